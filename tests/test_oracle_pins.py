"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here re-types an oracle formula or re-calls the library routine the oracle uses for
the same step: each expected value comes from an independent construction (a brute-force
DFT sum, an analytic Haar basis, a closed form, a grid search, an algebraic identity of the
iteration).
"""
import numpy as np
import pytest

from oracle import lps_oracle as O
from paper_1411_6206_gb300 import phantom as P

RNG = np.random.default_rng(12345)


def crandn(*shape, rng=RNG):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rand_mask(ny, nz, frac, rng=RNG):
    m = (rng.random((nz, ny)) < frac).astype(np.uint8)
    m[0, 0] = 1
    return m


# ---------------------------------------------------------------- acquisition operator

def brute_E(x, coils, mask, fft_z):
    """d[c][l][kx] = sum_{z,x,y} C x exp(-2 pi i (kx x/nx + ky y/ny [+ kz z/nz])) / sqrt(N)."""
    ncoil, nz, nx, ny = coils.shape
    lines = np.argwhere(mask)          # raster order over [first][ky]
    out = np.zeros((ncoil, len(lines), nx), complex)
    zz, xx, yy = np.meshgrid(np.arange(nz), np.arange(nx), np.arange(ny), indexing="ij")
    for c in range(ncoil):
        img = coils[c] * x
        for l, (a, ky) in enumerate(lines):
            for kx in range(nx):
                if fft_z:
                    ph = np.exp(-2j * np.pi * (kx * xx / nx + ky * yy / ny + a * zz / nz))
                    out[c, l, kx] = (img * ph).sum() / np.sqrt(nx * ny * nz)
                else:
                    ph = np.exp(-2j * np.pi * (kx * xx[a] / nx + ky * yy[a] / ny))
                    out[c, l, kx] = (img[a] * ph).sum() / np.sqrt(nx * ny)
    return out


@pytest.mark.parametrize("fft_z", [1, 0])
def test_E_matches_brute_force_dft(fft_z):
    nz, nx, ny, nc = 3, 4, 6, 2
    x = crandn(nz, nx, ny)
    coils = crandn(nc, nz, nx, ny)
    mask = rand_mask(ny, nz, 0.5)
    got = O.E(x, coils, mask, fft_z)
    ref = brute_E(x, coils, mask, fft_z)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("fft_z", [1, 0])
@pytest.mark.parametrize("shape", [(4, 8, 8, 3), (5, 6, 10, 1), (8, 16, 12, 4)])
def test_adjoint_identity(fft_z, shape):
    nz, nx, ny, nc = shape
    coils = crandn(nc, nz, nx, ny)
    mask = rand_mask(ny, nz, 0.4)
    x = crandn(nz, nx, ny)
    y = crandn(nc, int(mask.sum()), nx)
    lhs = np.vdot(O.E(x, coils, mask, fft_z), y)
    rhs = np.vdot(x, O.EH(y, coils, mask, fft_z))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_full_mask_sos_coils_is_identity():
    nz, nx, ny, nc = 4, 8, 8, 3
    coils = P.coil_maps(nx, ny, nz, nc, seed=3)
    mask = np.ones((nz, ny), np.uint8)
    x = crandn(nz, nx, ny)
    assert np.abs(O.EH(O.E(x, coils, mask), coils, mask) - x).max() < 1e-12


def test_line_order_is_raster():
    mask = np.zeros((3, 4), np.uint8)
    mask[2, 1] = mask[0, 3] = mask[1, 0] = 1
    kz, ky = O.line_index(mask)
    assert list(zip(kz, ky)) == [(0, 3), (1, 0), (2, 1)]


# ---------------------------------------------------------------- 3D frames as Casorati columns

def brute_E_blocks(x, coils, mask, zb):
    """d[c][l][kx] for line l = (z, ky), z = b zb + kz: the DFT of frame volume b alone,
    sum over its zb slices, x and y of C x exp(-2 pi i (kx x/nx + ky y/ny + kz s/zb)) / sqrt(zb nx ny)."""
    ncoil, nz, nx, ny = coils.shape
    lines = np.argwhere(mask)
    out = np.zeros((ncoil, len(lines), nx), complex)
    ss, xx, yy = np.meshgrid(np.arange(zb), np.arange(nx), np.arange(ny), indexing="ij")
    for c in range(ncoil):
        img = coils[c] * x
        for l, (z, ky) in enumerate(lines):
            b, kz = divmod(z, zb)
            vol = img[b * zb:(b + 1) * zb]
            for kx in range(nx):
                ph = np.exp(-2j * np.pi * (kx * xx / nx + ky * yy / ny + kz * ss / zb))
                out[c, l, kx] = (vol * ph).sum() / np.sqrt(zb * nx * ny)
    return out


@pytest.mark.parametrize("zb", [2, 3])
def test_E_frame_volumes_match_brute_force(zb):
    nz, nx, ny, nc = 2 * zb, 4, 4, 2
    coils = crandn(nc, nz, nx, ny)
    mask = rand_mask(ny, nz, 0.5)
    x = crandn(nz, nx, ny)
    got = O.E(x, coils, mask, 1, zb)
    assert np.abs(got - brute_E_blocks(x, coils, mask, zb)).max() < 1e-12
    # adjoint identity of the frame-volume encode
    y = crandn(nc, int(mask.sum()), nx)
    lhs = np.vdot(got, y)
    rhs = np.vdot(x, O.EH(y, coils, mask, 1, zb))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # one block is the whole-volume encode, a block of one slice the per-slice encode
    assert np.abs(O.E(x, coils, mask, 1, nz) - O.E(x, coils, mask, 1)).max() < 1e-12
    assert np.abs(O.E(x, coils, mask, 1, 1) - O.E(x, coils, mask, 0)).max() < 1e-12


def test_volume_columns_gram_and_rank_one_closed_form():
    """Columns of cs slices: the Gram is the sum, over the slice position s inside a column, of
    the slice Gram's entries (i cs + s, j cs + s); a separable sequence x[t cs + s] = v[t] u[s]
    (one volume u scaled per frame) is a rank-1 Casorati with sigma_1 = ||u|| ||v||, which
    initial_lambdas returns times lambda_L_rel."""
    cs, T, nx, ny = 3, 4, 8, 8
    X = crandn(cs * T, nx, ny)
    G1 = O.casorati_gram(X)
    G = O.casorati_gram(X, None, cs)
    want = np.array([[sum(G1[i * cs + s, j * cs + s] for s in range(cs)) for j in range(T)] for i in range(T)])
    assert np.abs(G - want).max() < 1e-10
    u = crandn(cs, nx, ny)
    v = np.array([1.0, -2.0j, 0.5, 3.0 + 1.0j])
    x = np.concatenate([v[t] * u for t in range(T)])
    sv = np.linalg.svd(O.casorati(x, cs), compute_uv=False)
    assert abs(sv[0] - np.linalg.norm(u) * np.linalg.norm(v)) < 1e-10 * sv[0] and sv[1] < 1e-10 * sv[0]
    p = O.Params(lambda_L_rel=0.01, frame_slices=cs)
    assert abs(O.initial_lambdas(x, p)[0] - 0.01 * np.linalg.norm(u) * np.linalg.norm(v)) < 1e-12 * sv[0]
    # the slice columns of the same sequence are not rank 1 (u varies over its slices)
    assert np.linalg.svd(O.casorati(x), compute_uv=False)[1] > 1e-3


@pytest.mark.parametrize("fft_z", [1, 0])
def test_frame_volumes_exact_recovery_full_mask_zero_thresholds(fft_z):
    cs, T, nx, ny = 2, 3, 8, 8
    nz = cs * T
    rng = np.random.default_rng(7)
    x = rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny))
    coils = P.coil_maps(nx, ny, nz, 2, seed=5)
    mask = np.ones((nz, ny), np.uint8)
    p = O.Params(lambda_L_rel=0.0, lambda_S_rel=0.0, lambda_p=0.0, rank_tau=0.0, max_iters=3,
                 fft_z=fft_z, frame_slices=cs)
    # data from the brute-force per-frame DFT (3D encode) or the per-slice encode
    d = brute_E_blocks(x, coils, mask, cs) if fft_z else O.E(x, coils, mask, 0)
    r = O.priori_ls(d, coils, mask, p)
    assert O.nrmse(r.recon, x) < 1e-12
    assert r.sigma.shape == (T,)


# ---------------------------------------------------------------- Haar transform

def haar_basis(nx, ny, J):
    """Analytic orthonormal 2D Haar basis (Mallat positions) built from its definition:
    level-j details are +-1 / 2^j on aligned 2^j x 2^j blocks (first half +, second half -),
    the level-J approximation is 1 / 2^J on aligned 2^J x 2^J blocks."""
    basis = {}
    for j in range(1, J + 1):
        b = 2 ** j
        h = b // 2
        for bi in range(nx // b):
            for bj in range(ny // b):
                sx = np.zeros(nx)
                sx[bi * b: bi * b + h] = 1
                sx[bi * b + h: bi * b + b] = -1
                sy = np.zeros(ny)
                sy[bj * b: bj * b + h] = 1
                sy[bj * b + h: bj * b + b] = -1
                ax = np.zeros(nx)
                ax[bi * b: bi * b + b] = 1
                ay = np.zeros(ny)
                ay[bj * b: bj * b + b] = 1
                basis[(bi, ny // b + bj)] = np.outer(ax, sy) / b          # x-low / y-high
                basis[(nx // b + bi, bj)] = np.outer(sx, ay) / b          # x-high / y-low
                basis[(nx // b + bi, ny // b + bj)] = np.outer(sx, sy) / b
                if j == J:
                    basis[(bi, bj)] = np.outer(ax, ay) / b
    return basis


@pytest.mark.parametrize("nx,ny,J", [(8, 8, 3), (16, 24, 3), (8, 16, 2), (4, 4, 1)])
def test_haar_equals_analytic_basis(nx, ny, J):
    x = crandn(nx, ny)
    c = O.haar2(x, J)
    basis = haar_basis(nx, ny, J)
    assert len(basis) == nx * ny
    for (i, j), f in basis.items():
        assert abs(c[i, j] - (f * x).sum()) < 1e-12


def test_haar_orthonormal_and_invertible():
    x = crandn(5, 16, 24)
    c = O.T(x, 3)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert np.abs(O.Tinv(c, 3) - x).max() < 1e-12


def test_haar_constant_block_single_coefficient():
    x = np.zeros((1, 16, 16), complex)
    x[0, 8:16, 0:8] = 2 - 1j
    c = O.T(x, 3)
    nzc = np.argwhere(np.abs(c) > 1e-12)
    assert nzc.tolist() == [[0, 1, 0]]
    assert abs(c[0, 1, 0] - 8 * (2 - 1j)) < 1e-12


def haar1_basis(n, J):
    """Analytic orthonormal 1D Haar functions (Mallat positions): level-j details are
    +-1 / sqrt(2^j) on aligned blocks of 2^j (first half +, second half -), the level-J
    approximation 1 / sqrt(2^J) on aligned blocks of 2^J."""
    basis = {}
    for j in range(1, J + 1):
        b = 2 ** j
        for k in range(n // b):
            f = np.zeros(n)
            f[k * b: k * b + b // 2] = 1 / np.sqrt(b)
            f[k * b + b // 2: k * b + b] = -1 / np.sqrt(b)
            basis[n // b + k] = f
            if j == J:
                a = np.zeros(n)
                a[k * b: k * b + b] = 1 / np.sqrt(b)
                basis[k] = a
    return basis


@pytest.mark.parametrize("nz,nx,ny,J", [(8, 8, 8, 3), (16, 8, 16, 3), (4, 8, 8, 2), (2, 8, 4, 1)])
def test_haar3_equals_analytic_basis(nz, nx, ny, J):
    """The 3D variant is the tensor product of the 1D Haar along z with the 2D pyramid: its
    coefficient (k, i, j) is <f_k (x) g_ij, x> for the analytic functions f (1D) and g (2D)."""
    x = crandn(nz, nx, ny)
    c = O.T3(x, J)
    fz = haar1_basis(nz, J)
    g2 = haar_basis(nx, ny, J)
    assert len(fz) == nz and len(g2) == nx * ny
    for k, f in fz.items():
        for (i, j), g in g2.items():
            assert abs(c[k, i, j] - (f[:, None, None] * g[None] * x).sum()) < 1e-12


def test_haar3_orthonormal_and_invertible():
    x = crandn(16, 16, 24)
    c = O.T3(x, 3)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert np.abs(O.T3inv(c, 3) - x).max() < 1e-12
    # not the per-slice transform: the z pass moves energy between slices
    assert np.abs(c - O.T(x, 3)).max() > 0.1


def test_haar3_constant_cube_single_coefficient():
    """A constant a on the aligned 8 x 8 x 8 cube (z, x, y) in [8, 16) x [0, 8) x [8, 16)
    has one 3D coefficient, a sqrt(512), at the approximation position (1, 0, 1); the 2D
    transform gives eight coefficients 8a instead (one per slice)."""
    a = 0.5 + 1.5j
    x = np.zeros((16, 16, 16), complex)
    x[8:16, 0:8, 8:16] = a
    c = O.T3(x, 3)
    assert np.argwhere(np.abs(c) > 1e-12).tolist() == [[1, 0, 1]]
    assert abs(c[1, 0, 1] - a * np.sqrt(512)) < 1e-12
    assert (np.abs(O.T(x, 3)) > 1e-12).sum() == 8


def test_initial_lambdas_and_sparse_step_use_the_3d_transform():
    """With wavelet_dims = 3, lambda_S = rel_S max|T3(X_0)| and step (3) shrinks the 3D
    coefficients. X_0 = the constant cube a on 8 x 8 x 8 (full mask, unit coil, so E^H E = I):
    sigma_1 = |a| sqrt(512) (eight equal Casorati columns of norm 8|a|), max|T3 X_0| =
    |a| sqrt(512). One iteration from the state (X = cube, S = 0, L_prev = 0) with lambda_S = l
    gives S = (1 - l / (|a| sqrt(512))) X; the per-slice transform would give (1 - l / (8|a|)) X."""
    a = 2.0 - 1.0j
    nz, nx, ny = 8, 8, 8
    x = np.full((nz, nx, ny), a)
    coils = np.ones((1, nz, nx, ny), complex)
    mask = np.ones((nz, ny), np.uint8)
    d = O.E(x, coils, mask)
    p3 = O.Params(lambda_L_rel=0.01, lambda_S_rel=0.005, max_iters=1, wavelet_dims=3)
    lL, lS = O.initial_lambdas(x, p3)
    assert abs(lL - 0.01 * abs(a) * np.sqrt(512)) < 1e-12
    assert abs(lS - 0.005 * abs(a) * np.sqrt(512)) < 1e-12
    lam = 4.0
    zero = np.zeros_like(x)
    r3 = O.priori_ls(d, coils, mask, p3, iters=1, state=(x, zero, zero, 0.0, lam))
    assert np.abs(r3.S - (1 - lam / (abs(a) * np.sqrt(512))) * x).max() < 1e-12
    p2 = O.Params(lambda_L_rel=0.01, lambda_S_rel=0.005, max_iters=1)
    r2 = O.priori_ls(d, coils, mask, p2, iters=1, state=(x, zero, zero, 0.0, lam))
    assert np.abs(r2.S - (1 - lam / (8 * abs(a))) * x).max() < 1e-12


# ---------------------------------------------------------------- soft threshold

def read_golden(name):
    rows = []
    with open(f"{__file__.rsplit('/', 1)[0]}/golden/{name}") as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def test_soft_threshold_closed_forms():
    g = read_golden("soft_threshold.txt")
    for re_, im_, lam, ore, oim in g:
        got = O.soft(np.array([re_ + 1j * im_]), lam)[0]
        assert abs(got - (ore + 1j * oim)) < 1e-15


def test_soft_threshold_is_prox_by_grid_search():
    rng = np.random.default_rng(7)
    grid = np.linspace(-3, 3, 601)
    Zr, Zi = np.meshgrid(grid, grid, indexing="ij")
    Zc = Zr + 1j * Zi
    for _ in range(5):
        cval = complex(*rng.uniform(-2, 2, 2))
        lam = rng.uniform(0.1, 1.5)
        f = 0.5 * np.abs(Zc - cval) ** 2 + lam * np.abs(Zc)
        zbest = Zc.ravel()[np.argmin(f)]
        assert abs(zbest - O.soft(np.array([cval]), lam)[0]) < 0.015


def test_support_shrink_special_cases():
    c = crandn(3, 8, 8)
    lam = 0.7
    assert np.array_equal(O.support_shrink(c, lam, None), O.soft(c, lam))
    assert np.array_equal(O.support_shrink(c, lam, np.ones(c.shape, bool)), c)
    keep = RNG.random(c.shape) < 0.3
    out = O.support_shrink(c, lam, keep)
    assert np.array_equal(out[keep], c[keep])
    # off the support: the prox of lam*|.| (closed form checked above)
    off = ~keep
    a = np.abs(c[off])
    assert np.allclose(np.abs(out[off]), np.maximum(a - lam, 0), atol=1e-14)


# ---------------------------------------------------------------- SVT and prior pull

def rand_unitary_cols(n, k, rng):
    q, _ = np.linalg.qr(crandn(n, k, rng=rng))
    return q


def test_svt_closed_form():
    rng = np.random.default_rng(1)
    N, n = 40, 6
    U = rand_unitary_cols(N, n, rng)
    V = rand_unitary_cols(n, n, rng)
    s = np.array([5.0, 3.0, 2.0, 1.0, 0.5, 0.1])
    M = (U * s) @ V.conj().T
    lam = 0.8
    L, sig, s2 = O.svt(M, lam)
    ref = (U * np.maximum(s - lam, 0)) @ V.conj().T
    assert np.abs(L - ref).max() < 1e-12
    assert np.allclose(sig, s, atol=1e-12)
    # zero threshold is the identity
    L0, _, _ = O.svt(M, 0.0)
    assert np.abs(L0 - M).max() < 1e-12


def test_casorati_gram_closed_form_and_svd():
    rng = np.random.default_rng(7)
    nz, nx, ny = 5, 4, 6
    # slices with disjoint supports: orthogonal Casorati columns, diagonal Gram of squared norms
    X = np.zeros((nz, nx, ny), complex)
    for z in range(nz):
        X[z].flat[z * 4:(z + 1) * 4] = crandn(4, rng=rng)
    G = O.casorati_gram(X)
    norms2 = np.array([np.sum(np.abs(X[z]) ** 2) for z in range(nz)])
    assert np.abs(G - np.diag(norms2)).max() < 1e-12
    # general case: eigenvalues = squared singular values of the Casorati (LAPACK SVD), and
    # S enters as M = X - S
    X = crandn(nz, nx, ny, rng=rng)
    S = crandn(nz, nx, ny, rng=rng)
    G = O.casorati_gram(X, S)
    assert np.abs(G - G.conj().T).max() < 1e-12
    M = np.stack([(X - S)[z].ravel() for z in range(nz)], axis=1)
    sv = np.linalg.svd(M, compute_uv=False)
    ev = np.sort(np.linalg.eigvalsh(G))[::-1]
    assert np.allclose(ev, sv ** 2, rtol=1e-12, atol=1e-12 * sv[0] ** 2)


def test_reproject_gram_route_equals_svt():
    rng = np.random.default_rng(8)
    N, n = 30, 5
    U = rand_unitary_cols(N, n, rng)
    V = rand_unitary_cols(n, n, rng)
    s = np.array([4.0, 2.5, 1.5, 0.7, 0.2])
    M = (U * s) @ V.conj().T
    X = M.T.reshape(n, 5, 6)
    lam = 0.6
    f = np.maximum(s - lam, 0) / s
    W = (V * f) @ V.conj().T
    Lr = O.reproject(X, None, W)
    ref = (U * np.maximum(s - lam, 0)) @ V.conj().T
    assert np.abs(Lr - ref.T.reshape(n, 5, 6)).max() < 1e-12
    # W = I gives X - S; W = 0 gives 0
    S = crandn(n, 5, 6, rng=rng)
    assert np.abs(O.reproject(X, S, np.eye(n)) - (X - S)).max() < 1e-12
    assert np.abs(O.reproject(X, S, np.zeros((n, n)))).max() == 0


def test_svt_rectangular_diagonal_with_phases():
    n = 4
    ph = np.exp(1j * np.array([0.3, -1.2, 2.0, 0.7]))
    s = np.array([4.0, 2.5, 1.0, 0.2])
    M = np.zeros((7, n), complex)
    M[np.arange(n), np.arange(n)] = s * ph
    L, _, _ = O.svt(M, 0.5)
    ref = np.zeros_like(M)
    ref[np.arange(n), np.arange(n)] = np.maximum(s - 0.5, 0) * ph
    assert np.abs(L - ref).max() < 1e-12


def test_prior_pull_special_cases_and_linearity():
    rng = np.random.default_rng(2)
    N, n = 30, 5
    U = rand_unitary_cols(N, n, rng)
    V = rand_unitary_cols(n, n, rng)
    s = np.array([6.0, 4.0, 3.0, 2.0, 1.5])
    M = (U * s) @ V.conj().T
    sp = np.array([5.0, 4.5, 2.0, 1.0, 0.0])
    lam = 0.5
    L0, _, a0 = O.svt(M, lam, 0.0, sp)
    Lplain, _, _ = O.svt(M, lam)
    assert np.abs(L0 - Lplain).max() < 1e-12                     # lambda_p = 0: plain SVT
    L1, _, a1 = O.svt(M, lam, 1.0, sp)
    assert np.allclose(a1, sp, atol=1e-12)                       # lambda_p = 1: sigma_prev
    assert np.abs(L1 - (U * sp) @ V.conj().T).max() < 1e-12
    Lh, _, _ = O.svt(M, lam, 0.3, sp)
    assert np.abs(Lh - (0.7 * L0 + 0.3 * L1)).max() < 1e-12     # linear in lambda_p


def test_rank_guard_drops_small_directions():
    rng = np.random.default_rng(3)
    U = rand_unitary_cols(20, 3, rng)
    V = rand_unitary_cols(3, 3, rng)
    s = np.array([1.0, 0.5, 1e-4])
    M = (U * s) @ V.conj().T
    _, _, s2 = O.svt(M, 0.0, 1.0, np.array([1.0, 0.5, 0.3]), tau=1e-3)
    assert s2[2] == 0.0 and abs(s2[0] - 1.0) < 1e-12


# ---------------------------------------------------------------- the whole iteration

def small_problem(seed=0, nz=4, nx=16, ny=16, nc=2, frac=0.35, noise=0.0, full=False):
    rng = np.random.default_rng(seed)
    coils = P.coil_maps(nx, ny, nz, nc, seed=seed + 1)
    Z, X, Y = np.meshgrid(np.arange(nz), np.arange(nx), np.arange(ny), indexing="ij")
    bg = np.exp(-((X - nx / 2) ** 2 + (Y - ny / 2) ** 2) / (2 * (nx / 4) ** 2)) * (1 + 0.2 * Z)
    x = bg * np.exp(0.3j * Y / ny) + 0.0j
    x[:, 3:6, 5:9] += 0.8
    x[1:3, 10:12, 2:4] += 0.6j
    mask = np.ones((nz, ny), np.uint8) if full else rand_mask(ny, nz, frac, rng)
    d = O.E(x, coils, mask)
    if noise:
        d = d + noise * crandn(*d.shape, rng=rng)
    return x, coils, mask, d


def test_exact_recovery_full_mask_zero_thresholds():
    x, coils, mask, d = small_problem(full=True)
    p = O.Params(lambda_L_rel=0.0, lambda_S_rel=0.0, lambda_p=0.0, rank_tau=0.0, max_iters=4)
    r = O.priori_ls(d, coils, mask, p)
    assert O.nrmse(r.recon, x) < 1e-12
    for k in (1, 2, 3):
        rk = O.priori_ls(d, coils, mask, p, iters=k)
        assert O.nrmse(rk.recon, x) < 1e-12
    assert np.abs(O.priori_ls(d, coils, mask, p, iters=1).S).max() == 0.0   # L_0 := X_0


@pytest.mark.parametrize("with_support", [False, True])
def test_objective_non_increasing(with_support):
    x, coils, mask, d = small_problem(seed=4, noise=1e-3)
    p = O.Params(lambda_L_rel=0.05, lambda_S_rel=0.02, lambda_p=0.0, rank_tau=1e-3,
                 max_iters=25)
    prior = None
    if with_support:
        sup = np.abs(O.T(x)) > 0.3
        prior = O.Prior(support=sup, sigma=np.ones(x.shape[0]))
    r = O.priori_ls(d, coils, mask, p, prior)
    F = [h["objective"] for h in r.history]
    for a, b in zip(F[1:], F[2:]):
        assert b <= a * (1 + 1e-12), (a, b)
    assert F[-1] < F[1]
    # the monitored objective equals F(L, S) evaluated from scratch
    keep = None if prior is None else prior.support
    Fk = O.objective(r.L, r.S, d, coils, mask, r.lambda_L, r.lambda_S, keep, p)
    assert abs(Fk - F[-1]) < 1e-10 * abs(Fk)


def test_monotonicity_pin_catches_ascent_sign():
    """A4 check: the printed sign of the residual (ascent) makes the objective grow."""
    x, coils, mask, d = small_problem(seed=5, noise=1e-3)
    X = O.EH(d, coils, mask)
    L = X.copy()
    S = np.zeros_like(X)
    R = O.E(L + S, coils, mask) - d
    descent = L + S - O.EH(R, coils, mask)
    ascent = L + S + O.EH(R, coils, mask)
    f = lambda Z: np.linalg.norm(O.E(Z, coils, mask) - d)
    assert f(descent) < f(L + S) < f(ascent)


def test_empty_prior_with_zero_pull_equals_plain_ls():
    x, coils, mask, d = small_problem(seed=6, noise=1e-3)
    p = O.Params(max_iters=8, lambda_p=0.0)
    a = O.priori_ls(d, coils, mask, p)
    b = O.priori_ls(d, coils, mask, p,
                    O.Prior(support=np.zeros(x.shape, bool), sigma=np.full(x.shape[0], 3.0)))
    assert np.array_equal(a.L, b.L) and np.array_equal(a.S, b.S)


def test_lambda_p_one_pins_singular_values_to_prior():
    x, coils, mask, d = small_problem(seed=7, noise=1e-3)
    p = O.Params(max_iters=3, lambda_p=1.0, rank_tau=0.0)
    sp = np.linspace(2.0, 0.5, x.shape[0])
    r = O.priori_ls(d, coils, mask, p, O.Prior(support=None, sigma=sp))
    s = np.linalg.svd(O.casorati(r.L), compute_uv=False)
    assert np.allclose(np.sort(s)[::-1], sp, atol=1e-10)


def test_recovery_improves_over_iterations():
    x, coils, mask, d = small_problem(seed=8, frac=0.5, noise=1e-3)
    p = O.Params(max_iters=40)
    e0 = O.nrmse(O.EH(d, coils, mask), x)
    r = O.priori_ls(d, coils, mask, p)
    assert O.nrmse(r.recon, x) < 0.7 * e0


def test_sequence_passes_prior():
    """Recursion of Sec. 3 (Fig. 2): frame t runs Algorithm 1 with the support and singular
    values of frame t-1. With lambda_p = 1, step (2) sets sigma'' to the prior exactly, so
    frame 2's singular values must be frame 1's; and on the prior support step (3) keeps the
    coefficients unshrunk, so T(S) of frame 2 equals its c there and equals soft(c) elsewhere.
    A recursion that dropped either prior (or passed frame 2's own) fails one of the two."""
    w = P.SMALL
    pr = P.problem(w, frames=2)
    datas = [O.E(pr["x"][t], pr["coils"], pr["masks"][t]) + pr["noise"][t] for t in range(2)]
    p = O.Params(max_iters=5, lambda_p=1.0, rank_tau=0.0)
    seq = O.sequence(datas, pr["coils"], pr["masks"], p)
    assert len(seq) == 2
    sup1 = seq[0].support
    assert sup1.any() and not sup1.all()
    # sigma: the singular values of L of frame 2 are frame 1's sigma'' (independent SVD)
    s_L2 = np.linalg.svd(O.casorati(seq[1].L), compute_uv=False)
    assert np.allclose(np.sort(s_L2)[::-1], np.sort(seq[0].sigma)[::-1], atol=1e-10 * seq[0].sigma.max())
    # support: coefficients of S of frame 2 on frame 1's support are the unshrunk c
    cS = O.T(seq[1].S, w_levels := p.wavelet_levels)
    c2 = seq[1].c
    assert np.abs(cS[sup1] - c2[sup1]).max() < 1e-12 * np.abs(c2).max()
    off = ~sup1
    lam = seq[1].lambda_S
    assert np.allclose(np.abs(cS[off]), np.maximum(np.abs(c2[off]) - lam, 0.0), atol=1e-12 * np.abs(c2).max())
    # the kept coefficients include some below the threshold (otherwise the test proves nothing)
    assert (np.abs(c2[sup1]) < lam).any()
    # frame 1 is plain L+S: the same call without a prior
    r1 = O.priori_ls(datas[0], pr["coils"], pr["masks"][0], p)
    assert np.array_equal(seq[0].L, r1.L) and np.array_equal(seq[0].S, r1.S)


def two_block_image(nz, nx, ny, s, v1, v2, blocks):
    """Image whose Casorati matrix is s[0] u1 v1^H + s[1] u2 v2^H, with u_k the normalised
    indicator of an aligned 8 x 8 in-plane block (so its J = 3 Haar transform is a single
    coefficient of value 1 at the block's approximation position)."""
    x = np.zeros((nz, nx, ny), complex)
    for sk, vk, (bx, by) in zip(s, (v1, v2), blocks):
        for z in range(nz):
            x[z, bx:bx + 8, by:by + 8] += sk * np.conj(vk[z]) / 8.0
    return x


def test_initial_lambdas_closed_form():
    """R2: lambda_L = rel_L sigma_1(X_0) and lambda_S = rel_S max|T(X_0)|, with X_0 = E^H d.
    Full mask and one unit coil make E^H E = I, so X_0 is the image itself. The image is a
    rank-2 Casorati matrix with singular values (5, 3) whose columns live on two 8 x 8 blocks,
    so sigma_1 = 5 (not ||X||_F = sqrt(34), not the nuclear norm 8) and the Haar coefficients
    are 5 conj(v1[z]) and 3 conj(v2[z]), so max|T X_0| = 5 * 0.8 = 4 (the image-domain
    maximum is 0.5)."""
    nz, nx, ny = 4, 16, 16
    v1 = np.array([3, 4j, 0, 0]) / 5.0
    v2 = np.array([0, 0, 1, -1j]) / np.sqrt(2)
    x = two_block_image(nz, nx, ny, (5.0, 3.0), v1, v2, ((0, 0), (8, 8)))
    coils = np.ones((1, nz, nx, ny), complex)
    mask = np.ones((nz, ny), np.uint8)
    d = O.E(x, coils, mask)
    p = O.Params(lambda_L_rel=0.01, lambda_S_rel=0.005, max_iters=1)
    r = O.priori_ls(d, coils, mask, p)
    assert abs(r.lambda_L - 0.01 * 5.0) < 1e-12
    assert abs(r.lambda_S - 0.005 * 4.0) < 1e-12
    # the same through initial_lambdas directly
    lL, lS = O.initial_lambdas(x, p)
    assert abs(lL - 0.05) < 1e-12 and abs(lS - 0.02) < 1e-12


def support_case(rule, keep=None):
    """A state (X, S, L_prev) with X - L_prev = T^{-1}(c) for a designed coefficient array c:
    one iteration from it computes c = T(X - L_prev) (step 3) and the output support from c.
    Magnitudes relative to lambda_S = 1: 2.0 and 1.5 above it, 1.0 exactly at it, 0.6 below,
    0 elsewhere."""
    nz, nx, ny = 2, 16, 16
    c = np.zeros((nz, nx, ny), complex)
    pos = {"above2": (0, 3, 5), "above15": (1, 9, 2), "at": (0, 12, 12), "below": (1, 0, 0)}
    c[pos["above2"]] = 2.0 * np.exp(0.3j)
    c[pos["above15"]] = -1.5j
    c[pos["at"]] = 1.0
    c[pos["below"]] = 0.6 * np.exp(-2.0j)
    D = O.Tinv(c, 3)
    assert np.abs(O.T(D, 3) - c).max() < 1e-14
    coils = np.ones((1, nz, nx, ny), complex)
    mask = np.ones((nz, ny), np.uint8)
    d = O.E(D, coils, mask)
    p = O.Params(max_iters=1, lambda_p=0.0, rank_tau=0.0, support_rule=rule)
    prior = None if keep is None else O.Prior(support=keep, sigma=None)
    # lambda_S is set to the rounded magnitude of the "at" coefficient as step (3) computes it
    # (c = T(X - L_prev) = T(D)), so that the tie is exact in floating point
    lam = float(np.abs(O.T(D, 3)[pos["at"]]))
    assert abs(lam - 1.0) < 1e-14
    r = O.priori_ls(d, coils, mask, p, prior, iters=1,
                    state=(D, np.zeros_like(D), np.zeros_like(D), 0.0, lam))
    assert np.abs(r.c[pos["at"]]) == r.lambda_S
    return r, pos


def test_output_support_threshold_rule():
    """R5: T^(t) = {i : |c_i| > lambda_S} for c of the last iteration; a tie at lambda_S is
    off-support. A '>=' rule takes the tie; a support read from the shrunk c' (|c'| = |c| -
    lambda_S off the prior) drops the 1.5 lambda_S coefficient."""
    r, pos = support_case("threshold")
    want = np.zeros(r.c.shape, bool)
    want[pos["above2"]] = want[pos["above15"]] = True
    assert np.array_equal(r.support, want)


def test_output_support_nonzero_rule():
    """The literal rule supp T(S^(t)): nonzero shrunk coefficients. Off the prior support that
    is |c| > lambda_S; on it every nonzero c is kept unshrunk, so the 0.6 lambda_S coefficient
    on the prior support is in the support under this rule and out of it under the threshold
    rule."""
    keep = np.zeros((2, 16, 16), bool)
    r0, pos = support_case("nonzero")
    keep[pos["below"]] = True
    keep[pos["above2"]] = True
    r, _ = support_case("nonzero", keep)
    want = np.zeros(r.c.shape, bool)
    want[pos["above2"]] = want[pos["above15"]] = want[pos["below"]] = True
    assert np.array_equal(r.support, want)
    want0 = np.zeros(r.c.shape, bool)
    want0[pos["above2"]] = want0[pos["above15"]] = True
    assert np.array_equal(r0.support, want0)
    rt, _ = support_case("threshold", keep)
    assert not rt.support[pos["below"]] and rt.support[pos["above2"]]


def rel_change_case():
    """Full mask, one unit coil (E^H E = I), lambda_S = 0, lambda_L = 2, no prior, no rank
    guard, and an image whose Casorati matrix is U diag(5, 3, 1) V^H. Every iterate stays of
    the form U diag(.) V^H (T is orthonormal and lambda_S = 0, so S_k = X_{k-1} - L_{k-1}), and
    step (4) returns X_k = x. With (5, 3, 1) written s and svt(a) = max(a - 2, 0):
      k = 1: L = svt(s) = (3, 1, 0), S = 0,               Z = (3, 1, 0)
      k = 2: L = (3, 1, 0),          S = s - L_1 = (2, 2, 1), Z = (5, 3, 1)
      k = 3: L = svt(s - S_2) = (1, 0, 0), S = (2, 2, 1),  Z = (3, 2, 1)
      k = 4: L = (1, 0, 0),          S = s - L_3 = (4, 3, 1), Z = (5, 3, 1)
      k = 5: L = svt(s - S_4) = 0,   S = (4, 3, 1),        Z = (4, 3, 1)
    with Z_0 = L_0 + S_0 = x, so the relative changes ||Z_k - Z_{k-1}|| / ||Z_{k-1}|| are
    3/sqrt(35), 3/sqrt(10), 1/sqrt(7), sqrt(5/14), 1/sqrt(35) and the nuclear norms 4, 4, 1, 1, 0."""
    nz, nx, ny = 3, 16, 8
    rng = np.random.default_rng(21)
    U, _ = np.linalg.qr(rng.standard_normal((nx * ny, 3)) + 1j * rng.standard_normal((nx * ny, 3)))
    V, _ = np.linalg.qr(rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)))
    M = (U * np.array([5.0, 3.0, 1.0])) @ V.conj().T
    x = M.T.reshape(nz, nx, ny)
    coils = np.ones((1, nz, nx, ny), complex)
    mask = np.ones((nz, ny), np.uint8)
    return x, coils, mask, O.E(x, coils, mask)


@pytest.mark.parametrize("tol,stop_at", [(0.0, 5), (0.6, 1), (0.4, 3)])
def test_rel_change_and_tol_stop_closed_form(tol, stop_at):
    """Sec. 3 stopping rule: stop at the first iteration whose relative change of the
    solution Z = L + S, ||Z_k - Z_{k-1}|| / ||Z_{k-1}||, is below the tolerance. The closed
    forms fail if X is normed instead of Z (X_k = x for every k, so the change would be 0),
    if Z_{k-1} is taken after the update, or if the new Z is the denominator."""
    x, coils, mask, d = rel_change_case()
    lam_rel = 2.0 / 5.0   # lambda_L = 2 (sigma_1 = 5)
    p = O.Params(lambda_L_rel=lam_rel, lambda_S_rel=0.0, lambda_p=0.0, rank_tau=0.0, max_iters=5, tol=tol)
    r = O.priori_ls(d, coils, mask, p)
    assert abs(r.lambda_L - 2.0) < 1e-12 and r.lambda_S == 0.0
    want = [3.0 / np.sqrt(35.0), 3.0 / np.sqrt(10.0), 1.0 / np.sqrt(7.0), np.sqrt(5.0 / 14.0), 1.0 / np.sqrt(35.0)]
    got = [h["rel_change"] for h in r.history]
    assert r.iters == stop_at and len(got) == stop_at
    for g, w_ in zip(got, want):
        assert abs(g - w_) < 1e-12
    nuc = [4.0, 4.0, 1.0, 1.0, 0.0]
    for h, n_ in zip(r.history, nuc):
        assert abs(h["nuclear"] - n_) < 1e-12


@pytest.mark.parametrize("fft_z", [1, 0])
def test_data_consistency_step_is_a_projection_for_one_unit_coil(fft_z):
    """With C = 1, E^H E = F^H M F is a projection, so step (4) with unit step makes the
    new estimate agree with the samples exactly: E(X_it) = d (pins the step length)."""
    rng = np.random.default_rng(9)
    nz, nx, ny = 4, 8, 16
    coils = np.ones((1, nz, nx, ny), complex)
    mask = rand_mask(ny, nz, 0.3, rng)
    d = crandn(1, int(mask.sum()), nx, rng=rng)
    p = O.Params(max_iters=1, fft_z=fft_z)
    for k in (1, 2, 3):
        r = O.priori_ls(d, coils, mask, p, iters=k)
        assert np.abs(O.E(r.X, coils, mask, fft_z) - d).max() < 1e-12
