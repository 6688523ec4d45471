"""Layout "frames" with 3D frames (frame_slices > 1): the Casorati columns are whole frame
volumes, each encoded by its own 3D DFT (or per slice) under its own (kz, ky) lines. Operators,
one iteration from a common state and a whole segment against the FP64 oracle with the same
columns (Params.frame_slices), plus the shapes the library refuses."""
import numpy as np
import pytest

from oracle import lps_oracle as O
from tests.gpu_cases import c64, oracle_params, rel, up

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
E2E_TOL = 1e-3


@pytest.fixture(scope="module")
def L():
    from paper_1411_6206_gb300 import lps
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    lps.load()
    return lps


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def segment(T, fs, nx, ny, ncoil, fft_z=1, seed=3, frac=0.3, phantom="ellipsoids"):
    """T frame volumes of fs slices (a 3D + t phantom), per-frame (kz, ky) masks with a fully
    sampled centre, the same coil maps in every frame, k-space by the oracle's per-frame encode."""
    from paper_1411_6206_gb300 import phantom as P
    w = P.Workload("seg", nx, ny, fs, ncoil, T, 10, 1.0 / frac, seed, phantom=phantom, frac_lines=frac)
    x = P.phantom_sequence(w).reshape(T * fs, nx, ny)
    cm = P.coil_maps(nx, ny, fs, ncoil, seed + 17)
    coils = c64(np.concatenate([cm] * T, axis=1))
    masks = [P.vd_mask(ny, fs, max(1, int(round(frac * ny * fs))), min(4, fs, ny), seed + 31 * t, fft_z)
             for t in range(T)]
    mask = np.ascontiguousarray(np.concatenate(masks, axis=0))
    zb = fs if fft_z else 1
    d = O.E(x, up(coils), mask, fft_z, zb) + P.noise(ncoil, int(mask.sum()), nx, 1e-3, seed + 5)
    return dict(x=x, coils=coils, mask=mask, d=c64(d), nlines=int(mask.sum()), fs=fs, fft_z=fft_z)


def plan_for(L, case, T, nx, ny, ncoil, **kw):
    fs = case["fs"]
    pl = L.Plan(nx, ny, T * fs, ncoil, layout=L.LAYOUT_FRAMES, frame_slices=fs, fft_z=case["fft_z"], **kw)
    pl.set_coils(dev(case["coils"]))
    assert pl.set_mask(dev(case["mask"])) == case["nlines"]
    pl.set_data(dev(case["d"]))
    return pl


@pytest.mark.parametrize("T,fs,nx,ny,nc,fz", [(4, 4, 16, 32, 2, 1), (3, 8, 16, 16, 1, 1), (4, 2, 24, 16, 3, 0),
                                             (6, 5, 16, 24, 2, 1)])
def test_operators_match_oracle(L, T, fs, nx, ny, nc, fz):
    case = segment(T, fs, nx, ny, nc, fz)
    pl = plan_for(L, case, T, nx, ny, nc)
    zb = fs if fz else 1
    nz = T * fs
    rng = np.random.default_rng(1)
    x = c64(rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny)))
    kd = torch.empty((nc, case["nlines"], nx), dtype=torch.complex64, device="cuda")
    L.forward(pl.handle, dev(x), kd)
    assert rel(kd.cpu().numpy(), O.E(up(x), up(case["coils"]), case["mask"], fz, zb)) < OP_TOL
    img = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    L.adjoint(pl.handle, dev(case["d"]), img)
    assert rel(img.cpu().numpy(), O.EH(up(case["d"]), up(case["coils"]), case["mask"], fz, zb)) < OP_TOL
    # step (4) alone
    X = torch.empty_like(img)
    r2 = L.data_consistency(pl.handle, dev(x), X)
    R = O.E(up(x), up(case["coils"]), case["mask"], fz, zb) - up(case["d"])
    Xref = up(x) - O.EH(R, up(case["coils"]), case["mask"], fz, zb)
    assert rel(X.cpu().numpy(), Xref) < OP_TOL
    assert abs(r2 - np.vdot(R, R).real) < 1e-5 * np.vdot(R, R).real
    # the T x T Gram of the volume columns
    G = torch.empty((T, T), dtype=torch.complex64, device="cuda")
    L.casorati_gram(pl.handle, dev(x), None, G)
    Gref = O.casorati_gram(up(x), None, fs)
    assert np.abs(G.cpu().numpy() - Gref).max() < 1e-5 * np.abs(Gref).max()
    pl.close()


@pytest.mark.parametrize("T,fs,nx,ny,nc", [(4, 4, 16, 32, 2), (8, 8, 32, 32, 1)])
def test_one_iteration_from_state(L, T, fs, nx, ny, nc):
    case = segment(T, fs, nx, ny, nc)
    pl = plan_for(L, case, T, nx, ny, nc, lambda_p=0.5)
    p = oracle_params(pl.params)
    assert p.frame_slices == fs
    coils, d, mask = up(case["coils"]), up(case["d"]), case["mask"]
    r0 = O.priori_ls(d, coils, mask, p, iters=3)
    X, S, Lp = c64(r0.X), c64(r0.S), c64(r0.L)
    lamL, lamS = float(np.float32(r0.lambda_L)), float(np.float32(r0.lambda_S))
    L.set_state(pl.handle, dev(X), dev(S), dev(Lp), lamL, lamS, 3)
    pl.iterate(1)
    Xg = torch.empty((T * fs, nx, ny), dtype=torch.complex64, device="cuda")
    Lg, Sg = torch.empty_like(Xg), torch.empty_like(Xg)
    L.get_state(pl.handle, Xg, Lg, Sg)
    ref = O.priori_ls(d, coils, mask, p, None, iters=1, state=(up(X), up(S), up(Lp), lamL, lamS))
    s = ref.sigma_in
    keep = s > ref.lambda_L
    tol = max(OP_TOL, 8 * 2.0 ** -24 * s[0] ** 2 * np.sqrt(np.sum(1.0 / s[keep] ** 2)) / np.linalg.norm(ref.L))
    assert rel(Lg.cpu().numpy(), ref.L) < tol
    assert rel(Xg.cpu().numpy(), ref.X) < tol
    assert rel(Sg.cpu().numpy(), ref.S) < OP_TOL
    sig = np.empty(T)
    L.get_support(pl.handle, None, sig)
    np.testing.assert_allclose(sig, ref.sigma, rtol=1e-3, atol=1e-4 * ref.sigma.max())
    pl.close()


@pytest.mark.parametrize("T,fs,nx,ny,nc,wdims,iters", [(8, 8, 32, 32, 1, 2, 30), (4, 8, 16, 32, 2, 3, 20),
                                                       (5, 4, 16, 16, 2, 2, 20)])
def test_segment_end_to_end(L, T, fs, nx, ny, nc, wdims, iters):
    """A 3D + t segment (the first shape is the 32 x 32 x 8 volume x 8 frames single-coil
    workload with its frames as the Casorati columns) against the oracle after the stated
    iterations; lambda_L and lambda_S of step (0) from the volume-column Casorati."""
    case = segment(T, fs, nx, ny, nc, frac=0.25)
    pl = plan_for(L, case, T, nx, ny, nc, max_iters=iters, wavelet_dims=wdims)
    recon = torch.empty((T * fs, nx, ny), dtype=torch.complex64, device="cuda")
    st = pl.reconstruct_frame(recon=recon)
    ref = O.priori_ls(up(case["d"]), up(case["coils"]), case["mask"], oracle_params(pl.params))
    assert st.iters == iters
    assert abs(st.lambda_L - ref.lambda_L) < 1e-5 * ref.lambda_L
    assert abs(st.lambda_S - ref.lambda_S) < 1e-5 * ref.lambda_S
    err = O.nrmse(recon.cpu().numpy(), ref.recon)
    assert err <= E2E_TOL, err
    pl.close()


def test_refused_shapes(L):
    def code(**kw):
        base = dict(nx=16, ny=16, nz=16, ncoil=1, layout=L.LAYOUT_FRAMES, frame_slices=4)
        base.update(kw)
        with pytest.raises(L.LpsError) as e:
            L.plan_create(L.params_init(**base))
        return e.value.code
    assert code(frame_slices=3) == L.ERR_INVALID_ARG                  # nz not a multiple
    assert code(layout=L.LAYOUT_SLICES) == L.ERR_INVALID_ARG          # slices layout has one slice per column
    assert code(precision=L.BF16_REFINE) == L.ERR_UNSUPPORTED
    assert code(nz=8 * 40, frame_slices=8) == L.ERR_UNSUPPORTED   # more than 128 slices
    assert code(wavelet_dims=3, frame_slices=4, nz=16) == L.ERR_INVALID_ARG   # 3D Haar blocks would cross frames


def test_recursion_over_two_segments(L):
    """With recursive = 1 the second segment starts from the first segment's support and its
    T singular values (one per frame column); the oracle reconstructs segment 2 with the prior
    the GPU installed."""
    from tests.abi_layout import bits_to_mallat
    T, fs, nx, ny, nc, iters = 4, 4, 16, 32, 2, 20
    c1 = segment(T, fs, nx, ny, nc, seed=3)
    x2 = segment(T, fs, nx, ny, nc, seed=8)["x"]
    d2 = c64(O.E(x2, up(c1["coils"]), c1["mask"], 1, fs))
    pl = plan_for(L, c1, T, nx, ny, nc, max_iters=iters, recursive=1, lambda_p=0.5)
    pl.reconstruct_frame(stats=False)
    words = np.empty(pl.support_words(), np.uint32)
    sig = np.empty(T)
    L.get_support(pl.handle, words, sig)
    prior = O.Prior(support=bits_to_mallat(words, T * fs, nx, ny, 3), sigma=sig.copy())
    assert prior.support.any() and np.all(sig >= 0)
    pl.set_data(dev(d2))
    recon = torch.empty((T * fs, nx, ny), dtype=torch.complex64, device="cuda")
    pl.reconstruct_frame(recon=recon)
    ref = O.priori_ls(up(d2), up(c1["coils"]), c1["mask"], oracle_params(pl.params), prior)
    assert O.nrmse(recon.cpu().numpy(), ref.recon) <= E2E_TOL
    pl.close()
