"""The 3D Haar variant of the sparsifying transform (wavelet_dims = 3: the per-slice 2D pyramid
times the J-level 1D Haar along z) through the C ABI against the FP64 oracle's T3: one iteration
from a common state (with and without a prior support in the 3D numbering), the support bits,
lambda_S of step (0), whole frames and the recursion over two frames."""
import numpy as np
import pytest

from oracle import lps_oracle as O
from tests.abi_layout import bits_to_mallat, mallat_to_bits
from tests.gpu_cases import c64, make_case, oracle_params, rel, up

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
E2E_TOL = 1e-3
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def L():
    from paper_1411_6206_gb300 import lps
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    lps.load()
    return lps


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def plan_for(L, case, nz, nx, ny, nc, **kw):
    pl = L.Plan(nx, ny, nz, nc, wavelet_dims=3, **kw)
    pl.set_coils(dev(case["coils"]))
    assert pl.set_mask(dev(case["mask"])) == case["nlines"]
    pl.set_data(dev(case["d"]))
    return pl


def support_diff_in_band(words, ref, nz, nx, ny, J, band=1e-5):
    got = bits_to_mallat(words, nz, nx, ny, J, 3)
    diff = got != ref.support
    cabs = np.abs(ref.c)
    near = np.abs(cabs - ref.lambda_S) / cabs.max() <= band
    assert not (diff & ~near).any(), f"{int((diff & ~near).sum())} support bits differ off the tie band"
    return int(diff.sum())


@pytest.mark.parametrize("with_prior", [False, True])
@pytest.mark.parametrize("nz,nx,ny,nc,J", [(8, 32, 32, 2, 3), (16, 16, 24, 3, 3), (16, 128, 128, 8, 3),
                                           (12, 16, 16, 2, 2), (6, 16, 8, 2, 1), (32, 16, 16, 2, 3)])
def test_one_iteration_from_state_3d(L, nz, nx, ny, nc, J, with_prior):
    case = make_case(nz, nx, ny, nc, seed=17 + nz)
    pl = plan_for(L, case, nz, nx, ny, nc, lambda_p=0.5, wavelet_levels=J)
    coils, d, mask = up(case["coils"]), up(case["d"]), case["mask"]
    p = oracle_params(pl.params)
    assert p.wavelet_dims == 3
    r0 = O.priori_ls(d, coils, mask, p, iters=3)
    X, S, Lp = c64(r0.X), c64(r0.S), c64(r0.L)
    lamL, lamS = float(np.float32(r0.lambda_L)), float(np.float32(r0.lambda_S))
    prior = None
    if with_prior:
        sup = np.abs(O.T3(up(X) - up(Lp), J)) > 1.5 * lamS
        sig = r0.sigma * (1.0 + 0.04 * np.cos(np.arange(nz)))
        prior = O.Prior(support=sup, sigma=sig)
        pl.set_prior(dev(mallat_to_bits(sup, J, 3)), dev(sig))
    L.set_state(pl.handle, dev(X), dev(S), dev(Lp), lamL, lamS, 3)
    pl.iterate(1)
    Xg = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    Lg, Sg = torch.empty_like(Xg), torch.empty_like(Xg)
    L.get_state(pl.handle, Xg, Lg, Sg)
    words = np.empty(pl.support_words(), np.uint32)
    L.get_support(pl.handle, words, None)
    ref = O.priori_ls(d, coils, mask, p, prior, iters=1, state=(up(X), up(S), up(Lp), lamL, lamS))
    # the sparse step thresholds T3(X - L_prev) of the common state: the operator bound
    eS = rel(Sg.cpu().numpy(), ref.S)
    assert eS < OP_TOL, eS
    # L and X go through the float32 Gram of step (1): its bound (rank-weighted u sigma_1^2)
    s = ref.sigma_in
    keep = s > ref.lambda_L
    tol = max(OP_TOL, 8 * U32 * s[0] ** 2 * np.sqrt(np.sum(1.0 / s[keep] ** 2)) / np.linalg.norm(ref.L))
    assert rel(Lg.cpu().numpy(), ref.L) < tol
    assert rel(Xg.cpu().numpy(), ref.X) < tol
    support_diff_in_band(words, ref, nz, nx, ny, J)
    # the 3D transform is in use: the per-slice one gives another sparse part
    if not with_prior:
        r2 = O.priori_ls(d, coils, mask, oracle_params(pl.params, wavelet_dims=2), None, iters=1,
                         state=(up(X), up(S), up(Lp), lamL, lamS))
        assert rel(r2.S, ref.S) > 100 * OP_TOL
    pl.close()


@pytest.mark.parametrize("nz,nx,ny,nc,J,iters", [(8, 32, 32, 2, 3, 30), (16, 16, 24, 3, 3, 20),
                                                 (12, 32, 16, 2, 2, 20)])
def test_frame_end_to_end_3d(L, nz, nx, ny, nc, J, iters):
    case = make_case(nz, nx, ny, nc, seed=29, frac=0.3)
    pl = plan_for(L, case, nz, nx, ny, nc, max_iters=iters, wavelet_levels=J)
    recon = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    sup = torch.empty(pl.support_words(), dtype=torch.int32, device="cuda")
    st = pl.reconstruct_frame(recon=recon, support=sup)
    ref = O.priori_ls(up(case["d"]), up(case["coils"]), case["mask"], oracle_params(pl.params))
    assert st.iters == iters
    # lambda_S of step (0) is rel_S max|T3(X_0)| (the max-only pass of the 3D kernel)
    assert abs(st.lambda_S - ref.lambda_S) < 1e-5 * ref.lambda_S
    lam2 = O.initial_lambdas(O.EH(up(case["d"]), up(case["coils"]), case["mask"]),
                             oracle_params(pl.params, wavelet_dims=2))[1]
    assert abs(lam2 - ref.lambda_S) > 1e-3 * ref.lambda_S
    assert O.nrmse(recon.cpu().numpy(), ref.recon) <= E2E_TOL
    # the full frame's support: bits away from the threshold agree (tie band of 1e-3 max|c|
    # after the iterations' float32 rounding), at most 0.5 % differ
    words = sup.cpu().numpy().view(np.uint32)
    got = bits_to_mallat(words, nz, nx, ny, J, 3)
    diff = got != ref.support
    cabs = np.abs(ref.c)
    near = np.abs(cabs - ref.lambda_S) / cabs.max() <= 1e-3
    assert not (diff & ~near).any()
    assert diff.sum() <= 0.005 * ref.support.sum() + 2
    pl.close()


def test_recursion_over_two_frames_3d(L):
    """Frame 2 starts from frame 1's support (3D numbering) and sigma''; the oracle runs frame 2
    with the prior the GPU installed."""
    nz, nx, ny, nc, iters = 16, 32, 32, 2, 20
    c0 = make_case(nz, nx, ny, nc, seed=41, frac=0.3)
    # frame 2: another image, the same coils and lines
    x2 = make_case(nz, nx, ny, nc, seed=42, frac=0.3)["x"]
    d2 = c64(O.E(x2, up(c0["coils"]), c0["mask"]))
    pl = plan_for(L, c0, nz, nx, ny, nc, max_iters=iters, recursive=1, lambda_p=0.5)
    pl.reconstruct_frame(stats=False)
    words = np.empty(pl.support_words(), np.uint32)
    sig = np.empty(nz)
    L.get_support(pl.handle, words, sig)
    prior = O.Prior(support=bits_to_mallat(words, nz, nx, ny, 3, 3), sigma=sig.copy())
    assert prior.support.any()
    pl.set_data(dev(d2))
    recon = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    pl.reconstruct_frame(recon=recon)
    ref = O.priori_ls(up(d2), up(c0["coils"]), c0["mask"], oracle_params(pl.params), prior)
    assert O.nrmse(recon.cpu().numpy(), ref.recon) <= E2E_TOL
    pl.close()


def test_3d_support_has_no_column_shift(L):
    case = make_case(8, 16, 16, 2, seed=3)
    pl = plan_for(L, case, 8, 16, 16, 2)
    with pytest.raises(L.LpsError) as e:
        L.shift_prior_columns(pl.handle, 1)
    assert e.value.code == -1
    pl.close()
