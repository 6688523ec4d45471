"""The data-consistency update on register transforms (planes of ny = 16 Q, Q = 4..10, by
nz in {8, 10, 12, 14, 16, 20, 24, 28, 32}; lps_tune_result.dc_variant 5): step (4) against the
oracle to the operator bound for every Q and column count, both encodes, samples staged in
shared memory or read from L2 (dense masks on the largest planes); one iteration from a
common state and a frame against the oracle; equal to the runtime-sized kernel's output
within the operator bound."""
import numpy as np
import pytest

from oracle import lps_oracle as O
from tests.gpu_cases import c64, make_case, oracle_params, rel, up

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


def plan_for(L, case, nz, nx, ny, nc, **kw):
    pl = L.Plan(nx, ny, nz, nc, **kw)
    pl.set_coils(dev(case["coils"]))
    assert pl.set_mask(dev(case["mask"])) == case["nlines"]
    pl.set_data(dev(case["d"]))
    return pl


def radix_plan(n):
    out = []
    for r in (16, 8, 4, 2, 3, 5, 7):
        while n % r == 0 and n > 1:
            out.append(r)
            n //= r
    assert n == 1
    return tuple(out)


RT_SHAPES = [
    # nz, ny, ncoil, fft_z, dense mask
    (8, 64, 2, 1, False), (10, 80, 3, 1, False), (12, 96, 2, 1, False), (14, 112, 3, 1, False),
    (16, 144, 2, 1, False), (20, 160, 3, 1, False), (24, 64, 2, 1, False), (28, 144, 2, 1, False),
    (32, 160, 2, 1, False), (32, 112, 3, 0, False), (14, 160, 5, 0, False), (20, 96, 1, 1, False),
    (32, 160, 2, 1, True), (28, 128, 2, 1, True),
]


@pytest.mark.parametrize("nz,ny,nc,fz,full", RT_SHAPES)
def test_rt_data_consistency_step(L, nz, ny, nc, fz, full):
    nx = 16
    case = make_case(nz, nx, ny, nc, seed=nz * 7 + ny, fft_z=fz, full=full)
    pl = plan_for(L, case, nz, nx, ny, nc, fft_z=fz)
    rng = np.random.default_rng(5)
    Z = c64(rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny)))
    X = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    r2 = L.data_consistency(pl.handle, dev(Z), X)
    coils, d = up(case["coils"]), up(case["d"])
    R = O.E(up(Z), coils, case["mask"], fz) - d
    Xref = up(Z) - O.EH(R, coils, case["mask"], fz)
    e = rel(X.cpu().numpy(), Xref)
    assert e < OP_TOL, e
    assert abs(r2 - np.vdot(R, R).real) < 1e-5 * np.vdot(R, R).real
    # the same step on the runtime-sized kernel (variant 2, coil maps read from L2)
    X2 = torch.empty_like(X)
    L.apply_tune(pl.handle, 2, radix_plan(ny), radix_plan(nz), lrs_tiles=1)
    L.data_consistency(pl.handle, dev(Z), X2)
    assert rel(X.cpu().numpy(), X2.cpu().numpy().astype(np.complex128)) < OP_TOL
    pl.close()


def test_rt_is_the_default_and_the_tuned_variant(L):
    """Plans of these planes start on the register-transform update; the autotuner measures it
    against the runtime-sized candidates and reports variant 5 where it wins."""
    nz, nx, ny, nc = 14, 160, 160, 8
    case = make_case(nz, nx, ny, nc, seed=8, frac=0.1)
    pl = plan_for(L, case, nz, nx, ny, nc, max_iters=2)
    L.autotune_clear_cache()
    r = pl.autotune()
    assert r.dc_variant == 5, r.as_dict()
    pl.close()


@pytest.mark.parametrize("nz,nx,ny,nc", [(14, 16, 160, 3), (20, 16, 96, 2), (32, 16, 144, 2)])
def test_rt_one_iteration_from_state(L, nz, nx, ny, nc):
    case = make_case(nz, nx, ny, nc, seed=nz + ny)
    pl = plan_for(L, case, nz, nx, ny, nc, lambda_p=0.5)
    coils, d, mask = up(case["coils"]), up(case["d"]), case["mask"]
    p = oracle_params(pl.params)
    r0 = O.priori_ls(d, coils, mask, p, iters=3)
    X, S, Lp = c64(r0.X), c64(r0.S), c64(r0.L)
    lamL, lamS = float(np.float32(r0.lambda_L)), float(np.float32(r0.lambda_S))
    L.set_state(pl.handle, dev(X), dev(S), dev(Lp), lamL, lamS, 3)
    pl.iterate(1)
    Xg = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    Lg, Sg = torch.empty_like(Xg), torch.empty_like(Xg)
    L.get_state(pl.handle, Xg, Lg, Sg)
    ref = O.priori_ls(d, coils, mask, p, None, iters=1, state=(up(X), up(S), up(Lp), lamL, lamS))
    s = ref.sigma_in
    keep = s > ref.lambda_L
    tol = max(OP_TOL, 8 * 2.0 ** -24 * s[0] ** 2 * np.sqrt(np.sum(1.0 / s[keep] ** 2)) / np.linalg.norm(ref.L))
    assert rel(Lg.cpu().numpy(), ref.L) < tol
    assert rel(Xg.cpu().numpy(), ref.X) < tol
    assert rel(Sg.cpu().numpy(), ref.S) < OP_TOL
    pl.close()


@pytest.mark.parametrize("nz,nx,ny,nc,iters", [(28, 16, 112, 2, 20), (10, 32, 80, 4, 30)])
def test_rt_frame_end_to_end(L, nz, nx, ny, nc, iters):
    case = make_case(nz, nx, ny, nc, seed=11, frac=0.3)
    pl = plan_for(L, case, nz, nx, ny, nc, max_iters=iters)
    recon = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    st = pl.reconstruct_frame(recon=recon)
    ref = O.priori_ls(up(case["d"]), up(case["coils"]), case["mask"], oracle_params(pl.params))
    assert st.iters == iters
    assert O.nrmse(recon.cpu().numpy(), ref.recon) <= E2E_TOL
    pl.close()
