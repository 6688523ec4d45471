"""Precision modes (LPS_TF32_REFINE, LPS_BF16_REFINE): the Casorati Gram and the low-rank
reprojection on the tensor cores with split operands (one refinement step), against the FP64
oracle, and whole frames against the oracle at the end-to-end tolerance.

Operator bounds. With unit roundoff u of the operand type (bf16: 2^-9, tf32: 2^-11), the split
x = hi + lo leaves |x - hi - lo| <= u^2 |x| and the dropped lo*lo term is <= u^2 |x||y|, so one
product carries at most ~3 u^2 |x||y| beyond float32 rounding. Summed over the Casorati rows,
|dG_ij| <= 3 u^2 ||m_i|| ||m_j|| (Cauchy-Schwarz), i.e. ||dG||_F <= 3 u^2 trace(G); float32
accumulation adds about (K + P) 2^-24 trace(G) for K rows per partial and P partials.
"""
import os

import numpy as np
import pytest

from oracle import lps_oracle as O
from tests.abi_layout import bits_to_mallat
from tests.gpu_cases import c64, make_case, oracle_params, rel, up

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E2E_TOL = 1e-3
U_OP = {1: 2.0 ** -11, 2: 2.0 ** -9}          # TF32_REFINE, BF16_REFINE
NAMES = {0: "fp32", 1: "tf32", 2: "bf16"}


@pytest.fixture(scope="module")
def L():
    from paper_1411_6206_gb300 import lps
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    lps.load()
    return lps


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gram_bound(G, mode, K, P):
    tr = float(np.real(np.trace(G)))
    u2 = 3 * U_OP[mode] ** 2 if mode else 0.0
    return 2.0 * (u2 + (K + P) * 2.0 ** -24) * tr


SHAPES = [(8, 32, 32), (5, 16, 24), (16, 64, 48), (32, 64, 64), (12, 40, 48)]


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("nz,nx,ny", SHAPES)
def test_casorati_gram_matches_definition(L, mode, nz, nx, ny):
    rng = np.random.default_rng(nz * 1000 + nx + mode)
    X = c64(rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny)))
    S = c64(0.3 * (rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny))))
    pl = L.Plan(nx, ny, nz, 1, precision=mode)
    G = torch.empty((nz, nz), dtype=torch.complex64, device="cuda")
    for s_arg, s_ref in ((dev(S), up(S)), (None, None)):
        L.casorati_gram(pl.handle, dev(X), s_arg, G)
        torch.cuda.synchronize()
        Gg = G.cpu().numpy().astype(np.complex128)
        Gr = O.casorati_gram(up(X), s_ref)
        # K rows per partial: 128-pixel tiles (tensor cores) or ny per x-plane (float32)
        K = 2 * 128 if mode else ny
        P = 148 if mode else nx
        assert np.linalg.norm(Gg - Gr) <= gram_bound(Gr, mode, K, P), (NAMES[mode], rel(Gg, Gr))
        assert np.array_equal(Gg, Gg.conj().T)   # exactly Hermitian
    pl.close()


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("nz,nx,ny", SHAPES)
def test_lowrank_reproject_matches_definition(L, mode, nz, nx, ny):
    rng = np.random.default_rng(nz * 7 + nx + mode)
    X = c64(rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny)))
    S = c64(0.3 * (rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny))))
    # W = V diag(f) V^H with f in [0, 1]: the shape of the SVT's reprojection matrix
    Q, _ = np.linalg.qr(rng.standard_normal((nz, nz)) + 1j * rng.standard_normal((nz, nz)))
    f = np.sort(rng.random(nz))[::-1]
    W = c64((Q * f) @ Q.conj().T)
    pl = L.Plan(nx, ny, nz, 1, precision=mode)
    Lg = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    L.lowrank_reproject(pl.handle, dev(X), dev(S), dev(W), Lg)
    torch.cuda.synchronize()
    Lr = O.reproject(up(X), up(S), up(W))
    M = up(X) - up(S)
    # per element: sum over nz terms of |m_i||w_ij| with (3 u^2 + nz 2^-24) relative error
    u2 = 3 * U_OP[mode] ** 2 if mode else 0.0
    bound = 2.0 * (u2 + nz * 2.0 ** -24) * np.linalg.norm(M) * np.linalg.norm(np.abs(up(W)), 2) * np.sqrt(nz)
    assert np.linalg.norm(Lg.cpu().numpy() - Lr) <= bound, (NAMES[mode], rel(Lg.cpu().numpy(), Lr))
    pl.close()


def run_frame(L, case, nz, nx, ny, nc, iters, mode):
    pl = L.Plan(nx, ny, nz, nc, max_iters=iters, precision=mode, eig_precision=L.EIG_FP64)
    pl.set_coils(dev(case["coils"]))
    pl.set_mask(case["mask"])
    pl.set_data(dev(case["d"]))
    recon = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    st = pl.reconstruct_frame(recon=recon)
    return pl, st, recon.cpu().numpy()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("nz,nx,ny,nc,iters", [(8, 32, 32, 1, 30), (16, 32, 64, 4, 30), (5, 16, 24, 3, 20)])
def test_frame_end_to_end_precision(L, mode, nz, nx, ny, nc, iters):
    case = make_case(nz, nx, ny, nc, seed=5, frac=0.3)
    pl, st, recon = run_frame(L, case, nz, nx, ny, nc, iters, mode)
    ref = O.priori_ls(up(case["d"]), up(case["coils"]), case["mask"], oracle_params(pl.params))
    err = O.nrmse(recon, ref.recon)
    assert err <= E2E_TOL, (NAMES[mode], err)
    assert st.iters == iters
    assert abs(st.lambda_L - ref.lambda_L) < 1e-4 * ref.lambda_L
    pl.close()


def test_precision_workload_per_mode_nrmse(L, capsys):
    """Config of the precision study (192 x 192 x 32, 12 coils, 10x): frames 1 and 2 of the
    recursive sequence in float32, tf32 and bf16 modes (FP64 eigendecomposition in the latter
    two), each against the oracle given the same inputs and the prior that mode produced."""
    import scipy.fft as sfft
    from paper_1411_6206_gb300 import phantom as P
    w = P.PRECISION
    pr = P.problem(w, frames=2)
    coils = c64(pr["coils"])
    datas = [c64(O.E(pr["x"][t], up(coils), pr["masks"][t]) + pr["noise"][t]) for t in range(2)]
    recon = torch.empty((w.nz, w.nx, w.ny), dtype=torch.complex64, device="cuda")
    report = {}
    ref1 = None
    for mode in (0, 1, 2):
        pl = L.Plan(w.nx, w.ny, w.nz, w.ncoil, max_iters=w.iters, recursive=1, precision=mode,
                    eig_precision=L.EIG_FP64 if mode else L.EIG_FP32)
        pl.set_coils(dev(coils))
        p = oracle_params(pl.params)
        sup = np.empty(pl.support_words(), np.uint32)
        sig = np.empty(w.nz)
        prior = None
        errs = []
        for t in range(2):
            pl.set_mask(pr["masks"][t])
            pl.set_data(dev(datas[t]))
            pl.reconstruct_frame(recon=recon, support=sup, sigma=sig)
            with sfft.set_workers(os.cpu_count()):
                if t == 0 and ref1 is not None:
                    ref = ref1
                else:
                    ref = O.priori_ls(up(datas[t]), up(coils), pr["masks"][t], p, prior)
                    if t == 0:
                        ref1 = ref
            errs.append(O.nrmse(recon.cpu().numpy(), ref.recon))
            prior = O.Prior(support=bits_to_mallat(sup, w.nz, w.nx, w.ny, 3), sigma=sig.copy())
        pl.close()
        report[NAMES[mode]] = errs
    with capsys.disabled():
        print(f"\nprecision workload NRMSE vs FP64 oracle (frames 1, 2): {report}")
    for k, errs in report.items():
        assert max(errs) <= E2E_TOL, (k, errs)
