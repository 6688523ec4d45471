"""Half-precision samples (LPS_DATA_FP16): the plan rounds its hybrid copy d' = F_x^H d to
binary16 and the per-iteration kernels read the half pairs. Step (4) equals the oracle's step
on the same rounding (d' rounded in float64 then mapped back by F_x) to the operator bound; a
frame stays within the end-to-end bound of the oracle on the unrounded samples, and the
rounding's effect on the frame is reported."""
import numpy as np
import pytest
import scipy.fft as sfft

from oracle import lps_oracle as O
from tests.gpu_cases import c64, make_case, oracle_params, rel, up

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def rounded_data(d):
    """k-space whose hybrid samples are the binary16 rounding of F_x^H d (float64 transform)."""
    h = sfft.ifft(up(d), axis=-1, norm="ortho")
    hr = h.real.astype(np.float16).astype(np.float64) + 1j * h.imag.astype(np.float16).astype(np.float64)
    return sfft.fft(hr, axis=-1, norm="ortho")


@pytest.mark.parametrize("nz,nx,ny,nc,variant", [(16, 16, 128, 4, 3), (14, 16, 160, 3, 5), (12, 24, 48, 2, 2),
                                                 (32, 16, 112, 2, 5)])
def test_dc_step_reads_rounded_samples(L, nz, nx, ny, nc, variant):
    case = make_case(nz, nx, ny, nc, seed=ny + nz)
    pl = L.Plan(nx, ny, nz, nc, data_format=L.DATA_FP16)
    pl.set_coils(dev(case["coils"]))
    pl.set_mask(case["mask"])
    pl.set_data(dev(case["d"]))
    if variant == 2:
        L.apply_tune(pl.handle, 2, (16, 3), (4, 3), lrs_tiles=1)
    else:
        L.apply_tune(pl.handle, variant, (), (), lrs_tiles=1)
    rng = np.random.default_rng(4)
    Z = c64(rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny)))
    X = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    L.data_consistency(pl.handle, dev(Z), X)
    coils, dr = up(case["coils"]), rounded_data(case["d"])
    R = O.E(up(Z), coils, case["mask"]) - dr
    Xref = up(Z) - O.EH(R, coils, case["mask"])
    # the GPU rounds its float32 F_x^H d: an element within float32 error of a binary16 tie may
    # round the other way (one binary16 ulp), far below this bound
    assert rel(X.cpu().numpy(), Xref) < 2e-5
    pl.close()


def test_frame_with_half_samples(L):
    nz, nx, ny, nc, iters = 16, 32, 64, 4, 30
    case = make_case(nz, nx, ny, nc, seed=9, frac=0.3)
    outs = {}
    for fmt in (L.DATA_FP32, L.DATA_FP16):
        pl = L.Plan(nx, ny, nz, nc, max_iters=iters, data_format=fmt)
        pl.set_coils(dev(case["coils"]))
        pl.set_mask(case["mask"])
        pl.set_data(dev(case["d"]))
        recon = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
        pl.reconstruct_frame(recon=recon)
        outs[fmt] = recon.cpu().numpy()
        params = pl.params
        pl.close()
    ref = O.priori_ls(up(case["d"]), up(case["coils"]), case["mask"], oracle_params(params))
    e16 = O.nrmse(outs[L.DATA_FP16], ref.recon)
    e32 = O.nrmse(outs[L.DATA_FP32], ref.recon)
    print(f"frame NRMSE vs oracle: float32 samples {e32:.3e}, binary16 samples {e16:.3e}")
    assert e16 <= E2E_TOL
    assert O.nrmse(outs[L.DATA_FP16], outs[L.DATA_FP32]) < 1e-3
