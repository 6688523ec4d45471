"""Half-precision coil maps (LPS_COILS_FP16): the acquisition operator of Sec. 2 with its coil
sensitivities rounded to IEEE binary16, read by the per-iteration kernels as 4-byte pairs.

On maps that are already half-representable the format changes nothing: a plan with
LPS_COILS_FP16 reproduces the LPS_COILS_FP32 plan bitwise (same kernels, the half pairs widen
exactly), and both match the oracle given the rounded maps. On float32 maps the plan rounds them
(round to nearest even, as numpy's float16 cast does), which the forward operator shows against
the oracle's E with maps rounded on the host.
"""
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


def rounded(c):
    """Re and Im rounded to IEEE binary16 (nearest, ties to even), back in complex64."""
    c = np.asarray(c, np.complex64)
    return c64(c.real.astype(np.float16).astype(np.float32) + 1j * c.imag.astype(np.float16).astype(np.float32))


def frame(L, case, nz, nx, ny, nc, iters, coil_format, tune=None):
    pl = L.Plan(nx, ny, nz, nc, max_iters=iters, coil_format=coil_format)
    pl.set_coils(dev(case["coils"]))
    pl.set_mask(case["mask"])
    pl.set_data(dev(case["d"]))
    if tune is not None:
        L.apply_tune(pl.handle, tune[0], tune[1], tune[2], lrs_tiles=1)
    recon = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    pl.reconstruct_frame(recon=recon)
    params = pl.params
    pl.close()
    return recon.cpu().numpy(), params


@pytest.mark.parametrize("nz,nx,ny,nc,tune", [
    (16, 32, 128, 8, None),             # register-transform kernel, coil sums in shared memory
    (16, 16, 128, 3, None),             # register-transform kernel, one coil per group
    (12, 48, 64, 3, (2, (8, 8), (4, 3))),   # runtime-sized kernel reading coil maps from global memory
    (12, 48, 64, 3, (1, (8, 8), (4, 3))),   # runtime-sized kernel with staged (float32) coil planes
])
def test_fp16_coils_equal_fp32_on_rounded_maps(L, nz, nx, ny, nc, tune):
    case = make_case(nz, nx, ny, nc, seed=71 + nc, frac=0.3)
    case["coils"] = rounded(case["coils"])
    r32, params = frame(L, case, nz, nx, ny, nc, 15, L.COILS_FP32, tune)
    r16, _ = frame(L, case, nz, nx, ny, nc, 15, L.COILS_FP16, tune)
    assert np.array_equal(r16, r32)
    ref = O.priori_ls(up(case["d"]), up(case["coils"]), case["mask"], oracle_params(params))
    assert O.nrmse(r16, ref.recon) <= E2E_TOL


def test_fp16_plan_rounds_float32_maps_to_nearest(L):
    """Float32 maps given to an LPS_COILS_FP16 plan: its forward operator is E with the maps
    rounded to binary16 (oracle E on host-rounded maps, operator bound), and differs from E with
    the float32 maps by about the binary16 rounding (2^-11 relative)."""
    nz, nx, ny, nc = 16, 16, 128, 4
    case = make_case(nz, nx, ny, nc, seed=77)
    pl = L.Plan(nx, ny, nz, nc, coil_format=L.COILS_FP16)
    pl.set_coils(dev(case["coils"]))
    m = pl.set_mask(case["mask"])
    rng = np.random.default_rng(5)
    x = c64(rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny)))
    kd = torch.empty((nc, m, nx), dtype=torch.complex64, device="cuda")
    L.forward(pl.handle, dev(x), kd)
    got = kd.cpu().numpy()
    pl.close()
    ref16 = O.E(up(x), up(rounded(case["coils"])), case["mask"])
    ref32 = O.E(up(x), up(case["coils"]), case["mask"])
    assert rel(got, ref16) < OP_TOL
    assert 1e-5 < rel(got, ref32) < 2.0 ** -10


def test_fp16_coils_cardiac_frame_against_float32_maps(L, capsys):
    """The cardiac-shaped frame (128 x 128 x 16, 8 coils) with float32 maps: the FP16 plan's
    reconstruction against the FP32 plan's (the effect of rounding the maps) and against the
    oracle given the rounded maps (parity)."""
    from paper_1411_6206_gb300 import phantom as P
    w = P.CARDIAC
    pr = P.problem(w, frames=1)
    coils = c64(pr["coils"])
    mask = pr["masks"][0]
    d = c64(O.E(pr["x"][0], up(coils), mask) + pr["noise"][0])
    case = dict(coils=coils, mask=mask, d=d)
    r32, params = frame(L, case, w.nz, w.nx, w.ny, w.ncoil, w.iters, L.COILS_FP32)
    r16, _ = frame(L, case, w.nz, w.nx, w.ny, w.ncoil, w.iters, L.COILS_FP16)
    ref16 = O.priori_ls(up(d), up(rounded(coils)), mask, oracle_params(params))
    e_model = O.nrmse(r16, r32)
    e_parity = O.nrmse(r16, ref16.recon)
    e_truth16, e_truth32 = O.nrmse(r16, pr["x"][0]), O.nrmse(r32, pr["x"][0])
    with capsys.disabled():
        print(f"\ncoil maps in binary16, cardiac frame 1: NRMSE vs float32-map recon {e_model:.3e}, vs oracle "
              f"(rounded maps) {e_parity:.3e}; vs phantom {e_truth16:.4e} (fp16) / {e_truth32:.4e} (fp32)")
    assert e_parity <= E2E_TOL
    assert e_model < 1e-2
