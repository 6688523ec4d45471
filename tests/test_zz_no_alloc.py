"""The allocation-free adjoint (lps_adjoint_noalloc) against the plan-based one.

lps_adjoint_noalloc serves callers that cannot allocate device memory where they need the
operator (another component owns the memory pool, allocation is forbidden after start-up,
or an allocation's device synchronisation is not acceptable); it keeps its scratch in a
fixed device array of the library. This file is collected last on purpose; it must pass
alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from tests.gpu_cases import make_case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5   # the operator tolerance of the other GPU parity tests


@pytest.fixture(scope="module")
def L():
    from paper_1411_6206_gb300 import lps
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    lps.load()
    return lps


def plan_adjoint(L, case, nz, nx, ny, nc):
    pl = L.Plan(nx, ny, nz, nc)
    pl.set_coils(torch.from_numpy(case["coils"]).cuda())
    pl.set_mask(case["mask"])
    out = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    L.adjoint(pl.handle, torch.from_numpy(case["d"]).cuda(), out)
    torch.cuda.synchronize()
    pl.close()
    return out.cpu().numpy()


@pytest.mark.parametrize("nz,nx,ny,nc", [(16, 128, 128, 8), (5, 16, 24, 3)])
def test_noalloc_adjoint_matches_plan_adjoint_twice(L, nz, nx, ny, nc):
    # two calls in a row with different data and masks: nothing of the first call's scratch
    # may leak into the second
    for seed in (31, 32):
        case = make_case(nz, nx, ny, nc, seed=seed, frac=0.3 if seed == 31 else 0.45)
        ref = plan_adjoint(L, case, nz, nx, ny, nc)
        img = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
        L.adjoint_noalloc(nx, ny, nz, nc, case["mask"], torch.from_numpy(case["coils"]).cuda(),
                          torch.from_numpy(case["d"]).cuda(), case["nlines"], img)
        torch.cuda.synchronize()
        assert rel(img.cpu().numpy(), ref) < TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(L):
    # 192 x 192 x 32 with 12 coils at 50% of the lines needs about 57 MB of scratch
    nz, nx, ny, nc = 32, 192, 192, 12
    mask = np.zeros((nz, ny), np.uint8)
    mask.ravel()[::2] = 1
    m = int(mask.sum())
    coils = torch.zeros((nc, nz, nx, ny), dtype=torch.complex64, device="cuda")
    kd = torch.zeros((nc, m, nx), dtype=torch.complex64, device="cuda")
    img = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    with pytest.raises(L.LpsError) as e:
        L.adjoint_noalloc(nx, ny, nz, nc, mask, coils, kd, m, img)
    assert e.value.code == L.ERR_UNSUPPORTED
