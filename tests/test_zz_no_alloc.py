"""The allocation-free adjoint (lps_adjoint_noalloc) against the plan-based one and the oracle.

lps_adjoint_noalloc serves callers that cannot allocate device memory where they need the
operator (another component owns the memory pool, allocation is forbidden after start-up,
or an allocation's device synchronisation is not acceptable); it keeps its scratch in a
fixed device array of the library. This file is collected last on purpose; it must pass
alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from oracle import lps_oracle as O
from tests.gpu_cases import make_case, rel, up

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


def oracle_adjoint(case):
    return O.EH(up(case["d"]), up(case["coils"]), case["mask"], 1)


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
        got = img.cpu().numpy()
        assert rel(got, ref) < TOL
        assert rel(got, oracle_adjoint(case)) < TOL


def test_noalloc_back_to_back_on_one_stream(L):
    """Two calls queued on one stream with different masks and data and no host
    synchronisation between them: both results match the oracle's adjoint."""
    nz, nx, ny, nc = 16, 128, 128, 8
    cases = [make_case(nz, nx, ny, nc, seed=41, frac=0.25), make_case(nz, nx, ny, nc, seed=42, frac=0.5)]
    dev = [(torch.from_numpy(c["coils"]).cuda(), torch.from_numpy(c["d"]).cuda()) for c in cases]
    outs = [torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda") for _ in cases]
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        for c, (co, d), o in zip(cases, dev, outs):
            L.adjoint_noalloc(nx, ny, nz, nc, c["mask"], co, d, c["nlines"], o, stream=st)
    st.synchronize()
    for c, o in zip(cases, outs):
        assert rel(o.cpu().numpy(), oracle_adjoint(c)) < TOL


def test_noalloc_rejects_host_buffers(L):
    """Host coils, samples or output (and a device mask) are refused on the host, before
    anything is enqueued: nothing is launched on memory the kernels cannot address."""
    nz, nx, ny, nc = 5, 16, 24, 3
    case = make_case(nz, nx, ny, nc, seed=33)
    coils_d = torch.from_numpy(case["coils"]).cuda()
    d_d = torch.from_numpy(case["d"]).cuda()
    img_d = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    img_h = torch.empty((nz, nx, ny), dtype=torch.complex64)
    bad = [
        (case["mask"], torch.from_numpy(case["coils"]), d_d, img_d),
        (case["mask"], coils_d, torch.from_numpy(case["d"]), img_d),
        (case["mask"], coils_d, d_d, img_h),
        (torch.from_numpy(case["mask"]).cuda(), coils_d, d_d, img_d),
    ]
    for mask, co, d, img in bad:
        with pytest.raises(L.LpsError) as e:
            L.adjoint_noalloc(nx, ny, nz, nc, mask, co, d, case["nlines"], img)
        assert e.value.code == L.ERR_INVALID_ARG
    with pytest.raises(L.LpsError) as e:
        L.adjoint_noalloc(nx, ny, nz, nc, case["mask"], coils_d, d_d, case["nlines"] + 1, img_d)
    assert e.value.code == L.ERR_INVALID_ARG and "nlines" in str(e.value)
    torch.cuda.synchronize()


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
    assert e.value.code == L.ERR_UNSUPPORTED and "scratch" in str(e.value)
