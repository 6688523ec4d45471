"""The bounded-wait failure path on the GPU without a fault: a one-shot test hook makes every CTA
of the staged-coil data-consistency kernel wait on an mbarrier that nothing completes, with a
short poll budget. The call returns LPS_ERR_TIMEOUT after the kernel drained its in-flight coil
copies, and the same plan then runs the step normally (the context stays usable)."""
import numpy as np
import pytest

from oracle import lps_oracle as O
from tests.gpu_cases import c64, make_case, rel, up

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1411_6206_gb300 import lps
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    lps.load()
    return lps


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("nc", [1, 3])
def test_wait_runs_out_and_the_plan_recovers(L, nc):
    nz, nx, ny = 8, 16, 48
    case = make_case(nz, nx, ny, nc, seed=21)
    pl = L.Plan(nx, ny, nz, nc)
    pl.set_coils(dev(case["coils"]))
    pl.set_mask(case["mask"])
    pl.set_data(dev(case["d"]))
    with pytest.raises(L.LpsError) as e:      # the hook needs the staged-coil kernel
        L.test_stall_wait(pl.handle, 100)
    assert e.value.code == L.ERR_STATE
    L.apply_tune(pl.handle, 1, (16, 3), (8,), lrs_tiles=1)
    rng = np.random.default_rng(6)
    Z = c64(rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny)))
    X = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    L.test_stall_wait(pl.handle, 2000)
    with pytest.raises(L.LpsError) as e:
        L.data_consistency(pl.handle, dev(Z), X)
    assert e.value.code == L.ERR_TIMEOUT
    # the hook is one-shot: the next call runs the step, and matches the oracle
    r2 = L.data_consistency(pl.handle, dev(Z), X)
    coils, d = up(case["coils"]), up(case["d"])
    R = O.E(up(Z), coils, case["mask"]) - d
    assert rel(X.cpu().numpy(), up(Z) - O.EH(R, coils, case["mask"])) < 1e-5
    assert abs(r2 - np.vdot(R, R).real) < 1e-5 * np.vdot(R, R).real
    # and a whole frame still runs on the same plan
    st = pl.reconstruct_frame(stats=True)
    assert st.iters == pl.params.max_iters
    pl.close()
