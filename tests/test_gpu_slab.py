"""x-slab sharding through the C ABI on one GPU: a volume held by two slab plans whose records
the driver reduces after every call (the reduction a multi-GPU run does with one all-reduce),
against the plan that holds the whole volume and against the oracle."""
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


def whole_frame(L, case, nz, nx, ny, nc, iters):
    pl = L.Plan(nx, ny, nz, nc, max_iters=iters, stream=torch.cuda.current_stream())
    pl.set_coils(dev(case["coils"]))
    pl.set_mask(case["mask"])
    pl.set_data(dev(case["d"]))
    recon = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    sig = np.empty(nz)
    pl.reconstruct_frame(recon=recon, sigma=sig)
    params = pl.params
    pl.close()
    return recon.cpu().numpy(), sig, params


@pytest.mark.parametrize("nz,nx,ny,nc,parts", [(16, 128, 128, 8, 2), (12, 48, 64, 3, 2), (8, 40, 32, 2, 3)])
def test_slab_plans_equal_the_whole_volume(L, nz, nx, ny, nc, parts):
    from paper_1411_6206_gb300 import shard
    iters = 30
    case = make_case(nz, nx, ny, nc, seed=91 + nx, frac=0.3)
    ref_gpu, sig_gpu, params = whole_frame(L, case, nz, nx, ny, nc, iters)
    ranges = shard.slab_ranges(nx, parts)
    slabs, plans = [], []
    for x0, n in ranges:
        pl = L.Plan(n, ny, nz, nc, max_iters=iters, nx_total=nx, x0=x0, stream=torch.cuda.current_stream())
        pl.set_coils(dev(case["coils"][:, :, x0:x0 + n, :]))
        pl.set_mask(case["mask"])
        pl.set_data(dev(case["d"]))
        plans.append(pl)
        slabs.append(shard.LibrarySlab(L, pl, "cuda"))
    stats = shard.reconstruct_frame(slabs, shard.Reducer(slabs[0].nsum), iters)
    assert all(s.iters == iters for s in stats)
    recon = np.zeros((nz, nx, ny), np.complex64)
    sigs = []
    for (x0, n), pl in zip(ranges, plans):
        part = torch.empty((nz, n, ny), dtype=torch.complex64, device="cuda")
        L.get_recon(pl.handle, part)
        recon[:, x0:x0 + n, :] = part.cpu().numpy()
        sg = np.empty(nz)
        L.get_support(pl.handle, None, sg)
        sigs.append(sg)
        pl.close()
    for sg in sigs[1:]:
        assert np.array_equal(sg, sigs[0])   # every slab takes the same steps (1)-(2)
    assert O.nrmse(recon, ref_gpu) < 1e-4
    ref = O.priori_ls(up(case["d"]), up(case["coils"]), case["mask"], oracle_params(params))
    assert O.nrmse(recon, ref.recon) <= E2E_TOL
    assert abs(stats[0].lambda_L - ref.lambda_L) < 1e-5 * ref.lambda_L
    assert abs(stats[0].lambda_S - ref.lambda_S) < 1e-5 * ref.lambda_S


def test_slab_operators_share_the_volume(L):
    """The slabs' forward outputs add up to E x; the adjoint of whole readouts gives each slab
    its planes of E^H d."""
    from paper_1411_6206_gb300 import shard
    nz, nx, ny, nc = 8, 48, 32, 3
    case = make_case(nz, nx, ny, nc, seed=5)
    rng = np.random.default_rng(2)
    x = c64(rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny)))
    tot = None
    for x0, n in shard.slab_ranges(nx, 2):
        pl = L.Plan(n, ny, nz, nc, nx_total=nx, x0=x0)
        pl.set_coils(dev(case["coils"][:, :, x0:x0 + n, :]))
        m = pl.set_mask(case["mask"])
        kd = torch.empty((nc, m, nx), dtype=torch.complex64, device="cuda")
        L.forward(pl.handle, dev(x[:, x0:x0 + n, :]), kd)
        tot = kd.cpu().numpy().astype(np.complex128) + (0 if tot is None else tot)
        img = torch.empty((nz, n, ny), dtype=torch.complex64, device="cuda")
        L.adjoint(pl.handle, dev(case["d"]), img)
        refa = O.EH(up(case["d"]), up(case["coils"]), case["mask"])[:, x0:x0 + n, :]
        assert rel(img.cpu().numpy(), refa) < OP_TOL
        pl.set_data(dev(case["d"]))
        with pytest.raises(L.LpsError) as e:
            pl.reconstruct_frame()
        assert e.value.code == L.ERR_STATE
        pl.close()
    assert rel(tot, O.E(up(x), up(case["coils"]), case["mask"])) < OP_TOL
