"""Degenerate inputs against the oracle: one Casorati column (a single slice; 3D frames with one
frame), one sampled line, the smallest plane the library takes (8 x 8, 3 slices, one coil),
all-zero samples (every threshold zero, a zero Gram: the reconstruction is exactly zero), and
an empty mask (refused on the host)."""
import numpy as np
import pytest

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


def run(L, case, nz, nx, ny, nc, iters=20, **kw):
    pl = L.Plan(nx, ny, nz, nc, max_iters=iters, **kw)
    pl.set_coils(dev(case["coils"]))
    pl.set_mask(case["mask"])
    pl.set_data(dev(case["d"]))
    recon = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    st = pl.reconstruct_frame(recon=recon)
    params = pl.params
    pl.close()
    return recon.cpu().numpy(), st, params


@pytest.mark.parametrize("nz,nx,ny,nc,fz", [(1, 16, 32, 2, 1), (1, 16, 16, 1, 0), (3, 8, 8, 1, 1)])
def test_single_column_and_smallest_plane(L, nz, nx, ny, nc, fz):
    case = make_case(nz, nx, ny, nc, seed=3 + nz, fft_z=fz, frac=0.5, centre=min(4, ny, nz))
    recon, st, params = run(L, case, nz, nx, ny, nc, fft_z=fz)
    ref = O.priori_ls(up(case["d"]), up(case["coils"]), case["mask"], oracle_params(params))
    assert O.nrmse(recon, ref.recon) <= E2E_TOL
    assert abs(st.lambda_L - ref.lambda_L) < 1e-5 * ref.lambda_L


def test_one_frame_volume_as_the_only_column(L):
    from paper_1411_6206_gb300 import phantom as P
    fs, nx, ny, nc = 8, 16, 16, 2
    x = P.phantom_sequence(P.Workload("one", nx, ny, fs, nc, 1, 10, 3.0, 5, phantom="ellipsoids"))[0]
    coils = c64(P.coil_maps(nx, ny, fs, nc, 7))
    mask = P.vd_mask(ny, fs, int(0.4 * ny * fs), 4, 9, 1)
    d = c64(O.E(x, up(coils), mask, 1, fs) + P.noise(nc, int(mask.sum()), nx, 1e-3, 11))
    case = dict(coils=coils, mask=mask, d=d)
    recon, st, params = run(L, case, fs, nx, ny, nc, layout=L.LAYOUT_FRAMES, frame_slices=fs)
    assert params.frame_slices == fs
    ref = O.priori_ls(up(d), up(coils), mask, oracle_params(params))
    assert O.nrmse(recon, ref.recon) <= E2E_TOL


def test_one_sampled_line(L):
    nz, nx, ny, nc = 8, 16, 32, 2
    case = make_case(nz, nx, ny, nc, seed=4)
    mask = np.zeros((nz, ny), np.uint8)
    mask[0, 0] = 1
    case["mask"] = mask
    case["d"] = c64(O.E(case["x"], up(case["coils"]), mask))
    pl = L.Plan(nx, ny, nz, nc)
    pl.set_coils(dev(case["coils"]))
    assert pl.set_mask(mask) == 1
    pl.set_data(dev(case["d"]))
    rng = np.random.default_rng(2)
    Z = c64(rng.standard_normal((nz, nx, ny)) + 1j * rng.standard_normal((nz, nx, ny)))
    X = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
    L.data_consistency(pl.handle, dev(Z), X)
    R = O.E(up(Z), up(case["coils"]), mask) - up(case["d"])
    assert rel(X.cpu().numpy(), up(Z) - O.EH(R, up(case["coils"]), mask)) < 1e-5
    pl.close()
    recon, st, params = run(L, case, nz, nx, ny, nc)
    ref = O.priori_ls(up(case["d"]), up(case["coils"]), mask, oracle_params(params))
    assert O.nrmse(recon, ref.recon) <= E2E_TOL


def test_zero_samples_give_zero(L):
    nz, nx, ny, nc = 8, 16, 32, 2
    case = make_case(nz, nx, ny, nc, seed=6)
    case["d"] = np.zeros_like(case["d"])
    recon, st, params = run(L, case, nz, nx, ny, nc, iters=5)
    assert st.iters == 5
    assert np.all(recon == 0)
    assert st.lambda_L == 0 and st.lambda_S == 0


def test_empty_mask_is_refused(L):
    pl = L.Plan(16, 16, 4, 1)
    with pytest.raises(L.LpsError) as e:
        pl.set_mask(np.zeros((4, 16), np.uint8))
    assert e.value.code == L.ERR_INVALID_ARG
    pl.close()
