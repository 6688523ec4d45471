"""Sliding temporal window over a 2D + time stream (layout "frames"): every window against the
oracle given the same samples and the prior the GPU passed on, moved one column on the host;
the window's output frame is its last column."""
import numpy as np
import pytest

from oracle import lps_oracle as O
from tests.abi_layout import bits_to_mallat
from tests.gpu_cases import c64, oracle_params, up

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


def test_sliding_window_matches_oracle_per_window(L):
    from paper_1411_6206_gb300 import phantom as P
    from paper_1411_6206_gb300.window import SlidingWindow
    T, W, nx, ny, nc, iters = 12, 8, 32, 32, 2, 20
    w = P.Workload("stream", nx, ny, 1, nc, T, iters, 4.0, 13, phantom="heart")
    x = P.phantom_sequence(w)[:, 0]                      # [T][nx][ny]
    c1 = c64(P.coil_maps(nx, ny, 1, nc, 29)[:, 0])       # [nc][nx][ny]
    masks, samples = [], []
    for t in range(T):
        m = P.vd_mask(ny, 1, int(round(0.3 * ny)), 4, 40 + t, 0)      # [1][ny]
        d = O.E(x[t][None], up(c1)[:, None], m, 0) + P.noise(nc, int(m.sum()), nx, 1e-3, 60 + t)
        masks.append(m)
        samples.append(c64(d))
    sw = SlidingWindow(L, nx, ny, nc, W, dev(c1), max_iters=iters)
    params = oracle_params(sw.plan.params)
    coils_w = up(np.repeat(c1[:, None], W, axis=1))
    prior = None
    nwin = 0
    for t in range(T):
        out = sw.push(masks[t][0], dev(samples[t]))
        if out is None:
            assert t < W - 1
            continue
        frames = range(t - W + 1, t + 1)
        mask_w = np.concatenate([masks[s] for s in frames], axis=0)
        data_w = np.concatenate([samples[s] for s in frames], axis=1)
        ref = O.priori_ls(up(data_w), coils_w, mask_w, params, prior)
        got = sw.recon.cpu().numpy()
        err = O.nrmse(got, ref.recon)
        assert err <= E2E_TOL, (t, err)
        assert np.array_equal(out.cpu().numpy(), got[W - 1])
        # the prior of the next window: this window's support, one column on, and its sigma''
        words = np.empty(sw.plan.support_words(), np.uint32)
        sig = np.empty(W)
        L.get_support(sw.plan.handle, words, sig)
        sup = bits_to_mallat(words, W, nx, ny, 3)
        shifted = np.concatenate([sup[1:], sup[-1:]], axis=0)
        prior = O.Prior(support=shifted, sigma=sig.copy())
        nwin += 1
    assert nwin == T - W + 1
    sw.close()
