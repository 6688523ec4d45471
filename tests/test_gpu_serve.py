"""Serving loop: sessions admitted by a device-memory budget, frames of concurrent sessions
overlapping on the device; each result is the same alone and in the mix, and latencies are
accounted on the server clock."""
import time

import numpy as np
import pytest

from tests.gpu_cases import make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SESSIONS = [(8, 32, 32, 2), (16, 48, 64, 3), (12, 40, 40, 4), (5, 64, 48, 1)]
FRAMES = 3
ITERS = 10


@pytest.fixture(scope="module")
def L():
    from paper_1411_6206_gb300 import lps
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    lps.load()
    return lps


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def session_frames(k, nz, nx, ny, nc):
    fr = [make_case(nz, nx, ny, nc, seed=60 + 11 * k + t, frac=0.35) for t in range(FRAMES)]
    return fr[0]["coils"], [(f["mask"], dev(f["d"])) for f in fr]


def params(L, nz, nx, ny, nc):
    return L.params_init(nx=nx, ny=ny, nz=nz, ncoil=nc, max_iters=ITERS, recursive=1)


def test_each_result_same_alone_and_in_the_mix(L):
    data = [session_frames(k, *s) for k, s in enumerate(SESSIONS)]
    # alone: one session at a time, one frame at a time
    alone = []
    for (nz, nx, ny, nc), (coils, frames) in zip(SESSIONS, data):
        srv = L.Server(1 << 40, max_inflight=1)
        sid = srv.open(params(L, nz, nx, ny, nc), dev(coils))
        outs = []
        for mask, kd in frames:
            t = srv.submit(sid, mask, kd, srv.now())
            srv.wait(t)
            out = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
            outs.append(srv.result(sid, out).cpu().numpy())
            srv.release(t)
        srv.close()
        alone.append(outs)
    # in the mix: every session's frame t submitted together, no slot limit
    srv = L.Server(1 << 40, max_inflight=0)
    sids = [srv.open(params(L, *s), dev(c)) for s, (c, _) in zip(SESSIONS, data)]
    for t in range(FRAMES):
        tickets = [srv.submit(sid, *data[k][1][t], srv.now()) for k, sid in enumerate(sids)]
        for k, (sid, tk) in enumerate(zip(sids, tickets)):
            lat, comp = srv.wait(tk)
            assert lat >= 0.0 and comp > 0.0
            nz, nx, ny, _ = SESSIONS[k]
            out = torch.empty((nz, nx, ny), dtype=torch.complex64, device="cuda")
            got = srv.result(sid, out).cpu().numpy()
            assert np.array_equal(got, alone[k][t]), (k, t)   # bitwise
            srv.release(tk)
    srv.close()


def test_admission_by_budget(L):
    from paper_1411_6206_gb300 import lps
    nz, nx, ny, nc = SESSIONS[1]
    p = params(L, nz, nx, ny, nc)
    need = lps.estimate_device_bytes(p)
    srv = L.Server(need + need // 2, max_inflight=0)
    coils, frames = session_frames(1, nz, nx, ny, nc)
    a = srv.open(p, dev(coils))
    assert srv.bytes_in_use() == need
    with pytest.raises(L.LpsError) as e:
        srv.open(p, dev(coils))
    assert e.value.code == L.ERR_ADMISSION
    t = srv.submit(a, *frames[0], srv.now())
    with pytest.raises(L.LpsError):
        srv.close_session(a)              # a frame is still queued or on the device
    srv.wait(t)
    srv.release(t)
    srv.close_session(a)
    assert srv.bytes_in_use() == 0
    b = srv.open(p, dev(coils))           # admitted once memory is free again
    srv.close_session(b)
    srv.close()


def test_slots_limit_frames_on_device_and_latency_accounting(L):
    data = [session_frames(k, *s) for k, s in enumerate(SESSIONS)]
    srv = L.Server(1 << 40, max_inflight=2)
    sids = [srv.open(params(L, *s), dev(c)) for s, (c, _) in zip(SESSIONS, data)]
    rng = np.random.default_rng(3)
    arrivals = np.cumsum(rng.exponential(0.002, size=len(sids) * FRAMES))
    t0 = srv.now()
    tickets = []
    for i, a in enumerate(arrivals):
        k, t = i % len(sids), i // len(sids)
        while srv.now() < t0 + a:
            time.sleep(0.0002)
        tickets.append(srv.submit(sids[k], *data[k][1][t], t0 + a))
    comps = []
    for tk in tickets:
        lat, comp = srv.wait(tk)
        assert lat > 0.0
        comps.append(comp)
        srv.release(tk)
    # frames of one session complete in submission order
    for k in range(len(sids)):
        ck = comps[k::len(sids)]
        assert all(x < y for x, y in zip(ck, ck[1:]))
    srv.close()
