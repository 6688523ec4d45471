"""x-slab sharding on the CPU: the partition, and the sharded iteration over gloo ranks against
the unsharded oracle.

The driver (paper_1411_6206_gb300/shard.py: partition, call order, record reduction) runs
unchanged over slabs of the FP64 oracle's Algorithm 1 (tests/slab_oracle.py): two gloo ranks,
one slab each, the records all-reduced every iteration; the assembled reconstruction and the
singular values equal those of the unsharded oracle.
"""
import os
import socket

import numpy as np
import pytest

from oracle import lps_oracle as O
from paper_1411_6206_gb300 import phantom as P
from paper_1411_6206_gb300 import shard

torch = pytest.importorskip("torch")

NZ, NXT, NY, NC, ITERS = 4, 32, 16, 2, 8


def problem():
    w = P.Workload("slab", NXT, NY, NZ, NC, 2, ITERS, 3.0, 23, phantom="heart")
    pr = P.problem(w, frames=1)
    x = pr["x"][0]
    coils = pr["coils"]
    mask = pr["masks"][0]
    d = O.E(x, coils, mask) + pr["noise"][0]
    return d, coils, mask


def params():
    return O.Params(max_iters=ITERS, lambda_p=0.5)


def test_slab_ranges_partition_whole_tiles():
    assert shard.slab_ranges(128, 2) == [(0, 64), (64, 64)]
    assert shard.slab_ranges(40, 3) == [(0, 16), (16, 16), (32, 8)]
    for nxt, parts in ((128, 5), (64, 8), (24, 1)):
        r = shard.slab_ranges(nxt, parts)
        assert sum(n for _, n in r) == nxt and all(n % 8 == 0 and n > 0 for _, n in r)
        assert all(a + n == b for (a, n), (b, _) in zip(r, r[1:]))
    with pytest.raises(ValueError):
        shard.slab_ranges(36, 2)
    with pytest.raises(ValueError):
        shard.slab_ranges(16, 3)


def assemble(results, ranges, key):
    out = np.zeros((NZ, NXT, NY), np.complex128)
    for (x0, n), r in zip(ranges, results):
        out[:, x0:x0 + n, :] = r[key]
    return out


@pytest.mark.parametrize("parts", [1, 3])
def test_slabs_in_one_process_equal_the_oracle(parts):
    """All slabs in one process, the records reduced by the driver's local fixed-order sum."""
    from tests.slab_oracle import NumpySlab
    d, coils, mask = problem()
    ranges = shard.slab_ranges(NXT, parts)
    slabs = [NumpySlab(x0, n, d, coils, mask, params()) for x0, n in ranges]
    res = shard.reconstruct_frame(slabs, shard.Reducer(slabs[0].nsum), ITERS)
    ref = O.priori_ls(d, coils, mask, params())
    assert O.nrmse(assemble(res, ranges, "recon"), ref.recon) < 1e-9
    for r in res:
        assert np.allclose(r["sigma"], ref.sigma, rtol=1e-9, atol=1e-12 * ref.sigma.max())


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, world, port, out_dir):
    import torch.distributed as dist
    from tests.slab_oracle import NumpySlab
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d, coils, mask = problem()
        x0, n = shard.slab_ranges(NXT, world)[rank]
        slab = NumpySlab(x0, n, d, coils, mask, params())
        (res,) = shard.reconstruct_frame([slab], shard.Reducer(slab.nsum, distributed=True), ITERS)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), recon=res["recon"], sigma=res["sigma"])
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sharded_iteration_equals_unsharded_oracle(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(worker, args=(world, free_port(), str(tmp_path)), nprocs=world, start_method="spawn",
                       join=True)
    ranges = shard.slab_ranges(NXT, world)
    res = [dict(np.load(tmp_path / f"rank{r}.npz")) for r in range(world)]
    d, coils, mask = problem()
    ref = O.priori_ls(d, coils, mask, params())
    assert O.nrmse(assemble(res, ranges, "recon"), ref.recon) < 1e-9
    assert np.array_equal(res[0]["sigma"], res[1]["sigma"])   # every rank takes the same step (1)-(2)
    assert np.allclose(res[0]["sigma"], ref.sigma, rtol=1e-9, atol=1e-12 * ref.sigma.max())
