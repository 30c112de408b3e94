"""The multi-rank path on CPU: instance sharding, the end-of-run gather and the
timing reduction, run as world-size-2 gloo process groups.

Each rank advances its shard with the CPU oracle standing in for its GPU (the
sharding layer is the same whatever steps the instances); the gathered results
must equal one process advancing every instance.
"""
import multiprocessing as mp
import os
import socket
import time

import numpy as np
import pytest

from paper_1902_08933_gb300 import sharding as sh
from paper_1902_08933_gb300 import workloads as wl


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tiny_batch():
    cfgs = [wl.static_droplet(n=12, R=3.0), wl.static_droplet(n=16, R=4.0, rho_ratio=2.0),
            wl.rising_bubble(nx=16, ny=20, R=4.0, cy=7.0, Re=5.0),
            wl.static_droplet(n=8, R=2.5, qim=0), wl.spinodal(n=10),
            wl.rising_bubble(nx=12, ny=16, R=3.0, cy=6.0, Re=5.0, qim=0)]
    return cfgs


def _advance(cfg, nsteps):
    from oracle import oracle as orc
    P = orc.params(cfg)
    st = orc.init(P, wl.initial_phi(cfg))
    orc.step(P, st, nsteps)
    f = orc.fields(P, st)
    return {k: np.asarray(v).copy() for k, v in f.items()}


def _rank_main(rank, world, port, outdir, mode):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), OMP_NUM_THREADS="1")
    import datetime
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    try:
        cfgs = _tiny_batch()
        cells = [c["nx"] * c["ny"] for c in cfgs]
        mine = sh.shard(cells, rank, world)
        if mode == "fail" and rank == 1:
            raise RuntimeError("rank 1 fails before the gather")
        t0 = time.perf_counter()
        local = {i: _advance(cfgs[i], 15) for i in mine}
        secs = time.perf_counter() - t0
        t_job = sh.max_over_ranks(secs + rank)          # rank-dependent on purpose
        allres = sh.gather_by_instance(local, len(cfgs))
        if rank == 0:
            np.save(os.path.join(outdir, "gathered.npy"),
                    np.array([allres[i]["phi"] for i in range(len(cfgs))], dtype=object),
                    allow_pickle=True)
            with open(os.path.join(outdir, "meta.txt"), "w") as f:
                f.write("%r %r %r\n" % (t_job, secs, mine))
    except RuntimeError as e:
        with open(os.path.join(outdir, "rank%d_error.txt" % rank), "w") as f:
            f.write(str(e))
        if not (mode == "fail" and rank == 0):
            raise
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _launch(world, outdir, mode="ok", timeout=120):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(outdir), mode)) for r in range(world)]
    for p in procs:
        p.start()
    deadline = time.time() + timeout
    for p in procs:
        p.join(max(1.0, deadline - time.time()))
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
        p.join()
    assert not alive, "a rank did not finish in time"
    return [p.exitcode for p in procs]


def test_partition_covers_every_instance_once():
    cells = [c["nx"] * c["ny"] for c in wl.batched_mixed(512)]
    for world in (1, 2, 3, 4, 8):
        parts = sh.partition(cells, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(cells)))
        assert parts == sh.partition(cells, world)          # deterministic
        loads = [sum(cells[i] for i in p) for p in parts]
        # greedy largest-first: no two ranks differ by more than the largest instance
        assert max(loads) - min(loads) <= max(cells)
        assert sh.imbalance(cells, world) < 1.01


def test_partition_edge_cases():
    assert sh.partition([], 3) == [[], [], []]
    assert sh.partition([5], 2) == [[0], []]
    assert sh.partition([4, 4, 4, 4], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        sh.partition([1, 2], 0)
    with pytest.raises(ValueError):
        sh.partition([1, -2], 2)
    with pytest.raises(ValueError):
        sh.shard([1, 2], 2, 2)


def test_two_ranks_gather_equals_one_process(tmp_path):
    codes = _launch(2, tmp_path)
    assert codes == [0, 0]
    gathered = np.load(tmp_path / "gathered.npy", allow_pickle=True)
    for i, cfg in enumerate(_tiny_batch()):
        np.testing.assert_array_equal(gathered[i], _advance(cfg, 15)["phi"])
    t_job, secs, mine = open(tmp_path / "meta.txt").read().split(" ", 2)
    # rank 1 added one second: the job time is the slowest rank's
    assert float(t_job) >= 1.0


def test_rank_failure_is_seen_by_the_other_rank(tmp_path):
    t0 = time.time()
    codes = _launch(2, tmp_path, mode="fail", timeout=90)
    assert codes[1] != 0 and codes[0] == 0
    assert (tmp_path / "rank1_error.txt").exists()
    assert (tmp_path / "rank0_error.txt").exists()     # the gather failed instead of hanging
    assert time.time() - t0 < 90
