"""The multi-GPU path of the benchmark on CPU: two gloo ranks (one process each, as torchrun
would start them) shard the slots with no data-path collective and time the job by its
slowest rank.  Slots are independent problems, so ranks run as replicas on disjoint slot
ids; the only collectives are the timing barrier and the max over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from oracle import sim as osim
        from workloads import WORKLOADS
        w = WORKLOADS["plain_14x72_b16_fp32"]
        B = 3
        slot0 = bench.rank_slot0(rank)
        s = osim.simulate(w.net, w.sim, 1, slot0, B)
        # each rank's slots: gather ids and a fingerprint of the transmitted bits
        ids = torch.arange(slot0, slot0 + B, dtype=torch.int64)
        all_ids = [torch.zeros_like(ids) for _ in range(world)]
        dist.all_gather(all_ids, ids)
        fp = torch.tensor([float(np.sum(s["bits"][0] * np.arange(s["bits"][0].size).reshape(s["bits"][0].shape)))],
                          dtype=torch.float64)
        all_fp = [torch.zeros_like(fp) for _ in range(world)]
        dist.all_gather(all_fp, fp)
        # per-rank step times: the job's is the largest
        my_ms = 10.0 + 5.0 * rank
        job_ms = bench.max_over_ranks(my_ms, dist)
        out[rank] = dict(ids=[t.tolist() for t in all_ids], fp=[float(t.item()) for t in all_fp], job_ms=job_ms,
                         rate=bench.job_rate(B, world, job_ms))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_slots_and_time_by_the_slowest():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    ids = res[0]["ids"]
    assert ids == res[1]["ids"]
    assert not set(ids[0]) & set(ids[1]), "ranks must process disjoint slots"
    assert res[0]["fp"][0] != res[0]["fp"][1], "different slots carry different bits"
    for r in (0, 1):
        assert res[r]["job_ms"] == 15.0          # the slower rank's time
        assert res[r]["rate"] == pytest.approx(3 * 2 / 0.015)


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.rank_slot0(0) == 0 and bench.rank_slot0(3) == 3 * bench.RANK_SLOT_STRIDE
    assert bench.job_rate(256, 1, 100.0) == pytest.approx(2560.0)
