"""Host-side logic of bench.py, without a GPU: the max-over-ranks timing of
the replicas-only multi-GPU mode (two gloo ranks on the CPU), the clock sample
parsing, and the staleness rule of the committed DRAM-traffic figure."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(0.5 + rank, dist, "cpu")
        out[rank] = t
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert dict(out) == {0: 1.5, 1: 1.5}


def test_max_over_ranks_without_process_group_is_identity():
    assert bench.max_over_ranks(0.25, None, "cpu") == 0.25


def test_clock_summary_flags_throttle_reasons():
    s = bench.ClockSampler(0)
    s.rows = [["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "1950", "2070", "1300", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["0", "300", "2070", "100", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    summ = s.summary()
    assert summ["sm_max_mhz"] == 2070
    assert summ["sm_mhz"] == pytest.approx(2010)  # median of the samples under load
    assert summ["reasons"] == ["sw_power_cap"]


def test_traffic_figure_is_dropped_when_the_kernel_source_changed(tmp_path, monkeypatch):
    val, sha = bench.read_traffic("k_ab1<f32>")
    # the committed figure either matches the current source (a number) or is stale (None, current sha)
    assert (val is None and sha) or (val is not None and 100 < val < 200)
    assert bench.read_traffic("no_such_kernel") == (None, None)


def test_parse_defaults():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.impl == "native" and a.n == 256 and a.precision == "f32"
