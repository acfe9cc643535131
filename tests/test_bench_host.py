"""Host-side logic of bench.py without a GPU: the max-over-ranks barrier on
two gloo ranks, the clock-record parser, the workload inputs and the
roofline arithmetic."""
import os
import socket

import numpy as np
import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.barrier_max(10.0 + 5 * rank, world)
    q.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


def test_barrier_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res == [(0, 15.0), (1, 15.0)]


def test_clock_parser():
    c = bench.Clocks(0)
    c.lines = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1900, 2070, 1390.1, 0x4, Not Active, Not Active, Not Active, Active",
               "garbage"]
    s = c.summary()
    assert s["sm_max_mhz"] == 2070 and s["sm_mhz"] == pytest.approx(1985)
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 2


def test_workload_inputs_delete_existing_points():
    wl = dict(n=5000, d=3, m=700, kind="uniform")
    X, Y, yid, zid = bench.make_inputs(wl, 0)
    assert X.shape == (5000, 3) and Y.shape == (700, 3)
    assert len(np.unique(zid)) == 700 and zid.max() < 5700  # existing ids, each once
    assert np.array_equal(yid, np.arange(5000, 5700, dtype=np.uint32))


def test_roofline_bytes_and_config():
    assert bench.algo_bytes("scatter", 3) == 32 and bench.algo_bytes("count", 2) == 8
    assert bench.algo_bytes("unknown", 3) is None
    peak, src = bench.measured_peaks()
    assert peak > 1000 and src in ("measured", "fallback")
    class A:
        workload = bench.DEFAULT_WORKLOAD
        gpus = 1
    cfg = bench.config_of(A, bench.WORKLOADS[bench.DEFAULT_WORKLOAD])
    assert cfg["n"] == 100_000_000 and cfg["d"] == 3 and "larger than L2" in cfg["l2"]


def test_cpu_oracle_step_small():
    pts, dt, desc = bench.cpu_oracle_step(dict(n=20000, d=2, m=2000, kind="uniform"), scale=10)
    assert pts == 2000 + 2 * 200 and dt > 0 and "oracle" in desc


def test_dram_traffic_is_dropped_when_a_kernel_source_changed(tmp_path, monkeypatch):
    import hashlib
    import json

    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text("kernel v1")
    j = {"sources": {"k.cu": hashlib.sha1(b"kernel v1").hexdigest()},
         "kernels": {"scatter": {"dram_bytes_per_item": 25.0}}}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(j))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.dram_traffic()["scatter"]["dram_bytes_per_item"] == 25.0
    (tmp_path / "k.cu").write_text("kernel v2")
    assert bench.dram_traffic() == {}


def test_sieve_rooflines():
    import bench

    kernels = {"scatter": {"achieved_gbs": 3400.0, "items_per_launch": 1e8},
               "count": {"achieved_gbs": None, "items_per_launch": 0.0},
               "smem_build": {"achieved_gbs": 340.0, "items_per_launch": 1e8},
               "sample": {"achieved_gbs": 1000.0, "items_per_launch": 5e7}}
    traffic = {"scatter": {"dram_bytes_per_item": 33.0}}
    r = bench.sieve_rooflines(kernels, 6800.0, traffic)
    assert set(r) == {"scatter", "sample"}          # count had no point count; smem_build is not a sieve kernel
    assert r["scatter"]["frac"] == 0.5 and r["scatter"]["traffic"] == 33.0 * 1e8
    assert r["sample"]["traffic"] is None and r["sample"]["unit"] == "GB/s"
