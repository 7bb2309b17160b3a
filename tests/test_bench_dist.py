"""The benchmark's multi-rank host logic on CPU: two gloo ranks (the layout
torchrun gives `bench.py --gpus 2`, one replica per GPU).  Each rank times its
own replica; the job's time is the maximum over ranks and the work the sum, so
the reported throughput is total work / slowest rank.  No data-path collective
exists: the replicas share nothing but these scalars."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    r, w, local, dist = bench.dist_setup(world)
    assert (r, w, local) == (rank, world, rank) and dist is not None
    bench.barrier(dist)
    t = bench.max_over_ranks(dist, 10.0 + rank, "cpu")       # per-rank times 10 ms and 11 ms
    n = bench.sum_over_ranks(dist, 1000.0 * (rank + 1), "cpu")  # per-rank work 1000 and 2000 units
    out.put((rank, t, n))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_sum_work():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 11.0, 3000.0), (1, 11.0, 3000.0)]


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import importlib
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr("oracle.oracle.from_workload", lambda *a, **k: called.append(1), raising=False)

    class Args:
        cells, particles, workload, steps, warmup = 16, 1000, "plasma_ball", 1, 3
    assert bench.reference_arm(Args()) is None
    assert not called


def test_clock_record_rejection_rule():
    """A timing whose clock record shows a hardware or thermal slowdown, or SM
    clocks well below their maximum with no reason, is measured again; a power
    cap alone is kept."""
    sys.path.insert(0, ROOT)
    import bench
    ok = {"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": []}
    assert not bench.clock_rejected(ok)
    assert not bench.clock_rejected(dict(ok, sm_mhz=1500, reasons=["sw_power_cap"]))
    assert bench.clock_rejected(dict(ok, sm_mhz=1500))                       # a leftover clock lock
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clock_rejected(dict(ok, reasons=[r]))
    assert not bench.clock_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]})


def test_oracle_replicas_on_two_cores():
    """The CPU baseline and the reference arm run the single-threaded oracle
    as one replica per core: two spawned replicas of a small sample both step
    it, and the reported rate is all their particle-steps over the slower
    replica's time."""
    sys.path.insert(0, ROOT)
    import bench
    rate, res = bench.oracle_runs("thermal_cube", 4, 1000, 1, 2, None, 2)
    assert len(res) == 2
    assert all(k == 2 and n == res[0][0] and el > 0 for n, k, el in res)
    assert rate == pytest.approx(sum(n * k for n, k, _ in res) / max(el for _, _, el in res))


def test_push_issue_roofline():
    """The push's issue roofline: the captured launch (245M warp instructions
    for 8M particles in 0.434 ms) on 152 SMs at 2070 MHz issues at 0.45 of the
    four schedulers' one instruction per cycle, as ncu's issue-active share
    (45.5%) says; the count scales with the particles pushed."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.issue_roofline(8_000_000, 0.434, 152, 2070.0)
    assert r["warp_instructions_per_particle"] == pytest.approx(30.62, abs=0.01)
    assert r["peak_warp_inst_per_s"] == pytest.approx(152 * 4 * 2.07e9)
    assert r["frac"] == pytest.approx(245e6 / 0.434e-3 / (152 * 4 * 2.07e9), abs=1e-4)
    assert 0.44 < r["frac"] < 0.46
    r2 = bench.issue_roofline(33_554_432, 1.88, 152, 2070.0)
    assert r2["achieved_warp_inst_per_s"] == pytest.approx(245e6 / 8e6 * 33_554_432 / 1.88e-3)
    assert bench.measured_sm_mhz() > 1000.0
