"""bench.py host logic on CPU: the max-over-ranks timing reduction and the
whole-job value on two gloo ranks, the FLOP model, the clock-log parser."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    out.put((rank, ms, bench.whole_job_value(world, 256, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_scale_value():
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
    for rank, ms, v in res:
        assert ms == 11.0
        assert abs(v - 2 * 256 / 0.011) < 1e-6


def test_flop_model_counts():
    import bench
    reps = {"n_inner": np.array([6, 2]), "n_blocks": np.array([81, 3]), "mix_qubits": np.array([[6, 2], [2, 2]])}
    fwd = bench.algorithmic_flops(reps, 2, grad=False)
    a0, a1 = 81 * 2 ** 6, 3 * 2 ** 2
    assert fwd == a0 * (6 + 4 * 8 + 4) + a1 * (6 + 4 * 4 + 4)
    both = bench.algorithmic_flops(reps, 2, grad=True)
    # both cones are register-resident with a last layer of qubits 0 and 1: pair terms once (-4)
    assert both == fwd + a0 * (2 + 12 * 2 + 8 * 6 + 10 + 12 - 4) + a1 * (2 + 12 * 2 + 8 * 2 + 10 + 12 - 4)
    # depth 1: blocks of 4 amplitudes mixed on qubits u, v
    r1 = {"n_inner": np.array([2, 2]), "n_blocks": np.array([9, 169]), "mix_qubits": np.array([[2], [2]])}
    a = 4 * (9 + 169)
    assert bench.algorithmic_flops(r1, 1, grad=False) == a * 12
    assert bench.algorithmic_flops(r1, 1, grad=True) == a * (12 + 2 + 16 + 5 - 4)
    assert bench.algorithmic_flops(r1, 1, grad=True, depth1=True) == a * (12 + 4 + 8 + 3.75)


def test_clock_log_parser(tmp_path):
    """Samples are read with their timestamps; those before the timed region's
    start are left out, and those up to its end are counted as inside it."""
    import datetime
    import bench
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "c.csv")
    c.proc = object()
    with open(c.path, "w") as f:
        f.write("2026/12/03 10:00:00.000, 0, 1200, 2070, 300.0, 0x0, Not Active, Active, Not Active, Not Active\n")
        f.write("2026/12/03 10:00:00.100, 0, 1900, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("2026/12/03 10:00:00.120, 0, 1950, 2070, 950.2, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("2026/12/03 10:00:00.140, 0, 2000, 2070, 990.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("2026/12/03 10:00:00.160, 0, 20")  # a sample still being written
    s = c.summary()  # no region marked: every complete sample
    assert s["samples"] == 4 and s["sm_mhz"] == 1925 and s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    c.t0 = datetime.datetime(2026, 12, 3, 10, 0, 0, 50000)
    c.t1 = datetime.datetime(2026, 12, 3, 10, 0, 0, 125000)
    s = c.summary()
    assert s["sm_mhz"] == 1950 and s["sm_max_mhz"] == 2070 and s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3 and s["samples_in_timed_region"] == 2 and c.count_since_start() == 3


def test_oracle_sample_reports_parallel_and_one_core_rates():
    """The CPU baseline leg: a pool of oracle processes and a one-core run of
    the same kind of terms, both scaled to whole evaluations."""
    import bench
    v, cores, dt, nt, v1 = bench.oracle_sample(target_s=1.0)
    assert v > 0 and v1 > 0 and cores >= 1 and dt > 0 and nt >= cores
    assert v1 <= v * 1.5  # one process is not faster than the pool
