#!/usr/bin/env python3
"""Benchmark: QAOA MaxCut energy + adjoint gradient evaluations per second,
orbit-reduced against plain all-edge, on one GPU.

Workload (one step): the 48-graph mix shaped like the paper's benchmark set
(Sec. 5; 100 to 10,000 vertices: random 3-, 4- and 5-regular graphs,
Erdos-Renyi graphs of mean degree 4, tori, hypercubes Q_8..Q_13 and
circulants), depth p = 1, 256 parameter points per graph drawn with the
project's recipe, orbit reduction on (one cone per edge orbit of Aut(G),
weighted by the orbit size; Sec. 3), energies and gradients of all
48 x 256 = 12,288 (graph, point) evaluations in one batched call: the
autotuned evaluation (launch shape and register tile, searched once per plan
shape and cached) replayed as a captured CUDA graph.  The same
workload with every edge its own cone (orbit reduction off, same kernels) is
timed the same way and reported beside it (``plain_all_edge_evals_per_s``):
the contrast the metric names.  The inputs are synthetic stand-ins for the
paper's benchmark files, which are not available.

Side measurements (none enters ``value``): 4 random 3-regular graphs with
n = 2000 at p = 2 and 64 points (graphs without symmetry, where the orbit
step must cost nothing), the energy-only rate, every shell count vector
evolved as its own block, the cone-class plan, a training run, and the
large-state path on a plan whose cones exceed on-chip memory.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on
the launching stream, with a 512 MB L2 flush written between steps outside the
events; barrier + synchronize on both sides; max over ranks.  With N > 1 every
rank runs its own replica (the path shards into independent problems; there
is no data-path collective), so the whole-job value is N x per-rank evals.

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload: random cone terms at one parameter point, scaled
to whole evaluations by a cost model calibrated on the sample (extrapolated,
as the paper extrapolates its infeasible runs in Sec. 5).
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QAOA energy+grad evals/s on 1 GB300, orbit-reduced batched vs plain all-edge"
UNIT = "evals/s"
WORKLOAD = ("mix48-p1-P256: the 48-graph benchmark-shaped mix (100-10,000 vertices: random 3/4/5-regular, "
            "Erdos-Renyi <k>=4, tori, hypercubes Q8-Q13, circulants), p=1, 256 points per graph, energy+grad, "
            "orbit-reduced")
P_DEPTH, N_POINTS = 1, 256
PARAM_SEED0 = 1000  # graph k draws its points with seed PARAM_SEED0 + k
SIDE_SEEDS = (1, 2, 3, 4)

# DRAM bytes per launch of the dominant kernel (the depth-1 adjoint kernel on
# this workload) from a one-pass ncu capture of `bench.py --case reg-mix48`
# (dram__bytes_read.sum + dram__bytes_write.sum: 12,878,592 + 0), with the
# hash of the sources they were taken on; a change to any of them reports
# null until it is captured again.
TRAFFIC = {"kernels_sha1": "7f85fecc87ccd76559b4bf100cd0afd576bea2e7", "bytes_per_launch": 12878592,
           "source": "ncu one-pass capture (dram__bytes_read.sum + dram__bytes_write.sum) of "
                     "`python bench.py --case reg-mix48` (default tuning: 12 points per task, 6 blocks per SM), "
                     "summarised in profiles/reg_p1_mix48_p1.md"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload():
    """The 48 graphs of the mix and their parameter points [48, 256, 2]."""
    from paper_2101_10296_gb300 import inputs as I
    graphs = [b() for _, b in I.mixed_benchmark_graphs()]
    theta = np.stack([I.draw_params(P_DEPTH, N_POINTS, PARAM_SEED0 + k) for k in range(len(graphs))])
    return graphs, theta


def side_workload():
    """4 random 3-regular graphs n = 2000 (seeds 1-4), p = 2, 64 points each."""
    from paper_2101_10296_gb300 import inputs as I
    graphs = [I.random_regular(2000, 3, s) for s in SIDE_SEEDS]
    theta = np.stack([I.draw_params(2, 64, s) for s in SIDE_SEEDS])
    return graphs, theta


def config_dict(world, info=None):
    """The workload's config keys (the same on both arms)."""
    d = {
        "workload": WORKLOAD,
        "graphs": 48, "p": P_DEPTH, "points_per_graph": N_POINTS, "evals_per_step": 48 * N_POINTS,
        "orbit_reduction": True,
        "l2": "512 MB buffer written between timed steps (outside the events)",
        "parallelism": f"replicas x{world}",
    }
    if info is not None:
        d.update({"n_edges": int(info["n_edges_total"]), "n_reps": int(info["n_reps"]),
                  "max_cone_qubits": int(info["max_qubits"]), "max_inner_qubits": int(info["max_inner"])})
    return d


# ------------------------------------------------------------------ roofline

def algorithmic_flops(reps, p, grad, depth1=False):
    """FP32 FLOPs of the pruned state-vector circuit per point, summed over reps.

    Counted for the cheapest formulation the kernels use (FMA = 2 FLOPs), per
    cone with A = n_blocks * 2^n_inner evolved amplitudes (one inner block per
    shell-class count vector) and k_l qubits mixed in layer l:
      forward = A (6 (p-1) + 4 sum_l k_l + 4): the phase complex multiply (6)
        from layer 2 on (layer 1 is a table read), exp(-i beta X) as
        kappa (I - i tau X) with kappa kept as a scalar (one FMA per real
        output: 4 per amplitude per mixed qubit), |psi|^2 with the signed
        accumulation (4);
      adjoint adds A (2 + 12 sum_{l>=2} k_l + 8 k_1 + 5 p + 12 (p-1)): the
        co-state (2); per mixed qubit the Im<lam|X_q|psi> term (4) and undoing
        the butterfly on both states (8), on the co-state only in layer 1 (4);
        per layer the Im<lam|C|psi> term (5); undoing the phase on both states
        above layer 1 (12).
    For register-resident cones (<= 9 inner qubits) at p <= 3 whose last layer
    mixes qubits 0 and 1 only, that layer's pair terms are taken once (the
    co-state is Z_u Z_v psi there): 2 per amplitude per qubit instead of 4.
    With depth1 (p = 1 plans on the depth-1 kernel, k_1 = 2 for every cone)
    the adjoint is A (4 + 8 + 3.75): the co-state's signs fold into the next
    FMAs (0); the two pair terms of a mixed qubit coincide once the co-state
    is Z_u Z_v psi, so Im<lam|X_q|psi> takes 2 per amplitude per qubit; undoing
    the butterflies on the co-state (4 per qubit); Im<lam|C|psi> (5) on the
    three amplitudes of each 4-amplitude block whose cut value differs from
    the block's first, against which C is shifted.
    """
    A = reps["n_blocks"].astype(np.float64) * np.ldexp(1.0, reps["n_inner"].astype(np.int64))
    k = reps["mix_qubits"][:, :p].astype(np.float64)
    ksum = k.sum(axis=1)
    flops = A * (6 * (p - 1) + 4 * ksum + 4)
    if grad and depth1:
        flops = flops + A * (2 * ksum + 4 * ksum + 3.75)
    elif grad:
        flops = flops + A * (2 + 12 * (ksum - k[:, 0]) + 8 * k[:, 0] + 5 * p + 12 * (p - 1))
        if p <= 3:
            # the general register kernel (inner parts of <= 9 qubits) takes the last
            # layer's pair terms once when it mixes qubits 0 and 1 only: 2 per
            # amplitude per qubit instead of 4
            last2 = (reps["n_inner"] <= 9) & (k[:, p - 1] == 2)
            flops = flops - A * 4 * last2
    return float(flops.sum())


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path))
        except Exception:
            pass
    return {}


def fp32_peak_tflops(sm_count):
    """FP32 peak: the device's SM count x 128 FP32 lanes x 2 FLOP (FMA) x the
    maximum SM clock (measured file, else the part's 2070 MHz)."""
    mhz = float(_peaks().get("sm_max_mhz", 2070.0))
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12, mhz


def hbm_peak_gbs():
    pk = _peaks()
    if "hbm_gbs" in pk:
        return float(pk["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernels_sha1():
    """Hash of the dominant kernel's sources (the depth-1 kernel) and of the
    planner and upload code that decide what it reads (the block records)."""
    h = hashlib.sha1()
    for f in ("p1_kernel.cu", "reg_common.cuh", "device.cuh", "capi.cu", "plan.cpp", "block_orbits.cpp"):
        h.update(open(os.path.join(ROOT, "paper_2101_10296_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def large_state_measurement(device, flush, product=True):
    """The large-state path: energy of the 6x6 torus at p = 3 (one 28-qubit
    cone: an 18-qubit inner block per merged shell block, 2 MiB each; the
    product plan) or the Q_12 full cone at p = 1 (24-qubit blocks, a
    cross-check plan), 32 points.  Algorithmic bytes per (cone, point, block)
    = one write and one read of the complex64 block: the minimum once a block
    exceeds on-chip memory."""
    import torch
    from paper_2101_10296_gb300 import inputs as I
    from paper_2101_10296_gb300 import qaoa
    P = 32
    if product:
        plan = qaoa.Plan(I.torus(6, 6), 3)
        params = torch.tensor(I.draw_params(3, P, 36)[None], device=device)
        what = "6x6 torus, p=3, 32 points, energy (product plan: 28-qubit cone, 18-qubit inner blocks)"
    else:
        plan = qaoa.Plan(I.hypercube(12), 1, full_cone=True)
        params = torch.tensor(I.draw_params(1, P, 12)[None], device=device)
        what = "Q12 full cone, p=1, 32 points, energy (cross-check plan: 24-qubit blocks)"
    plan.upload()
    reps = plan.reps()
    blocks = plan.shell_blocks()
    for _ in range(3):
        plan.energy(params)
    torch.cuda.synchronize()
    plan.set_timing(True)
    plan.kernel_time()
    for k in range(5):
        flush.fill_(k & 0xFF)
        plan.energy(params)
    ms, launches, _ = plan.kernel_time()
    plan.set_timing(False)
    ms /= max(launches, 1)
    alg = float(sum(2 * 8 * (2 ** int(n)) * int(b) for n, b in zip(reps["n_inner"], blocks))) * P
    peak, basis = hbm_peak_gbs()
    status = plan.device_status()
    plan.close()
    return {
        "workload": what,
        "ms_per_call": ms,
        "algorithmic_bytes_per_call": alg,
        "achieved_algorithmic_gbs": alg / (ms / 1e3) / 1e9,
        "peak_gbs": peak,
        "peak_basis": basis,
        "frac_algorithmic": alg / (ms / 1e3) / 1e9 / peak,
        "device_status": status,
    }


# -------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of the SM clock and the throttle reasons, every
    period_ms, with their timestamps.  mark_start()/mark_end() bracket the
    timed region; the summary uses the samples from its start on (the caller
    keeps the same load running after the region until a few have arrived:
    a timed region of a few milliseconds is shorter than the sampling period)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index, period_ms=50):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.t0 = self.t1 = None
        # the raw samples go to $QAOA_BENCH_CLOCKS_DIR (default: the temp directory);
        # the JSON line carries their summary
        out_dir = os.environ.get("QAOA_BENCH_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"qaoa_clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            # start timing only once the sampler is producing samples
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                self.fh.flush()
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def mark_start(self):
        self.t0 = datetime.datetime.now()

    def mark_end(self):
        self.t1 = datetime.datetime.now()

    def _rows(self):
        """(time, sm MHz, max sm MHz, active reasons) of every complete sample."""
        rows = []
        if not self.proc:
            return rows
        try:
            lines = open(self.path).read().splitlines()
        except OSError:
            return rows
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
                sm, smax = float(f[2]), float(f[3])
            except ValueError:
                continue
            rows.append((ts, sm, smax, {nm for nm, v in zip(self.REASONS, f[6:10]) if v.lower() == "active"}))
        return rows

    def count_since_start(self):
        return sum(1 for r in self._rows() if self.t0 is None or r[0] >= self.t0)

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = [r for r in self._rows() if self.t0 is None or r[0] >= self.t0]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        reasons = set().union(*(r[3] for r in rows))
        inside = sum(1 for r in rows if self.t1 is None or r[0] <= self.t1)
        return {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "samples_in_timed_region": inside,
                "period_ms": self.period_ms,
                "window": "from the start of the timed region through an untimed replay of the same step "
                          "after it (the region is shorter than the sampling period)"}


# --------------------------------------------------------------- CPU oracle

_W = {}


def _init_oracle_worker():
    """Pool initializer: each worker rebuilds the seeded graphs once."""
    from oracle import qaoa_oracle as O
    graphs, theta = workload()
    _W["graphs"] = graphs
    _W["theta"] = theta
    _W["adj"] = [O.adjacency(n, e) for n, e in graphs]


def _oracle_term_job(job):
    from oracle import qaoa_oracle as O
    g, ei, j = job
    n, edges = _W["graphs"][g]
    verts, _, ledges = O.lightcone(n, edges, edges[ei], P_DEPTH, _W["adj"][g])
    return O.term_grad_adjoint(len(verts), ledges, _W["theta"][g, j], P_DEPTH)


def _oracle_serial_job(jobs):
    """Runs the given terms one after another in one worker; returns seconds."""
    t0 = time.perf_counter()
    for job in jobs:
        _oracle_term_job(job)
    return time.perf_counter() - t0


def _worker_ready(_):
    return os.getpid()


def make_oracle_pool(cores):
    """One single-threaded oracle process per host core (spawned, so it is safe
    to create after CUDA is initialised).  Returns once every worker has run
    its initializer, so that no worker competes for the host cores while the
    GPU is timed."""
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    pool = mp.get_context("spawn").Pool(cores, initializer=_init_oracle_worker)
    pool.map(_worker_ready, range(4 * cores), chunksize=1)
    return pool


_REPS = {}


def workload_reps():
    """(graph, edge, cone qubits, cone edges) of every representative of the
    orbit-reduced workload, from the host planner (plan time, like the paper's
    t_aut, is outside every rate on both arms)."""
    if "reps" not in _REPS:
        from paper_2101_10296_gb300 import qaoa
        graphs, _ = workload()
        plan = qaoa.Plan(graphs, P_DEPTH, orbits=True)
        r = plan.reps()
        plan.close()
        _REPS["reps"] = (r["graph"].astype(np.int64), r["edge"].astype(np.int64),
                         r["n_qubits"].astype(np.int64), r["n_cone_edges"].astype(np.int64))
    return _REPS["reps"]


def oracle_cost(nq, ne):
    """The oracle's work on one cone, up to a constant: a cut table of ne edges
    and about 3 nq butterfly passes over 2^nq amplitudes."""
    return (np.asarray(ne, dtype=np.float64) + 3.0 * np.asarray(nq, dtype=np.float64)) * np.ldexp(
        1.0, np.asarray(nq, dtype=np.int64))


def oracle_sample(target_s=15.0, pool=None, seed=0, max_qubits=18):
    """Times the FP64 oracle (per-cone energy + adjoint gradient) on a random
    sample of the workload's representatives (cones of at most max_qubits
    qubits) at point 0, sized to about target_s of wall time, and a smaller
    sample on one core.  The time of one whole evaluation point (every
    representative of the 48 graphs) is extrapolated with the cost model
    ``oracle_cost`` calibrated on the sample.  Returns (evals/s, processes,
    seconds, terms, one-core evals/s)."""
    rng = np.random.default_rng(seed)
    cores = os.cpu_count() or 1
    g_of, e_of, nq, ne = workload_reps()
    total_cost = float(oracle_cost(nq, ne).sum())
    small = np.nonzero(nq <= max_qubits)[0]
    own = pool is None
    if own:
        pool = make_oracle_pool(cores)
    try:
        probe = [(int(g_of[r]), int(e_of[r]), 0) for r in rng.choice(small, cores)]
        pool.map(_oracle_term_job, probe, chunksize=1)  # warms the workers
        t0 = time.perf_counter()
        pool.map(_oracle_term_job, probe, chunksize=1)
        t_one = (time.perf_counter() - t0)  # ~ one term per process
        n_terms = int(max(cores, min(50000, 0.8 * target_s / max(t_one, 1e-4) * cores)))
        pick = rng.choice(small, n_terms)
        jobs = [(int(g_of[r]), int(e_of[r]), 0) for r in pick]
        t0 = time.perf_counter()
        pool.map(_oracle_term_job, jobs, chunksize=max(1, n_terms // (8 * cores)))
        dt = time.perf_counter() - t0
        cost = float(oracle_cost(nq[pick], ne[pick]).sum())
        # the same kind of terms on one core, about a tenth of the time budget
        n_one = int(max(1, min(n_terms, 0.1 * target_s / max(t_one, 1e-4))))
        dt_one = pool.apply(_oracle_serial_job, (jobs[:n_one],))
        cost_one = float(oracle_cost(nq[pick[:n_one]], ne[pick[:n_one]]).sum())
    finally:
        if own:
            pool.close()
            pool.join()
    n_graphs = int(g_of.max()) + 1
    t_point = dt / cost * total_cost            # all representatives of every graph, one point, on the pool
    t_point_one = dt_one / cost_one * total_cost  # the same on one core
    return n_graphs / t_point, cores, dt, n_terms, n_graphs / t_point_one


def max_over_ranks(x, dist, device):
    """Max of a float over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, evals_per_rank, ms_per_step):
    """Evals/s of the whole job: every rank processes its own evals in parallel."""
    return world * evals_per_rank / (ms_per_step / 1e3)


# ---------------------------------------------------------------- GPU arm

def timed_steps(fn, steps, warmup, flush, stream):
    """W warm-up calls, then K calls each between CUDA events on ``stream``
    with the L2 flush written before the first event; returns ms per call."""
    import torch
    for k in range(warmup):  # the same as a timed call, flush included
        flush.fill_(k & 0xFF)
        fn()
    torch.cuda.synchronize()
    out = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        out.append(a.elapsed_time(b))
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2101_10296_gb300 import qaoa

    dist = None
    if world > 1:
        import torch.distributed as dist
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    sm_count = torch.cuda.get_device_properties(device).multi_processor_count
    graphs, theta = workload()
    G, P, p = len(graphs), N_POINTS, P_DEPTH
    evals = G * P

    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        workload_reps()  # plan the representatives before the pool spawns
        pool = make_oracle_pool(os.cpu_count() or 1)  # spawned before the first GPU call

    from paper_2101_10296_gb300 import autotune
    t0 = time.perf_counter()
    plan = qaoa.Plan(graphs, p, orbits=True)
    t_plan = time.perf_counter() - t0
    plan.upload()
    info = plan.info()
    reps = plan.reps()
    reps["n_blocks"] = plan.shell_blocks()
    params = torch.tensor(theta, device=device)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream()

    def tuned_graph(pl, prm):
        """Autotuned launch shape and tile (cached per plan shape), then one
        evaluation captured as a CUDA graph; returns (graph, tuning, tune s,
        kernel launches per replay)."""
        t = time.perf_counter()
        tun, _ = autotune.autotune(pl, prm, grad=True, reps=2)
        t = time.perf_counter() - t
        pl.kernel_time()  # resets the launch counter
        g = pl.graph(prm, grad=True)
        return g, tun, t, pl.kernel_time()[2]

    # the step: one replay of a captured graph of the autotuned evaluation
    graph, tuning, t_tune, launches_per_step = tuned_graph(plan, params)

    def step():
        return graph.run()

    for k in range(args.warmup):  # the same as a timed step, flush included
        flush.fill_(k & 0xFF)
        step()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        clk.mark_start()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clk.mark_end()
        # the same load, untimed, until the sampler has caught up with the region (at most 1 s)
        hold0 = time.perf_counter()
        while clk.proc and clk.count_since_start() < 5 and time.perf_counter() - hold0 < 1.0:
            for _ in range(8):
                step()
            torch.cuda.synchronize()
    clocks = clk.summary()
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    all_launches = launches_per_step * args.steps
    ms_per_step = max_over_ranks(sum(step_ms) / len(step_ms), dist, device)
    value = whole_job_value(world, evals, ms_per_step)
    # the dominant kernel's own duration: the same tuned evaluation, uncaptured, with
    # the library's events around its cone kernels on the launching stream
    plan.set_timing(True)
    plan.kernel_time()
    for k in range(max(5, args.steps // 2)):
        flush.fill_(k & 0xFF)
        plan.energy_grad(params)
    kern_ms, kern_launches, _ = plan.kernel_time()
    plan.set_timing(False)

    # plain all-edge: the same workload with every edge its own cone, same kernels, same timing
    t0 = time.perf_counter()
    plain = qaoa.Plan(graphs, p, orbits=False)
    t_plain = time.perf_counter() - t0
    plain.upload()
    pgraph, ptuning, _, _ = tuned_graph(plain, params)
    plain_ms = max_over_ranks(statistics.mean(timed_steps(lambda: pgraph.run(), args.steps,
                                                          args.warmup, flush, stream)), dist, device)
    plain_reps = int(plain.info()["n_reps"])
    pgraph.close()
    plain.close()

    # e2e: public API with host buffers, copies inside the timed region
    host_params = torch.tensor(theta).pin_memory()
    host_e = torch.empty(G, P, dtype=torch.float64).pin_memory()
    host_g = torch.empty(G, P, 2 * p, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.fill_(k & 0xFF)
        s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_ev.record(stream)
        e_dev, g_dev = graph.run(host_params)  # pinned host parameters into the graph's buffer
        host_e.copy_(e_dev, non_blocking=True)
        host_g.copy_(g_dev, non_blocking=True)
        e_ev.record(stream)
        e_ev.synchronize()
        if k >= args.warmup:
            e2e_ms.append(s_ev.elapsed_time(e_ev))
    e2e_step = max_over_ranks(sum(e2e_ms) / len(e2e_ms), dist, device)

    def timed(fn, reps_=5):
        return statistics.mean(timed_steps(fn, reps_, 2, flush, stream))

    energy_ms = timed(lambda: plan.energy(params))
    # every shell count vector evolved as its own block (no merging by the cones' symmetries)
    every = qaoa.Plan(graphs, p, block_plain=True)
    every.upload()
    every_ms = timed(lambda: every.energy_grad(params))
    blocks = {"merged": int(reps["n_blocks"].sum()), "every_count_vector": int(every.shell_blocks().sum()),
              "every_block_evals_per_s": world * evals / (every_ms / 1e3)}
    every.close()
    # local-symmetry reduction: one cone per isomorphism class of cones
    t_cc = time.perf_counter()
    ccplan = qaoa.Plan(graphs, p, cone_classes=True)
    t_cc = time.perf_counter() - t_cc
    ccplan.upload()
    cc_ms = timed(lambda: ccplan.energy_grad(params))
    cc_e, _ = ccplan.energy_grad(params)
    ref_e, _ = plan.energy_grad(params)
    cc_err = float((cc_e - ref_e).abs().max() / ref_e.abs().max())
    cc_reps = int(ccplan.info()["n_reps"])
    ccplan.close()

    # graphs without symmetry: 4 x random 3-regular n = 2000, p = 2, 64 points
    sg, stheta = side_workload()
    sparams = torch.tensor(stheta, device=device)
    splan = qaoa.Plan(sg, 2, orbits=True)
    splan.upload()
    s_graph, s_tuning, _, _ = tuned_graph(splan, sparams)
    s_ms = timed(lambda: s_graph.run())
    splain = qaoa.Plan(sg, 2, orbits=False)
    splain.upload()
    sp_graph, _, _, _ = tuned_graph(splain, sparams)
    sp_ms = timed(lambda: sp_graph.run())
    s_graph.close()
    sp_graph.close()
    s_evals = len(sg) * stheta.shape[1]
    s_reps = splan.reps()
    s_reps["n_blocks"] = splan.shell_blocks()
    s_flops = algorithmic_flops(s_reps, 2, grad=True) * stheta.shape[1]
    side = {"workload": "rr3-n2000x4-p2-P64: 4 random 3-regular graphs n=2000 (seeds 1-4), p=2, 64 points each, "
                        "energy+grad",
            "energy_grad_evals_per_s": world * s_evals / (s_ms / 1e3),
            "plain_all_edge_evals_per_s": world * s_evals / (sp_ms / 1e3),
            "n_reps": int(splan.info()["n_reps"]), "tuning": s_tuning,
            # the general adjoint register kernel's algorithmic FP32 work over the whole step
            # (prep_kernel + that kernel), against the same FP32 peak as the roofline
            "fp32_tflops_alg": s_flops / (s_ms / 1e3) / 1e12}
    # the training driver: Adam on -E from 64 starts per graph, timed after a warm-up step
    from paper_2101_10296_gb300 import train as qtrain
    tr_steps = 50
    target = 0.75 * np.array([len(e) for _, e in sg], dtype=np.float64)
    tr = qtrain.train(sg, 2, points=64, steps=tr_steps, lr=0.03, seed=1, plan=splan, device=device, target=target)
    training = {"workload": side["workload"], "steps": tr_steps, "points_per_graph": 64, "seconds": tr["seconds"],
                "energy_grad_evals_per_s": world * tr["evals"] / tr["seconds"],
                "best_energy_per_edge": float(np.mean(tr["energy"] / np.array([len(e) for _, e in sg]))),
                "target_energy_per_edge": 0.75,
                "steps_to_target": [None if s is None else int(s) for s in tr["steps_to_target"]],
                "seconds_to_target": tr["seconds_to_target"],
                "note": "Adam (torch.optim) on the autograd energy; one warm-up step before the clock starts; "
                        "best point tracked on the device, one host read per step"}
    splan.close()
    splain.close()

    # roofline of the dominant kernel: the adjoint register kernel (every cone of the
    # workload is register-resident at p = 1; the events bracket its launch)
    depth1 = bool(info["depth1_kernel"])
    flops = algorithmic_flops(reps, p, grad=True, depth1=depth1) * P
    kern_avg_ms = kern_ms / max(kern_launches, 1)
    achieved = flops / (kern_avg_ms / 1e3) / 1e12
    peak, mhz = fp32_peak_tflops(sm_count)
    side["fp32_frac_of_peak"] = side["fp32_tflops_alg"] / peak
    traffic = TRAFFIC["bytes_per_launch"] if TRAFFIC["kernels_sha1"] == kernels_sha1() else None
    amp_updates = float((np.ldexp(1.0, reps["n_qubits"].astype(np.int64)) * p).sum()) * P
    evolved = float((reps["n_blocks"] * np.ldexp(1.0, reps["n_inner"].astype(np.int64)) * p).sum()) * P

    large = None
    if not args.no_aux:
        large = {"product": large_state_measurement(device, flush, product=True),
                 "full_cone_q12": large_state_measurement(device, flush, product=False)}
    status = plan.device_status()
    graph.close()
    plan.close()
    if rank != 0:
        return None
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded stand-ins for the paper's benchmark graphs)",
        "config": config_dict(world, info),
        "plain_all_edge_evals_per_s": whole_job_value(world, evals, plain_ms),
        "orbit_speedup_vs_plain": plain_ms / ms_per_step,
        "plain_all_edge": {"n_reps": plain_reps, "ms_per_step": plain_ms, "plan_s": t_plain, "tuning": ptuning},
        "step": {"launch": "replay of a captured CUDA graph of one evaluation", "tuning": tuning,
                 "autotune_s": t_tune, "kernel_launches_per_step": launches_per_step},
        "roofline": {
            "bound": "alu",
            "kernel": "reg_p1_kernel<adjoint>" if depth1 else "reg_cone_kernel<adjoint, p=1>",
            "achieved": achieved,
            "peak": peak,
            "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": traffic,
            "traffic_source": TRAFFIC["source"] if traffic is not None else
            "null: the kernel or planner sources changed since the last ncu capture",
            "algorithmic_flops_per_launch": flops,
            "kernel_ms_per_launch": kern_avg_ms,
            "peak_basis": f"FP32: {sm_count} SMs (device property) x 128 lanes x 2 FLOP x {mhz:.0f} MHz "
                          f"(maximum SM clock, MEASURED_PEAKS.json)",
        },
        "e2e": {"value": whole_job_value(world, evals, e2e_step), "unit": UNIT,
                "h2d_bytes_per_step": int(theta.nbytes), "d2h_bytes_per_step": int(G * P * (1 + 2 * p) * 8)},
        "gpu_launches": int(all_launches),
        "clocks": clocks,
        "energy_only_evals_per_s": world * evals / (energy_ms / 1e3),
        "shell_blocks": blocks,
        "cone_classes": {"n_classes": cc_reps, "plan_s": t_cc,
                         "energy_grad_evals_per_s": world * evals / (cc_ms / 1e3),
                         "max_rel_energy_diff_vs_orbit_path": cc_err},
        "no_symmetry_side": side,
        "training": training,
        "amp_updates_per_s": world * amp_updates / (ms_per_step / 1e3),
        "evolved_amp_updates_per_s": world * evolved / (ms_per_step / 1e3),
        "plan_s": t_plan,
        "t_orbits_s": info["t_orbits_s"],
        "wall_s_timed_region": wall,
        "device_status": status,
        "large_state": large,
    }
    if pool is not None:
        try:
            v, cores, dt, nt, v1 = oracle_sample(target_s=args.cpu_seconds, pool=pool)
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": f"{nt} random representative cone terms (<= 18 qubits) at point 0, "
                                             f"FP64 energy + adjoint gradient, {dt:.1f} s on {cores} processes; "
                                             f"extrapolated to whole evals (all {len(workload_reps()[0])} "
                                             f"representatives) by a cost model calibrated on the sample",
                                   "extrapolated": True,
                                   "one_core_value": v1}
        finally:
            pool.close()
            pool.join()
    return out


def run_reference(args, rank, world):
    """The FP64 CPU oracle on the host cores, as the reference arm."""
    if rank != 0:
        return None
    cores = os.cpu_count() or 1
    workload_reps()
    pool = make_oracle_pool(cores)
    try:
        budget = max(5.0, min(30.0, 150.0 / max(args.steps + args.warmup, 1)))
        vals = []
        samples = []
        ones = []
        for k in range(args.warmup + args.steps):
            v, c, dt, nt, v1 = oracle_sample(target_s=budget, pool=pool, seed=k)
            if k >= args.warmup:
                vals.append(v)
                samples.append(nt)
                ones.append(v1)
    finally:
        pool.close()
        pool.join()
    value = statistics.mean(vals)
    sample = (f"per step {statistics.mean(samples):.0f} random representative cone terms (<= 18 qubits) at point 0 "
              f"(FP64 energy + adjoint gradient) on {cores} processes, extrapolated to whole evals by a cost "
              f"model calibrated on the sample")
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * 48 * N_POINTS / value if value else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded stand-ins for the paper's benchmark graphs)", "impl": "reference",
        "extrapolated": True,
        "config": config_dict(world, {"n_edges_total": sum(len(e) for _, e in workload()[0]),
                                      "n_reps": len(workload_reps()[0]),
                                      "max_qubits": int(workload_reps()[2].max()), "max_inner": 2}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "extrapolated": True, "one_core_value": statistics.mean(ones)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------------------------ suite

def suite_configs():
    """The five benchmark configurations (3 split by depth, 4 by graph: Q_12 and C_5000(1,7,23)
    have cones of 134 and 38 qubits at p = 2, the 8x8 torus 32 at p = 3), plus a signed
    objective on configuration 2's graphs."""
    from paper_2101_10296_gb300 import inputs as I
    return [
        ("1. C_20(1,4) p=1, 1 point", [I.circulant(20, [1, 4])], 1, 1),
        ("2. rr3 n=2000 x4, p=2, 64 points", [I.random_regular(2000, 3, s) for s in SIDE_SEEDS], 2, 64),
        ("3a. torus 100x100 + C_5000(1,7), p=2, 32 points", [I.torus(100, 100), I.circulant(5000, [1, 7])], 2, 32),
        ("3b. Q_12 + C_5000(1,7,23), p=1, 32 points", [I.hypercube(12), I.circulant(5000, [1, 7, 23])], 1, 32),
        ("4a. rr3 n=24 x4, p=3, 128 points", [I.random_regular(24, 3, s) for s in SIDE_SEEDS], 3, 128),
        ("4b. torus 8x8, p=2, 128 points", [I.torus(8, 8)], 2, 128),
        ("4c. torus 6x6, p=3, 128 points", [I.torus(6, 6)], 3, 128),
        ("5. 48-graph mix, p=1, 256 points", [b() for _, b in I.mixed_benchmark_graphs()], 1, 256),
        # beyond the five: a signed (edge-coloured) objective of Sec. 4 on configuration 2's graphs
        ("6. rr3 n=2000 x4 with random +-1 weights, p=2, 64 points",
         [I.random_regular(2000, 3, s) for s in SIDE_SEEDS], 2, 64,
         [np.random.default_rng(10 + s).choice([1, -1], 3000) for s in SIDE_SEEDS]),
    ]


def _suite_term_job(job):
    from oracle import qaoa_oracle as O
    n, edges, e, theta, p, w = job
    import time as _t
    t0 = _t.perf_counter()
    val = O.lightcone_term(n, edges, e, theta, p, weights=w)
    return val, _t.perf_counter() - t0


def run_suite(args):
    """Measures every configuration; prints one JSON object per configuration."""
    import multiprocessing as mp
    import torch
    from oracle import qaoa_oracle as O
    from paper_2101_10296_gb300 import inputs as I
    from paper_2101_10296_gb300 import qaoa
    cores = os.cpu_count() or 1
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    pool = mp.get_context("spawn").Pool(cores)
    device = torch.device("cuda", 0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=device)

    def timed(fn, reps=3, warmup=3):
        return statistics.mean(timed_steps(fn, reps, warmup, flush, torch.cuda.current_stream()))

    rows = []
    for cfg in suite_configs():
        name, graphs, p, P = cfg[:4]
        wts = cfg[4] if len(cfg) > 4 else None
        theta = np.stack([I.draw_params(p, P, 1000 + k) for k in range(len(graphs))])
        params = torch.tensor(theta, device=device)
        evals = len(graphs) * P
        t0 = time.perf_counter()
        plan = qaoa.Plan(graphs, p, weights=wts)
        t_plan = time.perf_counter() - t0
        plan.upload()
        info = plan.info()
        plain = qaoa.Plan(graphs, p, orbits=False, weights=wts)
        plain.upload()
        ms_g = timed(lambda: plan.energy_grad(params))
        ms_e = timed(lambda: plan.energy(params))
        ms_pg = timed(lambda: plain.energy_grad(params))
        every = qaoa.Plan(graphs, p, weights=wts, block_plain=True)  # every shell count vector its own block
        every.upload()
        ms_bp = timed(lambda: every.energy_grad(params))
        blocks_every = int(every.shell_blocks().sum())
        every.close()
        ccplan = qaoa.Plan(graphs, p, cone_classes=True, weights=wts)
        ccplan.upload()
        ms_cc = timed(lambda: ccplan.energy_grad(params))
        e_cc = ccplan.energy(params).cpu().numpy()
        e_gpu, terms = plan.energy(params, terms=True)
        e_gpu = e_gpu.cpu().numpy()
        terms = terms.cpu().numpy()
        reps = plan.reps()
        reps["n_blocks"] = plan.shell_blocks()
        flops = algorithmic_flops(reps, p, grad=True, depth1=bool(plan.info()["depth1_kernel"])) * P
        amps = float((np.ldexp(1.0, reps["n_qubits"].astype(np.int64)) * p).sum()) * P
        # accuracy: per-term against the FP64 oracle on sampled representatives
        # (cones of at most 20 qubits), total energy against the closed form at p = 1
        rng = np.random.default_rng(0)
        small = np.nonzero(reps["n_qubits"] <= 20)[0]
        pick = rng.choice(small, min(24, small.size), replace=False) if small.size else []
        jobs = []
        for r in pick:
            gi = int(reps["graph"][r])
            n, edges = graphs[gi]
            jobs.append((n, edges, edges[reps["edge"][r]], theta[gi, 0], p, None if wts is None else wts[gi]))
        res = pool.map(_suite_term_job, jobs) if jobs else []
        dterm = max([abs(0.5 * (1 - terms[r, 0]) - 0.5 * (1 - v)) for r, (v, _) in zip(pick, res)] or [float("nan")])
        t_term = float(np.mean([dt for _, dt in res])) if res else float("nan")
        drel = float("nan")
        if p == 1 and wts is None:
            worst = 0.0
            for gi in range(min(len(graphs), 8)):
                n, edges = graphs[gi]
                adj = O.adjacency(n, edges)
                ref = sum(O.closed_form_p1_term(n, edges, e, theta[gi, 0, 0], theta[gi, 0, 1], adj) for e in edges)
                worst = max(worst, abs(e_gpu[gi, 0] - ref) / abs(ref))
            drel = worst
        # oracle CPU rate: mean single-process time per cone term x terms per eval / processes
        n_terms = int(info["n_reps"])
        n_terms_plain = int(info["n_edges_total"])
        cpu_eval_s = t_term * n_terms / len(graphs) / cores
        row = {
            "config": name, "graphs": len(graphs), "p": p, "points": P, "n_reps": n_terms,
            "n_edges": n_terms_plain, "max_cone_qubits": int(info["max_qubits"]), "max_inner": int(info["max_inner"]),
            "large_state_cones": int(info["n_big"]), "plan_s": t_plan, "t_orbits_s": info["t_orbits_s"],
            "energy_grad_evals_per_s": evals / (ms_g / 1e3), "energy_evals_per_s": evals / (ms_e / 1e3),
            "plain_energy_grad_evals_per_s": evals / (ms_pg / 1e3),
            "shell_blocks": int(reps["n_blocks"].sum()), "shell_blocks_every_count_vector": blocks_every,
            "every_block_energy_grad_evals_per_s": evals / (ms_bp / 1e3),
            "cone_class_reps": int(ccplan.info()["n_reps"]),
            "cone_class_energy_grad_evals_per_s": evals / (ms_cc / 1e3),
            "cone_class_max_rel_energy_diff": float(np.max(np.abs(e_cc - e_gpu) / np.abs(e_gpu))),
            "amp_updates_per_s": amps / (ms_g / 1e3), "fp32_tflops_alg": flops / (ms_g / 1e3) / 1e12,
            "max_term_err_vs_fp64": dterm, "max_rel_energy_err_vs_closed_form": drel,
            "cpu_oracle_evals_per_s": (1.0 / cpu_eval_s) if cpu_eval_s == cpu_eval_s and cpu_eval_s > 0 else None,
            "cpu_oracle_basis": f"{len(res)} sampled cone terms (<= 20 qubits) x {n_terms} terms per eval, {cores} processes",
            "device_status": plan.device_status(),
        }
        rows.append(row)
        print(json.dumps(row), flush=True)
    pool.close()
    pool.join()
    # RQAOA (Sec. 4.1) end to end on a random cubic graph: training, terms and
    # re-planning every round, enumeration of the last eight vertices
    from paper_2101_10296_gb300 import rqaoa
    n, edges = I.random_regular(60, 3, 1)
    # untimed warm-up: the first use of the optimiser's and reductions' kernels
    # on a fresh device loads them (seconds)
    rqaoa.rqaoa(*I.random_regular(20, 3, 2), p=1, n_brute=8, steps=3, points=8, seed=1)
    t0 = time.perf_counter()
    out = rqaoa.rqaoa(n, edges, p=1, n_brute=8, steps=100, points=8, seed=1)
    secs = time.perf_counter() - t0
    row = {"config": "7. RQAOA, rr3 n=60, p=1 (100 Adam steps x 8 starts per round)", "rounds": len(out["rounds"]),
           "seconds": secs, "cut": out["cut"], "edges": len(edges), "cut_fraction": out["cut"] / len(edges),
           "mean_representatives_per_round": float(np.mean([r["representatives"] for r in out["rounds"]]))}
    print(json.dumps(row), flush=True)


# Small fixed workloads for profiler captures (ncu replays each launch many
# times, so these hold at most a few GB on the device).  Each runs the call
# twice: a warm-up and the one to capture.
PROFILE_CASES = {
    "reg-mix48": "the benchmark workload (48-graph mix, p=1, 256 points): energy+grad",
    "reg-mix48-small": "the 48-graph mix, p=1, 16 points: energy+grad",
    "reg-mix48-p32": "the 48-graph mix, p=1, 32 points: energy+grad",
    "reg-adjoint-rr3-n2000": "1 random 3-regular graph n=2000 (seed 1), p=2, 8 points: energy+grad "
                             "(5 register qubits per thread)",
    "reg-adjoint-rr3-n2000-p64": "1 random 3-regular graph n=2000 (seed 1), p=2, 64 points: energy+grad "
                                 "(5 register qubits per thread)",
    "reg-rr3-x4": "4 x rr3 n=2000, p=2, 64 points: energy+grad",
    "split-adjoint-rr3-n24": "1 random 3-regular graph n=24 (seed 1), p=3, 8 points: energy+grad",
    "split-adjoint-torus6": "6x6 torus, p=3, 2 points: energy+grad",
    "split-energy-torus6": "6x6 torus, p=3, 4 points: energy",
    "split-energy-q12-fullcone": "Q_12 full cone, p=1, 2 points: energy",
}


def run_case(name):
    import torch
    from paper_2101_10296_gb300 import inputs as I
    from paper_2101_10296_gb300 import qaoa
    tuning = {}
    if name in ("reg-mix48", "reg-mix48-small", "reg-mix48-p32"):
        graphs, theta = workload()
        if name != "reg-mix48":
            theta = np.ascontiguousarray(theta[:, :16 if name == "reg-mix48-small" else 32])
        p, grad, kw = 1, True, {}
    elif name == "reg-rr3-x4":
        graphs, theta = side_workload()
        p, grad, kw = 2, True, {}
    else:
        if name.startswith("reg-adjoint-rr3-n2000"):
            # the width the untuned plan of the 4-graph side workload takes
            tuning = {"reg_bits_grad": 5}
        spec = {"reg-adjoint-rr3-n2000": ([I.random_regular(2000, 3, 1)], 2, 8, True, {}),
                "reg-adjoint-rr3-n2000-p64": ([I.random_regular(2000, 3, 1)], 2, 64, True, {}),
                "split-adjoint-rr3-n24": ([I.random_regular(24, 3, 1)], 3, 8, True, {}),
                "split-adjoint-torus6": ([I.torus(6, 6)], 3, 2, True, {}),
                "split-energy-torus6": ([I.torus(6, 6)], 3, 4, False, {}),
                "split-energy-q12-fullcone": ([I.hypercube(12)], 1, 2, False, {"full_cone": True})}[name]
        graphs, p, P, grad, kw = spec
        theta = np.stack([I.draw_params(p, P, s + 1) for s in range(len(graphs))])
    plan = qaoa.Plan(graphs, p, **kw)
    plan.upload()
    if tuning:
        plan.set_tuning(**tuning)
    th = torch.tensor(theta, device="cuda")
    for _ in range(2):
        out = plan.energy_grad(th) if grad else plan.energy(th)
    torch.cuda.synchronize()
    e = out[0] if grad else out
    print(json.dumps({"case": name, "what": PROFILE_CASES[name], "energy_0": float(e[0, 0]),
                      "device_status": plan.device_status()}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-aux", action="store_true", help="skip the auxiliary large-state measurements")
    ap.add_argument("--suite", action="store_true", help="measure every benchmark configuration instead")
    ap.add_argument("--case", choices=sorted(PROFILE_CASES), help="run one small profiling workload and exit")
    args = ap.parse_args()
    if args.case:
        run_case(args.case)
        return
    if args.warmup < 3:
        log("warning: fewer than 3 warm-up steps")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.suite:
        run_suite(args)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        out = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
