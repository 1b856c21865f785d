"""Launch autotuner for a plan: times candidate tunings once and keeps the best.

Candidates (see qaoa_tuning_t in include/qaoa.h): the number of parameter
points a warp task of the register kernels evaluates (1, 2, 4, 8, 16 when the
phase tables fit), the persistent grid's blocks per SM, and, when the plan
has large-state cones, the scratch per call, i.e. how many state blocks a
wave holds (waves that fit the L2 keep their passes on chip).  Each
candidate is timed with the library's kernel events on real parameters; the
winner is applied to the plan and cached in a JSON file keyed by device name
and plan shape, so later plans of the same shape skip the search.
"""
from __future__ import annotations

import json
import os

_DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuning_cache.json")


def _key(plan, n_points, grad):
    import torch
    info = plan.info()
    dev = torch.cuda.get_device_name()
    return (f"{dev}|p={info['p']}|reps={info['n_reps']}|maxq={info['max_qubits']}|maxin={info['max_inner']}"
            f"|big={info['n_big']}|P={n_points}|grad={int(bool(grad))}")


def _time(plan, params, grad, reps):
    import torch
    fn = plan.energy_grad if grad else plan.energy
    fn(params)
    torch.cuda.synchronize()
    plan.set_timing(True)
    plan.kernel_time()
    for _ in range(reps):
        fn(params)
    ms, launches, _ = plan.kernel_time()
    plan.set_timing(False)
    return ms / max(reps, 1)


def candidates(plan, n_points):
    info = plan.info()
    row_bytes = info["p"] * (info["max_edges"] + 1) * 8
    jpts = [j for j in (1, 2, 4, 8, 16, 32) if j <= max(1, n_points) and j * row_bytes * 4 <= 48 * 1024]
    bpsm = [0, 1, 2]
    bigs = [0] if info["n_big"] == 0 else [0, 32 << 20, 96 << 20, 256 << 20]
    return [(j, b, g) for j in jpts for b in bpsm for g in bigs]


def autotune(plan, params, grad=True, reps=2, cache_path=_DEFAULT_CACHE, use_cache=True):
    """Times every candidate tuning on ``params`` and applies the fastest.

    Returns ``(best_tuning_dict, {candidate: ms})``.
    """
    n_points = int(params.shape[-2])
    key = _key(plan, n_points, grad)
    cache = {}
    if use_cache and cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except Exception:
            cache = {}
    if use_cache and key in cache:
        best = cache[key]
        plan.set_tuning(**best)
        return best, {}
    results = {}
    for j, b, g in candidates(plan, n_points):
        plan.set_tuning(points_per_task=j, blocks_per_sm=b, big_scratch_bytes=g)
        results[(j, b, g)] = _time(plan, params, grad, reps)
    j, b, g = min(results, key=results.get)
    best = {"points_per_task": j, "blocks_per_sm": b, "big_scratch_bytes": g}
    plan.set_tuning(**best)
    if cache_path:
        cache[key] = best
        try:
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
        except OSError:
            pass
    return best, results
