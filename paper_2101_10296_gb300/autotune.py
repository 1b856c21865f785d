"""Launch autotuner for a plan: times candidate tunings once and keeps the best.

Candidates (see qaoa_tuning_t in include/qaoa.h), searched one group at a
time (coordinate descent, each group timed with the best values found for
the groups before it):

1. the number of parameter points a warp task of the register kernels
   evaluates (1, 2, 4, 8, 12, 16, 32 while the phase tables fit) and the persistent grid's
   blocks per SM;
2. with gradients and register-resident cones on the general register
   kernel (not depth-1 plans): the adjoint register kernel's tile,
   2^(bits + 5) amplitudes per warp with 4 or 5 register qubits per thread;
3. with large-state cones: the scratch per call, i.e. how many state blocks a
   wave holds (waves that fit the L2 keep their passes on chip), and the
   widest window of outer qubits a shared-memory chunk pass mixes (the chunk
   tile: a window of w outer qubits over contiguous runs of 2^(13 - w)
   amplitudes).

Each candidate is timed with the library's kernel events on real parameters;
the winner is applied to the plan and cached in a JSON file keyed by device
name and plan shape, so later plans of the same shape skip the search.
Results do not depend on the tuning (every candidate computes the same sums).
"""
from __future__ import annotations

import json
import os

_DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuning_cache.json")
_FIELDS = ("points_per_task", "blocks_per_sm", "big_scratch_bytes", "reg_bits_grad", "chunk_window")


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


def candidate_groups(plan, n_points, grad):
    """The groups of tuning values the search walks through, in order: a list
    of lists of partial tunings (dicts over qaoa_tuning_t's fields)."""
    info = plan.info()
    row_bytes = info["p"] * (info["max_edges"] + 1) * 8
    jpts = [j for j in (1, 2, 4, 8, 12, 16, 32) if j <= max(1, n_points) and j * row_bytes * 4 <= 48 * 1024]
    groups = [[{"points_per_task": j, "blocks_per_sm": b} for j in jpts for b in (0, 1, 2)]]
    # the adjoint register tile matters only to the general register kernel
    # (depth-1 plans run their register cones on the depth-1 kernel)
    has_reg = info["n_reps"] > info["n_big"] and not info["depth1_kernel"]
    if grad and has_reg:
        groups.append([{"reg_bits_grad": r} for r in (4, 5)])
    if info["n_big"] > 0:
        groups.append([{"big_scratch_bytes": g, "chunk_window": w}
                       for g in (0, 96 << 20, 256 << 20) for w in (8, 10)])
    return groups


def candidates(plan, n_points, grad=True):
    """Every partial tuning the search may time (flattened groups)."""
    return [c for grp in candidate_groups(plan, n_points, grad) for c in grp]


def autotune(plan, params, grad=True, reps=2, cache_path=_DEFAULT_CACHE, use_cache=True):
    """Times the candidate tunings on ``params`` and applies the fastest.

    Returns ``(best_tuning_dict, {candidate: ms})`` with candidates as tuples
    of (field, value) pairs.
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
        best = {k: cache[key].get(k, 0) for k in _FIELDS}
        plan.set_tuning(**best)
        return best, {}
    best = {k: 0 for k in _FIELDS}
    results = {}
    for group in candidate_groups(plan, n_points, grad):
        timed = []
        for cand in group:
            trial = dict(best, **cand)
            plan.set_tuning(**trial)
            ms = _time(plan, params, grad, reps)
            results[tuple(sorted(trial.items()))] = ms
            timed.append((ms, cand))
        best.update(min(timed, key=lambda t: t[0])[1])
    plan.set_tuning(**best)
    if cache_path:
        cache[key] = best
        try:
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
        except OSError:
            pass
    return best, results
