"""QAOA parameter training: maximise the expected cut E(gamma, beta).

The reason to evaluate E fast is training (Sec. 1, Sec. 2.2): an optimiser
asks for E and its gradient over and over, so the one-off cost of finding
the symmetry (the plan) is amortised over many evaluations (Sec. 5).  This
driver plans once -- with an optional search budget, after which the orbit
finder falls back to the verified subgroup it has (Sec. 6) -- and then runs
Adam on -E for many starting points of every graph at once: each step is one
call of the adjoint kernels through the autograd function.  It reports the
best energy per graph, the wall-clock time spent, and the step and time at
which a target energy was first reached.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs
from . import qaoa


def train(graphs, p, *, points=16, steps=200, lr=0.05, seed=0, target=None, plan=None, orbits=True,
          cone_classes=False, search_budget=0, device="cuda"):
    """Maximise E for every graph from ``points`` random starts each.

    graphs: (n, edges) or a list of them; target: None, a number, or one per
    graph.  Returns a dict with ``theta`` [G, 2p] and ``energy`` [G] (the best
    point seen), ``history`` (best energy per graph after every step),
    ``steps_to_target`` / ``seconds_to_target`` per graph (None if not
    reached), ``seconds`` (optimisation wall-clock after one untimed warm-up
    step on a copy of the starting points), ``plan_seconds`` and ``evals``
    (energy+gradient evaluations of the timed steps).
    """
    import torch

    if isinstance(graphs, tuple):
        graphs = [graphs]
    t0 = time.perf_counter()
    if plan is None:
        plan = qaoa.Plan(graphs, p, orbits=orbits, cone_classes=cone_classes, search_budget=search_budget)
    plan.upload()
    plan_s = time.perf_counter() - t0
    G = len(graphs)
    theta0 = np.stack([inputs.draw_params(p, points, seed + g) for g in range(G)])
    rows = torch.arange(G, device=device)

    def step_once(theta, opt, best_e, best_theta):
        e = qaoa.qaoa_energy(theta, plan)  # [G, points]
        loss = -e.sum()
        opt.zero_grad()
        loss.backward()
        with torch.no_grad():
            # best point so far, tracked on the device (before the step moves theta)
            e_max, j_max = e.detach().max(dim=1)
            better = e_max > best_e
            best_e = torch.where(better, e_max, best_e)
            best_theta = torch.where(better[:, None], theta.detach()[rows, j_max], best_theta)
        opt.step()
        return best_e, best_theta

    def start():
        theta = torch.tensor(theta0, device=device, requires_grad=True)
        return (theta, torch.optim.Adam([theta], lr=lr),
                torch.full((G,), -np.inf, dtype=torch.float64, device=device),
                torch.zeros(G, 2 * p, dtype=torch.float64, device=device))

    # one warm-up step on a throwaway copy (first launches of the library's and
    # the optimiser's kernels, the host read) so that the clock measures
    # steady-state steps only
    warm = start()
    warm[2].copy_(step_once(*warm)[0])
    warm[2].cpu()
    del warm
    theta, opt, best_e, best_theta = start()
    if target is not None:
        target = np.broadcast_to(np.asarray(target, dtype=np.float64), (G,))
    history = []
    hit_step = [None] * G
    hit_time = [None] * G
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for step in range(steps):
        best_e, best_theta = step_once(theta, opt, best_e, best_theta)
        history.append(best_e.clone())
        if target is not None and any(h is None for h in hit_step):
            be = best_e.cpu().numpy()  # the one host read of the step
            now = time.perf_counter() - t1
            for g in range(G):
                if hit_step[g] is None and be[g] >= target[g]:
                    hit_step[g] = step
                    hit_time[g] = now
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t1
    return {
        "theta": best_theta.cpu().numpy(),
        "energy": best_e.cpu().numpy(),
        "history": torch.stack(history).cpu().numpy() if history else np.zeros((0, G)),
        "steps_to_target": hit_step,
        "seconds_to_target": hit_time,
        "seconds": seconds,
        "plan_seconds": plan_s,
        "evals": steps * G * points,
    }
