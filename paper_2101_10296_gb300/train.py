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
    reached), ``seconds`` (optimisation wall-clock), ``plan_seconds`` and
    ``evals`` (energy+gradient evaluations).
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
    theta = torch.tensor(theta0, device=device, requires_grad=True)
    opt = torch.optim.Adam([theta], lr=lr)
    if target is not None:
        target = np.broadcast_to(np.asarray(target, dtype=np.float64), (G,))
    best_e = np.full(G, -np.inf)
    best_theta = np.zeros((G, 2 * p))
    history = []
    hit_step = [None] * G
    hit_time = [None] * G
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for step in range(steps):
        e = qaoa.qaoa_energy(theta, plan)  # [G, points]
        loss = -e.sum()
        opt.zero_grad()
        loss.backward()
        e_host = e.detach().cpu().numpy()
        th_host = theta.detach().cpu().numpy()
        opt.step()
        now = time.perf_counter() - t1
        for g in range(G):
            j = int(np.argmax(e_host[g]))
            if e_host[g, j] > best_e[g]:
                best_e[g] = e_host[g, j]
                best_theta[g] = th_host[g, j]
            if target is not None and hit_step[g] is None and best_e[g] >= target[g]:
                hit_step[g] = step
                hit_time[g] = now
        history.append(best_e.copy())
    torch.cuda.synchronize()
    return {
        "theta": best_theta,
        "energy": best_e,
        "history": np.array(history),
        "steps_to_target": hit_step,
        "seconds_to_target": hit_time,
        "seconds": time.perf_counter() - t1,
        "plan_seconds": plan_s,
        "evals": steps * G * points,
    }
