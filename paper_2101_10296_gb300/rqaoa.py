"""Recursive QAOA (RQAOA) on weighted cut objectives (Sec. 4.1).

Each round optimises the QAOA parameters for the current objective
C(z) = sum_e w_e [z_u != z_v] (``train``), reads <Z_u Z_v> for every edge
(one value per orbit -- or per cone class -- from the terms of the plan:
edges related by a symmetry share it, Theorem 1), picks the edge with the
largest |<Z_u Z_v>| and eliminates its larger endpoint v by imposing
z_v = sgn(<Z_u Z_v>) z_u.  In cut terms: with sigma = +1 an edge (v, k)
becomes (u, k) with the same weight; with sigma = -1, [z_v != z_k] =
1 - [z_u != z_k], so (v, k) becomes (u, k) with weight -w plus the constant w,
and the eliminated edge (u, v) itself contributes w to the constant when
sigma = -1.  Weights of parallel edges add; an edge whose weight sums to 0
disappears.  When at most ``n_brute`` vertices still carry edges the rest is
solved by enumeration, and the eliminated spins are filled in backwards.
"""
from __future__ import annotations

import numpy as np

from . import qaoa
from . import train as qtrain


def cut_value(edges, weights, bits):
    """sum_e w_e [bits_u != bits_v] for a 0/1 assignment."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.ones(len(edges)) if weights is None else np.asarray(weights)
    return float(np.sum(w * (bits[edges[:, 0]] != bits[edges[:, 1]])))


def _brute(verts, W):
    """Best 0/1 assignment of ``verts`` for the weighted cut W {(a, b): w}."""
    k = len(verts)
    idx = {v: i for i, v in enumerate(verts)}
    z = np.arange(1 << k, dtype=np.int64)
    c = np.zeros(1 << k)
    for (a, b), w in W.items():
        c += w * (((z >> idx[a]) ^ (z >> idx[b])) & 1)
    best = int(np.argmax(c))
    return {v: (best >> i) & 1 for v, i in idx.items()}, float(c[best])


def rqaoa(n, edges, weights=None, p=1, n_brute=8, steps=150, points=8, lr=0.05, seed=0, orbits=True,
          cone_classes=False):
    """Run RQAOA to an assignment.  Returns a dict with ``bits`` (0/1 per
    vertex), ``cut`` (its value on the input objective), ``rounds`` (per
    elimination: the vertex, its partner, the sign, |<ZZ>|, the trained
    energy and the number of simulated representatives) and ``brute_vertices``."""
    import torch

    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w0 = np.ones(len(edges), dtype=np.int64) if weights is None else np.asarray(weights, dtype=np.int64)
    W = {}
    for (a, b), w in zip(edges, w0):
        key = (int(min(a, b)), int(max(a, b)))
        W[key] = W.get(key, 0) + int(w)
    W = {k: v for k, v in W.items() if v != 0}
    rounds = []
    eliminated = []  # (v, u, sigma): z_v = sigma z_u, in order
    while True:
        verts = sorted({x for e in W for x in e})
        if len(verts) <= n_brute or not W:
            break
        idx = {v: i for i, v in enumerate(verts)}
        keys = sorted(W)
        local = np.array([(idx[a], idx[b]) for a, b in keys], dtype=np.int64)
        lw = np.array([W[k] for k in keys], dtype=np.int64)
        try:
            plan = qaoa.Plan((len(verts), local), p, orbits=orbits, cone_classes=cone_classes, weights=lw)
        except qaoa.QAOAError:
            # merged weights can outgrow a cone's 64-bit cut word: finish by enumeration if small
            if len(verts) <= 20:
                break
            raise
        out = qtrain.train((len(verts), local), p, points=points, steps=steps, lr=lr, seed=seed + len(rounds),
                           plan=plan)
        th = torch.tensor(out["theta"][:, None, :], device="cuda")
        _, terms = plan.energy(th, terms=True)
        terms = terms[:, 0].cpu().numpy()
        reps = plan.reps()
        row = {int(e): r for r, e in enumerate(reps["edge"])}
        cid, _ = plan.cone_classes(0)
        m = np.array([terms[row[int(c)]] for c in cid])  # <Z_u Z_v> of every edge
        e_star = int(np.argmax(np.abs(m)))
        u, v = verts[local[e_star, 0]], verts[local[e_star, 1]]
        sigma = 1 if m[e_star] >= 0 else -1
        rounds.append({"eliminate": v, "onto": u, "sigma": sigma, "abs_zz": float(abs(m[e_star])),
                       "energy": float(out["energy"][0]), "representatives": int(len(reps["edge"]))})
        eliminated.append((v, u, sigma))
        # substitute z_v = sigma z_u
        new = {}
        for (a, b), w in W.items():
            if (a, b) == (min(u, v), max(u, v)):
                continue  # constant: contributes w when sigma = -1
            if v in (a, b):
                k = b if a == v else a
                key = (min(u, k), max(u, k))
                new[key] = new.get(key, 0) + (w if sigma > 0 else -w)
            else:
                new[(a, b)] = new.get((a, b), 0) + w
        W = {k: x for k, x in new.items() if x != 0}
    rest = sorted({x for e in W for x in e})
    assign, _ = _brute(rest, W) if W else ({}, 0.0)
    bits = np.zeros(n, dtype=np.int64)
    for x, b in assign.items():
        bits[x] = b
    for v, u, sigma in reversed(eliminated):  # z_v = sigma z_u
        bits[v] = bits[u] if sigma > 0 else 1 - bits[u]
    return {"bits": bits, "cut": cut_value(edges, w0, bits), "rounds": rounds, "brute_vertices": len(rest)}
