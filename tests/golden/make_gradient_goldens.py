#!/usr/bin/env python3
"""Writes the FP64 oracle's energies and gradients that the GPU gradient tests
compare against.  It calls only ``oracle/`` and the seeded input generators
(``paper_2101_10296_gb300/inputs.py``, which hold no QAOA arithmetic); nothing
here runs the CUDA path.

Two files:

``near_stationary.json`` -- points close to a local maximum of E, where the
gradient is small and its FP32 evaluation is hardest (the terms of each
derivative cancel to 1e-3 .. 1e-4 of their size).  For every case: the
maximiser theta* (Q_d at p = 1 from the published p = 1 formula, which for a
hypercube edge -- no triangles, both endpoints of degree d -- reduces to
1/2 + 1/2 sin(4 beta) sin(gamma) cos^(d-1)(gamma), maximal at beta = pi/8,
tan^2(gamma) = 1/(d-1); the other cases by L-BFGS on the oracle's energy and
adjoint gradient from a linear-ramp start), then, for each rho in RHOS, six
points theta* + delta u (u a seeded random unit vector) with delta set so
that |grad E| = rho * |E edges|, and the oracle's
orbit-weighted energy and adjoint gradient there (Sec. 3: one cone per orbit,
weighted by the orbit size; Sec. 2.3: each term on its reverse causal cone).
Orbits are those of symmetries read off each family's definition: every edge
of Q_d and of K_{a,b} is equivalent, and an edge i -- i + j of a circulant
is equivalent to every other edge of jump j (rotations).

``full_size_gradient.json`` -- the gradient configuration at full size: four
random 3-regular graphs with n = 24 (seeds 1-4, no symmetry, so every edge is
its own cone: up to 24 qubits) at p = 3, energies and gradients at two of
the test's points, with the terms of each graph's two largest cones; and the
6x6 torus at p = 3, whose 72 edges form one orbit (translations and the swap
of the two coordinates, checked here edge by edge) with a 28-qubit cone,
term and gradient of that cone at one point.

Run once on a CPU (it takes about an hour; the 28-qubit cone needs ~30 GB):
    python tests/golden/make_gradient_goldens.py [near|full|all]
``near`` computes only the cases not yet in near_stationary.json and keeps the rest.
"""
from __future__ import annotations

import json
import math
import os
import sys
import time
from multiprocessing import get_context

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import qaoa_oracle as O  # noqa: E402
from paper_2101_10296_gb300 import inputs as I  # noqa: E402

RHOS = (1e-3, 2e-4)  # |grad E| / |E| at the near-stationary points
N_NEAR = 6          # points per case


def circulant_orbits(n, edges):
    """Orbit of each edge under the rotations i -> i + 1: its jump length."""
    a, b = edges[:, 0], edges[:, 1]
    d = np.abs(a - b)
    return np.minimum(d, n - d)


def near_cases():
    """(name, builder, p, orbit ids, theta* or None)."""
    out = []
    for d in (8, 9, 10):
        n, e = I.hypercube(d)
        star = np.array([math.atan(1.0 / math.sqrt(d - 1)), math.pi / 8])
        out.append((f"Q{d}", ("hypercube", [d]), 1, np.zeros(len(e), dtype=np.int64), star))
    n, e = I.circulant(30, [1, 2])
    out.append(("C30(1,2)", ("circulant", [30, [1, 2]]), 4, circulant_orbits(n, e), None))
    n, e = I.complete_bipartite(8, 8)
    out.append(("K8,8", ("complete_bipartite", [8, 8]), 3, np.zeros(len(e), dtype=np.int64), None))
    # p = 3 default plans on the core-tile schedule: 15-qubit cones with 11 inner
    # qubits, and 20-qubit cones with 14 (later layers mix at most nine qubits)
    for nn, jumps in ((30, [1, 2]), (40, [1, 3])):
        n, e = I.circulant(nn, jumps)
        name = f"C{nn}({','.join(str(j) for j in jumps)})p3"
        out.append((name, ("circulant", [nn, jumps]), 3, circulant_orbits(n, e), None))
    return out


def build(spec):
    name, args = spec
    return getattr(I, name)(*args)


def eg(graph, p, oid, th):
    n, e = graph
    return O.orbit_grad_adjoint(n, e, th, p, oid)


def maximise(graph, p, oid):
    """L-BFGS from the linear ramp gamma_l = 0.2 + 0.4 l / p, beta_l = 0.5 - 0.4 l / p
    (the shape optimal QAOA parameters take on regular graphs)."""
    from scipy.optimize import minimize
    ramp = np.arange(1, p + 1) / p
    th0 = np.concatenate([0.2 + 0.4 * ramp, 0.5 - 0.4 * ramp])

    def f(th):
        en, g = eg(graph, p, oid, th)
        return -en, -g
    r = minimize(f, th0, jac=True, method="L-BFGS-B", options={"maxiter": 200, "gtol": 1e-9, "ftol": 1e-15})
    return r.x


_NW = {}


def _near_job(args):
    """One near-stationary point: secant on delta along u, then the oracle there."""
    spec, p, oid, star, m, u, rho = args
    graph = build(spec)
    target = rho * m
    d0, d1 = 1e-5, 1e-3
    f0 = np.linalg.norm(eg(graph, p, oid, star + d0 * u)[1]) - target
    f1 = np.linalg.norm(eg(graph, p, oid, star + d1 * u)[1]) - target
    for _ in range(30):
        d2 = d1 - f1 * (d1 - d0) / (f1 - f0)
        d0, f0 = d1, f1
        d1 = min(max(d2, 0.1 * d1), 10.0 * d1)
        f1 = np.linalg.norm(eg(graph, p, oid, star + d1 * u)[1]) - target
        if abs(f1) <= 1e-3 * target:
            break
    th = star + d1 * u
    en, g = eg(graph, p, oid, th)
    return th, en, g


def make_near(only_missing=True):
    """Computes the cases not yet in near_stationary.json (all of them with
    only_missing=False) and writes the file with every case."""
    path = os.path.join(HERE, "near_stationary.json")
    rows = []
    if only_missing and os.path.exists(path):
        rows = json.load(open(path))["rows"]
    have = {r["case"] for r in rows}
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    pool = get_context("spawn").Pool(os.cpu_count() or 1)
    for k, (name, spec, p, oid, star) in enumerate(near_cases()):
        if name in have:
            continue
        t0 = time.time()
        graph = build(spec)
        m = len(graph[1])
        if star is None:
            star = maximise(graph, p, oid)
        e_star, g_star = eg(graph, p, oid, star)
        rng = np.random.default_rng(70 + k)
        dirs = [rng.normal(size=star.size) for _ in range(N_NEAR)]
        dirs = [u / np.linalg.norm(u) for u in dirs]
        jobs = [(spec, p, oid, star, m, u, rho) for rho in RHOS for u in dirs]
        for (_, _, _, _, _, _, rho), (th, en, g) in zip(jobs, pool.map(_near_job, jobs, chunksize=1)):
            rows.append({"case": name, "graph": list(spec), "p": p, "rho": rho, "theta": th.tolist(), "energy": en,
                         "grad": g.tolist(), "grad_norm_over_edges": float(np.linalg.norm(g) / m),
                         "theta_star": star.tolist(), "energy_star": e_star})
        print(f"{name}: theta*={star.tolist()} E*={e_star:.9f} |g*|={np.linalg.norm(g_star):.2e} "
              f"({time.time() - t0:.0f} s)", flush=True)
    pool.close()
    doc = {"about": "FP64 oracle energies and adjoint gradients at points near a local maximum of E "
                    "(|grad E| = rho |E|); written by tests/golden/make_gradient_goldens.py from oracle/ only",
           "rhos": list(RHOS), "orbits": "Q_d, K_{a,b}: one orbit; circulants: one orbit per jump (rotations)",
           "rows": rows}
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)


# ------------------------------------------------------------ full size

def _term_job(job):
    seed, ei, j, p, th = job
    n, e = I.random_regular(24, 3, seed)
    verts, _, le = O.lightcone(n, e, e[ei], p)
    val, g = O.term_grad_adjoint(len(verts), le, th, p)
    return seed, ei, j, len(verts), val, g


def torus_orbit_is_all_edges(r, c):
    """Edge 0's images under the translations (and the coordinate swap, r = c)
    are every edge of the torus: one orbit of 2 r c edges."""
    n, e = I.torus(r, c)
    eset = {(int(a), int(b)) for a, b in e}
    a0, b0 = (int(x) for x in e[0])
    seen = set()
    maps = []
    for dr in range(r):
        for dc in range(c):
            maps.append(lambda v, dr=dr, dc=dc: ((v // c + dr) % r) * c + (v % c + dc) % c)
    if r == c:
        base = list(maps)
        maps += [lambda v, f=f: f((v % c) * c + v // c) for f in base]
    for f in maps:
        img = tuple(sorted((f(a0), f(b0))))
        assert img in eset
        seen.add(img)
    return len(seen) == len(e)


def make_full():
    p = 3
    seeds = (1, 2, 3, 4)
    P = 128
    pts = (0, 64)
    jobs = []
    size = {}
    for s in seeds:
        n, e = I.random_regular(24, 3, s)
        adj = O.adjacency(n, e)
        th = I.draw_params(p, P, s)
        for ei in range(len(e)):
            size[(s, ei)] = len(O.lightcone(n, e, e[ei], p, adj)[0])
        for j in pts:
            for ei in range(len(e)):
                jobs.append((s, ei, j, p, th[j]))
    t0 = time.time()
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    with get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        # largest cones first, so that the pool ends evenly
        res = pool.map(_term_job, sorted(jobs, key=lambda j: -size[(j[0], j[1])]), chunksize=1)
    print(f"rr3 n=24 p=3: {len(jobs)} cone adjoints in {time.time() - t0:.0f} s", flush=True)
    rr3 = []
    for s in seeds:
        for j in pts:
            mine = [r for r in res if r[0] == s and r[2] == j]
            energy = float(sum(r[4] for r in mine))
            grad = np.sum([r[5] for r in mine], axis=0)
            big = sorted(mine, key=lambda r: (-r[3], r[1]))[:2]
            rr3.append({"seed": s, "point": j, "energy": energy, "grad": grad.tolist(),
                        "largest_cones": [{"edge": int(r[1]), "qubits": int(r[3]), "term_cut": float(r[4]),
                                           "term_grad": r[5].tolist()} for r in big]})
    assert torus_orbit_is_all_edges(6, 6)
    n, e = I.torus(6, 6)
    th = I.draw_params(p, 4, 6)
    torus = []
    for j in (0,):
        t0 = time.time()
        verts, _, le = O.lightcone(n, e, e[0], p)
        val, g = O.term_grad_adjoint(len(verts), le, th[j], p)
        torus.append({"point": j, "qubits": len(verts), "edges": len(e), "energy": len(e) * val,
                      "grad": (len(e) * g).tolist(), "term_cut": val})
        print(f"torus 6x6 p=3 point {j}: {len(verts)} qubits, {time.time() - t0:.0f} s", flush=True)
    doc = {"about": "FP64 oracle energies and adjoint gradients of the gradient configuration at full size; "
                    "written by tests/golden/make_gradient_goldens.py from oracle/ only",
           "rr3_n24_p3": {"points_per_graph": P, "points": list(pts), "param_seed": "graph seed", "rows": rr3},
           "torus6_p3": {"points": 4, "param_seed": 6, "orbit": "all 72 edges (edge 0's cone)", "rows": torus}}
    with open(os.path.join(HERE, "full_size_gradient.json"), "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    if what in ("near", "all"):
        make_near()
    if what in ("full", "all"):
        make_full()
