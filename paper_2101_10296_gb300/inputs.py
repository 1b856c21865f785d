"""Seeded synthetic inputs: graphs and QAOA parameter points.

This module holds only input generation -- no QAOA arithmetic -- so that the
FP64 oracle and the CUDA path can both draw the same inputs from it without
sharing any of the method's code.

Graphs are returned as ``(n_vertices, edges)`` with ``edges`` an ``int32``
array of shape ``[m, 2]``, each row ``(a, b)`` with ``a < b``, rows sorted
lexicographically.  All families are simple and undirected, as the MaxCut
problem of the paper (Sec. 2.4) requires.

The random families use the project's own generators seeded through
``numpy.random.default_rng(seed)`` so that streams do not depend on any
third-party graph library:

* random d-regular: configuration (pairing) model, rejecting and re-drawing
  pairings that contain a loop or a repeated edge;
* Erdos-Renyi G(n, q): every pair independently with probability q.

The structured families (tori, hypercubes, circulants, complete, Paley,
rook's graphs) stand in for the highly symmetric graphs of the paper's
benchmark (Sec. 5, Tables 1-2), whose files are not available.
"""
from __future__ import annotations

import math

import numpy as np


def _normalize(edges, n):
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if e.size == 0:
        return np.zeros((0, 2), dtype=np.int32)
    a = np.minimum(e[:, 0], e[:, 1])
    b = np.maximum(e[:, 0], e[:, 1])
    if np.any(a == b):
        raise ValueError("self-loop in generated graph")
    key = np.unique(a * n + b)
    out = np.stack([key // n, key % n], axis=1).astype(np.int32)
    return out


def random_regular(n, d, seed, max_tries=100000):
    """Uniform random simple d-regular graph on n vertices (pairing model)."""
    if (n * d) % 2 or d >= n:
        raise ValueError("need n*d even and d < n")
    rng = np.random.default_rng(seed)
    points = np.repeat(np.arange(n, dtype=np.int64), d)
    for _ in range(max_tries):
        perm = rng.permutation(points)
        a = perm[0::2]
        b = perm[1::2]
        if np.any(a == b):
            continue
        lo = np.minimum(a, b)
        hi = np.maximum(a, b)
        key = lo * n + hi
        if np.unique(key).size != key.size:
            continue
        return n, _normalize(np.stack([lo, hi], axis=1), n)
    raise RuntimeError("pairing model did not produce a simple graph")


def erdos_renyi(n, q, seed, chunk=1 << 22):
    """G(n, q): each of the n(n-1)/2 pairs present independently with prob. q.

    Pairs are enumerated in lexicographic order (a < b) and tested in chunks.
    """
    rng = np.random.default_rng(seed)
    total = n * (n - 1) // 2
    sel = []
    for start in range(0, total, chunk):
        cnt = min(chunk, total - start)
        hit = np.nonzero(rng.random(cnt) < q)[0].astype(np.int64) + start
        sel.append(hit)
    idx = np.concatenate(sel) if sel else np.zeros(0, np.int64)
    # invert the lexicographic pair index k -> (a, b)
    # row a starts at s(a) = a*(2n-a-1)/2
    a = np.floor((2 * n - 1 - np.sqrt((2 * n - 1) ** 2 - 8.0 * idx)) / 2).astype(np.int64)
    s = a * (2 * n - a - 1) // 2
    # guard against floating error at row boundaries
    over = idx < s
    a[over] -= 1
    s = a * (2 * n - a - 1) // 2
    nxt = (a + 1) * (2 * n - a - 2) // 2
    under = idx >= nxt
    a[under] += 1
    s = a * (2 * n - a - 1) // 2
    b = idx - s + a + 1
    return n, _normalize(np.stack([a, b], axis=1), n)


def torus(rows, cols):
    """Periodic rows x cols grid (4-regular for rows, cols >= 3)."""
    n = rows * cols
    e = []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            e.append((v, r * cols + (c + 1) % cols))
            e.append((v, ((r + 1) % rows) * cols + c))
    return n, _normalize(e, n)


def hypercube(d):
    """Q_d: vertices are d-bit words, edges join words at Hamming distance 1."""
    n = 1 << d
    e = [(v, v ^ (1 << k)) for v in range(n) for k in range(d) if v < v ^ (1 << k)]
    return n, _normalize(e, n)


def circulant(n, jumps):
    """C_n(j1, j2, ...): vertex i adjacent to i +- j (mod n) for every jump j."""
    e = []
    for j in jumps:
        for i in range(n):
            e.append((i, (i + j) % n))
    return n, _normalize(e, n)


def complete(n):
    e = [(a, b) for a in range(n) for b in range(a + 1, n)]
    return n, _normalize(e, n)


def cycle(n):
    return circulant(n, [1])


def path(n):
    return n, _normalize([(i, i + 1) for i in range(n - 1)], n)


def star(leaves):
    return leaves + 1, _normalize([(0, i) for i in range(1, leaves + 1)], leaves + 1)


def complete_bipartite(a, b):
    return a + b, _normalize([(i, a + j) for i in range(a) for j in range(b)], a + b)


def petersen():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return 10, _normalize(outer + spokes + inner, 10)


def paley(q):
    """Paley graph on the prime q = 1 (mod 4): a ~ b iff a - b is a nonzero square."""
    if q % 4 != 1:
        raise ValueError("Paley graph needs q = 1 mod 4")
    for f in range(2, int(math.isqrt(q)) + 1):
        if q % f == 0:
            raise ValueError("this generator needs q prime")
    squares = {(x * x) % q for x in range(1, q)}
    e = [(a, b) for a in range(q) for b in range(a + 1, q) if (b - a) % q in squares]
    return q, _normalize(e, q)


def rook(m):
    """Rook's graph K_m x K_m (Cartesian product): cells sharing a row or column."""
    n = m * m
    e = []
    for r in range(m):
        for c in range(m):
            v = r * m + c
            for c2 in range(c + 1, m):
                e.append((v, r * m + c2))
            for r2 in range(r + 1, m):
                e.append((v, r2 * m + c))
    return n, _normalize(e, n)


def wheel(spokes):
    """W_n: a hub joined to every vertex of a cycle of length ``spokes``."""
    n = spokes + 1
    e = [(0, i) for i in range(1, n)] + [(i, 1 + (i % spokes)) for i in range(1, n)]
    return n, _normalize(e, n)


def draw_params(p, n_points, seed):
    """QAOA parameter points: gamma ~ U[0, pi)^p first, then beta ~ U[0, pi/2)^p.

    Returns a float64 array ``[n_points, 2p]`` laid out (gamma_1..gamma_p,
    beta_1..beta_p) per row.
    """
    rng = np.random.default_rng(seed)
    g = rng.uniform(0.0, math.pi, size=(n_points, p))
    b = rng.uniform(0.0, math.pi / 2, size=(n_points, p))
    return np.ascontiguousarray(np.concatenate([g, b], axis=1))


def mixed_benchmark_graphs():
    """48 graph specs shaped like the paper's benchmark (Sec. 5): 100 to 10,000
    vertices, asymmetric random graphs mixed with highly symmetric families.

    Returns a list of ``(name, builder)`` with ``builder()`` -> (n, edges).
    """
    specs = []
    seed = 100
    for d in (3, 4, 5):
        for n in (100, 1000, 3000, 10000):
            if (n * d) % 2:
                n += 1
            specs.append((f"rr{d}-{n}", (lambda n=n, d=d, s=seed: random_regular(n, d, s))))
            seed += 1
    for n in (100, 300, 1000, 3000, 5000, 10000):
        specs.append((f"er4-{n}", (lambda n=n, s=seed: erdos_renyi(n, 4.0 / (n - 1), s))))
        seed += 1
    for r, c in ((10, 10), (20, 20), (30, 30), (50, 50), (100, 100), (10, 20), (25, 40), (50, 100)):
        specs.append((f"torus-{r}x{c}", (lambda r=r, c=c: torus(r, c))))
    for d in range(8, 14):
        specs.append((f"Q{d}", (lambda d=d: hypercube(d))))
    circ = [
        (100, (1, 7)), (500, (1, 7)), (1000, (1, 7, 23)), (2000, (1, 3)),
        (5000, (1, 7, 23)), (5000, (1, 7)), (10000, (1, 2)), (10000, (1, 7, 23)),
        (200, (1, 5)), (300, (1, 4, 9)), (700, (1, 3, 11)), (1500, (1, 10)),
        (2500, (1, 6, 15)), (4000, (1, 9)), (6000, (1, 5, 13)), (8000, (1, 11)),
    ]
    for n, j in circ:
        specs.append((f"C{n}({','.join(map(str, j))})", (lambda n=n, j=j: circulant(n, j))))
    assert len(specs) == 48
    return specs


def torus3d(m):
    """Periodic m x m x m cubic grid (6-regular for m >= 3)."""
    n = m * m * m
    e = []
    for x in range(m):
        for y in range(m):
            for z in range(m):
                v = (x * m + y) * m + z
                e.append((v, (((x + 1) % m) * m + y) * m + z))
                e.append((v, (x * m + (y + 1) % m) * m + z))
                e.append((v, (x * m + y) * m + (z + 1) % m))
    return n, _normalize(e, n)
