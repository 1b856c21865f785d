"""FP64 CPU oracle for the depth-p QAOA MaxCut energy and its gradient.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs may call it.  It shares no code with the CUDA path.

Everything here is the plain definition, written out slowly in float64 /
complex128 NumPy (arXiv:2101.10296):

* QAOA state (Sec. 2.2): |beta,gamma>_p = U_B(beta_p) U_P(gamma_p) ...
  U_B(beta_1) U_P(gamma_1) |+>^n with U_P(gamma) = exp(-i gamma H),
  U_B(beta) = prod_j exp(-i beta X_j).
* MaxCut Hamiltonian (Sec. 2.4): H = 1/2 sum_{(u,v) in E} (I - Z_u Z_v),
  i.e. the diagonal cut count C(z) = #{(u,v) in E : z_u != z_v}.
* Term-wise energy (Sec. 2.3, the linearity equation):
  E = sum_{(u,v)} 1/2 (1 - <Z_u Z_v>).
* Reverse causal cone (Sec. 2.3): a term on {u,v} only sees the vertices
  within distance p of the edge.  ``lightcone`` extracts that ball with its
  own BFS and the term is simulated on the induced subgraph, with the mixer on
  every cone qubit in every layer (no pruning).
* Symmetry (Sec. 3, Theorem 1 and the orbit-weighted sum that follows it):
  E = sum_m |orbit_m| * 1/2 (1 - <Z Z>_{rep_m}).
* Weighted objective (Sec. 4, the Ising objective with coloured edges):
  with an integer weight w_e per edge (``weights``; None = all 1),
  C(z) = sum_e w_e [z_u != z_v] and E = sum_e w_e 1/2 (1 - <Z_u Z_v>);
  symmetries must map every edge to an edge of the same weight.

Bit convention: bit q of the basis index z is the value of qubit (vertex) q.
Readings where the paper is silent: the mixer is exp(-i beta X) with no 1/2
(Sec. 2.2), phase before mixer in each layer, the identity part of H is
dropped from U_P (a global phase).

``closed_form_p1_term`` is not from this paper: it is the published p = 1
MaxCut edge expectation with the triangle correction (Wang, Hadfield, Jiang,
Rieffel, Phys. Rev. A 97, 022304 (2018)), used as an independent pin.
``grad_adjoint`` is the standard reverse-mode (adjoint) derivative of an
expectation value; ``grad_fd`` is central finite differences of the
definition.  Parity pins for every function live in ``tests/test_oracle_*``.
"""
from __future__ import annotations

from collections import deque

import numpy as np


# ---------------------------------------------------------------- basics

def cut_table(n, edges, weights=None):
    """C(z) for z in [0, 2^n): the number (total weight) of edges (a, b) with
    z_a != z_b."""
    z = np.arange(1 << n, dtype=np.int64)
    c = np.zeros(1 << n, dtype=np.int64)
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.ones(len(edges), dtype=np.int64) if weights is None else np.asarray(weights, dtype=np.int64)
    for (a, b), we in zip(edges, w):
        c += we * (((z >> a) ^ (z >> b)) & 1)
    return c


def plus_state(n):
    """|+>^n: every amplitude 2^(-n/2)."""
    return np.full(1 << n, 2.0 ** (-n / 2.0), dtype=np.complex128)


def apply_phase(psi, cut, gamma):
    """U_P(gamma) = exp(-i gamma H) with H diagonal = C(z)."""
    return psi * np.exp(-1j * gamma * cut)


def apply_rx(psi, q, beta):
    """exp(-i beta X_q) = cos(beta) I - i sin(beta) X_q on qubit q."""
    c, s = np.cos(beta), np.sin(beta)
    v = psi.reshape(-1, 2, 1 << q)
    a = v[:, 0, :].copy()
    b = v[:, 1, :].copy()
    out = np.empty_like(v)
    out[:, 0, :] = c * a - 1j * s * b
    out[:, 1, :] = -1j * s * a + c * b
    return out.reshape(-1)


def apply_mixer(psi, n, beta, qubits=None):
    """U_B(beta) = prod_j exp(-i beta X_j) over ``qubits`` (default: all n)."""
    for q in range(n) if qubits is None else qubits:
        psi = apply_rx(psi, q, beta)
    return psi


def qaoa_state(n, edges, gammas, betas, weights=None):
    """|beta, gamma>_p on n qubits for the graph ``edges`` (Sec. 2.2)."""
    cut = cut_table(n, edges, weights)
    psi = plus_state(n)
    for g, b in zip(gammas, betas):
        psi = apply_phase(psi, cut, g)
        psi = apply_mixer(psi, n, b)
    return psi


def zz_expectation(psi, u, v):
    """<psi| Z_u Z_v |psi> = sum_z |psi_z|^2 (-1)^(z_u xor z_v)."""
    z = np.arange(psi.size, dtype=np.int64)
    sign = 1.0 - 2.0 * (((z >> u) ^ (z >> v)) & 1)
    return float(np.sum(np.abs(psi) ** 2 * sign))


def split_params(theta, p):
    theta = np.asarray(theta, dtype=np.float64).reshape(-1)
    return theta[:p], theta[p:2 * p]


# ------------------------------------------------ O1: whole-graph state

def full_energy(n, edges, theta, p, weights=None):
    """E_p = <psi| C |psi> on the whole graph (n <= ~22)."""
    g, b = split_params(theta, p)
    psi = qaoa_state(n, edges, g, b, weights)
    return float(np.sum(np.abs(psi) ** 2 * cut_table(n, edges, weights)))


def full_edge_terms(n, edges, theta, p):
    """<Z_u Z_v> for every edge, on the whole-graph state."""
    g, b = split_params(theta, p)
    psi = qaoa_state(n, edges, g, b)
    return np.array([zz_expectation(psi, int(u), int(v)) for u, v in edges])


def full_norm(n, edges, theta, p):
    g, b = split_params(theta, p)
    psi = qaoa_state(n, edges, g, b)
    return float(np.sum(np.abs(psi) ** 2))


# ---------------------------------------- O2: per-edge reverse causal cone

def adjacency(n, edges):
    adj = [[] for _ in range(n)]
    for a, b in np.asarray(edges, dtype=np.int64).reshape(-1, 2):
        adj[a].append(int(b))
        adj[b].append(int(a))
    return adj


def lightcone(n, edges, edge, p, adj=None):
    """Ball of radius p around the edge (u, v) (Sec. 2.3).

    Returns ``(verts, dist, local_edges)``: ``verts`` lists the global vertex of
    each local qubit -- u first, v second, the rest ordered by (distance to
    {u, v}, global id) -- and ``local_edges`` is the induced subgraph on the
    ball in local labels.
    """
    if adj is None:
        adj = adjacency(n, edges)
    u, v = int(min(edge)), int(max(edge))
    dist = {u: 0, v: 0}
    queue = deque([u, v])
    while queue:
        x = queue.popleft()
        if dist[x] == p:
            continue
        for y in adj[x]:
            if y not in dist:
                dist[y] = dist[x] + 1
                queue.append(y)
    rest = sorted((w for w in dist if w not in (u, v)), key=lambda w: (dist[w], w))
    verts = [u, v] + rest
    local = {w: i for i, w in enumerate(verts)}
    ledges = []
    for a in verts:
        for b in adj[a]:
            if b in local and a < b:
                ledges.append((local[a], local[b]))
    ledges.sort()
    return verts, [dist[w] for w in verts], np.array(ledges, dtype=np.int64).reshape(-1, 2)


def cone_weights(edges, weights, verts, ledges):
    """Weights of a cone's local edges (None for an unweighted graph)."""
    if weights is None:
        return None
    w = {(int(min(a, b)), int(max(a, b))): int(x) for (a, b), x in zip(np.asarray(edges).reshape(-1, 2), weights)}
    return np.array([w[(min(verts[a], verts[b]), max(verts[a], verts[b]))] for a, b in ledges], dtype=np.int64)


def lightcone_term(n, edges, edge, theta, p, adj=None, weights=None):
    """<Z_u Z_v> of one edge, simulated on its cone's induced subgraph."""
    verts, _, ledges = lightcone(n, edges, edge, p, adj)
    g, b = split_params(theta, p)
    psi = qaoa_state(len(verts), ledges, g, b, cone_weights(edges, weights, verts, ledges))
    return zz_expectation(psi, 0, 1)


def lightcone_energy(n, edges, theta, p, adj=None, weights=None):
    """E_p = sum over every edge of w_e 1/2 (1 - <Z_u Z_v>_cone) (no symmetry)."""
    if adj is None:
        adj = adjacency(n, edges)
    w = np.ones(len(edges)) if weights is None else np.asarray(weights, dtype=np.float64)
    return float(sum(we * 0.5 * (1.0 - lightcone_term(n, edges, e, theta, p, adj, weights))
                     for e, we in zip(edges, w)))


def orbit_energy(n, edges, theta, p, orbit_id, adj=None):
    """E_p = sum_m |orbit_m| 1/2 (1 - <Z Z>_{rep_m}) (Sec. 3).

    ``orbit_id[i]`` labels the orbit of edge i; the representative of an orbit
    is its first edge in input order.
    """
    if adj is None:
        adj = adjacency(n, edges)
    orbit_id = np.asarray(orbit_id)
    total = 0.0
    for m in np.unique(orbit_id):
        members = np.nonzero(orbit_id == m)[0]
        rep = edges[members[0]]
        total += members.size * 0.5 * (1.0 - lightcone_term(n, edges, rep, theta, p, adj))
    return total


# --------------------------------------------- O3: p = 1 closed form (pin)

def closed_form_p1_term(n, edges, edge, gamma, beta, adj=None):
    """Published p = 1 expectation of the edge's cut indicator 1/2(1 - Z_u Z_v).

    With d_u = deg(u) - 1, d_v = deg(v) - 1 and t = number of triangles on
    the edge: 1/2 + 1/4 sin(4b) sin(g) (cos^d_u g + cos^d_v g)
    - 1/4 sin^2(2b) cos^(d_u + d_v - 2t) g (1 - cos^t 2g).
    """
    if adj is None:
        adj = adjacency(n, edges)
    u, v = int(edge[0]), int(edge[1])
    du = len(adj[u]) - 1
    dv = len(adj[v]) - 1
    t = len(set(adj[u]) & set(adj[v]))
    cg = np.cos(gamma)
    return (0.5 + 0.25 * np.sin(4 * beta) * np.sin(gamma) * (cg ** du + cg ** dv)
            - 0.25 * np.sin(2 * beta) ** 2 * cg ** (du + dv - 2 * t) * (1.0 - np.cos(2 * gamma) ** t))


# ------------------------------------------------ O4: brute-force orbits

def brute_automorphisms(n, edges, weights=None):
    """Every automorphism of the graph, by backtracking over vertex images.

    An automorphism is a vertex permutation preserving adjacency (Sec. 2.6),
    and with weights the weight of every edge (Sec. 4: edge colours).
    Vertices are mapped in the order 0..n-1; a partial map is extended only if
    degree and adjacency to every already-mapped vertex are preserved.
    """
    adjm = np.zeros((n, n), dtype=np.int64)  # edge weight, 0 = no edge
    w = np.ones(len(np.asarray(edges).reshape(-1, 2))) if weights is None else weights
    for (a, b), we in zip(np.asarray(edges, dtype=np.int64).reshape(-1, 2), w):
        adjm[a, b] = adjm[b, a] = int(we)
    deg = (adjm != 0).sum(axis=1)
    out = []
    img = [-1] * n
    used = [False] * n

    def extend(v):
        if v == n:
            out.append(tuple(img))
            return
        for w in range(n):
            if used[w] or deg[w] != deg[v]:
                continue
            ok = True
            for x in range(v):
                if adjm[x, v] != adjm[img[x], w]:
                    ok = False
                    break
            if ok:
                img[v] = w
                used[w] = True
                extend(v + 1)
                used[w] = False
                img[v] = -1

    extend(0)
    return out


def brute_edge_orbits(n, edges, weights=None):
    """Edge orbits under the full automorphism group (weight-preserving when
    weights are given).

    Returns ``orbit_id[m]`` with orbits numbered by their smallest edge index
    (edge order as given).
    """
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    index = {(int(a), int(b)): i for i, (a, b) in enumerate(edges)}
    m = len(edges)
    orbit = [-1] * m
    autos = brute_automorphisms(n, edges, weights)
    nxt = 0
    for i in range(m):
        if orbit[i] >= 0:
            continue
        a, b = int(edges[i, 0]), int(edges[i, 1])
        for s in autos:
            x, y = s[a], s[b]
            j = index[(min(x, y), max(x, y))]
            orbit[j] = nxt
        nxt += 1
    return np.array(orbit, dtype=np.int64)


# ---------------------------------------------------- O5: gradients

def energy_lightcone_theta(n, edges, theta, p, adj=None, weights=None):
    return lightcone_energy(n, edges, theta, p, adj, weights)


def grad_fd(n, edges, theta, p, h=1e-4, adj=None, weights=None):
    """Central finite differences of the cone-sum energy, FP64, step h."""
    if adj is None:
        adj = adjacency(n, edges)
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros(2 * p)
    for k in range(2 * p):
        tp = theta.copy()
        tm = theta.copy()
        tp[k] += h
        tm[k] -= h
        g[k] = (lightcone_energy(n, edges, tp, p, adj, weights) - lightcone_energy(n, edges, tm, p, adj, weights)) / (2 * h)
    return g


def term_grad_adjoint(nq, ledges, theta, p, lweights=None):
    """d/dtheta of 1/2 (1 - <Z_0 Z_1>) on one cone, by the adjoint method.

    Forward: phi_l = U_P(g_l) psi_{l-1}, psi_l = U_B(b_l) phi_l.  With the
    co-state lambda = O psi_p for O = -1/2 Z_0 Z_1 (the identity part of the
    observable contributes nothing), each derivative is twice the imaginary
    part of <lambda| G |psi> taken right after the gate exp(-i theta G):
    G = sum_j X_j for beta_l, G = C for gamma_l.  Both states are then taken
    back through the inverse gate.
    """
    gam, bet = split_params(theta, p)
    cut = cut_table(nq, ledges, lweights)
    psi = plus_state(nq)
    for g_, b_ in zip(gam, bet):
        psi = apply_phase(psi, cut, g_)
        psi = apply_mixer(psi, nq, b_)
    z = np.arange(1 << nq, dtype=np.int64)
    sign = 1.0 - 2.0 * ((z ^ (z >> 1)) & 1)
    lam = -0.5 * sign * psi
    value = 0.5 * (1.0 - float(np.sum(np.abs(psi) ** 2 * sign)))
    grad = np.zeros(2 * p)
    for l in range(p - 1, -1, -1):
        bpsi = np.zeros_like(psi)
        for q in range(nq):
            bpsi += psi.reshape(-1, 2, 1 << q)[:, ::-1, :].reshape(-1)
        grad[p + l] = 2.0 * float(np.imag(np.vdot(lam, bpsi)))
        psi = apply_mixer(psi, nq, -bet[l])
        lam = apply_mixer(lam, nq, -bet[l])
        grad[l] = 2.0 * float(np.imag(np.vdot(lam, cut * psi)))
        psi = apply_phase(psi, cut, -gam[l])
        lam = apply_phase(lam, cut, -gam[l])
    return value, grad


def grad_adjoint(n, edges, theta, p, adj=None, weights=None):
    """(E, dE/dtheta) summed over every edge's cone (times its weight), FP64 adjoint."""
    if adj is None:
        adj = adjacency(n, edges)
    w = np.ones(len(edges)) if weights is None else np.asarray(weights, dtype=np.float64)
    e_tot = 0.0
    g_tot = np.zeros(2 * p)
    for e, we in zip(edges, w):
        verts, _, ledges = lightcone(n, edges, e, p, adj)
        val, gr = term_grad_adjoint(len(verts), ledges, theta, p, cone_weights(edges, weights, verts, ledges))
        e_tot += we * val
        g_tot += we * gr
    return e_tot, g_tot


def orbit_grad_adjoint(n, edges, theta, p, orbit_id, adj=None, weights=None):
    """(E, dE/dtheta) from one cone per orbit weighted by the orbit size (and
    the representative's edge weight)."""
    if adj is None:
        adj = adjacency(n, edges)
    orbit_id = np.asarray(orbit_id)
    e_tot = 0.0
    g_tot = np.zeros(2 * p)
    for m in np.unique(orbit_id):
        members = np.nonzero(orbit_id == m)[0]
        rep = members[0]
        we = 1.0 if weights is None else float(weights[rep])
        verts, _, ledges = lightcone(n, edges, edges[rep], p, adj)
        val, gr = term_grad_adjoint(len(verts), ledges, theta, p, cone_weights(edges, weights, verts, ledges))
        e_tot += members.size * we * val
        g_tot += members.size * we * gr
    return e_tot, g_tot
