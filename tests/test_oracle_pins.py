"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a dense
matrix-exponential construction built from Pauli matrices, the published p = 1
closed form, exact special values, symmetries of the energy, textbook
automorphism-group orders, and finite differences of the definition.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import qaoa_oracle as O
from paper_2101_10296_gb300 import inputs as I

SMALL_GRAPHS = {
    "K2": (2, np.array([[0, 1]])),
    "K3": I.complete(3),
    "K4": I.complete(4),
    "P4": I.path(4),
    "C5": I.cycle(5),
    "W5": I.wheel(5),
    "star4": I.star(4),
    "K23": I.complete_bipartite(2, 3),
    "petersen": I.petersen(),
    "rr3-10": I.random_regular(10, 3, 7),
    "er-9": I.erdos_renyi(9, 0.4, 3),
}


def _rand_theta(p, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.uniform(-np.pi, np.pi, p), rng.uniform(-np.pi / 2, np.pi / 2, p)])


# ------------------------------------------------------------------ O1 vs expm

def _pauli_on(n, q, P):
    """Dense operator acting as P on qubit q (bit q of the basis index)."""
    mats = [np.eye(2)] * n
    mats = list(mats)
    mats[n - 1 - q] = P
    out = np.array([[1.0]])
    for m in mats:
        out = np.kron(out, m)
    return out


def _dense_state(n, edges, gam, bet):
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)
    dim = 1 << n
    H = np.zeros((dim, dim), dtype=complex)
    for u, v in edges:
        H += 0.5 * (np.eye(dim) - _pauli_on(n, int(u), Z) @ _pauli_on(n, int(v), Z))
    B = sum(_pauli_on(n, q, X) for q in range(n))
    psi = np.ones(dim, dtype=complex) / math.sqrt(dim)
    for g, b in zip(gam, bet):
        psi = scipy.linalg.expm(-1j * b * B) @ (scipy.linalg.expm(-1j * g * H) @ psi)
    return psi, H


@pytest.mark.parametrize("name", ["K2", "K3", "P4", "C5", "W5", "K23"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_state_matches_dense_expm(name, p):
    n, edges = SMALL_GRAPHS[name]
    theta = _rand_theta(p, 11 * p + n)
    gam, bet = theta[:p], theta[p:]
    psi_ref, H = _dense_state(n, edges, gam, bet)
    psi = O.qaoa_state(n, edges, gam, bet)
    # identity part of H is a global phase: compare up to one phase
    ov = np.vdot(psi_ref, psi)
    assert abs(abs(ov) - 1.0) < 1e-12
    assert np.allclose(psi * np.conj(ov) / abs(ov), psi_ref, atol=1e-12)
    e_ref = float(np.real(np.vdot(psi_ref, H @ psi_ref)))
    assert abs(O.full_energy(n, edges, theta, p) - e_ref) < 1e-11


def test_cut_table_matches_hamiltonian_diagonal():
    n, edges = SMALL_GRAPHS["W5"]
    _, H = _dense_state(n, edges, [], [])
    assert np.array_equal(O.cut_table(n, edges), np.rint(np.real(np.diag(H))).astype(np.int64))


# ------------------------------------------------------- closed form, p = 1

@pytest.mark.parametrize("name", sorted(SMALL_GRAPHS))
def test_p1_terms_match_closed_form(name):
    n, edges = SMALL_GRAPHS[name]
    for seed in range(3):
        g, b = _rand_theta(1, seed)
        terms = O.full_edge_terms(n, edges, [g, b], 1)
        for e, t in zip(edges, terms):
            cf = O.closed_form_p1_term(n, edges, e, g, b)
            assert abs(0.5 * (1 - t) - cf) < 1e-13


def test_k2_special_case():
    for g, b in [(0.3, 0.2), (2.0, 0.42), (-1.1, 1.3)]:
        e = O.full_energy(2, np.array([[0, 1]]), [g, b], 1)
        assert abs(e - (0.5 + 0.5 * np.sin(4 * b) * np.sin(g))) < 1e-14


# ------------------------------------------------------- exact special values

@pytest.mark.parametrize("p", [1, 2, 3])
def test_zero_beta_or_gamma_gives_half_edges(p):
    n, edges = SMALL_GRAPHS["petersen"]
    th = _rand_theta(p, 5)
    zb = th.copy()
    zb[p:] = 0
    zg = th.copy()
    zg[:p] = 0
    assert abs(O.full_energy(n, edges, zb, p) - len(edges) / 2) < 1e-12
    assert abs(O.full_energy(n, edges, zg, p) - len(edges) / 2) < 1e-12


@pytest.mark.parametrize("p", [1, 2])
def test_energy_symmetries_and_norm(p):
    n, edges = SMALL_GRAPHS["rr3-10"]
    th = _rand_theta(p, 9)
    e0 = O.full_energy(n, edges, th, p)
    assert abs(O.full_energy(n, edges, -th, p) - e0) < 1e-11
    for k in range(p):
        t2 = th.copy()
        t2[k] += 2 * np.pi
        assert abs(O.full_energy(n, edges, t2, p) - e0) < 1e-10
        t3 = th.copy()
        t3[p + k] += np.pi / 2
        assert abs(O.full_energy(n, edges, t3, p) - e0) < 1e-10
    assert abs(O.full_norm(n, edges, th, p) - 1.0) < 1e-13


# ------------------------------------------------ locality: O1 == sum of O2

@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("name", ["petersen", "rr3-10", "er-9", "W5"])
def test_lightcone_sum_equals_full_energy(name, p):
    n, edges = SMALL_GRAPHS[name]
    th = _rand_theta(p, 21 + p)
    assert abs(O.lightcone_energy(n, edges, th, p) - O.full_energy(n, edges, th, p)) < 1e-11


def test_lightcone_sum_equals_full_energy_larger():
    n, edges = I.random_regular(16, 3, 4)
    th = _rand_theta(2, 4)
    full = O.full_edge_terms(n, edges, th, 2)
    for e, t in zip(edges, full):
        assert abs(O.lightcone_term(n, edges, e, th, 2) - t) < 1e-12


def test_lightcone_ball_shape():
    # on a long cycle the radius-p ball around an edge has 2 + 2p vertices
    n, edges = I.cycle(30)
    for p in (1, 2, 3):
        verts, dist, le = O.lightcone(n, edges, (0, 1), p)
        assert len(verts) == 2 + 2 * p
        assert verts[:2] == [0, 1]
        assert dist == sorted(dist)
        assert len(le) == 2 * p + 1


# --------------------------------------------------- orbits (brute force)

@pytest.mark.parametrize("graph,order,n_orb", [
    (I.cycle(7), 14, 1),
    (I.complete(5), 120, 1),
    (I.path(6), 2, 3),
    (I.path(5), 2, 2),
    (I.petersen(), 120, 1),
    (I.hypercube(3), 48, 1),
    (I.complete_bipartite(2, 3), 12, 1),
    (I.star(4), 24, 1),
    (I.wheel(5), 10, 2),
])
def test_brute_automorphism_group_orders(graph, order, n_orb):
    n, edges = graph
    autos = O.brute_automorphisms(n, edges)
    assert len(autos) == order
    assert len(set(autos)) == order
    assert len(np.unique(O.brute_edge_orbits(n, edges))) == n_orb


def test_brute_orbits_are_unions_under_every_automorphism():
    n, edges = I.random_regular(8, 3, 2)
    orb = O.brute_edge_orbits(n, edges)
    idx = {tuple(e): i for i, e in enumerate(edges.tolist())}
    for s in O.brute_automorphisms(n, edges):
        for i, (a, b) in enumerate(edges.tolist()):
            j = idx[(min(s[a], s[b]), max(s[a], s[b]))]
            assert orb[i] == orb[j]


# -------------------------------------------- Theorem 1 and orbit weighting

@pytest.mark.parametrize("name", ["petersen", "W5", "K23", "C5", "star4"])
def test_theorem1_equal_terms_within_orbits(name):
    n, edges = SMALL_GRAPHS[name]
    orb = O.brute_edge_orbits(n, edges)
    for p in (1, 2):
        terms = O.full_edge_terms(n, edges, _rand_theta(p, 3), p)
        for m in np.unique(orb):
            t = terms[orb == m]
            assert np.ptp(t) < 1e-12


@pytest.mark.parametrize("p", [1, 2])
def test_orbit_weighted_energy_equals_full(p):
    n, edges = I.circulant(12, [1, 3])
    orb = O.brute_edge_orbits(n, edges)
    th = _rand_theta(p, 8)
    assert abs(O.orbit_energy(n, edges, th, p, orb) - O.full_energy(n, edges, th, p)) < 1e-11


# ------------------------------------------------------------- gradients

@pytest.mark.parametrize("p", [1, 2, 3])
def test_adjoint_matches_finite_differences(p):
    n, edges = SMALL_GRAPHS["rr3-10"]
    th = _rand_theta(p, 30 + p)
    e, g = O.grad_adjoint(n, edges, th, p)
    assert abs(e - O.full_energy(n, edges, th, p)) < 1e-11
    fd = O.grad_fd(n, edges, th, p, h=1e-4)
    assert np.max(np.abs(g - fd)) < 1e-6 * max(1.0, np.max(np.abs(g)))


def test_adjoint_matches_closed_form_derivative_p1():
    sympy = pytest.importorskip("sympy")
    gs, bs = sympy.symbols("g b")
    n, edges = SMALL_GRAPHS["W5"]
    adj = O.adjacency(n, edges)
    g0, b0 = 0.7, -0.35
    for e in edges:
        u, v = int(e[0]), int(e[1])
        du, dv = len(adj[u]) - 1, len(adj[v]) - 1
        t = len(set(adj[u]) & set(adj[v]))
        expr = (sympy.Rational(1, 2) + sympy.Rational(1, 4) * sympy.sin(4 * bs) * sympy.sin(gs)
                * (sympy.cos(gs) ** du + sympy.cos(gs) ** dv)
                - sympy.Rational(1, 4) * sympy.sin(2 * bs) ** 2 * sympy.cos(gs) ** (du + dv - 2 * t)
                * (1 - sympy.cos(2 * gs) ** t))
        dg = float(sympy.diff(expr, gs).subs({gs: g0, bs: b0}))
        db = float(sympy.diff(expr, bs).subs({gs: g0, bs: b0}))
        verts, _, le = O.lightcone(n, edges, e, 1)
        val, gr = O.term_grad_adjoint(len(verts), le, np.array([g0, b0]), 1)
        assert abs(val - float(expr.subs({gs: g0, bs: b0}))) < 1e-13
        assert abs(gr[0] - dg) < 1e-12 and abs(gr[1] - db) < 1e-12


def test_orbit_grad_equals_plain_grad():
    n, edges = I.circulant(14, [1, 4])
    orb = O.brute_edge_orbits(n, edges)
    th = _rand_theta(2, 2)
    e1, g1 = O.grad_adjoint(n, edges, th, 2)
    e2, g2 = O.orbit_grad_adjoint(n, edges, th, 2, orb)
    assert abs(e1 - e2) < 1e-11 and np.max(np.abs(g1 - g2)) < 1e-11


def test_params_recipe_first_draw():
    # gamma ~ U[0, pi) first, then beta ~ U[0, pi/2), default_rng(seed)
    th = I.draw_params(1, 1, 0)
    u = np.random.default_rng(0).random(2)
    assert th[0, 0] == u[0] * np.pi and th[0, 1] == u[1] * np.pi / 2


# --------------------------------------------- O6: weighted (coloured) edges

def _signs(m, seed, values=(1, -1)):
    return np.random.default_rng(seed).choice(values, m)


def _dense_weighted(n, edges, weights, gam, bet):
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)
    dim = 1 << n
    H = np.zeros((dim, dim), dtype=complex)
    for (u, v), w in zip(edges, weights):
        H += 0.5 * w * (np.eye(dim) - _pauli_on(n, int(u), Z) @ _pauli_on(n, int(v), Z))
    B = sum(_pauli_on(n, q, X) for q in range(n))
    psi = np.ones(dim, dtype=complex) / math.sqrt(dim)
    for g, b in zip(gam, bet):
        psi = scipy.linalg.expm(-1j * b * B) @ (scipy.linalg.expm(-1j * g * H) @ psi)
    return psi, H


@pytest.mark.parametrize("name", ["K3", "P4", "C5", "W5", "K23"])
@pytest.mark.parametrize("p", [1, 2])
def test_weighted_state_matches_dense_expm(name, p):
    """Weighted cost H = sum_e w_e (I - Z_u Z_v)/2 (Sec. 4's objective with edge
    colours) built from Pauli matrices, weights in {-2, -1, 1, 3}."""
    n, edges = SMALL_GRAPHS[name]
    w = _signs(len(edges), 5 + p, (-2, -1, 1, 3))
    theta = _rand_theta(p, 7 * p + n)
    gam, bet = theta[:p], theta[p:]
    psi_ref, H = _dense_weighted(n, edges, w, gam, bet)
    psi = O.qaoa_state(n, edges, gam, bet, w)
    ov = np.vdot(psi_ref, psi)
    assert abs(abs(ov) - 1.0) < 1e-12
    assert np.allclose(psi * np.conj(ov) / abs(ov), psi_ref, atol=1e-12)
    assert np.array_equal(O.cut_table(n, edges, w), np.real(np.diag(H)).round().astype(np.int64))
    e_ref = float(np.real(np.vdot(psi_ref, H @ psi_ref)))
    assert abs(O.full_energy(n, edges, theta, p, w) - e_ref) < 1e-10


@pytest.mark.parametrize("p", [1, 2, 3])
def test_weighted_lightcone_sum_equals_full_energy(p):
    n, edges = SMALL_GRAPHS["petersen"]
    w = _signs(len(edges), p)
    th = _rand_theta(p, 40 + p)
    assert abs(O.lightcone_energy(n, edges, th, p, weights=w) - O.full_energy(n, edges, th, p, w)) < 1e-10


def test_all_negative_weights_mirror_the_unweighted_energy():
    """C -> -C maps E(gamma, beta) to -E(-gamma, beta): an identity that ties the
    weighted code path to the unweighted one."""
    n, edges = SMALL_GRAPHS["rr3-10"]
    for p in (1, 2):
        th = _rand_theta(p, 60 + p)
        mirrored = th.copy()
        mirrored[:p] *= -1
        e_neg = O.full_energy(n, edges, th, p, -np.ones(len(edges), dtype=np.int64))
        assert abs(e_neg + O.full_energy(n, edges, mirrored, p)) < 1e-11


@pytest.mark.parametrize("p", [1, 2])
def test_weighted_adjoint_matches_finite_differences(p):
    n, edges = SMALL_GRAPHS["W5"]
    w = _signs(len(edges), 3 + p, (-1, 1, 2))
    th = _rand_theta(p, 80 + p)
    e, g = O.grad_adjoint(n, edges, th, p, weights=w)
    assert abs(e - O.lightcone_energy(n, edges, th, p, weights=w)) < 1e-11
    assert np.max(np.abs(g - O.grad_fd(n, edges, th, p, h=1e-5, weights=w))) < 1e-7


def test_weighted_orbits_respect_colours():
    """An 8-cycle with alternating signs keeps only the rotations by two and the
    reflections that map signs to signs: 8 automorphisms, two edge orbits (the
    positive and the negative edges); all-positive gives the dihedral 16 and one."""
    n, edges = I.cycle(8)
    # edge (i, i+1) gets sign (-1)^i, the closing edge (0, 7) sign -1
    alt = np.array([(-1) ** int(min(a, b)) if abs(int(a) - int(b)) == 1 else -1 for a, b in edges])
    assert len(O.brute_automorphisms(n, edges)) == 16
    assert len(O.brute_automorphisms(n, edges, alt)) == 8
    orb = O.brute_edge_orbits(n, edges, alt)
    assert len(set(orb)) == 2
    for s in set(orb):
        assert len(set(alt[orb == s])) == 1
    th = _rand_theta(2, 5)
    e1, g1 = O.grad_adjoint(n, edges, th, 2, weights=alt)
    e2, g2 = O.orbit_grad_adjoint(n, edges, th, 2, orb, weights=alt)
    assert abs(e1 - e2) < 1e-11 and np.max(np.abs(g1 - g2)) < 1e-11
