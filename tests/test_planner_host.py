"""Host planner through the C ABI (no GPU): edge orbits and reverse causal cones.

Orbits are checked against the oracle's brute-force enumeration and against
textbook group orders and the paper's printed orbit counts; cones against the
oracle's own BFS lightcone.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import qaoa_oracle as O
from paper_2101_10296_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_orbit_counts.txt")


def _canon(labels):
    """Relabel a partition by order of first occurrence."""
    seen = {}
    return np.array([seen.setdefault(int(x), len(seen)) for x in labels])


# ------------------------------------------------------------ vs brute force

def test_orbits_match_brute_force_all_graphs_on_5_vertices(qlib):
    pairs = list(itertools.combinations(range(5), 2))
    for mask in range(1, 1 << len(pairs)):
        edges = np.array([pairs[i] for i in range(len(pairs)) if mask >> i & 1])
        oid, norb, _, l10, comp = qlib.edge_orbits(5, edges)
        ref = O.brute_edge_orbits(5, edges)
        assert comp
        assert np.array_equal(_canon(oid), _canon(ref)), edges
        assert norb == len(np.unique(ref))
        assert abs(10 ** l10 - len(O.brute_automorphisms(5, edges))) < 1e-6 * 10 ** l10


@pytest.mark.parametrize("n,q,count", [(7, 0.3, 60), (8, 0.5, 40), (9, 0.35, 30), (10, 0.3, 12)])
def test_orbits_match_brute_force_random_graphs(qlib, n, q, count):
    rng = np.random.default_rng(n)
    for _ in range(count):
        _, edges = I.erdos_renyi(n, q, int(rng.integers(1 << 30)))
        if len(edges) == 0:
            continue
        oid, norb, _, l10, comp = qlib.edge_orbits(n, edges)
        ref = O.brute_edge_orbits(n, edges)
        assert comp
        assert np.array_equal(_canon(oid), _canon(ref))
        assert abs(10 ** l10 / len(O.brute_automorphisms(n, edges)) - 1) < 1e-9


@pytest.mark.parametrize("graph", [I.petersen(), I.wheel(6), I.hypercube(3), I.circulant(10, [1, 3]),
                                   I.complete_bipartite(3, 4), I.random_regular(10, 3, 5)])
def test_orbits_match_brute_force_families(qlib, graph):
    n, edges = graph
    oid, _, _, _, _ = qlib.edge_orbits(n, edges)
    assert np.array_equal(_canon(oid), _canon(O.brute_edge_orbits(n, edges)))


@pytest.mark.parametrize("n,q,count,values", [(7, 0.4, 40, (1, -1)), (8, 0.5, 30, (1, -1, 2)),
                                              (9, 0.35, 20, (1, -1))])
def test_weighted_orbits_match_brute_force(qlib, n, q, count, values):
    """Edge colours (Sec. 4): the planner's orbits are those of the
    weight-preserving automorphisms, as brute force enumerates them."""
    rng = np.random.default_rng(100 + n)
    for _ in range(count):
        _, edges = I.erdos_renyi(n, q, int(rng.integers(1 << 30)))
        if len(edges) == 0:
            continue
        w = rng.choice(values, len(edges))
        plan = qlib.Plan((n, edges), 1, weights=w)
        oid, norb, l10, comp = plan.orbits(0)
        ref = O.brute_edge_orbits(n, edges, w)
        assert comp and np.array_equal(_canon(oid), _canon(ref))
        assert abs(10 ** l10 / len(O.brute_automorphisms(n, edges, w)) - 1) < 1e-9
        reps = plan.reps()
        for r in range(len(reps["edge"])):
            e = int(reps["edge"][r])
            assert reps["weight"][r] == int(np.sum(oid == e)) * int(w[e])


def test_weighted_input_errors_and_caps(qlib):
    n, edges = I.cycle(6)
    for bad in (0, 65, -65):
        w = np.ones(len(edges), dtype=np.int64)
        w[2] = bad
        with pytest.raises(qlib.QAOAError) as ei:
            qlib.Plan((n, edges), 1, weights=w)
        assert ei.value.code == qlib.QAOA_E_INVALID and "weight" in str(ei.value)
    # a p = 1 cone of C_6 has 3 edges; weights 30 + 30 + 30 exceed the 64-bit cut word
    with pytest.raises(qlib.QAOAError) as ei:
        qlib.Plan((n, edges), 1, weights=np.full(len(edges), 30))
    assert ei.value.code == qlib.QAOA_E_CONE_TOO_LARGE and "weight" in str(ei.value)
    # the boundary: a star's cone holds all its edges; 8 x 8 = 64 bits fit, 5 x 13 = 65 do not
    plan = qlib.Plan(I.star(8), 1, weights=np.full(8, 8))
    assert plan.info()["max_edges"] == 8 and plan.info()["n_reps"] == 1
    with pytest.raises(qlib.QAOAError) as ei:
        qlib.Plan(I.star(5), 1, weights=np.full(5, 13))
    assert ei.value.code == qlib.QAOA_E_CONE_TOO_LARGE and "65 > cap 64" in str(ei.value)


def test_orbit_id_is_smallest_edge_of_orbit(qlib):
    n, edges = I.circulant(12, [1, 5])
    oid, *_ = qlib.edge_orbits(n, edges)
    for i, r in enumerate(oid):
        assert r <= i and oid[r] == r


# ----------------------------------------------------- textbook group orders

def _log10_fact(k):
    return math.lgamma(k + 1) / math.log(10)


@pytest.mark.parametrize("name,graph,log10_order,n_orb", [
    ("K12", I.complete(12), _log10_fact(12), 1),
    ("C31", I.cycle(31), math.log10(62), 1),
    ("Q6", I.hypercube(6), 6 * math.log10(2) + _log10_fact(6), 1),
    ("Q10", I.hypercube(10), 10 * math.log10(2) + _log10_fact(10), 1),
    ("petersen", I.petersen(), math.log10(120), 1),
    ("torus7x7", I.torus(7, 7), math.log10(8 * 49), 1),
    ("torus5x7", I.torus(5, 7), math.log10(4 * 35), 2),
    ("torus3d-5", I.torus3d(5), math.log10(48 * 125), 1),
    ("paley13", I.paley(13), math.log10(13 * 12 / 2), 1),
    ("paley29", I.paley(29), math.log10(29 * 28 / 2), 1),
    ("rook6", I.rook(6), math.log10(2) + 2 * _log10_fact(6), 1),
    ("star9", I.star(9), _log10_fact(9), 1),
    ("K34", I.complete_bipartite(3, 4), _log10_fact(3) + _log10_fact(4), 1),
    ("P9", I.path(9), math.log10(2), 4),
])
def test_group_order_and_orbit_count(qlib, name, graph, log10_order, n_orb):
    n, edges = graph
    oid, norb, ngen, l10, comp = qlib.edge_orbits(n, edges)
    assert comp
    assert norb == n_orb
    assert abs(l10 - log10_order) < 1e-9


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            name, m, n, norb = line.split()[:4]
            rows.append((name, int(m), int(n), int(norb)))
    return rows


def _family(name):
    if name.startswith("k-"):
        return I.complete(int(name[2:]))
    if name.startswith("paley-"):
        return I.paley(int(name[6:]))
    if name.startswith("lattice-"):
        return I.rook(int(name[8:]))
    if name.startswith("grid-w-2-"):
        m = int(name[9:])
        return I.torus(m, m)
    if name.startswith("grid-w-3-"):
        return I.torus3d(int(name[9:]))
    raise KeyError(name)


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_paper_printed_orbit_counts(qlib, row):
    name, m, n, norb_paper = row
    nv, edges = _family(name)
    assert (nv, len(edges)) == (n, m)
    _, norb, _, _, comp = qlib.edge_orbits(nv, edges)
    assert comp and norb == norb_paper


@pytest.mark.parametrize("graph,n_orb", [
    (I.circulant(20, [1, 4]), 2),
    (I.circulant(5000, [1, 7, 23]), 3),
    (I.circulant(5000, [1, 7]), 2),
    (I.torus(100, 100), 1),
    (I.torus(50, 200), 2),
    (I.hypercube(12), 1),
])
def test_benchmark_family_orbit_counts(qlib, graph, n_orb):
    n, edges = graph
    _, norb, _, _, comp = qlib.edge_orbits(n, edges)
    assert comp and norb == n_orb


def test_c20_orbits_match_brute_force(qlib):
    n, edges = I.circulant(20, [1, 4])
    oid, *_ = qlib.edge_orbits(n, edges)
    assert np.array_equal(_canon(oid), _canon(O.brute_edge_orbits(n, edges)))


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_random_3_regular_are_asymmetric(qlib, seed):
    # Sec. 2.6: random 3-regular graphs almost surely have no automorphism
    n, edges = I.random_regular(2000, 3, seed)
    _, norb, _, l10, comp = qlib.edge_orbits(n, edges)
    assert comp and norb == len(edges) and l10 == 0.0


def test_budget_fallback_gives_sub_orbits(qlib):
    n, edges = I.rook(7)
    oid_small, norb_small, _, _, comp = qlib.edge_orbits(n, edges, budget=3)
    assert not comp
    oid_full, norb_full, *_ = qlib.edge_orbits(n, edges)
    assert norb_full == 1 and norb_small >= norb_full
    # every orbit of the subgroup lies inside an orbit of the full group
    for r in np.unique(oid_small):
        assert len(np.unique(oid_full[oid_small == r])) == 1


# ---------------------------------------------------------------- cones

@pytest.mark.parametrize("graph,p", [
    (I.petersen(), 1), (I.petersen(), 2), (I.random_regular(40, 3, 3), 2), (I.random_regular(24, 3, 1), 3),
    (I.torus(8, 8), 2), (I.erdos_renyi(60, 0.07, 2), 1), (I.hypercube(5), 1), (I.circulant(30, [1, 4]), 2),
])
def test_cones_match_oracle_lightcone(qlib, graph, p):
    n, edges = graph
    plan = qlib.Plan((n, edges), p, orbits=False)
    reps = plan.reps()
    assert len(reps["edge"]) == len(edges)
    adj = O.adjacency(n, edges)
    for r in range(0, len(edges), max(1, len(edges) // 25)):
        verts, dist, ce = plan.cone(r)
        e = edges[reps["edge"][r]]
        ov, od, oe = O.lightcone(n, edges, e, p, adj)
        assert list(verts) == ov and list(dist) == od
        # cone terms: induced edges with an endpoint within distance p-1
        keep = sorted((min(a, b), max(a, b)) for a, b in oe.tolist() if min(od[a], od[b]) <= p - 1)
        assert [tuple(x) for x in ce.tolist()] == keep
        assert reps["n_inner"][r] == sum(d <= p - 1 for d in od)
        assert reps["n_qubits"][r] == len(ov)


def test_full_cone_flag_marks_every_qubit_inner(qlib):
    n, edges = I.random_regular(30, 3, 2)
    plan = qlib.Plan((n, edges), 2, orbits=False, full_cone=True)
    reps = plan.reps()
    assert np.array_equal(reps["n_inner"], reps["n_qubits"])


def test_multi_graph_plan_weights_sum_to_edges(qlib):
    gs = [I.circulant(20, [1, 4]), I.torus(6, 6), I.random_regular(30, 3, 1), I.petersen()]
    plan = qlib.Plan(gs, 1)
    reps = plan.reps()
    info = plan.info()
    assert info["n_graphs"] == 4 and info["n_edges_total"] == sum(len(e) for _, e in gs)
    for g, (_, e) in enumerate(gs):
        assert reps["weight"][reps["graph"] == g].sum() == len(e)
    assert info["n_reps"] == sum(qlib.edge_orbits(n, e)[1] for n, e in gs)
    for g, (n, e) in enumerate(gs):
        assert np.array_equal(plan.orbits(g)[0], qlib.edge_orbits(n, e)[0])
    assert info["orbits_complete"] == 1


def test_orbits_off_every_edge_is_a_rep(qlib):
    n, edges = I.torus(6, 6)
    plan = qlib.Plan((n, edges), 1, orbits=False)
    reps = plan.reps()
    assert np.array_equal(reps["edge"], np.arange(len(edges))) and np.all(reps["weight"] == 1)


def test_empty_and_isolated_graphs(qlib):
    plan = qlib.Plan((6, np.zeros((0, 2), dtype=np.int32)), 2)
    assert plan.info()["n_reps"] == 0
    plan = qlib.Plan((9, np.array([[0, 1], [2, 3]])), 2)  # isolated vertices 4..8
    reps = plan.reps()
    assert plan.info()["n_reps"] == 1 and reps["weight"][0] == 2 and reps["n_qubits"][0] == 2


# ----------------------------------------------------------- error paths

@pytest.mark.parametrize("n,edges,p,msg", [
    (4, [[0, 0]], 1, "self-loop"),
    (4, [[0, 1], [1, 0]], 1, "repeated"),
    (4, [[0, 4]], 1, "outside"),
    (4, [[0, 1]], 0, "p must"),
    (4, [[0, 1]], 9, "p must"),
])
def test_invalid_inputs_are_rejected(qlib, n, edges, p, msg):
    with pytest.raises(qlib.QAOAError) as ei:
        qlib.Plan((n, np.array(edges)), p)
    assert ei.value.code == qlib.QAOA_E_INVALID and msg in str(ei.value)


def test_cone_caps(qlib):
    n, edges = I.random_regular(200, 3, 1)
    with pytest.raises(qlib.QAOAError) as ei:
        qlib.Plan((n, edges), 3, max_cone_qubits=20)
    assert ei.value.code == qlib.QAOA_E_CONE_TOO_LARGE
    n, edges = I.complete(40)  # p = 1 cone of K_40 has 2*38+1 = 77 edges > 64
    with pytest.raises(qlib.QAOAError) as ei:
        qlib.Plan((n, edges), 1)
    assert ei.value.code == qlib.QAOA_E_CONE_TOO_LARGE
    # the qubit cap, QAOA_MAX_CONE_QUBITS = 32: a p = 1 cone of a star holds the whole star
    assert qlib.Plan(I.star(31), 1).info()["max_qubits"] == 32
    assert qlib.Plan(I.torus(8, 8), 3).info()["max_qubits"] == 32
    with pytest.raises(qlib.QAOAError) as ei:
        qlib.Plan(I.star(32), 1)
    assert ei.value.code == qlib.QAOA_E_CONE_TOO_LARGE and "33 qubits" in str(ei.value)


def test_bad_call_arguments(qlib):
    import ctypes as C
    h = C.c_void_p()
    nv = np.array([3], dtype=np.int32)
    offs = np.array([1, 2], dtype=np.int64)
    e = np.array([[0, 1]], dtype=np.int32)
    rc = qlib.lib().qaoa_plan_graphs(1, qlib._ptr(nv, C.c_int32), qlib._ptr(offs, C.c_int64),
                                     qlib._ptr(e, C.c_int32), 1, 1, 0, 0, C.byref(h))
    assert rc == qlib.QAOA_E_INVALID
    assert qlib.lib().qaoa_plan_graph(3, 1, qlib._ptr(e, C.c_int32), 1, 1, 0, 0, None) == qlib.QAOA_E_INVALID
    assert qlib.lib().qaoa_plan_info(None, None) == qlib.QAOA_E_INVALID
    assert qlib.lib().qaoa_energy(None, 1, None, None, None, None) == qlib.QAOA_E_INVALID
    nb = C.c_int64()
    assert qlib.lib().qaoa_plan_blocks(None, 0, C.byref(nb), None, None, None) == qlib.QAOA_E_INVALID
    plan = qlib.Plan(I.petersen(), 1)
    for rep in (-1, plan.info()["n_reps"]):
        assert qlib.lib().qaoa_plan_blocks(plan.handle, rep, C.byref(nb), None, None, None) == qlib.QAOA_E_INVALID
    # counts only, weights only: the same rows as both together
    counts, w = plan.blocks(0)
    nc = counts.shape[1]
    c2 = np.zeros_like(counts)
    w2 = np.zeros_like(w)
    assert qlib.lib().qaoa_plan_blocks(plan.handle, 0, None, None, qlib._ptr(c2, C.c_uint8), None) == qlib.QAOA_OK
    assert qlib.lib().qaoa_plan_blocks(plan.handle, 0, None, None, None, qlib._ptr(w2, C.c_double)) == qlib.QAOA_OK
    assert np.array_equal(c2, counts) and np.array_equal(w2, w) and nc >= 1


def test_plan_flags(qlib):
    """Every documented flag is accepted (the large-state schedule switch
    changes nothing on the host), an unknown bit is refused."""
    import ctypes as C
    n, edges = I.random_regular(24, 3, 1)
    a = qlib.Plan((n, edges), 3)
    b = qlib.Plan((n, edges), 3, big_general=True)
    for key in ("n_qubits", "n_inner", "weight"):
        assert np.array_equal(a.reps()[key], b.reps()[key])
    assert np.array_equal(a.shell_blocks(), b.shell_blocks())
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32))
    h = C.c_void_p()
    rc = qlib.lib().qaoa_plan_graph(n, len(edges), qlib._ptr(e, C.c_int32), 3, 64, 0, 0, C.byref(h))
    assert rc == qlib.QAOA_E_INVALID


# ------------------------------------------------------------ cone classes

def _cone_nx(plan, rep):
    nx = pytest.importorskip("networkx")
    verts, dist, ce = plan.cone(rep)
    g = nx.Graph()
    for i, d in enumerate(dist):
        g.add_node(i, dist=int(d))
    g.add_edges_from(map(tuple, ce))
    return g


@pytest.mark.parametrize("graph,p", [(I.random_regular(30, 3, 2), 2), (I.erdos_renyi(40, 0.15, 5), 1),
                                     (I.random_regular(24, 3, 1), 3), (I.circulant(30, [1, 4]), 2),
                                     (I.petersen(), 2)])
def test_cone_classes_are_the_isomorphism_classes(qlib, graph, p):
    """Edges share a cone class exactly when their cones are isomorphic with
    the root edge fixed setwise: networkx's matcher (distance from the edge
    as the node label, so the root edge maps onto itself) gives the same
    partition of the edges."""
    nx = pytest.importorskip("networkx")
    from networkx.algorithms.isomorphism import GraphMatcher, categorical_node_match
    n, edges = graph
    plain = qlib.Plan((n, edges), p, orbits=False)  # one cone per edge, in edge order
    cc = qlib.Plan((n, edges), p, orbits=False, cone_classes=True)
    cid, ncls = cc.cone_classes(0)
    cones = [_cone_nx(plain, e) for e in range(len(edges))]
    match = categorical_node_match("dist", -1)
    ref = [-1] * len(edges)
    reps = []
    for e, g in enumerate(cones):
        for r in reps:
            if GraphMatcher(g, cones[r], node_match=match).is_isomorphic():
                ref[e] = r
                break
        if ref[e] < 0:
            ref[e] = e
            reps.append(e)
    assert list(cid) == ref
    assert ncls == len(reps) == cc.info()["n_reps"]
    assert int(cc.reps()["weight"].sum()) == len(edges)


def test_weighted_cone_classes_are_the_coloured_isomorphism_classes(qlib):
    """With edge weights a class joins only cones isomorphic as edge-coloured
    graphs (networkx with an edge-weight match)."""
    pytest.importorskip("networkx")
    from networkx.algorithms.isomorphism import GraphMatcher, categorical_edge_match, categorical_node_match
    n, edges = I.random_regular(30, 3, 2)
    w = np.random.default_rng(4).choice([1, -1], len(edges))
    plain = qlib.Plan((n, edges), 2, orbits=False, weights=w)
    cc = qlib.Plan((n, edges), 2, orbits=False, cone_classes=True, weights=w)
    cid, ncls = cc.cone_classes(0)
    cones = []
    for e in range(len(edges)):
        g = _cone_nx(plain, e)
        for (a, b), x in zip(plain.cone(e)[2], plain.cone_weights(e)):
            g.edges[int(a), int(b)]["w"] = int(x)
        cones.append(g)
    nm, em = categorical_node_match("dist", -1), categorical_edge_match("w", 0)
    ref, reps = [-1] * len(edges), []
    for e, g in enumerate(cones):
        for r in reps:
            if GraphMatcher(g, cones[r], node_match=nm, edge_match=em).is_isomorphic():
                ref[e] = r
                break
        if ref[e] < 0:
            ref[e] = e
            reps.append(e)
    assert list(cid) == ref and ncls == len(reps)
    assert int(cc.reps()["weight"].sum()) == int(np.sum(w))


def test_cone_classes_refine_orbits_and_keep_weights(qlib):
    """With orbit reduction on, every Aut(G) orbit lies in one cone class, the
    class weights sum to |E|, and a class's row carries its smallest edge."""
    for graph, p in ((I.circulant(40, [1, 3]), 2), (I.random_regular(200, 3, 4), 2), (I.torus(6, 6), 2)):
        n, edges = graph
        plan = qlib.Plan((n, edges), p, cone_classes=True)
        oid, _, _, _ = plan.orbits(0)
        cid, ncls = plan.cone_classes(0)
        for e in range(len(edges)):
            assert cid[oid[e]] == cid[e] and cid[e] <= e
        reps = plan.reps()
        assert ncls == len(reps["edge"]) and int(reps["weight"].sum()) == len(edges)
        assert sorted(reps["edge"]) == sorted(set(cid))
        # without the flag the classes are the orbits
        o = qlib.Plan((n, edges), p)
        assert np.array_equal(o.cone_classes(0)[0], o.orbits(0)[0])


def test_cone_classes_have_equal_oracle_terms(qlib):
    """The FP64 oracle gives every edge of a class the same term (Theorem 1's
    argument applied to cone isomorphisms), while different classes differ."""
    n, edges = I.random_regular(60, 3, 7)
    p = 2
    plan = qlib.Plan((n, edges), p, orbits=False, cone_classes=True)
    cid, ncls = plan.cone_classes(0)
    assert ncls < len(edges)
    adj = O.adjacency(n, edges)
    theta = I.draw_params(p, 1, 3)[0]
    classes = {}
    for e, c in enumerate(cid):
        classes.setdefault(int(c), []).append(e)
    vals = {}
    for c, members in sorted(classes.items(), key=lambda kv: -len(kv[1]))[:4]:
        terms = [O.lightcone_term(n, edges, edges[e], theta, p, adj) for e in members[:3]]
        assert max(terms) - min(terms) <= 1e-12
        vals[c] = terms[0]
    assert len(set(round(v, 9) for v in vals.values())) == len(vals)


# ------------------------------------------------------------ shell classes

@pytest.mark.parametrize("graph,p", [
    (I.random_regular(2000, 3, 1), 2), (I.hypercube(12), 1), (I.torus(8, 8), 2), (I.petersen(), 2),
    (I.erdos_renyi(300, 4 / 299, 9), 1), (I.circulant(5000, [1, 7, 23]), 1), (I.complete(6), 1),
])
def test_shell_classes_partition_the_shell(qlib, graph, p):
    n, edges = graph
    plan = qlib.Plan((n, edges), p, orbits=False, block_plain=True)
    plain = qlib.Plan((n, edges), p, orbits=False, shell_plain=True)
    reps = plan.reps()
    for r in range(0, len(edges), max(1, len(edges) // 20)):
        verts, dist, ce = plan.cone(r)
        cls, nb = plan.shell(r)
        n_in = reps["n_inner"][r]
        assert np.all(cls[:n_in] == -1) and np.all(cls[n_in:] >= 0)
        assert np.all(np.asarray(dist)[n_in:] == p)
        inner_nb = {q: frozenset(a for a, b in ce.tolist() for a, b in [(a, b), (b, a)] if b == q and a < n_in)
                    for q in range(n_in, len(verts))}
        # same class <=> same inner neighbours
        for q1 in range(n_in, len(verts)):
            for q2 in range(n_in, len(verts)):
                assert (cls[q1] == cls[q2]) == (inner_nb[q1] == inner_nb[q2])
        sizes = np.bincount(cls[n_in:]) if len(verts) > n_in else np.zeros(0, int)
        assert nb == int(np.prod(sizes + 1))
        pc, pnb = plain.shell(r)
        assert pnb == 2 ** (len(verts) - n_in) and len(set(pc[n_in:].tolist())) == len(verts) - n_in


def test_shell_blocks_of_known_cones(qlib):
    # random cubic graph at p = 2: tree-like cones have 4 classes of 2 -> 3^4 blocks
    n, edges = I.random_regular(2000, 3, 1)
    nbs = [qlib.Plan((n, edges), 2, orbits=False, block_plain=True).shell(r)[1] for r in range(50)]
    assert max(set(nbs), key=nbs.count) == 81
    # hypercube Q_12 at p = 1: neighbours of u only and of v only -> 12 x 12 blocks
    assert qlib.Plan(I.hypercube(12), 1, block_plain=True).shell(0)[1] == 144


def _orbit_count(vectors, generators):
    """Number of orbits of a finite set of tuples under the group the given
    maps (tuple -> tuple) generate, by breadth-first search."""
    seen, count = set(), 0
    for v in vectors:
        if v in seen:
            continue
        count += 1
        seen.add(v)
        stack = [v]
        while stack:
            x = stack.pop()
            for gen in generators:
                y = gen(x)
                if y not in seen:
                    seen.add(y)
                    stack.append(y)
    return count


def _tree_orbits(p):
    """Blocks of a tree cone of a cubic graph at depth p after merging: the
    2^p leaf classes (two shell qubits under each inner qubit at distance
    p - 1) give the phase vector entries 2 - 2 n_k in {2, 0, -2}; the cone's
    symmetries exchange the two subtrees below any inner vertex and the two
    ends of the root edge (a complete binary tree over the leaf classes); the
    global spin flip negates the vector."""
    L = 1 << p
    gens = [lambda v: tuple(-x for x in v)]
    for size in (L >> d for d in range(p)):  # subtree sizes L, L/2, ..., 2
        for off in range(0, L, size):
            def swap(v, off=off, h=size // 2):
                v = list(v)
                v[off:off + h], v[off + h:off + 2 * h] = v[off + h:off + 2 * h], v[off:off + h]
                return tuple(v)
            gens.append(swap)
    return _orbit_count(itertools.product((2, 0, -2), repeat=L), gens)


def test_block_orbits_of_known_cones(qlib):
    """Block counts after merging, against counts from an independent orbit
    enumeration: a tree cone of a cubic graph at depth p (binary-tree
    symmetries plus the spin flip, 3^(2^p) count vectors); Q_12 at p = 1 (two
    classes of 11 exchanged by swapping the root edge's ends, phase entries
    11 - 2n odd, so the flip fixes nothing: (144 + 12 + 0 + 12) / 4 = 42)."""
    assert [_tree_orbits(p) for p in (1, 2)] == [4, 13]  # Burnside by hand: 16 / 4, 208 / 16
    n, edges = I.random_regular(2000, 3, 1)
    for p in (1, 2, 3):
        expect = _tree_orbits(p)
        plan = qlib.Plan((n, edges), p, orbits=False)
        reps = plan.reps()
        tree = [r for r in range(60) if reps["n_cone_edges"][r] == reps["n_qubits"][r] - 1]
        assert len(tree) >= 40
        for r in tree:
            counts, w = plan.blocks(r)
            assert len(counts) == expect == plan.shell(r)[1]
            assert w.sum() == 2.0 ** (reps["n_qubits"][r] - reps["n_inner"][r])
    plan = qlib.Plan(I.hypercube(12), 1)
    counts, w = plan.blocks(0)
    assert len(counts) == 42 and w.sum() == 2.0 ** 22


def test_block_merging_is_independent_of_batching(qlib):
    """Cones with the same local structure share one merging result within a
    planning call; every representative's blocks come out the same whether
    its graph is planned alone or in a batch (and whichever thread merged
    that structure first)."""
    graphs = [I.random_regular(300, 3, s) for s in (1, 2)] + [I.torus(6, 6)]
    batch = qlib.Plan(graphs, 2)
    rows = [r for r in range(batch.info()["n_reps"])]
    graph_of = batch.reps()["graph"]
    alone = [qlib.Plan(g, 2) for g in graphs]
    start = {}
    for r in rows:
        start.setdefault(int(graph_of[r]), r)
    for r in rows:
        g = int(graph_of[r])
        c1, w1 = batch.blocks(r)
        c2, w2 = alone[g].blocks(r - start[g])
        assert np.array_equal(c1, c2) and np.array_equal(w1, w2)


def test_block_merging_cap_keeps_every_count_vector(qlib):
    """A cone with more than 2^16 count vectors keeps the plain enumeration
    (Q_6 at p = 2: twenty singleton shell classes, 2^20 blocks), and the
    block query still lists every one with weight 1."""
    plan = qlib.Plan(I.hypercube(6), 2)
    cls, nb = plan.shell(0)
    assert nb == 2 ** 20 == 2 ** int((cls >= 0).sum())
    counts, w = plan.blocks(0)
    assert counts.shape == (2 ** 20, 20) and np.all(w == 1.0)
    assert np.array_equal(counts[5], [1, 0, 1] + [0] * 17)  # mixed radix, least significant class first


def _phase_vector(plan, rep, counts):
    """The coefficient of z_q in the shell edges' part of the cut, for the
    assignment that sets the first n_k members of each class to 1: a shell
    neighbour t of q adds w [z_q != t] = w t + w (1 - 2t) z_q."""
    verts, dist, ce = plan.cone(rep)
    cw = plan.cone_weights(rep)
    cls, _ = plan.shell(rep)
    n_in = int(plan.reps()["n_inner"][rep])
    bits = _shell_bits(cls, counts)
    c = [0] * n_in
    for (a, b), w in zip(ce.tolist(), cw.tolist()):
        if a >= n_in:
            a, b = b, a
        if a < n_in <= b:
            c[a] += w * (1 - 2 * bits[b])
    return tuple(c)


def _shell_bits(cls, counts):
    bits, seen = {}, {}
    for q, k in enumerate(cls):
        if k >= 0:
            bits[q] = 1 if seen.get(k, 0) < counts[k] else 0
            seen[k] = seen.get(k, 0) + 1
    return bits


def _block_orbits_brute(plan_plain, rep, nx):
    """Merged blocks from first principles: count vectors with equal phase
    vectors, count vectors whose phase vectors are related by an automorphism
    of the cone's inner part (networkx enumerates every isomorphism of the
    inner subgraph onto itself that keeps distances from the root edge and
    edge weights), and complementary count vectors (s - n, the global spin
    flip) fall together; returns, per count vector, the total number of shell
    assignments of its class, or None if there are too many automorphisms to
    list."""
    from networkx.algorithms.isomorphism import GraphMatcher, categorical_edge_match, categorical_node_match
    n_in = int(plan_plain.reps()["n_inner"][rep])
    g = _cone_nx(plan_plain, rep)
    for (a, b), x in zip(plan_plain.cone(rep)[2], plan_plain.cone_weights(rep)):
        g.edges[int(a), int(b)]["w"] = int(x)
    inner = g.subgraph(range(n_in)).copy()
    cls, _ = plan_plain.shell(rep)
    counts, w = plan_plain.blocks(rep)
    rows = [tuple(c) for c in counts.tolist()]
    index = {c: i for i, c in enumerate(rows)}
    ncls = counts.shape[1]
    sizes = np.bincount(cls[cls >= 0], minlength=ncls)
    parent = list(range(len(rows)))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    def union(a, b):
        a, b = find(a), find(b)
        if a != b:
            parent[max(a, b)] = min(a, b)

    by_vec = {}
    for i, x in enumerate(rows):
        union(i, index[tuple(int(s) - v for s, v in zip(sizes, x))])
        by_vec.setdefault(_phase_vector(plan_plain, rep, x), []).append(i)
    for members in by_vec.values():
        for i in members[1:]:
            union(members[0], i)
    gm = GraphMatcher(inner, inner, node_match=categorical_node_match("dist", -1),
                      edge_match=categorical_edge_match("w", 0))
    for k, phi in enumerate(gm.isomorphisms_iter()):
        if k > 20000:
            return None
        for c, members in by_vec.items():
            img = [0] * n_in
            for q in range(n_in):
                img[phi[q]] = c[q]
            other = by_vec.get(tuple(img))
            if other is not None:
                union(members[0], other[0])
    total = {}
    for i in range(len(rows)):
        total[find(i)] = total.get(find(i), 0.0) + w[i]
    return {x: total[find(i)] for i, x in enumerate(rows)}, total


@pytest.mark.parametrize("graph,p,weighted", [
    (I.petersen(), 1, False), (I.petersen(), 2, False), (I.torus(5, 5), 2, False), (I.circulant(20, [1, 4]), 1, False),
    (I.circulant(24, [1, 5]), 2, False), (I.hypercube(4), 2, False), (I.complete_bipartite(3, 4), 1, False),
    (I.random_regular(40, 3, 3), 2, False), (I.random_regular(30, 4, 2), 1, False), (I.random_regular(30, 3, 5), 2, True),
    (I.erdos_renyi(30, 0.2, 3), 1, False), (I.erdos_renyi(30, 0.2, 4), 1, True), (I.random_regular(24, 3, 1), 3, False),
])
def test_block_orbits_match_brute_force(qlib, graph, p, weighted):
    """The planner's merged blocks are exactly the classes of count vectors
    under equal phase vectors, the full automorphism group of the cone's
    inner part (distances kept, so the root edge is fixed setwise) and the
    spin flip, each carrying its class's number of shell assignments."""
    nx = pytest.importorskip("networkx")
    n, edges = graph
    w = np.random.default_rng(1).choice([1, 2, -1], len(edges)) if weighted else None
    plain = qlib.Plan((n, edges), p, orbits=False, block_plain=True, weights=w)
    plan = qlib.Plan((n, edges), p, orbits=False, weights=w)
    checked = 0
    for r in range(0, len(edges), max(1, len(edges) // 12)):
        ref = _block_orbits_brute(plain, r, nx)
        if ref is None:
            continue
        of_block, total = ref
        counts, wt = plan.blocks(r)
        assert len(counts) == len(total) == plan.shell(r)[1]
        got = sorted(wt.tolist())
        for c, x in zip(counts.tolist(), wt):
            assert x == of_block[tuple(c)]
        assert got == sorted(total.values())
        assert wt.sum() == 2.0 ** (plan.reps()["n_qubits"][r] - plan.reps()["n_inner"][r])
        checked += 1
    assert checked >= 6


def _block_zz(plan, rep, counts, theta, p):
    """<Z_0 Z_1> of one shell block, simulated from the definition: the inner
    qubits start in |+>, the shell qubits hold the assignment (first n_k
    members of class k set to 1); each layer applies exp(-i gamma C) with C
    the weighted cut of the cone's edges and then exp(-i beta X) on the inner
    qubits within distance p - l of the edge (the pruned circuit, Sec. 2.3)."""
    verts, dist, ce = plan.cone(rep)
    cw = plan.cone_weights(rep)
    cls, _ = plan.shell(rep)
    n_in = int(plan.reps()["n_inner"][rep])
    bits = _shell_bits(cls, counts)
    z = np.arange(1 << n_in, dtype=np.int64)
    C = np.zeros(z.size)
    for (a, b), w in zip(ce.tolist(), cw.tolist()):
        za = (z >> a) & 1 if a < n_in else bits[a]
        zb = (z >> b) & 1 if b < n_in else bits[b]
        C += w * (za != zb)
    psi = np.full(z.size, 2.0 ** (-n_in / 2), dtype=np.complex128)
    g, b = theta[:p], theta[p:]
    for l in range(p):
        psi = psi * np.exp(-1j * g[l] * C)
        for q in range(n_in):
            if dist[q] <= p - 1 - l:
                psi = O.apply_rx(psi, q, b[l])
    return float(np.sum(np.abs(psi) ** 2 * (1 - 2 * (((z >> 0) ^ (z >> 1)) & 1))))


@pytest.mark.parametrize("graph,p,weighted", [(I.torus(5, 5), 2, False), (I.random_regular(30, 3, 5), 2, True),
                                              (I.erdos_renyi(24, 0.25, 3), 1, False), (I.circulant(24, [1, 5]), 2, False),
                                              (I.random_regular(24, 3, 1), 3, False), (I.erdos_renyi(20, 0.2, 6), 2, True),
                                              (I.circulant(16, [1, 3]), 2, True)])
def test_merged_blocks_have_equal_contributions(qlib, graph, p, weighted):
    """Every count vector merged into a block has the same <Z_0 Z_1> as the
    block's own (simulated from the definition in FP64), and the merged
    blocks weighted by their shell assignments give the oracle's term."""
    n, edges = graph
    w = np.random.default_rng(1).choice([1, 2, -1], len(edges)) if weighted else None
    plain = qlib.Plan((n, edges), p, orbits=False, block_plain=True, weights=w)
    plan = qlib.Plan((n, edges), p, orbits=False, weights=w)
    theta = I.draw_params(p, 1, 5)[0]
    adj = O.adjacency(n, edges)
    merged_any = False
    for r in range(0, len(edges), max(1, len(edges) // 5)):
        counts, wt = plan.blocks(r)
        all_counts, all_w = plain.blocks(r)
        if len(counts) < len(all_counts):
            merged_any = True
        vals = {tuple(c): _block_zz(plain, r, c, theta, p) for c in all_counts.tolist()}
        rep_vals = [_block_zz(plan, r, c, theta, p) for c in counts.tolist()]
        # each count vector's value equals that of a kept block with the same class weight
        kept = sorted(zip(rep_vals, wt.tolist()))
        for c, x in zip(all_counts.tolist(), all_w):
            assert any(abs(vals[tuple(c)] - v) <= 1e-12 for v, _ in kept)
        shell = plan.reps()["n_qubits"][r] - plan.reps()["n_inner"][r]
        term = float(np.dot(rep_vals, wt)) / 2.0 ** shell
        ref = O.lightcone_term(n, edges, edges[plan.reps()["edge"][r]], theta, p, adj, weights=w)
        assert abs(term - ref) <= 1e-12
    assert merged_any


# ------------------------------------------------------- failure injection

def test_corrupted_generators_are_rejected(qlib):
    n, edges = I.petersen()
    try:
        qlib.inject_fault(qlib.FAULT_GENERATOR, 10 ** 6)  # corrupt every candidate
        oid, norb, ngen, l10, comp = qlib.edge_orbits(n, edges)
    finally:
        qlib.inject_fault(qlib.FAULT_NONE, 0)
    # no corrupted candidate passes verification: the group found is trivial
    assert ngen == 0 and norb == len(edges) and np.array_equal(oid, np.arange(len(edges)))
    oid2, norb2, ngen2, *_ = qlib.edge_orbits(n, edges)
    assert norb2 == 1 and ngen2 > 0


def test_some_corrupted_generators_leave_a_valid_subgroup(qlib):
    n, edges = I.rook(5)
    true_oid, *_ = qlib.edge_orbits(n, edges)
    try:
        qlib.inject_fault(qlib.FAULT_GENERATOR, 2)
        oid, norb, ngen, _, comp = qlib.edge_orbits(n, edges)
    finally:
        qlib.inject_fault(qlib.FAULT_NONE, 0)
    for r in np.unique(oid):
        assert len(np.unique(true_oid[oid == r])) == 1


def test_inject_fault_rejects_unknown_kinds(qlib):
    with pytest.raises(qlib.QAOAError):
        qlib.inject_fault(7, 1)
