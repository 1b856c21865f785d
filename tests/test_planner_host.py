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


def _tree_orbits(levels, k=3):
    """Colourings of the leaves of the tree cone with k colours each, counted
    up to the tree's symmetries: a vertex with two exchangeable subtrees of f
    orbits each has f (f + 1) / 2 (unordered pairs), and the root edge's two
    ends are exchangeable too."""
    f = k
    for _ in range(levels):
        f = f * (f + 1) // 2
    return f


def test_block_orbits_of_known_cones(qlib):
    """Block counts after merging along the cone's symmetries, against counts
    fixed by hand (Burnside's lemma): a tree cone of a cubic graph at depth p
    has 2^(p+1) shell classes of two qubits hanging from a binary tree whose
    automorphisms fixing the root edge form an iterated wreath product; Q_12
    at p = 1 has two classes of 11 exchanged by swapping the root edge's ends,
    so 12 x 12 count pairs fall into 12 * 13 / 2 orbits."""
    n, edges = I.random_regular(2000, 3, 1)
    for p, expect in ((1, 6), (2, 21), (3, 231)):
        assert _tree_orbits(p) == expect
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
    assert len(counts) == 78 and w.sum() == 2.0 ** 22
    # every unordered pair of counts once
    assert sorted(tuple(sorted(c)) for c in counts.tolist()) == sorted(
        (a, b) for a in range(12) for b in range(a, 12))


def _block_orbits_brute(plan_plain, rep, nx):
    """Orbits of the class count vectors under every automorphism of the cone
    (networkx enumerates the isomorphisms of the cone onto itself that keep
    distances from the root edge and edge weights), with each orbit's number
    of shell assignments; None if there are too many automorphisms to list."""
    from networkx.algorithms.isomorphism import GraphMatcher, categorical_edge_match, categorical_node_match
    g = _cone_nx(plan_plain, rep)
    for (a, b), x in zip(plan_plain.cone(rep)[2], plan_plain.cone_weights(rep)):
        g.edges[int(a), int(b)]["w"] = int(x)
    cls, _ = plan_plain.shell(rep)
    counts, w = plan_plain.blocks(rep)
    index = {tuple(c): i for i, c in enumerate(counts.tolist())}
    ncls = counts.shape[1]
    perms = []
    gm = GraphMatcher(g, g, node_match=categorical_node_match("dist", -1), edge_match=categorical_edge_match("w", 0))
    for k, phi in enumerate(gm.isomorphisms_iter()):
        if k > 20000:
            return None
        pm = [-1] * ncls
        for q, img in phi.items():
            if cls[q] >= 0:
                assert pm[cls[q]] in (-1, cls[img])
                pm[cls[q]] = int(cls[img])
        perms.append(pm)
    orbit = [-1] * len(counts)
    for b in range(len(counts)):
        if orbit[b] >= 0:
            continue
        stack, orbit[b] = [b], b
        while stack:
            x = counts[stack.pop()]
            for pm in perms:
                y = [0] * ncls
                for k in range(ncls):
                    y[pm[k]] = int(x[k])
                j = index[tuple(y)]
                if orbit[j] < 0:
                    orbit[j] = b
                    stack.append(j)
    total = {}
    for b, o in enumerate(orbit):
        total[o] = total.get(o, 0.0) + w[b]
    return {tuple(counts[b].tolist()): total[o] for b, o in enumerate(orbit)}, total


@pytest.mark.parametrize("graph,p,weighted", [
    (I.petersen(), 1, False), (I.petersen(), 2, False), (I.torus(5, 5), 2, False), (I.circulant(20, [1, 4]), 1, False),
    (I.circulant(24, [1, 5]), 2, False), (I.hypercube(4), 2, False), (I.complete_bipartite(3, 4), 1, False),
    (I.random_regular(40, 3, 3), 2, False), (I.random_regular(30, 4, 2), 1, False), (I.random_regular(30, 3, 5), 2, True),
])
def test_block_orbits_match_brute_force(qlib, graph, p, weighted):
    """The planner's merged blocks are exactly the orbits of the class count
    vectors under the cone's full automorphism group (root edge fixed
    setwise), each carrying its orbit's number of shell assignments."""
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
        # one block per orbit, each with the orbit's weight
        keys = {}
        for c, x in zip(counts.tolist(), wt):
            o = of_block[tuple(c)]
            assert x == o
            keys[tuple(c)] = x
        assert sorted(keys.values()) == sorted(total.values())
        assert wt.sum() == 2.0 ** (plan.reps()["n_qubits"][r] - plan.reps()["n_inner"][r])
        checked += 1
    assert checked >= 6


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
