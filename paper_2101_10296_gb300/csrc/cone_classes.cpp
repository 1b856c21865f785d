// Cone classes: edges whose reverse causal cones are isomorphic have equal
// terms.
//
// The term of edge (u, v) (Sec. 2.3) is a function of its cone alone: the
// ball of radius p around {u, v} with the edges the phase keeps, each layer
// mixing the qubits within a given distance of the edge.  A bijection
// between two cones that maps edges onto edges and the root edge onto the
// root edge preserves those distances, so it carries one circuit and its
// observable (Z_u Z_v, symmetric in u and v) onto the other and the two
// terms are equal.  This is the symmetry argument of Sec. 3 (Theorem 1)
// applied to isomorphisms between cones instead of automorphisms of the
// whole graph: the local symmetries that Sec. 6 names as the next step.
// Edges in different Aut(G) orbits -- in a graph with no symmetry at all --
// share a term whenever their neighbourhoods look alike.
//
// Per graph, cones are bucketed by a colour-refinement invariant and each
// cone is tested against the class representatives in its bucket by an
// individualisation-refinement search whose leaves are checked edge by
// edge, so a class only ever joins cones proven isomorphic.
#include <algorithm>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "host.hpp"

namespace qaoa {
namespace {

constexpr int kMaxN = QAOA_MAX_CONE_QUBITS;

struct ConeGraph {
    int n = 0;
    int m = 0;
    uint32_t adj[kMaxN] = {0};
    int32_t dist[kMaxN] = {0};
    int8_t w[kMaxN][kMaxN] = {{0}};  // edge weights (colours)
};

ConeGraph cone_graph(const Cone &c) {
    ConeGraph g;
    g.n = c.n;
    g.m = int(c.ea.size());
    for (int v = 0; v < c.n; ++v) g.dist[v] = c.dist[v];
    for (size_t e = 0; e < c.ea.size(); ++e) {
        g.adj[c.ea[e]] |= 1u << c.eb[e];
        g.adj[c.eb[e]] |= 1u << c.ea[e];
        g.w[c.ea[e]][c.eb[e]] = g.w[c.eb[e]][c.ea[e]] = int8_t(c.ew[e]);
    }
    return g;
}

uint64_t mix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

int distinct(const uint64_t *c, int n) {
    uint64_t s[kMaxN];
    std::copy(c, c + n, s);
    std::sort(s, s + n);
    return int(std::unique(s, s + n) - s);
}

// One round of colour refinement with colours that are a function of the
// structure only (a hash of the own colour and the multiset of neighbour
// colours), so that colours of different cones can be compared.
void refine_round(const ConeGraph &g, uint64_t *col) {
    uint64_t nxt[kMaxN];
    for (int v = 0; v < g.n; ++v) {
        uint64_t s = 0;
        for (uint32_t a = g.adj[v]; a; a &= a - 1) {
            const int u = __builtin_ctz(a);
            s += mix64(col[u] ^ (uint64_t(uint8_t(g.w[v][u])) << 56));
        }
        nxt[v] = mix64(col[v] * 0x2545f4914f6cdd1dull ^ s);
    }
    std::copy(nxt, nxt + g.n, col);
}

// Refines both colourings by the same number of rounds until neither
// partition splits further.
void refine_both(const ConeGraph &A, const ConeGraph &B, uint64_t *ca, uint64_t *cb) {
    int da = distinct(ca, A.n), db = distinct(cb, B.n);
    for (int round = 0; round < A.n; ++round) {
        uint64_t ta[kMaxN], tb[kMaxN];
        std::copy(ca, ca + A.n, ta);
        std::copy(cb, cb + B.n, tb);
        refine_round(A, ta);
        refine_round(B, tb);
        const int na = distinct(ta, A.n), nb = distinct(tb, B.n);
        std::copy(ta, ta + A.n, ca);
        std::copy(tb, tb + B.n, cb);
        if (na == da && nb == db) break;
        da = na;
        db = nb;
    }
}

bool same_multiset(const uint64_t *ca, const uint64_t *cb, int n) {
    uint64_t sa[kMaxN], sb[kMaxN];
    std::copy(ca, ca + n, sa);
    std::copy(cb, cb + n, sb);
    std::sort(sa, sa + n);
    std::sort(sb, sb + n);
    return std::equal(sa, sa + n, sb);
}

// Search budget per test (tree nodes); a test that runs out answers "not
// isomorphic", which only costs reduction, never correctness.
constexpr int kSearchNodes = 20000;

bool iso_search(const ConeGraph &A, const ConeGraph &B, uint64_t *ca, uint64_t *cb, int depth, int &budget) {
    if (--budget < 0) return false;
    refine_both(A, B, ca, cb);
    if (!same_multiset(ca, cb, A.n)) return false;
    // the smallest non-singleton colour cell of A
    int best = -1, best_count = kMaxN + 1;
    for (int v = 0; v < A.n; ++v) {
        int count = 0;
        for (int w = 0; w < A.n; ++w) count += ca[w] == ca[v];
        if (count > 1 && (count < best_count || (count == best_count && ca[v] < ca[best]))) {
            best = v;
            best_count = count;
        }
    }
    if (best < 0) {  // discrete: the colours define the bijection; check it
        int phi[kMaxN];
        for (int a = 0; a < A.n; ++a) {
            phi[a] = -1;
            for (int b = 0; b < B.n; ++b)
                if (cb[b] == ca[a]) phi[a] = b;
            if (phi[a] < 0 || B.dist[phi[a]] != A.dist[a]) return false;
        }
        for (int a = 0; a < A.n; ++a) {
            uint32_t img = 0;
            for (uint32_t s = A.adj[a]; s; s &= s - 1) {
                const int u = __builtin_ctz(s);
                if (B.w[phi[a]][phi[u]] != A.w[a][u]) return false;
                img |= 1u << phi[u];
            }
            if (img != B.adj[phi[a]]) return false;
        }
        return true;
    }
    const uint64_t cell = ca[best];
    const uint64_t fresh = mix64(cell ^ (0x51afd7ed558ccd1dull * uint64_t(depth + 1)));
    for (int b = 0; b < B.n; ++b) {
        if (cb[b] != cell) continue;
        uint64_t na[kMaxN], nb[kMaxN];
        std::copy(ca, ca + A.n, na);
        std::copy(cb, cb + B.n, nb);
        na[best] = fresh;
        nb[b] = fresh;
        if (iso_search(A, B, na, nb, depth + 1, budget)) return true;
    }
    return false;
}

void initial_colours(const ConeGraph &g, uint64_t *col) {
    for (int v = 0; v < g.n; ++v) col[v] = mix64(uint64_t(g.dist[v]) + 1);
}

// Invariant of a cone: sizes, mixer prefixes and its stable colours.
uint64_t cone_invariant(const Cone &c, const ConeGraph &g, int p) {
    uint64_t col[kMaxN], other[kMaxN];
    initial_colours(g, col);
    std::copy(col, col + g.n, other);
    refine_both(g, g, col, other);
    std::sort(col, col + g.n);
    uint64_t h = mix64(uint64_t(g.n) << 32 | uint32_t(g.m));
    h = mix64(h ^ uint64_t(c.n_in));
    for (int l = 0; l < p; ++l) h = mix64(h ^ uint64_t(c.k[l]) * 0x100000001b3ull);
    for (int v = 0; v < g.n; ++v) h = mix64(h ^ col[v]);
    return h;
}

}  // namespace

bool cones_isomorphic(const Cone &a, const Cone &b, int p) {
    if (a.n != b.n || a.n_in != b.n_in || a.ea.size() != b.ea.size() || a.n_blocks != b.n_blocks) return false;
    for (int l = 0; l < p; ++l)
        if (a.k[l] != b.k[l]) return false;
    const ConeGraph A = cone_graph(a), B = cone_graph(b);
    uint64_t ca[kMaxN], cb[kMaxN];
    initial_colours(A, ca);
    initial_colours(B, cb);
    int budget = kSearchNodes;
    return iso_search(A, B, ca, cb, 0, budget);
}

void cone_classes(const std::vector<const Cone *> &cones, int p, std::vector<int32_t> &class_of) {
    class_of.assign(cones.size(), -1);
    std::unordered_map<uint64_t, std::vector<int32_t>> bucket;  // invariant -> class representatives
    for (size_t i = 0; i < cones.size(); ++i) {
        const uint64_t h = cone_invariant(*cones[i], cone_graph(*cones[i]), p);
        auto &reps = bucket[h];
        for (int32_t r : reps) {
            if (cones_isomorphic(*cones[i], *cones[r], p)) {
                class_of[i] = r;
                break;
            }
        }
        if (class_of[i] < 0) {
            class_of[i] = int32_t(i);
            reps.push_back(int32_t(i));
        }
    }
}

}  // namespace qaoa
