// Edge orbits of the automorphism group of a graph.
//
// The paper computes Aut(G) with an external solver (Sec. 2.6, Sec. 4) and
// then partitions the Hamiltonian terms -- the edges, for MaxCut -- into
// orbits (Sec. 3).  This file is the project's own solver:
//
//  1. colour refinement to the coarsest equitable partition (splitting cells
//     by the number of neighbours in a splitter cell until stable), started
//     from a vertex invariant read off the balls of radius 1..3 around each
//     vertex (cycles near a vertex show up there, so in a graph without
//     symmetry the few vertices on short cycles are told apart before any
//     search);
//  2. an individualisation-refinement search: along a first path of the
//     search tree (individualise the first element of the first smallest
//     non-singleton cell, refine, repeat until discrete) the tree is explored
//     level by level from the deepest, looking under every cell element that
//     is not yet known to be in the base point's orbit for a leaf whose
//     position-wise correspondence with the first leaf is an automorphism;
//     nodes whose refinement trace differs from the first path's are pruned;
//  3. every candidate permutation is verified to map every edge to an edge
//     before it becomes a generator;
//  4. edge orbits by union-find over (edge, image of edge) for every generator.
//
// The order of the group follows from the orbit-stabiliser theorem as the
// product of the base points' orbit sizes.  With a budget on refinement calls
// the search may stop early; the generators found so far are all verified, so
// the orbits are those of a subgroup, which is still a valid reduction.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "host.hpp"

namespace qaoa {
namespace {

struct UnionFind {
    std::vector<int64_t> parent, size;
    explicit UnionFind(int64_t n) : parent(size_t(n)), size(size_t(n), 1) {
        std::iota(parent.begin(), parent.end(), 0);
    }
    int64_t find(int64_t x) {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];
            x = parent[x];
        }
        return x;
    }
    // returns the new root
    int64_t unite(int64_t a, int64_t b) {
        a = find(a);
        b = find(b);
        if (a == b) return a;
        if (size[a] < size[b]) std::swap(a, b);
        parent[b] = a;
        size[a] += size[b];
        return a;
    }
};

// Ordered partition of the vertices: cells are contiguous runs of `lab`;
// a cell is named by its start position.
struct Partition {
    std::vector<int32_t> lab, pos, cell, len;
    int32_t ncells = 0;
};

inline uint64_t hmix(uint64_t h, uint64_t x) {
    x *= 0x9e3779b97f4a7c15ull;
    x ^= x >> 29;
    h ^= x + 0x7f4a7c159e3779b9ull + (h << 6) + (h >> 2);
    return h;
}

class Refiner {
   public:
    explicit Refiner(const Graph &g) : g_(g), cnt_(size_t(g.n), 0), inq_(size_t(g.n), 0) {}

    // A neighbour across an edge of weight w counts as ecode(w): 1 for the
    // unweighted case, a distinct hash per weight otherwise, so the split
    // respects edge colours (Sec. 4: colours = equal weights).
    static uint64_t ecode(int32_t w) {
        return w == 1 ? 1ull : hmix(0x5bd1e9955bd1e995ull, uint64_t(uint32_t(w))) | (1ull << 40);
    }

    // Refines P to the coarsest equitable partition finer than P, starting
    // from the splitter cells in `queue` (consumed).  Each split is one event
    // hash; with `record` the events are appended, with `expect` they are
    // compared and the call returns false at the first difference.
    bool refine(Partition &P, std::vector<int32_t> &queue, std::vector<uint64_t> *record,
                const std::vector<uint64_t> *expect) {
        size_t ev = 0;
        for (int32_t s : queue) inq_[s] = 1;
        size_t head = 0;
        bool ok = true;
        while (head < queue.size()) {
            int32_t S = queue[head++];
            inq_[S] = 0;
            int32_t slen = P.len[S];
            touched_.clear();
            for (int32_t i = S; i < S + slen; ++i) {
                int32_t x = P.lab[i];
                for (int64_t k = g_.off[x]; k < g_.off[x + 1]; ++k) {
                    int32_t y = g_.adj[k];
                    if (cnt_[y] == 0) touched_.push_back(y);
                    cnt_[y] += ecode(g_.ew[g_.eid[k]]);
                }
            }
            keys_.clear();
            for (int32_t y : touched_) keys_.push_back({{P.cell[y], cnt_[y]}, y});
            std::sort(keys_.begin(), keys_.end());
            size_t a = 0;
            while (a < keys_.size() && ok) {
                int32_t X = keys_[a].first.first;
                size_t b = a;
                while (b < keys_.size() && keys_[b].first.first == X) ++b;
                int32_t L = P.len[X];
                int32_t t = int32_t(b - a);
                bool split = (t < L) || (keys_[a].first.second != keys_[b - 1].first.second);
                if (split && L > 1) {
                    uint64_t h = hmix(hmix(hmix(hmix(0, uint64_t(S)), uint64_t(slen)), uint64_t(X)),
                                      uint64_t(L));
                    // move the touched vertices (sorted by count) to the back
                    int32_t back = X + L - t;
                    for (int32_t k = 0; k < t; ++k) {
                        int32_t y = keys_[a + k].second;
                        int32_t py = P.pos[y], tp = back + k;
                        int32_t z = P.lab[tp];
                        P.lab[tp] = y;
                        P.pos[y] = tp;
                        P.lab[py] = z;
                        P.pos[z] = py;
                    }
                    // fragments: [zero-count group], then equal-count runs
                    frag_.clear();
                    if (t < L) frag_.push_back({X, L - t, 0u});
                    for (size_t k = a; k < b;) {
                        size_t r = k;
                        while (r < b && keys_[r].first.second == keys_[k].first.second) ++r;
                        frag_.push_back({back + int32_t(k - a), int32_t(r - k), keys_[k].first.second});
                        k = r;
                    }
                    bool was_in = inq_[X] != 0;
                    size_t largest = 0;
                    for (size_t f = 1; f < frag_.size(); ++f)
                        if (frag_[f].size > frag_[largest].size) largest = f;
                    for (size_t f = 0; f < frag_.size(); ++f) {
                        const Frag &fr = frag_[f];
                        P.len[fr.start] = fr.size;
                        if (f > 0)
                            for (int32_t i = fr.start; i < fr.start + fr.size; ++i) P.cell[P.lab[i]] = fr.start;
                        h = hmix(hmix(h, fr.count), uint64_t(fr.size));
                        bool push = was_in ? (f > 0) : (f != largest);
                        if (push && !inq_[fr.start]) {
                            inq_[fr.start] = 1;
                            queue.push_back(fr.start);
                        }
                    }
                    P.ncells += int32_t(frag_.size()) - 1;
                    if (record) record->push_back(h);
                    if (expect) {
                        if (ev >= expect->size() || (*expect)[ev] != h) ok = false;
                    }
                    ++ev;
                }
                a = b;
            }
            for (int32_t y : touched_) cnt_[y] = 0;
            if (!ok) break;
        }
        for (size_t i = head; i < queue.size(); ++i) inq_[queue[i]] = 0;
        queue.clear();
        if (expect && ok && ev != expect->size()) ok = false;
        return ok;
    }

   private:
    struct Frag {
        int32_t start, size;
        uint64_t count;
    };
    const Graph &g_;
    std::vector<uint64_t> cnt_;
    std::vector<char> inq_;
    std::vector<int32_t> touched_;
    std::vector<std::pair<std::pair<int32_t, uint64_t>, int32_t>> keys_;  // ((cell, count), vertex)
    std::vector<Frag> frag_;
};

// Vertex invariant, from a breadth-first search of radius 1..3 around each
// vertex (stopped once the ball holds more than kBallCap vertices): per
// radius r the number of vertices first reached at distance r, and the edge
// codes summed separately over the edges scanned from distance r - 1 that
// lead back to distance <= r - 1 and over those that reach a vertex at
// distance r already reached from another vertex (both zero in a tree, so
// cycles near a vertex show).  The counts do not depend on the order of the
// search, and an automorphism maps a vertex's balls onto its image's, so
// vertices of one orbit get equal values.
constexpr int kBallRadius = 3;
constexpr int32_t kBallCap = 512;

void ball_invariants(const Graph &g, std::vector<uint64_t> &col) {
    const int32_t n = g.n;
    col.assign(size_t(n), 0);
    std::vector<int32_t> stamp(size_t(n), -1), dist(size_t(n), 0), ball;
    for (int32_t v = 0; v < n; ++v) {
        ball.assign(1, v);
        stamp[v] = v;
        dist[v] = 0;
        uint64_t h = hmix(0x243f6a8885a308d3ull, uint64_t(g.degree(v)));
        size_t frontier = 0;
        for (int r = 1; r <= kBallRadius && int32_t(ball.size()) <= kBallCap; ++r) {
            const size_t end = ball.size();
            uint64_t back = 0, cross = 0;
            for (size_t i = frontier; i < end; ++i) {
                const int32_t x = ball[i];
                for (int64_t k = g.off[x]; k < g.off[x + 1]; ++k) {
                    const int32_t y = g.adj[k];
                    const uint64_t code = Refiner::ecode(g.ew[g.eid[k]]);
                    if (stamp[y] != v) {
                        stamp[y] = v;
                        dist[y] = r;
                        ball.push_back(y);
                    } else if (dist[y] < r) {
                        back += code;
                    } else {
                        cross += code;
                    }
                }
            }
            frontier = end;
            h = hmix(hmix(hmix(h, uint64_t(ball.size() - end)), back), cross);
        }
        col[v] = h;
    }
}

void individualize(Partition &P, int32_t v, std::vector<int32_t> &queue) {
    int32_t X = P.cell[v], L = P.len[X];
    if (L == 1) return;
    int32_t pv = P.pos[v], z = P.lab[X];
    P.lab[X] = v;
    P.pos[v] = X;
    P.lab[pv] = z;
    P.pos[z] = pv;
    P.len[X] = 1;
    P.len[X + 1] = L - 1;
    for (int32_t i = X + 1; i < X + L; ++i) P.cell[P.lab[i]] = X + 1;
    P.ncells += 1;
    queue.push_back(X);
}

class AutSearch {
   public:
    AutSearch(const Graph &g, int64_t budget) : g_(g), budget_(budget), ref_(g), iso_(size_t(g.n), 0) {
        for (int32_t v = 0; v < g.n; ++v) iso_[v] = g.degree(v) == 0;
    }

    void run(std::vector<std::vector<int32_t>> &gens, double &log10_aut, bool &complete) {
        const int32_t n = g_.n;
        log10_aut = 0.0;
        int64_t n_iso = 0;
        for (int32_t v = 0; v < n; ++v) n_iso += iso_[v];
        log10_aut += std::lgamma(double(n_iso) + 1.0) / std::log(10.0);
        if (n == 0) {
            complete = true;
            return;
        }
        // the initial partition: cells of equal ball invariants, ordered by value
        std::vector<uint64_t> col;
        ball_invariants(g_, col);
        Partition P0;
        P0.lab.resize(n);
        P0.pos.resize(n);
        P0.cell.assign(n, 0);
        P0.len.assign(n, 0);
        std::iota(P0.lab.begin(), P0.lab.end(), 0);
        std::sort(P0.lab.begin(), P0.lab.end(), [&](int32_t a, int32_t b) {
            return col[a] != col[b] ? col[a] < col[b] : a < b;
        });
        std::vector<int32_t> queue;
        for (int32_t i = 0; i < n;) {
            int32_t j = i;
            while (j < n && col[P0.lab[j]] == col[P0.lab[i]]) ++j;
            P0.len[i] = j - i;
            for (int32_t k = i; k < j; ++k) {
                P0.pos[P0.lab[k]] = k;
                P0.cell[P0.lab[k]] = i;
            }
            queue.push_back(i);
            ++P0.ncells;
            i = j;
        }
        std::vector<uint64_t> ev;
        ref_.refine(P0, queue, &ev, nullptr);
        path_.push_back(P0);
        // first path
        const double mem_cap = 4.0e8;  // bytes of stored partitions
        for (;;) {
            int32_t t = target_cell(path_.back());
            if (t < 0) break;
            if (double(path_.size() + 1) * 16.0 * n > mem_cap) {
                aborted_ = true;
                break;
            }
            int32_t v = path_.back().lab[t];
            tgt_.push_back(t);
            base_.push_back(v);
            Partition P = path_.back();
            individualize(P, v, queue);
            ev.clear();
            ref_.refine(P, queue, &ev, nullptr);
            events_.push_back(ev);
            path_.push_back(std::move(P));
            ++calls_;
        }
        if (aborted_) {
            complete = false;
            return;
        }
        leaf_ = path_.back().lab;
        depth_ = int32_t(path_.size()) - 1;
        UnionFind uf(n);
        std::vector<char> bad(size_t(n), 0);
        std::vector<int32_t> perm(size_t(n), 0);
        for (int32_t j = depth_ - 1; j >= 0 && !aborted_; --j) {
            const Partition &Pj = path_[j];
            int32_t s = tgt_[j], L = Pj.len[s], v = base_[j];
            std::fill(bad.begin(), bad.end(), 0);
            for (int32_t idx = s; idx < s + L; ++idx) {
                int32_t w = Pj.lab[idx];
                if (w == v) continue;
                int64_t rw = uf.find(w), rv = uf.find(v);
                if (rw == rv || bad[rw]) continue;
                bool found = explore(Pj, w, j, perm);
                if (aborted_) break;
                if (found) {
                    gens.push_back(perm);
                    for (int32_t x = 0; x < n; ++x) {
                        int64_t ra = uf.find(x), rb = uf.find(perm[x]);
                        if (ra == rb) continue;
                        char b = bad[ra] | bad[rb];
                        int64_t r = uf.unite(ra, rb);
                        bad[r] = b;
                    }
                } else {
                    bad[uf.find(w)] = 1;
                }
            }
            if (!aborted_) log10_aut += std::log10(double(uf.size[uf.find(v)]));
        }
        complete = !aborted_;
    }

   private:
    int32_t target_cell(const Partition &P) const {
        int32_t best = -1, bestL = 0;
        for (int32_t i = 0; i < g_.n;) {
            int32_t L = P.len[i];
            if (L > 1 && !iso_[P.lab[i]] && (best < 0 || L < bestL)) {
                best = i;
                bestL = L;
            }
            i += L;
        }
        return best;
    }

    bool verify(const std::vector<int32_t> &perm) const {
        for (int64_t e = 0; e < g_.m; ++e) {
            const int64_t f = find_edge(g_, perm[g_.eu[e]], perm[g_.ev[e]]);
            if (f < 0 || g_.ew[f] != g_.ew[e]) return false;
        }
        return true;
    }

    // Looks under (Pp, individualise w) for a leaf equivalent to the first leaf.
    bool explore(const Partition &Pp, int32_t w, int32_t j, std::vector<int32_t> &perm) {
        if (++calls_ > budget_) {
            aborted_ = true;
            return false;
        }
        Partition P = Pp;
        std::vector<int32_t> queue;
        individualize(P, w, queue);
        if (!ref_.refine(P, queue, nullptr, &events_[j])) return false;
        const Partition &ref = path_[j + 1];
        if (P.ncells != ref.ncells) return false;
        int32_t t = target_cell(P);
        if (t < 0) {
            if (j + 1 != depth_) return false;
            for (int32_t x = 0; x < g_.n; ++x) perm[x] = x;
            for (int32_t q = 0; q < g_.n; ++q)
                if (!iso_[leaf_[q]]) perm[leaf_[q]] = P.lab[q];
            if (take_fault(QAOA_FAULT_GENERATOR)) {
                // injected corruption: exchange the images of an edge's endpoints'
                // first non-neighbour pair so that the candidate is not an automorphism
                for (int64_t e = 0; e < g_.m; ++e) {
                    const int32_t a = g_.eu[e];
                    int32_t b = -1;
                    for (int32_t y = 0; y < g_.n; ++y)
                        if (y != a && find_edge(g_, a, y) < 0 && g_.degree(y) > 0) {
                            b = y;
                            break;
                        }
                    if (b >= 0) {
                        std::swap(perm[a], perm[b]);
                        break;
                    }
                }
            }
            return verify(perm);
        }
        if (j + 1 >= depth_ || t != tgt_[j + 1] || P.len[t] != ref.len[t]) return false;
        int32_t L = P.len[t];
        for (int32_t idx = t; idx < t + L; ++idx) {
            if (explore(P, P.lab[idx], j + 1, perm)) return true;
            if (aborted_) return false;
        }
        return false;
    }

    const Graph &g_;
    int64_t budget_;
    int64_t calls_ = 0;
    bool aborted_ = false;
    Refiner ref_;
    std::vector<char> iso_;
    std::vector<Partition> path_;
    std::vector<int32_t> tgt_, base_, leaf_;
    std::vector<std::vector<uint64_t>> events_;
    int32_t depth_ = 0;
};

}  // namespace

void trivial_orbits(const Graph &g, OrbitResult &out) {
    out.orbit_id.resize(size_t(g.m));
    std::iota(out.orbit_id.begin(), out.orbit_id.end(), 0);
    out.n_orbits = g.m;
    out.n_generators = 0;
    out.log10_aut = 0.0;
    out.complete = true;
}

void edge_orbits(const Graph &g, int64_t budget, OrbitResult &out) {
    std::vector<std::vector<int32_t>> gens;
    AutSearch s(g, budget > 0 ? budget : 2000000);
    double l10 = 0.0;
    bool complete = true;
    s.run(gens, l10, complete);
    UnionFind uf(g.m);
    for (const auto &gam : gens) {
        for (int64_t e = 0; e < g.m; ++e) {
            int64_t f = find_edge(g, gam[g.eu[e]], gam[g.ev[e]]);
            uf.unite(e, f);  // f >= 0: every generator was verified
        }
    }
    out.orbit_id.assign(size_t(g.m), -1);
    std::vector<int64_t> rep_of_root(size_t(g.m), -1);
    int64_t norb = 0;
    for (int64_t e = 0; e < g.m; ++e) {
        int64_t r = uf.find(e);
        if (rep_of_root[r] < 0) {
            rep_of_root[r] = e;
            ++norb;
        }
        out.orbit_id[e] = int32_t(rep_of_root[r]);
    }
    out.n_orbits = norb;
    out.n_generators = int64_t(gens.size());
    out.log10_aut = l10;
    out.complete = complete;
}

}  // namespace qaoa
