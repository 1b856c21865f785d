// Block merging: shell blocks whose evolutions are related contribute
// equally, and are evolved once.
//
// A cone's term is a sum over its shell blocks (one per vector n of per-class
// counts of shell qubits set to 1, weighted by the product of binomials).
// Three exact relations between blocks are used.
//
// 1. The phase vector.  A shell qubit with value t adds sum_q w_q [z_q != t]
//    over its inner neighbours q; a class of s such qubits with n of them 1
//    adds n W + (s - 2n) sum_q w_q z_q, with W = sum_q w_q.  So up to a
//    constant (a global phase of the block, which leaves its expectation and
//    every derivative unchanged) block n sees the inner cut function
//    C_in(z) + sum_q c_q z_q with c_q = sum_k (s_k - 2 n_k) w_kq: blocks with
//    the same integer vector c evolve identically.
// 2. Symmetries of the inner part.  A block evolves on the inner qubits
//    under C_in(z) + sum_q c_q z_q and the mixers, so a permutation pi of the
//    inner qubits that keeps the inner edges and their weights and every
//    distance from the root edge (hence every layer's mixer set, and the root
//    edge itself, which alone has distance 0) carries block c onto block
//    c o pi^-1 with the qubits relabelled: Z_0 Z_1 is unchanged by it, so
//    both contribute the same to the term and to every derivative (sums over
//    all qubits of a layer) -- Theorem 1's argument (Sec. 3) inside one cone,
//    whenever c o pi^-1 occurs as a phase vector as well.
// 3. The global spin flip.  Flipping every bit leaves any cut value, the
//    mixers, |+>^n and Z_0 Z_1 unchanged; it maps block c onto block -c
//    (C_in(~z) = C_in(z) and sum_q c_q (1 - z_q) = const - sum_q c_q z_q).
//
// Count vectors are grouped by c; generators of the inner graph's
// automorphism group are found by backtracking (with a budget: any set of
// genuine automorphisms gives valid merges); the occurring phase vectors are
// merged into their orbits under that group and c -> -c by union-find, and
// one count vector per orbit is kept with the orbit's total number of shell
// assignments.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "host.hpp"

namespace qaoa {
namespace {

constexpr int64_t kMaxBlocks = int64_t(1) << 16;  // larger block sets keep the plain enumeration
constexpr int kMaxGens = 256;
constexpr int64_t kMaxNodes = 200000;

// The inner part of a cone as a coloured, edge-weighted graph: vertices are
// the inner qubits coloured by their distance from the root edge (so an
// automorphism keeps every layer's mixer set and maps the root edge onto
// itself), edges the inner edges with their weights.
struct InnerGraph {
    int V = 0;
    std::vector<int> colour;          // distance from the root edge
    std::vector<std::vector<int>> w;  // edge weight, 0 = no edge
    std::vector<int> wdeg;            // an invariant for pruning: sum over edges of a weight code
};

InnerGraph inner_graph(const Cone &c) {
    InnerGraph g;
    g.V = c.n_in;
    g.colour.assign(size_t(g.V), 0);
    g.w.assign(size_t(g.V), std::vector<int>(size_t(g.V), 0));
    for (int v = 0; v < c.n_in; ++v) g.colour[v] = c.dist[v];
    for (size_t e = 0; e < c.ea.size(); ++e) {
        const int a = c.ea[e], b = c.eb[e];
        if (a < c.n_in && b < c.n_in) g.w[a][b] = g.w[b][a] = c.ew[e];
    }
    g.wdeg.assign(size_t(g.V), 0);
    for (int v = 0; v < g.V; ++v)
        for (int u = 0; u < g.V; ++u)
            if (g.w[v][u]) g.wdeg[v] += 1 + 64 * (g.w[v][u] + 64);
    return g;
}

// Generators of the inner graph's automorphism group: for base points
// v = 0, 1, ... (the earlier ones fixed) one automorphism per image t of v
// outside the orbit already reached -- a transversal at every level, which
// together generate the whole group.  Each search stops at its first leaf.
struct Enumerator {
    const InnerGraph &g;
    std::vector<int> img, used;
    std::vector<std::vector<int>> gens;  // full vertex permutations
    int64_t nodes = 0;

    explicit Enumerator(const InnerGraph &cg) : g(cg), img(size_t(cg.V), -1), used(size_t(cg.V), 0) {}

    bool fits(int v, int t) const {
        if (used[t] || g.colour[t] != g.colour[v] || g.wdeg[t] != g.wdeg[v]) return false;
        for (int x = 0; x < v; ++x)
            if (g.w[x][v] != g.w[img[x]][t]) return false;
        return true;
    }
    bool extend(int v) {
        if (++nodes > kMaxNodes) return false;
        if (v == g.V) return true;
        for (int t = 0; t < g.V; ++t) {
            if (!fits(v, t)) continue;
            img[v] = t;
            used[t] = 1;
            if (extend(v + 1)) return true;
            used[t] = 0;
            img[v] = -1;
            if (nodes > kMaxNodes) return false;
        }
        return false;
    }
    void run() {
        for (int base = 0; base < g.V; ++base) {
            // orbit of `base` under the generators that fix 0..base-1
            std::vector<char> orbit(size_t(g.V), 0);
            orbit[base] = 1;
            for (bool grown = true; grown;) {
                grown = false;
                for (const auto &pm : gens) {
                    bool fixes = true;
                    for (int x = 0; x < base && fixes; ++x) fixes = pm[x] == x;
                    if (!fixes) continue;
                    for (int x = 0; x < g.V; ++x)
                        if (orbit[x] && !orbit[pm[x]]) {
                            orbit[pm[x]] = 1;
                            grown = true;
                        }
                }
            }
            for (int t = 0; t < g.V; ++t) {
                if (orbit[t] || int(gens.size()) >= kMaxGens) continue;
                std::fill(img.begin(), img.end(), -1);
                std::fill(used.begin(), used.end(), 0);
                bool ok = true;
                for (int x = 0; x < base && ok; ++x) {
                    ok = fits(x, x);
                    img[x] = x;
                    used[x] = 1;
                }
                if (!ok || !fits(base, t)) continue;
                img[base] = t;
                used[t] = 1;
                if (!extend(base + 1)) continue;
                gens.push_back(img);
                // t joins the orbit together with everything the new generator reaches
                for (bool grown = true; grown;) {
                    grown = false;
                    for (int x = 0; x < g.V; ++x)
                        if (orbit[x] && !orbit[img[x]]) {
                            orbit[img[x]] = 1;
                            grown = true;
                        }
                }
            }
        }
    }
};

constexpr int64_t kMaxOrbitNodes = int64_t(1) << 18;  // phase vectors reached by the orbit search

struct VecHash {
    size_t operator()(const std::vector<int32_t> &v) const {
        uint64_t h = 0x9e3779b97f4a7c15ull;
        for (int32_t x : v) {
            h ^= uint64_t(uint32_t(x)) + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
            h *= 0xff51afd7ed558ccdull;
        }
        return size_t(h ^ (h >> 33));
    }
};

int64_t find(std::vector<int64_t> &parent, int64_t x) {
    while (parent[x] != x) x = parent[x] = parent[parent[x]];
    return x;
}

// Everything the merging reads from a cone, in its local labels: the inner
// distances and edges, and per shell class its size and the inner
// neighbours (with weights) of its first member.  Cones with equal keys get
// equal block lists; tree-like cones of one graph share a handful of keys.
std::string structure_key(const Cone &c, const std::vector<int> &cls_of) {
    std::vector<int32_t> k;
    k.push_back(c.n_in);
    k.push_back(int32_t(c.shell_classes.size()));
    for (int q = 0; q < c.n_in; ++q) k.push_back(c.dist[q]);
    for (const auto &cls : c.shell_classes) k.push_back(int32_t(cls.size()));
    for (size_t e = 0; e < c.ea.size(); ++e) {
        int a = c.ea[e], b = c.eb[e];
        if (a < c.n_in && b < c.n_in) {
            k.insert(k.end(), {a, b, c.ew[e]});
            continue;
        }
        if (a < c.n_in) std::swap(a, b);  // a: the shell end
        if (a < c.n_in || b >= c.n_in || c.shell_classes[cls_of[a]][0] != a) continue;
        k.insert(k.end(), {-1 - cls_of[a], b, c.ew[e]});
    }
    std::string out(k.size() * sizeof(int32_t), '\0');
    std::memcpy(&out[0], k.data(), out.size());
    return out;
}

void merge_blocks(Cone &c, int n_in, int ncls);

}  // namespace

struct BlockMemo {
    std::mutex mu;
    std::unordered_map<std::string, std::pair<std::vector<std::vector<uint8_t>>, std::vector<double>>> done;
};

BlockMemo *block_memo_new() { return new BlockMemo(); }
void block_memo_free(BlockMemo *m) { delete m; }

void block_orbits(Cone &c, BlockMemo *memo) {
    c.blk_counts.clear();
    c.blk_weight.clear();
    const int ncls = int(c.shell_classes.size());
    if (ncls == 0 || c.n_blocks < 2 || c.n_blocks > kMaxBlocks) return;
    const int n_in = c.n_in;
    std::string key;
    if (memo) {
        std::vector<int> cls(size_t(c.n), -1);
        for (int k = 0; k < ncls; ++k)
            for (int32_t q : c.shell_classes[k]) cls[q] = k;
        key = structure_key(c, cls);
        std::lock_guard<std::mutex> lk(memo->mu);
        const auto it = memo->done.find(key);
        if (it != memo->done.end()) {
            c.blk_counts = it->second.first;
            c.blk_weight = it->second.second;
            if (!c.blk_counts.empty()) c.n_blocks = int64_t(c.blk_counts.size());
            return;
        }
    }
    merge_blocks(c, n_in, ncls);
    if (memo) {
        std::lock_guard<std::mutex> lk(memo->mu);
        memo->done.emplace(std::move(key), std::make_pair(c.blk_counts, c.blk_weight));
    }
}

namespace {

void merge_blocks(Cone &c, const int n_in, const int ncls) {
    // inner neighbours of each class with their weights (shared by its members)
    std::vector<int> cls_of(size_t(c.n), -1);
    for (int k = 0; k < ncls; ++k)
        for (int32_t q : c.shell_classes[k]) cls_of[q] = k;
    std::vector<std::vector<std::pair<int, int>>> nbr(static_cast<size_t>(ncls));
    for (size_t e = 0; e < c.ea.size(); ++e) {
        int a = c.ea[e], b = c.eb[e];
        if (a < n_in) std::swap(a, b);
        if (a < n_in || b >= n_in) continue;  // inner-inner (shell-shell edges are not kept)
        if (c.shell_classes[cls_of[a]][0] == a) nbr[cls_of[a]].emplace_back(b, c.ew[e]);
    }
    // the phase vector of every count vector, and its number of shell assignments
    std::vector<int64_t> radix(size_t(ncls) + 1, 1);
    for (int k = 0; k < ncls; ++k) radix[k + 1] = radix[k] * int64_t(c.shell_classes[k].size() + 1);
    const int64_t nb = c.n_blocks;
    std::unordered_map<std::vector<int32_t>, int64_t, VecHash> id_of;  // phase vector -> id
    std::vector<std::vector<int32_t>> vec;                             // id -> phase vector
    std::vector<int64_t> first;                                        // id -> first count vector
    std::vector<double> weight;                                        // id -> shell assignments
    std::vector<int32_t> cv(static_cast<size_t>(n_in));
    for (int64_t b = 0; b < nb; ++b) {
        std::fill(cv.begin(), cv.end(), 0);
        double mult = 1.0;
        for (int k = 0; k < ncls; ++k) {
            const int s = int(c.shell_classes[k].size());
            const int nk = int((b / radix[k]) % int64_t(s + 1));
            for (const auto &qw : nbr[k]) cv[qw.first] += (s - 2 * nk) * qw.second;
            double bin = 1.0;  // binomial(s, nk), exact in double for s <= 32
            for (int i = 0; i < nk; ++i) bin = bin * double(s - i) / double(i + 1);
            mult *= bin;
        }
        auto it = id_of.find(cv);
        if (it == id_of.end()) {
            it = id_of.emplace(cv, int64_t(vec.size())).first;
            vec.push_back(cv);
            first.push_back(b);
            weight.push_back(0.0);
        }
        weight[size_t(it->second)] += mult;
    }
    const int64_t nid = int64_t(vec.size());
    // A block's evolution depends on the shell only through c, so a symmetry
    // of the inner part alone (inner edges and weights, distances from the
    // root edge, the root edge) relates block c to block c o pi^-1 whenever
    // that phase vector occurs.  Orbits of the occurring vectors under the
    // inner group: breadth-first search from each along the generators,
    // through vectors that do not occur as well (two occurring vectors of one
    // orbit may only be joined through such), by union-find over all vectors
    // reached; up to kMaxOrbitNodes vectors, beyond which the search stops
    // (every merge made is still valid).
    const InnerGraph gi = inner_graph(c);
    Enumerator ei(gi);
    ei.run();
    std::vector<int64_t> parent(static_cast<size_t>(nid));
    std::iota(parent.begin(), parent.end(), 0);
    std::vector<char> visited(static_cast<size_t>(nid), 0);
    auto node = [&](const std::vector<int32_t> &v) {  // id of v, added if new
        const auto it = id_of.emplace(v, int64_t(vec.size()));
        if (it.second) {
            vec.push_back(v);
            parent.push_back(int64_t(parent.size()));
            visited.push_back(0);
        }
        return it.first->second;
    };
    auto unite = [&](int64_t x, int64_t y) {
        const int64_t ra = find(parent, x), rb = find(parent, y);
        if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
    };
    std::vector<int32_t> img(static_cast<size_t>(n_in));
    std::vector<int64_t> queue;
    for (int64_t i = 0; i < nid && !ei.gens.empty(); ++i) {
        if (visited[i] || int64_t(vec.size()) > kMaxOrbitNodes) continue;
        visited[i] = 1;
        queue.assign(1, i);
        while (!queue.empty()) {
            const int64_t x = queue.back();
            queue.pop_back();
            for (const auto &pi : ei.gens) {
                for (int q = 0; q < n_in; ++q) img[pi[q]] = vec[x][q];
                if (int64_t(vec.size()) > kMaxOrbitNodes && id_of.find(img) == id_of.end()) continue;
                const int64_t y = node(img);
                unite(x, y);
                if (!visited[y]) {
                    visited[y] = 1;
                    queue.push_back(y);
                }
            }
        }
    }
    // the spin flip maps orbits onto orbits, and -c of an occurring c occurs
    for (int64_t i = 0; i < nid; ++i) {
        for (int q = 0; q < n_in; ++q) img[q] = -vec[i][q];
        const auto it = id_of.find(img);
        if (it != id_of.end()) unite(i, it->second);
    }
    std::vector<double> total(static_cast<size_t>(nid), 0.0);
    for (int64_t i = 0; i < nid; ++i) total[find(parent, i)] += weight[i];
    int64_t n_orbits = 0;
    for (int64_t i = 0; i < nid; ++i) n_orbits += find(parent, i) == i;
    if (n_orbits == nb) return;  // nothing merged: keep the class table
    for (int64_t i = 0; i < nid; ++i) {
        if (find(parent, i) != i) continue;
        std::vector<uint8_t> cnt(static_cast<size_t>(ncls));
        for (int k = 0; k < ncls; ++k)
            cnt[k] = uint8_t((first[i] / radix[k]) % int64_t(c.shell_classes[k].size() + 1));
        c.blk_counts.push_back(std::move(cnt));
        c.blk_weight.push_back(total[i]);
    }
    c.n_blocks = int64_t(c.blk_counts.size());
}

}  // namespace
}  // namespace qaoa
