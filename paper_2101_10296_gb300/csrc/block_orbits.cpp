// Block orbits: shell blocks related by a symmetry of the cone contribute
// equally.
//
// A cone's term is a sum over its shell blocks (one per vector of per-class
// counts of shell qubits set to 1, weighted by the product of binomials).  A
// permutation of the cone's qubits that maps edges onto edges of the same
// weight, keeps every distance from the root edge and maps the root edge
// onto itself carries the evolution of block b onto that of its image, with
// the inner qubits relabelled: Z_0 Z_1, the cut value C and the mixers are
// all unchanged by it, so the block's share of the term and of every
// derivative (sums over all qubits of a layer) is the same -- Theorem 1's
// argument (Sec. 3) inside one cone.  On shell classes such a permutation
// acts as a permutation of classes of equal size with equal neighbourhoods'
// images, i.e. as an automorphism of the small "class graph": the inner
// qubits plus one vertex per class, joined to the class's inner neighbours.
// Generators of its automorphism group are found by backtracking (with a
// budget: any set of genuine automorphisms gives valid merges), blocks are
// merged along them by union-find, and one block per orbit is kept with the
// orbit's total multiplicity.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

#include "host.hpp"

namespace qaoa {
namespace {

constexpr int64_t kMaxBlocks = int64_t(1) << 16;  // larger block sets keep the plain enumeration
constexpr int kMaxGens = 256;
constexpr int64_t kMaxNodes = 200000;

struct ClassGraph {
    int V = 0, n_in = 0;
    std::vector<int> colour;             // inner: distance; class: 1000 + size
    std::vector<std::vector<int>> w;     // edge weight, 0 = no edge
    std::vector<int> wdeg;               // sorted-signature proxy: sum over edges of (weight code)
};

ClassGraph class_graph(const Cone &c) {
    ClassGraph g;
    g.n_in = c.n_in;
    const int ncls = int(c.shell_classes.size());
    g.V = c.n_in + ncls;
    g.colour.assign(size_t(g.V), 0);
    g.w.assign(size_t(g.V), std::vector<int>(size_t(g.V), 0));
    for (int v = 0; v < c.n_in; ++v) g.colour[v] = c.dist[v];
    std::vector<int> cls_of(size_t(c.n), -1);
    for (int k = 0; k < ncls; ++k) {
        g.colour[c.n_in + k] = 1000 + int(c.shell_classes[k].size());
        for (int32_t q : c.shell_classes[k]) cls_of[q] = k;
    }
    for (size_t e = 0; e < c.ea.size(); ++e) {
        int a = c.ea[e], b = c.eb[e];
        const int w = c.ew[e];
        // a shell endpoint stands for its class (all members share neighbours and weights)
        if (a >= c.n_in) a = c.n_in + cls_of[a];
        if (b >= c.n_in) b = c.n_in + cls_of[b];
        g.w[a][b] = g.w[b][a] = w;
    }
    g.wdeg.assign(size_t(g.V), 0);
    for (int v = 0; v < g.V; ++v)
        for (int u = 0; u < g.V; ++u)
            if (g.w[v][u]) g.wdeg[v] += 1 + 64 * (g.w[v][u] + 64);
    return g;
}

// Generators of the class graph's automorphism group: for base points
// v = 0, 1, ... (the earlier ones fixed) one automorphism per image t of v
// outside the orbit already reached -- a transversal at every level, which
// together generate the whole group.  Each search stops at its first leaf.
struct Enumerator {
    const ClassGraph &g;
    std::vector<int> img, used;
    std::vector<std::vector<int>> gens;  // full vertex permutations
    int64_t nodes = 0;

    explicit Enumerator(const ClassGraph &cg) : g(cg), img(size_t(cg.V), -1), used(size_t(cg.V), 0) {}

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

int64_t find(std::vector<int64_t> &parent, int64_t x) {
    while (parent[x] != x) x = parent[x] = parent[parent[x]];
    return x;
}

}  // namespace

void block_orbits(Cone &c) {
    c.blk_counts.clear();
    c.blk_weight.clear();
    const int ncls = int(c.shell_classes.size());
    if (ncls == 0 || c.n_blocks < 2 || c.n_blocks > kMaxBlocks) return;
    const ClassGraph g = class_graph(c);
    Enumerator en(g);
    en.run();
    // their action on the classes; those that move no class act trivially on blocks
    std::vector<std::vector<int>> perms;
    for (const auto &a : en.gens) {
        std::vector<int> pm(static_cast<size_t>(ncls));
        bool moves = false;
        for (int k = 0; k < ncls; ++k) {
            pm[k] = a[g.n_in + k] - g.n_in;
            moves |= pm[k] != k;
        }
        if (moves) perms.push_back(pm);
    }
    if (perms.empty()) return;
    // blocks as mixed-radix numbers, least significant class first (the device order)
    std::vector<int64_t> radix(size_t(ncls) + 1, 1);
    for (int k = 0; k < ncls; ++k) radix[k + 1] = radix[k] * int64_t(c.shell_classes[k].size() + 1);
    const int64_t nb = c.n_blocks;
    std::vector<int64_t> parent(static_cast<size_t>(nb));
    std::iota(parent.begin(), parent.end(), 0);
    std::vector<int> digit(static_cast<size_t>(ncls));
    for (int64_t b = 0; b < nb; ++b) {
        for (int k = 0; k < ncls; ++k) digit[k] = int((b / radix[k]) % int64_t(c.shell_classes[k].size() + 1));
        for (const auto &pm : perms) {
            int64_t image = 0;
            for (int k = 0; k < ncls; ++k) image += int64_t(digit[k]) * radix[pm[k]];
            const int64_t ra = find(parent, b), rb = find(parent, image);
            if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
        }
    }
    std::vector<int64_t> size(size_t(nb), 0);
    for (int64_t b = 0; b < nb; ++b) size[find(parent, b)]++;
    for (int64_t b = 0; b < nb; ++b) {
        if (find(parent, b) != b) continue;
        std::vector<uint8_t> cnt(static_cast<size_t>(ncls));
        double mult = 1.0;
        for (int k = 0; k < ncls; ++k) {
            const int s = int(c.shell_classes[k].size());
            const int nk = int((b / radix[k]) % int64_t(s + 1));
            cnt[k] = uint8_t(nk);
            double bin = 1.0;  // binomial(s, nk), exact in double for s <= 32
            for (int i = 0; i < nk; ++i) bin = bin * double(s - i) / double(i + 1);
            mult *= bin;
        }
        c.blk_counts.push_back(std::move(cnt));
        c.blk_weight.push_back(mult * double(size[b]));
    }
    c.n_blocks = int64_t(c.blk_counts.size());
}

}  // namespace qaoa
