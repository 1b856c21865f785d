// Plan construction (host only): validation, edge orbits, reverse causal
// cones, and the host-side C-ABI queries.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host.hpp"

namespace qaoa {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

static std::atomic<int32_t> g_faults[3];

bool take_fault(int kind) {
    if (kind < 1 || kind > 2) return false;
    int32_t v = g_faults[kind].load();
    while (v > 0)
        if (g_faults[kind].compare_exchange_weak(v, v - 1)) return true;
    return false;
}

// Reverse causal cone of edge e (Sec. 2.3): the operator Z_u Z_v conjugated
// by the last layer's mixer stays on {u, v}; each phase layer adds the
// qubits of every term meeting the current support, so after p layers the
// support is the ball of radius p around the edge.  Mixers of layer l only
// matter on qubits within distance p-l, and the terms that matter are the
// edges with an endpoint within distance p-1.
int extract_cone(const Graph &g, int64_t e, int32_t p, bool full_cone, bool shell_plain, int32_t max_qubits,
                 std::vector<int32_t> &dist, Cone &c, std::string &err) {
    const int32_t u = g.eu[e], v = g.ev[e];
    std::vector<int32_t> ball{u, v};
    dist[u] = 0;
    dist[v] = 0;
    size_t lo = 0;
    for (int32_t d = 1; d <= p; ++d) {
        size_t hi = ball.size();
        for (size_t i = lo; i < hi; ++i) {
            int32_t x = ball[i];
            for (int64_t k = g.off[x]; k < g.off[x + 1]; ++k) {
                int32_t y = g.adj[k];
                if (dist[y] < 0) {
                    dist[y] = d;
                    ball.push_back(y);
                }
            }
        }
        lo = hi;
    }
    auto restore = [&]() {
        for (int32_t x : ball) dist[x] = -1;
    };
    if (int32_t(ball.size()) > max_qubits) {
        char buf[160];
        snprintf(buf, sizeof buf, "cone of edge %lld has %zu qubits > cap %d", (long long)e, ball.size(),
                 max_qubits);
        err = buf;
        restore();
        return QAOA_E_CONE_TOO_LARGE;
    }
    std::sort(ball.begin() + 2, ball.end(), [&](int32_t a, int32_t b) {
        return dist[a] != dist[b] ? dist[a] < dist[b] : a < b;
    });
    c.n = int32_t(ball.size());
    c.verts = ball;
    c.dist.resize(ball.size());
    for (size_t i = 0; i < ball.size(); ++i) c.dist[i] = dist[ball[i]];
    // local index by binary search over (dist, id) order for i >= 2
    auto local = [&](int32_t y) -> int32_t {
        if (y == u) return 0;
        if (y == v) return 1;
        auto it = std::lower_bound(ball.begin() + 2, ball.end(), y, [&](int32_t a, int32_t b) {
            return dist[a] != dist[b] ? dist[a] < dist[b] : a < b;
        });
        return int32_t(it - ball.begin());
    };
    std::vector<std::pair<std::pair<int32_t, int32_t>, int32_t>> le;  // ((a, b), weight)
    for (size_t i = 0; i < ball.size(); ++i) {
        int32_t x = ball[i];
        if (dist[x] > p - 1) continue;
        for (int64_t k = g.off[x]; k < g.off[x + 1]; ++k) {
            int32_t y = g.adj[k];
            if (dist[y] < 0) continue;
            if (dist[y] <= p - 1 && y < x) continue;  // inner-inner edge: add once
            int32_t a = int32_t(i), b = local(y);
            le.push_back({{std::min(a, b), std::max(a, b)}, g.ew[g.eid[k]]});
        }
    }
    std::sort(le.begin(), le.end());
    restore();
    // an edge of weight w takes |w| bits of the 64-bit cut word
    size_t bits = 0;
    for (const auto &x : le) bits += size_t(x.second < 0 ? -x.second : x.second);
    if (bits > size_t(QAOA_MAX_CONE_EDGES)) {
        char buf[160];
        if (bits == le.size())
            snprintf(buf, sizeof buf, "cone of edge %lld has %zu edges > cap %d", (long long)e, le.size(),
                     QAOA_MAX_CONE_EDGES);
        else
            snprintf(buf, sizeof buf, "cone of edge %lld has %zu edges of total |weight| %zu > cap %d",
                     (long long)e, le.size(), bits, QAOA_MAX_CONE_EDGES);
        err = buf;
        return QAOA_E_CONE_TOO_LARGE;
    }
    c.ea.resize(le.size());
    c.eb.resize(le.size());
    c.ew.resize(le.size());
    for (size_t i = 0; i < le.size(); ++i) {
        c.ea[i] = le[i].first.first;
        c.eb[i] = le[i].first.second;
        c.ew[i] = le[i].second;
    }
    int32_t n_in = 0;
    for (int32_t d : c.dist) n_in += (d <= p - 1);
    c.n_in = full_cone ? c.n : n_in;
    for (int32_t l = 0; l < QAOA_MAX_P; ++l) {
        int32_t k = 0;
        if (l < p) {
            for (int32_t d : c.dist) k += (d <= p - 1 - l);
        }
        c.k[l] = full_cone ? (l < p ? c.n : 0) : k;
    }
    // Shell classes.  A shell qubit (distance p) is never mixed and meets the
    // phases only through its cone edges, all of which go to inner qubits; two
    // shell qubits with the same inner neighbours (and edge weights) can be
    // exchanged without changing any cut value, so an inner block's evolution
    // depends on the shell assignment only through how many qubits of each
    // class are 1.
    c.shell_classes.clear();
    c.n_blocks = 1;
    if (c.n_in < c.n) {
        std::vector<std::vector<std::pair<int32_t, int32_t>>> nb(size_t(c.n));  // (inner neighbour, weight)
        for (size_t i = 0; i < c.ea.size(); ++i) {
            const int32_t a = c.ea[i], b = c.eb[i];
            if (a >= c.n_in && b < c.n_in) nb[a].emplace_back(b, c.ew[i]);
            if (b >= c.n_in && a < c.n_in) nb[b].emplace_back(a, c.ew[i]);
        }
        for (auto &x : nb) std::sort(x.begin(), x.end());
        for (int32_t q = c.n_in; q < c.n; ++q) {
            bool placed = false;
            if (!shell_plain) {
                for (auto &cls : c.shell_classes) {
                    if (nb[cls[0]] == nb[q]) {
                        cls.push_back(q);
                        placed = true;
                        break;
                    }
                }
            }
            if (!placed) c.shell_classes.push_back({q});
        }
        for (auto &cls : c.shell_classes) c.n_blocks *= int64_t(cls.size()) + 1;
    }
    return QAOA_OK;
}

template <class F>
static void parallel_for(int64_t count, F fn) {
    int64_t nt = std::min<int64_t>(std::max(1u, std::thread::hardware_concurrency()), 16);
    nt = std::min(nt, count);
    if (nt <= 1) {
        for (int64_t i = 0; i < count; ++i) fn(i, 0);
        return;
    }
    std::vector<std::thread> th;
    std::atomic_int64_t next{0};
    for (int64_t t = 0; t < nt; ++t) {
        th.emplace_back([&, t]() {
            for (;;) {
                int64_t i = next.fetch_add(1);
                if (i >= count) break;
                fn(i, int(t));
            }
        });
    }
    for (auto &x : th) x.join();
}

}  // namespace qaoa

using namespace qaoa;

extern "C" void qaoa_device_release(qaoa_plan *plan);  // defined in the CUDA unit

extern "C" const char *qaoa_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *qaoa_version(void) { return "qaoa-gb300 0.1 (sm_103a)"; }

extern "C" int qaoa_plan_graphs(int32_t n_graphs, const int32_t *n_vertices, const int64_t *edge_offsets,
                                const int32_t *edges, int32_t p, uint32_t flags, int32_t max_cone_qubits,
                                int64_t search_budget, qaoa_plan **out) {
    return qaoa_plan_graphs_weighted(n_graphs, n_vertices, edge_offsets, edges, nullptr, p, flags, max_cone_qubits,
                                     search_budget, out);
}

extern "C" int qaoa_plan_graphs_weighted(int32_t n_graphs, const int32_t *n_vertices, const int64_t *edge_offsets,
                                         const int32_t *edges, const int32_t *weights, int32_t p, uint32_t flags,
                                         int32_t max_cone_qubits, int64_t search_budget, qaoa_plan **out) {
    g_last_error.clear();
    if (!out) {
        set_error("out is NULL");
        return QAOA_E_INVALID;
    }
    *out = nullptr;
    if (n_graphs < 1 || !n_vertices || !edge_offsets) {
        set_error("need n_graphs >= 1 and non-NULL n_vertices / edge_offsets");
        return QAOA_E_INVALID;
    }
    if (p < 1 || p > QAOA_MAX_P) {
        set_error("p must be in [1, QAOA_MAX_P]");
        return QAOA_E_INVALID;
    }
    if (flags & ~uint32_t(QAOA_ORBITS | QAOA_FULL_CONE | QAOA_SHELL_PLAIN | QAOA_BIG_GENERAL | QAOA_CONE_CLASSES |
                            QAOA_BLOCK_PLAIN)) {
        set_error("unknown flag bits");
        return QAOA_E_INVALID;
    }
    if (max_cone_qubits == 0) max_cone_qubits = QAOA_MAX_CONE_QUBITS;
    if (max_cone_qubits < 2 || max_cone_qubits > QAOA_MAX_CONE_QUBITS) {
        set_error("max_cone_qubits must be in [2, QAOA_MAX_CONE_QUBITS]");
        return QAOA_E_INVALID;
    }
    if (edge_offsets[0] != 0) {
        set_error("edge_offsets[0] must be 0");
        return QAOA_E_INVALID;
    }
    for (int32_t g = 0; g < n_graphs; ++g) {
        if (edge_offsets[g + 1] < edge_offsets[g] || n_vertices[g] < 0) {
            set_error("edge_offsets must be non-decreasing and n_vertices >= 0");
            return QAOA_E_INVALID;
        }
    }
    if (edge_offsets[n_graphs] > 0 && !edges) {
        set_error("edges is NULL");
        return QAOA_E_INVALID;
    }
    qaoa_plan *pl = new (std::nothrow) qaoa_plan;
    if (!pl) {
        set_error("host allocation failed");
        return QAOA_E_OOM;
    }
    try {
        pl->p = p;
        pl->flags = flags;
        pl->n_graphs = n_graphs;
        pl->n_vertices.assign(n_vertices, n_vertices + n_graphs);
        pl->n_edges.resize(n_graphs);
        pl->weight_sum.resize(n_graphs);
        std::vector<Graph> graphs(n_graphs);
        for (int32_t g = 0; g < n_graphs; ++g) {
            std::string err;
            int64_t m = edge_offsets[g + 1] - edge_offsets[g];
            int rc = build_graph(n_vertices[g], m, edges + 2 * edge_offsets[g],
                                 weights ? weights + edge_offsets[g] : nullptr, graphs[g], err);
            if (rc != QAOA_OK) {
                set_error("graph " + std::to_string(g) + ": " + err);
                delete pl;
                return rc;
            }
            pl->n_edges[g] = m;
            pl->weight_sum[g] = 0;
            for (int32_t w : graphs[g].ew) {
                pl->weight_sum[g] += w;
                pl->weighted |= w != 1;
            }
        }
        auto t0 = std::chrono::steady_clock::now();
        pl->orbits.resize(n_graphs);
        parallel_for(n_graphs, [&](int64_t g, int) {
            if (flags & QAOA_ORBITS)
                edge_orbits(graphs[g], search_budget, pl->orbits[g]);
            else
                trivial_orbits(graphs[g], pl->orbits[g]);
        });
        auto t1 = std::chrono::steady_clock::now();
        // representatives: smallest edge index of each orbit, in edge order
        std::vector<std::pair<int32_t, int64_t>> reps;
        std::vector<std::vector<int32_t>> size_of(n_graphs);
        for (int32_t g = 0; g < n_graphs; ++g) {
            const auto &oid = pl->orbits[g].orbit_id;
            size_of[g].assign(oid.size(), 0);
            for (int32_t r : oid) size_of[g][r]++;
            for (int64_t e = 0; e < int64_t(oid.size()); ++e)
                if (oid[e] == e) reps.emplace_back(g, e);
        }
        pl->cones.resize(reps.size());
        std::vector<std::vector<int32_t>> scratch(16);
        std::vector<int> rcs(reps.size(), QAOA_OK);
        std::vector<std::string> errs(16);
        parallel_for(int64_t(reps.size()), [&](int64_t i, int t) {
            int32_t g = reps[i].first;
            auto &dist = scratch[t];
            if (int32_t(dist.size()) < graphs[g].n) dist.assign(graphs[g].n, -1);
            Cone &c = pl->cones[i];
            c.graph = g;
            c.edge = reps[i].second;
            c.weight = size_of[g][reps[i].second] * graphs[g].ew[reps[i].second];  // orbit size x edge weight
            rcs[i] = extract_cone(graphs[g], c.edge, p, (flags & QAOA_FULL_CONE) != 0,
                                  (flags & QAOA_SHELL_PLAIN) != 0, max_cone_qubits, dist, c, errs[t]);
        });
        for (size_t i = 0; i < reps.size(); ++i) {
            if (rcs[i] != QAOA_OK) {
                // recompute the message deterministically for the first failing cone
                std::vector<int32_t> dist(graphs[reps[i].first].n, -1);
                Cone c;
                std::string err;
                extract_cone(graphs[reps[i].first], reps[i].second, p, (flags & QAOA_FULL_CONE) != 0,
                             (flags & QAOA_SHELL_PLAIN) != 0, max_cone_qubits, dist, c, err);
                set_error("graph " + std::to_string(reps[i].first) + ": " + err);
                int rc = rcs[i];
                delete pl;
                return rc;
            }
        }
        // cone classes: per graph, one cone per isomorphism class of its cones,
        // weighted by the class's total orbit size
        pl->cone_class.resize(n_graphs);
        pl->n_classes.assign(n_graphs, 0);
        std::vector<int64_t> first(n_graphs + 1, 0);  // graph g's cones: [first[g], first[g+1])
        for (const Cone &c : pl->cones) first[c.graph + 1]++;
        for (int32_t g = 0; g < n_graphs; ++g) first[g + 1] += first[g];
        std::vector<std::vector<int32_t>> class_of(n_graphs);
        if (flags & QAOA_CONE_CLASSES) {
            parallel_for(n_graphs, [&](int64_t g, int) {
                std::vector<const Cone *> list;
                for (int64_t i = first[g]; i < first[g + 1]; ++i) list.push_back(&pl->cones[i]);
                cone_classes(list, p, class_of[g]);
            });
        }
        std::vector<Cone> kept;
        std::vector<int64_t> rep_edge_of_cone(pl->cones.size());
        for (int32_t g = 0; g < n_graphs; ++g) {
            for (int64_t i = first[g]; i < first[g + 1]; ++i) {
                const int64_t r = (flags & QAOA_CONE_CLASSES) ? first[g] + class_of[g][i - first[g]] : i;
                rep_edge_of_cone[i] = pl->cones[r].edge;
            }
            std::unordered_map<int64_t, size_t> slot;  // class representative's edge -> kept index
            for (int64_t i = first[g]; i < first[g + 1]; ++i) {
                auto it = slot.find(rep_edge_of_cone[i]);
                if (it == slot.end()) {
                    slot.emplace(rep_edge_of_cone[i], kept.size());
                    kept.push_back(pl->cones[i]);
                } else {
                    kept[it->second].weight += pl->cones[i].weight;
                }
            }
            pl->n_classes[g] = int64_t(slot.size());
            // edge -> its orbit's representative cone -> that cone's class representative
            std::unordered_map<int64_t, int64_t> cone_of_edge;
            for (int64_t i = first[g]; i < first[g + 1]; ++i) cone_of_edge[pl->cones[i].edge] = i;
            const auto &oid = pl->orbits[g].orbit_id;
            pl->cone_class[g].resize(oid.size());
            for (size_t e = 0; e < oid.size(); ++e)
                pl->cone_class[g][e] = int32_t(rep_edge_of_cone[cone_of_edge[oid[e]]]);
        }
        pl->cones.swap(kept);
        // block merging: shell blocks that contribute equally (phase vectors,
        // symmetries of the inner part, the global spin flip)
        if (!(flags & (QAOA_SHELL_PLAIN | QAOA_BLOCK_PLAIN))) {
            // one memo per worker thread (parallel_for runs at most 16): no lock contention
            std::vector<std::unique_ptr<BlockMemo, void (*)(BlockMemo *)>> memo;
            for (int t = 0; t < 16; ++t) memo.emplace_back(block_memo_new(), block_memo_free);
            parallel_for(int64_t(pl->cones.size()),
                         [&](int64_t i, int t) { block_orbits(pl->cones[i], memo[size_t(t)].get()); });
        }
        auto t2 = std::chrono::steady_clock::now();
        pl->t_orbits = std::chrono::duration<double>(t1 - t0).count();
        pl->t_cones = std::chrono::duration<double>(t2 - t1).count();
    } catch (const std::bad_alloc &) {
        delete pl;
        set_error("host allocation failed");
        return QAOA_E_OOM;
    }
    *out = pl;
    return QAOA_OK;
}

extern "C" int qaoa_plan_graph(int32_t n_vertices, int64_t n_edges, const int32_t *edges, int32_t p,
                               uint32_t flags, int32_t max_cone_qubits, int64_t search_budget, qaoa_plan **out) {
    if (n_edges < 0) {
        set_error("n_edges < 0");
        return QAOA_E_INVALID;
    }
    int64_t off[2] = {0, n_edges};
    return qaoa_plan_graphs(1, &n_vertices, off, edges, p, flags, max_cone_qubits, search_budget, out);
}

extern "C" void qaoa_plan_free(qaoa_plan *plan) {
    if (!plan) return;
    qaoa_device_release(plan);
    delete plan;
}

extern "C" int qaoa_plan_cone_classes(const qaoa_plan *plan, int32_t graph, int32_t *class_id, int64_t *n_classes) {
    if (!plan || graph < 0 || graph >= plan->n_graphs) {
        set_error("bad plan or graph index");
        return QAOA_E_INVALID;
    }
    const auto &cc = plan->cone_class[graph];
    if (class_id) std::copy(cc.begin(), cc.end(), class_id);
    if (n_classes) *n_classes = plan->n_classes[graph];
    return QAOA_OK;
}

extern "C" int qaoa_plan_orbits(const qaoa_plan *plan, int32_t graph, int32_t *orbit_id, int64_t *n_orbits,
                                double *log10_aut, int32_t *complete) {
    if (!plan || graph < 0 || graph >= plan->n_graphs) {
        set_error("bad plan or graph index");
        return QAOA_E_INVALID;
    }
    const OrbitResult &o = plan->orbits[graph];
    if (orbit_id) std::copy(o.orbit_id.begin(), o.orbit_id.end(), orbit_id);
    if (n_orbits) *n_orbits = o.n_orbits;
    if (log10_aut) *log10_aut = o.log10_aut;
    if (complete) *complete = o.complete ? 1 : 0;
    return QAOA_OK;
}

extern "C" int qaoa_plan_reps(const qaoa_plan *plan, int32_t *graph, int64_t *edge, int32_t *weight,
                              int32_t *n_qubits, int32_t *n_inner, int32_t *n_cone_edges,
                              int32_t *mix_qubits) {
    if (!plan) {
        set_error("plan is NULL");
        return QAOA_E_INVALID;
    }
    for (size_t i = 0; i < plan->cones.size(); ++i) {
        const Cone &c = plan->cones[i];
        if (graph) graph[i] = c.graph;
        if (edge) edge[i] = c.edge;
        if (weight) weight[i] = c.weight;
        if (n_qubits) n_qubits[i] = c.n;
        if (n_inner) n_inner[i] = c.n_in;
        if (n_cone_edges) n_cone_edges[i] = int32_t(c.ea.size());
        if (mix_qubits)
            for (int32_t l = 0; l < plan->p; ++l) mix_qubits[i * plan->p + l] = c.k[l];
    }
    return QAOA_OK;
}

extern "C" int qaoa_plan_cone(const qaoa_plan *plan, int64_t rep, int32_t *verts, int32_t *dist,
                              int32_t *cone_edges) {
    if (!plan || rep < 0 || rep >= int64_t(plan->cones.size())) {
        set_error("bad plan or representative index");
        return QAOA_E_INVALID;
    }
    const Cone &c = plan->cones[rep];
    if (verts) std::copy(c.verts.begin(), c.verts.end(), verts);
    if (dist) std::copy(c.dist.begin(), c.dist.end(), dist);
    if (cone_edges)
        for (size_t i = 0; i < c.ea.size(); ++i) {
            cone_edges[2 * i] = c.ea[i];
            cone_edges[2 * i + 1] = c.eb[i];
        }
    return QAOA_OK;
}

extern "C" int qaoa_plan_cone_weights(const qaoa_plan *plan, int64_t rep, int32_t *weights) {
    if (!plan || rep < 0 || rep >= int64_t(plan->cones.size()) || !weights) {
        set_error("bad plan, representative index or NULL weights");
        return QAOA_E_INVALID;
    }
    const Cone &c = plan->cones[size_t(rep)];
    std::copy(c.ew.begin(), c.ew.end(), weights);
    return QAOA_OK;
}

extern "C" int qaoa_edge_orbits(int32_t n_vertices, int64_t n_edges, const int32_t *edges, int64_t search_budget,
                                int32_t *orbit_id, int64_t *n_orbits, int64_t *n_generators, double *log10_aut,
                                int32_t *complete) {
    g_last_error.clear();
    Graph g;
    std::string err;
    int rc = build_graph(n_vertices, n_edges, edges, nullptr, g, err);
    if (rc != QAOA_OK) {
        set_error(err);
        return rc;
    }
    OrbitResult o;
    try {
        edge_orbits(g, search_budget, o);
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return QAOA_E_OOM;
    }
    if (orbit_id) std::copy(o.orbit_id.begin(), o.orbit_id.end(), orbit_id);
    if (n_orbits) *n_orbits = o.n_orbits;
    if (n_generators) *n_generators = o.n_generators;
    if (log10_aut) *log10_aut = o.log10_aut;
    if (complete) *complete = o.complete ? 1 : 0;
    return QAOA_OK;
}

extern "C" int qaoa_plan_shell(const qaoa_plan *plan, int64_t rep, int32_t *class_of, int64_t *n_blocks) {
    if (!plan || rep < 0 || rep >= int64_t(plan->cones.size())) {
        set_error("bad plan or representative index");
        return QAOA_E_INVALID;
    }
    const Cone &c = plan->cones[rep];
    if (class_of) {
        std::fill(class_of, class_of + c.n, -1);
        for (size_t k = 0; k < c.shell_classes.size(); ++k)
            for (int32_t q : c.shell_classes[k]) class_of[q] = int32_t(k);
    }
    if (n_blocks) *n_blocks = c.n_blocks;
    return QAOA_OK;
}

extern "C" int qaoa_plan_blocks(const qaoa_plan *plan, int64_t rep, int64_t *n_blocks, int32_t *n_classes,
                                uint8_t *counts, double *weight) {
    if (!plan || rep < 0 || rep >= int64_t(plan->cones.size())) {
        set_error("bad plan or representative index");
        return QAOA_E_INVALID;
    }
    const Cone &c = plan->cones[rep];
    const int32_t ncls = int32_t(c.shell_classes.size());
    if (n_blocks) *n_blocks = c.n_blocks;
    if (n_classes) *n_classes = ncls;
    if (!counts && !weight) return QAOA_OK;
    for (int64_t b = 0; b < c.n_blocks; ++b) {
        double w = 1.0;
        if (!c.blk_counts.empty()) {
            if (counts) std::copy(c.blk_counts[b].begin(), c.blk_counts[b].end(), counts + b * ncls);
            w = c.blk_weight[b];
        } else {
            int64_t r = b;  // mixed radix, least significant class first
            for (int32_t k = 0; k < ncls; ++k) {
                const int s = int(c.shell_classes[k].size());
                const int nk = int(r % (s + 1));
                r /= s + 1;
                if (counts) counts[b * ncls + k] = uint8_t(nk);
                for (int i = 0; i < nk; ++i) w = w * double(s - i) / double(i + 1);
            }
        }
        if (weight) weight[b] = w;
    }
    return QAOA_OK;
}

extern "C" int qaoa_inject_fault(int32_t kind, int32_t count) {
    if (kind == QAOA_FAULT_NONE) {
        for (auto &f : g_faults) f.store(0);
        return QAOA_OK;
    }
    if (kind < 1 || kind > 2 || count < 0) {
        set_error("unknown fault kind or negative count");
        return QAOA_E_INVALID;
    }
    g_faults[kind].store(count);
    return QAOA_OK;
}
