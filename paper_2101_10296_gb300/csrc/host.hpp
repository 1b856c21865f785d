// Host-side planner internals: graph, edge-orbit finder, lightcone extractor,
// plan object.  Nothing here touches CUDA.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qaoa.h"

namespace qaoa {

// Simple undirected graph in CSR form.  Edge e joins eu[e] < ev[e]; adj lists
// are sorted and eid[k] is the edge id of adjacency entry k.
struct Graph {
    int32_t n = 0;
    int64_t m = 0;
    std::vector<int64_t> off;
    std::vector<int32_t> adj;
    std::vector<int64_t> eid;
    std::vector<int32_t> eu, ev;
    std::vector<int32_t> ew;  // edge weights (colours), input order; all 1 for MaxCut
    int32_t degree(int32_t v) const { return int32_t(off[v + 1] - off[v]); }
};

// Validates and builds; weights may be NULL (all 1).  Returns QAOA_OK or
// QAOA_E_INVALID with `err` set.
int build_graph(int32_t n, int64_t m, const int32_t *edges, const int32_t *weights, Graph &g, std::string &err);
int64_t find_edge(const Graph &g, int32_t a, int32_t b);

struct OrbitResult {
    std::vector<int32_t> orbit_id;  // per edge: smallest edge index of its orbit
    int64_t n_orbits = 0;
    int64_t n_generators = 0;
    double log10_aut = 0.0;
    bool complete = true;
};

// Edge orbits of Aut(G) (or of the verified subgroup found within budget).
void edge_orbits(const Graph &g, int64_t budget, OrbitResult &out);
// Every edge its own orbit.
void trivial_orbits(const Graph &g, OrbitResult &out);

// One representative's reverse causal cone.
struct Cone {
    int32_t graph = 0;
    int64_t edge = 0;     // representative edge index within its graph
    int32_t weight = 1;   // orbit size
    int32_t n = 0;        // qubits (ball of radius p)
    int32_t n_in = 0;     // qubits within distance p-1 (mixed in layer 1)
    int32_t k[QAOA_MAX_P] = {0};  // layer l mixes local qubits [0, k[l])
    std::vector<int32_t> verts, dist;
    std::vector<int32_t> ea, eb;  // local edges (a < b), sorted
    std::vector<int32_t> ew;      // their weights
    // Shell (never-mixed) qubits grouped by their set of inner neighbours;
    // one block per vector of per-class counts of shell qubits set to 1.
    std::vector<std::vector<int32_t>> shell_classes;
    int64_t n_blocks = 1;  // prod over classes of (size + 1), or blk_counts.size()
    // Block merging (block_orbits.cpp): when blocks that contribute equally merge,
    // one count vector per orbit and its total multiplicity; empty = every block.
    std::vector<std::vector<uint8_t>> blk_counts;
    std::vector<double> blk_weight;
};

// Fills cone for edge `e` of g at depth p.  full_cone: mix every qubit in
// every layer.  shell_plain: one class per shell qubit (every assignment its
// own block).  Returns QAOA_OK or QAOA_E_CONE_TOO_LARGE.
int extract_cone(const Graph &g, int64_t e, int32_t p, bool full_cone, bool shell_plain, int32_t max_qubits,
                 std::vector<int32_t> &dist_scratch, Cone &c, std::string &err);

// Cone classes (cone_classes.cpp): whether two cones are isomorphic with the
// root edge fixed setwise (then their terms are equal), and the classes of a
// list of cones: class_of[i] = index of the first cone of i's class.
bool cones_isomorphic(const Cone &a, const Cone &b, int p);
void cone_classes(const std::vector<const Cone *> &cones, int p, std::vector<int32_t> &class_of);

// Merges the cone's shell blocks that contribute equally (block_orbits.cpp).
// With a memo (shared by the threads of one planning call), cones whose
// local structure was merged before reuse that result.
struct BlockMemo;
BlockMemo *block_memo_new();
void block_memo_free(BlockMemo *m);
void block_orbits(Cone &c, BlockMemo *memo = nullptr);

void set_error(const std::string &msg);

// Injected failures (qaoa_inject_fault): true if one of `kind` is pending,
// consuming it.
bool take_fault(int kind);

}  // namespace qaoa

struct qaoa_device_plan;  // defined in the CUDA translation unit

struct qaoa_plan {
    int32_t p = 1;
    uint32_t flags = 0;
    int32_t n_graphs = 0;
    std::vector<int32_t> n_vertices;
    std::vector<int64_t> n_edges;
    std::vector<int64_t> weight_sum;  // per graph: sum of edge weights (|E| for MaxCut)
    bool weighted = false;
    std::vector<qaoa::OrbitResult> orbits;
    std::vector<qaoa::Cone> cones;  // plan order (rows of terms)
    // per graph and edge: the smallest edge of its cone class (QAOA_CONE_CLASSES),
    // else of its orbit; and the number of classes
    std::vector<std::vector<int32_t>> cone_class;
    std::vector<int64_t> n_classes;
    double t_orbits = 0.0, t_cones = 0.0;
    qaoa_device_plan *dev = nullptr;
};
