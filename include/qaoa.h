/*
 * qaoa.h -- C ABI of libqaoa: orbit-reduced depth-p QAOA MaxCut energies and
 * their adjoint gradients on one GB300 (sm_103a).
 *
 * What is computed (arXiv:2101.10296):
 *   E_p(gamma, beta) = sum_{(u,v) in E} 1/2 (1 - <Z_u Z_v>)       (Sec. 2.3-2.4)
 * for the QAOA state U_B(beta_p) U_P(gamma_p) ... U_B(beta_1) U_P(gamma_1)|+>^n
 * with U_P(gamma) = exp(-i gamma H), H the diagonal cut count, and
 * U_B(beta) = prod_j exp(-i beta X_j) (Sec. 2.2).  Each edge term is simulated
 * on the state vector of the edge's reverse causal cone, the vertices within
 * distance p of the edge (Sec. 2.3), and with orbit reduction only one
 * representative edge per orbit of Aut(G) is simulated, its term weighted by
 * the orbit size (Sec. 3, Theorem 1 and the orbit-weighted sum after it).
 *
 * Conventions used by every entry point:
 *   - A graph is simple and undirected: vertices 0..n-1, edges given as
 *     int32 pairs [m][2] (either order), no self-loops, no repeated edges.
 *   - Parameter rows are (gamma_1..gamma_p, beta_1..beta_p), float64.
 *   - Return value: QAOA_OK (0) or a negative qaoa_status.  On error a
 *     message is available from qaoa_last_error() (thread-local) and no
 *     output has been written unless stated.  Argument errors are found on
 *     the host before anything is launched.
 *   - Device pointers (suffix _dev) are caller-owned CUDA device memory on
 *     the current device; host pointers (no suffix) are caller-owned host
 *     memory.  Device-side work is enqueued on `stream` (a cudaStream_t;
 *     NULL = legacy default stream) and is asynchronous: outputs are ready
 *     when the stream reaches that point.
 *   - A plan is immutable after qaoa_plan_upload and may be used from
 *     several streams at once; each call gets its own stream-ordered scratch.
 */
#ifndef QAOA_H
#define QAOA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qaoa_plan qaoa_plan;
typedef void *qaoa_stream_t; /* cudaStream_t */

enum qaoa_status {
    QAOA_OK = 0,
    QAOA_E_INVALID = -1,        /* bad argument, graph or state */
    QAOA_E_CONE_TOO_LARGE = -2, /* a cone exceeds the qubit or edge cap */
    QAOA_E_OOM = -3,            /* host or device allocation failed */
    QAOA_E_CUDA = -4,           /* a CUDA runtime call failed */
    QAOA_E_DEVICE = -5          /* a kernel's own guard tripped (status word) */
};

enum qaoa_flags {
    QAOA_ORBITS_OFF = 0u, /* every edge is its own representative */
    QAOA_ORBITS = 1u,     /* one representative per edge orbit of Aut(G) */
    QAOA_FULL_CONE = 2u,  /* simulate the whole 2^n cone state with the mixer on
                             every cone qubit in every layer (no pruning of the
                             gates that cancel); slower, used for cross-checks */
    QAOA_SHELL_PLAIN = 4u, /* evolve every assignment of the never-mixed shell
                              qubits as its own block instead of one block per
                              shell class count vector; slower, for cross-checks */
    QAOA_BIG_GENERAL = 8u, /* large-state cones always use the general pass
                              schedule (psi and lambda both stored), never the
                              core-tile schedule; slower, for cross-checks */
    QAOA_CONE_CLASSES = 16u, /* simulate one cone per isomorphism class of the
                               graph's cones (root edge fixed setwise), weighted
                               by the class's total orbit size: edges with
                               isomorphic cones have equal terms (the argument
                               of Sec. 3 applied to cone isomorphisms, the
                               local symmetries of Sec. 6); a coarser partition
                               than the Aut(G) orbits, found by a verified
                               search (qaoa_plan_cone_classes) */
    QAOA_BLOCK_PLAIN = 32u /* keep every shell class count vector as its own
                              block instead of merging those that contribute
                              equally (qaoa_plan_blocks); slower, for
                              cross-checks */
};

/* Largest cone handled: qubits per cone and local edges per cone. */
#define QAOA_MAX_CONE_QUBITS 32
#define QAOA_MAX_CONE_EDGES 64
#define QAOA_MAX_P 8

/*
 * qaoa_plan_graphs -- plan a batch of graphs (host only; no CUDA call).
 *
 * Steps, per graph: validate and build adjacency; if QAOA_ORBITS, find the
 * edge orbits of Aut(G) (Sec. 2.6 and Sec. 4: colour refinement, then an
 * individualisation-refinement search for automorphism generators, each
 * verified to preserve every edge; orbits by union-find); pick the smallest
 * edge index of each orbit as its representative (the paper's arbitrary
 * representative, Sec. 3); extract each representative's reverse causal cone
 * (Sec. 2.3): BFS to depth p from {u, v}, local qubit 0 = min(u,v),
 * 1 = max(u,v), the rest ordered by (distance, vertex id); the cone's edges
 * are the edges with at least one endpoint within distance p-1 (the terms
 * whose support meets the growing operator support, Sec. 2.3).
 *
 *   n_graphs        number of graphs G >= 1
 *   n_vertices      host int32[G]
 *   edge_offsets    host int64[G+1]; graph g owns edge rows
 *                   edge_offsets[g] .. edge_offsets[g+1]-1 of `edges`
 *   edges           host int32[edge_offsets[G]][2]
 *   p               QAOA depth, 1..QAOA_MAX_P
 *   flags           qaoa_flags
 *   max_cone_qubits cap on qubits per cone (<= QAOA_MAX_CONE_QUBITS;
 *                   0 = QAOA_MAX_CONE_QUBITS); a larger cone fails the
 *                   call with QAOA_E_CONE_TOO_LARGE
 *   search_budget   cap on refinement calls of the automorphism search per
 *                   graph (0 = default 2,000,000).  When reached, the search
 *                   stops and the orbits of the verified subgroup found so far
 *                   are used: still exact (any subgroup of symmetries gives a
 *                   valid reduction, Sec. 3), only less reduced.
 *   out             receives the new plan (caller frees with qaoa_plan_free)
 *
 * Errors: QAOA_E_INVALID (bad sizes, vertex out of range, self-loop,
 * repeated edge, p out of range), QAOA_E_CONE_TOO_LARGE, QAOA_E_OOM.
 */
int qaoa_plan_graphs(int32_t n_graphs, const int32_t *n_vertices,
                     const int64_t *edge_offsets, const int32_t *edges,
                     int32_t p, uint32_t flags, int32_t max_cone_qubits,
                     int64_t search_budget, qaoa_plan **out);

/*
 * Weighted (edge-coloured) form of qaoa_plan_graphs: weights (host
 * int32[total edges], same order as edges; NULL = all 1) gives each edge an
 * integer weight w_e with 1 <= |w_e| <= QAOA_MAX_CONE_EDGES.  The objective
 * becomes the weighted cut C(z) = sum_e w_e [z_u != z_v] and
 * E = sum_e w_e (1 - <Z_u Z_v>) / 2; the Ising objective
 * f(z) = sum J_ij z_i z_j of Sec. 4 is this with w = -J (up to a constant
 * and gamma -> 2 gamma).  Orbits are those of the automorphisms that map
 * every edge to an edge of the same weight (Sec. 4: edge colours), shell and
 * cone classes respect weights too.  An edge of weight w takes |w| bits of a
 * cone's 64-bit cut word, so a cone's total |w| is capped at
 * QAOA_MAX_CONE_EDGES (QAOA_E_CONE_TOO_LARGE).  QAOA_E_INVALID for a zero or
 * out-of-range weight; otherwise as qaoa_plan_graphs.
 */
int qaoa_plan_graphs_weighted(int32_t n_graphs, const int32_t *n_vertices,
                              const int64_t *edge_offsets, const int32_t *edges,
                              const int32_t *weights, int32_t p, uint32_t flags,
                              int32_t max_cone_qubits, int64_t search_budget,
                              qaoa_plan **out);

/* Single-graph form of qaoa_plan_graphs (edges: host int32[n_edges][2]). */
int qaoa_plan_graph(int32_t n_vertices, int64_t n_edges, const int32_t *edges,
                    int32_t p, uint32_t flags, int32_t max_cone_qubits,
                    int64_t search_budget, qaoa_plan **out);

/* Frees the plan and all host and device memory it owns.  NULL is a no-op.
 * The caller must make sure no stream still uses the plan. */
void qaoa_plan_free(qaoa_plan *plan);

typedef struct qaoa_plan_info_t {
    int32_t p;
    int32_t n_graphs;
    int64_t n_edges_total;  /* sum of |E_g| */
    int64_t n_reps;         /* simulated cones (= orbits, or edges if OFF) */
    int32_t max_qubits;     /* largest cone */
    int32_t max_inner;      /* largest inner part (qubits within distance p-1) */
    int32_t max_edges;      /* largest cone edge count */
    int32_t on_device;      /* 1 after qaoa_plan_upload */
    int64_t n_big;          /* cones routed to the large-state path */
    double amps_per_point;  /* sum over reps of 2^n_c (one eval, one layer) */
    double t_orbits_s;      /* wall time of orbit finding (all graphs) */
    double t_cones_s;       /* wall time of cone extraction */
    int32_t orbits_complete; /* 1 if every graph's search finished in budget */
    /* large-state cones by schedule (0 without large-state cones): on the
     * general schedule for the energy, and for the gradient (the rest of
     * n_big runs on the core-tile schedule) */
    int64_t n_big_general_energy;
    int64_t n_big_general_grad;
    /* 1 when the register-resident cones run on the depth-1 kernel: p = 1 and
     * every such cone's inner part is the edge {u, v}, the qubits the only
     * mixer acts on (Sec. 2.3), so its shell blocks evolve independently and
     * are processed as one flat list per graph.  Calls that ask for terms_dev
     * use the general register kernel. */
    int32_t depth1_kernel;
} qaoa_plan_info_t;

int qaoa_plan_info(const qaoa_plan *plan, qaoa_plan_info_t *info);

/*
 * Per-graph orbit summary.  orbit_id: host int32[|E_g|] (may be NULL)
 * receives, for each edge in input order, the index of the smallest edge in
 * its orbit.  n_orbits, log10_aut (log10 of the order of the group found,
 * from the orbit-stabiliser product along the search's first path) and
 * complete (1 if the search finished within budget) may each be NULL.
 */
int qaoa_plan_orbits(const qaoa_plan *plan, int32_t graph, int32_t *orbit_id,
                     int64_t *n_orbits, double *log10_aut, int32_t *complete);

/* Cone classes of graph `graph` (0-based): class_id[e] (host, n_edges of the
 * graph, may be NULL) = the smallest edge index of edge e's class, and
 * *n_classes (may be NULL) = the number of classes = the graph's rows in the
 * plan.  Without QAOA_CONE_CLASSES the classes are the orbits.  Every class
 * only joins edges whose cones were proven isomorphic (search with the
 * root edge fixed setwise, leaves checked edge by edge), so all its edges
 * have the same term.  Host only.  Returns QAOA_E_INVALID on a bad plan or
 * graph index. */
int qaoa_plan_cone_classes(const qaoa_plan *plan, int32_t graph, int32_t *class_id, int64_t *n_classes);

/*
 * Representatives, in plan order (the row order of terms_dev).  Each array
 * is host memory of length n_reps and may be NULL.  weight = orbit size
 * (total over the class with QAOA_CONE_CLASSES) times the edge's weight.
 * mix_qubits (host int32[n_reps][p], may be NULL): qubits mixed in each
 * layer -- the local qubits within distance p-l of the edge for layer l
 * (all n_qubits with QAOA_FULL_CONE).
 */
int qaoa_plan_reps(const qaoa_plan *plan, int32_t *graph, int64_t *edge,
                   int32_t *weight, int32_t *n_qubits, int32_t *n_inner,
                   int32_t *n_cone_edges, int32_t *mix_qubits);

/*
 * One representative's cone.  verts: host int32[n_qubits] global vertex of
 * each local qubit; dist: host int32[n_qubits] distance to the edge;
 * cone_edges: host int32[n_cone_edges][2] local pairs (a < b), in the bit
 * order used by the cut table.  Any pointer may be NULL.
 */
int qaoa_plan_cone(const qaoa_plan *plan, int64_t rep, int32_t *verts,
                   int32_t *dist, int32_t *cone_edges);

/* Weights of one representative's cone edges (host int32[n_cone_edges], the
 * order of qaoa_plan_cone; all 1 for an unweighted plan).  QAOA_E_INVALID on
 * a bad plan, index or NULL pointer. */
int qaoa_plan_cone_weights(const qaoa_plan *plan, int64_t rep, int32_t *weights);

/*
 * Shell classes of one representative's cone.  The shell qubits (distance p,
 * never mixed) with the same set of inner neighbours form a class; an inner
 * block is evolved once per vector of per-class counts of shell qubits set
 * to 1 and weighted by the product of binomial coefficients, which sums
 * exactly the same terms as one block per shell assignment (Sec. 2.3: the
 * shell enters only through the phase, and exchanging two shell qubits of a
 * class leaves every cut value unchanged).  class_of: host int32[n_qubits],
 * -1 for inner qubits, else the class index; n_blocks: number of blocks.
 * Either pointer may be NULL.
 */
int qaoa_plan_shell(const qaoa_plan *plan, int64_t rep, int32_t *class_of,
                    int64_t *n_blocks);

/*
 * The shell blocks one representative's cone is evolved for.  Unless the plan
 * has QAOA_BLOCK_PLAIN, count vectors that contribute equally are merged into
 * one block: (1) those with the same phase vector c_q = sum_k (s_k - 2 n_k)
 * w_kq (a class of s shell qubits with n set to 1 adds n W + (s - 2n) times
 * the weighted sum of its inner neighbours' bits to the cut, so c fixes the
 * block's evolution up to a global phase); (2) those related by a symmetry of
 * the cone (a permutation of its qubits that keeps every edge and weight,
 * every distance from the root edge and the root edge itself), which carries
 * one block's evolution onto the other's with the inner qubits relabelled
 * (the argument of Sec. 3, Theorem 1, inside one cone); (3) c and -c (the
 * global spin flip leaves the cut, the mixers, |+> and Z_u Z_v unchanged).
 * counts: host uint8[n_blocks * n_classes], row b = the number of shell
 * qubits set to 1 in each class (qaoa_plan_shell's class order) for the
 * block evolved; weight: host double[n_blocks], the number of shell
 * assignments block b stands for (the weights sum to 2^(shell qubits)).
 * Call with both NULL to learn n_blocks and n_classes; either output pointer
 * may be NULL.  QAOA_E_INVALID on a bad plan or index.
 */
int qaoa_plan_blocks(const qaoa_plan *plan, int64_t rep, int64_t *n_blocks,
                     int32_t *n_classes, uint8_t *counts, double *weight);

/*
 * Host-only edge-orbit finder on one graph (the plan's orbit step alone),
 * for callers that only want symmetry.  orbit_id: host int32[n_edges] as in
 * qaoa_plan_orbits.  n_generators, log10_aut and complete may be NULL.
 */
int qaoa_edge_orbits(int32_t n_vertices, int64_t n_edges, const int32_t *edges,
                     int64_t search_budget, int32_t *orbit_id,
                     int64_t *n_orbits, int64_t *n_generators,
                     double *log10_aut, int32_t *complete);

/*
 * Copies the plan's cone descriptors to the current device (synchronous).
 * Called implicitly by the first energy call if not done; calling it first
 * keeps allocation out of later calls.  Errors: QAOA_E_CUDA, QAOA_E_OOM.
 */
int qaoa_plan_upload(qaoa_plan *plan);

/*
 * Integer cut table of one representative's cone (Sec. 2.4: the MaxCut
 * Hamiltonian is diagonal with value C(z) = number of cone edges (a, b) with
 * z_a != z_b; bit q of z is local qubit q).  out_dev: device uint8[2^n]
 * with n = the cone's qubit count; computed by the same device routine the
 * energy kernels use.  Bit-exact.  For a weighted plan the table holds
 * C(z) + (sum of |w| over the cone's negative edges), which is >= 0.
 */
int qaoa_cut_table(const qaoa_plan *plan, int64_t rep, uint8_t *out_dev,
                   qaoa_stream_t stream);

/*
 * Energies at n_points parameter points per graph.
 *   params_dev  device float64[n_graphs][n_points][2p]
 *   energy_dev  device float64[n_graphs][n_points]  E_p of each graph
 *   terms_dev   optional device float64[n_reps][n_points]: <Z_u Z_v> of each
 *               representative (NULL to skip)
 * State: complex64 amplitudes, FP32 arithmetic; cut values are integers;
 * the phase table exp(-i gamma c) is computed in FP64 and rounded to FP32;
 * per-cone and orbit-weighted sums are accumulated in FP64.
 * Errors: QAOA_E_INVALID (n_points < 1, NULL params/energy),
 * QAOA_E_CUDA / QAOA_E_OOM.
 */
int qaoa_energy(const qaoa_plan *plan, int64_t n_points, const double *params_dev,
                double *energy_dev, double *terms_dev, qaoa_stream_t stream);

/*
 * State norms: the forward sweep of qaoa_energy with the identity in place of
 * Z_u Z_v, so that norms_dev receives sum_z |psi_z|^2 of every representative's
 * cone state at every point (exactly 1 for the unitary evolution of Sec. 2.2;
 * the departure from 1 is the FP32 state's accumulated rounding).  The
 * energies are not renormalised by it: this is a diagnostic.
 *   norms_dev   device float64[n_reps][n_points], overwritten
 * Other arguments and errors as qaoa_energy; allocates one stream-ordered
 * float64[n_graphs][n_points] scratch for the unused energies.
 */
int qaoa_norms(const qaoa_plan *plan, int64_t n_points, const double *params_dev,
               double *norms_dev, qaoa_stream_t stream);

/*
 * Energies and their gradients dE/d(gamma_1..gamma_p, beta_1..beta_p) by the
 * adjoint method: after the forward sweep, the state psi and the co-state
 * lambda = -1/2 Z_u Z_v psi are taken back through the inverse gates; each
 * derivative is 2 Im <lambda| G |psi> at the gate exp(-i theta G).
 *   grad_dev  device float64[n_graphs][n_points][2p]
 * Other arguments and errors as qaoa_energy.
 */
int qaoa_energy_grad(const qaoa_plan *plan, int64_t n_points,
                     const double *params_dev, double *energy_dev,
                     double *grad_dev, double *terms_dev, qaoa_stream_t stream);

/*
 * qaoa_energy_noalloc -- qaoa_energy that makes no device allocation.  The
 * paper has no counterpart: this is an interface for callers that must not
 * allocate GPU memory while they run (code inside another allocator's
 * callbacks, under a budget manager that forbids new allocations, or in a
 * process whose memory pool belongs to another runtime), so neither
 * cudaMalloc nor stream-ordered allocation may happen inside the call.
 *
 * Same arguments, outputs and results as qaoa_energy.  Its temporary memory
 * -- the phase tables and the state blocks of cones on the large-state
 * path -- is carved from one static device array of QAOA_NOALLOC_SCRATCH_MB
 * MiB that every device loading the library keeps until the process exits.
 * The plan must already be on the device (qaoa_plan_upload, which does
 * allocate; call it during set-up).  The array occupies device memory from
 * the moment its module is loaded on a device; qaoa_plan_upload forces that
 * load and looks up the array's device address, so the memory is committed
 * during set-up and a qaoa_energy_noalloc call allocates nothing, not even
 * its first.  Should that lookup fail at upload (it is not reported there),
 * the first qaoa_energy_noalloc call on the device repeats it, which loads
 * the module then; make that first call before any stream capture.  A call whose tables plus one state block would not fit returns
 * QAOA_E_INVALID with the sizes in the message, before launching anything.
 * Every call uses the same array and leaves its contents behind (all of it
 * is rewritten before being read, nothing needs clearing); calls that
 * overlap on the GPU -- on different streams, or from different host
 * threads -- race on it, so callers must serialise them.
 */
#define QAOA_NOALLOC_SCRATCH_MB 64
int qaoa_energy_noalloc(const qaoa_plan *plan, int64_t n_points,
                        const double *params_dev, double *energy_dev,
                        double *terms_dev, qaoa_stream_t stream);

/*
 * Reads and clears the plan's device status word (synchronises the device).
 * *status = 0 if no kernel guard tripped since the last read; otherwise a
 * nonzero code, the OR of 1: descriptor out of range, 2: non-finite result,
 * 4: a tensor-memory-accelerator load into shared memory did not complete
 * within its time limit (the block stopped; results of that call are
 * incomplete).
 */
int qaoa_device_status(const qaoa_plan *plan, int32_t *status);

/*
 * Launch tuning of a plan (applies to every later call).  Any field 0 means
 * "default".
 *   points_per_task  parameter points one warp task of the register kernels
 *                    evaluates for the same cone slots (default: up to 32,
 *                    while their phase tables fit 8 KB of shared memory;
 *                    larger values are cut to what fits 12 KB per warp; the
 *                    depth-1 kernel's default is what leaves room for its
 *                    resident blocks: the multiprocessor's shared memory
 *                    split among them, less the per-block reservation)
 *   blocks_per_sm    resident blocks per SM of the persistent grid (default:
 *                    the occupancy limit)
 *   big_scratch_bytes scratch per call for large-state cones, which sets how
 *                    many state blocks a wave holds (default 1 GiB; a wave
 *                    that fits the 129 MB L2 keeps its passes on chip)
 *   reg_bits_grad    register qubits per thread of the adjoint register
 *                    kernel, 4 or 5: a tile of 2^(bits + 5) amplitudes per
 *                    warp, 5 holding twice the amplitudes per thread at half
 *                    the resident blocks (default: 5 when the plan's
 *                    register work fills the GPU for at least four waves of
 *                    8 warps per SM at 32 points per task, else 4; the
 *                    autotuner times both)
 *   chunk_window     largest window of outer qubits a shared-memory chunk
 *                    pass of the large-state path mixes, 6..10 (default 10):
 *                    the 2^13-amplitude chunk is a window of w outer qubits
 *                    over contiguous runs of 2^(13 - w) amplitudes
 * Errors: QAOA_E_INVALID for negative values, reg_bits_grad other than
 * 0, 4, 5, or chunk_window outside 6..10 (0 = default).
 */
typedef struct qaoa_tuning_t {
    int32_t points_per_task;
    int32_t blocks_per_sm;
    int64_t big_scratch_bytes;
    int32_t reg_bits_grad;
    int32_t chunk_window;
} qaoa_tuning_t;

int qaoa_plan_set_tuning(qaoa_plan *plan, const qaoa_tuning_t *tuning);
int qaoa_plan_get_tuning(const qaoa_plan *plan, qaoa_tuning_t *tuning);

/*
 * Captured CUDA graphs (batching: one replayable graph per evaluation).
 * qaoa_graph_create records one qaoa_energy (grad_dev == NULL) or
 * qaoa_energy_grad call with these fixed device buffers into a CUDA graph
 * (its scratch becomes graph-owned memory nodes) and instantiates it; the
 * plan is uploaded first if needed.  qaoa_graph_launch replays it on
 * `stream`: write new parameters into params_dev before each launch; the
 * outputs are overwritten.  The plan and the buffers must outlive the graph.
 * Errors: as qaoa_energy / qaoa_energy_grad, or QAOA_E_CUDA if capture fails.
 */
typedef struct qaoa_graph qaoa_graph;
int qaoa_graph_create(qaoa_plan *plan, int64_t n_points, const double *params_dev,
                      double *energy_dev, double *grad_dev, double *terms_dev,
                      qaoa_graph **out);
int qaoa_graph_launch(qaoa_graph *graph, qaoa_stream_t stream);
void qaoa_graph_free(qaoa_graph *graph);

/*
 * Kernel timing, for measurement.  With enable != 0 every later energy or
 * gradient call records a pair of CUDA events on its own stream around each
 * of its cone kernels (the FP64 phase-table kernel that precedes them is not
 * included).  qaoa_kernel_time waits for those events, returns the summed
 * kernel milliseconds in *ms, the number of cone-kernel launches timed in
 * *launches and the number of all kernel launches made by those calls in
 * *all_launches (any of the three may be NULL), and forgets them.
 */
int qaoa_plan_timing(qaoa_plan *plan, int32_t enable);
int qaoa_kernel_time(qaoa_plan *plan, double *ms, int64_t *launches, int64_t *all_launches);

/*
 * Failure injection for testing error handling; nothing here faults the GPU.
 * The next `count` events of `kind` are made to fail on the host:
 *   QAOA_FAULT_GENERATOR  a candidate automorphism of the orbit search gets
 *                         two images exchanged before verification (which
 *                         must then reject it; the orbits stay those of a
 *                         verified subgroup)
 *   QAOA_FAULT_DEVICE_ALLOC  a device allocation of an energy call reports
 *                         out-of-memory (the call returns QAOA_E_OOM before
 *                         launching anything)
 * kind QAOA_FAULT_NONE clears every pending injection.  Process-wide.
 */
enum qaoa_fault { QAOA_FAULT_NONE = 0, QAOA_FAULT_GENERATOR = 1, QAOA_FAULT_DEVICE_ALLOC = 2 };
int qaoa_inject_fault(int32_t kind, int32_t count);

/* Last error message of the calling thread ("" if none). */
const char *qaoa_last_error(void);

/* Library version string. */
const char *qaoa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QAOA_H */
