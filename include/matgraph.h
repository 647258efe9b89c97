/*
 * matgraph: batched periodic cutoff and k-nearest-neighbour multigraphs of crystal
 * structures on one GB300 GPU (sm_103a), with edge vectors and their gradients.
 *
 * Method: Klipfel, Fregier, Sayede, Bouraoui, "Optimized Crystallographic Graph
 * Generation for Material Science" (IJCAI 2023 workshop; arXiv 2307.05380).
 *
 * Conventions (Sec. 2.1, Def. 1 and Def. 3)
 *   A structure s is a lattice L_s (3x3 float, ROW r = lattice vector r, Angstrom; the
 *   paper's rho is L^T) and fractional coordinates x (float [n][3], any finite value;
 *   never wrapped).  A batch concatenates structures: atom rows
 *   atom_ptr[s] .. atom_ptr[s+1]-1 belong to structure s.
 *   An edge is (src i, dst j, t), i and j GLOBAL atom rows of one structure, t an
 *   integer cell offset, with edge vector v = (x_j - x_i + t) L and length |v|.
 *   Cutoff graph (Def. 3, constant c per structure): every (i, j, t) with |v| < c,
 *   strictly, except (i, i, 0).  Images of an atom itself, (i, i, t != 0), are edges.
 *   KNN graph (Sec. 2.1, the special case after Def. 3; Alg. 1 and 2): exactly k edges
 *   per atom, the k smallest by (d2, j, t) lexicographically, t signed.
 *   Membership and ranking use the canonical FP64 distance: with inputs promoted to
 *   double and every operation rounded to nearest without fused multiply-add,
 *     df_c = (x_j[c] - x_i[c]) + t_c;  v_c = (df_0 L_0c + df_1 L_1c) + df_2 L_2c;
 *     d2 = (v_0^2 + v_1^2) + v_2^2;    edge iff d2 < (double)c * (double)c.
 *   Output order is canonical: (src, dst, tx, ty, tz) ascending; structures in order.
 *
 * Memory and streams
 *   Every pointer named "device" is device memory owned by the caller.  The library
 *   never allocates device memory: scratch comes from a caller workspace sized by
 *   mg_workspace_size.  All calls are ordered on the caller's stream (a cudaStream_t
 *   passed as void*; NULL = legacy default stream) and none synchronises the host,
 *   except mg_autotune and mg_measure_fp_peaks.  The host-side mg_context_t owns only
 *   host state (device
 *   properties, tuned schedules, captured CUDA graphs).
 *
 * Errors
 *   Arguments the host can check (null pointers, k <= 0, cutoff <= 0, too small a
 *   workspace) make a call return an error code before anything is launched.
 *   Problems found on the device (non-finite input, singular lattice, too small an
 *   edge capacity, an offset that does not fit a sort key, a bounded wait that ran
 *   out) are written to the graph's device status word; read it after synchronising
 *   the stream.  A CUDA launch error returns MG_ERR_CUDA.
 */
#ifndef MATGRAPH_H
#define MATGRAPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_context *mg_context_t;

typedef enum {
    MG_OK = 0,
    MG_ERR_INVALID_ARGUMENT = 1,
    MG_ERR_NONFINITE_INPUT = 2,
    MG_ERR_SINGULAR_LATTICE = 3,
    MG_ERR_CAPACITY = 4,     /* more edges than graph capacity; nothing past it written */
    MG_ERR_OFFSET_RANGE = 5, /* an offset component outside [-511, 511] where a packed
                                sort key needs it, or a KNN radius that could not grow */
    MG_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
    MG_ERR_CUDA = 7,
    MG_ERR_WORKSPACE = 8,    /* workspace pointer NULL or smaller than required */
    MG_ERR_NOT_BUILT = 9,    /* mg_update_graph on a graph no build call has filled */
    MG_ERR_INTERNAL = 10     /* an internal consistency check failed (a library bug) */
} mg_status_t;

/* Device status word, written by the kernels of a build. */
typedef struct {
    int32_t code;                /* mg_status_t of the first device-side problem, else 0 */
    int32_t first_bad_structure; /* structure index for input errors, else -1 */
    int64_t num_edges;           /* edges in the graph (also edge_ptr[B]) */
    int64_t required_capacity;   /* edges needed; equals num_edges on success */
    int64_t rechecked;           /* FP32 candidates re-tested in FP64 (opts.collect_stats) */
    int64_t candidates;          /* FP32 candidates evaluated (opts.collect_stats) */
} mg_device_status_t;

/* A batch of structures.  Counts are host values (no synchronisation needed). */
typedef struct {
    int32_t num_structures;   /* B >= 1 */
    int32_t total_atoms;      /* N = atom_ptr[B] */
    int32_t max_atoms;        /* max atoms in one structure, 0 if unknown (picks schedule) */
    const float *lattice;     /* device [B][3][3], row r = lattice vector r, Angstrom */
    const float *frac;        /* device [N][3] fractional coordinates */
    const int32_t *atom_ptr;  /* device [B+1], atom_ptr[0] = 0, non-decreasing */
} mg_batch_t;

/* Graph buffers, all device memory owned by the caller. */
typedef struct {
    int64_t capacity;          /* edges the arrays below can hold */
    int32_t *src;              /* [capacity] global atom row i */
    int32_t *dst;              /* [capacity] global atom row j */
    int32_t *offset;           /* [capacity][3] cell offset t */
    float *vec;                /* [capacity][3] (x_j - x_i + t) L, or NULL */
    float *len;                /* [capacity] |vec|, or NULL */
    int64_t *edge_ptr;         /* [B+1] edges of structure s: edge_ptr[s] .. edge_ptr[s+1]-1 */
    int64_t *src_ptr;          /* [N+1] CSR by source atom (needed by fwd/bwd), or NULL */
    int32_t *perm_dst;         /* [capacity] edge ids ordered by (dst, src, t), or NULL */
    int64_t *dst_ptr;          /* [N+1] CSR of perm_dst by destination atom; with perm_dst */
    mg_device_status_t *status;/* device status word */
} mg_graph_t;

/* Options; pass NULL for the defaults shown. */
typedef struct {
    float band_rel;        /* 1e-5: FP64 re-test band, relative to the cutoff distance
                              (candidates within band_rel*c of c are re-tested in FP64,
                              widened further to the FP32 error bound when that is larger) */
    int32_t knn_keep_ties; /* 0: exactly k edges per atom.  1: Alg. 2's final filter, every
                              image whose canonical d2 is <= the k-th one (ties at the k-th
                              distance all kept, so >= k edges per atom; the capacity then
                              works as for a cutoff graph).  Other values: invalid argument */
    int32_t schedule;      /* 0 auto (tuned where mg_autotune ran for the size class).
                              KNN graphs (exact k): 5 (auto from 8192 atoms; 1 below) the
                              pair-lane KNN (a warp per
                              source, a lane per target evaluating that pair's offset box,
                              candidates sorted in shared memory; sources whose boxes are too
                              large go to the warp-enumeration KNN; k <= 64, larger k
                              takes schedule 1), 1 the warp-enumeration
                              KNN on a flat grid for every source, 2 on a persistent work
                              queue.  Cutoff builds: auto picks the one-pass build (decoupled
                              look-back) below 8192 atoms; from there the pair-lane build
                              (a cost-sorted work list pulled by a persistent grid: count
                              pass, scan of the counts, write pass) for a constant radius
                              when max_atoms is known and at most 1024, else the staged
                              build (scan and stage keys, scan the counts, write) when the
                              workspace covers the capacity (when it does not, the
                              one-pass pair-lane build for a constant radius); 3 forces
                              the one-pass build, 4 the staged one (if the workspace covers
                              the capacity), 5 the pair-lane one, 6 the one-pass pair-lane
                              one (items of the pair-lane scan in canonical order, a
                              decoupled look-back, no staging; 5 and 6: constant radius,
                              other builds ignore them) */
    int32_t collect_stats; /* 1: count FP32 candidates and FP64 re-tests into status */
    int32_t fault_tile;    /* -1.  Testing only: the one-pass cutoff build's tile with this
                              index never publishes its offset, so the bounded waits of the
                              tiles after it run out and the build reports MG_ERR_TIMEOUT
                              (edges then wrong) instead of hanging */
} mg_opts_t;

#define MG_KIND_CUTOFF 1
#define MG_KIND_KNN 2

/* Create a context bound to CUDA device `device`.  Reads device properties. */
mg_status_t mg_create(mg_context_t *ctx, int device);
mg_status_t mg_destroy(mg_context_t ctx);
const char *mg_status_string(mg_status_t status);

/* Workspace bytes that suffice for every call on batches with this many structures
 * and atoms (any values) and graphs of up to max_edges edges: about 2.3 KB per atom
 * (2 KB of it the pair table of symmetric graphs, for structures of up to 512 atoms),
 * 160 B per structure and 8 B per edge (staged keys, or sort scratch). */
mg_status_t mg_workspace_size(mg_context_t ctx, const mg_batch_t *batch, int64_t max_edges,
                              size_t *bytes);

/* Cutoff multigraph (Def. 3 with a constant cutoff per structure).
 * cutoff: radius for every structure, or cutoff_per_structure (device [B]) if not NULL.
 * Writes src, dst, offset, vec/len (if not NULL), edge_ptr, src_ptr (if not NULL), and
 * perm_dst/dst_ptr (if not NULL).  If the edge count exceeds capacity, the status word
 * reports MG_ERR_CAPACITY with required_capacity; edge arrays are then not written.
 * Canonical order holds whichever schedule runs. */
mg_status_t mg_cutoff_graph(mg_context_t ctx, const mg_batch_t *batch, float cutoff,
                            const float *cutoff_per_structure, const mg_opts_t *opts,
                            mg_graph_t *graph, void *workspace, size_t workspace_bytes,
                            void *stream);

/* Cutoff multigraph with one cutoff per atom (Def. 3 in full): every (i, j, t) with
 * |v| < c_i, the SOURCE atom's radius (so (i, j, t) and (j, i, -t) need not both be
 * edges), (i, i, 0) excluded; the FP64 test is d2 < (double)c_i * (double)c_i.
 * cutoff_atom: device [N], every value finite and > 0 (else the status word reports
 * MG_ERR_INVALID_ARGUMENT for the structure).  Outputs, capacity handling and order as
 * mg_cutoff_graph; the graph is not symmetric, so its backward needs perm_dst. */
mg_status_t mg_cutoff_graph_atoms(mg_context_t ctx, const mg_batch_t *batch, const float *cutoff_atom,
                                  const mg_opts_t *opts, mg_graph_t *graph, void *workspace,
                                  size_t workspace_bytes, void *stream);

/* KNN multigraph (Alg. 1 output): exactly k edges per atom, k * N in total, so the
 * capacity needed is known up front.  Search radii start from the number density and
 * grow until the k-th distance is covered (Alg. 1's loop).  Same outputs as above.
 * With opts->knn_keep_ties = 1 (Alg. 2's filter, d <= d^k_i) the k-th canonical distance
 * of every atom is found first and every image at most that far is emitted: >= k edges
 * per atom, capacity and MG_ERR_CAPACITY as for mg_cutoff_graph. */
mg_status_t mg_knn_graph(mg_context_t ctx, const mg_batch_t *batch, int32_t k,
                         const mg_opts_t *opts, mg_graph_t *graph, void *workspace,
                         size_t workspace_bytes, void *stream);

/* Rebuild `graph` for new coordinates/lattices held in the same device buffers, with
 * the kind, parameters, shapes and pointers of the last build of this graph (Sec. 1:
 * the graph follows the geometry inside a generative model's forward pass).  The
 * first call captures the build into a CUDA graph; later calls replay it.
 * Returns MG_ERR_NOT_BUILT if no build call has filled this graph. */
mg_status_t mg_update_graph(mg_context_t ctx, const mg_batch_t *batch, mg_graph_t *graph,
                            void *workspace, size_t workspace_bytes, void *stream);

/* The plain comparison build: the same kernels, launched once per structure (one launch
 * sequence per structure, device-chained offsets, no host synchronisation).
 * atom_ptr_host: host copy of batch->atom_ptr.  kind: MG_KIND_CUTOFF or MG_KIND_KNN
 * (cutoff or k used accordingly).  Output identical to the batched build. */
mg_status_t mg_build_per_structure(mg_context_t ctx, const mg_batch_t *batch, int32_t kind,
                                   float cutoff, int32_t k, const int32_t *atom_ptr_host,
                                   const mg_opts_t *opts, mg_graph_t *graph, void *workspace,
                                   size_t workspace_bytes, void *stream);

/* Edge vectors for a fixed edge set (Def. 3's rho (x_j - x_i + t)): vec [E][3] and
 * len [E] from the current batch coordinates.  Needs graph->src_ptr and edge_ptr; the
 * edge count is read on the device (edge_ptr[B]).  Either output may be NULL. */
mg_status_t mg_edge_vectors_fwd(mg_context_t ctx, const mg_batch_t *batch, const mg_graph_t *graph,
                                float *vec, float *len, void *stream);

/* Backward of mg_edge_vectors_fwd with the edge set held fixed:
 *   g_e = grad_vec_e + grad_len_e * vec_e / len_e   (len_e > 0)
 *   grad_frac[j] = sum_{e: dst=j} g_e L^T - sum_{e: src=j} g_e L^T
 *   grad_lattice[s] = sum_{e in s} (x_j - x_i + t)^T g_e          (3x3)
 * Deterministic: fixed-order compensated (float-float) sums, no floating-point atomics.
 * A graph last built on this context by mg_cutoff_graph (one radius per structure) or
 * mg_symmetrize is symmetric: the in-edge matching out-edge (j, i, t) is its reverse (i, j, -t), found in
 * i's source segment, so only src_ptr is needed.  Every other graph is summed over src
 * segments and over dst segments through perm_dst, so it needs src_ptr, perm_dst and
 * dst_ptr (else MG_ERR_INVALID_ARGUMENT).  grad_vec or grad_len may be NULL (zero);
 * vec/len are the forward outputs.  Outputs (device float [N][3] and [B][3][3]) are
 * overwritten. */
mg_status_t mg_edge_vectors_bwd(mg_context_t ctx, const mg_batch_t *batch, const mg_graph_t *graph,
                                const float *grad_vec, const float *grad_len, const float *vec,
                                const float *len, float *grad_frac, float *grad_lattice,
                                void *workspace, size_t workspace_bytes, void *stream);

/* Triplet buffers (device memory owned by the caller). */
typedef struct {
    int64_t capacity;           /* triplets the arrays below can hold */
    int32_t *edge_a;            /* [capacity] first edge id e of each triplet, or NULL
                                   (then implied by trip_ptr) */
    int32_t *edge_b;            /* [capacity] second edge id e' */
    int64_t *trip_ptr;          /* [E+1] triplets with first edge e: trip_ptr[e] ..
                                   trip_ptr[e+1]-1, or NULL */
    mg_device_status_t *status; /* num_edges = triplet count; MG_ERR_CAPACITY with
                                   required_capacity when capacity is too small */
} mg_triplets_t;

/* Triplets of a built graph: Gamma_2 of Def. 3, the ordered pairs (e, e') of edges with
 * the same source (the paper's tool list after Alg. 2), as ids into the graph's edge
 * arrays.  include_self = 1 keeps (e, e) as the definition does; 0 drops it.  Order:
 * (e, e') ascending, so source by source a deg x deg block (deg x (deg-1) without the
 * diagonal).  Needs graph->src_ptr and at most INT32_MAX edges; reads only src_ptr.
 * The count is sum_i deg_i * (deg_i - 1 + include_self); nothing is written past
 * `capacity` (the status word then reports MG_ERR_CAPACITY and the exact count). */
mg_status_t mg_triplets(mg_context_t ctx, const mg_batch_t *batch, const mg_graph_t *graph,
                        int32_t include_self, mg_triplets_t *out, void *workspace,
                        size_t workspace_bytes, void *stream);

/* Symmetric closure of a graph (the paper's tool list after Alg. 2): every edge of `in`
 * plus every reversed edge (j, i, -t), each distinct edge once, in canonical order.
 * `in` must hold distinct edges in canonical order with src_ptr, perm_dst and dst_ptr
 * (any graph this library built with a destination order).  `out` gets src, dst,
 * offset, vec/len (if not NULL, from the batch's geometry), src_ptr (required),
 * edge_ptr, and perm_dst/dst_ptr (if not NULL); capacity as for mg_cutoff_graph.  The
 * result is recorded as symmetric, so mg_edge_vectors_bwd needs no perm_dst for it.
 * The workspace must cover `in`'s capacity in edges (mg_workspace_size). */
mg_status_t mg_symmetrize(mg_context_t ctx, const mg_batch_t *batch, const mg_graph_t *in,
                          mg_graph_t *out, void *workspace, size_t workspace_bytes, void *stream);

/* Time the available schedules for this batch shape on the caller's buffers and keep
 * the fastest per size class (largest structure: <= 32, <= 128, <= 512 atoms, larger;
 * times batches below 8192 atoms and from there: class = 0..3 + 4 for the latter) in
 * the context: KNN schedules 1, 2 and 5; cutoff graphs the one-pass builds (3, 6), and
 * the staged and pair-lane builds when the workspace covers graph->capacity.  Each schedule
 * is timed as a loop rebuilds: a build that records it, then mg_update_graph replays
 * (CUDA events around three replays after a first one).
 * Synchronises; results are identical for every schedule.  kind/cutoff/k as in
 * mg_build_per_structure. */
mg_status_t mg_autotune(mg_context_t ctx, const mg_batch_t *batch, int32_t kind, float cutoff,
                        int32_t k, mg_graph_t *graph, void *workspace, size_t workspace_bytes,
                        void *stream);

/* The context's tuned schedules, table[kind - 1][size class] (the size classes of
 * mg_autotune; 0 = not tuned, else the schedule mg_autotune chose), read into table
 * (set = 0) or replaced from it (set = 1; values outside 0..5 are rejected), so that a
 * caller can keep them across processes (e.g. in a per-device cache file). */
#define MG_SIZE_CLASSES 8
mg_status_t mg_tuned_table(mg_context_t ctx, int32_t table[2][MG_SIZE_CLASSES], int32_t set);

/* Host buffers for mg_graph_to_host, all owned by the caller; any may be NULL (not
 * copied).  Page-locked (pinned) memory lets the copies run asynchronously. */
typedef struct {
    mg_device_status_t *status; /* one status word */
    int32_t *src;               /* [num_edges] */
    int32_t *dst;               /* [num_edges] */
    int32_t *offset;            /* [num_edges][3] */
    float *vec;                 /* [num_edges][3]; needs graph->vec */
    float *len;                 /* [num_edges]; needs graph->len */
    int64_t *edge_ptr;          /* [B+1] */
    int64_t *src_ptr;           /* [N+1]; needs graph->src_ptr */
} mg_graph_host_t;

/* Copy a built graph to host memory (data movement only, no counterpart in the paper):
 * the first num_edges rows of src, dst, offset, vec and len, the pointer arrays and the
 * status word, for every non-NULL field of `out`, as one cudaMemcpyAsync each on
 * `stream` (asynchronous: synchronise the stream before reading).  num_edges is a host
 * value, e.g. from an earlier status read; rows past the edge count the device holds
 * are undefined.  MG_ERR_INVALID_ARGUMENT for num_edges outside [0, capacity], or a
 * requested field whose device array the graph does not have; MG_ERR_CUDA if a copy
 * cannot be issued. */
mg_status_t mg_graph_to_host(mg_context_t ctx, const mg_batch_t *batch, const mg_graph_t *graph,
                             int64_t num_edges, const mg_graph_host_t *out, void *stream);

/* Number of kernel launches the last build/fwd/bwd call on this context issued
 * (graph replays count their kernel nodes). */
int64_t mg_last_launch_count(mg_context_t ctx);

/* Measurement support (not needed for results).  When on, the batched builds and the
 * edge-vector calls of this context record CUDA events on the caller's stream between
 * their kernel stages.  A plan is recorded again at its next replay when the switch has
 * changed since it was recorded: with the event records when on, without them (and
 * with kernels launched behind their predecessors) when off.
 * mg_stage_times waits for the events of the last call of kind `which`
 * (MG_PROF_CUTOFF, MG_PROF_KNN, MG_PROF_FWD, MG_PROF_BWD), then writes up to max_stages
 * stage names (static strings) and durations in milliseconds.  Returns the number of
 * stages, or -1 if that kind has not run with profiling on. */
/* Cutoff graph without a caller workspace (no counterpart in the paper; a library
 * convenience).  Some callers cannot hand the library a workspace: code that runs
 * inside another framework's allocator (which owns all device memory through its own
 * pool), plug-ins that may not call cudaMalloc because it can synchronise the device,
 * or real-time loops that must not allocate after start-up.  This entry point takes
 * the same inputs and outputs as mg_cutoff_graph but keeps its scratch in a fixed
 * array of MG_NOALLOC_SCRATCH_BYTES bytes that the library holds in device memory on
 * every GPU where it is loaded, until the process exits.  It never allocates.
 *   - Limit: a batch whose scratch (mg_workspace_size with max_edges = capacity when
 *     perm_dst is requested, else 0) exceeds MG_NOALLOC_SCRATCH_BYTES is rejected
 *     with MG_ERR_WORKSPACE before anything is launched.
 *   - The first call on a device looks up the array's device address (with that device
 *     current); make that first call before any stream capture.
 *   - All calls on one device share the array, and the previous call's contents stay
 *     in it (the kernels clear what they need).  Calls whose work overlaps on the GPU
 *     (different streams, no ordering between them) race on the array: order them.
 * Output is identical to mg_cutoff_graph's.  The build is not recorded: mg_update_graph
 * on these buffers returns MG_ERR_NOT_BUILT, and a plan of an earlier mg_cutoff_graph
 * into the same buffers is dropped.  The graph is recorded as symmetric, so
 * mg_edge_vectors_bwd needs only its src_ptr (no perm_dst) and any workspace that
 * mg_workspace_size sizes for the batch; it finds reverse edges by binary search. */
#define MG_NOALLOC_SCRATCH_BYTES (32u << 20)
mg_status_t mg_cutoff_graph_noalloc(mg_context_t ctx, const mg_batch_t *batch, float cutoff,
                                    const mg_opts_t *opts, mg_graph_t *graph, void *stream);

/* One step of a generative loop in one call (no counterpart in the paper; it saves the
 * host time of a call per stage): new geometry in, the graphs rebuilt, edge vectors and
 * their gradients, results out.  Every pointer is caller-owned; NULL skips that part.
 * In order, on the caller's streams:
 *   1. frac_host / lattice_host / atom_ptr_host (pinned host memory, the batch's sizes)
 *      are copied into the batch's device buffers on stream[0];
 *   2. graph[1] (if not NULL) is rebuilt by mg_update_graph on stream[1] after the
 *      copies, and copied out by mg_graph_to_host (graph_host[1], host_edges[1] rows)
 *      behind it on the same stream;
 *   3. graph[0] is rebuilt on stream[0]; its host copy runs on stream[2] behind it (or on
 *      stream[0] when stream[2] is NULL), beside the rest of the step;
 *   4. mg_edge_vectors_fwd into vec / len and mg_edge_vectors_bwd of grad_vec / grad_len
 *      into grad_frac / grad_lattice on graph[0] (ws[0] as the backward's workspace), each
 *      skipped when its outputs are NULL; vec_host and len_host (host_edges[0] rows) are
 *      copied out behind the forward on stream[2] (after graph[0]'s copy) while the
 *      backward runs, grad_frac_host and grad_lattice_host behind the backward;
 *   5. stream[0] waits for streams 1 and 2: synchronise stream[0] to read the results.
 * Each graph must have been built before on this context (mg_update_graph's
 * conditions); errors are those of the calls named.  Does not synchronise.
 * capture = 1: the first call records all of the above as one CUDA graph and launches
 * it; a later call whose arguments are identical (the same pointers, sizes and edge
 * counts, compared byte for byte with the batch, the graphs and the host buffer lists)
 * launches that graph again: one launch per step instead of about 25 calls.  Other
 * arguments record a new graph.  The context keeps one recorded step. */
typedef struct {
    const mg_batch_t *batch;
    const float *frac_host, *lattice_host;   /* [N][3], [B][3][3] pinned host, or NULL */
    const int32_t *atom_ptr_host;             /* [B+1] pinned host, or NULL */
    mg_graph_t *graph[2];                     /* graph[1] may be NULL */
    void *ws[2];
    size_t ws_bytes[2];
    void *stream[3];                          /* stream[1], stream[2] may be NULL (= stream[0]) */
    const mg_graph_host_t *graph_host[2];     /* host copies of the graphs, or NULL */
    int64_t host_edges[2];                    /* rows to copy (e.g. the last read edge count) */
    const float *grad_vec, *grad_len;         /* device [E][3], [E] incoming gradients, or NULL */
    float *vec, *len;                         /* device forward outputs, or NULL (no forward) */
    float *grad_frac, *grad_lattice;          /* device backward outputs, or NULL (no backward) */
    float *vec_host, *len_host, *grad_frac_host, *grad_lattice_host;  /* pinned host, or NULL */
    int32_t capture;                          /* 1: record once, replay (see above) */
} mg_step_t;
mg_status_t mg_graph_step(mg_context_t ctx, const mg_step_t *step);

/* Measurement support (no counterpart in the paper): the FP32 and FP64 fused
 * multiply-add issue rates of this GPU, in TFLOP/s (2 flops per FMA), from the library's
 * own kernel: every thread runs 16 independent FMA chains, a full-occupancy grid, CUDA
 * events around each launch, the best of three timed launches after one warm-up.  No
 * clock or power setting is read or changed.  sink: 16 bytes of device memory the
 * kernels may write (they never do for these inputs).  Synchronises the stream. */
mg_status_t mg_measure_fp_peaks(mg_context_t ctx, void *sink, double *fp32_tflops, double *fp64_tflops,
                                void *stream);

#define MG_PROF_CUTOFF 0
#define MG_PROF_KNN 1
#define MG_PROF_FWD 2
#define MG_PROF_BWD 3
mg_status_t mg_profile_enable(mg_context_t ctx, int32_t on);
int32_t mg_stage_times(mg_context_t ctx, int32_t which, int32_t max_stages, const char **names, float *ms);

#ifdef __cplusplus
}
#endif
#endif /* MATGRAPH_H */
