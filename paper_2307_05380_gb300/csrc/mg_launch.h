// Internal launch interface between the C-ABI host layer (api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "matgraph.h"

namespace mg {

struct StructRec;

// Device scratch carved from the caller's workspace.
struct Work {
    StructRec *recs;          // [B]
    float4 *pos;              // [N] Cartesian positions (FP32)
    int32_t *atom_struct;     // [N] structure of each atom row
    int32_t *cnt;             // [N] per-atom counts (edges out / edges in)
    int32_t *cursor;          // [N] scatter cursors
    long long *tile_sum;      // [n_tiles + 1] scan partials
    int64_t *src_ptr;         // [N+1] used when the graph has none
    float2 *gpart;            // [N][3] source-side gradient partials (float-float)
    float2 *lpart;            // [N][9] per-atom lattice-gradient partials (float-float)
    int32_t *sort_tmp;        // [max_edges] scratch for long destination segments (aliases stage)
    unsigned long long *stage;      // [max_edges] staged (j, t) keys of the decoupled build
    long long *stage_off;           // [N] slot of each source's keys in `stage` (-1: spilled)
    unsigned long long *stage_ctr;  // next free slot (queue[4..5])
    unsigned int *queue;      // [4] work-queue counters
    int32_t *bin_cnt;         // [N+B] atoms per cell-list bin
    int32_t *bin_cursor;      // [N+B] scatter cursors of the bins
    int64_t *cell_start;      // [N+B+1] first slot of each bin
    float4 *cell_fx;          // [N] fractional coordinates of each slot, .w = local index bits
    float4 *cell_p;           // [N] FP32 Cartesian position of each slot (bin order)
    int32_t *atom_bin;        // [N] global bin of each atom (-1: all-pairs structure)
    unsigned long long *tile_flags;  // [N/BUILD_TILE + 2] look-back words of the one-pass build
    double *rr_atom;          // [N] per-source squared radius (keep-ties KNN: the k-th distance)
    uint16_t *pair_lo;        // [N][PAIR_MAX] run of edges i -> j in i's segment: first and
    uint16_t *pair_hi;        //   one-past-last position (structures of <= PAIR_MAX atoms)
    int32_t *pair_ok;         // [B] 1: the pair table of the structure is complete
    int32_t *lat_cnt;         // [B] atoms of the structure whose lattice partial is stored
    int2 *items;              // [N] pair-lane build: work items (structure, item within it)
    int32_t *spill_list;      // [N] staged builds: sources whose keys were not staged
                              // (queue[12] of them, taken through cursor queue[13]); aliases cursor
    int32_t *plan_items;      // [B] work items of each structure
    int32_t *plan_class;      // [B] cost class of each structure's items
    int32_t *item_base;       // [B] first slot of each structure's items in `items`
    int64_t max_edges;
};

constexpr int SCAN_TILE = 4096;
constexpr int BUILD_TILE = 4;    // source atoms (one warp each) per look-back tile of the one-pass build
constexpr int PAIR_MAX = 512;    // largest structure with a pair table (run of i -> j per (i, j)):
                                 // 2 KB of workspace per atom

struct PrepArgs {
    int B, N;
    const float *lattice, *frac;
    const int32_t *atom_ptr;
    float cutoff;              // cutoff graphs: constant radius (if cutoff_ps NULL)
    const float *cutoff_ps;    // per-structure radii or NULL
    int knn_k;                 // > 0: KNN graph (starting radius from density)
    float band_rel;
    mg_device_status_t *status;
    int struct_offset;         // global index of the first structure of this call
    int zero_tiles;            // 1: clear the one-pass build's look-back words and ticket
    int init_status;           // 1: reset the status word (first kernel of a build)
    int64_t *src_ptr;          // KNN: written here (k per atom); may be NULL otherwise
    int64_t *edge_ptr;         // KNN: written here
    int max_atoms;             // host-known bound on atoms per structure (0: unknown)
    const float *cutoff_atom = nullptr;  // per-atom radii [N]: the structure's reach is their maximum
    int32_t *pair_ok = nullptr;          // [B] set to (n <= PAIR_MAX) when a pair table is written
    int32_t *lat_cnt = nullptr;          // [B] zeroed with the pair table (backward's counters)
    int32_t *plan_items = nullptr;       // [B] pair-lane build: work items of each structure
    int32_t *plan_class = nullptr;       // [B] pair-lane build: cost class of its items (0..31)
};

cudaError_t launch_prep(const PrepArgs &a, const Work &w, cudaStream_t s);

// Fractional cell list of the structures that use one (after prep): bins counted,
// scanned and filled.  Batched form: all atoms [0, N) and every bin.  Per-structure
// form (atom_lo..atom_hi of one structure with host-known first bin and atom row):
// slots of that structure start at its first atom row.
cudaError_t launch_bins(int B, int N, const float *frac, const Work &w, cudaStream_t s);
cudaError_t launch_bins_one(int atom_lo, int atom_hi, int bin_base, const float *frac, const Work &w,
                            cudaStream_t s);

struct ScanArgs {
    int n;                     // counts
    const int32_t *cnt;
    int64_t *out_ptr;          // [n+1] exclusive prefix, out_ptr[n] = total
};
cudaError_t launch_scan(const ScanArgs &a, const Work &w, cudaStream_t s);

struct BuildArgs {
    int B, N;
    const float *frac;
    const int32_t *atom_ptr;
    int schedule;              // 1 flat, 2 persistent queue
    int collect_stats;
    mg_graph_t g;
    int64_t *src_ptr;          // graph's or workspace's
    int knn_k;
    float band_rel;
    int atom_lo, atom_hi;      // atom row range to process (per-structure builds)
    int struct_offset;         // global index of local structure 0 (per-structure builds)
    int fault_tile;            // testing: a one-pass build tile that never publishes (-1: none)
    // per-source radius of the one-pass build (default: the structure's cutoff)
    const float *cut_atom = nullptr;   // [N] radius c_i; edge iff d2 < c_i^2
    const double *rr_atom = nullptr;   // [N] squared radius in FP64 (keep-ties KNN)
    int inclusive = 0;                 // 1: edge iff d2 <= rr (Alg. 2's filter)
    double *knn_dk = nullptr;          // KNN: write the k-th canonical d2 per atom, no edges
    int write_pairs = 0;               // 1: record the pair table (symmetric cutoff graphs)
    int knn_list = 0;                  // 1: the KNN kernel takes only the sources of the fallback
                                       // list (w.items as int [queue[10]]) the pair-lane KNN left
    int pdl = 0;                       // host: launch the first build kernel with programmatic
                                       // stream serialization (it directly follows prep)
};

// Pair-lane cutoff build (batched, constant radius): a cost-sorted work list of the
// structures' source groups (plan: 2 launches), then a stage pass over the list that
// counts every source and stages its keys like the staged build's stage kernel; the
// staged build's count scan and emit finish it.  Structures whose pair boxes are too
// large or that use a cell list are scanned by the warp enumeration inside the pass.
cudaError_t launch_pair_plan(const BuildArgs &a, const Work &w, cudaStream_t s);
cudaError_t launch_pair_stage(const BuildArgs &a, const Work &w, cudaStream_t s);
// One-pass pair-lane build (constant radius, small batches): items of the pair-lane
// scan in canonical order (1 launch), then masks, a decoupled look-back over tiles of
// items and the edges written from the masks (1 launch).
cudaError_t launch_pair_onepass(const BuildArgs &a, const Work &w, cudaStream_t s);
// One-pass cutoff build (batched): scan once, stage keys, look-back offsets, write.
cudaError_t launch_cutoff_build(const BuildArgs &a, const Work &w, cudaStream_t s);
// Staged cutoff build: scan and stage keys globally (stage), scan the counts and write
// the pointers and status (counts: 4 launches), write the edges (emit).  Sources whose
// keys do not fit the staging area (w.max_edges) are enumerated again by emit.
cudaError_t launch_cutoff_stage(const BuildArgs &a, const Work &w, cudaStream_t s);
cudaError_t launch_cutoff_counts(const BuildArgs &a, const Work &w, cudaStream_t s);
cudaError_t launch_cutoff_emit(const BuildArgs &a, const Work &w, cudaStream_t s);
// Two-pass form (per-structure builds): count, separate scan, write.
cudaError_t launch_cutoff_count(const BuildArgs &a, const Work &w, cudaStream_t s);
// Edge pointers, status and capacity check after the scan of counts.
cudaError_t launch_cutoff_finalize(const BuildArgs &a, const Work &w, cudaStream_t s);
cudaError_t launch_cutoff_write(const BuildArgs &a, const Work &w, cudaStream_t s);
cudaError_t launch_knn(const BuildArgs &a, const Work &w, cudaStream_t s);
constexpr int PL_KNN_MAX_K = 64;  // largest k of the pair-lane KNN (its buffer holds 2k candidates)
// Pair-lane KNN (exact k, batched): a warp per source, lanes over targets evaluating
// their pairs' offset boxes at a growing search radius; sources it cannot take go to a
// list that launch_knn (with knn_list = 1) builds afterwards.
cudaError_t launch_knn_pairs(const BuildArgs &a, const Work &w, cudaStream_t s);
cudaError_t launch_knn_pointers(const BuildArgs &a, const Work &w, cudaStream_t s);
cudaError_t launch_dst_sort(const BuildArgs &a, const Work &w, cudaStream_t s, int *launches);
// Destination order of a symmetric (cutoff) graph from its source order, one kernel.
cudaError_t launch_dst_perm_symmetric(const BuildArgs &a, const Work &w, cudaStream_t s);
cudaError_t launch_reset_queue(const Work &w, cudaStream_t s);

struct EdgeVecArgs {
    int B, N;
    int max_atoms;             // host-known bound on atoms per structure (0: unknown)
    const float *lattice, *frac;
    const int32_t *atom_ptr;
    mg_graph_t g;
    const float *grad_vec, *grad_len, *vec, *len;
    float *out_vec, *out_len;
    float *grad_frac, *grad_lattice;
    // symmetric backward: the pair table of the graph's build (NULL: binary searches)
    const uint16_t *pair_lo, *pair_hi;
    const int32_t *pair_ok, *atom_struct;
    int32_t *lat_cnt;          // non-NULL: the last warp of a structure reduces its lattice
                               // gradient (counters start at zero and are left at zero)
};
cudaError_t launch_edgevec_fwd(const EdgeVecArgs &a, cudaStream_t s);
cudaError_t launch_bwd_sym(const EdgeVecArgs &a, const Work &w, cudaStream_t s);  // symmetric graphs
cudaError_t launch_bwd_src(const EdgeVecArgs &a, const Work &w, cudaStream_t s);
cudaError_t launch_bwd_dst(const EdgeVecArgs &a, const Work &w, cudaStream_t s);
cudaError_t launch_bwd_lat(const EdgeVecArgs &a, const Work &w, cudaStream_t s);

// Triplets (Gamma_2): ordered pairs of edges with a common source, as edge ids.
struct TripArgs {
    int N;
    const int64_t *src_ptr;    // [N+1] CSR by source of the graph
    int excl;                  // 1: leave out (e, e)
    int64_t capacity;
    int32_t *edge_a, *edge_b;  // [capacity]; edge_a may be NULL
    int64_t *trip_ptr;         // [E+1] CSR by first edge, or NULL
    mg_device_status_t *status;
};
cudaError_t launch_triplets(const TripArgs &a, const Work &w, cudaStream_t s, int *launches);

// Symmetric closure of a graph (needs its destination order).
struct SymArgs {
    int B, N;
    const float *lattice, *frac;
    const int32_t *atom_ptr;
    mg_graph_t in, out;
};
cudaError_t launch_symmetrize(const SymArgs &a, const Work &w, cudaStream_t s, int *launches);

int num_sms();

}  // namespace mg
