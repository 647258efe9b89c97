// C-ABI host layer of matgraph (include/matgraph.h): argument checks, workspace
// carving, launch sequences, CUDA-graph plans for mg_update_graph, the per-structure
// comparison build and the schedule autotuner.  It allocates no device memory.
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "matgraph.h"
#include "mg_device.cuh"
#include "mg_launch.h"

namespace mg {

static int g_num_sms = 0;
int num_sms() { return g_num_sms > 0 ? g_num_sms : 152; }

}  // namespace mg

using namespace mg;

// Stage events of one call (measurement support).
struct Prof {
    static constexpr int MAX = 16;
    cudaEvent_t ev[MAX] = {};
    const char *name[MAX] = {};
    int n = 0;
    bool valid = false;
    bool create() {
        for (auto &e : ev)
            if (!e && cudaEventCreate(&e) != cudaSuccess) return false;
        return true;
    }
    void destroy() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        *this = Prof();
    }
};

// A recorded build: everything a rebuild of the same graph needs.  A captured plan
// owns its own stage events (they are nodes of its CUDA graph).
struct Plan {
    int kind = 0;
    float cutoff = 0.f;
    const float *cutoff_ps = nullptr;
    const float *cutoff_atom = nullptr;
    int k = 0;
    mg_opts_t opts{};
    mg_batch_t batch{};
    mg_graph_t graph{};
    void *ws = nullptr;
    size_t ws_bytes = 0;
    cudaGraphExec_t exec = nullptr;
    bool exec_profiled = false;  // exec was recorded with stage events (profiling on)
    int launches = 0;
    Prof prof;
};

struct mg_context {
    int device = 0;
    int sms = 152;
    bool prof_on = false;
    Prof prof[4];                // events of direct (not replayed) calls, per kind
    Prof *last_prof[4] = {};     // events of the last call of each kind
    std::mutex mu;
    std::map<const void *, Plan> plans;      // keyed by graph->src
    std::map<const void *, mg_graph_t> sym;  // symmetric closures written here, keyed by src
    std::map<const void *, const void *> pair_owner;  // workspace -> graph (src) whose pair table it holds
    int tuned[2][MG_SIZE_CLASSES] = {};  // [kind-1][size class] -> schedule (0: not tuned)
    int64_t last_launches = 0;
    cudaEvent_t step_ev[4] = {};  // mg_graph_step's fork and join events (no timing)
    struct StepRec {              // the step mg_graph_step recorded as a CUDA graph
        mg_step_t st{};
        mg_batch_t batch{};
        mg_graph_t g[2]{};
        mg_graph_host_t h[2]{};
        cudaGraphExec_t exec = nullptr;
    } step;
};

namespace {

constexpr size_t ALIGN = 256;
constexpr int KIND_CUTOFF_ATOMS = 3;  // plans only: a cutoff graph with per-atom radii
constexpr int STAGED_MIN_ATOMS = 8192; // smallest batch built by the decoupled form by default
constexpr int PAIR_AUTO_MAX_ATOMS = 1024;  // largest structure of a batch the pair-lane build takes by default

// Stage marks: with profiling on, record the next event of `prof` (default: the
// context's set for `which`) on the stream.
struct Marker {
    mg_context *ctx;
    int which;
    cudaStream_t st;
    Prof *pr;
    Marker(mg_context *c, int w, cudaStream_t s, Prof *p = nullptr) : ctx(c), which(w), st(s), pr(p) {
        if (on()) {
            if (!pr) pr = &ctx->prof[which];
            pr->n = 0;
            pr->valid = false;
            ctx->last_prof[which] = pr;
            mark("start");
        }
    }
    bool on() const { return ctx && which >= 0 && ctx->prof_on; }
    void mark(const char *name) {
        if (!on()) return;
        Prof &p = *pr;
        if (p.n >= Prof::MAX) return;
        if (!p.ev[p.n]) return;
        // inside a capture the record must become a timing node of the graph
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (st) cudaStreamIsCapturing(st, &cs);
        if (cs == cudaStreamCaptureStatusActive)
            cudaEventRecordWithFlags(p.ev[p.n], st, cudaEventRecordExternal);
        else
            cudaEventRecord(p.ev[p.n], st);
        p.name[p.n] = name;
        ++p.n;
        p.valid = true;
    }
};

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    size_t recs, pos, atom_struct, cnt, cursor, tile_sum, src_ptr, gpart, lpart, queue, bin_cnt, bin_cursor,
        cell_start, cell_fx, cell_p, atom_bin, tile_flags, rr_atom, pair_lo, pair_hi, pair_ok, lat_cnt, stage_off,
        items, plan_items, plan_class, item_base, sort_tmp, total;
};

// Workspace regions, 256-byte aligned; the edge-sized sort scratch comes last so that
// any workspace size maps to an exact edge limit.
Layout layout(int B, int N, int64_t max_edges) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += align_up(bytes > 0 ? bytes : 1);
        return at;
    };
    const size_t n = (size_t)(N > 0 ? N : 1);
    const size_t nbins = (size_t)N + (size_t)(B > 0 ? B : 1);
    const size_t tiles = (nbins + 1 + SCAN_TILE - 1) / SCAN_TILE + 2;
    L.recs = take(sizeof(StructRec) * (size_t)(B > 0 ? B : 1));
    L.pos = take(sizeof(float4) * n);
    L.atom_struct = take(sizeof(int32_t) * n);
    L.cnt = take(sizeof(int32_t) * n);
    L.cursor = take(sizeof(int32_t) * n);
    L.tile_sum = take(sizeof(long long) * tiles);
    L.src_ptr = take(sizeof(int64_t) * (n + 1));
    L.gpart = take(sizeof(float2) * 3 * n);
    L.lpart = take(sizeof(float2) * 9 * n);
    L.queue = take(16 * sizeof(unsigned int));
    L.bin_cnt = take(sizeof(int32_t) * nbins);
    L.bin_cursor = take(sizeof(int32_t) * nbins);
    L.cell_start = take(sizeof(int64_t) * (nbins + 1));
    L.cell_fx = take(sizeof(float4) * n);
    L.cell_p = take(sizeof(float4) * n);
    L.atom_bin = take(sizeof(int32_t) * n);
    L.tile_flags = take(sizeof(unsigned long long) * (n / BUILD_TILE + 2));
    L.rr_atom = take(sizeof(double) * n);
    L.pair_lo = take(sizeof(uint16_t) * n * PAIR_MAX);
    L.pair_hi = take(sizeof(uint16_t) * n * PAIR_MAX);
    L.pair_ok = take(sizeof(int32_t) * (size_t)(B > 0 ? B : 1));
    L.lat_cnt = take(sizeof(int32_t) * (size_t)(B > 0 ? B : 1));
    L.stage_off = take(sizeof(long long) * n);
    L.items = take(sizeof(int2) * n);
    L.plan_items = take(sizeof(int32_t) * (size_t)(B > 0 ? B : 1));
    L.plan_class = take(sizeof(int32_t) * (size_t)(B > 0 ? B : 1));
    L.item_base = take(sizeof(int32_t) * (size_t)(B > 0 ? B : 1));
    L.sort_tmp = off;  // edge-sized region, 8 bytes per edge: staged keys, or sort scratch
    off += sizeof(unsigned long long) * (size_t)(max_edges > 0 ? max_edges : 0);
    L.total = align_up(off);
    return L;
}

Work carve(void *ws, int B, int N, int64_t max_edges) {
    const Layout L = layout(B, N, max_edges);
    char *b = static_cast<char *>(ws);
    Work w;
    w.recs = reinterpret_cast<StructRec *>(b + L.recs);
    w.pos = reinterpret_cast<float4 *>(b + L.pos);
    w.atom_struct = reinterpret_cast<int32_t *>(b + L.atom_struct);
    w.cnt = reinterpret_cast<int32_t *>(b + L.cnt);
    w.cursor = reinterpret_cast<int32_t *>(b + L.cursor);
    w.tile_sum = reinterpret_cast<long long *>(b + L.tile_sum);
    w.src_ptr = reinterpret_cast<int64_t *>(b + L.src_ptr);
    w.gpart = reinterpret_cast<float2 *>(b + L.gpart);
    w.lpart = reinterpret_cast<float2 *>(b + L.lpart);
    w.queue = reinterpret_cast<unsigned int *>(b + L.queue);
    w.bin_cnt = reinterpret_cast<int32_t *>(b + L.bin_cnt);
    w.bin_cursor = reinterpret_cast<int32_t *>(b + L.bin_cursor);
    w.cell_start = reinterpret_cast<int64_t *>(b + L.cell_start);
    w.cell_fx = reinterpret_cast<float4 *>(b + L.cell_fx);
    w.cell_p = reinterpret_cast<float4 *>(b + L.cell_p);
    w.atom_bin = reinterpret_cast<int32_t *>(b + L.atom_bin);
    w.tile_flags = reinterpret_cast<unsigned long long *>(b + L.tile_flags);
    w.rr_atom = reinterpret_cast<double *>(b + L.rr_atom);
    w.pair_lo = reinterpret_cast<uint16_t *>(b + L.pair_lo);
    w.pair_hi = reinterpret_cast<uint16_t *>(b + L.pair_hi);
    w.pair_ok = reinterpret_cast<int32_t *>(b + L.pair_ok);
    w.lat_cnt = reinterpret_cast<int32_t *>(b + L.lat_cnt);
    w.sort_tmp = reinterpret_cast<int32_t *>(b + L.sort_tmp);
    w.stage = reinterpret_cast<unsigned long long *>(b + L.sort_tmp);
    w.stage_off = reinterpret_cast<long long *>(b + L.stage_off);
    w.stage_ctr = reinterpret_cast<unsigned long long *>(w.queue + 4);
    w.items = reinterpret_cast<int2 *>(b + L.items);
    w.spill_list = w.cursor;  // the scatter cursors are not in use during a cutoff build
    w.plan_items = reinterpret_cast<int32_t *>(b + L.plan_items);
    w.plan_class = reinterpret_cast<int32_t *>(b + L.plan_class);
    w.item_base = reinterpret_cast<int32_t *>(b + L.item_base);
    w.max_edges = max_edges;
    return w;
}

// Largest edge count a workspace of ws_bytes supports for this batch (-1: too small).
int64_t ws_max_edges(int B, int N, size_t ws_bytes) {
    const Layout L0 = layout(B, N, 0);
    if (ws_bytes < L0.total) return -1;
    return (int64_t)((ws_bytes - L0.sort_tmp) / sizeof(unsigned long long));
}

mg_opts_t defaults(const mg_opts_t *o) {
    mg_opts_t d;
    d.band_rel = 1e-5f;
    d.knn_keep_ties = 0;
    d.schedule = 0;
    d.collect_stats = 0;
    d.fault_tile = -1;
    if (o) d = *o;
    return d;
}

mg_status_t check_batch(const mg_batch_t *b) {
    if (!b || b->num_structures < 1 || b->total_atoms < 0 || !b->lattice || !b->atom_ptr ||
        (b->total_atoms > 0 && !b->frac))
        return MG_ERR_INVALID_ARGUMENT;
    return MG_OK;
}

mg_status_t check_graph(const mg_graph_t *g, const mg_batch_t *b) {
    if (!g || !g->status || !g->edge_ptr || g->capacity < 0) return MG_ERR_INVALID_ARGUMENT;
    if (g->capacity > 0 && (!g->src || !g->dst || !g->offset)) return MG_ERR_INVALID_ARGUMENT;
    if (g->perm_dst && !g->dst_ptr) return MG_ERR_INVALID_ARGUMENT;
    if (g->perm_dst && g->capacity > (int64_t)INT_MAX) return MG_ERR_INVALID_ARGUMENT;
    (void)b;
    return MG_OK;
}

// Size class of a batch: its largest structure (<= 32, <= 128, <= 512 atoms, larger or
// unknown as <= 128), plus 4 from 8192 atoms in the batch (where the staged and
// pair-lane forms start to pay for their extra launches).
int size_class(const mg_batch_t *b) {
    const int m = b->max_atoms;
    const int c = m <= 0 ? 1 : m <= 32 ? 0 : m <= 128 ? 1 : m <= 512 ? 2 : 3;
    return c + (b->total_atoms >= STAGED_MIN_ATOMS ? 4 : 0);
}

// KNN schedule: 1 / 2 the warp-enumeration KNN on a flat or persistent grid, 5 the
// pair-lane KNN, as requested or as mg_autotune measured for the size class; untuned,
// the pair-lane KNN from 8192 atoms and the warp enumeration below (batches of 32-512
// small structures: 0.034-0.063 against 0.040-0.081 ms for k = 32).
int pick_schedule(mg_context *ctx, int kind, const mg_batch_t *b, const mg_opts_t &o) {
    if (o.schedule == 1 || o.schedule == 2 || (kind == MG_KIND_KNN && o.schedule == 5)) return o.schedule;
    const int t = ctx->tuned[kind == MG_KIND_KNN ? 1 : 0][size_class(b)];
    if (kind == MG_KIND_KNN) return t ? t : (b->total_atoms >= STAGED_MIN_ATOMS ? 5 : 1);
    return t == 1 || t == 2 ? t : 1;
}

__global__ void status_init_kernel(mg_device_status_t *st) {
    st->code = 0;
    st->first_bad_structure = INT_MAX;
    st->num_edges = 0;
    st->required_capacity = 0;
    st->rechecked = 0;
    st->candidates = 0;
}

// The batched build's launch sequence (no host synchronisation).
mg_status_t enqueue_build(mg_context *ctx, int kind, const mg_batch_t *b, float cutoff, const float *cutoff_ps,
                          const float *cutoff_atom, int k, const mg_opts_t &o, const mg_graph_t *g, void *ws,
                          size_t ws_bytes, cudaStream_t st, int *launches, Prof *prof = nullptr) {
    const int B = b->num_structures, N = b->total_atoms;
    const int64_t me = ws_max_edges(B, N, ws_bytes);
    if (!ws || me < 0) return MG_ERR_WORKSPACE;
    if (g->perm_dst && me < g->capacity) return MG_ERR_WORKSPACE;  // destination sort scratch
    const Work w = carve(ws, B, N, me);
    int n = 0;
    const bool knn = kind == MG_KIND_KNN;
    const bool ties = knn && o.knn_keep_ties;  // edges come from the one-pass build
    Marker mk(ctx, knn ? MG_PROF_KNN : MG_PROF_CUTOFF, st, prof);
    int64_t *src_ptr = g->src_ptr ? g->src_ptr : w.src_ptr;
    // prep also resets the status word and, for exact-k KNN, writes the k-per-atom pointers
    PrepArgs pa{B, N, b->lattice, b->frac, b->atom_ptr, cutoff, cutoff_ps, knn ? k : 0, o.band_rel, g->status,
                0, (!knn || ties) ? 1 : 0, 1, src_ptr, (knn && !ties) ? g->edge_ptr : nullptr, b->max_atoms};
    pa.cutoff_atom = kind == KIND_CUTOFF_ATOMS ? cutoff_atom : nullptr;
    const bool pairs = kind == MG_KIND_CUTOFF;  // symmetric: record the pair table for the backward
    // The cutoff build's form: the pair-lane build (a cost-sorted work list, count pass,
    // scan, write pass; no keys staged in global memory) for constant-radius graphs of
    // large batches, the staged build (scan and stage keys, scan of the counts, write)
    // or the one-pass build (decoupled look-back) otherwise.  schedule 3 / 4 / 5 force
    // the one-pass / staged / pair-lane form, as does a form mg_autotune measured for this
    // size class; the one-pass form's testing hook forces it.
    int csched = o.schedule;
    if (csched == 0) csched = ctx->tuned[0][size_class(b)];
    const bool can_stage = o.fault_tile < 0 && me >= g->capacity;
    // auto: large batches of structures that are known to be small enough for the
    // pair-lane scan (batches of supercells, whose sources use a cell list, keep the
    // staged build, which enumerates them once)
    const bool pair_auto = N >= STAGED_MIN_ATOMS && b->max_atoms > 0 && b->max_atoms <= PAIR_AUTO_MAX_ATOMS;
    const bool pair_form = kind == MG_KIND_CUTOFF && can_stage &&
                           (csched == 5 || (csched != 3 && csched != 4 && pair_auto));
    const bool staged = !pair_form && can_stage && (csched == 4 || (csched != 3 && N >= STAGED_MIN_ATOMS));
    // schedule 6: the one-pass pair-lane build (constant radius; not with the testing hook).
    // It needs no staging area, so it also takes the large batches of small structures
    // whose workspace does not cover the capacity (where the others would fall back to
    // the one-pass warp enumeration: 0.27 against 0.47 ms at 1024 structures of up to
    // 400 atoms); below 8192 atoms the one-pass warp enumeration is faster (42 against
    // 54 us at 256 structures of up to 64 atoms).
    const bool pair_onepass = kind == MG_KIND_CUTOFF && !pair_form && !staged && o.fault_tile < 0 &&
                              (csched == 6 || (csched != 3 && !can_stage && pair_auto));
    if (pair_form || pair_onepass) {
        pa.plan_items = w.plan_items;
        pa.plan_class = w.plan_class;
    }
    pa.pair_ok = pairs ? w.pair_ok : nullptr;
    pa.lat_cnt = pairs ? w.lat_cnt : nullptr;
    if (launch_prep(pa, w, st)) return MG_ERR_CUDA;
    ++n;
    mk.mark("prep");
    bool after_prep = !mk.on();  // the next launch directly follows prep in the stream
    if (b->max_atoms <= 0 || b->max_atoms >= CELL_MIN_ATOMS) {  // some structure may use a cell list
        if (launch_bins(B, N, b->frac, w, st)) return MG_ERR_CUDA;
        n += 6;
        mk.mark("bin");
        after_prep = false;
    }
    BuildArgs ba;
    ba.pdl = after_prep ? 1 : 0;  // the build kernel may launch while prep finishes
    ba.struct_offset = 0;
    ba.B = B;
    ba.N = N;
    ba.frac = b->frac;
    ba.atom_ptr = b->atom_ptr;
    ba.schedule = pick_schedule(ctx, kind, b, o);
    ba.collect_stats = o.collect_stats;
    ba.fault_tile = o.fault_tile;
    ba.g = *g;
    ba.src_ptr = src_ptr;
    ba.knn_k = k;
    ba.band_rel = o.band_rel;
    ba.atom_lo = 0;
    ba.atom_hi = N;
    auto cutoff_build = [&](const BuildArgs &args) -> bool {  // false on a launch error
        if (pair_form && !args.cut_atom && !args.rr_atom) {
            if (launch_pair_plan(args, w, st)) return false;
            mk.mark("plan");
            if (launch_pair_stage(args, w, st)) return false;
            mk.mark("stage");
            if (launch_cutoff_counts(args, w, st)) return false;
            mk.mark("count_scan");
            if (launch_cutoff_emit(args, w, st)) return false;
            mk.mark("emit");
            n += 9;
            return true;
        }
        if (pair_onepass && !args.cut_atom && !args.rr_atom) {  // item scan, then one pass
            if (launch_pair_onepass(args, w, st)) return false;
            n += 2;
            mk.mark("build");
            return true;
        }
        if (!staged) {  // one pass: scan, look-back offsets, write (also src_ptr, edge_ptr, count)
            if (launch_cutoff_build(args, w, st)) return false;
            ++n;
            mk.mark("build");
            return true;
        }
        if (launch_cutoff_stage(args, w, st)) return false;
        mk.mark("stage");
        if (launch_cutoff_counts(args, w, st)) return false;
        mk.mark("count_scan");
        if (launch_cutoff_emit(args, w, st)) return false;
        mk.mark("emit");
        n += 7;
        return true;
    };
    if (!knn) {
        if (kind == KIND_CUTOFF_ATOMS) ba.cut_atom = cutoff_atom;
        ba.write_pairs = pairs ? 1 : 0;
        if (!cutoff_build(ba)) return MG_ERR_CUDA;
    } else if (ties) {
        // the k-th canonical distance of every atom, then every image at most that far
        ba.knn_dk = w.rr_atom;
        if (launch_knn(ba, w, st)) return MG_ERR_CUDA;
        n += 1 + (ba.schedule == 2);
        mk.mark("knn");
        ba.knn_dk = nullptr;
        ba.rr_atom = w.rr_atom;
        ba.inclusive = 1;
        if (!cutoff_build(ba)) return MG_ERR_CUDA;
    } else if (ba.schedule == 1 || ba.schedule == 2 || k > PL_KNN_MAX_K) {  // the warp-enumeration KNN
        if (ba.schedule != 1 && ba.schedule != 2) ba.schedule = 1;  // k beyond the pair-lane buffer
        if (launch_knn(ba, w, st)) return MG_ERR_CUDA;
        n += 1 + (ba.schedule == 2);
        mk.mark("knn");
    } else {  // the pair-lane KNN; the sources it leaves go to the warp-enumeration KNN
        if (launch_knn_pairs(ba, w, st)) return MG_ERR_CUDA;
        BuildArgs bl = ba;
        bl.knn_list = 1;
        bl.pdl = 0;
        if (launch_knn(bl, w, st)) return MG_ERR_CUDA;
        n += 2;
        mk.mark("knn");
    }
    if (g->perm_dst) {
        if (kind == MG_KIND_CUTOFF) {  // symmetric: destination order from the source order
            if (launch_dst_perm_symmetric(ba, w, st)) return MG_ERR_CUDA;
            ++n;
        } else {
            if (launch_dst_sort(ba, w, st, &n)) return MG_ERR_CUDA;
        }
        mk.mark("dst_sort");
    }
    if (launches) *launches = n;
    return MG_OK;
}

bool same_batch(const mg_batch_t &a, const mg_batch_t &b) {
    return a.num_structures == b.num_structures && a.total_atoms == b.total_atoms && a.max_atoms == b.max_atoms &&
           a.lattice == b.lattice && a.frac == b.frac && a.atom_ptr == b.atom_ptr;
}

bool same_graph(const mg_graph_t &a, const mg_graph_t &b) {
    return a.capacity == b.capacity && a.src == b.src && a.dst == b.dst && a.offset == b.offset && a.vec == b.vec &&
           a.len == b.len && a.edge_ptr == b.edge_ptr && a.src_ptr == b.src_ptr && a.perm_dst == b.perm_dst &&
           a.dst_ptr == b.dst_ptr && a.status == b.status;
}

bool same_opts(const mg_opts_t &a, const mg_opts_t &b) {
    return a.band_rel == b.band_rel && a.knn_keep_ties == b.knn_keep_ties && a.schedule == b.schedule &&
           a.collect_stats == b.collect_stats && a.fault_tile == b.fault_tile;
}

mg_status_t check_build_args(mg_context *ctx, const mg_batch_t *b, const mg_opts_t &o, const mg_graph_t *g) {
    if (!ctx) return MG_ERR_INVALID_ARGUMENT;
    mg_status_t r = check_batch(b);
    if (r) return r;
    r = check_graph(g, b);
    if (r) return r;
    if (o.knn_keep_ties < 0 || o.knn_keep_ties > 1 || !(o.band_rel >= 0.f) || o.schedule < 0 || o.schedule > 6)
        return MG_ERR_INVALID_ARGUMENT;
    return MG_OK;
}

mg_status_t build_and_record(mg_context *ctx, int kind, const mg_batch_t *b, float cutoff, const float *cutoff_ps,
                             const float *cutoff_atom, int k, const mg_opts_t *opts, mg_graph_t *g, void *ws,
                             size_t ws_bytes, void *stream) {
    const mg_opts_t o = defaults(opts);
    mg_status_t r = check_build_args(ctx, b, o, g);
    if (r) return r;
    if (kind == MG_KIND_CUTOFF && !cutoff_ps && !(cutoff > 0.f)) return MG_ERR_INVALID_ARGUMENT;
    if (kind == KIND_CUTOFF_ATOMS && !cutoff_atom && b->total_atoms > 0) return MG_ERR_INVALID_ARGUMENT;
    if (kind == MG_KIND_KNN) {
        if (k <= 0 || k > KNN_MAX_K) return MG_ERR_INVALID_ARGUMENT;
        if (!o.knn_keep_ties && (int64_t)k * b->total_atoms > g->capacity) return MG_ERR_CAPACITY;
    }
    int launches = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    r = enqueue_build(ctx, kind, b, cutoff, cutoff_ps, cutoff_atom, k, o, g, ws, ws_bytes, st, &launches);
    if (r) return r;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_launches = launches;
    ctx->sym.erase((const void *)g->src);
    if (kind == MG_KIND_CUTOFF)  // this build wrote the workspace's pair table
        ctx->pair_owner[ws] = (const void *)g->src;
    else
        ctx->pair_owner.erase(ws);
    Plan &p = ctx->plans[(const void *)g->src];
    const bool same = p.kind == kind && p.cutoff == cutoff && p.cutoff_ps == cutoff_ps &&
                      p.cutoff_atom == cutoff_atom && p.k == k &&
                      same_opts(p.opts, o) && same_batch(p.batch, *b) && same_graph(p.graph, *g) && p.ws == ws &&
                      p.ws_bytes == ws_bytes;
    if (!same) {
        if (p.exec) cudaGraphExecDestroy(p.exec);
        const int which = p.kind == MG_KIND_KNN ? MG_PROF_KNN : MG_PROF_CUTOFF;
        if (p.kind && ctx->last_prof[which] == &p.prof) ctx->last_prof[which] = nullptr;
        p.prof.destroy();
        p = Plan();
        p.kind = kind;
        p.cutoff = cutoff;
        p.cutoff_ps = cutoff_ps;
        p.cutoff_atom = cutoff_atom;
        p.k = k;
        p.opts = o;
        p.batch = *b;
        p.graph = *g;
        p.ws = ws;
        p.ws_bytes = ws_bytes;
        p.launches = launches;
    }
    return MG_OK;
}

}  // namespace

// Scratch for mg_cutoff_graph_noalloc: a fixed device array, so that callers which
// cannot provide a workspace (see matgraph.h) never make the library allocate.  Its
// name in host code is only a host-side handle: kernels receive the device address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MG_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of the scratch array in the current device's context.  Looked up on
// every call (a table lookup once the module is loaded): a cached address would go stale
// when the context is torn down and created again (cudaDeviceReset), and kernels would
// then write to memory that is no longer mapped.  The first lookup on a device loads the
// library's module into its context.
mg_status_t noalloc_scratch(void **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MG_ERR_CUDA;
    *out = p;
    return MG_OK;
}

}  // namespace

// Issue-rate probes for mg_measure_fp_peaks: every thread runs PEAK_CHAINS independent
// fused multiply-add chains (enough to cover the pipe latency) for `iters` steps; the
// result is stored only under a condition the data never meets, so the chains are kept.
constexpr int PEAK_CHAINS = 16;

template <class T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T b, T c, T *sink) {
    T acc[PEAK_CHAINS];
#pragma unroll
    for (int q = 0; q < PEAK_CHAINS; ++q) acc[q] = (T)(threadIdx.x + q) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < PEAK_CHAINS; ++q) acc[q] = fma(acc[q], b, c);
    }
    T sum = 0;
#pragma unroll
    for (int q = 0; q < PEAK_CHAINS; ++q) sum += acc[q];
    if (sum == (T)-1.2345e30) *sink = sum;
}

extern "C" {

mg_status_t mg_create(mg_context_t *ctx, int device) {
    if (!ctx) return MG_ERR_INVALID_ARGUMENT;
    *ctx = nullptr;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return MG_ERR_CUDA;
    mg_context *c = new (std::nothrow) mg_context();
    if (!c) return MG_ERR_INVALID_ARGUMENT;
    c->device = device;
    c->sms = prop.multiProcessorCount;
    g_num_sms = prop.multiProcessorCount;
    *ctx = c;
    return MG_OK;
}

mg_status_t mg_destroy(mg_context_t ctx) {
    if (!ctx) return MG_ERR_INVALID_ARGUMENT;
    for (auto &kv : ctx->plans) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        kv.second.prof.destroy();
    }
    for (auto &p : ctx->prof) p.destroy();
    for (auto &e : ctx->step_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->step.exec) cudaGraphExecDestroy(ctx->step.exec);
    delete ctx;
    return MG_OK;
}

const char *mg_status_string(mg_status_t s) {
    switch (s) {
    case MG_OK: return "MG_OK";
    case MG_ERR_INVALID_ARGUMENT: return "MG_ERR_INVALID_ARGUMENT: invalid argument";
    case MG_ERR_NONFINITE_INPUT: return "MG_ERR_NONFINITE_INPUT: non-finite lattice or coordinate";
    case MG_ERR_SINGULAR_LATTICE: return "MG_ERR_SINGULAR_LATTICE: singular lattice";
    case MG_ERR_CAPACITY: return "MG_ERR_CAPACITY: edge capacity too small";
    case MG_ERR_OFFSET_RANGE: return "MG_ERR_OFFSET_RANGE: cell offset outside the packed-key range";
    case MG_ERR_TIMEOUT: return "MG_ERR_TIMEOUT: a bounded device wait gave up";
    case MG_ERR_CUDA: return "MG_ERR_CUDA: CUDA error";
    case MG_ERR_WORKSPACE: return "MG_ERR_WORKSPACE: workspace missing or too small";
    case MG_ERR_NOT_BUILT: return "MG_ERR_NOT_BUILT: graph was never built";
    case MG_ERR_INTERNAL: return "MG_ERR_INTERNAL: internal consistency check failed";
    }
    return "unknown matgraph status";
}

mg_status_t mg_workspace_size(mg_context_t ctx, const mg_batch_t *batch, int64_t max_edges, size_t *bytes) {
    if (!ctx || !batch || !bytes || max_edges < 0 || batch->num_structures < 1 || batch->total_atoms < 0)
        return MG_ERR_INVALID_ARGUMENT;
    *bytes = layout(batch->num_structures, batch->total_atoms, max_edges).total;
    return MG_OK;
}

mg_status_t mg_cutoff_graph(mg_context_t ctx, const mg_batch_t *batch, float cutoff, const float *cutoff_ps,
                            const mg_opts_t *opts, mg_graph_t *graph, void *ws, size_t ws_bytes, void *stream) {
    return build_and_record(ctx, MG_KIND_CUTOFF, batch, cutoff, cutoff_ps, nullptr, 0, opts, graph, ws, ws_bytes,
                            stream);
}

mg_status_t mg_cutoff_graph_atoms(mg_context_t ctx, const mg_batch_t *batch, const float *cutoff_atom,
                                  const mg_opts_t *opts, mg_graph_t *graph, void *ws, size_t ws_bytes, void *stream) {
    return build_and_record(ctx, KIND_CUTOFF_ATOMS, batch, 0.f, nullptr, cutoff_atom, 0, opts, graph, ws, ws_bytes,
                            stream);
}

mg_status_t mg_knn_graph(mg_context_t ctx, const mg_batch_t *batch, int32_t k, const mg_opts_t *opts,
                         mg_graph_t *graph, void *ws, size_t ws_bytes, void *stream) {
    return build_and_record(ctx, MG_KIND_KNN, batch, 0.f, nullptr, nullptr, k, opts, graph, ws, ws_bytes, stream);
}

mg_status_t mg_update_graph(mg_context_t ctx, const mg_batch_t *batch, mg_graph_t *graph, void *ws, size_t ws_bytes,
                            void *stream) {
    if (!ctx || !graph) return MG_ERR_INVALID_ARGUMENT;
    mg_status_t r = check_batch(batch);
    if (r) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->plans.find((const void *)graph->src);
    if (it == ctx->plans.end()) return MG_ERR_NOT_BUILT;
    Plan &p = it->second;
    if (!same_batch(p.batch, *batch) || !same_graph(p.graph, *graph) || p.ws != ws || p.ws_bytes != ws_bytes)
        return MG_ERR_INVALID_ARGUMENT;  // shapes, pointers or workspace differ from the recorded build
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (st != nullptr && cudaStreamIsCapturing(st, &cap) != cudaSuccess) return MG_ERR_CUDA;
    if (st == nullptr || cap != cudaStreamCaptureStatusNone) {
        // legacy stream or a capture already in progress: enqueue the launches directly
        int n = 0;
        r = enqueue_build(ctx, p.kind, batch, p.cutoff, p.cutoff_ps, p.cutoff_atom, p.k, p.opts, graph, ws,
                          ws_bytes, st, &n);
        ctx->last_launches = n;
        if (p.kind == MG_KIND_CUTOFF)
            ctx->pair_owner[ws] = (const void *)graph->src;
        else
            ctx->pair_owner.erase(ws);
        return r;
    }
    const int which = p.kind == MG_KIND_KNN ? MG_PROF_KNN : MG_PROF_CUTOFF;
    if (p.exec && p.exec_profiled != ctx->prof_on) {
        // recorded under the other profiling setting: record again, with stage events when
        // profiling is on, without them (and with programmatic launches) when it is off
        cudaGraphExecDestroy(p.exec);
        p.exec = nullptr;
    }
    if (!p.exec) {
        // with profiling on, the plan gets its own stage events (created before capture)
        Prof *prof = nullptr;
        if (ctx->prof_on) {
            if (!p.prof.create()) return MG_ERR_CUDA;
            prof = &p.prof;
        }
        cudaGraph_t cg = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MG_ERR_CUDA;
        int n = 0;
        r = enqueue_build(ctx, p.kind, batch, p.cutoff, p.cutoff_ps, p.cutoff_atom, p.k, p.opts, graph, ws,
                          ws_bytes, st, &n, prof);
        const cudaError_t ce = cudaStreamEndCapture(st, &cg);
        if (r) {
            if (cg) cudaGraphDestroy(cg);
            return r;
        }
        if (ce != cudaSuccess || !cg) return MG_ERR_CUDA;
        const cudaError_t ie = cudaGraphInstantiate(&p.exec, cg, 0);
        cudaGraphDestroy(cg);
        if (ie != cudaSuccess) {
            p.exec = nullptr;
            return MG_ERR_CUDA;
        }
        p.launches = n;
        p.exec_profiled = ctx->prof_on;
    }
    if (cudaGraphLaunch(p.exec, st) != cudaSuccess) return MG_ERR_CUDA;
    ctx->last_launches = p.launches;
    if (p.kind == MG_KIND_CUTOFF)
        ctx->pair_owner[ws] = (const void *)graph->src;
    else
        ctx->pair_owner.erase(ws);
    if (p.prof.valid) ctx->last_prof[which] = &p.prof;  // the replay re-records the plan's events
    return MG_OK;
}

__global__ void per_structure_final_kernel(int B, int N, const int64_t *__restrict__ edge_ptr, int64_t capacity,
                                           mg_device_status_t *status) {
    Status *st = reinterpret_cast<Status *>(status);
    const long long tot = edge_ptr[B];
    st->num_edges = (unsigned long long)tot;
    st->required_capacity = (unsigned long long)tot;
    if (tot > capacity) set_error(status, MG_ERR_CAPACITY, -1);
    (void)N;
}

__global__ void edge_ptr_link_kernel(int64_t *__restrict__ edge_ptr, int s, const int64_t *__restrict__ src_ptr,
                                     int hi) {
    edge_ptr[s + 1] = src_ptr[hi];
}

__global__ void add_base_kernel2(int64_t *__restrict__ out, int n, const int64_t *__restrict__ base) {
    const int64_t b = *base;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q <= n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] += b;
}

mg_status_t mg_build_per_structure(mg_context_t ctx, const mg_batch_t *b, int32_t kind, float cutoff, int32_t k,
                                   const int32_t *atom_ptr_host, const mg_opts_t *opts, mg_graph_t *g, void *ws,
                                   size_t ws_bytes, void *stream) {
    const mg_opts_t o = defaults(opts);
    mg_status_t r = check_build_args(ctx, b, o, g);
    if (r) return r;
    if (!atom_ptr_host || (kind != MG_KIND_CUTOFF && kind != MG_KIND_KNN)) return MG_ERR_INVALID_ARGUMENT;
    if (o.knn_keep_ties) return MG_ERR_INVALID_ARGUMENT;  // the comparison build has exact-k KNN only
    if (kind == MG_KIND_CUTOFF && !(cutoff > 0.f)) return MG_ERR_INVALID_ARGUMENT;
    if (kind == MG_KIND_KNN && (k <= 0 || k > KNN_MAX_K)) return MG_ERR_INVALID_ARGUMENT;
    if (kind == MG_KIND_KNN && (int64_t)k * b->total_atoms > g->capacity) return MG_ERR_CAPACITY;
    const int B = b->num_structures, N = b->total_atoms;
    const int64_t me = ws_max_edges(B, N, ws_bytes);
    if (!ws || me < 0) return MG_ERR_WORKSPACE;
    if (g->perm_dst && me < g->capacity) return MG_ERR_WORKSPACE;
    const Work w0 = carve(ws, B, N, me);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int n = 0;
    status_init_kernel<<<1, 1, 0, st>>>(g->status);
    ++n;
    int64_t *src_ptr = g->src_ptr ? g->src_ptr : w0.src_ptr;
    cudaMemsetAsync(g->edge_ptr, 0, sizeof(int64_t), st);
    for (int s = 0; s < B; ++s) {
        const int lo = atom_ptr_host[s], hi = atom_ptr_host[s + 1];
        Work w = w0;
        w.recs = w0.recs + s;  // the structure's record sits at local index 0
        PrepArgs pa{1, hi - lo, b->lattice + 9 * (size_t)s, b->frac, b->atom_ptr + s, cutoff, nullptr,
                    kind == MG_KIND_KNN ? k : 0, o.band_rel, g->status, s, 0, 0, nullptr, nullptr, hi - lo};
        if (launch_prep(pa, w, st)) return MG_ERR_CUDA;
        ++n;
        if (hi - lo >= CELL_MIN_ATOMS) {  // this structure may use a cell list
            if (launch_bins_one(lo, hi, lo + s, b->frac, w, st)) return MG_ERR_CUDA;
            n += 7;
        }
        BuildArgs ba;
        ba.struct_offset = s;
        ba.B = B;
        ba.N = N;
        ba.frac = b->frac;
        ba.atom_ptr = b->atom_ptr;
        ba.schedule = 1;
        ba.collect_stats = o.collect_stats;
        ba.fault_tile = -1;
        ba.g = *g;
        ba.src_ptr = src_ptr;
        ba.knn_k = k;
        ba.band_rel = o.band_rel;
        ba.atom_lo = lo;
        ba.atom_hi = hi;
        if (hi == lo) {
            if (kind == MG_KIND_CUTOFF) {
                edge_ptr_link_kernel<<<1, 1, 0, st>>>(g->edge_ptr, s, g->edge_ptr, s);  // edge_ptr[s+1] = edge_ptr[s]
                ++n;
            }
            continue;
        }
        if (kind == MG_KIND_CUTOFF) {
            if (launch_cutoff_count(ba, w, st)) return MG_ERR_CUDA;
            ScanArgs sa{hi - lo, w.cnt + lo, src_ptr + lo};
            if (launch_scan(sa, w, st)) return MG_ERR_CUDA;
            add_base_kernel2<<<1, 256, 0, st>>>(src_ptr + lo, hi - lo, g->edge_ptr + s);
            edge_ptr_link_kernel<<<1, 1, 0, st>>>(g->edge_ptr, s, src_ptr, hi);
            if (launch_cutoff_write(ba, w, st)) return MG_ERR_CUDA;
            n += 7;
        } else {
            if (launch_knn(ba, w, st)) return MG_ERR_CUDA;
            n += 1;
        }
    }
    BuildArgs fa;
    fa.struct_offset = 0;
    fa.B = B;
    fa.N = N;
    fa.frac = b->frac;
    fa.atom_ptr = b->atom_ptr;
    fa.schedule = 1;
    fa.collect_stats = 0;
    fa.fault_tile = -1;
    fa.g = *g;
    fa.src_ptr = src_ptr;
    fa.knn_k = k;
    fa.band_rel = o.band_rel;
    fa.atom_lo = 0;
    fa.atom_hi = N;
    if (kind == MG_KIND_KNN) {
        if (launch_knn_pointers(fa, w0, st)) return MG_ERR_CUDA;
        ++n;
    }
    per_structure_final_kernel<<<1, 1, 0, st>>>(B, N, g->edge_ptr, g->capacity, g->status);
    ++n;
    if (g->perm_dst) {
        if (kind == MG_KIND_CUTOFF) {
            if (launch_dst_perm_symmetric(fa, w0, st)) return MG_ERR_CUDA;
            ++n;
        } else {
            if (launch_dst_sort(fa, w0, st, &n)) return MG_ERR_CUDA;
        }
    }
    if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_launches = n;
    ctx->pair_owner.erase(ws);  // the per-structure build records no pair table
    return MG_OK;
}

mg_status_t mg_edge_vectors_fwd(mg_context_t ctx, const mg_batch_t *b, const mg_graph_t *g, float *vec, float *len,
                                void *stream) {
    if (!ctx) return MG_ERR_INVALID_ARGUMENT;
    mg_status_t r = check_batch(b);
    if (r) return r;
    if (!g || !g->src_ptr || !g->edge_ptr || !g->dst || !g->offset) return MG_ERR_INVALID_ARGUMENT;
    EdgeVecArgs a{};
    a.B = b->num_structures;
    a.N = b->total_atoms;
    a.lattice = b->lattice;
    a.frac = b->frac;
    a.atom_ptr = b->atom_ptr;
    a.g = *g;
    a.out_vec = vec;
    a.out_len = len;
    Marker mk(ctx, MG_PROF_FWD, static_cast<cudaStream_t>(stream));
    if (launch_edgevec_fwd(a, static_cast<cudaStream_t>(stream))) return MG_ERR_CUDA;
    mk.mark("fwd");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_launches = 1;
    return MG_OK;
}

mg_status_t mg_edge_vectors_bwd(mg_context_t ctx, const mg_batch_t *b, const mg_graph_t *g, const float *grad_vec,
                                const float *grad_len, const float *vec, const float *len, float *grad_frac,
                                float *grad_lattice, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx) return MG_ERR_INVALID_ARGUMENT;
    mg_status_t r = check_batch(b);
    if (r) return r;
    if (!g || !g->src_ptr || !g->edge_ptr || !g->dst || !g->offset || !grad_frac || !grad_lattice)
        return MG_ERR_INVALID_ARGUMENT;
    if (grad_len && (!vec || !len)) return MG_ERR_INVALID_ARGUMENT;
    // A cutoff graph built on this context with one radius per structure is symmetric:
    // its in-edges are found as the reverses of out-edges and no destination order is
    // needed.  Other graphs (KNN, per-atom radii, foreign edge lists) need one.
    // The pair table in the workspace serves it when the last build that used this
    // workspace was this graph's own.
    bool symmetric = false, pairs = false;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->plans.find((const void *)g->src);
        symmetric = it != ctx->plans.end() && it->second.kind == MG_KIND_CUTOFF && same_graph(it->second.graph, *g);
        if (symmetric) {
            auto po = ctx->pair_owner.find(ws);
            pairs = po != ctx->pair_owner.end() && po->second == (const void *)g->src && it->second.ws == ws &&
                    it->second.ws_bytes == ws_bytes;
        } else {
            auto sit = ctx->sym.find((const void *)g->src);
            symmetric = sit != ctx->sym.end() && same_graph(sit->second, *g);
        }
    }
    if (!symmetric && (!g->perm_dst || !g->dst_ptr)) return MG_ERR_INVALID_ARGUMENT;
    const int B = b->num_structures, N = b->total_atoms;
    const int64_t me = ws_max_edges(B, N, ws_bytes);
    if (!ws || me < 0) return MG_ERR_WORKSPACE;
    const Work w = carve(ws, B, N, me);
    EdgeVecArgs a{};
    a.B = B;
    a.N = N;
    a.max_atoms = b->max_atoms;
    a.lattice = b->lattice;
    a.frac = b->frac;
    a.atom_ptr = b->atom_ptr;
    a.g = *g;
    a.grad_vec = grad_vec;
    a.grad_len = grad_len;
    a.vec = vec;
    a.len = len;
    a.grad_frac = grad_frac;
    a.grad_lattice = grad_lattice;
    if (pairs) {
        a.pair_lo = w.pair_lo;
        a.pair_hi = w.pair_hi;
        a.pair_ok = w.pair_ok;
        a.atom_struct = w.atom_struct;
        // the build's prep zeroed the counters: for small batches the lattice reduction
        // joins bwd_sym (one launch less; measured 3.7 us faster at 3.6k atoms, while the
        // fence and count per warp cost more than the launch from 37k atoms up)
        if (N > 0 && N < STAGED_MIN_ATOMS && b->max_atoms > 0 && b->max_atoms <= 1024) a.lat_cnt = w.lat_cnt;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Marker mk(ctx, MG_PROF_BWD, st);
    int n = 0;
    if (symmetric) {
        if (launch_bwd_sym(a, w, st)) return MG_ERR_CUDA;
        mk.mark("bwd_sym");
        n = 2;
        if (a.lat_cnt) {  // lattice gradient already reduced
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->last_launches = 1;
            return MG_OK;
        }
    } else {
        if (launch_bwd_src(a, w, st)) return MG_ERR_CUDA;
        mk.mark("bwd_src");
        if (launch_bwd_dst(a, w, st)) return MG_ERR_CUDA;
        mk.mark("bwd_dst");
        n = 3;
    }
    if (launch_bwd_lat(a, w, st)) return MG_ERR_CUDA;
    mk.mark("bwd_lat");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_launches = n;
    return MG_OK;
}

mg_status_t mg_graph_to_host(mg_context_t ctx, const mg_batch_t *b, const mg_graph_t *g, int64_t num_edges,
                             const mg_graph_host_t *out, void *stream) {
    if (!ctx || !out) return MG_ERR_INVALID_ARGUMENT;
    mg_status_t r = check_batch(b);
    if (r) return r;
    if (!g || num_edges < 0 || num_edges > g->capacity) return MG_ERR_INVALID_ARGUMENT;
    if ((out->status && !g->status) || (out->src && !g->src) || (out->dst && !g->dst) ||
        (out->offset && !g->offset) || (out->vec && !g->vec) || (out->len && !g->len) ||
        (out->edge_ptr && !g->edge_ptr) || (out->src_ptr && !g->src_ptr))
        return MG_ERR_INVALID_ARGUMENT;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t E = (size_t)num_edges;
    struct Copy {
        void *dst;
        const void *src;
        size_t bytes;
    };
    const Copy copies[] = {
        {out->status, g->status, sizeof(mg_device_status_t)},
        {out->src, g->src, E * sizeof(int32_t)},
        {out->dst, g->dst, E * sizeof(int32_t)},
        {out->offset, g->offset, 3 * E * sizeof(int32_t)},
        {out->vec, g->vec, 3 * E * sizeof(float)},
        {out->len, g->len, E * sizeof(float)},
        {out->edge_ptr, g->edge_ptr, ((size_t)b->num_structures + 1) * sizeof(int64_t)},
        {out->src_ptr, g->src_ptr, ((size_t)b->total_atoms + 1) * sizeof(int64_t)},
    };
    for (const Copy &c : copies)
        if (c.dst && c.bytes && cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return MG_ERR_CUDA;
    return MG_OK;
}

mg_status_t mg_triplets(mg_context_t ctx, const mg_batch_t *b, const mg_graph_t *g, int32_t include_self,
                        mg_triplets_t *out, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || !out || !out->status || !out->edge_b || out->capacity < 0 || (include_self != 0 && include_self != 1))
        return MG_ERR_INVALID_ARGUMENT;
    mg_status_t r = check_batch(b);
    if (r) return r;
    if (!g || !g->src_ptr || g->capacity > (int64_t)INT_MAX) return MG_ERR_INVALID_ARGUMENT;
    const int B = b->num_structures, N = b->total_atoms;
    const int64_t me = ws_max_edges(B, N, ws_bytes);
    if (!ws || me < 0) return MG_ERR_WORKSPACE;
    const Work w = carve(ws, B, N, me);
    TripArgs ta{N, g->src_ptr, include_self ? 0 : 1, out->capacity, out->edge_a, out->edge_b, out->trip_ptr,
                out->status};
    int n = 0;
    if (launch_triplets(ta, w, static_cast<cudaStream_t>(stream), &n)) return MG_ERR_CUDA;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_launches = n;
    return MG_OK;
}

mg_status_t mg_symmetrize(mg_context_t ctx, const mg_batch_t *b, const mg_graph_t *in, mg_graph_t *out, void *ws,
                          size_t ws_bytes, void *stream) {
    if (!ctx) return MG_ERR_INVALID_ARGUMENT;
    mg_status_t r = check_batch(b);
    if (r) return r;
    if (!in || !in->src_ptr || !in->perm_dst || !in->dst_ptr || !in->src || !in->dst || !in->offset)
        return MG_ERR_INVALID_ARGUMENT;
    r = check_graph(out, b);
    if (r) return r;
    if (!out->src_ptr || out->src == in->src || out->capacity > (int64_t)INT_MAX) return MG_ERR_INVALID_ARGUMENT;
    const int B = b->num_structures, N = b->total_atoms;
    const int64_t me = ws_max_edges(B, N, ws_bytes);
    if (!ws || me < 0) return MG_ERR_WORKSPACE;
    if (me < in->capacity) return MG_ERR_WORKSPACE;  // per-edge twin counts of the input
    const Work w = carve(ws, B, N, me);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SymArgs sa{B, N, b->lattice, b->frac, b->atom_ptr, *in, *out};
    int n = 0;
    if (launch_symmetrize(sa, w, st, &n)) return MG_ERR_CUDA;
    if (out->perm_dst) {  // symmetric: destination order from reverse runs
        BuildArgs ba;
        ba.B = B;
        ba.N = N;
        ba.g = *out;
        ba.src_ptr = out->src_ptr;
        if (launch_dst_perm_symmetric(ba, w, st)) return MG_ERR_CUDA;
        ++n;
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_launches = n;
    ctx->plans.erase((const void *)out->src);  // no longer the graph of a recorded build
    ctx->sym[(const void *)out->src] = *out;
    return MG_OK;
}

mg_status_t mg_cutoff_graph_noalloc(mg_context_t ctx, const mg_batch_t *b, float cutoff, const mg_opts_t *opts,
                                    mg_graph_t *g, void *stream) {
    // Same launch sequence as mg_cutoff_graph, with the fixed scratch array as workspace.
    // Nothing here allocates device memory; the sequence's own memset nodes clear the
    // scratch words that must start at zero (work-queue counters, histogram cursors).
    const mg_opts_t o = defaults(opts);
    mg_status_t r = check_build_args(ctx, b, o, g);
    if (r) return r;
    if (!(cutoff > 0.f)) return MG_ERR_INVALID_ARGUMENT;
    const size_t need = layout(b->num_structures, b->total_atoms, g->perm_dst ? g->capacity : 0).total;
    if (need > (size_t)MG_NOALLOC_SCRATCH_BYTES) return MG_ERR_WORKSPACE;  // batch too large for the array
    void *scratch = nullptr;
    r = noalloc_scratch(&scratch);
    if (r) return r;
    int launches = 0;
    r = enqueue_build(ctx, MG_KIND_CUTOFF, b, cutoff, nullptr, nullptr, 0, o, g, scratch, need,
                      static_cast<cudaStream_t>(stream), &launches);
    if (r) return r;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->last_launches = launches;
    // The buffers now hold a graph that no recorded build describes: forget an earlier
    // workspace build into them (its plan would replay another radius, and its pair table
    // indexes another edge set), and record the graph as symmetric, so that the backward
    // finds reverse edges by search rather than through a pair table.
    const void *key = (const void *)g->src;
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        Plan &p = it->second;
        if (p.exec) cudaGraphExecDestroy(p.exec);
        const int which = p.kind == MG_KIND_KNN ? MG_PROF_KNN : MG_PROF_CUTOFF;
        if (ctx->last_prof[which] == &p.prof) ctx->last_prof[which] = nullptr;
        p.prof.destroy();
        ctx->plans.erase(it);
    }
    for (auto po = ctx->pair_owner.begin(); po != ctx->pair_owner.end();) {
        if (po->second == key) po = ctx->pair_owner.erase(po);
        else ++po;
    }
    ctx->sym[key] = *g;
    return MG_OK;
}

mg_status_t mg_autotune(mg_context_t ctx, const mg_batch_t *b, int32_t kind, float cutoff, int32_t k, mg_graph_t *g,
                        void *ws, size_t ws_bytes, void *stream) {
    if (!ctx || (kind != MG_KIND_CUTOFF && kind != MG_KIND_KNN)) return MG_ERR_INVALID_ARGUMENT;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return MG_ERR_CUDA;
    // KNN: the warp enumeration on a flat grid (1) or a persistent queue (2), or the
    // pair-lane KNN (5); cutoff graphs: the one-pass build (3), the staged build (4) or the
    // pair-lane build (5), the last two only when the workspace can stage the capacity
    int cands[4], nc = 0;
    if (kind == MG_KIND_KNN) {
        cands[nc++] = 1;
        cands[nc++] = 2;
        cands[nc++] = 5;
    } else {
        cands[nc++] = 3;
        cands[nc++] = 6;
        if (g && ws_max_edges(b->num_structures, b->total_atoms, ws_bytes) >= g->capacity) {
            cands[nc++] = 4;
            cands[nc++] = 5;
        }
    }
    float best = 1e30f;
    int best_s = cands[0];
    for (int ci = 0; ci < nc; ++ci) {
        const int sched = cands[ci];
        mg_opts_t o = defaults(nullptr);
        o.schedule = sched;
        float tot = 0.f;
        // the build once with this schedule (which records it), then replays of the
        // recorded plan, as a rebuild inside a loop runs (mg_update_graph); the first
        // replay records the CUDA graph and is not counted
        mg_status_t r0 = kind == MG_KIND_CUTOFF ? mg_cutoff_graph(ctx, b, cutoff, nullptr, &o, g, ws, ws_bytes, stream)
                                                : mg_knn_graph(ctx, b, k, &o, g, ws, ws_bytes, stream);
        if (r0) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return r0;
        }
        for (int rep = 0; rep < 4; ++rep) {
            mg_status_t r;
            cudaEventRecord(e0, st);
            r = mg_update_graph(ctx, b, g, ws, ws_bytes, stream);
            cudaEventRecord(e1, st);
            if (r) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return r;
            }
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tot += ms;  // first repetition warms up
        }
        if (tot < best) {
            best = tot;
            best_s = sched;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->tuned[kind - 1][size_class(b)] = best_s;
    return MG_OK;
}

}  // extern "C"

namespace {

bool same_step(const mg_context::StepRec &r, const mg_step_t &p) {
    const mg_step_t &q = r.st;
    bool same = q.frac_host == p.frac_host && q.lattice_host == p.lattice_host && q.atom_ptr_host == p.atom_ptr_host &&
                q.grad_vec == p.grad_vec && q.grad_len == p.grad_len && q.vec == p.vec && q.len == p.len &&
                q.grad_frac == p.grad_frac && q.grad_lattice == p.grad_lattice && q.vec_host == p.vec_host &&
                q.len_host == p.len_host && q.grad_frac_host == p.grad_frac_host &&
                q.grad_lattice_host == p.grad_lattice_host && q.capture == p.capture && same_batch(r.batch, *p.batch);
    for (int k = 0; k < 3; ++k) same = same && q.stream[k] == p.stream[k];
    for (int g = 0; g < 2; ++g) {
        same = same && (q.graph[g] != nullptr) == (p.graph[g] != nullptr) && q.ws[g] == p.ws[g] &&
               q.ws_bytes[g] == p.ws_bytes[g] && q.host_edges[g] == p.host_edges[g] &&
               (q.graph_host[g] != nullptr) == (p.graph_host[g] != nullptr);
        if (same && p.graph[g]) same = same_graph(r.g[g], *p.graph[g]);
        if (same && p.graph_host[g]) same = std::memcmp(&r.h[g], p.graph_host[g], sizeof(mg_graph_host_t)) == 0;
    }
    return same;
}

mg_status_t enqueue_step(mg_context_t ctx, const mg_step_t *p) {
    const mg_batch_t *b = p->batch;
    mg_status_t r = MG_OK;
    cudaStream_t s0 = static_cast<cudaStream_t>(p->stream[0]);
    cudaStream_t s1 = p->stream[1] ? static_cast<cudaStream_t>(p->stream[1]) : s0;
    cudaStream_t s2 = p->stream[2] ? static_cast<cudaStream_t>(p->stream[2]) : s0;
    cudaEvent_t ev_in = ctx->step_ev[0], ev_g0 = ctx->step_ev[1], ev_done = ctx->step_ev[2], ev_fwd = ctx->step_ev[3];
    // 1. inputs
    const size_t N = (size_t)b->total_atoms, B = (size_t)b->num_structures;
    if (p->frac_host && N &&
        cudaMemcpyAsync(const_cast<float *>(b->frac), p->frac_host, 12 * N, cudaMemcpyHostToDevice, s0) != cudaSuccess)
        return MG_ERR_CUDA;
    if (p->lattice_host && cudaMemcpyAsync(const_cast<float *>(b->lattice), p->lattice_host, 36 * B,
                                           cudaMemcpyHostToDevice, s0) != cudaSuccess)
        return MG_ERR_CUDA;
    if (p->atom_ptr_host && cudaMemcpyAsync(const_cast<int32_t *>(b->atom_ptr), p->atom_ptr_host, 4 * (B + 1),
                                            cudaMemcpyHostToDevice, s0) != cudaSuccess)
        return MG_ERR_CUDA;
    // 2. the second graph on its own stream, its copy behind it
    if (p->graph[1]) {
        if (s1 != s0) {
            if (cudaEventRecord(ev_in, s0) != cudaSuccess || cudaStreamWaitEvent(s1, ev_in, 0) != cudaSuccess)
                return MG_ERR_CUDA;
        }
        r = mg_update_graph(ctx, b, p->graph[1], p->ws[1], p->ws_bytes[1], s1);
        if (r) return r;
        if (p->graph_host[1]) {
            r = mg_graph_to_host(ctx, b, p->graph[1], p->host_edges[1], p->graph_host[1], s1);
            if (r) return r;
        }
    }
    // 3. the first graph; its copy beside the rest of the step
    r = mg_update_graph(ctx, b, p->graph[0], p->ws[0], p->ws_bytes[0], s0);
    if (r) return r;
    if (p->graph_host[0]) {
        if (s2 != s0) {
            if (cudaEventRecord(ev_g0, s0) != cudaSuccess || cudaStreamWaitEvent(s2, ev_g0, 0) != cudaSuccess)
                return MG_ERR_CUDA;
        }
        r = mg_graph_to_host(ctx, b, p->graph[0], p->host_edges[0], p->graph_host[0], s2);
        if (r) return r;
    }
    // 4. edge vectors and their backward, results out
    const size_t E = p->host_edges[0] > 0 ? (size_t)p->host_edges[0] : 0;
    if (p->vec || p->len) {
        r = mg_edge_vectors_fwd(ctx, b, p->graph[0], p->vec, p->len, s0);
        if (r) return r;
    }
    // the vectors and lengths go out behind the forward, on the copy stream (after the
    // graph's rows), while the backward runs: the host link stays busy through the step
    cudaStream_t sv = s2 != s0 ? s2 : s0;
    if (sv != s0 && (p->vec_host || p->len_host)) {
        if (cudaEventRecord(ev_fwd, s0) != cudaSuccess || cudaStreamWaitEvent(sv, ev_fwd, 0) != cudaSuccess)
            return MG_ERR_CUDA;
    }
    if (p->vec_host && p->vec && E && cudaMemcpyAsync(p->vec_host, p->vec, 12 * E, cudaMemcpyDeviceToHost, sv) != cudaSuccess)
        return MG_ERR_CUDA;
    if (p->len_host && p->len && E && cudaMemcpyAsync(p->len_host, p->len, 4 * E, cudaMemcpyDeviceToHost, sv) != cudaSuccess)
        return MG_ERR_CUDA;
    if (p->grad_frac && p->grad_lattice) {
        r = mg_edge_vectors_bwd(ctx, b, p->graph[0], p->grad_vec, p->grad_len, p->vec, p->len, p->grad_frac,
                                p->grad_lattice, p->ws[0], p->ws_bytes[0], s0);
        if (r) return r;
    }
    struct Out {
        void *dst;
        const void *src;
        size_t bytes;
    };
    const Out outs[] = {{p->grad_frac_host, p->grad_frac, 12 * N},
                        {p->grad_lattice_host, p->grad_lattice, 36 * B}};
    for (const Out &o : outs)
        if (o.dst && o.src && o.bytes && cudaMemcpyAsync(o.dst, o.src, o.bytes, cudaMemcpyDeviceToHost, s0) != cudaSuccess)
            return MG_ERR_CUDA;
    // 5. join
    for (cudaStream_t sx : {s1, s2}) {
        if (sx == s0) continue;
        if (cudaEventRecord(ev_done, sx) != cudaSuccess || cudaStreamWaitEvent(s0, ev_done, 0) != cudaSuccess)
            return MG_ERR_CUDA;
    }
    return MG_OK;
}

}  // namespace

extern "C" {

mg_status_t mg_graph_step(mg_context_t ctx, const mg_step_t *p) {
    if (!ctx || !p || !p->batch || !p->graph[0] || (p->capture != 0 && p->capture != 1)) return MG_ERR_INVALID_ARGUMENT;
    mg_status_t r = check_batch(p->batch);
    if (r) return r;
    cudaStream_t s0 = static_cast<cudaStream_t>(p->stream[0]);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (auto &e : ctx->step_ev)
            if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return MG_ERR_CUDA;
        if (p->capture && ctx->step.exec && same_step(ctx->step, *p))
            return cudaGraphLaunch(ctx->step.exec, s0) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
    }
    if (!p->capture || !s0) return enqueue_step(ctx, p);  // the legacy stream cannot be captured
    // record the step as one CUDA graph (the streams it forks to join the capture through
    // its events), then launch it
    if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MG_ERR_CUDA;
    r = enqueue_step(ctx, p);
    cudaGraph_t cg = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s0, &cg);
    if (r || ce != cudaSuccess || !cg) {
        if (cg) cudaGraphDestroy(cg);
        return r ? r : MG_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, cg, 0);
    cudaGraphDestroy(cg);
    if (ie != cudaSuccess) return MG_ERR_CUDA;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->step.exec) cudaGraphExecDestroy(ctx->step.exec);
    ctx->step = mg_context::StepRec();
    ctx->step.st = *p;
    ctx->step.batch = *p->batch;
    for (int g = 0; g < 2; ++g) {
        if (p->graph[g]) ctx->step.g[g] = *p->graph[g];
        if (p->graph_host[g]) ctx->step.h[g] = *p->graph_host[g];
    }
    ctx->step.exec = exec;
    return cudaGraphLaunch(exec, s0) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

mg_status_t mg_measure_fp_peaks(mg_context_t ctx, void *sink, double *fp32_tflops, double *fp64_tflops,
                                void *stream) {
    if (!ctx || !sink || !fp32_tflops || !fp64_tflops) return MG_ERR_INVALID_ARGUMENT;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MG_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MG_ERR_CUDA;
    }
    int per_sm = 0;
    const int blocks_f = (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<float>, 256, 0) ==
                          cudaSuccess && per_sm > 0 ? per_sm : 8) * ctx->sms;
    const int blocks_d = (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<double>, 256, 0) ==
                          cudaSuccess && per_sm > 0 ? per_sm : 8) * ctx->sms;
    auto best_rate = [&](bool dbl, int iters, int blocks, double *out) -> bool {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {  // the first repetition warms up
            cudaEventRecord(e0, st);
            if (dbl)
                fma_peak_kernel<double><<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7, static_cast<double *>(sink));
            else
                fma_peak_kernel<float><<<blocks, 256, 0, st>>>(iters, 0.9999f, 1e-4f, static_cast<float *>(sink));
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return false;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        const double flops = 2.0 * PEAK_CHAINS * (double)iters * 256.0 * blocks;
        *out = flops / (best * 1e-3) / 1e12;
        return true;
    };
    const bool ok = best_rate(false, 4096, blocks_f, fp32_tflops) && best_rate(true, 64, blocks_d, fp64_tflops);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok && cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

mg_status_t mg_tuned_table(mg_context_t ctx, int32_t table[2][MG_SIZE_CLASSES], int32_t set) {
    if (!ctx || !table || (set != 0 && set != 1)) return MG_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (int k = 0; k < 2; ++k)
        for (int c = 0; c < MG_SIZE_CLASSES; ++c) {
            if (set && (table[k][c] < 0 || table[k][c] > 6)) return MG_ERR_INVALID_ARGUMENT;
        }
    for (int k = 0; k < 2; ++k)
        for (int c = 0; c < MG_SIZE_CLASSES; ++c) {
            if (set) ctx->tuned[k][c] = table[k][c];
            else table[k][c] = ctx->tuned[k][c];
        }
    return MG_OK;
}

mg_status_t mg_profile_enable(mg_context_t ctx, int32_t on) {
    if (!ctx) return MG_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (on)  // create every event up front: nothing is created while a plan is captured
        for (auto &p : ctx->prof)
            for (auto &e : p.ev)
                if (!e && cudaEventCreate(&e) != cudaSuccess) return MG_ERR_CUDA;
    ctx->prof_on = on != 0;
    return MG_OK;
}

int32_t mg_stage_times(mg_context_t ctx, int32_t which, int32_t max_stages, const char **names, float *ms) {
    if (!ctx || which < 0 || which > 3) return -1;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->last_prof[which]) return -1;
    const Prof &p = *ctx->last_prof[which];
    if (!p.valid || p.n < 2) return -1;
    if (cudaEventSynchronize(p.ev[p.n - 1]) != cudaSuccess) return -1;
    const int stages = p.n - 1;
    for (int q = 0; q < stages && q < max_stages; ++q) {
        float t = 0.f;
        cudaEventElapsedTime(&t, p.ev[q], p.ev[q + 1]);
        if (names) names[q] = p.name[q + 1];
        if (ms) ms[q] = t;
    }
    return stages;
}

int64_t mg_last_launch_count(mg_context_t ctx) {
    if (!ctx) return -1;
    std::lock_guard<std::mutex> lk(ctx->mu);
    return ctx->last_launches;
}

}  // extern "C"
