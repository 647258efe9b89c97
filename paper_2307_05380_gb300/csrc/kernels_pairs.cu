// Pair-lane cutoff build (Def. 3, Sec. 2.1) for large batches on sm_103a.
//
// The evaluated area of Alg. 1 is, per pair of atoms (i, j), the box of cell offsets t
// with |x_j,k - x_i,k + t_k| <= c / d_k on every axis (d_k the interplanar spacing): every
// image closer than c lies in it.  In crystal batches almost every pair's box is small
// (at most 64 cells), so here one lane owns one (source, target) pair and evaluates its
// whole box: FP32 distance, FP64 canonical re-test in the band, the pair's edges marked
// in a 64-bit mask.  Lanes are grouped G per source (G the smallest power of two >= the
// structure's atom count, at most 32), so a warp covers 32 / G sources of one structure
// and loops over its targets in chunks of G.  Lane order is target order and each lane's
// mask is in offset order, so a scan of the mask counts gives every edge its canonical
// position.
//
//   plan   each structure's work items (source groups; one item per source for
//          structures scanned by the warp enumeration) are bucketed by cost class and
//          laid out heaviest first (a cost-sorted work list)
//   stage  a persistent grid pulls the items: masks, per-source counts, then the (j, t)
//          keys of the item's sources at their canonical positions in one slot range of
//          the staging area (one atomic add per item)
//   scan   of the counts: src_ptr, edge_ptr, edge count and capacity check
//   emit   a thread per edge row writes src, dst, t, vec and len from the staged key
//          (the staged build's emit kernel), sources that did not fit are enumerated
//          again
//
// Structures whose boxes are larger, that use a cell list or whose offsets exceed the
// packed key are scanned by the warp enumeration of mg_enum.cuh inside the same passes.
#include "mg_build.cuh"
#include "mg_device.cuh"
#include "mg_launch.h"

namespace mg {

constexpr int PAIR_WARPS = 4;
constexpr int PLAN_THREADS = 1024;

// ============================================================================ plan

// One block: histogram of work items by cost class (classes 32..63 for structures of
// the warp enumeration, 0..31 for pair-lane ones), class bases with the warp-enumeration
// items first and each kind heaviest first, and the first slot of every structure's items
// (within a class in arrival order: the order of equally costly items does not affect
// any output).  queue[8] gets the total, queue[9] the number of warp-enumeration items.
__global__ void __launch_bounds__(PLAN_THREADS) pair_plan_kernel(int B, const int32_t *__restrict__ plan_items,
                                                                 const int32_t *__restrict__ plan_class,
                                                                 int32_t *__restrict__ item_base,
                                                                 unsigned int *__restrict__ queue) {
    __shared__ int hist[64], base[64];
    if (threadIdx.x < 64) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < B; s += PLAN_THREADS) atomicAdd(&hist[plan_class[s]], plan_items[s]);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int c = 63; c >= 0; --c) {
            base[c] = run;
            run += hist[c];
            if (c == 32) queue[9] = (unsigned)run;
        }
        queue[8] = (unsigned)run;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < B; s += PLAN_THREADS) item_base[s] = atomicAdd(&base[plan_class[s]], plan_items[s]);
}

// A warp per structure writes its items (structure, item index) at its slots.
__global__ void __launch_bounds__(256) pair_fill_kernel(int B, const int32_t *__restrict__ plan_items,
                                                        const int32_t *__restrict__ item_base, int2 *__restrict__ items) {
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= B) return;
    const int n = plan_items[s], b0 = item_base[s];
    for (int q = lane_id(); q < n; q += 32) items[b0 + q] = make_int2(s, q);
}

// ============================================================================ pair boxes

// Constants of one structure that the lanes keep in registers.
struct PairStruct {
    float L[9];
    float reach[3];       // c / d_k plus the structure's margin: reach of the box along each axis
    float thr_lo, thr_hi; // FP32 d2 below thr_lo: edge; above thr_hi: not; between: FP64 test
    double rr;            // canonical squared cutoff
    int begin, n;
    int G, spw;           // lanes per source, sources per warp
    int B1, B2;           // largest box extents along L_1 and L_2: the strides of a pair's mask
};

__device__ __forceinline__ void load_pair_struct(PairStruct &P, const StructRec &R) {
#pragma unroll
    for (int q = 0; q < 9; ++q) P.L[q] = R.L[q];
#pragma unroll
    for (int k = 0; k < 3; ++k) P.reach[k] = R.reach[k];
    P.thr_lo = R.thr_lo;
    P.thr_hi = R.thr_hi;
    P.rr = R.rr;
    P.begin = R.atom_begin;
    P.n = R.n_atoms;
    int G = 1;
    while (G < P.n && G < 32) G <<= 1;
    P.G = G;
    P.spw = 32 / G;
    P.B2 = R.pl & 255;
    P.B1 = (R.pl >> 8) & 255;
}

// The canonical FP64 test of one candidate in the band, out of line: inlined, the
// compiler hoists its float-to-double conversions out of the branch into every pair,
// and on this GPU the FP64 pipe runs at a small fraction of the FP32 rate.
__device__ __noinline__ bool band_is_edge(const StructRec *__restrict__ rec, float xi0, float xi1, float xi2,
                                          float xj0, float xj1, float xj2, float t0, float t1, float t2) {
    return canon_d2(rec->L, xi0, xi1, xi2, xj0, xj1, xj2, (int)t0, (int)t1, (int)t2) < rec->rr;
}

// The offset box of pair (i, j): the integers t_k with |x_j,k - x_i,k + t_k| <= reach_k,
// lo[k] .. lo[k] + nn[k] - 1 on axis k, and the mask of its edges, bit q0 nn1 nn2 + q1 nn2
// + q2 for offset lo + (q0, q1, q2).  FP32 distances come from the same fused operations
// in the same order as the warp enumeration, so the structure's FP32 error bound (the
// re-test band) holds; candidates inside the band take the canonical FP64 test.  Bounds
// and offsets stay in FP32 (exact for these small integers), so that the loop converts
// nothing.  A box larger than the mask cannot occur for a structure marked pair-lane (its
// record bounds every pair's box); if it did, the box would be left out and
// MG_ERR_INTERNAL reported.
struct PairBox {
    float lo[3], nn[3];
};

// Small integers in floats by exponent alignment (adding 1.5 * 2^23 moves the value's
// integer part into the low mantissa bits, rounded to nearest): exact for |v| < 2^22.
// Conversions and float rounding to integers run on a low-rate pipe of this GPU; these
// use additions and compares only.
__device__ __forceinline__ float frnd(float v) { return __fsub_rn(__fadd_rn(v, 12582912.0f), 12582912.0f); }
__device__ __forceinline__ float ffloor(float v) {
    const float r = frnd(v);
    return r > v ? __fsub_rn(r, 1.0f) : r;
}
__device__ __forceinline__ float fceil(float v) {
    const float r = frnd(v);
    return r < v ? __fadd_rn(r, 1.0f) : r;
}
__device__ __forceinline__ int fint(float v) { return __float_as_int(__fadd_rn(v, 12582912.0f)) - 0x4B400000; }
__device__ __forceinline__ float ifloat(int v) { return __fsub_rn(__int_as_float(v + 0x4B400000), 12582912.0f); }

__device__ __forceinline__ void pair_box(const PairStruct &P, bool ok, float xi0, float xi1, float xi2, float xj0,
                                         float xj1, float xj2, PairBox &bx) {
    const float dx[3] = {__fsub_rn(xj0, xi0), __fsub_rn(xj1, xi1), __fsub_rn(xj2, xi2)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        bx.lo[k] = fceil(__fsub_rn(-P.reach[k], dx[k]));
        const float hi = ffloor(__fsub_rn(P.reach[k], dx[k]));
        bx.nn[k] = ok ? fmaxf(0.0f, __fadd_rn(__fsub_rn(hi, bx.lo[k]), 1.0f)) : 0.0f;
    }
}


// The cells of one row (t0, t1) of a pair's box: U offsets t2 = lo2 + q (U the
// structure's largest extent along L_2, so every lane runs the same unrolled code), FP32
// distances from the row base b.  Returns the bits of the cells certainly inside and
// sets `le` to the bits of those at most at the band's upper threshold; cells past the
// pair's extent are masked by the caller.
template <int U>
__device__ __forceinline__ unsigned row_cells(const PairStruct &P, float bx_, float by_, float bz_, float lo2,
                                              unsigned &le) {
    unsigned in = 0u, lo_hi = 0u;
#pragma unroll
    for (int q = 0; q < U; ++q) {
        const float ft2 = __fadd_rn(lo2, (float)q);
        const float vx = __fmaf_rn(ft2, P.L[6], bx_);
        const float vy = __fmaf_rn(ft2, P.L[7], by_);
        const float vz = __fmaf_rn(ft2, P.L[8], bz_);
        const float d2 = __fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx)));
        if (d2 < P.thr_lo) in |= 1u << q;
        if (d2 <= P.thr_hi) lo_hi |= 1u << q;
    }
    le = lo_hi;
    return in;
}

// U beyond the unrolled sizes: the same cells in a loop (up to 32 cells per row).
__device__ __forceinline__ unsigned row_cells_loop(const PairStruct &P, float bx_, float by_, float bz_, float lo2,
                                                   int n2, unsigned &le) {
    unsigned in = 0u, lo_hi = 0u;
    float ft2 = lo2;
    for (int q = 0; q < n2; ++q, ft2 = __fadd_rn(ft2, 1.0f)) {
        const float vx = __fmaf_rn(ft2, P.L[6], bx_);
        const float vy = __fmaf_rn(ft2, P.L[7], by_);
        const float vz = __fmaf_rn(ft2, P.L[8], bz_);
        const float d2 = __fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx)));
        if (d2 < P.thr_lo) in |= 1u << q;
        if (d2 <= P.thr_hi) lo_hi |= 1u << q;
    }
    le = lo_hi;
    return in;
}

// The pair's box and the mask of its edges: rows (t0, t1) in order as one flat loop (a
// warp runs as many rows as its busiest lane); the cell lo + (q0, q1, q2) is bit
// (q0 B1 + q1) B2 + q2, with the structure's largest extents as strides, so that the
// decode divides by warp-uniform numbers.  Cells in the band take the canonical FP64
// test (rare); the source's own cell (i, i, 0) is cleared once per pair.
template <int U>
__device__ __forceinline__ unsigned long long pair_box_mask(const PairStruct &P, const StructRec *__restrict__ rec,
                                                            bool ok, int i_loc, int j_loc, float xi0, float xi1,
                                                            float xi2, float3 pi, float xj0, float xj1, float xj2,
                                                            float4 pj, PairBox &bx, mg_device_status_t *status,
                                                            unsigned long long &nre) {
    pair_box(P, ok, xi0, xi1, xi2, xj0, xj1, xj2, bx);
    // more cells than the mask holds, or a row longer than the unrolled code: cannot
    // happen for a pair-lane structure (its record bounds them)
    const int B2 = U > 0 ? U : P.B2, B1 = P.B1;
    if (bx.nn[2] > (float)B2 || bx.nn[1] > (float)B1 || __fmul_rn(bx.nn[0], (float)(B1 * B2)) > (float)PL_BOX_MAX) {
        set_error(status, MG_ERR_INTERNAL, -1);
        bx.nn[0] = 0.0f;
    }
    const float ax = __fsub_rn(pj.x, pi.x), ay = __fsub_rn(pj.y, pi.y), az = __fsub_rn(pj.z, pi.z);
    const int n2 = fint(bx.nn[2]);
    const unsigned rowmask = n2 >= 32 ? ~0u : (1u << n2) - 1u;
    const float rows = __fmul_rn(bx.nn[0], bx.nn[1]);
    const float e1 = __fadd_rn(bx.lo[1], bx.nn[1]);
    const int skip = (B1 - fint(bx.nn[1])) * B2;  // stride from a row's end to the next t0
    unsigned long long mask = 0ull;
    float ft0 = bx.lo[0], ft1 = bx.lo[1];
    int shift = 0;
    for (float r = 0.0f; r < rows; r = __fadd_rn(r, 1.0f), shift += B2) {
        // row base b = a + t0 L0 + t1 L1, then v = b + t2 L2
        const float bx_ = __fmaf_rn(ft1, P.L[3], __fmaf_rn(ft0, P.L[0], ax));
        const float by_ = __fmaf_rn(ft1, P.L[4], __fmaf_rn(ft0, P.L[1], ay));
        const float bz_ = __fmaf_rn(ft1, P.L[5], __fmaf_rn(ft0, P.L[2], az));
        unsigned le;
        unsigned in = U > 0 ? row_cells<(U > 0 ? U : 1)>(P, bx_, by_, bz_, bx.lo[2], le)
                            : row_cells_loop(P, bx_, by_, bz_, bx.lo[2], n2, le);
        in &= rowmask;
        unsigned band = (le & rowmask) & ~in;
        while (band) {  // the band: canonical FP64 distance decides
            const int q = __ffs(band) - 1;
            band &= band - 1;
            if (band_is_edge(rec, xi0, xi1, xi2, xj0, xj1, xj2, ft0, ft1, __fadd_rn(bx.lo[2], (float)q)))
                in |= 1u << q;
            ++nre;
        }
        mask |= (unsigned long long)in << shift;
        ft1 = __fadd_rn(ft1, 1.0f);
        if (ft1 >= e1) {
            ft1 = bx.lo[1];
            ft0 = __fadd_rn(ft0, 1.0f);
            shift += skip;
        }
    }
    if (i_loc == j_loc && mask) {  // (i, i, 0) is not an edge: the cell of offset 0, if in the box
        const int z0 = -fint(bx.lo[0]), z1 = -fint(bx.lo[1]), z2 = -fint(bx.lo[2]);
        if (z0 >= 0 && z0 < fint(bx.nn[0]) && z1 >= 0 && z1 < fint(bx.nn[1]) && z2 >= 0 && z2 < n2)
            mask &= ~(1ull << ((z0 * B1 + z1) * B2 + z2));
    }
    return mask;
}

// A pair's box origin as one word: lo_k + 512 in 10 bits each (the extents are the
// structure's strides).
__device__ __forceinline__ unsigned pack_box(const PairBox &bx) {
    return pack_t(fint(bx.lo[0]), fint(bx.lo[1]), fint(bx.lo[2]));
}

// The next work item of this warp's pass (queue word `which`), or -1 when the list is done.
__device__ __forceinline__ int next_item(unsigned int *queue, int which, int total) {
    unsigned int v = 0;
    if (lane_id() == 0) v = atomicAdd(&queue[which], 1u);
    v = __shfl_sync(FULL, v, 0);
    return (int)v < total ? (int)v : -1;
}

// Structures outside the pair-lane scan: one source by the warp enumeration (an unusable
// structure reports its error at its first atom and counts zero), its keys staged in
// shared memory and then copied to the staging area at a slot taken with one atomic add
// (-1: the keys did not fit, and the spill kernel enumerates the source again).
__device__ __forceinline__ void warp_source_stage(const BuildArgs &a, const Work &w, int i, unsigned long long *keys) {
    const int lane = lane_id();
    SrcScan c;
    int m = 0;
    bool spill = false;
    if (source_setup<false>(a, w, i, c)) m = scan_source<false>(a, w, c, keys, nullptr, spill);
    long long off = -1;
    if (!spill && m > 0) {
        if (lane == 0) off = (long long)atomicAdd(w.stage_ctr, (unsigned long long)m);
        off = __shfl_sync(FULL, off, 0);
        if (off + m <= w.max_edges) {
            for (int q = lane; q < m; q += 32) w.stage[off + q] = keys[q];
        } else {
            spill = true;  // staging area full (more edges than the workspace covers)
            if (a.write_pairs && lane == 0) w.pair_ok[c.s] = 0;
        }
    }
    if (lane == 0) {
        w.cnt[i] = m;
        w.stage_off[i] = spill ? -1 : off;
        if (spill && m > 0) note_spill(w.spill_list, w.queue, i);
    }
    __syncwarp();
}

// ============================================================================ stage pass

// The warp-enumeration items (the front of the work list), one source each.
__global__ void __launch_bounds__(PAIR_WARPS * 32, 2) pair_legacy_kernel(const __grid_constant__ BuildArgs a,
                                                                          const __grid_constant__ Work w) {
    __shared__ unsigned long long keys_all[PAIR_WARPS][BUILD_CAP];
    unsigned long long *keys = keys_all[threadIdx.x >> 5];
    const int total = (int)w.queue[9];
    for (int it = next_item(w.queue, 6, total); it >= 0; it = next_item(w.queue, 6, total)) {
        const int2 item = w.items[it];
        warp_source_stage(a, w, w.recs[item.x].atom_begin + item.y, keys);
    }
}

constexpr int MASK_CHUNKS = PL_MAX_ATOMS / 32;  // target chunks of a source: masks and boxes kept in shared memory

// Phase 1 of a pair-lane item: every chunk of G targets, each lane's pair mask and packed
// box into shared memory; returns the lane's edge count and the number of chunks.
template <int U>
__device__ __forceinline__ int pair_masks(const PairStruct &P, const StructRec *__restrict__ rec, const BuildArgs &a,
                                          const Work &w, int jg, int i_loc, bool src_ok, float xi0, float xi1,
                                          float xi2, float3 pi, unsigned long long *buf, unsigned *boxes,
                                          int &nchunks, unsigned long long &nre, unsigned long long &ncand) {
    const int lane = lane_id();
    int cnt = 0;
    nchunks = 0;
    for (int jb = 0; jb < P.n; jb += P.G, ++nchunks) {
        const int j_loc = jb + jg;
        const bool ok = src_ok && j_loc < P.n;
        const int64_t jr = (int64_t)P.begin + (ok ? j_loc : 0);
        PairBox bx;
        const unsigned long long mask =
            pair_box_mask<U>(P, rec, ok, i_loc, j_loc, xi0, xi1, xi2, pi, a.frac[3 * jr], a.frac[3 * jr + 1],
                             a.frac[3 * jr + 2], w.pos[jr], bx, a.g.status, nre);
        buf[32 * nchunks + lane] = mask;
        boxes[32 * nchunks + lane] = mask ? pack_box(bx) : 0u;
        cnt += __popcll(mask);
        if (a.collect_stats) ncand += (unsigned long long)(bx.nn[0] * bx.nn[1] * bx.nn[2]);
    }
    return cnt;
}

// A persistent grid pulls the work items.  A pair-lane item: every lane evaluates its
// pair's box for each target chunk (mask and box kept in shared memory), each source's
// count is summed over its lanes, the item's keys take one slot range of the staging
// area (one atomic add), and every lane writes its pairs' keys there at their canonical
// positions: the source's start, plus its edges in earlier chunks, plus the edges of
// the pairs before it in this chunk.  cnt[i] and stage_off[i] go to every source, as
// from the staged build, whose count scan and emit kernel finish the graph.  8 blocks of 4
// warps per SM (64 registers, a few spilled values; 6 KB of shared memory per warp):
// 0.869 ms at 8192 structures against 0.901 at 6 blocks and 80 registers.
__global__ void __launch_bounds__(PAIR_WARPS * 32, 8) pair_stage_kernel(const __grid_constant__ BuildArgs a,
                                                                         const __grid_constant__ Work w) {
    __shared__ unsigned long long mask_all[PAIR_WARPS][32 * MASK_CHUNKS];  // pair masks by chunk and lane
    __shared__ unsigned box_all[PAIR_WARPS][32 * MASK_CHUNKS];             // their packed box origins
    const int wid = threadIdx.x >> 5, lane = lane_id();
    unsigned long long *buf = mask_all[wid];
    unsigned *boxes = box_all[wid];
    const int first = (int)w.queue[9], total = (int)w.queue[8] - first;
    unsigned long long nre = 0, ncand = 0;
    for (int it = next_item(w.queue, 7, total); it >= 0; it = next_item(w.queue, 7, total)) {
        const int2 item = w.items[first + it];
        const StructRec &R = w.recs[item.x];
        PairStruct P;
        load_pair_struct(P, R);
        const int G = P.G;
        const int g = lane / G, jg = lane % G;
        const int i_loc = item.y * P.spw + g;
        const bool src_ok = i_loc < P.n;
        const int64_t ir = (int64_t)P.begin + (src_ok ? i_loc : 0);
        const float xi0 = a.frac[3 * ir], xi1 = a.frac[3 * ir + 1], xi2 = a.frac[3 * ir + 2];
        const float4 pi4 = w.pos[ir];
        const float3 pi = make_float3(pi4.x, pi4.y, pi4.z);
        // ---- masks and counts (at most MASK_CHUNKS chunks: n <= PL_MAX_ATOMS), the cells
        // along L_2 unrolled to the structure's extent
        int cnt = 0, nchunks = 0;
#define MG_PAIR_MASKS(U_)                                                                                    \
    cnt = pair_masks<U_>(P, &R, a, w, jg, i_loc, src_ok, xi0, xi1, xi2, pi, buf, boxes, nchunks, nre, ncand)
        switch (R.pl & 255) {
        case 1: MG_PAIR_MASKS(1); break;
        case 2: MG_PAIR_MASKS(2); break;
        case 3: MG_PAIR_MASKS(3); break;
        case 4: MG_PAIR_MASKS(4); break;
        case 5: MG_PAIR_MASKS(5); break;
        case 6: MG_PAIR_MASKS(6); break;
        case 7: MG_PAIR_MASKS(7); break;
        case 8: MG_PAIR_MASKS(8); break;
        default: MG_PAIR_MASKS(0); break;
        }
#undef MG_PAIR_MASKS
        // ---- one slot range for the item; each source's start within it
        const int incl = warp_incl_scan(cnt);
        const int T = __shfl_sync(FULL, incl, 31);
        const int lead = g * G;
        const int src_first = __shfl_sync(FULL, incl - cnt, lead);  // edges of earlier sources
        const int src_count = __shfl_sync(FULL, incl, lead + G - 1) - src_first;
        long long off = 0;
        if (lane == 0 && T > 0) off = (long long)atomicAdd(w.stage_ctr, (unsigned long long)T);
        off = __shfl_sync(FULL, off, 0);
        const bool spill = off + T > w.max_edges;  // staging area full: the spill kernel takes them
        if (jg == 0 && src_ok) {
            w.cnt[ir] = src_count;
            w.stage_off[ir] = spill ? -1ll : off + src_first;
            if (spill && src_count > 0) note_spill(w.spill_list, w.queue, (int)ir);
        }
        if (spill) {
            if (a.write_pairs && lane == 0 && T > 0) w.pair_ok[item.x] = 0;
            __syncwarp();
            continue;
        }
        // ---- keys at their canonical positions, from the stored masks and boxes
        const unsigned mB2 = (65536u + P.B2 - 1) / P.B2, mB1 = (65536u + P.B1 - 1) / P.B1;
        long long pos_src = off + src_first;  // this lane's source: its next free slot
        const long long item_end = off + T;
        __syncwarp();
        for (int c = 0; c < nchunks; ++c) {
            unsigned long long mask = buf[32 * c + lane];
            const unsigned bw = boxes[32 * c + lane];
            const int m = __popcll(mask);
            const int ci = warp_incl_scan(m);
            const int cfirst = __shfl_sync(FULL, ci - m, lead);
            const int ccount = __shfl_sync(FULL, ci, lead + G - 1) - cfirst;
            long long p = pos_src + (ci - m - cfirst);
            const unsigned long long jkey = (unsigned long long)(unsigned)(c * G + jg) << 32;
            int t0, t1, t2;
            unpack_t((uint32_t)bw, t0, t1, t2);
            // set bit b is offset lo + (r / B1, r % B1, b % B2) with r = b / B2; the quotients
            // of these small numbers (b < 64, B <= 64) by multiply and shift: floor(b / d) =
            // (b ceil(2^16 / d)) >> 16
            while (mask) {
                const unsigned b = (unsigned)(__ffsll((long long)mask) - 1);
                mask &= mask - 1;
                const unsigned r = (b * mB2) >> 16;
                const unsigned q0 = (r * mB1) >> 16;
                const int q2 = (int)(b - r * (unsigned)P.B2), q1 = (int)(r - q0 * (unsigned)P.B1);
                if (p < item_end) w.stage[p++] = jkey | pack_t(t0 + (int)q0, t1 + q1, t2 + q2);
            }
            pos_src += ccount;
        }
        __syncwarp();
    }
    if (a.collect_stats) {
        nre = warp_sum(nre);
        ncand = warp_sum(ncand);
        if (lane == 0 && ncand) {
            Status *st = reinterpret_cast<Status *>(a.g.status);
            atomicAdd(&st->rechecked, nre);
            atomicAdd(&st->candidates, ncand);
        }
    }
}

// ============================================================================ one-pass pair-lane build

// The one-pass form's items in canonical order (structure by structure): item_base[s] is
// the first item of structure s, queue[8] the number of items.  One block: each thread
// sums a contiguous range of structures, a block scan gives the ranges' starts.
__global__ void __launch_bounds__(PLAN_THREADS) pair_item_scan_kernel(int B, const int32_t *__restrict__ plan_items,
                                                                    int32_t *__restrict__ item_base,
                                                                    unsigned int *__restrict__ queue) {
    __shared__ int part[PLAN_THREADS];
    const int t = threadIdx.x;
    const int per = (B + PLAN_THREADS - 1) / PLAN_THREADS;
    const int s0 = min(B, t * per), s1 = min(B, s0 + per);
    int sum = 0;
    for (int s = s0; s < s1; ++s) sum += plan_items[s];
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < PLAN_THREADS; off <<= 1) {  // inclusive scan of the ranges' sums
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - sum;
    for (int s = s0; s < s1; ++s) {
        item_base[s] = run;
        run += plan_items[s];
    }
    if (t == PLAN_THREADS - 1) queue[8] = (unsigned)part[t];
}

// The pair-lane build in one pass (small batches, where the count scan and the staging
// of the other forms cost more than they save): blocks take tiles of PAIR_WARPS
// consecutive items in canonical order (a ticket per block, so a tile only waits on tiles
// already running).  A warp computes its item's pair masks into shared memory (or, for a
// structure outside the pair-lane scan, scans its one source by the warp enumeration,
// keys in shared memory); the tile's total is published and its offset found by the
// decoupled look-back; then every lane writes its pairs' edges at their canonical
// positions (or the warp emits its source).  Writes src_ptr, edge_ptr, the pair table of
// symmetric graphs, and (the last tile) the edge count and the capacity check.  4 blocks
// of 4 warps per SM at up to 128 registers (at 80 both scans spill; the batches this form
// serves fill less than a wave of blocks anyway).
__global__ void __launch_bounds__(PAIR_WARPS * 32, 4) pair_onepass_kernel(const __grid_constant__ BuildArgs a,
                                                                           const __grid_constant__ Work w) {
    __shared__ unsigned long long buf_all[PAIR_WARPS][BUILD_CAP];  // source keys, or masks and boxes
    static_assert(32 * MASK_CHUNKS + 16 * MASK_CHUNKS <= BUILD_CAP, "mask buffer");
    __shared__ int s_tile;
    __shared__ long long s_cnt[PAIR_WARPS];
    __shared__ long long s_prefix;
    const int wid = threadIdx.x >> 5, lane = lane_id();
    unsigned long long *buf = buf_all[wid];
    unsigned *boxes = reinterpret_cast<unsigned *>(buf + 32 * MASK_CHUNKS);
    const mg_graph_t &g = a.g;
    pdl_wait();  // prep's records, positions, items and zeroed look-back words
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(&w.queue[3], 1u);
    __syncthreads();
    const int tile = s_tile;
    const int total = (int)w.queue[8];
    const int last_tile = (total + PAIR_WARPS - 1) / PAIR_WARPS - 1;
    if (tile > last_tile) return;  // the whole block: more blocks than tiles
    const int it = tile * PAIR_WARPS + wid;
    const bool have = it < total;
    // the item's structure: the last s with item_base[s] <= it (structures without items
    // share their base with the next one and precede it)
    int s = 0;
    if (have) {
        int lo = 0, hi = a.B;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (w.item_base[mid] <= it) lo = mid;
            else hi = mid;
        }
        s = lo;
    }
    const StructRec &R = w.recs[s];
    const int q_item = have ? it - w.item_base[s] : 0;
    const bool pairs = have && R.pl != 0;
    unsigned long long nre = 0, ncand = 0;
    // ---- pass 1: masks and counts (pair-lane) or the source's keys (warp enumeration)
    PairStruct P;
    int G = 32, jg = 0, lead = 0, nchunks = 0, src_first = 0, i_loc = 0;
    bool src_ok = false;
    int64_t ir = 0;
    float xi0 = 0.f, xi1 = 0.f, xi2 = 0.f;
    long long item_total = 0;
    SrcScan c;
    c.s = 0;
    int m_src = 0;
    bool spill = false;
    if (pairs) {
        load_pair_struct(P, R);
        G = P.G;
        const int grp = lane / G;
        jg = lane % G;
        lead = grp * G;
        i_loc = q_item * P.spw + grp;
        src_ok = i_loc < P.n;
        ir = (int64_t)P.begin + (src_ok ? i_loc : 0);
        xi0 = a.frac[3 * ir];
        xi1 = a.frac[3 * ir + 1];
        xi2 = a.frac[3 * ir + 2];
        const float4 pi4 = w.pos[ir];
        const float3 pi = make_float3(pi4.x, pi4.y, pi4.z);
        int cnt = 0;
#define MG_PAIR_MASKS1(U_)                                                                                   \
    cnt = pair_masks<U_>(P, &R, a, w, jg, i_loc, src_ok, xi0, xi1, xi2, pi, buf, boxes, nchunks, nre, ncand)
        switch (R.pl & 255) {
        case 1: MG_PAIR_MASKS1(1); break;
        case 2: MG_PAIR_MASKS1(2); break;
        case 3: MG_PAIR_MASKS1(3); break;
        case 4: MG_PAIR_MASKS1(4); break;
        case 5: MG_PAIR_MASKS1(5); break;
        case 6: MG_PAIR_MASKS1(6); break;
        case 7: MG_PAIR_MASKS1(7); break;
        case 8: MG_PAIR_MASKS1(8); break;
        default: MG_PAIR_MASKS1(0); break;
        }
#undef MG_PAIR_MASKS1
        const int incl = warp_incl_scan(cnt);
        item_total = __shfl_sync(FULL, incl, 31);
        src_first = __shfl_sync(FULL, incl - cnt, lead);
    } else if (have) {
        const int i = R.atom_begin + q_item;
        if (source_setup<false>(a, w, i, c)) m_src = scan_source<false>(a, w, c, buf, nullptr, spill);
        item_total = m_src;
    }
    if (lane == 0) s_cnt[wid] = item_total;
    __syncthreads();
    if (wid == 0) {  // the tile's total and prefix: one warp looks back
        long long agg = 0;
        for (int q = 0; q < PAIR_WARPS; ++q) agg += s_cnt[q];
        long long prefix = 0;
        unsigned long long *flags = w.tile_flags;
        if (tile == 0) {
            if (lane == 0) atomicExch(&flags[0], TILE_PREFIX | (unsigned long long)agg);
        } else {
            if (lane == 0) atomicExch(&flags[tile], TILE_AGG | (unsigned long long)agg);
            __syncwarp();
            prefix = tile_lookback_warp(flags, tile, g.status);
            if (lane == 0) atomicExch(&flags[tile], TILE_PREFIX | (unsigned long long)(prefix + agg));
        }
        if (lane == 0) s_prefix = prefix;
        if (lane == 0 && tile == last_tile) {  // the last tile knows the edge count
            const long long tot = prefix + agg;
            Status *st = reinterpret_cast<Status *>(g.status);
            st->num_edges = (unsigned long long)tot;
            st->required_capacity = (unsigned long long)tot;
            if (tot > g.capacity) set_error(g.status, MG_ERR_CAPACITY, -1);
            a.src_ptr[a.N] = tot;
            g.edge_ptr[a.B] = tot;
            for (int q = a.B - 1; q >= 0 && a.atom_ptr[q] == a.N; --q) g.edge_ptr[q] = tot;
        }
    }
    __syncthreads();
    if (!have) return;
    long long base = s_prefix;
    for (int q = 0; q < wid; ++q) base += s_cnt[q];
    const bool fits = base + item_total <= g.capacity;
    if (!pairs) {  // ---- a source of the warp enumeration
        const int i = R.atom_begin + q_item;
        if (lane == 0) {
            a.src_ptr[i] = base;
            for (int q = s; q >= 0 && a.atom_ptr[q] == i; --q) g.edge_ptr[q] = base;  // structures starting at i
        }
        if (m_src > 0 && fits) emit_source<false>(a, w, c, i, base, m_src, buf, nullptr, spill);
        return;
    }
    // ---- the pair-lane item: every lane writes its pairs' edges, chunk by chunk
    const long long seg = base + src_first;  // this lane's source: its first row
    if (jg == 0 && src_ok) {
        a.src_ptr[ir] = seg;
        if (i_loc == 0)
            for (int q = s; q >= 0 && a.atom_ptr[q] == (int)ir; --q) g.edge_ptr[q] = seg;
    }
    if (fits) {
        const bool ptab = a.write_pairs && P.n <= PAIR_MAX;
        const unsigned mB2 = (65536u + P.B2 - 1) / P.B2, mB1 = (65536u + P.B1 - 1) / P.B1;
        long long pos_src = seg;
        for (int cc = 0; cc < nchunks; ++cc) {
            unsigned long long mask = buf[32 * cc + lane];
            const int m = __popcll(mask);
            const int ci = warp_incl_scan(m);
            const int cfirst = __shfl_sync(FULL, ci - m, lead);
            const int ccount = __shfl_sync(FULL, ci, lead + G - 1) - cfirst;
            long long p = pos_src + (ci - m - cfirst);
            if (m) {
                const int jl = cc * G + jg;
                const int64_t jr = (int64_t)P.begin + jl;
                if (ptab) {
                    w.pair_lo[ir * PAIR_MAX + jl] = (uint16_t)(p - seg);
                    w.pair_hi[ir * PAIR_MAX + jl] = (uint16_t)(p - seg + m);
                }
                int t0, t1, t2;
                unpack_t(boxes[32 * cc + lane], t0, t1, t2);
                while (mask) {  // bit b is offset lo + (r / B1, r % B1, b % B2), r = b / B2
                    const unsigned b = (unsigned)(__ffsll((long long)mask) - 1);
                    mask &= mask - 1;
                    const unsigned r = (b * mB2) >> 16;
                    const unsigned q0 = (r * mB1) >> 16;
                    const int q2 = (int)(b - r * (unsigned)P.B2), q1 = (int)(r - q0 * (unsigned)P.B1);
                    g.src[p] = (int32_t)ir;
                    g.dst[p] = (int32_t)jr;
                    g.offset[3 * p + 0] = t0 + (int)q0;
                    g.offset[3 * p + 1] = t1 + q1;
                    g.offset[3 * p + 2] = t2 + q2;
                    ++p;
                }
            }
            pos_src += ccount;
        }
        // the vectors of the item's rows, a lane per row (the rows' lanes vary in their
        // edge counts; this part does not): read back what the warp just wrote
        __syncwarp();
        if (g.vec || g.len) {
            for (long long e = base + lane; e < base + item_total; e += 32) {
                const int64_t si = g.src[e], sj = g.dst[e];
                const float3 v =
                    edge_vec_ff(P.L, a.frac[3 * si], a.frac[3 * si + 1], a.frac[3 * si + 2], a.frac[3 * sj],
                                a.frac[3 * sj + 1], a.frac[3 * sj + 2], g.offset[3 * e], g.offset[3 * e + 1],
                                g.offset[3 * e + 2]);
                if (g.vec) {
                    g.vec[3 * e + 0] = v.x;
                    g.vec[3 * e + 1] = v.y;
                    g.vec[3 * e + 2] = v.z;
                }
                if (g.len) g.len[e] = vec_len(v);
            }
        }
    }
    if (a.collect_stats) {
        nre = warp_sum(nre);
        ncand = warp_sum(ncand);
        if (lane == 0 && ncand) {
            Status *st = reinterpret_cast<Status *>(g.status);
            atomicAdd(&st->rechecked, nre);
            atomicAdd(&st->candidates, ncand);
        }
    }
}

cudaError_t launch_pair_onepass(const BuildArgs &a, const Work &w, cudaStream_t s) {
    if (a.N <= 0) return cudaSuccess;
    pair_item_scan_kernel<<<1, PLAN_THREADS, 0, s>>>(a.B, w.plan_items, w.item_base, w.queue);
    const int blocks = (a.N + PAIR_WARPS - 1) / PAIR_WARPS;  // at most one item per atom
    pair_onepass_kernel<<<blocks, PAIR_WARPS * 32, 0, s>>>(a, w);
    return cudaGetLastError();
}

// ============================================================================ pair-lane KNN

constexpr int KNN_CAP = 2 * PL_KNN_MAX_K;  // candidates one warp collects for its source

// Canonical FP64 squared distance of one candidate, out of line (see band_is_edge).
__device__ __noinline__ double canon_pair_d2(const StructRec *__restrict__ rec, float xi0, float xi1, float xi2,
                                             float xj0, float xj1, float xj2, int t0, int t1, int t2) {
    return canon_d2(rec->L, xi0, xi1, xi2, xj0, xj1, xj2, t0, t1, t2);
}

// 64-bit keys, one per lane, sorted ascending across the warp (bitonic network).
__device__ __forceinline__ unsigned long long warp_sort_u64(unsigned long long v) {
    const int lane = lane_id();
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
        const bool desc = (lane & size) != 0;
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const unsigned long long y = __shfl_xor_sync(FULL, v, stride);
            const bool lower = (lane & stride) == 0;
            v = (lower != desc) ? (v < y ? v : y) : (v < y ? y : v);
        }
    }
    return v;
}

// 64 keys, two per lane (element r 32 + lane in register r), sorted ascending by the
// same bitonic network over 64 elements: strides below 32 across lanes, stride 32 within
// the lane.
__device__ __forceinline__ void warp_sort_u64x2(unsigned long long &a, unsigned long long &b) {
    const int lane = lane_id();
#pragma unroll
    for (int size = 2; size <= 64; size <<= 1) {
        const bool d0 = (lane & size) != 0, d1 = ((lane + 32) & size) != 0;
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride == 32) {  // size 64, ascending: element lane against lane + 32
                const unsigned long long lo = a < b ? a : b, hi = a < b ? b : a;
                a = lo;
                b = hi;
            } else {
                const bool lower = (lane & stride) == 0;
                unsigned long long y = __shfl_xor_sync(FULL, a, stride);
                a = (lower != d0) ? (a < y ? a : y) : (a < y ? y : a);
                y = __shfl_xor_sync(FULL, b, stride);
                b = (lower != d1) ? (b < y ? b : y) : (b < y ? y : b);
            }
        }
    }
}

// Sort n (<= KNN_CAP) 64-bit keys in shared memory with one warp: in registers up to 64,
// by the shared-memory network beyond (padded to a power of two >= 128).
__device__ __forceinline__ void warp_sort_n(unsigned long long *b, int n) {
    const int lane = lane_id();
    if (n <= 32) {
        unsigned long long v = lane < n ? b[lane] : ~0ull;
        v = warp_sort_u64(v);
        __syncwarp();
        if (lane < n) b[lane] = v;
        __syncwarp();
        return;
    }
    if (n <= 64) {
        unsigned long long v0 = b[lane], v1 = lane + 32 < n ? b[lane + 32] : ~0ull;
        warp_sort_u64x2(v0, v1);
        __syncwarp();
        b[lane] = v0;
        if (lane + 32 < n) b[lane + 32] = v1;
        __syncwarp();
        return;
    }
    int P = 128;
    while (P < n) P <<= 1;
    warp_smem_sort_u64(b, n, P);
}

// The KNN candidates of one chunk of targets: every lane's cells with FP32 d2 < rho^2
// (not (i, i, 0)) are placed in shared memory after the C candidates already there, in
// lane order (a warp scan of the counts); ord gets (d2 bits << 32 | slot), keys the
// slot's (j << 32 | packed t).  Returns false (and sets over) when they would pass
// KNN_CAP.  knn_small_cells: boxes of at most E cells per axis, unrolled with the cells'
// distances kept in registers; knn_box_cells: any box (at most PL_BOX_MAX cells).
template <int E>
__device__ __forceinline__ bool knn_small_cells(const float L[9], float ax, float ay, float az, const float lo[3],
                                                const float nn[3], float rho2, bool same, int j_loc, int &C,
                                                unsigned long long *ord, unsigned long long *keys, bool &over) {
    // cell c = (q0 E + q1) E + q2; the cells inside the pair's box, from its extents
    // (0 .. E per axis) as per-axis bit patterns
    unsigned valid;
    if (E == 1) {
        valid = (nn[0] > 0.0f && nn[1] > 0.0f && nn[2] > 0.0f) ? 1u : 0u;
    } else {
        const unsigned v0 = nn[0] >= 2.0f ? 0xFFu : (nn[0] >= 1.0f ? 0x0Fu : 0u);
        const unsigned v1 = nn[1] >= 2.0f ? 0xFFu : (nn[1] >= 1.0f ? 0x33u : 0u);
        const unsigned v2 = nn[2] >= 2.0f ? 0xFFu : (nn[2] >= 1.0f ? 0x55u : 0u);
        valid = v0 & v1 & v2;
    }
    unsigned mask = 0u;
#pragma unroll
    for (int q0 = 0; q0 < E; ++q0) {
        const float t0 = __fadd_rn(lo[0], (float)q0);
#pragma unroll
        for (int q1 = 0; q1 < E; ++q1) {
            const float t1 = __fadd_rn(lo[1], (float)q1);
            const float bx_ = __fmaf_rn(t1, L[3], __fmaf_rn(t0, L[0], ax));
            const float by_ = __fmaf_rn(t1, L[4], __fmaf_rn(t0, L[1], ay));
            const float bz_ = __fmaf_rn(t1, L[5], __fmaf_rn(t0, L[2], az));
#pragma unroll
            for (int q2 = 0; q2 < E; ++q2) {
                const float t2 = __fadd_rn(lo[2], (float)q2);
                const float vx = __fmaf_rn(t2, L[6], bx_);
                const float vy = __fmaf_rn(t2, L[7], by_);
                const float vz = __fmaf_rn(t2, L[8], bz_);
                const float d2 = __fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx)));
                if (d2 < rho2) mask |= 1u << ((q0 * E + q1) * E + q2);
            }
        }
    }
    mask &= valid;
    if (same && mask) {  // (i, i, 0) is not a candidate: the cell of offset 0, if in the box
        const float z0 = -lo[0], z1 = -lo[1], z2 = -lo[2];
        if (z0 >= 0.0f && z0 < (float)E && z1 >= 0.0f && z1 < (float)E && z2 >= 0.0f && z2 < (float)E)
            mask &= ~(1u << ((fint(z0) * E + fint(z1)) * E + fint(z2)));
    }
    const int m = __popc(mask);
    int incl, tot;
    if (E == 1) {  // at most one candidate per lane: a ballot is the scan
        const unsigned bal = __ballot_sync(FULL, m != 0);
        incl = __popc(bal & (0xffffffffu >> (31 - lane_id())));
        tot = __popc(bal);
    } else {
        incl = warp_incl_scan(m);
        tot = __shfl_sync(FULL, incl, 31);
    }
    if (C + tot > KNN_CAP) {
        over = true;
        return false;
    }
    int slot = C + incl - m;
    const int t0i = fint(lo[0]), t1i = fint(lo[1]), t2i = fint(lo[2]);
    while (mask) {  // the set cells, their distance again (the same operations)
        const int c = __ffs(mask) - 1;
        mask &= mask - 1;
        const int q0 = c / (E * E), q1 = (c / E) % E, q2 = c % E;
        const float t0 = __fadd_rn(lo[0], ifloat(q0)), t1 = __fadd_rn(lo[1], ifloat(q1)),
                    t2 = __fadd_rn(lo[2], ifloat(q2));
        const float bx_ = __fmaf_rn(t1, L[3], __fmaf_rn(t0, L[0], ax));
        const float by_ = __fmaf_rn(t1, L[4], __fmaf_rn(t0, L[1], ay));
        const float bz_ = __fmaf_rn(t1, L[5], __fmaf_rn(t0, L[2], az));
        const float vx = __fmaf_rn(t2, L[6], bx_);
        const float vy = __fmaf_rn(t2, L[7], by_);
        const float vz = __fmaf_rn(t2, L[8], bz_);
        const float d2 = __fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx)));
        ord[slot] = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)slot;
        keys[slot] = ((unsigned long long)(unsigned)j_loc << 32) | pack_t(t0i + q0, t1i + q1, t2i + q2);
        ++slot;
    }
    C += tot;
    return true;
}

__device__ __forceinline__ bool knn_box_cells(const float L[9], float ax, float ay, float az, const float lo[3],
                                              const float nn[3], float rho2, bool same, int j_loc, int &C,
                                              unsigned long long *ord, unsigned long long *keys, bool &over) {
    unsigned long long mask = 0ull, bit = 1ull;
    for (float t0 = lo[0]; t0 < lo[0] + nn[0]; t0 = __fadd_rn(t0, 1.0f))
        for (float t1 = lo[1]; t1 < lo[1] + nn[1]; t1 = __fadd_rn(t1, 1.0f)) {
            const float bx_ = __fmaf_rn(t1, L[3], __fmaf_rn(t0, L[0], ax));
            const float by_ = __fmaf_rn(t1, L[4], __fmaf_rn(t0, L[1], ay));
            const float bz_ = __fmaf_rn(t1, L[5], __fmaf_rn(t0, L[2], az));
            const bool row0 = same && t0 == 0.0f && t1 == 0.0f;
            for (float t2 = lo[2]; t2 < lo[2] + nn[2]; t2 = __fadd_rn(t2, 1.0f), bit <<= 1) {
                const float vx = __fmaf_rn(t2, L[6], bx_);
                const float vy = __fmaf_rn(t2, L[7], by_);
                const float vz = __fmaf_rn(t2, L[8], bz_);
                const float d2 = __fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx)));
                if (d2 < rho2 && !(row0 && t2 == 0.0f)) mask |= bit;
            }
        }
    const int m = __popcll(mask);
    const int incl = warp_incl_scan(m);
    const int tot = __shfl_sync(FULL, incl, 31);
    if (C + tot > KNN_CAP) {
        over = true;
        return false;
    }
    // place this lane's candidates at C + (its exclusive prefix) + its order
    int slot = C + incl - m;
    const int t0i = fint(lo[0]), t1i = fint(lo[1]), t2i = fint(lo[2]);
    const int n1 = fint(nn[1]), n2 = fint(nn[2]);
    for (int q0 = 0; q0 < fint(nn[0]) && mask; ++q0)
        for (int q1 = 0; q1 < n1 && mask; ++q1) {
            const float ft0 = ifloat(t0i + q0), ft1 = ifloat(t1i + q1);
            const float bx_ = __fmaf_rn(ft1, L[3], __fmaf_rn(ft0, L[0], ax));
            const float by_ = __fmaf_rn(ft1, L[4], __fmaf_rn(ft0, L[1], ay));
            const float bz_ = __fmaf_rn(ft1, L[5], __fmaf_rn(ft0, L[2], az));
            for (int q2 = 0; q2 < n2; ++q2, mask >>= 1) {
                if (!(mask & 1ull)) continue;
                const float ft2 = ifloat(t2i + q2);
                const float vx = __fmaf_rn(ft2, L[6], bx_);
                const float vy = __fmaf_rn(ft2, L[7], by_);
                const float vz = __fmaf_rn(ft2, L[8], bz_);
                const float d2 = __fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx)));
                ord[slot] = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)slot;
                keys[slot] = ((unsigned long long)(unsigned)j_loc << 32) | pack_t(t0i + q0, t1i + q1, t2i + q2);
                ++slot;
            }
        }
    C += tot;
    return true;
}

// A warp per source atom.  Alg. 1's loop with a radius rho that starts from the number
// density: every lane evaluates its target's offset box for rho (at most 64 cells; a
// source whose boxes grow past that, or whose offsets exceed the packed key, goes to the
// fallback list) and the images with FP32 d2 < rho^2 are collected in shared memory (a
// warp scan of the lanes' counts places them).  Sorted by FP32 d2, the k-th is tau; rho
// grows until tau + 3 delta < rho^2 (delta the FP32 error bound plus the band), so every
// image whose canonical d2 can reach tau + 2 delta is among the candidates.  Then the
// selection of the warp-enumeration KNN: certain members below tau - 2 delta, the band
// ranked by (canonical FP64 d2, j, t) when it holds more candidates than the slots left,
// the k winners sorted by (j, t) and written at rows i k .. i k + k - 1.
__global__ void __launch_bounds__(PAIR_WARPS * 32, 7) knn_pairs_kernel(const __grid_constant__ BuildArgs a,
                                                                        const __grid_constant__ Work w) {
    __shared__ unsigned long long ord_all[PAIR_WARPS][KNN_CAP];  // (FP32 d2 bits << 32 | slot)
    __shared__ unsigned long long key_all[PAIR_WARPS][KNN_CAP];  // (j << 32 | packed t) by slot
    __shared__ unsigned long long aux_all[PAIR_WARPS][KNN_CAP];  // FP64 d2 bits of the band
    __shared__ unsigned long long win_all[PAIR_WARPS][KNN_CAP];  // the k winners' keys
    const int wid = threadIdx.x >> 5, lane = lane_id();
    unsigned long long *ord = ord_all[wid], *keys = key_all[wid], *aux = aux_all[wid], *win = win_all[wid];
    pdl_wait();  // prep's records and positions (a no-op unless launched behind prep)
    const int i = a.atom_lo + blockIdx.x * PAIR_WARPS + wid;
    if (i >= a.atom_hi) return;
    const mg_graph_t &g = a.g;
    const int s = w.atom_struct[i];
    const StructRec &R = w.recs[s];
    if (R.bad) {
        if (lane == 0 && i == R.atom_begin) set_error(g.status, R.bad, s + a.struct_offset);
        return;
    }
    const int k = a.knn_k;
    const int n = R.n_atoms, begin = R.atom_begin, i_loc = i - begin;
    float L[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) L[q] = R.L[q];
    const float xi0 = a.frac[3 * (int64_t)i], xi1 = a.frac[3 * (int64_t)i + 1], xi2 = a.frac[3 * (int64_t)i + 2];
    const float4 pi4 = w.pos[i];
    unsigned long long ncand = 0;
    float rho = R.cut, tau = 0.f, delta = 0.f;
    int C = 0;
    bool ok = false, fallback = false;
    for (int iter = 0; iter < 32 && !ok && !fallback; ++iter) {
        const float rho2 = __fmul_rn(rho, rho);
        float reach[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) reach[d] = __fadd_rn(__fmul_rn(__fmul_rn(rho, 1.00001f), R.invd[d]), R.reach[d]);
        if (!(fmaxf(reach[0], fmaxf(reach[1], reach[2])) < 32.0f)) {  // no box of 64 cells reaches that far
            fallback = true;
            break;
        }
        // boxes of at most one or two cells per axis when the reach is below a half or a
        // whole cell (an interval shorter than 1 or 2 holds at most 1 or 2 integers)
        const float rmax = fmaxf(reach[0], fmaxf(reach[1], reach[2]));
        const int E = rmax < 0.49f ? 1 : (rmax < 0.99f ? 2 : 0);
        C = 0;
        bool over = false;
        // one chunk of targets (a target per lane): the pair boxes, then the cells with
        // FP32 d2 < rho^2 except (i, i, 0), with the same fused operations as the warp
        // enumeration, so the structure's FP32 error bound holds.  false: stop the scan
        // (the source falls back, or the buffer is full)
        auto chunk = [&](float xj0, float xj1, float xj2, float4 pj, int j_loc, bool okj) -> bool {
            const float dx[3] = {__fsub_rn(xj0, xi0), __fsub_rn(xj1, xi1), __fsub_rn(xj2, xi2)};
            float lo[3], nn[3];
            bool big = false;
            if (E == 1) {
                // reach below half a cell: the only integer that can lie within reach of
                // -dx is the nearest one (a cell at the interval's edge lies beyond rho
                // by the reach's margin, so either test keeps every image closer than rho)
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    lo[d] = frnd(-dx[d]);
                    nn[d] = (okj && fabsf(__fadd_rn(dx[d], lo[d])) <= reach[d]) ? 1.0f : 0.0f;
                    big |= okj && fabsf(lo[d]) > (float)OFFSET_KEY_LIM;
                }
            } else {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    lo[d] = fceil(__fsub_rn(-reach[d], dx[d]));
                    const float hi = ffloor(__fsub_rn(reach[d], dx[d]));
                    nn[d] = okj ? fmaxf(0.0f, __fadd_rn(__fsub_rn(hi, lo[d]), 1.0f)) : 0.0f;
                    big |= okj && (lo[d] < -(float)OFFSET_KEY_LIM || hi > (float)OFFSET_KEY_LIM);
                }
            }
            big |= __fmul_rn(__fmul_rn(nn[0], nn[1]), nn[2]) > (float)PL_BOX_MAX;
            if (E > 0) big |= fmaxf(nn[0], fmaxf(nn[1], nn[2])) > (float)E;  // cannot happen
            if (__any_sync(FULL, big)) {
                fallback = true;
                return false;
            }
            const float ax = __fsub_rn(pj.x, pi4.x), ay = __fsub_rn(pj.y, pi4.y), az = __fsub_rn(pj.z, pi4.z);
            const bool same = okj && j_loc == i_loc;
            if (a.collect_stats) ncand += (unsigned long long)__fmul_rn(__fmul_rn(nn[0], nn[1]), nn[2]);
            if (E == 1) return knn_small_cells<1>(L, ax, ay, az, lo, nn, rho2, same, j_loc, C, ord, keys, over);
            if (E == 2) return knn_small_cells<2>(L, ax, ay, az, lo, nn, rho2, same, j_loc, C, ord, keys, over);
            return knn_box_cells(L, ax, ay, az, lo, nn, rho2, same, j_loc, C, ord, keys, over);
        };
        if (R.nb[0] == 0 || n <= PL_MAX_ATOMS) {
            // every atom of the structure, in order (up to PL_MAX_ATOMS atoms this is
            // faster than the cell list: measured 0.81 against 0.90 ms for k = 16 on
            // 8192 structures of up to 400 atoms); the targets' coordinates one chunk
            // ahead (their loads overlap this chunk's cells)
            int64_t jr = (int64_t)begin + (lane < n ? lane : 0);
            float nx0 = a.frac[3 * jr], nx1 = a.frac[3 * jr + 1], nx2 = a.frac[3 * jr + 2];
            float4 npj = w.pos[jr];
            for (int jb = 0; jb < n; jb += 32) {
                const int j_loc = jb + lane;
                const float xj0 = nx0, xj1 = nx1, xj2 = nx2;
                const float4 pj = npj;
                if (jb + 32 < n) {
                    jr = (int64_t)begin + (j_loc + 32 < n ? j_loc + 32 : 0);
                    nx0 = a.frac[3 * jr];
                    nx1 = a.frac[3 * jr + 1];
                    nx2 = a.frac[3 * jr + 2];
                    npj = w.pos[jr];
                }
                if (!chunk(xj0, xj1, xj2, pj, j_loc, j_loc < n)) break;
            }
        } else {
            // larger structures with a cell list (20.4 against 1.48 ms for k = 32 on 32
            // supercells of 1,728 to 21,952 atoms): the atoms of the bins that the reach interval
            // [x_i - reach_k, x_i + reach_k] (wrapped) touches on each axis, each bin
            // once; every image with FP32 d2 < rho^2 lies in the pair boxes of these
            // targets.  Candidates then come in bin order: only the ranking by distance
            // and the final (j, t) sort see them, so the result does not depend on it.
            int blo[3], bcnt[3];
            const float xw[3] = {wrap01(xi0), wrap01(xi1), wrap01(xi2)};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int nk = R.nb[d];
                const float m = 1e-5f * (1.0f + reach[d]);
                const int blo_d = (int)floorf((xw[d] - reach[d] - m) * (float)nk);
                const int bhi_d = (int)floorf((xw[d] + reach[d] + m) * (float)nk);
                blo[d] = bhi_d - blo_d + 1 >= nk ? 0 : blo_d;
                bcnt[d] = bhi_d - blo_d + 1 >= nk ? nk : bhi_d - blo_d + 1;
            }
            const int nbins = bcnt[0] * bcnt[1] * bcnt[2];
            bool go = true;
            for (int bb = 0; bb < nbins && go; bb += 32) {
                const int q = bb + lane;
                int64_t st = 0;
                int cnt = 0;
                if (q < nbins) {
                    const int c2 = q % bcnt[2], c1 = (q / bcnt[2]) % bcnt[1], c0 = q / (bcnt[2] * bcnt[1]);
                    const int b0 = ((blo[0] + c0) % R.nb[0] + R.nb[0]) % R.nb[0];
                    const int b1 = ((blo[1] + c1) % R.nb[1] + R.nb[1]) % R.nb[1];
                    const int b2 = ((blo[2] + c2) % R.nb[2] + R.nb[2]) % R.nb[2];
                    const int64_t gb = (int64_t)R.bin_base + (b0 * R.nb[1] + b1) * R.nb[2] + b2;
                    st = w.cell_start[gb];
                    cnt = (int)(w.cell_start[gb + 1] - st);
                }
                const int incl = warp_incl_scan(cnt);
                const int total = __shfl_sync(FULL, incl, 31);
                const int excl = incl - cnt;
                for (int ab = 0; ab < total && go; ab += 32) {
                    const int q2 = ab + lane;
                    const bool va = q2 < total;
                    const int ow = warp_owner(incl, va ? q2 : total - 1);
                    const int64_t ost = __shfl_sync(FULL, st, ow);
                    const int oex = __shfl_sync(FULL, excl, ow);
                    float4 xj = make_float4(0.f, 0.f, 0.f, 0.f), pj = xj;
                    if (va) {
                        xj = w.cell_fx[ost + (q2 - oex)];
                        pj = w.cell_p[ost + (q2 - oex)];
                    }
                    go = chunk(xj.x, xj.y, xj.z, pj, va ? __float_as_int(xj.w) : 0, va);
                }
            }
        }
        __syncwarp();
        if (fallback) break;
        if (over) {  // more candidates than the buffer: a smaller radius
            rho = __fmul_rn(rho, 0.8f);
            continue;
        }
        if (C < k) {  // too few: a larger radius, by the expected count's cube root (at most 1.5)
            rho = __fmul_rn(rho, C > 0 ? fminf(1.5f, fmaxf(1.1f, cbrtf(1.4f * (float)k / (float)C))) : 1.5f);
            continue;
        }
        warp_sort_n(ord, C);
        tau = __uint_as_float((unsigned)(ord[k - 1] >> 32));
        delta = fp32_d2_error(R, rho, rho2) + 2.0f * a.band_rel * rho2;
        if (tau + 3.0f * delta < rho2) ok = true;
        else rho = sqrtf(tau + 3.0f * delta) * 1.0005f + 1e-6f;
        if (!(rho < 1e6f)) break;
    }
    if (!ok) {  // the warp-enumeration KNN takes this source
        if (lane == 0) {
            const unsigned p = atomicAdd(&w.queue[10], 1u);
            reinterpret_cast<int *>(w.items)[p] = i;
        }
        return;
    }
    // ---- selection: ord[0 .. m0) certain, ord[m0 .. m0 + nb) the band
    const float lo_thr = tau - 2.0f * delta, hi_thr = tau + 2.0f * delta;
    int m0 = 0, nb = 0;
    for (int q = lane; q < C; q += 32) {
        const float d = __uint_as_float((unsigned)(ord[q] >> 32));
        m0 += d < lo_thr ? 1 : 0;
        nb += (d >= lo_thr && d <= hi_thr) ? 1 : 0;
    }
    m0 = warp_sum(m0);
    nb = warp_sum(nb);
    if (m0 >= k || m0 + nb < k) {  // cannot happen: fewer than k FP32 distances lie below tau
        if (lane == 0) set_error(g.status, MG_ERR_INTERNAL, s);
        return;
    }
    const int need = k - m0;
    for (int q = lane; q < m0; q += 32) win[q] = keys[(unsigned)ord[q]];
    if (nb == need) {  // every band member fills a remaining slot
        for (int q = lane; q < nb; q += 32) win[m0 + q] = keys[(unsigned)ord[m0 + q]];
    } else {  // rank the band by (canonical FP64 d2, j, t)
        for (int q = lane; q < nb; q += 32) {
            const unsigned long long key = keys[(unsigned)ord[m0 + q]];
            int t0, t1, t2;
            unpack_t((uint32_t)(key & 0xffffffffull), t0, t1, t2);
            const int64_t jr = (int64_t)begin + (int)(key >> 32);
            aux[q] = (unsigned long long)__double_as_longlong(
                canon_pair_d2(&R, xi0, xi1, xi2, a.frac[3 * jr], a.frac[3 * jr + 1], a.frac[3 * jr + 2], t0, t1, t2));
            ord[m0 + q] = key;  // this lane's own band slot: now its key
        }
        __syncwarp();
        for (int q = lane; q < nb; q += 32) {
            const unsigned long long dq = aux[q], kq = ord[m0 + q];
            int rank = 0;
            for (int p = 0; p < nb; ++p) {
                const unsigned long long dp = aux[p], kp = ord[m0 + p];
                rank += (dp < dq || (dp == dq && kp < kq)) ? 1 : 0;
            }
            if (rank < need) win[m0 + rank] = kq;
        }
    }
    __syncwarp();
    // ---- the k winners in canonical (j, t) order, written at rows i k ..
    warp_sort_n(win, k);
    for (int q = lane; q < k; q += 32) {
        const unsigned long long jt = win[q];
        int t0, t1, t2;
        unpack_t((uint32_t)(jt & 0xffffffffull), t0, t1, t2);
        const int64_t jr = (int64_t)begin + (int)(jt >> 32);
        const int64_t e = (int64_t)i * k + q;
        g.src[e] = i;
        g.dst[e] = (int32_t)jr;
        g.offset[3 * e + 0] = t0;
        g.offset[3 * e + 1] = t1;
        g.offset[3 * e + 2] = t2;
        if (g.vec || g.len) {
            const float3 v = edge_vec_ff(L, xi0, xi1, xi2, a.frac[3 * jr], a.frac[3 * jr + 1], a.frac[3 * jr + 2], t0,
                                         t1, t2);
            if (g.vec) {
                g.vec[3 * e + 0] = v.x;
                g.vec[3 * e + 1] = v.y;
                g.vec[3 * e + 2] = v.z;
            }
            if (g.len) g.len[e] = vec_len(v);
        }
    }
    if (a.collect_stats) {
        ncand = warp_sum(ncand);
        if (lane == 0) {
            Status *st = reinterpret_cast<Status *>(g.status);
            atomicAdd(&st->candidates, ncand);
            if (nb != need) atomicAdd(&st->rechecked, (unsigned long long)nb);
        }
    }
}

// ============================================================================ launch

static int g_pair_blocks = 0;  // resident blocks per SM of the stage pass

cudaError_t launch_knn_pairs(const BuildArgs &a, const Work &w, cudaStream_t s) {
    const int atoms = a.atom_hi - a.atom_lo;
    if (atoms <= 0) return cudaSuccess;
    const int blocks = (atoms + PAIR_WARPS - 1) / PAIR_WARPS;
    if (a.pdl) return launch_pdl(knn_pairs_kernel, dim3(blocks), dim3(PAIR_WARPS * 32), s, a, w);
    knn_pairs_kernel<<<blocks, PAIR_WARPS * 32, 0, s>>>(a, w);
    return cudaGetLastError();
}

cudaError_t launch_pair_plan(const BuildArgs &a, const Work &w, cudaStream_t s) {
    pair_plan_kernel<<<1, PLAN_THREADS, 0, s>>>(a.B, w.plan_items, w.plan_class, w.item_base, w.queue);
    pair_fill_kernel<<<(a.B + 7) / 8, 256, 0, s>>>(a.B, w.plan_items, w.item_base, w.items);
    return cudaGetLastError();
}

cudaError_t launch_pair_stage(const BuildArgs &a, const Work &w, cudaStream_t s) {
    if (a.N <= 0) return cudaSuccess;
    if (!g_pair_blocks) {
        int c = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, pair_stage_kernel, PAIR_WARPS * 32, 0);
        g_pair_blocks = max(1, c);
    }
    // persistent grids; never more warps than sources (items never outnumber them).  The
    // warp-enumeration items are usually few: two blocks per SM pull them.
    const int cap = (a.N + PAIR_WARPS - 1) / PAIR_WARPS;
    pair_legacy_kernel<<<max(1, min(cap, 2 * num_sms())), PAIR_WARPS * 32, 0, s>>>(a, w);
    pair_stage_kernel<<<max(1, min(cap, g_pair_blocks * num_sms())), PAIR_WARPS * 32, 0, s>>>(a, w);
    return cudaGetLastError();
}

}  // namespace mg
