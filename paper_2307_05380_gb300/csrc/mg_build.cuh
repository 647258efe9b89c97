// Per-source scan and emission shared by the cutoff-type builds (Def. 3, Sec. 2.1):
// a warp scans one source atom's candidates (mg_enum.cuh), classifies them by FP32
// distance with an FP64 canonical re-test in the band, stages the edges' (j, t) keys in
// shared memory in canonical order, and writes the source's edges (src, dst, t, vec,
// len) at a given row.
#pragma once

#include "mg_device.cuh"
#include "mg_enum.cuh"
#include "mg_launch.h"

namespace mg {

// Emission of one source's edges: edge q of the source goes to row base + q.
__device__ __forceinline__ void emit_edge(const mg_graph_t &g, const Source &S, int i, int64_t e, int64_t jr,
                                          float xj0, float xj1, float xj2, int t0, int t1, int t2) {
    g.src[e] = i;
    g.dst[e] = (int32_t)jr;
    g.offset[3 * e + 0] = t0;
    g.offset[3 * e + 1] = t1;
    g.offset[3 * e + 2] = t2;
    if (g.vec || g.len) {
        const float3 v = edge_vec_ff(S.L, S.xi0, S.xi1, S.xi2, xj0, xj1, xj2, t0, t1, t2);
        if (g.vec) {
            g.vec[3 * e + 0] = v.x;
            g.vec[3 * e + 1] = v.y;
            g.vec[3 * e + 2] = v.z;
        }
        if (g.len) g.len[e] = vec_len(v);
    }
}

constexpr int BUILD_WARPS = BUILD_TILE;
constexpr int BUILD_CAP = 1024;  // edges of one source staged in shared memory

// Per-source state of a cutoff-type build: the source's constants and its radius,
// thresholds and FP64 squared radius (the structure's, or per source).
struct SrcScan {
    Source S;
    float thr_lo, thr_hi, cut;
    double rr;
    int s;  // structure of the source
};

// Source constants; false when the structure is unusable (its first atom reports it).
// `permute`: the scan may enumerate in the structure's axis order (the staged scan only:
// where the scan is issue-bound the rows it saves outweigh the reordering of the keys;
// in the one-pass build the reordering lengthens each warp's latency chain instead).
template <bool PERSRC>
__device__ __forceinline__ bool source_setup(const BuildArgs &a, const Work &w, int i, SrcScan &c,
                                             bool permute = false) {
    c.s = w.atom_struct[i];
    const StructRec &R = w.recs[c.s];
    if (R.bad) {
        if (lane_id() == 0 && i == R.atom_begin) set_error(a.g.status, R.bad, c.s + a.struct_offset);
        return false;
    }
    load_source(c.S, w.recs, c.s, a.frac, w.pos, i, permute);
    c.thr_lo = R.thr_lo;
    c.thr_hi = R.thr_hi;
    c.cut = R.cut;
    c.rr = R.rr;
    if (PERSRC && a.cut_atom) {  // the source's own radius c_i (Def. 3)
        c.cut = a.cut_atom[i];
        c.rr = (double)c.cut * (double)c.cut;
        band_thresholds(R, c.cut, c.rr, a.band_rel, c.thr_lo, c.thr_hi);
    } else if (PERSRC && a.rr_atom) {  // a squared radius given in FP64 (keep-ties KNN)
        c.rr = a.rr_atom[i];
        c.cut = __double2float_ru(sqrt(c.rr)) * (1.0f + 1e-6f);
        band_thresholds(R, c.cut, c.rr, a.band_rel, c.thr_lo, c.thr_hi);
    }
    return true;
}

// One scan of a source: FP32 test, FP64 re-test in the band, the edges' (j, t) keys
// staged in `keys` (canonical order; sorted for cell-list sources and for sources
// enumerated in another axis order, whose keys are first put back in lattice order).
// Returns the edge count; `spill` when the keys did not fit or an offset exceeds the
// packed key.  With keys NULL the source is only counted.
template <bool PERSRC>
__device__ __forceinline__ int scan_source(const BuildArgs &a, const Work &w, const SrcScan &c,
                                           unsigned long long *keys, unsigned char *trim, bool &spill) {
    const Source &S = c.S;
    const Cells cells{w.cell_start, w.cell_fx, w.cell_p};
    const unsigned lt = (1u << lane_id()) - 1u;
    const bool incl = PERSRC && a.inclusive != 0;
    const float thr_lo = c.thr_lo, thr_hi = c.thr_hi;
    const double rr = c.rr;
    int m = 0;
    bool range_bad = false;
    unsigned long long nre = 0, ncand = 0;
    for_each_candidate(S, a.frac, w.pos, cells, true, c.cut, trim, [&](bool vc, float d2, bool self, int ow, int t2,
                                                                  const RowRegs &rw) {
        const bool cand = vc && !self;
        bool in = cand && d2 < thr_lo;
        const bool band = cand && !in && d2 <= thr_hi;
        if (__any_sync(FULL, in || band)) {
            const int jj = __shfl_sync(FULL, rw.j, ow);
            const int t0 = __shfl_sync(FULL, rw.t0, ow);
            const int t1 = __shfl_sync(FULL, rw.t1, ow);
            if (band) {
                // the canonical distance in lattice axis order (the identity for ax == 2)
                const int64_t jr = (int64_t)S.begin + jj;
                float Lr[9];
#pragma unroll
                for (int q = 0; q < 3; ++q) to_lattice_order(S.ax, S.L[q], S.L[3 + q], S.L[6 + q], Lr[q], Lr[3 + q], Lr[6 + q]);
                float x0, x1, x2;
                int T0, T1, T2;
                to_lattice_order(S.ax, S.xi0, S.xi1, S.xi2, x0, x1, x2);
                to_lattice_order(S.ax, t0, t1, t2, T0, T1, T2);
                const double d = canon_d2(Lr, x0, x1, x2, a.frac[3 * jr], a.frac[3 * jr + 1], a.frac[3 * jr + 2],
                                          T0, T1, T2);
                in = incl ? d <= rr : d < rr;
            }
            if (a.collect_stats) nre += __popc(__ballot_sync(FULL, band));
            const unsigned bal = __ballot_sync(FULL, in);
            if (in) {
                if (abs(t0) > OFFSET_KEY_LIM || abs(t1) > OFFSET_KEY_LIM || abs(t2) > OFFSET_KEY_LIM)
                    range_bad = true;
                const int p = m + __popc(bal & lt);
                if (keys && p < BUILD_CAP) keys[p] = ((unsigned long long)(unsigned)jj << 32) | pack_t(t0, t1, t2);
            }
            m += __popc(bal);
        }
        if (a.collect_stats) ncand += __popc(__ballot_sync(FULL, cand));
    });
    spill = m > BUILD_CAP || __any_sync(FULL, range_bad);
    if (keys && !spill && S.ax != 2) {  // offsets back in lattice order
        for (int q = lane_id(); q < m; q += 32) {
            const unsigned long long k = keys[q];
            int a0, a1, a2, t0, t1, t2;
            unpack_t((uint32_t)(k & 0xffffffffull), a0, a1, a2);
            to_lattice_order(S.ax, a0, a1, a2, t0, t1, t2);
            keys[q] = (k & 0xffffffff00000000ull) | pack_t(t0, t1, t2);
        }
        __syncwarp();
    }
    if (keys && !spill && (S.nb[0] != 0 || S.ax != 2) && m > 1) {
        if (S.nb[0] == 0 && 2 * m <= BUILD_CAP) {
            // all pairs: the keys are already in target order, only each target's run
            // (its offsets) needs reordering
            warp_smem_sort_runs_u64(keys, m);
        } else {
            int P = 64;
            while (P < m) P <<= 1;
            warp_smem_sort_u64(keys, m, P);
        }
    }
    if (a.collect_stats && lane_id() == 0 && ncand) {
        Status *st = reinterpret_cast<Status *>(a.g.status);
        atomicAdd(&st->rechecked, nre);
        atomicAdd(&st->candidates, ncand);
    }
    if (!PERSRC && a.write_pairs && spill && lane_id() == 0) w.pair_ok[c.s] = 0;  // no pair table here
    return m;
}

// The m edges of source i at rows base .. base + m - 1: from the staged keys (shared
// or global memory), recording the pair table of symmetric graphs of small structures;
// a spilled source is enumerated again in canonical all-pairs order.
template <bool PERSRC>
__device__ __forceinline__ void emit_source(const BuildArgs &a, const Work &w, const SrcScan &c, int i, int64_t base,
                                            int m, const unsigned long long *keys, unsigned char *trim, bool spill) {
    const Source &S = c.S;
    const mg_graph_t &g = a.g;
    const int lane = lane_id();
    if (!spill) {
        const bool pairs = !PERSRC && a.write_pairs && S.n <= PAIR_MAX;
        // two edges per lane and step: both targets' coordinates are loaded before
        // either edge is computed and stored, so their latencies overlap
        for (int q0 = lane; q0 < m; q0 += 64) {
            const int q1 = q0 + 32;
            const bool two = q1 < m;
            const unsigned long long k0 = keys[q0], k1 = two ? keys[q1] : k0;
            const int64_t j0 = (int64_t)S.begin + (int)(k0 >> 32), j1 = (int64_t)S.begin + (int)(k1 >> 32);
            const float x00 = a.frac[3 * j0], x01 = a.frac[3 * j0 + 1], x02 = a.frac[3 * j0 + 2];
            const float x10 = a.frac[3 * j1], x11 = a.frac[3 * j1 + 1], x12 = a.frac[3 * j1 + 2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && !two) break;
                const int q = h ? q1 : q0;
                const unsigned long long key = h ? k1 : k0;
                int t0, t1, t2;
                unpack_t((uint32_t)(key & 0xffffffffull), t0, t1, t2);
                const int jl = (int)(key >> 32);
                if (pairs) {
                    if (q == 0 || (int)(keys[q - 1] >> 32) != jl) w.pair_lo[(int64_t)i * PAIR_MAX + jl] = (uint16_t)q;
                    if (q == m - 1 || (int)(keys[q + 1] >> 32) != jl)
                        w.pair_hi[(int64_t)i * PAIR_MAX + jl] = (uint16_t)(q + 1);
                }
                if (h == 0)
                    emit_edge(g, S, i, base + q, j0, x00, x01, x02, t0, t1, t2);
                else
                    emit_edge(g, S, i, base + q, j1, x10, x11, x12, t0, t1, t2);
            }
        }
        return;
    }
    const Cells cells{w.cell_start, w.cell_fx, w.cell_p};
    const unsigned lt = (1u << lane) - 1u;
    const float thr_lo = c.thr_lo, thr_hi = c.thr_hi;
    const double rr = c.rr;
    int64_t out = base;
    const int64_t endp = base + m;
    for_each_candidate(S, a.frac, w.pos, cells, false, c.cut, trim,
                       [&](bool vc, float d2, bool self, int ow, int t2, const RowRegs &rw) {
        const bool cand = vc && !self;
        bool in = cand && d2 < thr_lo;
        const bool band = cand && !in && d2 <= thr_hi;
        if (__any_sync(FULL, in || band)) {
            const int jj = __shfl_sync(FULL, rw.j, ow);
            const int t0 = __shfl_sync(FULL, rw.t0, ow);
            const int t1 = __shfl_sync(FULL, rw.t1, ow);
            const int64_t jr = (int64_t)S.begin + jj;
            float xj0 = 0.f, xj1 = 0.f, xj2 = 0.f;
            if (in || band) {
                xj0 = a.frac[3 * jr];
                xj1 = a.frac[3 * jr + 1];
                xj2 = a.frac[3 * jr + 2];
            }
            if (band) {
                const double d = canon_d2(S.L, S.xi0, S.xi1, S.xi2, xj0, xj1, xj2, t0, t1, t2);
                in = (PERSRC && a.inclusive) ? d <= rr : d < rr;
            }
            const unsigned bal = __ballot_sync(FULL, in);
            if (in) {
                const int64_t e = out + __popc(bal & lt);
                if (e < endp) emit_edge(g, S, i, e, jr, xj0, xj1, xj2, t0, t1, t2);
            }
            out += __popc(bal);
        }
    });
    if (lane == 0 && out != endp) set_error(g.status, MG_ERR_INTERNAL, c.s);
}

// ============================================================================ look-back

// Tile status words of the decoupled look-back: value in the low 62 bits, flag on top.
constexpr unsigned long long TILE_AGG = 1ull << 62;      // tile total published
constexpr unsigned long long TILE_PREFIX = 2ull << 62;   // inclusive prefix published
constexpr unsigned long long TILE_VALUE = (1ull << 62) - 1;
constexpr int LOOKBACK_SPIN_LIMIT = 1 << 22;             // bounded wait per predecessor

__device__ __forceinline__ unsigned long long load_flag(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// Exclusive prefix of tile `tile` from its predecessors' published words.  Every wait is
// bounded: a predecessor that publishes nothing within the limit makes the build report
// MG_ERR_TIMEOUT (and the prefix is then wrong) instead of hanging.
// The warp reads the flags of the 32 nearest predecessors not yet accounted for and
// consumes them once every flag up to the nearest published prefix is set; a window with
// an unpublished flag is read again (nothing is skipped), so a tile never waits on a
// predecessor beyond its nearest prefix.  Called by a whole warp; every lane returns the
// prefix.
__device__ __forceinline__ long long tile_lookback_warp(const unsigned long long *flags, int tile, mg_device_status_t *status) {
    const int lane = lane_id();
    long long excl = 0;
    int top = tile - 1, spins = 0;
    while (top >= 0) {
        const int q = top - lane;
        const unsigned long long v = q >= 0 ? load_flag(&flags[q]) : TILE_PREFIX;  // before tile 0: prefix 0
        const unsigned long long f = v & ~TILE_VALUE;
        const unsigned pre = __ballot_sync(FULL, f == TILE_PREFIX);
        const unsigned none = __ballot_sync(FULL, f == 0);
        const int kp = pre ? __ffs(pre) - 1 : 31;  // nearest prefix in the window
        const unsigned need = kp == 31 ? FULL : ((2u << kp) - 1u);
        if (none & need) {
            if (++spins > LOOKBACK_SPIN_LIMIT) {
                // give up at the first unpublished predecessor, keeping what precedes it:
                // every tile stopped by the same silent predecessor then gets the same
                // shifted prefix, so the offsets stay monotone (the build still fails)
                const int kz = __ffs(none & need) - 1;
                excl += warp_sum(lane < kz ? (long long)(v & TILE_VALUE) : 0ll);
                if (lane == 0) set_error(status, MG_ERR_TIMEOUT, -1);
                break;
            }
            __nanosleep(32);
            continue;
        }
        excl += warp_sum(lane <= kp ? (long long)(v & TILE_VALUE) : 0ll);
        if (pre) break;
        top -= 32;
        spins = 0;
    }
    return excl;
}

}  // namespace mg
