// KNN multigraph construction (Sec. 2.1 after Def. 3; Alg. 1 and Alg. 2) on sm_103a.
//
// One warp per source atom.  Alg. 1 grows the evaluated area until the k-th distance
// d^max_i is covered; Alg. 2 keeps the k closest in an "ordered stack".  Here:
//   pass 1  scan every image within radius rho (interplanar box, mg_enum.cuh) and keep
//           the 32*S nearest images (FP32 d2 with their j and t) in registers: a sorted
//           array spread over the lanes, updated by warp-shuffle bitonic merges.  If
//           fewer than k images lie within rho, or the k-th distance tau is not covered
//           by rho with the error band to spare, rho grows and the pass repeats (the
//           covered-radius test plays the role of closest_distance(border, rho)).
//   select  images with FP32 d2 < tau - 2 delta are certainly among the k nearest;
//           images within tau +- 2 delta form the band.  When the kept images reach
//           past the band (32*S > k leaves slack) both sets are read from registers;
//           otherwise pass 2 scans again, staging the band in shared memory.  If the band
//           holds exactly the slots left, all of it is taken; otherwise it is ranked by
//           the canonical FP64 distance with the (d2, j, t) tie-break in a second
//           register top-k (GB300's FP64 rate is low, so FP64 runs only when the order
//           inside the band decides membership).  The k winners are sorted by (j, t) and
//           written in canonical order.
//           Keep-ties mode (Alg. 2's filter d <= d^k_i) writes only the k-th canonical
//           d2 of each atom; the one-pass cutoff build then emits every image that close.
// delta bounds the FP32 error (fp32_d2_error) plus the requested band.
#include <type_traits>

#include "mg_device.cuh"
#include "mg_enum.cuh"
#include "mg_launch.h"

namespace mg {

// ------------------------------------------------------------------ key types

struct FKey {
    float v;
};
__device__ __forceinline__ FKey kshfl(FKey k, int src) { return FKey{__shfl_sync(FULL, k.v, src)}; }
__device__ __forceinline__ FKey kxor(FKey k, int m) { return FKey{__shfl_xor_sync(FULL, k.v, m)}; }
__device__ __forceinline__ bool kless(FKey a, FKey b) { return a.v < b.v; }
__device__ __forceinline__ FKey kinf(FKey) { return FKey{F_INF}; }

// Exact key: canonical FP64 d2 (non-negative, so its bit pattern orders like the value),
// then (local j << 32 | packed t).
struct XKey {
    unsigned long long d, jt;
};
__device__ __forceinline__ XKey kshfl(XKey k, int src) {
    return XKey{__shfl_sync(FULL, k.d, src), __shfl_sync(FULL, k.jt, src)};
}
__device__ __forceinline__ XKey kxor(XKey k, int m) {
    return XKey{__shfl_xor_sync(FULL, k.d, m), __shfl_xor_sync(FULL, k.jt, m)};
}
__device__ __forceinline__ bool kless(XKey a, XKey b) { return a.d < b.d || (a.d == b.d && a.jt < b.jt); }
__device__ __forceinline__ XKey kinf(XKey) { return XKey{~0ull, ~0ull}; }

// FP32 key with the candidate's (local j << 32 | packed t): pass 1 keeps the 32 S nearest
// images themselves, ordered by (d2, j, t).
struct CKey {
    float v;
    unsigned long long jt;
};
__device__ __forceinline__ CKey kshfl(CKey k, int src) {
    return CKey{__shfl_sync(FULL, k.v, src), __shfl_sync(FULL, k.jt, src)};
}
__device__ __forceinline__ CKey kxor(CKey k, int m) {
    return CKey{__shfl_xor_sync(FULL, k.v, m), __shfl_xor_sync(FULL, k.jt, m)};
}
__device__ __forceinline__ bool kless(CKey a, CKey b) { return a.v < b.v || (a.v == b.v && a.jt < b.jt); }
__device__ __forceinline__ CKey kinf(CKey) { return CKey{F_INF, ~0ull}; }
constexpr unsigned long long JT_OUT_OF_RANGE = ~0ull - 1;  // an offset the packed key cannot hold

template <class K>
__device__ __forceinline__ K kmin(K a, K b) { return kless(b, a) ? b : a; }
template <class K>
__device__ __forceinline__ K kmax(K a, K b) { return kless(b, a) ? a : b; }

// Bitonic sort of one key per lane, ascending by lane.
template <class K>
__device__ __forceinline__ K warp_bitonic_sort(K x) {
    const int lane = lane_id();
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
        const bool desc = (lane & size) != 0;
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const K y = kxor(x, stride);
            const bool lower = (lane & stride) == 0;
            x = (lower != desc) ? kmin(x, y) : kmax(x, y);
        }
    }
    return x;
}

// A bitonic sequence across the lanes, sorted ascending.
template <class K>
__device__ __forceinline__ K warp_bitonic_merge(K x) {
    const int lane = lane_id();
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
        const K y = kxor(x, stride);
        x = ((lane & stride) == 0) ? kmin(x, y) : kmax(x, y);
    }
    return x;
}

// The 32*S smallest keys seen so far, sorted: slot s of lane l holds rank 32 s + l.
template <class K, int S>
struct TopK {
    K a[S];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int s = 0; s < S; ++s) a[s] = kinf(K{});
    }
    // Merge one key per lane (kinf for none).
    __device__ __forceinline__ void insert(K b) {
        const int lane = lane_id();
        b = warp_bitonic_sort(b);
        // the 32 smallest of the top block and b (a bitonic split), sorted
        K m = kmin(a[S - 1], kshfl(b, 31 - lane));
        m = warp_bitonic_merge(m);
        // ripple m down through the sorted blocks
#pragma unroll
        for (int s = 0; s < S - 1; ++s) {
            const K rm = kshfl(m, 31 - lane);
            const K lo = kmin(a[s], rm), hi = kmax(a[s], rm);
            a[s] = warp_bitonic_merge(lo);
            m = warp_bitonic_merge(hi);
        }
        a[S - 1] = m;
    }
    // The r-th smallest (1-based, r <= 32 S), the same in every lane.
    __device__ __forceinline__ K kth(int r) const {
        const int idx = r - 1, blk = idx >> 5, l = idx & 31;
        K v = a[0];
#pragma unroll
        for (int s = 1; s < S; ++s)
            if (s == blk) v = a[s];
        return kshfl(v, l);
    }
};

// Work distribution over source atoms (same scheme as the cutoff kernels): a flat grid
// (1), a persistent grid pulling atoms from a counter (2), or a persistent grid pulling
// the atoms of the pair-lane KNN's fallback list (3: list[0 .. queue[10]), cursor
// queue[11]).
template <int SCHED>
struct KnnLoop {
    int lo, hi;
    unsigned int *queue;
    const int *list = nullptr;
    __device__ __forceinline__ int first() {
        if (SCHED == 1) return lo + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
        return next();
    }
    __device__ __forceinline__ int next() {
        if (SCHED == 1) return hi;
        unsigned int v = 0;
        if (lane_id() == 0) v = atomicAdd(queue + (SCHED == 3 ? 11 : 1), 1u);
        v = __shfl_sync(FULL, v, 0);
        if (SCHED == 3) return v < queue[10] ? list[v] : hi;
        return lo + (int)v;
    }
};

constexpr int KNN_WARPS = 4;
constexpr int BAND_CAP = 64;  // band candidates staged per source in shared memory

// At most 85 registers (6 blocks of 4 warps per SM): measured faster than 128 registers
// (fewer resident warps) and than 64 (more spills) on the bench workloads.
// ONEPASS: pass 1 keeps (d2, j, t) keys and the selection usually reads them from
// registers; otherwise pass 1 keeps FP32 distances only (fewer registers and shuffles)
// and pass 2 always scans again.
template <int S, int SCHED, bool ONEPASS>
__global__ void __launch_bounds__(KNN_WARPS * 32, 6) knn_kernel(BuildArgs a, Work w) {
    using PKey = typename std::conditional<ONEPASS, CKey, FKey>::type;
    __shared__ unsigned long long sel_all[KNN_WARPS][S * 32 > 64 ? S * 32 : 64];
    __shared__ unsigned long long band_all[KNN_WARPS][BAND_CAP];
    __shared__ float bufv_all[KNN_WARPS][64];               // pass-1 candidates waiting for a merge
    __shared__ unsigned long long bufjt_all[KNN_WARPS][64];
    pdl_wait();  // prep's records and positions (a no-op unless launched behind prep)
    const int wid = threadIdx.x >> 5, lane = lane_id();
    unsigned long long *sel = sel_all[wid];
    unsigned long long *bl = band_all[wid];
    float *bufv = bufv_all[wid];
    unsigned long long *bufjt = bufjt_all[wid];
    const int k = a.knn_k;
    const unsigned lt = (1u << lane) - 1u;
    const mg_graph_t g = a.g;
    KnnLoop<SCHED> loop{a.atom_lo, a.atom_hi, w.queue, reinterpret_cast<const int *>(w.items)};
    const Cells cells{w.cell_start, w.cell_fx, w.cell_p};
    unsigned long long nre = 0, ncand = 0;

    for (int i = loop.first(); i < a.atom_hi; i = loop.next()) {
        const int s = w.atom_struct[i];
        const StructRec &R = w.recs[s];
        if (R.bad) {
            if (lane == 0 && i == R.atom_begin) set_error(g.status, R.bad, s + a.struct_offset);
            continue;
        }
        Source Src;
        load_source(Src, w.recs, s, a.frac, w.pos, i);

        // ---------------- pass 1: grow rho until the k-th FP32 distance is covered; the
        // 32 S nearest images are kept with their (j, t)
        float rho = R.cut, tau = F_INF, delta = 0.f;
        bool ok = false;
        TopK<PKey, S> tk;
        for (int iter = 0; iter < 64 && !ok; ++iter) {
            tk.init();
            float thr = F_INF;  // images at least this far cannot enter the kept set
            int found = 0, nbuf = 0;
            const float rho2 = rho * rho;
            // candidates below thr wait in shared memory; 32 at a time go through one
            // register merge (thr is refreshed then: a stale thr only admits more)
            auto merge = [&](int from, int cnt) {
                const int q = from + lane;
                const bool have = lane < cnt;
                const float v = have ? bufv[q] : F_INF;
                if constexpr (ONEPASS) {
                    tk.insert(CKey{v, have ? bufjt[q] : ~0ull});
                    thr = tk.kth(32 * S).v;  // the kept images are the 32 S nearest seen
                } else {
                    tk.insert(FKey{v});
                    thr = tk.kth(k).v;
                }
            };
            for_each_candidate(Src, a.frac, w.pos, cells, true, rho, nullptr, [&](bool vc, float d2, bool self, int ow,
                                                                          int t2, const RowRegs &rw) {
                const bool c = vc && !self && d2 < rho2;
                found += __popc(__ballot_sync(FULL, c));
                const bool ins = c && d2 < thr;
                const unsigned bal = __ballot_sync(FULL, ins);
                if (bal) {
                    const int p = nbuf + __popc(bal & lt);
                    if constexpr (ONEPASS) {
                        const int jj = __shfl_sync(FULL, rw.j, ow);
                        const int t0 = __shfl_sync(FULL, rw.t0, ow);
                        const int t1 = __shfl_sync(FULL, rw.t1, ow);
                        if (ins)
                            bufjt[p] = (abs(t0) > OFFSET_KEY_LIM || abs(t1) > OFFSET_KEY_LIM || abs(t2) > OFFSET_KEY_LIM)
                                           ? JT_OUT_OF_RANGE
                                           : (((unsigned long long)(unsigned)jj << 32) | pack_t(t0, t1, t2));
                    }
                    if (ins) bufv[p] = d2;
                    nbuf += __popc(bal);
                    if (nbuf >= 32) {  // merge the last 32, keep the rest waiting
                        __syncwarp();
                        nbuf -= 32;
                        merge(nbuf, 32);
                        __syncwarp();
                    }
                }
                if (a.collect_stats) ncand += __popc(__ballot_sync(FULL, vc && !self));
            });
            if (nbuf > 0) {
                __syncwarp();
                merge(0, nbuf);
                nbuf = 0;
                __syncwarp();
            }
            thr = tk.kth(k).v;
            delta = fp32_d2_error(R, rho, rho2) + 2.0f * a.band_rel * rho2;
            if (found >= k && thr + 3.0f * delta < rho2) {
                tau = thr;
                ok = true;
            } else if (found >= k) {
                rho = sqrtf(thr + 3.0f * delta) * 1.0005f + 1e-6f;
            } else {
                rho *= 1.5f;
            }
            if (!(rho < 1e6f)) break;
        }
        if (!ok) {
            if (lane == 0) set_error(g.status, MG_ERR_OFFSET_RANGE, s);
            continue;
        }

        const float lo_thr = tau - 2.0f * delta, hi_thr = tau + 2.0f * delta;
        unsigned long long dk_bits = 0;  // keep-ties mode: the k-th canonical d2
        bool spare = false;
        if constexpr (ONEPASS) spare = tk.kth(32 * S).v > hi_thr;
        if (spare) {
          if constexpr (ONEPASS) {
            // ---------------- the kept images hold every certain member (FP32 d2 below
            // tau - 2 delta) and the whole band: no second scan.  Ranks [0, m) are
            // certain, [m, m + nb) the band, ranked in FP64 only if it holds more
            // candidates than the slots left.
            int m = 0, nb = 0;
            bool range_bad = false;
#pragma unroll
            for (int q = 0; q < S; ++q) {
                const CKey c = tk.a[q];
                m += __popc(__ballot_sync(FULL, c.v < lo_thr));
                nb += __popc(__ballot_sync(FULL, c.v >= lo_thr && c.v <= hi_thr));
                if (c.v <= hi_thr && c.jt == JT_OUT_OF_RANGE) range_bad = true;
            }
            if (__any_sync(FULL, range_bad)) {
                if (lane == 0) set_error(g.status, MG_ERR_OFFSET_RANGE, s);
                continue;
            }
            if (m >= k || m + nb < k) {  // cannot happen: fewer than k FP32 distances lie below tau
                if (lane == 0) set_error(g.status, MG_ERR_INTERNAL, s);
                continue;
            }
            const int need = k - m;
            if (nb == need) {  // every band member fills a remaining slot
#pragma unroll
                for (int q = 0; q < S; ++q) {
                    const int r = 32 * q + lane;
                    if (r < k) sel[r] = tk.a[q].jt;
                    if (a.knn_dk && r >= m && r < k) {
                        const unsigned long long jt = tk.a[q].jt;
                        int t0, t1, t2;
                        unpack_t((uint32_t)(jt & 0xffffffffull), t0, t1, t2);
                        const int64_t jr = (int64_t)Src.begin + (int)(jt >> 32);
                        const double d = canon_d2(Src.L, Src.xi0, Src.xi1, Src.xi2, a.frac[3 * jr],
                                                  a.frac[3 * jr + 1], a.frac[3 * jr + 2], t0, t1, t2);
                        const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
                        dk_bits = bits > dk_bits ? bits : dk_bits;
                    }
                }
                if (a.knn_dk) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long y = __shfl_xor_sync(FULL, dk_bits, o);
                        dk_bits = y > dk_bits ? y : dk_bits;
                    }
                }
            } else {  // rank the band by (canonical FP64 d2, j, t)
                if (a.collect_stats) nre += nb;
                TopK<XKey, S> ek;
                ek.init();
#pragma unroll
                for (int q = 0; q < S; ++q) {
                    const int r = 32 * q + lane;
                    const unsigned long long jt = tk.a[q].jt;
                    if (r < m) sel[r] = jt;
                    XKey key = kinf(XKey{});
                    if (r >= m && r < m + nb) {
                        int t0, t1, t2;
                        unpack_t((uint32_t)(jt & 0xffffffffull), t0, t1, t2);
                        const int64_t jr = (int64_t)Src.begin + (int)(jt >> 32);
                        const double d = canon_d2(Src.L, Src.xi0, Src.xi1, Src.xi2, a.frac[3 * jr],
                                                  a.frac[3 * jr + 1], a.frac[3 * jr + 2], t0, t1, t2);
                        key = XKey{(unsigned long long)__double_as_longlong(d), jt};
                    }
                    ek.insert(key);
                }
#pragma unroll
                for (int q = 0; q < S; ++q) {
                    const int p = q * 32 + lane;
                    if (p < need) sel[m + p] = ek.a[q].jt;
                }
                if (a.knn_dk) dk_bits = ek.kth(need).d;
            }
            __syncwarp();
          }
        } else {
            // ---------------- pass 2 (the band reaches past the kept images): certain members;
            // the band is staged, then ranked only if it holds more candidates than the slots
            // left (FP64 only in that case)
            int m = 0, nb = 0;
            bool range_bad = false;
            for_each_candidate(Src, a.frac, w.pos, cells, true, rho, nullptr, [&](bool vc, float d2, bool self, int ow, int t2,
                                                                          const RowRegs &rw) {
                const bool c = vc && !self;
                const bool in = c && d2 < lo_thr;
                const bool band = c && !in && d2 <= hi_thr;
                if (__any_sync(FULL, in || band)) {
                    const int jj = __shfl_sync(FULL, rw.j, ow);
                    const int t0 = __shfl_sync(FULL, rw.t0, ow);
                    const int t1 = __shfl_sync(FULL, rw.t1, ow);
                    if ((in || band) && (abs(t0) > OFFSET_KEY_LIM || abs(t1) > OFFSET_KEY_LIM || abs(t2) > OFFSET_KEY_LIM))
                        range_bad = true;
                    const unsigned long long jt = ((unsigned long long)(unsigned)jj << 32) | pack_t(t0, t1, t2);
                    const unsigned bin = __ballot_sync(FULL, in);
                    if (in) {
                        const int p = m + __popc(bin & lt);
                        if (p < k) sel[p] = jt;
                    }
                    m += __popc(bin);
                    const unsigned bb = __ballot_sync(FULL, band);
                    if (band) {
                        const int p = nb + __popc(bb & lt);
                        if (p < BAND_CAP) bl[p] = jt;
                    }
                    nb += __popc(bb);
                }
            });
            if (__any_sync(FULL, range_bad)) {
                if (lane == 0) set_error(g.status, MG_ERR_OFFSET_RANGE, s);
                continue;
            }
            if (m >= k || m + nb < k) {  // cannot happen: fewer than k FP32 distances lie below tau
                if (lane == 0) set_error(g.status, MG_ERR_INTERNAL, s);
                continue;
            }
            const int need = k - m;
            __syncwarp();
            // the k-th canonical d2 (keep-ties mode): the largest selected band member, since
            // every certain member lies below tau - delta and the k-th distance does not
            if (nb == need && nb <= BAND_CAP) {  // every band member fills a remaining slot
                for (int q = lane; q < nb; q += 32) sel[m + q] = bl[q];
                if (a.knn_dk) {
                    for (int q = lane; q < nb; q += 32) {
                        const unsigned long long jt = bl[q];
                        int t0, t1, t2;
                        unpack_t((uint32_t)(jt & 0xffffffffull), t0, t1, t2);
                        const int64_t jr = (int64_t)Src.begin + (int)(jt >> 32);
                        const double d = canon_d2(Src.L, Src.xi0, Src.xi1, Src.xi2, a.frac[3 * jr], a.frac[3 * jr + 1],
                                                  a.frac[3 * jr + 2], t0, t1, t2);
                        const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
                        dk_bits = bits > dk_bits ? bits : dk_bits;  // non-negative: bits order like values
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long y = __shfl_xor_sync(FULL, dk_bits, o);
                        dk_bits = y > dk_bits ? y : dk_bits;
                    }
                }
            } else {  // rank the band by (canonical FP64 d2, j, t)
                TopK<XKey, S> ek;
                ek.init();
                if (a.collect_stats) nre += nb;
                if (nb <= BAND_CAP) {
                    for (int b0 = 0; b0 < nb; b0 += 32) {
                        const int q = b0 + lane;
                        XKey key = kinf(XKey{});
                        if (q < nb) {
                            const unsigned long long jt = bl[q];
                            int t0, t1, t2;
                            unpack_t((uint32_t)(jt & 0xffffffffull), t0, t1, t2);
                            const int64_t jr = (int64_t)Src.begin + (int)(jt >> 32);
                            const double d = canon_d2(Src.L, Src.xi0, Src.xi1, Src.xi2, a.frac[3 * jr], a.frac[3 * jr + 1],
                                                      a.frac[3 * jr + 2], t0, t1, t2);
                            key = XKey{(unsigned long long)__double_as_longlong(d), jt};
                        }
                        ek.insert(key);
                    }
                } else {  // the band did not fit in shared memory: stream it again with FP64 keys
                    XKey ethr = kinf(XKey{});
                    for_each_candidate(Src, a.frac, w.pos, cells, true, rho, nullptr, [&](bool vc, float d2, bool self, int ow,
                                                                                  int t2, const RowRegs &rw) {
                        const bool c = vc && !self;
                        const bool band = c && d2 >= lo_thr && d2 <= hi_thr;
                        if (__any_sync(FULL, band)) {
                            const int jj = __shfl_sync(FULL, rw.j, ow);
                            const int t0 = __shfl_sync(FULL, rw.t0, ow);
                            const int t1 = __shfl_sync(FULL, rw.t1, ow);
                            XKey key = kinf(XKey{});
                            if (band) {
                                const int64_t jr = (int64_t)Src.begin + jj;
                                const double d = canon_d2(Src.L, Src.xi0, Src.xi1, Src.xi2, a.frac[3 * jr],
                                                          a.frac[3 * jr + 1], a.frac[3 * jr + 2], t0, t1, t2);
                                key = XKey{(unsigned long long)__double_as_longlong(d),
                                           ((unsigned long long)(unsigned)jj << 32) | pack_t(t0, t1, t2)};
                            }
                            const bool ins = band && kless(key, ethr);
                            if (__any_sync(FULL, ins)) {
                                ek.insert(ins ? key : kinf(XKey{}));
                                ethr = ek.kth(k);
                            }
                        }
                    });
                }
#pragma unroll
                for (int q = 0; q < S; ++q) {
                    const int p = q * 32 + lane;
                    if (p < need) sel[m + p] = ek.a[q].jt;
                }
                if (a.knn_dk) dk_bits = ek.kth(need).d;
            }
            __syncwarp();
        }  // pass 2
        if (a.knn_dk) {  // keep-ties mode: the radius only; a cutoff pass emits the edges
            if (lane == 0) a.knn_dk[i] = __longlong_as_double((long long)dk_bits);
            continue;
        }
        // canonical (j, t) order of the k winners
        if (k <= 32) {
            unsigned long long v = lane < k ? sel[lane] : ~0ull;
            // 64-bit bitonic sort across lanes
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
            if (lane < k) sel[lane] = v;
            __syncwarp();
        } else {
            int P = 64;
            while (P < k) P <<= 1;
            warp_smem_sort_u64(sel, k, P);
        }
        // write k edges at rows i*k .. i*k + k - 1
        for (int q = lane; q < k; q += 32) {
            const unsigned long long jt = sel[q];
            const int jl = (int)(jt >> 32);
            int t0, t1, t2;
            unpack_t((uint32_t)(jt & 0xffffffffull), t0, t1, t2);
            const int64_t jr = (int64_t)Src.begin + jl;
            const int64_t e = (int64_t)i * k + q;
            g.src[e] = i;
            g.dst[e] = (int32_t)jr;
            g.offset[3 * e + 0] = t0;
            g.offset[3 * e + 1] = t1;
            g.offset[3 * e + 2] = t2;
            if (g.vec || g.len) {
                const float3 v = edge_vec_ff(Src.L, Src.xi0, Src.xi1, Src.xi2, a.frac[3 * jr], a.frac[3 * jr + 1],
                                             a.frac[3 * jr + 2], t0, t1, t2);
                if (g.vec) {
                    g.vec[3 * e + 0] = v.x;
                    g.vec[3 * e + 1] = v.y;
                    g.vec[3 * e + 2] = v.z;
                }
                if (g.len) g.len[e] = vec_len(v);
            }
        }
        __syncwarp();
    }
    if (a.collect_stats && lane == 0 && (ncand || nre)) {
        Status *st = reinterpret_cast<Status *>(g.status);
        atomicAdd(&st->rechecked, nre);
        atomicAdd(&st->candidates, ncand);
    }
}

template <int S, bool ONEPASS>
static cudaError_t launch_knn_s(const BuildArgs &a, const Work &w, cudaStream_t s) {
    const int atoms = a.atom_hi - a.atom_lo;
    const int threads = KNN_WARPS * 32;
    const int flat_blocks = (atoms + KNN_WARPS - 1) / KNN_WARPS;
    if (a.knn_list) {  // the sources the pair-lane KNN left: usually few, two blocks per SM
        knn_kernel<S, 3, ONEPASS><<<max(1, min(flat_blocks, 2 * num_sms())), threads, 0, s>>>(a, w);
    } else if (a.schedule == 2) {
        cudaError_t e = launch_reset_queue(w, s);
        if (e) return e;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, knn_kernel<S, 2, ONEPASS>, threads, 0);
        int blocks = max(1, per_sm) * num_sms();
        blocks = min(blocks, flat_blocks);
        knn_kernel<S, 2, ONEPASS><<<blocks, threads, 0, s>>>(a, w);
    } else {
        if (a.pdl) return launch_pdl(knn_kernel<S, 1, ONEPASS>, dim3(flat_blocks), dim3(threads), s, a, w);
        knn_kernel<S, 1, ONEPASS><<<flat_blocks, threads, 0, s>>>(a, w);
    }
    return cudaGetLastError();
}

// k <= 24: one warp-wide block of keys (d2, j, t) holds k plus at least 8 spare images,
// so the band usually fits and the second scan is skipped.  Larger k: FP32 distances
// only and two scans (measured faster at k = 32 than 64 keys with their (j, t)).
cudaError_t launch_knn(const BuildArgs &a, const Work &w, cudaStream_t s) {
    if (a.atom_hi <= a.atom_lo) return cudaSuccess;
    if (a.knn_k <= 24) return launch_knn_s<1, true>(a, w, s);
    if (a.knn_k <= 56) return launch_knn_s<2, true>(a, w, s);
    return launch_knn_s<4, false>(a, w, s);
}

// src_ptr[i] = k i, edge_ptr[s] = k atom_ptr[s], status counts.
__global__ void knn_pointers_kernel(int B, int N, int k, const int32_t *__restrict__ atom_ptr,
                                    int64_t *__restrict__ src_ptr, int64_t *__restrict__ edge_ptr,
                                    mg_device_status_t *status, int atom_lo, int atom_hi, int s_lo, int s_hi) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (src_ptr)
        for (int64_t q = atom_lo + tid; q <= atom_hi; q += stride) src_ptr[q] = q * k;
    for (int64_t q = s_lo + tid; q <= s_hi; q += stride) edge_ptr[q] = (int64_t)(q == B ? N : atom_ptr[q]) * k;
    if (tid == 0 && s_hi == B) {
        Status *st = reinterpret_cast<Status *>(status);
        st->num_edges = (unsigned long long)N * k;
        st->required_capacity = (unsigned long long)N * k;
    }
}

cudaError_t launch_knn_pointers(const BuildArgs &a, const Work &, cudaStream_t s) {
    // structures [0, B] and atoms [atom_lo, atom_hi] of this call
    const int n = max(a.atom_hi - a.atom_lo + 1, a.B + 1);
    const int threads = 256;
    const int blocks = min(1024, (n + threads - 1) / threads);
    knn_pointers_kernel<<<blocks, threads, 0, s>>>(a.B, a.N, a.knn_k, a.atom_ptr, a.src_ptr, a.g.edge_ptr,
                                                    a.g.status, a.atom_lo, a.atom_hi, 0, a.B);
    return cudaGetLastError();
}

}  // namespace mg
