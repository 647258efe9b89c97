// Device-side building blocks shared by the matgraph kernels (sm_103a).
//
// Geometry conventions follow Def. 1 and Def. 3 (Sec. 2.1): lattice rows are lattice
// vectors, an edge (i, j, t) has vector v = (x_j - x_i + t) L.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "matgraph.h"

namespace mg {

constexpr unsigned FULL = 0xffffffffu;
constexpr float F_INF = __builtin_huge_valf();
constexpr int KNN_MAX_K = 128;      // k limit of the register top-k (4 slots per lane)
constexpr int OFFSET_KEY_LIM = 511; // |t_k| bound of the 10-bit packed offset key

// Per-structure record written by the prep kernel.
struct StructRec {
    float L[9];        // lattice rows (caller's FP32 values)
    float invd[3];     // ||L^-1[:, k]|| = 1/d_k (interplanar spacing d_k), rounded up
    float cut;         // cutoff radius (cutoff graphs) or starting radius (KNN)
    float thr_lo;      // FP32 d2 below this: certainly an edge (cutoff graphs)
    float thr_hi;      // FP32 d2 above this: certainly not an edge
    float errP[3];     // per Cartesian component c: sum_k Xmax_k |L_kc|
    float errL[3];     // per component: sum_k invd_k |L_kc|
    float errC[3];     // per component: sum_k (2 Xmax_k + 1) |L_kc|
    float L2norm2;     // |L_2|^2
    float L2norm;      // |L_2|
    double rr;         // canonical squared cutoff, (double)c * (double)c
    int32_t atom_begin;
    int32_t n_atoms;
    int32_t bad;       // mg_status_t for this structure (0 = usable)
    int32_t nb[3];     // cell-list bins per axis; nb[0] == 0: the structure uses all pairs
    int32_t bin_base;  // first bin of the structure: atom_begin + structure index
    int32_t ax;        // lattice axis the cutoff scan runs its candidates along (2: none moved)
    int32_t pl;        // > 0: the pair-lane scan takes the structure: B0 B1 B2 <= PL_BOX_MAX
                       // for the largest extents B_k of any pair's offset box, whose offsets
                       // fit the packed key; pl = B2 | B1 << 8 | B0 << 16
    float reach[3];    // pair-lane scan: c / d_k plus the structure's margin; a pair's box
                       // along axis k is ceil(-reach_k - dx_k) .. floor(reach_k - dx_k).
                       // KNN graphs: the margin's constant part, 1e-5 (1 + 2 max|x_k|)
};
static_assert(sizeof(StructRec) == 160, "record layout");

constexpr int PL_BOX_MAX = 64;  // offset-box cells one lane evaluates for its pair (a 64-bit mask)
constexpr int PL_MAX_ATOMS = 512;  // largest structure of the pair-lane scan (16 chunks of 32 targets)

constexpr int CELL_MIN_ATOMS = 128;  // smallest structure that may use a cell list
constexpr int WRITE_CAP = 1024;      // edges of one source sorted in shared memory

struct alignas(8) Status {  // device mirror of mg_device_status_t
    int32_t code;
    int32_t first_bad_structure;
    unsigned long long num_edges;
    unsigned long long required_capacity;
    unsigned long long rechecked;
    unsigned long long candidates;
};
static_assert(sizeof(Status) == sizeof(mg_device_status_t), "status layout");

__device__ __forceinline__ void set_error(mg_device_status_t *st, int code, int structure) {
    Status *s = reinterpret_cast<Status *>(st);
    atomicCAS(&s->code, 0, code);
    if (structure >= 0) atomicMin(&s->first_bad_structure, structure);
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// A source whose keys a staged build could not stage: appended to the spill list, which
// the spill kernel enumerates again (list [N], count queue[12]).
__device__ __forceinline__ void note_spill(int32_t *list, unsigned int *queue, int i) {
    list[atomicAdd(&queue[12], 1u)] = i;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the kernel before it in the stream is still running;
// pdl_wait() returns once that kernel has completed and its writes are visible (at once
// for a kernel launched without the attribute).  pdl_trigger() lets the next kernel's
// launch begin as soon as every block of this one has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Host side: launch `kernel` with programmatic stream serialization (its first global
// access must follow pdl_wait()).
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, cudaStream_t s, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A &&>(args)...);
}

// ------------------------------------------------------------------ warp scans

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Index of the lane owning flat position q, given each lane's inclusive prefix `incl`
// (non-decreasing across lanes, q < incl of lane 31): the first lane with incl > q.
__device__ __forceinline__ int warp_owner(int incl, int q) {
    int owner = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        int v = __shfl_sync(FULL, incl, owner + s - 1);
        if (v <= q) owner += s;
    }
    return owner;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// ------------------------------------------------------------------ FP32 distance

// Cartesian position p = x L, FP32 fused multiply-adds in a fixed order.
__device__ __forceinline__ float3 cart(const float *L, float x0, float x1, float x2) {
    float3 p;
    p.x = __fmaf_rn(x2, L[6], __fmaf_rn(x1, L[3], __fmul_rn(x0, L[0])));
    p.y = __fmaf_rn(x2, L[7], __fmaf_rn(x1, L[4], __fmul_rn(x0, L[1])));
    p.z = __fmaf_rn(x2, L[8], __fmaf_rn(x1, L[5], __fmul_rn(x0, L[2])));
    return p;
}

__device__ __forceinline__ float norm2f(float3 v) {
    return __fmaf_rn(v.z, v.z, __fmaf_rn(v.y, v.y, __fmul_rn(v.x, v.x)));
}

// ------------------------------------------------------------------ canonical FP64

// The canonical distance that decides membership and ranking (identical to the
// definition the oracle follows): double inputs, every operation rounded to nearest,
// no contraction, left-to-right sums.
__device__ __forceinline__ double canon_d2(const float *L, float xi0, float xi1, float xi2,
                                           float xj0, float xj1, float xj2, int t0, int t1, int t2) {
    double df0 = __dadd_rn(__dsub_rn((double)xj0, (double)xi0), (double)t0);
    double df1 = __dadd_rn(__dsub_rn((double)xj1, (double)xi1), (double)t1);
    double df2 = __dadd_rn(__dsub_rn((double)xj2, (double)xi2), (double)t2);
    double v0 = __dadd_rn(__dadd_rn(__dmul_rn(df0, (double)L[0]), __dmul_rn(df1, (double)L[3])),
                          __dmul_rn(df2, (double)L[6]));
    double v1 = __dadd_rn(__dadd_rn(__dmul_rn(df0, (double)L[1]), __dmul_rn(df1, (double)L[4])),
                          __dmul_rn(df2, (double)L[7]));
    double v2 = __dadd_rn(__dadd_rn(__dmul_rn(df0, (double)L[2]), __dmul_rn(df1, (double)L[5])),
                          __dmul_rn(df2, (double)L[8]));
    return __dadd_rn(__dadd_rn(__dmul_rn(v0, v0), __dmul_rn(v1, v1)), __dmul_rn(v2, v2));
}

// ------------------------------------------------------------------ float-float vec

// Error-free transformations (Knuth's TwoSum; TwoProd through fused multiply-add).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Edge vector v = (x_j - x_i + t) L with the difference carried exactly as a
// float-float pair and the three-term dot products compensated (Ogita-Rump-Oishi
// Dot2), then rounded once: the result is within about one FP32 rounding of the exact
// vector even when the terms cancel (skewed cells, large offsets).
__device__ __forceinline__ float3 edge_vec_ff(const float *L, float xi0, float xi1, float xi2,
                                              float xj0, float xj1, float xj2, int t0, int t1, int t2) {
    float hi[3], lo[3];
    {
        const float xi[3] = {xi0, xi1, xi2}, xj[3] = {xj0, xj1, xj2};
        const int t[3] = {t0, t1, t2};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float s, e, s2, e2;
            two_sum(xj[k], -xi[k], s, e);
            two_sum(s, (float)t[k], s2, e2);
            hi[k] = s2;
            lo[k] = __fadd_rn(e2, e);
        }
    }
    float out[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float p0, q0, p1, q1, p2, q2;
        two_prod(hi[0], L[0 + c], p0, q0);
        two_prod(hi[1], L[3 + c], p1, q1);
        two_prod(hi[2], L[6 + c], p2, q2);
        float s, e1, e2;
        two_sum(p0, p1, s, e1);
        two_sum(s, p2, s, e2);
        float corr = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(q0, q1), q2));
        corr = __fmaf_rn(lo[0], L[0 + c], corr);
        corr = __fmaf_rn(lo[1], L[3 + c], corr);
        corr = __fmaf_rn(lo[2], L[6 + c], corr);
        out[c] = __fadd_rn(s, corr);
    }
    return make_float3(out[0], out[1], out[2]);
}

__device__ __forceinline__ float vec_len(float3 v) {
    return __fsqrt_rn(__fmaf_rn(v.z, v.z, __fmaf_rn(v.y, v.y, __fmul_rn(v.x, v.x))));
}

// ------------------------------------------------------------------ axis order

// A scan may enumerate a structure's offsets with lattice axis `ax` innermost: position q
// of its (a0, a1, a2) then holds axis (p0, p1, ax)[q], p0 < p1 the other two.  Back to
// lattice order (the identity for ax == 2):
template <class T>
__device__ __forceinline__ void to_lattice_order(int ax, T a0, T a1, T a2, T &t0, T &t1, T &t2) {
    t0 = ax == 0 ? a2 : a0;
    t1 = ax == 0 ? a0 : (ax == 1 ? a2 : a1);
    t2 = ax == 2 ? a2 : a1;
}

// ------------------------------------------------------------------ packed offsets

__device__ __forceinline__ uint32_t pack_t(int t0, int t1, int t2) {
    return ((uint32_t)(t0 + 512) << 20) | ((uint32_t)(t1 + 512) << 10) | (uint32_t)(t2 + 512);
}
__device__ __forceinline__ void unpack_t(uint32_t p, int &t0, int &t1, int &t2) {
    t0 = (int)((p >> 20) & 1023u) - 512;
    t1 = (int)((p >> 10) & 1023u) - 512;
    t2 = (int)(p & 1023u) - 512;
}

// Sort n (<= P, P a power of two >= 64) 64-bit keys in shared memory with one warp
// (bitonic network; pads [n, P) with the largest key).
__device__ __forceinline__ void warp_smem_sort_u64(unsigned long long *b, int n, int P) {
    const int lane = lane_id();
    for (int q = n + lane; q < P; q += 32) b[q] = ~0ull;
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
        for (int ls = __ffs(size) - 2; ls >= 0; --ls) {  // stride = 2^ls
            const int stride = 1 << ls;
            for (int q = lane; q < P / 2; q += 32) {
                const int x = ((q >> ls) << (ls + 1)) | (q & (stride - 1));
                const int y = x + stride;
                const bool asc = (x & size) == 0;
                const unsigned long long vx = b[x], vy = b[y];
                if ((vx > vy) == asc) {
                    b[x] = vy;
                    b[y] = vx;
                }
            }
            __syncwarp();
        }
    }
}

// Sort n distinct 64-bit keys in shared memory with one warp when they are already
// grouped into runs of equal high words in ascending order: each key moves to its run's
// first position plus its rank within the run (a scan over the run, which is short where
// this is used), through b[n, 2n) as scratch, so 2n must fit the buffer.
__device__ __forceinline__ void warp_smem_sort_runs_u64(unsigned long long *b, int n) {
    const int lane = lane_id();
    for (int q = lane; q < n; q += 32) {
        const unsigned long long k = b[q];
        const unsigned hk = (unsigned)(k >> 32);
        int lo = q, hi = q + 1;
        while (lo > 0 && (unsigned)(b[lo - 1] >> 32) == hk) --lo;
        while (hi < n && (unsigned)(b[hi] >> 32) == hk) ++hi;
        int r = 0;
        for (int p = lo; p < hi; ++p) r += b[p] < k ? 1 : 0;
        b[n + lo + r] = k;
    }
    __syncwarp();
    for (int q = lane; q < n; q += 32) b[q] = b[n + q];
    __syncwarp();
}

// ------------------------------------------------------------------ error model

// Bound on |d2_fp32 - d2_canonical| for candidates enumerated within radius rho of a
// structure (the FP32 path forms p = x L per atom, then v = (p_j - p_i) + t L with
// fused multiply-adds, then d2).  Per component the vector error is at most
// 8u (2 P_c + T_c) with T_c <= rho errL_c + errC_c the offset term; the squared norm
// then moves by at most 3.1u d2 + 2|v| |eps| + |eps|^2.  The result is doubled.
__device__ __forceinline__ float fp32_d2_error(const StructRec &R, float rho, float d2) {
    const float u8 = 8.0f * 5.9604645e-8f;
    float e0 = u8 * (2.0f * R.errP[0] + rho * R.errL[0] + R.errC[0]);
    float e1 = u8 * (2.0f * R.errP[1] + rho * R.errL[1] + R.errC[1]);
    float e2 = u8 * (2.0f * R.errP[2] + rho * R.errL[2] + R.errC[2]);
    float en = sqrtf(e0 * e0 + e1 * e1 + e2 * e2) * 1.01f;
    float dv = sqrtf(d2) * 1.01f + en;
    return 2.0f * (3.1f * 5.9604645e-8f * dv * dv + 2.0f * dv * en + en * en) + 1e-30f;
}

// Re-test thresholds around the squared radius rr (FP64) of radius rho: FP32 d2 below
// lo is certainly inside, above hi certainly outside, in between the FP64 test decides.
// The band is the FP32 error bound, widened to 2 band_rel rho^2 when that is larger.
__device__ __forceinline__ void band_thresholds(const StructRec &R, float rho, double rr, float band_rel,
                                                float &lo, float &hi) {
    const float r2 = rho * rho;
    const float band = fmaxf(fp32_d2_error(R, rho, r2), 2.0f * band_rel * r2) * (1.0f + 1e-5f);
    lo = __double2float_rd(rr - (double)band);
    hi = __double2float_ru(rr + (double)band);
}

}  // namespace mg
