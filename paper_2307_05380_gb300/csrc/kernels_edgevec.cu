// Edge vectors and their backward pass for a fixed edge set (Sec. 1 and Sec. 4: the
// graph is rebuilt from the geometry inside a generative model's forward pass, and the
// loss is differentiated through v = (x_j - x_i + t) L and |v|).
//
//   fwd       one warp per source atom over its CSR segment: vec (compensated
//             float-float evaluation, rounded once) and len.
//   bwd_src   one warp per atom over its out-edges: g_e = dvec_e + dlen_e vec_e / len_e,
//             the sum of g over out-edges and the per-atom lattice partial
//             sum_e (x_j - x_i + t)^T g_e (FP32 lane sums, compensated warp reduction).
//   bwd_dst   one warp per atom over its in-edges in (dst, src, t) order (perm_dst):
//             grad_frac[j] = (sum_in g - sum_out g) L^T.
//   bwd_lat   one warp per structure: grad_lattice = sum of the atoms' partials in
//             atom order.
// Every sum runs in a fixed order, so the result does not depend on scheduling.
#include "mg_device.cuh"
#include "mg_launch.h"

namespace mg {

// Structure of global atom row `row` (binary search over atom_ptr), same in all lanes.
__device__ __forceinline__ int structure_of(const int32_t *__restrict__ atom_ptr, int B, int row) {
    int lo = 0, hi = B;  // atom_ptr[lo] <= row < atom_ptr[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (atom_ptr[mid] <= row) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Largest s in [0, n) with ptr[s] <= key (ptr non-decreasing, ptr[0] <= key), found by
// the whole warp in rounds of 32 probes: about log32(n) dependent loads instead of
// log2(n) for a binary search.  Warp-uniform arguments.
__device__ __forceinline__ int warp_last_leq(const int64_t *__restrict__ ptr, int n, int64_t key) {
    const int lane = lane_id();
    int lo = 0, len = n;  // the answer lies in [lo, lo + len) and ptr[lo] <= key
    while (len > 1) {
        const int step = (len + 31) / 32;
        const int idx = lo + lane * step;
        const bool le = idx < lo + len && ptr[idx] <= key;
        const int c = __popc(__ballot_sync(FULL, le));  // probes 0 .. c-1 satisfy it (c >= 1)
        const int end = lo + len;
        lo += (c - 1) * step;
        len = min(step, end - lo);
    }
    return lo;
}

// A thread per edge: every edge is independent, so the forward runs at full occupancy
// whatever the degrees.  Each warp takes one contiguous range of edges, 32 at a time,
// so the structure of an edge (from edge_ptr) is found by one binary search per warp and
// then only moves forward.
__global__ void __launch_bounds__(256) edgevec_fwd_kernel(EdgeVecArgs a) {
    pdl_trigger();  // the backward may launch now; it waits for this grid before reading
    const int64_t E = a.g.edge_ptr[a.B];
    if (E > a.g.capacity) return;
    const int lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t chunk = ((E + warps - 1) / warps + 31) & ~(int64_t)31;
    const int64_t e0 = wid * chunk, e1 = min(E, e0 + chunk);
    if (e0 >= e1) return;
    int s = warp_last_leq(a.g.edge_ptr, a.B, e0);  // last structure whose first edge is <= e0
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        while (s + 1 < a.B && a.g.edge_ptr[s + 1] <= e) ++s;
        const float *L = a.lattice + 9 * (int64_t)s;
        const int64_t i = a.g.src[e], j = a.g.dst[e];
        const int t0 = a.g.offset[3 * e], t1 = a.g.offset[3 * e + 1], t2 = a.g.offset[3 * e + 2];
        const float Ls[9] = {L[0], L[1], L[2], L[3], L[4], L[5], L[6], L[7], L[8]};
        const float3 v = edge_vec_ff(Ls, a.frac[3 * i], a.frac[3 * i + 1], a.frac[3 * i + 2], a.frac[3 * j],
                                     a.frac[3 * j + 1], a.frac[3 * j + 2], t0, t1, t2);
        if (a.out_vec) {
            a.out_vec[3 * e] = v.x;
            a.out_vec[3 * e + 1] = v.y;
            a.out_vec[3 * e + 2] = v.z;
        }
        if (a.out_len) a.out_len[e] = vec_len(v);
    }
}

cudaError_t launch_edgevec_fwd(const EdgeVecArgs &a, cudaStream_t s) {
    if (a.N <= 0) return cudaSuccess;
    // the edge count lives on the device: one thread per edge of a graph of up to the
    // capacity, capped at 16 blocks per SM (longer ranges per warp beyond)
    const int64_t want = (a.g.capacity + 255) / 256;
    const int blocks = (int)(want < 16 * num_sms() ? (want > 0 ? want : 1) : 16 * num_sms());
    edgevec_fwd_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// g_e from the upstream gradients.
__device__ __forceinline__ float3 edge_g(const EdgeVecArgs &a, int64_t e) {
    float3 g = make_float3(0.f, 0.f, 0.f);
    if (a.grad_vec) g = make_float3(a.grad_vec[3 * e], a.grad_vec[3 * e + 1], a.grad_vec[3 * e + 2]);
    if (a.grad_len) {
        const float l = a.len[e];
        if (l > 0.f) {
            const float f = __fdiv_rn(a.grad_len[e], l);
            g.x = __fmaf_rn(f, a.vec[3 * e], g.x);
            g.y = __fmaf_rn(f, a.vec[3 * e + 1], g.y);
            g.z = __fmaf_rn(f, a.vec[3 * e + 2], g.z);
        }
    }
    return g;
}

// Compensated warp sum of one FP32 value per lane: a float-float pair (hi, lo) whose
// sum carries the total to about 2^-44 relative, in a fixed butterfly order.  TwoSum is
// exact and symmetric in its operands, so every lane ends with the same pair.  (GB300
// issues FP64 at a small fraction of its FP32 rate: the reductions stay on FP32 pipes.)
__device__ __forceinline__ float2 warp_sum_ff(float v) {
    float hi = v, lo = 0.f;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const float ho = __shfl_xor_sync(FULL, hi, o);
        const float lo2 = __shfl_xor_sync(FULL, lo, o);
        float s, e;
        two_sum(hi, ho, s, e);
        hi = s;
        lo = __fadd_rn(__fadd_rn(lo, lo2), e);
    }
    return make_float2(hi, lo);
}

// (a_hi + a_lo) + (b_hi + b_lo) as a float-float pair.
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    return make_float2(s, __fadd_rn(__fadd_rn(a.y, b.y), e));
}

// Compensated warp sums of 16 FP32 values per lane at once (reduce-scatter): at each
// butterfly step a lane keeps half of its values and sends the other half to its
// partner, so lane l ends with the sum of value l >> 1 after 24 shuffles instead of 160.
// Each value meets the same partners in the same order as in warp_sum_ff, and ff_add
// is exact in its TwoSum and symmetric, so the sums are bit-identical to it.
__device__ __forceinline__ float2 warp_reduce16_ff(const float v[16]) {
    const int lane = lane_id();
    float2 a[8];
    {
        const bool up = lane & 16;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float keep = up ? v[8 + k] : v[k], send = up ? v[k] : v[8 + k];
            a[k] = ff_add(make_float2(keep, 0.f), make_float2(__shfl_xor_sync(FULL, send, 16), 0.f));
        }
    }
    float2 b[4];
    {
        const bool up = lane & 8;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 keep = up ? a[4 + k] : a[k], send = up ? a[k] : a[4 + k];
            b[k] = ff_add(keep, make_float2(__shfl_xor_sync(FULL, send.x, 8), __shfl_xor_sync(FULL, send.y, 8)));
        }
    }
    float2 c[2];
    {
        const bool up = lane & 4;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float2 keep = up ? b[2 + k] : b[k], send = up ? b[k] : b[2 + k];
            c[k] = ff_add(keep, make_float2(__shfl_xor_sync(FULL, send.x, 4), __shfl_xor_sync(FULL, send.y, 4)));
        }
    }
    const bool up = lane & 2;
    const float2 keep = up ? c[1] : c[0], send = up ? c[0] : c[1];
    float2 d = ff_add(keep, make_float2(__shfl_xor_sync(FULL, send.x, 2), __shfl_xor_sync(FULL, send.y, 2)));
    return ff_add(d, make_float2(__shfl_xor_sync(FULL, d.x, 1), __shfl_xor_sync(FULL, d.y, 1)));
}


__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }

// (sum_c g_c L[k][c]) for a float-float gradient: FP32 terms, error within a few
// roundings of the contributions' magnitude.
__device__ __forceinline__ float ff_times_LT(const float2 g[3], const float *L, int k) {
    float h = __fmul_rn(g[0].x, L[3 * k + 0]);
    h = __fmaf_rn(g[1].x, L[3 * k + 1], h);
    h = __fmaf_rn(g[2].x, L[3 * k + 2], h);
    h = __fmaf_rn(g[0].y, L[3 * k + 0], h);
    h = __fmaf_rn(g[1].y, L[3 * k + 1], h);
    return __fmaf_rn(g[2].y, L[3 * k + 2], h);
}

// The same for 32 values: lane l ends with the sum of value l (62 shuffles instead of 320).
__device__ __forceinline__ float2 warp_reduce32_ff(const float v[32]) {
    const int lane = lane_id();
    float2 a[16];
    {
        const bool up = lane & 16;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float keep = up ? v[16 + k] : v[k], send = up ? v[k] : v[16 + k];
            a[k] = ff_add(make_float2(keep, 0.f), make_float2(__shfl_xor_sync(FULL, send, 16), 0.f));
        }
    }
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {  // keep half of the o-slot window, send the other half
        const bool up = lane & o;
#pragma unroll
        for (int k = 0; k < o; ++k) {
            const float2 keep = up ? a[o + k] : a[k], send = up ? a[k] : a[o + k];
            a[k] = ff_add(keep, make_float2(__shfl_xor_sync(FULL, send.x, o), __shfl_xor_sync(FULL, send.y, o)));
        }
    }
    return a[0];
}

// A source atom's three gradient sums and nine lattice partials in one reduce-scatter:
// grad_frac[j] from the gradient sums (lanes 0-2), lpart[j] from the lattice partials.
__device__ __forceinline__ void store_atom_sums(float *__restrict__ grad_frac, float2 *__restrict__ lpart, int64_t j,
                                                const float acc[3], const float M[9], const float *L) {
    const int lane = lane_id();
    float v[16];
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q] = acc[q];
#pragma unroll
    for (int q = 0; q < 9; ++q) v[3 + q] = M[q];
#pragma unroll
    for (int q = 12; q < 16; ++q) v[q] = 0.f;
    const float2 r = warp_reduce16_ff(v);  // lanes 2q, 2q + 1: value q
    float2 tot[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) tot[q] = make_float2(__shfl_sync(FULL, r.x, 2 * q), __shfl_sync(FULL, r.y, 2 * q));
    if (lane < 3) grad_frac[3 * j + lane] = ff_times_LT(tot, L, lane);
    if (!(lane & 1) && lane >= 6 && lane < 24) lpart[9 * j + (lane / 2 - 3)] = r;
}

// Lattice partial of one edge: M[k][c] += df_k g_c with df = x_j - x_i + t within about
// one rounding of its value: x_j - x_i exactly as s1 + e1 (TwoSum); s1 + t is exact when
// the two nearly cancel (Sterbenz) and otherwise rounds once relative to df itself.
__device__ __forceinline__ void add_lattice_term(float M[9], const float xs[3], const float xd[3], const int t[3],
                                                 float3 g) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float s1, e1;
        two_sum(xd[k], -xs[k], s1, e1);
        const float df = __fadd_rn(__fadd_rn(s1, (float)t[k]), e1);
        M[3 * k + 0] = __fmaf_rn(df, g.x, M[3 * k + 0]);
        M[3 * k + 1] = __fmaf_rn(df, g.y, M[3 * k + 1]);
        M[3 * k + 2] = __fmaf_rn(df, g.z, M[3 * k + 2]);
    }
}

// Per-atom lattice partial (9 float-float pairs) from the lanes' FP32 sums.
__device__ __forceinline__ void store_lattice_partial(float2 *__restrict__ lpart, int64_t atom, const float M[9]) {
    const int lane = lane_id();
    float2 r = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const float2 t = warp_sum_ff(M[q]);
        if (lane == q) r = t;
    }
    if (lane < 9) lpart[9 * atom + lane] = r;
}

__global__ void __launch_bounds__(256) bwd_src_kernel(EdgeVecArgs a, float2 *__restrict__ gpart,
                                                      float2 *__restrict__ lpart) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = lane_id();
    if (i >= a.N) return;
    const int64_t E = a.g.edge_ptr[a.B];
    const int64_t lo = a.g.src_ptr[i], hi = (E > a.g.capacity) ? lo : a.g.src_ptr[i + 1];
    const float xi[3] = {a.frac[3 * (int64_t)i], a.frac[3 * (int64_t)i + 1], a.frac[3 * (int64_t)i + 2]};
    float gs[3] = {0.f, 0.f, 0.f};
    float M[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) M[q] = 0.f;
    for (int64_t e = lo + lane; e < hi; e += 32) {
        const float3 g = edge_g(a, e);
        const int64_t j = a.g.dst[e];
        const int t[3] = {a.g.offset[3 * e], a.g.offset[3 * e + 1], a.g.offset[3 * e + 2]};
        const float xj[3] = {a.frac[3 * j], a.frac[3 * j + 1], a.frac[3 * j + 2]};
        gs[0] += g.x;
        gs[1] += g.y;
        gs[2] += g.z;
        add_lattice_term(M, xi, xj, t, g);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float2 t = warp_sum_ff(gs[q]);
        if (lane == 0) gpart[3 * (int64_t)i + q] = t;
    }
    store_lattice_partial(lpart, i, M);
}

__global__ void __launch_bounds__(256) bwd_dst_kernel(EdgeVecArgs a, const float2 *__restrict__ gpart) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = lane_id();
    if (j >= a.N) return;
    const int64_t E = a.g.edge_ptr[a.B];
    const int64_t lo = a.g.dst_ptr[j], hi = (E > a.g.capacity) ? lo : a.g.dst_ptr[j + 1];
    float gs[3] = {0.f, 0.f, 0.f};
    for (int64_t p = lo + lane; p < hi; p += 32) {
        const int64_t e = a.g.perm_dst[p];
        const float3 g = edge_g(a, e);
        gs[0] += g.x;
        gs[1] += g.y;
        gs[2] += g.z;
    }
    float2 tot[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) tot[q] = ff_add(warp_sum_ff(gs[q]), ff_neg(gpart[3 * (int64_t)j + q]));
    if (lane < 3) {
        const int s = structure_of(a.atom_ptr, a.B, j);
        a.grad_frac[3 * (int64_t)j + lane] = ff_times_LT(tot, a.lattice + 9 * (int64_t)s, lane);
    }
}

// One warp: the lattice gradient of structure s from its atoms' partials, in atom order
// per lane and a fixed butterfly (deterministic).
__device__ __forceinline__ void lattice_reduce_warp(const EdgeVecArgs &a, const float2 *__restrict__ lpart, int s) {
    const int lane = lane_id();
    const int lo = a.atom_ptr[s], hi = a.atom_ptr[s + 1];
    float2 acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int r = lo + lane; r < hi; r += 32)
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = ff_add(acc[q], __ldcg(&lpart[9 * (int64_t)r + q]));  // L2: written by other SMs
    // the nine high and nine low parts summed across the warp in one reduce-scatter
    float v[32];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        v[q] = acc[q].x;
        v[9 + q] = acc[q].y;
    }
#pragma unroll
    for (int q = 18; q < 32; ++q) v[q] = 0.f;
    const float2 h = warp_reduce32_ff(v);  // lane q: value q
    const float2 l = make_float2(__shfl_sync(FULL, h.x, (lane + 9) & 31), __shfl_sync(FULL, h.y, (lane + 9) & 31));
    if (lane < 9) a.grad_lattice[9 * (int64_t)s + lane] = __fadd_rn(h.x, __fadd_rn(h.y, __fadd_rn(l.x, l.y)));
}

__global__ void __launch_bounds__(256) bwd_lat_kernel(EdgeVecArgs a, const float2 *__restrict__ lpart) {
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= a.B) return;
    lattice_reduce_warp(a, lpart, s);
}

// Large structures: a block of LAT_WARPS warps per structure, warp w taking every
// LAT_WARPS-th chunk of 32 atoms; the warps' float-float partials are combined in warp
// order through shared memory (a fixed order: deterministic).
constexpr int LAT_WARPS = 8;
__global__ void __launch_bounds__(LAT_WARPS * 32) bwd_lat_block_kernel(EdgeVecArgs a,
                                                                     const float2 *__restrict__ lpart) {
    __shared__ float2 part[LAT_WARPS][9];
    const int s = blockIdx.x;
    const int lane = lane_id(), wid = threadIdx.x >> 5;
    const int lo = a.atom_ptr[s], hi = a.atom_ptr[s + 1];
    float2 acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int r = lo + 32 * wid + lane; r < hi; r += 32 * LAT_WARPS)
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = ff_add(acc[q], lpart[9 * (int64_t)r + q]);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const float2 h = warp_sum_ff(acc[q].x);
        const float2 l = warp_sum_ff(acc[q].y);
        if (lane == q) part[wid][q] = ff_add(h, l);
    }
    __syncthreads();
    if (wid == 0 && lane < 9) {
        float2 t = part[0][lane];
        for (int w = 1; w < LAT_WARPS; ++w) t = ff_add(t, part[w][lane]);
        a.grad_lattice[9 * (int64_t)s + lane] = __fadd_rn(t.x, t.y);
    }
}

// First position in [lo, hi) of the sorted keys with key >= v (or > v when upper).
__device__ __forceinline__ int64_t key_bound(const int32_t *__restrict__ keys, int64_t lo, int64_t hi, int v,
                                             bool upper) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int k = keys[mid];
        if (k < v || (upper && k == v)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Backward of a symmetric (cutoff) graph in one pass over source segments: the in-edge
// of j matching out-edge p = (j, i, t) is its reverse (i, j, -t), which sits in i's
// segment at s_ij + (rhi - 1 - p) (the run of i's edges to j holds the reversed run in
// the opposite offset order; s_ij its start, [rlo, rhi) the run of p in j's segment).
// PAIRS 0: the runs come from binary searches done once per run by its first lane;
// PAIRS 1: from the build's pair table where the structure has a complete one (none for
// a structure with a source that did not fit the build's staging), else searches.
// A reverse index outside i's segment (an inconsistent graph) is reported as
// MG_ERR_INTERNAL in the graph's status word and not followed.
// The reverse edge's vector and length are those of p negated (the forward evaluates
// both edges with sign-symmetric float-float arithmetic), so only its incoming
// gradients are gathered.
// grad_frac[j] = sum_p (g_rev(p) - g_p) L^T; the lattice partial sums (x_i - x_j + t)^T g_p.
// Fixed per-lane order and a fixed warp reduction (the 12 sums of an atom in one
// reduce-scatter): deterministic, no destination order.  A warp per source atom; its
// chunks of 32 out-edges are software-pipelined (see the loop).  BLOCKS blocks of 8 warps
// per SM: 5 (48 registers, a few spilled values) for large batches, at 8192 structures
// 0.722 ms against 0.747 at 4 blocks and 64 registers and 0.857 at 6 blocks and 40
// registers; 4 for batches in one partial wave (256 structures: 20.1 against 21.9 us).
template <int PAIRS, int BLOCKS>
__global__ void __launch_bounds__(256, BLOCKS) bwd_sym_kernel(EdgeVecArgs a, float2 *__restrict__ lpart) {
    pdl_wait();  // launched early behind the forward: its vectors must be complete
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = lane_id();
    if (j >= a.N) return;
    const int64_t E = a.g.edge_ptr[a.B];
    const int64_t lo = a.g.src_ptr[j], hi = (E > a.g.capacity) ? lo : a.g.src_ptr[j + 1];
    const float xj[3] = {a.frac[3 * (int64_t)j], a.frac[3 * (int64_t)j + 1], a.frac[3 * (int64_t)j + 2]};
    int sj = -1, begin = 0;  // structure of j when its pair table is usable
    if (PAIRS) {
        const int s = a.atom_struct[j];
        if (a.pair_ok[s]) {
            sj = s;
            begin = a.atom_ptr[s];
        }
    }
    float acc[3] = {0.f, 0.f, 0.f};
    float M[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) M[q] = 0.f;
    // software-pipelined: the next chunk's targets are loaded one chunk ahead, and every
    // load that depends on the edge alone is issued before the chain through the target
    // (pair table, segment bounds) to the reverse edge's gradient
    int i_next = (lo + lane < hi) ? a.g.dst[lo + lane] : -1;
    for (int64_t p0 = lo; p0 < hi; p0 += 32) {
        const int64_t p = p0 + lane;
        const bool valid = p < hi;
        const int i = i_next;
        i_next = (p + 32 < hi) ? a.g.dst[p + 32] : -1;
        float3 g = make_float3(0.f, 0.f, 0.f);
        float f = 0.f, il = 0.f, vx = 0.f, vy = 0.f, vz = 0.f, l = 0.f;
        int t[3] = {0, 0, 0};
        float xi[3] = {0.f, 0.f, 0.f};
        int64_t ilo = 0, ihi = 0;
        if (valid) {
            if (a.grad_vec) g = make_float3(a.grad_vec[3 * p], a.grad_vec[3 * p + 1], a.grad_vec[3 * p + 2]);
            if (a.grad_len) {
                l = a.len[p];
                vx = a.vec[3 * p];
                vy = a.vec[3 * p + 1];
                vz = a.vec[3 * p + 2];
                if (l > 0.f) {
                    il = __frcp_rn(l);
                    f = __fmul_rn(a.grad_len[p], il);
                }
            }
            t[0] = a.g.offset[3 * p];
            t[1] = a.g.offset[3 * p + 1];
            t[2] = a.g.offset[3 * p + 2];
            xi[0] = a.frac[3 * (int64_t)i];
            xi[1] = a.frac[3 * (int64_t)i + 1];
            xi[2] = a.frac[3 * (int64_t)i + 2];
            ilo = a.g.src_ptr[i];
            ihi = a.g.src_ptr[i + 1];
        }
        int64_t rev = 0;
        if (PAIRS && sj >= 0) {
            if (valid) {
                const int il = i - begin, jl = j - begin;
                const int64_t rhi = lo + a.pair_hi[(int64_t)j * PAIR_MAX + il];
                rev = ilo + a.pair_lo[(int64_t)i * PAIR_MAX + jl] + (rhi - 1 - p);
            }
        } else {
            // lanes of one run (same target i, contiguous) share the run's two searches
            const unsigned grp = __match_any_sync(FULL, i);
            const int leader = __ffs(grp) - 1;
            int64_t rhi = 0, sij = 0;
            if (valid && lane == leader) {
                int64_t e = p + 1;  // end of the run: a short probe, then a binary search
                while (e < hi && e < p + 4 && a.g.dst[e] == i) ++e;
                rhi = (e < hi && e == p + 4 && a.g.dst[e] == i) ? key_bound(a.g.dst, e, hi, i, true) : e;
                sij = key_bound(a.g.dst, ilo, ihi, j, false);
            }
            rhi = __shfl_sync(FULL, rhi, leader);
            sij = __shfl_sync(FULL, sij, leader);
            rev = sij + (rhi - 1 - p);
        }
        if (!valid) continue;
        if (rev < ilo || rev >= ihi) {  // never for a graph built here
            set_error(a.g.status, MG_ERR_INTERNAL, -1);
            rev = p;
        }
        float3 gr = make_float3(0.f, 0.f, 0.f);
        if (a.grad_vec) gr = make_float3(a.grad_vec[3 * rev], a.grad_vec[3 * rev + 1], a.grad_vec[3 * rev + 2]);
        if (a.grad_len && l > 0.f) {
            const float fr = __fmul_rn(a.grad_len[rev], il);
            g.x = __fmaf_rn(f, vx, g.x);
            g.y = __fmaf_rn(f, vy, g.y);
            g.z = __fmaf_rn(f, vz, g.z);
            gr.x = __fmaf_rn(fr, -vx, gr.x);  // the reverse edge's vector is -vec[p]
            gr.y = __fmaf_rn(fr, -vy, gr.y);
            gr.z = __fmaf_rn(fr, -vz, gr.z);
        }
        acc[0] += gr.x - g.x;
        acc[1] += gr.y - g.y;
        acc[2] += gr.z - g.z;
        add_lattice_term(M, xj, xi, t, g);
    }
    {
        const int s = sj >= 0 ? sj : structure_of(a.atom_ptr, a.B, j);
        store_atom_sums(a.grad_frac, lpart, j, acc, M, a.lattice + 9 * (int64_t)s);
    }
    if (a.lat_cnt) {
        // the last warp of the structure to store its partial reduces the structure's
        // lattice gradient (the order of the sum does not depend on which warp it is)
        const int s = sj >= 0 ? sj : structure_of(a.atom_ptr, a.B, j);
        __threadfence();
        int last = 0;
        if (lane == 0) last = atomicAdd(&a.lat_cnt[s], 1) == a.atom_ptr[s + 1] - a.atom_ptr[s] - 1;
        if (__shfl_sync(FULL, last, 0)) {
            __threadfence();
            lattice_reduce_warp(a, lpart, s);
            if (lane == 0) a.lat_cnt[s] = 0;  // ready for the next backward
            // empty structures after s (and before the first atom's) get a zero gradient
            for (int q = s + 1; q < a.B && a.atom_ptr[q] == a.atom_ptr[q + 1]; ++q)
                if (lane < 9) a.grad_lattice[9 * (int64_t)q + lane] = 0.f;
            if (a.atom_ptr[s] == 0)
                for (int q = s - 1; q >= 0; --q)
                    if (lane < 9) a.grad_lattice[9 * (int64_t)q + lane] = 0.f;
        }
    }
}

cudaError_t launch_bwd_sym(const EdgeVecArgs &a, const Work &w, cudaStream_t s) {
    if (a.N <= 0) return cudaSuccess;
    const int blocks = (a.N + 7) / 8;
    float2 *lpart = w.lpart;
    if (a.N < 8192) {  // one partial wave: the 64-register form
        if (!a.pair_lo) return launch_pdl(bwd_sym_kernel<0, 4>, dim3(blocks), dim3(256), s, a, lpart);
        return launch_pdl(bwd_sym_kernel<1, 4>, dim3(blocks), dim3(256), s, a, lpart);
    }
    if (!a.pair_lo) return launch_pdl(bwd_sym_kernel<0, 5>, dim3(blocks), dim3(256), s, a, lpart);
    return launch_pdl(bwd_sym_kernel<1, 5>, dim3(blocks), dim3(256), s, a, lpart);
}

cudaError_t launch_bwd_src(const EdgeVecArgs &a, const Work &w, cudaStream_t s) {
    if (a.N > 0) bwd_src_kernel<<<(a.N + 7) / 8, 256, 0, s>>>(a, w.gpart, w.lpart);
    return cudaGetLastError();
}

cudaError_t launch_bwd_dst(const EdgeVecArgs &a, const Work &w, cudaStream_t s) {
    if (a.N > 0) bwd_dst_kernel<<<(a.N + 7) / 8, 256, 0, s>>>(a, w.gpart);
    return cudaGetLastError();
}

cudaError_t launch_bwd_lat(const EdgeVecArgs &a, const Work &w, cudaStream_t s) {
    if (a.B <= 0) return cudaSuccess;
    if (a.max_atoms > 0 && a.max_atoms <= 1024)
        bwd_lat_kernel<<<(a.B + 7) / 8, 256, 0, s>>>(a, w.lpart);  // a warp per structure
    else
        bwd_lat_block_kernel<<<a.B, LAT_WARPS * 32, 0, s>>>(a, w.lpart);
    return cudaGetLastError();
}

}  // namespace mg
