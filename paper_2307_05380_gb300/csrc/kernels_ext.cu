// Operations on built graphs from the paper's tool list after Alg. 2 (Sec. 2.2):
//   triplets     Gamma_2 of Def. 3, the ordered pairs (e, e') of edges with a common
//                source, written as edge ids: per source a deg x deg block (without the
//                diagonal when (e, e) is excluded), offsets from a 64-bit scan of the
//                per-atom block sizes.  Pure index expansion: bound by HBM writes.
//   symmetrize   the symmetric closure in ∪ {(j, i, -t) : (i, j, t) in in}, each distinct
//                edge once, canonical order.  For atom j the out-list A (sorted by
//                (dst, t)) and the reversed in-list B (in-edges through perm_dst, sorted
//                by (src, t), hence by (src, -t) once every run of equal src is read
//                backwards) are merged; every position comes from binary searches, so
//                there is no degree limit and no shared-memory staging.
#include "mg_device.cuh"
#include "mg_launch.h"

namespace mg {

// ============================================================================ triplets

__device__ __forceinline__ long long trip_count(const int64_t *__restrict__ src_ptr, int i, int excl) {
    const long long d = src_ptr[i + 1] - src_ptr[i];
    return d * (d - excl > 0 ? d - excl : 0);
}

__device__ __forceinline__ long long block_sum_ll(long long v, long long *sm) {
    const int lane = lane_id(), wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sm[q];
    __syncthreads();
    return t;
}

constexpr int TRIP_TILE = 4096;  // atoms per scan tile (256 threads x 16)

// Per tile: the sum of the block sizes; block 0 also resets the status word.
__global__ void __launch_bounds__(256) trip_reduce_kernel(const int64_t *__restrict__ src_ptr, int n, int excl,
                                                          long long *__restrict__ tile_sum,
                                                          mg_device_status_t *status) {
    __shared__ long long sm[8];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Status *st = reinterpret_cast<Status *>(status);
        st->code = 0;
        st->first_bad_structure = 0x7fffffff;
        st->num_edges = 0;
        st->required_capacity = 0;
        st->rechecked = 0;
        st->candidates = 0;
    }
    const int64_t base = (int64_t)blockIdx.x * TRIP_TILE;
    long long v = 0;
    for (int q = threadIdx.x; q < TRIP_TILE; q += 256)
        if (base + q < n) v += trip_count(src_ptr, (int)(base + q), excl);
    const long long tot = block_sum_ll(v, sm);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// Exclusive prefix of the tile sums (one block), total in tile_sum[ntiles].
__global__ void __launch_bounds__(32) trip_top_kernel(long long *__restrict__ tile_sum, int ntiles) {
    long long carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += 32) {
        const int q = b0 + lane_id();
        const long long v = q < ntiles ? tile_sum[q] : 0;
        long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(FULL, x, o);
            if (lane_id() >= o) x += y;
        }
        if (q < ntiles) tile_sum[q] = carry + x - v;
        carry += __shfl_sync(FULL, x, 31);
    }
    if (lane_id() == 0) tile_sum[ntiles] = carry;
}

// atom_off[i] = triplets of the sources before i; atom_off[n] = total, also reported in
// the status word (MG_ERR_CAPACITY when it exceeds the capacity).
__global__ void __launch_bounds__(256) trip_apply_kernel(const int64_t *__restrict__ src_ptr, int n, int excl,
                                                         const long long *__restrict__ tile_off, int ntiles,
                                                         int64_t *__restrict__ atom_off, int64_t capacity,
                                                         int64_t *__restrict__ trip_ptr,
                                                         mg_device_status_t *status) {
    __shared__ long long sm[64];
    const int64_t base = (int64_t)blockIdx.x * TRIP_TILE + 16 * threadIdx.x;
    long long vals[16];
    long long mysum = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        vals[q] = (base + q < n) ? trip_count(src_ptr, (int)(base + q), excl) : 0;
        mysum += vals[q];
    }
    // block exclusive scan of the thread sums
    const int lane = lane_id(), wid = threadIdx.x >> 5;
    long long x = mysum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[wid] = x;
    __syncthreads();
    long long wpre = 0;
    for (int q = 0; q < wid; ++q) wpre += sm[q];
    long long run = tile_off[blockIdx.x] + wpre + x - mysum;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        if (base + q < n) atom_off[base + q] = run;
        run += vals[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const long long tot = tile_off[ntiles];
        atom_off[n] = tot;
        if (trip_ptr) trip_ptr[src_ptr[n]] = tot;
        Status *st = reinterpret_cast<Status *>(status);
        st->num_edges = (unsigned long long)tot;
        st->required_capacity = (unsigned long long)tot;
        if (tot > capacity) set_error(status, MG_ERR_CAPACITY, -1);
    }
}

// A warp per source atom writes its block row by row: row r (first edge lo + r) holds
// the second edges lo .. hi-1 (without lo + r when excl).  Lanes walk the flattened
// block with a running (row, column) instead of a division per element.
__global__ void __launch_bounds__(256) trip_write_kernel(const int64_t *__restrict__ src_ptr, int n, int excl,
                                                         const int64_t *__restrict__ atom_off, int64_t capacity,
                                                         int32_t *__restrict__ edge_a, int32_t *__restrict__ edge_b,
                                                         int64_t *__restrict__ trip_ptr) {
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = lane_id();
    if (i >= n) return;
    if (atom_off[n] > capacity) return;  // reported by the scan
    const int64_t lo = src_ptr[i], hi = src_ptr[i + 1];
    const int deg = (int)(hi - lo);
    const int w = deg - excl;
    const int64_t base = atom_off[i];
    if (trip_ptr)
        for (int r = lane; r < deg; r += 32) trip_ptr[lo + r] = base + (int64_t)r * (w > 0 ? w : 0);
    if (w <= 0) return;
    const int64_t total = (int64_t)deg * w;
    int r = lane / w, c = lane - (lane / w) * w;
    for (int64_t q = lane; q < total; q += 32) {
        const int e2 = (int)lo + c + ((excl && c >= r) ? 1 : 0);
        if (edge_a) edge_a[base + q] = (int32_t)(lo + r);
        edge_b[base + q] = e2;
        c += 32;
        while (c >= w) {
            c -= w;
            ++r;
        }
    }
}

cudaError_t launch_triplets(const TripArgs &a, const Work &w, cudaStream_t s, int *launches) {
    const int n = a.N;
    const int ntiles = (n + TRIP_TILE - 1) / TRIP_TILE;
    const int nt = ntiles > 0 ? ntiles : 1;
    trip_reduce_kernel<<<nt, 256, 0, s>>>(a.src_ptr, n, a.excl, w.tile_sum, a.status);
    trip_top_kernel<<<1, 32, 0, s>>>(w.tile_sum, ntiles);
    trip_apply_kernel<<<nt, 256, 0, s>>>(a.src_ptr, n, a.excl, w.tile_sum, ntiles, w.src_ptr, a.capacity, a.trip_ptr,
                                         a.status);
    int nl = 3;
    if (n > 0) {
        trip_write_kernel<<<(n + 7) / 8, 256, 0, s>>>(a.src_ptr, n, a.excl, w.src_ptr, a.capacity, a.edge_a, a.edge_b,
                                                      a.trip_ptr);
        ++nl;
    }
    if (launches) *launches = nl;
    return cudaGetLastError();
}

// ============================================================================ symmetrize

// Lexicographic order of (node, t0, t1, t2).
struct EKey {
    int n, t0, t1, t2;
};
__device__ __forceinline__ bool ekey_less(const EKey &a, const EKey &b) {
    if (a.n != b.n) return a.n < b.n;
    if (a.t0 != b.t0) return a.t0 < b.t0;
    if (a.t1 != b.t1) return a.t1 < b.t1;
    return a.t2 < b.t2;
}
__device__ __forceinline__ bool ekey_eq(const EKey &a, const EKey &b) {
    return a.n == b.n && a.t0 == b.t0 && a.t1 == b.t1 && a.t2 == b.t2;
}

__device__ __forceinline__ EKey out_key(const mg_graph_t &g, int64_t e) {
    return EKey{g.dst[e], g.offset[3 * e], g.offset[3 * e + 1], g.offset[3 * e + 2]};
}
// In-list element q (perm position) read as its reverse: (src, -t).
__device__ __forceinline__ EKey rev_key(const mg_graph_t &g, int64_t q) {
    const int64_t e = g.perm_dst[q];
    return EKey{g.src[e], -g.offset[3 * e], -g.offset[3 * e + 1], -g.offset[3 * e + 2]};
}

// First out-list position in [lo, hi) whose key is not below k.
__device__ __forceinline__ int64_t lower_out(const mg_graph_t &g, int64_t lo, int64_t hi, const EKey &k) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (ekey_less(out_key(g, mid), k)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Run of in-edges with source `src` in perm positions [lo, hi) (sorted by source).
__device__ __forceinline__ int64_t src_bound(const mg_graph_t &g, int64_t lo, int64_t hi, int src, bool upper) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int v = g.src[g.perm_dst[mid]];
        if (v < src || (upper && v == src)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Inside a run (sorted by t ascending): the first position whose t is above x (upper)
// or not below x (lower).
__device__ __forceinline__ int64_t t_bound(const mg_graph_t &g, int64_t lo, int64_t hi, int x0, int x1, int x2,
                                           bool upper) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int64_t e = g.perm_dst[mid];
        const EKey v{0, g.offset[3 * e], g.offset[3 * e + 1], g.offset[3 * e + 2]};
        const EKey x{0, x0, x1, x2};
        if (ekey_less(v, x) || (upper && ekey_eq(v, x))) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// For out-edge a = (j -> i, t): rank of a among the reversed in-list of j (how many
// reversed in-edges sort below it) and whether (i -> j, -t) is an in-edge (a twin).
__device__ __forceinline__ void rank_in_reversed(const mg_graph_t &g, int64_t b0, int64_t b1, const EKey &a,
                                                 int64_t &rank, bool &twin) {
    const int64_t r0 = src_bound(g, b0, b1, a.n, false);
    const int64_t r1 = src_bound(g, r0, b1, a.n, true);
    // reversed keys (i, -t'') below (i, t): t'' > -t
    const int64_t ub = t_bound(g, r0, r1, -a.t0, -a.t1, -a.t2, true);
    const int64_t lb = t_bound(g, r0, ub, -a.t0, -a.t1, -a.t2, false);
    rank = (r0 - b0) + (r1 - ub);
    twin = lb < ub;
}

// Pass 1: out-degree of every atom in the closure, |A| + |B| - twins.
__global__ void __launch_bounds__(256) sym_count_kernel(SymArgs a, int32_t *__restrict__ cnt) {
    const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = lane_id();
    if (j >= a.N) return;
    const mg_graph_t &g = a.in;
    const int64_t a0 = g.src_ptr[j], a1 = g.src_ptr[j + 1];
    const int64_t b0 = g.dst_ptr[j], b1 = g.dst_ptr[j + 1];
    int twins = 0;
    for (int64_t p = a0 + lane; p < a1; p += 32) {
        int64_t rank;
        bool twin;
        rank_in_reversed(g, b0, b1, out_key(g, p), rank, twin);
        twins += twin ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) twins += __shfl_xor_sync(FULL, twins, o);
    if (lane == 0) cnt[j] = (int32_t)((a1 - a0) + (b1 - b0) - twins);
}

// Out pointers per structure, edge count and capacity check.
__global__ void sym_finalize_kernel(SymArgs a) {
    const int64_t tot = a.out.src_ptr[a.N];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= a.B; s += gridDim.x * blockDim.x)
        a.out.edge_ptr[s] = s == a.B ? tot : a.out.src_ptr[a.atom_ptr[s]];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Status *st = reinterpret_cast<Status *>(a.out.status);
        st->code = 0;
        st->first_bad_structure = 0x7fffffff;
        st->num_edges = (unsigned long long)tot;
        st->required_capacity = (unsigned long long)tot;
        st->rechecked = 0;
        st->candidates = 0;
        if (tot > a.out.capacity) set_error(a.out.status, MG_ERR_CAPACITY, -1);
    }
}

__device__ __forceinline__ int structure_of_atom(const int32_t *__restrict__ atom_ptr, int B, int j) {
    int lo = 0, hi = B;  // last s with atom_ptr[s] <= j
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (atom_ptr[mid] <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void write_edge(const SymArgs &a, const float *L, int j, int64_t e, int i, int t0, int t1,
                                           int t2) {
    const mg_graph_t &o = a.out;
    o.src[e] = j;
    o.dst[e] = i;
    o.offset[3 * e] = t0;
    o.offset[3 * e + 1] = t1;
    o.offset[3 * e + 2] = t2;
    if (o.vec || o.len) {
        const float3 v = edge_vec_ff(L, a.frac[3 * (int64_t)j], a.frac[3 * (int64_t)j + 1], a.frac[3 * (int64_t)j + 2],
                                     a.frac[3 * (int64_t)i], a.frac[3 * (int64_t)i + 1], a.frac[3 * (int64_t)i + 2], t0,
                                     t1, t2);
        if (o.vec) {
            o.vec[3 * e] = v.x;
            o.vec[3 * e + 1] = v.y;
            o.vec[3 * e + 2] = v.z;
        }
        if (o.len) o.len[e] = vec_len(v);
    }
}

// Pass 2: the merged, de-duplicated list of atom j at out.src_ptr[j].  dup[a0 + p] holds
// the number of twins among A[0 .. p) (the out-edges whose reverse is also an in-edge),
// which turns ranks in A and in the reversed in-list into positions in the union.
__global__ void __launch_bounds__(256) sym_write_kernel(SymArgs a, int32_t *__restrict__ dup) {
    const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = lane_id();
    if (j >= a.N) return;
    if (a.out.src_ptr[a.N] > a.out.capacity) return;  // reported by the finalize kernel
    const mg_graph_t &g = a.in;
    const int64_t a0 = g.src_ptr[j], a1 = g.src_ptr[j + 1];
    const int64_t b0 = g.dst_ptr[j], b1 = g.dst_ptr[j + 1];
    const int64_t base = a.out.src_ptr[j];
    const int s = structure_of_atom(a.atom_ptr, a.B, j);
    float L[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) L[q] = a.lattice[9 * (int64_t)s + q];
    const unsigned lt = (1u << lane) - 1u;
    // out-list: twins, their prefix counts, positions
    int carry = 0;
    for (int64_t p0 = a0; p0 < a1; p0 += 32) {
        const int64_t p = p0 + lane;
        const bool v = p < a1;
        int64_t rank = 0;
        bool twin = false;
        EKey k{0, 0, 0, 0};
        if (v) {
            k = out_key(g, p);
            rank_in_reversed(g, b0, b1, k, rank, twin);
        }
        const unsigned tb = __ballot_sync(FULL, v && twin);
        const int before = carry + __popc(tb & lt);
        if (v) {
            dup[p] = before;
            write_edge(a, L, j, base + (p - a0) + rank - before, k.n, k.t0, k.t1, k.t2);
        }
        carry += __popc(tb);
    }
    __syncwarp();  // dup[] of this atom is complete and visible to the warp
    const int twins_total = carry;
    // reversed in-list: elements without a twin in A
    for (int64_t q0 = b0; q0 < b1; q0 += 32) {
        const int64_t q = q0 + lane;
        if (q >= b1) continue;
        const EKey k = rev_key(g, q);
        const int64_t lb = lower_out(g, a0, a1, k);
        if (lb < a1 && ekey_eq(out_key(g, lb), k)) continue;  // already in A
        const int64_t r0 = src_bound(g, b0, b1, k.n, false);
        const int64_t r1 = src_bound(g, r0, b1, k.n, true);
        const int64_t rank_b = (r0 - b0) + (r1 - 1 - q);  // reversed keys below this one
        const int dup_below = lb < a1 ? dup[lb] : twins_total;
        write_edge(a, L, j, base + (lb - a0) + rank_b - dup_below, k.n, k.t0, k.t1, k.t2);
    }
}

cudaError_t launch_symmetrize(const SymArgs &a, const Work &w, cudaStream_t s, int *launches) {
    int nl = 0;
    const int blocks = (a.N + 7) / 8;
    if (a.N > 0) {
        sym_count_kernel<<<blocks, 256, 0, s>>>(a, w.cnt);
        ++nl;
    }
    ScanArgs sa{a.N, w.cnt, a.out.src_ptr};
    cudaError_t e = launch_scan(sa, w, s);
    if (e) return e;
    nl += 3;
    sym_finalize_kernel<<<max(1, min(64, (a.B + 256) / 256)), 256, 0, s>>>(a);
    ++nl;
    if (a.N > 0) {
        sym_write_kernel<<<blocks, 256, 0, s>>>(a, w.sort_tmp);
        ++nl;
    }
    if (launches) *launches = nl;
    return cudaGetLastError();
}

}  // namespace mg
