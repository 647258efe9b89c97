// Batched cutoff-graph construction (Def. 3, Sec. 2.1) on sm_103a:
//   prep      a warp (or block) per structure: lattice cofactors in FP64, interplanar
//             spacings, FP32 Cartesian positions, FP32 error bound and re-test band,
//             cell-list shape; also resets the status word;
//   bins      the fractional cell list of large structures (count, scan, scatter);
//   build     one pass per source atom (one warp each): FP32 scan of the periodic
//             images inside the interplanar box (Sec. 2.2's evaluated area) with an FP64
//             re-test in the band, keys staged in shared memory, offsets by a bounded
//             decoupled look-back, edges (src, dst, t, vec, len) written in canonical
//             order;
//   count/scan/finalize/write  the two-pass form used by the per-structure build;
//   dst order edge ids ordered by (dst, src, t): from reverse runs for symmetric
//             (cutoff) graphs, by a counting sort plus segment sorts otherwise.
#include <cstdio>

#include "mg_build.cuh"
#include "mg_device.cuh"
#include "mg_enum.cuh"
#include "mg_launch.h"

namespace mg {

// ============================================================================ prep

// One group of GROUP threads per structure: a warp (small structures, four per block) or
// a whole block (large structures).  The group converts its atoms to FP32 Cartesian
// positions and finds max |x|; its first thread then derives the structure record.
// FP64 is used for the lattice cofactors and determinant (cancellation-prone) and the
// squared cutoff; the derived bounds are FP32, rounded up or inflated by 1e-5 so that
// they stay bounds.
template <int GROUP>
__global__ void __launch_bounds__(GROUP == 32 ? 128 : GROUP) prep_kernel(PrepArgs a, StructRec *__restrict__ recs,
                                                                        float4 *__restrict__ pos,
                                                                        int32_t *__restrict__ atom_struct,
                                                                        unsigned long long *__restrict__ tile_flags,
                                                                        unsigned int *__restrict__ queue) {
    __shared__ float red[GROUP == 32 ? 1 : 6 * (GROUP / 32)];
    pdl_trigger();  // a build kernel launched behind prep waits for it before reading
    if (a.zero_tiles) {  // the one-pass build's look-back words and tile ticket start at zero
        const int ntiles = (a.N + BUILD_TILE - 1) / BUILD_TILE + 1;
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x)
            tile_flags[t] = 0;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            queue[3] = 0;
            queue[4] = 0;  // queue[4..5]: 64-bit slot counter of the staged build
            queue[5] = 0;
            queue[6] = 0;  // queue[6], queue[7]: work-list cursors of the pair-lane build's passes
            queue[7] = 0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // queue[10], queue[11]: the KNN fallback list and its cursor
        queue[10] = 0;
        queue[11] = 0;
        queue[12] = 0;  // queue[12], queue[13]: the staged builds' spill list and its cursor
        queue[13] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (a.init_status || (a.knn_k > 0 && a.edge_ptr))) {
        // nothing else writes the status word before the kernels that follow prep
        Status *st = reinterpret_cast<Status *>(a.status);
        if (a.init_status) {
            st->code = 0;
            st->first_bad_structure = 0x7fffffff;
            st->rechecked = 0;
            st->candidates = 0;
            st->num_edges = 0;
            st->required_capacity = 0;
        }
        if (a.knn_k > 0 && a.edge_ptr) {  // exactly k edges per atom
            st->num_edges = (unsigned long long)a.N * a.knn_k;
            st->required_capacity = (unsigned long long)a.N * a.knn_k;
        }
    }
    const int s = GROUP == 32 ? (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) : (int)blockIdx.x;
    const int t = GROUP == 32 ? lane_id() : (int)threadIdx.x;
    if (s >= a.B) return;
    const int begin = a.atom_ptr[s], end = a.atom_ptr[s + 1];
    if (a.knn_k > 0 && a.edge_ptr) {  // KNN pointers: k edges per atom
        for (int r = begin + t; r < end; r += GROUP) a.src_ptr[r] = (int64_t)r * a.knn_k;
        if (t == 0) {
            a.edge_ptr[s] = (int64_t)begin * a.knn_k;
            if (s == a.B - 1) {
                a.edge_ptr[a.B] = (int64_t)a.N * a.knn_k;
                a.src_ptr[a.N] = (int64_t)a.N * a.knn_k;
            }
        }
    }
    float Lf[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Lf[q] = a.lattice[9 * (int64_t)s + q];
    float xm0 = 0.f, xm1 = 0.f, xm2 = 0.f, nonfinite = 0.f, cmax = 0.f, cbad = 0.f;
    for (int r = begin + t; r < end; r += GROUP) {
        const float x0 = a.frac[3 * (int64_t)r], x1 = a.frac[3 * (int64_t)r + 1], x2 = a.frac[3 * (int64_t)r + 2];
        if (!isfinite(x0) || !isfinite(x1) || !isfinite(x2)) nonfinite = 1.f;
        const float3 p = cart(Lf, x0, x1, x2);
        pos[r] = make_float4(p.x, p.y, p.z, 0.f);
        atom_struct[r] = s;
        xm0 = fmaxf(xm0, fabsf(x0));
        xm1 = fmaxf(xm1, fabsf(x1));
        xm2 = fmaxf(xm2, fabsf(x2));
        if (a.cutoff_atom) {  // per-atom radii: the structure reaches as far as the largest
            const float ca = a.cutoff_atom[r];
            if (!(ca > 0.f) || !isfinite(ca)) cbad = 1.f;
            else cmax = fmaxf(cmax, ca);
        }
    }
    xm0 = warp_max(xm0);
    xm1 = warp_max(xm1);
    xm2 = warp_max(xm2);
    nonfinite = warp_max(nonfinite);
    cmax = warp_max(cmax);
    cbad = warp_max(cbad);
    if (GROUP > 32) {
        const int wid = threadIdx.x >> 5;
        if (lane_id() == 0) {
            red[6 * wid + 0] = xm0;
            red[6 * wid + 1] = xm1;
            red[6 * wid + 2] = xm2;
            red[6 * wid + 3] = nonfinite;
            red[6 * wid + 4] = cmax;
            red[6 * wid + 5] = cbad;
        }
        __syncthreads();
        if (t == 0)
            for (int q = 1; q < GROUP / 32; ++q) {
                xm0 = fmaxf(xm0, red[6 * q + 0]);
                xm1 = fmaxf(xm1, red[6 * q + 1]);
                xm2 = fmaxf(xm2, red[6 * q + 2]);
                nonfinite = fmaxf(nonfinite, red[6 * q + 3]);
                cmax = fmaxf(cmax, red[6 * q + 4]);
                cbad = fmaxf(cbad, red[6 * q + 5]);
            }
    }
    if (t != 0) return;

    StructRec R;
    double L[9];
    int bad = 0;
    for (int q = 0; q < 9; ++q) {
        R.L[q] = Lf[q];
        L[q] = (double)Lf[q];
        if (!isfinite(Lf[q])) bad = MG_ERR_NONFINITE_INPUT;
    }
    if (nonfinite != 0.f) bad = MG_ERR_NONFINITE_INPUT;
    // cofactors (row-vector convention: f = v L^-1, column k of L^-1 = cofactor row k / det)
    const double c00 = L[4] * L[8] - L[5] * L[7], c01 = L[5] * L[6] - L[3] * L[8], c02 = L[3] * L[7] - L[4] * L[6];
    const double c10 = L[2] * L[7] - L[1] * L[8], c11 = L[0] * L[8] - L[2] * L[6], c12 = L[1] * L[6] - L[0] * L[7];
    const double c20 = L[1] * L[5] - L[2] * L[4], c21 = L[2] * L[3] - L[0] * L[5], c22 = L[0] * L[4] - L[1] * L[3];
    const double det = L[0] * c00 + L[1] * c01 + L[2] * c02;
    const float la = sqrtf(Lf[0] * Lf[0] + Lf[1] * Lf[1] + Lf[2] * Lf[2]);
    const float lb = sqrtf(Lf[3] * Lf[3] + Lf[4] * Lf[4] + Lf[5] * Lf[5]);
    const float lc = sqrtf(Lf[6] * Lf[6] + Lf[7] * Lf[7] + Lf[8] * Lf[8]);
    const float adet = fabsf((float)det);
    if (!bad && (!(adet > 1e-9f * la * lb * lc) || !isfinite(adet))) bad = MG_ERR_SINGULAR_LATTICE;
    const double cn2[3] = {c00 * c00 + c01 * c01 + c02 * c02, c10 * c10 + c11 * c11 + c12 * c12,
                           c20 * c20 + c21 * c21 + c22 * c22};
    const float xm[3] = {xm0, xm1, xm2};
    float invd[3];
    for (int k = 0; k < 3; ++k) {
        // ||L^-1[:, k]|| = 1 / d_k, inflated to stay an upper bound after FP32 rounding
        invd[k] = bad ? 1.0f : sqrtf((float)cn2[k]) / adet * (1.0f + 1e-5f);
        R.invd[k] = invd[k];
    }
    float c;
    const int n = end - begin;
    if (a.knn_k > 0) {
        c = 1.1f * cbrtf(3.0f * (a.knn_k + 1) * adet / (4.0f * 3.14159265f * (n > 0 ? n : 1)));
        if (!(c > 0.f) || !isfinite(c)) c = 1.0f;
    } else if (a.cutoff_atom) {
        c = n > 0 ? cmax : 1.0f;
        if (!bad && cbad != 0.f) bad = MG_ERR_INVALID_ARGUMENT;
    } else {
        c = a.cutoff_ps ? a.cutoff_ps[s] : a.cutoff;
        if (!bad && (!(c > 0.f) || !isfinite(c))) bad = MG_ERR_INVALID_ARGUMENT;
    }
    R.cut = c;
    for (int cc = 0; cc < 3; ++cc) {
        float P = 0.f, Lt = 0.f, C = 0.f;
        for (int k = 0; k < 3; ++k) {
            const float al = fabsf(Lf[3 * k + cc]);
            P += xm[k] * al;
            Lt += invd[k] * al;
            C += (2.0f * xm[k] + 1.0f) * al;
        }
        R.errP[cc] = P * (1.0f + 1e-5f);
        R.errL[cc] = Lt * (1.0f + 1e-5f);
        R.errC[cc] = C * (1.0f + 1e-5f);
    }
    R.L2norm2 = Lf[6] * Lf[6] + Lf[7] * Lf[7] + Lf[8] * Lf[8];
    R.L2norm = sqrtf(R.L2norm2);
    R.rr = (double)c * (double)c;
    band_thresholds(R, c, R.rr, a.band_rel, R.thr_lo, R.thr_hi);  // re-test band around the cutoff
    R.atom_begin = begin;
    R.n_atoms = n;
    R.bad = bad;
    R.ax = 2;
    // Cell list for large structures: bins at least half the radius wide along each
    // plane normal (n_k = floor(2 d_k / c)), at most n_atoms bins in total; used when the
    // bins a source visits cover less than half the cell.
    R.nb[0] = R.nb[1] = R.nb[2] = 0;
    R.bin_base = begin + s + a.struct_offset;
    if (!bad && n >= CELL_MIN_ATOMS) {
        int nk[3];
        float prod = 1.f;
        for (int k = 0; k < 3; ++k) {
            nk[k] = (int)fminf(fmaxf(floorf(2.0f / (invd[k] * c)), 1.0f), 1024.0f);
            prod *= nk[k];
        }
        if (prod > n) {
            const float f = cbrtf((float)n / prod);
            for (int k = 0; k < 3; ++k) nk[k] = max(1, (int)floorf(nk[k] * f));
        }
        while ((int64_t)nk[0] * nk[1] * nk[2] > n) {  // rounding left too many: trim the largest
            int kmax = 0;
            for (int k = 1; k < 3; ++k)
                if (nk[k] > nk[kmax]) kmax = k;
            --nk[kmax];
        }
        float visited = 1.f;
        for (int k = 0; k < 3; ++k) visited *= fminf(1.0f, (2.0f * c * invd[k] * nk[k] + 2.0f) / nk[k]);
        if (visited < 0.5f)
            for (int k = 0; k < 3; ++k) R.nb[k] = nk[k];
    }
    // Axis order of the staged cutoff scan: candidates along the axis of largest reach
    // (the shortest interplanar spacing), where each row holds the most of them.  Moved
    // only when that reach's box extent is at least 1.3 times the extent along L_2: the
    // scan then puts the source's keys back into canonical order, which pays for itself
    // only when the rows it saves are many (elongated or skewed cells).
    if (!bad && R.nb[0] == 0) {
        int ax = 2;
        if (invd[0] > invd[ax]) ax = 0;
        if (invd[1] > invd[ax]) ax = 1;
        if (ax != 2 && 2.0f * c * invd[ax] + 1.0f >= 1.3f * (2.0f * c * invd[2] + 1.0f)) R.ax = ax;
    }
    // Pair-lane scan: one lane evaluates a (source, target) pair's whole offset box, the
    // integers t_k with |x_j,k - x_i,k + t_k| <= reach_k = R_k + m_k.  The margin m_k =
    // 1e-5 (1 + 2 max|x_k| + R_k) is far above the FP32 rounding of x_j - x_i (at most
    // 2 max|x_k|) and of the bounds, so the box holds every offset within R_k.  An
    // interval of length 2 reach_k holds at most floor(2 reach_k) + 1 integers (counted
    // here with twice the margin, so that the count survives rounding); offsets stay
    // within reach_k + 2 max|x_k| + 1.
    int box[3] = {0, 0, 0};
    R.pl = 0;
    for (int k = 0; k < 3; ++k) {
        const float Rk = c * invd[k];
        // KNN graphs: the margin's constant part only (the search radius varies per source)
        R.reach[k] = a.knn_k > 0 ? 1e-5f * (1.0f + 2.0f * xm[k]) : Rk + 1e-5f * (1.0f + 2.0f * xm[k] + Rk);
    }
    if (!bad && R.nb[0] == 0 && n > 0 && n <= PL_MAX_ATOMS && a.knn_k == 0 && !a.cutoff_atom) {
        bool fits = true;
        int prod = 1;
        for (int k = 0; k < 3; ++k) {
            const float Rk = c * invd[k];
            const float ext = floorf(2.0f * Rk + 4e-5f * (1.0f + 2.0f * xm[k] + Rk)) + 1.0f;
            if (!(ext <= (float)PL_BOX_MAX) || !(Rk + 2.0f * xm[k] + 2.0f <= (float)OFFSET_KEY_LIM)) fits = false;
            box[k] = fits ? (int)ext : 0;
            prod *= fits ? (int)ext : 1;
        }
        // a row's cells fit one word; the extents, B2 | B1 << 8 | B0 << 16, are the mask's strides
        R.pl = (fits && prod <= PL_BOX_MAX && box[2] <= 32) ? box[2] | (box[1] << 8) | (box[0] << 16) : 0;
    }
    if (a.plan_items) {
        // work items and their cost class: a pair-lane structure is split into groups of
        // 32 / G sources (G = lanes per source, the smallest power of two >= n, at most 32),
        // each group's cost its target chunks times the box cells; any other structure is
        // one item per source (the warp enumeration), unusable structures included (their
        // items report the error and count zero edges)
        int items;
        float cost;
        if (R.pl) {
            int G = 1;
            while (G < n && G < 32) G <<= 1;
            const int spw = 32 / G;
            items = (n + spw - 1) / spw;
            cost = (float)((n + G - 1) / G) * (float)(box[0] * box[1] * box[2]);
        } else {
            items = n;
            cost = bad ? 1.0f
                       : 4.0f * (float)n * (2.0f * c * invd[0] + 1.0f) * (2.0f * c * invd[1] + 1.0f) *
                             (2.0f * c * invd[2] + 1.0f);
        }
        const unsigned ic = (unsigned)fminf(fmaxf(cost, 1.0f), 2.0e9f);
        a.plan_items[s] = items;
        a.plan_class[s] = (R.pl ? 0 : 32) + 31 - __clz(ic);  // classes 32..63: the warp enumeration
    }
    recs[s] = R;  // a bad structure is reported by the kernel that scans its first atom
    if (a.pair_ok) a.pair_ok[s] = n <= PAIR_MAX ? 1 : 0;
    if (a.lat_cnt) a.lat_cnt[s] = 0;
}

cudaError_t launch_prep(const PrepArgs &a, const Work &w, cudaStream_t s) {
    if (a.B <= 0) return cudaSuccess;
    if (a.max_atoms > 0 && a.max_atoms <= 2048) {  // a warp per structure (a few loads per lane)
        const int blocks = (a.B * 32 + 127) / 128;
        prep_kernel<32><<<blocks, 128, 0, s>>>(a, w.recs, w.pos, w.atom_struct, w.tile_flags, w.queue);
    } else {  // a block per structure
        prep_kernel<512><<<a.B, 512, 0, s>>>(a, w.recs, w.pos, w.atom_struct, w.tile_flags, w.queue);
    }
    return cudaGetLastError();
}

// ============================================================================ scan

__device__ __forceinline__ long long block_excl_scan_ll(long long v, long long *sm, long long &total) {
    // 256 threads: warp scans, then a scan of the 8 warp totals
    const int lane = lane_id(), wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long t = (lane < (int)(blockDim.x >> 5)) ? sm[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(FULL, t, o);
            if (lane >= o) t += y;
        }
        if (lane < 32) sm[lane + 32] = t;
    }
    __syncthreads();
    const long long warp_prefix = wid ? sm[32 + wid - 1] : 0;
    total = sm[32 + (blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

__global__ void __launch_bounds__(256) scan_reduce_kernel(const int32_t *__restrict__ cnt, int n,
                                                          long long *__restrict__ tile_sum) {
    __shared__ long long sm[64];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    long long v = 0;
    for (int q = threadIdx.x; q < SCAN_TILE; q += 256)
        if (base + q < n) v += cnt[base + q];
    long long tot;
    block_excl_scan_ll(v, sm, tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) scan_top_kernel(long long *__restrict__ tile_sum, int ntiles) {
    __shared__ long long sm[64];
    long long carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += 256) {
        const int q = b0 + threadIdx.x;
        const long long v = q < ntiles ? tile_sum[q] : 0;
        long long tot;
        const long long ex = block_excl_scan_ll(v, sm, tot);
        if (q < ntiles) tile_sum[q] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) tile_sum[ntiles] = carry;
}

// Each thread scans 16 consecutive counts of the tile.
__global__ void __launch_bounds__(256) scan_apply_kernel(const int32_t *__restrict__ cnt, int n,
                                                         const long long *__restrict__ tile_off,
                                                         int ntiles, int64_t *__restrict__ out) {
    __shared__ long long sm[64];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + 16 * threadIdx.x;
    int vals[16];
    long long mysum = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        vals[q] = (base + q < n) ? cnt[base + q] : 0;
        mysum += vals[q];
    }
    long long tot;
    long long run = block_excl_scan_ll(mysum, sm, tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        if (base + q < n) out[base + q] = run;
        run += vals[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tile_off[ntiles];
}

__global__ void add_base_kernel(int64_t *__restrict__ out, int n, const int64_t *__restrict__ base) {
    const int64_t b = *base;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q <= n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] += b;
}

cudaError_t launch_scan(const ScanArgs &a, const Work &w, cudaStream_t s) {
    const int ntiles = (a.n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles == 0) {
        cudaMemsetAsync(a.out_ptr, 0, sizeof(int64_t), s);
        return cudaGetLastError();
    }
    scan_reduce_kernel<<<ntiles, 256, 0, s>>>(a.cnt, a.n, w.tile_sum);
    scan_top_kernel<<<1, 256, 0, s>>>(w.tile_sum, ntiles);
    scan_apply_kernel<<<ntiles, 256, 0, s>>>(a.cnt, a.n, w.tile_sum, ntiles, a.out_ptr);
    return cudaGetLastError();
}

// ============================================================================ cell list

__global__ void bin_assign_kernel(int atom_lo, int atom_hi, const int32_t *__restrict__ atom_struct,
                                  const StructRec *__restrict__ recs, const float *__restrict__ frac,
                                  int32_t *__restrict__ bin_cnt, int32_t *__restrict__ atom_bin) {
    for (int r = atom_lo + blockIdx.x * blockDim.x + threadIdx.x; r < atom_hi; r += gridDim.x * blockDim.x) {
        const StructRec &R = recs[atom_struct[r]];
        if (R.nb[0] == 0) {
            atom_bin[r] = -1;
            continue;
        }
        const int b0 = bin_of(wrap01(frac[3 * (int64_t)r + 0]), R.nb[0]);
        const int b1 = bin_of(wrap01(frac[3 * (int64_t)r + 1]), R.nb[1]);
        const int b2 = bin_of(wrap01(frac[3 * (int64_t)r + 2]), R.nb[2]);
        const int g = R.bin_base + (b0 * R.nb[1] + b1) * R.nb[2] + b2;
        atom_bin[r] = g;
        atomicAdd(&bin_cnt[g], 1);
    }
}

__global__ void bin_scatter_kernel(int atom_lo, int atom_hi, const int32_t *__restrict__ atom_struct,
                                   const StructRec *__restrict__ recs, const int32_t *__restrict__ atom_bin,
                                   const int64_t *__restrict__ cell_start, int32_t *__restrict__ cursor,
                                   const float *__restrict__ frac, const float4 *__restrict__ pos,
                                   float4 *__restrict__ cell_fx, float4 *__restrict__ cell_p) {
    for (int r = atom_lo + blockIdx.x * blockDim.x + threadIdx.x; r < atom_hi; r += gridDim.x * blockDim.x) {
        const int g = atom_bin[r];
        if (g < 0) continue;
        const int64_t slot = cell_start[g] + atomicAdd(&cursor[g], 1);
        const int jl = r - recs[atom_struct[r]].atom_begin;
        cell_fx[slot] = make_float4(frac[3 * (int64_t)r], frac[3 * (int64_t)r + 1], frac[3 * (int64_t)r + 2],
                                    __int_as_float(jl));
        cell_p[slot] = pos[r];
    }
}

__global__ void add_const_kernel(int64_t *__restrict__ out, int n, int64_t c) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q <= n; q += gridDim.x * blockDim.x) out[q] += c;
}

cudaError_t launch_bins(int B, int N, const float *frac, const Work &w, cudaStream_t s) {
    const int nbins = N + B;
    cudaMemsetAsync(w.bin_cnt, 0, sizeof(int32_t) * (size_t)nbins, s);
    cudaMemsetAsync(w.bin_cursor, 0, sizeof(int32_t) * (size_t)nbins, s);
    const int grid = max(1, min(4 * num_sms(), (N + 255) / 256));
    bin_assign_kernel<<<grid, 256, 0, s>>>(0, N, w.atom_struct, w.recs, frac, w.bin_cnt, w.atom_bin);
    ScanArgs sa{nbins, w.bin_cnt, w.cell_start};
    cudaError_t e = launch_scan(sa, w, s);
    if (e) return e;
    bin_scatter_kernel<<<grid, 256, 0, s>>>(0, N, w.atom_struct, w.recs, w.atom_bin, w.cell_start, w.bin_cursor,
                                            frac, w.pos, w.cell_fx, w.cell_p);
    return cudaGetLastError();
}

cudaError_t launch_bins_one(int atom_lo, int atom_hi, int bin_base, const float *frac, const Work &w,
                            cudaStream_t s) {
    const int n = atom_hi - atom_lo;
    const int nbins = n + 1;
    cudaMemsetAsync(w.bin_cnt + bin_base, 0, sizeof(int32_t) * (size_t)nbins, s);
    cudaMemsetAsync(w.bin_cursor + bin_base, 0, sizeof(int32_t) * (size_t)nbins, s);
    const int grid = max(1, min(4 * num_sms(), (n + 255) / 256));
    bin_assign_kernel<<<grid, 256, 0, s>>>(atom_lo, atom_hi, w.atom_struct, w.recs, frac, w.bin_cnt, w.atom_bin);
    ScanArgs sa{nbins, w.bin_cnt + bin_base, w.cell_start + bin_base};
    cudaError_t e = launch_scan(sa, w, s);
    if (e) return e;
    add_const_kernel<<<max(1, min(64, (nbins + 255) / 256)), 256, 0, s>>>(w.cell_start + bin_base, nbins,
                                                                        (int64_t)atom_lo);
    bin_scatter_kernel<<<grid, 256, 0, s>>>(atom_lo, atom_hi, w.atom_struct, w.recs, w.atom_bin, w.cell_start,
                                            w.bin_cursor, frac, w.pos, w.cell_fx, w.cell_p);
    return cudaGetLastError();
}

// ============================================================================ schedule

// Work distribution over source atoms [lo, hi): flat (one warp per atom) or a persistent
// grid whose warps pull atoms from a counter (w.queue[0]) until the range is exhausted.
template <int SCHED>
struct AtomLoop {
    int lo, hi;
    unsigned int *queue;
    __device__ __forceinline__ int first() {
        if (SCHED == 1) {
            const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
            return lo + gw;
        }
        return next();
    }
    __device__ __forceinline__ int next() {
        if (SCHED == 1) return hi;
        unsigned int v = 0;
        if (lane_id() == 0) v = atomicAdd(queue, 1u);
        v = __shfl_sync(FULL, v, 0);
        return lo + (int)v;
    }
};

// ============================================================================ cutoff count

template <int SCHED>
__global__ void __launch_bounds__(256) cutoff_count_kernel(BuildArgs a, Work w) {
    AtomLoop<SCHED> loop{a.atom_lo, a.atom_hi, w.queue};
    unsigned long long nre = 0, ncand = 0;
    for (int i = loop.first(); i < a.atom_hi; i = loop.next()) {
        const int s = w.atom_struct[i];
        const StructRec &R = w.recs[s];
        if (R.bad) {
            if (lane_id() == 0) {
                w.cnt[i] = 0;
                if (i == R.atom_begin) set_error(a.g.status, R.bad, s + a.struct_offset);
            }
            continue;
        }
        Source S;
        load_source(S, w.recs, s, a.frac, w.pos, i);
        const float thr_lo = R.thr_lo, thr_hi = R.thr_hi;
        const double rr = R.rr;
        int count = 0;
        const Cells cells{w.cell_start, w.cell_fx, w.cell_p};
        for_each_candidate(S, a.frac, w.pos, cells, true, R.cut, nullptr, [&](bool vc, float d2, bool self, int ow, int t2,
                                                                      const RowRegs &rw) {
            const bool cand = vc && !self;
            bool in = cand && d2 < thr_lo;
            const bool band = cand && !in && d2 <= thr_hi;
            if (__any_sync(FULL, band)) {
                const int jj = __shfl_sync(FULL, rw.j, ow);
                const int t0 = __shfl_sync(FULL, rw.t0, ow);
                const int t1 = __shfl_sync(FULL, rw.t1, ow);
                if (band) {
                    const int64_t jr = (int64_t)S.begin + jj;
                    const double d = canon_d2(S.L, S.xi0, S.xi1, S.xi2, a.frac[3 * jr], a.frac[3 * jr + 1],
                                              a.frac[3 * jr + 2], t0, t1, t2);
                    in = d < rr;
                }
                nre += __popc(__ballot_sync(FULL, band));
            }
            count += __popc(__ballot_sync(FULL, in));
            ncand += __popc(__ballot_sync(FULL, cand));
        });
        if (lane_id() == 0) w.cnt[i] = count;
    }
    if (a.collect_stats && lane_id() == 0 && ncand) {
        Status *st = reinterpret_cast<Status *>(a.g.status);
        atomicAdd(&st->rechecked, nre);
        atomicAdd(&st->candidates, ncand);
    }
}

static int blocks_for(int atoms, int threads) {
    const int warps = threads / 32;
    return (atoms + warps - 1) / warps;
}

static int persistent_blocks(const void *kernel, int threads) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * num_sms();
}

cudaError_t launch_reset_queue(const Work &w, cudaStream_t s) {
    return cudaMemsetAsync(w.queue, 0, 4 * sizeof(unsigned int), s);
}

cudaError_t launch_cutoff_count(const BuildArgs &a, const Work &w, cudaStream_t s) {
    const int atoms = a.atom_hi - a.atom_lo;
    if (atoms <= 0) return cudaSuccess;
    const int threads = 256;
    if (a.schedule == 2) {
        cudaError_t e = launch_reset_queue(w, s);
        if (e) return e;
        int blocks = persistent_blocks((const void *)cutoff_count_kernel<2>, threads);
        blocks = min(blocks, blocks_for(atoms, threads));
        cutoff_count_kernel<2><<<blocks, threads, 0, s>>>(a, w);
    } else {
        cutoff_count_kernel<1><<<blocks_for(atoms, threads), threads, 0, s>>>(a, w);
    }
    return cudaGetLastError();
}

// ============================================================================ finalize

// After the scan of per-atom counts: edge_ptr[s] = src_ptr[atom_ptr[s]], edge count and
// capacity check.  For a per-structure build (B == 1 slice) the same holds with the
// pointers offset by the caller.
__global__ void cutoff_finalize_kernel(int B, const int32_t *__restrict__ atom_ptr, int N,
                                       const int64_t *__restrict__ src_ptr, int64_t *__restrict__ edge_ptr,
                                       int64_t capacity, mg_device_status_t *status) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= B; s += gridDim.x * blockDim.x) {
        const int a = (s == B) ? N : atom_ptr[s];
        edge_ptr[s] = src_ptr[a];
        if (s == B) {
            const long long tot = src_ptr[N];
            Status *st = reinterpret_cast<Status *>(status);
            st->num_edges = (unsigned long long)tot;
            st->required_capacity = (unsigned long long)tot;
            if (tot > capacity) set_error(status, MG_ERR_CAPACITY, -1);
        }
    }
}

cudaError_t launch_cutoff_finalize(const BuildArgs &a, const Work &w, cudaStream_t s) {
    const int threads = 256;
    const int blocks = min(1024, (a.B + 1 + threads - 1) / threads);
    cutoff_finalize_kernel<<<blocks, threads, 0, s>>>(a.B, a.atom_ptr, a.N, a.src_ptr, a.g.edge_ptr,
                                                      a.g.capacity, a.g.status);
    return cudaGetLastError();
}

// ============================================================================ cutoff write

constexpr int WRITE_WARPS = 4;

// The count kernel's scan again, emitting each source's edges at its scanned offset in
// canonical order.  All-pairs structures emit in enumeration order (already canonical,
// ballot/popc positions).  Cell-list structures gather the source's (j, t) keys in
// shared memory, sort them, then emit; a source with more edges than WRITE_CAP or an
// offset beyond the packed key range is emitted through the all-pairs enumeration.
template <int SCHED>
__global__ void __launch_bounds__(WRITE_WARPS * 32) cutoff_write_kernel(BuildArgs a, Work w) {
    __shared__ unsigned long long keys_all[WRITE_WARPS][WRITE_CAP];
    unsigned long long *keys = keys_all[threadIdx.x >> 5];
    AtomLoop<SCHED> loop{a.atom_lo, a.atom_hi, w.queue};
    const mg_graph_t g = a.g;
    const Cells cells{w.cell_start, w.cell_fx, w.cell_p};
    const unsigned lt = (1u << lane_id()) - 1u;
    for (int i = loop.first(); i < a.atom_hi; i = loop.next()) {
        const int s = w.atom_struct[i];
        const int64_t base = a.src_ptr[i];
        const int64_t endp = a.src_ptr[i + 1];
        if (endp > g.capacity || endp == base) continue;  // capacity error already reported
        const StructRec &R = w.recs[s];
        if (R.bad) continue;
        Source S;
        load_source(S, w.recs, s, a.frac, w.pos, i);
        const float thr_lo = R.thr_lo, thr_hi = R.thr_hi;
        const double rr = R.rr;
        const int64_t deg = endp - base;
        bool done = false;
        if (S.nb[0] != 0 && deg <= WRITE_CAP) {
            int m = 0;
            bool range_bad = false;
            for_each_candidate(S, a.frac, w.pos, cells, true, R.cut, nullptr, [&](bool vc, float d2, bool self, int ow,
                                                                          int t2, const RowRegs &rw) {
                const bool cand = vc && !self;
                bool in = cand && d2 < thr_lo;
                const bool band = cand && !in && d2 <= thr_hi;
                if (__any_sync(FULL, in || band)) {
                    const int jj = __shfl_sync(FULL, rw.j, ow);
                    const int t0 = __shfl_sync(FULL, rw.t0, ow);
                    const int t1 = __shfl_sync(FULL, rw.t1, ow);
                    if (band) {
                        const int64_t jr = (int64_t)S.begin + jj;
                        in = canon_d2(S.L, S.xi0, S.xi1, S.xi2, a.frac[3 * jr], a.frac[3 * jr + 1],
                                      a.frac[3 * jr + 2], t0, t1, t2) < rr;
                    }
                    const unsigned bal = __ballot_sync(FULL, in);
                    if (in) {
                        if (abs(t0) > OFFSET_KEY_LIM || abs(t1) > OFFSET_KEY_LIM || abs(t2) > OFFSET_KEY_LIM)
                            range_bad = true;
                        const int p = m + __popc(bal & lt);
                        if (p < WRITE_CAP)
                            keys[p] = ((unsigned long long)(unsigned)jj << 32) | pack_t(t0, t1, t2);
                    }
                    m += __popc(bal);
                }
            });
            if (!__any_sync(FULL, range_bad) && m == deg) {
                int P = 64;
                while (P < m) P <<= 1;
                warp_smem_sort_u64(keys, m, P);
                for (int q = lane_id(); q < m; q += 32) {
                    const unsigned long long key = keys[q];
                    int t0, t1, t2;
                    unpack_t((uint32_t)(key & 0xffffffffull), t0, t1, t2);
                    const int64_t jr = (int64_t)S.begin + (int)(key >> 32);
                    emit_edge(g, S, i, base + q, jr, a.frac[3 * jr], a.frac[3 * jr + 1], a.frac[3 * jr + 2], t0,
                              t1, t2);
                }
                done = true;
            }
            __syncwarp();
        }
        if (done) continue;
        int64_t out = base;
        for_each_candidate(S, a.frac, w.pos, cells, false, R.cut, nullptr, [&](bool vc, float d2, bool self, int ow,
                                                                       int t2, const RowRegs &rw) {
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
                if (band) in = canon_d2(S.L, S.xi0, S.xi1, S.xi2, xj0, xj1, xj2, t0, t1, t2) < rr;
                const unsigned bal = __ballot_sync(FULL, in);
                if (in) {
                    const int64_t e = out + __popc(bal & lt);
                    if (e < endp) emit_edge(g, S, i, e, jr, xj0, xj1, xj2, t0, t1, t2);
                }
                out += __popc(bal);
            }
        });
        if (lane_id() == 0 && out != endp) set_error(g.status, MG_ERR_INTERNAL, s);  // count/write mismatch
    }
}

cudaError_t launch_cutoff_write(const BuildArgs &a, const Work &w, cudaStream_t s) {
    const int atoms = a.atom_hi - a.atom_lo;
    if (atoms <= 0) return cudaSuccess;
    const int threads = WRITE_WARPS * 32;
    if (a.schedule == 2) {
        cudaError_t e = launch_reset_queue(w, s);
        if (e) return e;
        int blocks = persistent_blocks((const void *)cutoff_write_kernel<2>, threads);
        blocks = min(blocks, blocks_for(atoms, threads));
        cutoff_write_kernel<2><<<blocks, threads, 0, s>>>(a, w);
    } else {
        cutoff_write_kernel<1><<<blocks_for(atoms, threads), threads, 0, s>>>(a, w);
    }
    return cudaGetLastError();
}

// ============================================================================ single-pass build

// Cutoff graph in one pass.  Tiles of BUILD_WARPS consecutive source atoms are taken in
// order (a ticket per block, so every tile a block waits on is already running); each
// warp scans its source once and stages the edges' (j, t) keys in shared memory
// (canonical order from the all-pairs enumeration, sorted for cell-list sources); the
// tile's total is published, the tile's offset found by a decoupled look-back over the
// predecessors; then the edges are written from shared memory.  A source with more than
// BUILD_CAP edges (or an offset outside the packed key) is counted in the first scan
// and emitted by a second, canonical all-pairs scan.  Writes src_ptr, edge_ptr, the
// edge count and the capacity check too.  The radius is the structure's cutoff, or per
// source: c_i (Def. 3 with per-atom cutoffs) or an FP64 squared radius with an inclusive
// test (Alg. 2's filter, d <= d^k_i, for keep-ties KNN graphs).
// At most 85 registers (6 blocks of 4 warps per SM), the measured best register budget.
template <bool PERSRC>
__global__ void __launch_bounds__(BUILD_WARPS * 32, 6) cutoff_build_kernel(BuildArgs a, Work w) {
    __shared__ unsigned long long keys_all[BUILD_WARPS][BUILD_CAP];
    __shared__ __align__(4) unsigned char trim_all[BUILD_WARPS][32 * TRIM_STRIDE];  // row-trimming tables
    __shared__ int s_tile;
    __shared__ int s_cnt[BUILD_WARPS];
    __shared__ long long s_prefix;
    const int wid = threadIdx.x >> 5, lane = lane_id();
    unsigned long long *keys = keys_all[wid];
    unsigned char *trim = trim_all[wid];
    const mg_graph_t g = a.g;
    unsigned long long *flags = w.tile_flags;
    const int ntiles = gridDim.x;

    pdl_wait();  // prep's records, positions and zeroed counters
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(&w.queue[3], 1u);
    __syncthreads();
    const int tile = s_tile;
    const int i = a.atom_lo + tile * BUILD_WARPS + wid;
    const bool have = i < a.atom_hi;
    int m = 0;
    bool spill = false;  // edges not staged: emit through a second all-pairs scan
    SrcScan c;
    c.s = 0;
    bool usable = false;
    if (have) {
        usable = source_setup<PERSRC>(a, w, i, c);
        if (usable) m = scan_source<PERSRC>(a, w, c, keys, trim, spill);
    }
    if (lane == 0) s_cnt[wid] = m;
    __syncthreads();
    if (wid == 0) {  // the tile's count and prefix: one warp looks back
        long long agg = 0;
        for (int q = 0; q < BUILD_WARPS; ++q) agg += s_cnt[q];
        long long prefix = 0;
        if (tile == a.fault_tile) {
            // testing hook: this tile publishes nothing; the waits of later tiles run out
        } else if (tile == 0) {
            if (lane == 0) atomicExch(&flags[0], TILE_PREFIX | (unsigned long long)agg);
        } else {
            if (lane == 0) atomicExch(&flags[tile], TILE_AGG | (unsigned long long)agg);
            __syncwarp();
            prefix = tile_lookback_warp(flags, tile, g.status);
            if (lane == 0) atomicExch(&flags[tile], TILE_PREFIX | (unsigned long long)(prefix + agg));
        }
        if (lane == 0) s_prefix = prefix;
        if (lane == 0 && tile == ntiles - 1) {  // the last tile knows the edge count
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
    int64_t base = s_prefix;
    for (int q = 0; q < wid; ++q) base += s_cnt[q];
    if (lane == 0) {
        a.src_ptr[i] = base;
        const int s = w.atom_struct[i];
        for (int q = s; q >= 0 && a.atom_ptr[q] == i; --q) g.edge_ptr[q] = base;  // structures starting at i
    }
    if (m == 0 || base + m > g.capacity) return;  // nothing to write, or the capacity error
    emit_source<PERSRC>(a, w, c, i, base, m, keys, trim, spill);
}

// Decoupled build, part 1 (no dependence between sources): each warp scans a source and
// copies its staged keys to a global staging area at a slot taken with one atomic add;
// the count goes to cnt[i] and the slot to stage_off[i] (-1: spilled source).
template <bool PERSRC>
__global__ void __launch_bounds__(BUILD_WARPS * 32, 6) cutoff_stage_kernel(BuildArgs a, Work w) {
    __shared__ unsigned long long keys_all[BUILD_WARPS][BUILD_CAP];
    const int wid = threadIdx.x >> 5, lane = lane_id();
    unsigned long long *keys = keys_all[wid];
    pdl_wait();  // prep's records, positions and zeroed counters
    const int i = a.atom_lo + blockIdx.x * BUILD_WARPS + wid;
    if (i >= a.atom_hi) return;
    SrcScan c;
    int m = 0;
    bool spill = false;
    if (source_setup<PERSRC>(a, w, i, c, true)) m = scan_source<PERSRC>(a, w, c, keys, nullptr, spill);
    long long off = -1;
    if (!spill && m > 0) {
        if (lane == 0) off = (long long)atomicAdd(w.stage_ctr, (unsigned long long)m);
        off = __shfl_sync(FULL, off, 0);
        if (off + m <= w.max_edges) {
            for (int q = lane; q < m; q += 32) w.stage[off + q] = keys[q];
        } else {
            spill = true;  // staging area full (more edges than the workspace covers)
            if (!PERSRC && a.write_pairs && lane == 0) w.pair_ok[c.s] = 0;
        }
    }
    if (lane == 0) {
        w.cnt[i] = m;
        w.stage_off[i] = spill ? -1 : off;
        if (spill && m > 0) note_spill(w.spill_list, w.queue, i);
    }
}

// Staged build, part 2 (after the scan of the counts): a thread per edge row.  Each
// warp takes a contiguous range of rows, so the source of a row comes from src_ptr by one
// binary search per warp and then forward steps; its key is the staged one.  The pair
// table of symmetric graphs records each run's ends from the neighbouring keys.
// Spilled sources are left to cutoff_spill_kernel.
template <bool PERSRC>
__global__ void __launch_bounds__(256) cutoff_emit_kernel(BuildArgs a, Work w) {
    const mg_graph_t &g = a.g;
    const int64_t E = a.src_ptr[a.atom_hi];
    if (E > g.capacity) return;  // reported by the finalize kernel
    const int lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t lo_e = a.src_ptr[a.atom_lo];
    const int64_t span = E - lo_e;
    const int64_t chunk = ((span + warps - 1) / warps + 31) & ~(int64_t)31;
    const int64_t e0 = lo_e + wid * chunk, e1 = min(E, e0 + chunk);
    if (e0 >= e1) return;
    int i = a.atom_lo;  // last source whose first row is <= e0
    {
        int lo = a.atom_lo, hi = a.atom_hi;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.src_ptr[mid] <= e0) lo = mid;
            else hi = mid;
        }
        i = lo;
    }
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        while (i + 1 < a.atom_hi && a.src_ptr[i + 1] <= e) ++i;
        const long long off = w.stage_off[i];
        if (off < 0) continue;  // spilled source
        const int64_t base = a.src_ptr[i];
        const int m = (int)(a.src_ptr[i + 1] - base);
        const int q = (int)(e - base);
        const StructRec &R = w.recs[w.atom_struct[i]];
        const unsigned long long key = w.stage[off + q];
        int t0, t1, t2;
        unpack_t((uint32_t)(key & 0xffffffffull), t0, t1, t2);
        const int jl = (int)(key >> 32);
        const int64_t jr = (int64_t)R.atom_begin + jl;
        if (!PERSRC && a.write_pairs && R.n_atoms <= PAIR_MAX) {
            if (q == 0 || (int)(w.stage[off + q - 1] >> 32) != jl) w.pair_lo[(int64_t)i * PAIR_MAX + jl] = (uint16_t)q;
            if (q == m - 1 || (int)(w.stage[off + q + 1] >> 32) != jl)
                w.pair_hi[(int64_t)i * PAIR_MAX + jl] = (uint16_t)(q + 1);
        }
        g.src[e] = i;
        g.dst[e] = (int32_t)jr;
        g.offset[3 * e + 0] = t0;
        g.offset[3 * e + 1] = t1;
        g.offset[3 * e + 2] = t2;
        if (g.vec || g.len) {
            const float L[9] = {R.L[0], R.L[1], R.L[2], R.L[3], R.L[4], R.L[5], R.L[6], R.L[7], R.L[8]};
            const float3 v = edge_vec_ff(L, a.frac[3 * (int64_t)i], a.frac[3 * (int64_t)i + 1],
                                         a.frac[3 * (int64_t)i + 2], a.frac[3 * jr], a.frac[3 * jr + 1],
                                         a.frac[3 * jr + 2], t0, t1, t2);
            if (g.vec) {
                g.vec[3 * e + 0] = v.x;
                g.vec[3 * e + 1] = v.y;
                g.vec[3 * e + 2] = v.z;
            }
            if (g.len) g.len[e] = vec_len(v);
        }
    }
}

// Staged build, spilled sources (more edges than the shared staging holds, an offset
// outside the packed key, or a full staging area): a small persistent grid takes the
// spill list, a warp per source enumerating it again in canonical all-pairs order and
// writing at src_ptr[i].
template <bool PERSRC>
__global__ void __launch_bounds__(BUILD_WARPS * 32, 6) cutoff_spill_kernel(BuildArgs a, Work w) {
    if (a.src_ptr[a.atom_hi] > a.g.capacity) return;  // reported by the finalize kernel
    const unsigned total = w.queue[12];
    for (;;) {
        unsigned v = 0;
        if (lane_id() == 0) v = atomicAdd(&w.queue[13], 1u);
        v = __shfl_sync(FULL, v, 0);
        if (v >= total) return;
        const int i = w.spill_list[v];
        const int64_t base = a.src_ptr[i];
        const int m = (int)(a.src_ptr[i + 1] - base);
        if (m == 0) continue;
        SrcScan c;
        if (!source_setup<PERSRC>(a, w, i, c)) continue;
        emit_source<PERSRC>(a, w, c, i, base, m, nullptr, nullptr, true);
    }
}

cudaError_t launch_cutoff_build(const BuildArgs &a, const Work &w, cudaStream_t s) {
    const int atoms = a.atom_hi - a.atom_lo;
    if (atoms <= 0) return cudaSuccess;
    const int tiles = (atoms + BUILD_WARPS - 1) / BUILD_WARPS;
    void (*kern)(BuildArgs, Work) = (a.cut_atom || a.rr_atom) ? cutoff_build_kernel<true> : cutoff_build_kernel<false>;
    if (a.pdl) return launch_pdl(kern, dim3(tiles), dim3(BUILD_WARPS * 32), s, a, w);
    kern<<<tiles, BUILD_WARPS * 32, 0, s>>>(a, w);
    return cudaGetLastError();
}

cudaError_t launch_cutoff_stage(const BuildArgs &a, const Work &w, cudaStream_t s) {
    const int atoms = a.atom_hi - a.atom_lo;
    if (atoms <= 0) return cudaSuccess;
    const int blocks = (atoms + BUILD_WARPS - 1) / BUILD_WARPS;
    void (*kern)(BuildArgs, Work) = (a.cut_atom || a.rr_atom) ? cutoff_stage_kernel<true> : cutoff_stage_kernel<false>;
    if (a.pdl) return launch_pdl(kern, dim3(blocks), dim3(BUILD_WARPS * 32), s, a, w);
    kern<<<blocks, BUILD_WARPS * 32, 0, s>>>(a, w);
    return cudaGetLastError();
}

cudaError_t launch_cutoff_counts(const BuildArgs &a, const Work &w, cudaStream_t s) {
    const int atoms = a.atom_hi - a.atom_lo;
    ScanArgs sa{atoms, w.cnt + a.atom_lo, a.src_ptr + a.atom_lo};
    cudaError_t e = launch_scan(sa, w, s);
    if (e) return e;
    return launch_cutoff_finalize(a, w, s);
}

cudaError_t launch_cutoff_emit(const BuildArgs &a, const Work &w, cudaStream_t s) {
    const int atoms = a.atom_hi - a.atom_lo;
    if (atoms <= 0) return cudaSuccess;
    // rows live on the device: a thread per row of a graph up to the capacity, capped at
    // 16 blocks per SM (longer ranges per warp beyond)
    const int64_t want = (a.g.capacity + 255) / 256;
    const int blocks = (int)(want < 16 * num_sms() ? (want > 0 ? want : 1) : 16 * num_sms());
    const int sblocks = max(1, min((atoms + BUILD_WARPS - 1) / BUILD_WARPS, 2 * num_sms()));  // spill list: usually empty
    if (a.cut_atom || a.rr_atom) {
        cutoff_emit_kernel<true><<<blocks, 256, 0, s>>>(a, w);
        cutoff_spill_kernel<true><<<sblocks, BUILD_WARPS * 32, 0, s>>>(a, w);
    } else {
        cutoff_emit_kernel<false><<<blocks, 256, 0, s>>>(a, w);
        cutoff_spill_kernel<false><<<sblocks, BUILD_WARPS * 32, 0, s>>>(a, w);
    }
    return cudaGetLastError();
}

// ============================================================================ dst sort

__global__ void dst_hist_kernel(const int32_t *__restrict__ dst, const int64_t *__restrict__ E_dev,
                                int64_t capacity, int32_t *__restrict__ deg) {
    const int64_t E = *E_dev;
    if (E > capacity) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&deg[dst[e]], 1);
}

__global__ void dst_scatter_kernel(const int32_t *__restrict__ dst, const int64_t *__restrict__ E_dev,
                                   int64_t capacity, const int64_t *__restrict__ dst_ptr,
                                   int32_t *__restrict__ cursor, int32_t *__restrict__ perm) {
    const int64_t E = *E_dev;
    if (E > capacity) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int d = dst[e];
        perm[dst_ptr[d] + atomicAdd(&cursor[d], 1)] = (int32_t)e;
    }
}

constexpr int SEG_SMEM = 2048;  // per-warp shared-memory sort capacity (edge ids)

__device__ __forceinline__ int warp_sort32_int(int x) {
    const int lane = lane_id();
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
        const bool desc = (lane & size) != 0;
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int y = __shfl_xor_sync(FULL, x, stride);
            const bool lower = (lane & stride) == 0;
            x = (lower != desc) ? min(x, y) : max(x, y);
        }
    }
    return x;
}

// Warp per destination atom: sort its segment of perm_dst ascending (edge ids are in
// canonical (src, dst, t) order, so this yields (dst, src, t) order).
__global__ void __launch_bounds__(128) dst_segsort_kernel(int N, const int64_t *__restrict__ dst_ptr,
                                                          const int64_t *__restrict__ E_dev, int64_t capacity,
                                                          int32_t *__restrict__ perm, int32_t *__restrict__ tmp) {
    __shared__ int32_t sm[4][SEG_SMEM];
    if (*E_dev > capacity) return;
    const int wid = threadIdx.x >> 5, lane = lane_id();
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= N) return;
    const int64_t lo = dst_ptr[j], hi = dst_ptr[j + 1];
    const int n = (int)(hi - lo);
    if (n <= 1) return;
    if (n <= 32) {
        int v = lane < n ? perm[lo + lane] : 0x7fffffff;
        v = warp_sort32_int(v);
        if (lane < n) perm[lo + lane] = v;
        return;
    }
    if (n <= SEG_SMEM) {
        int P = 64;
        while (P < n) P <<= 1;
        int32_t *b = sm[wid];
        for (int q = lane; q < P; q += 32) b[q] = q < n ? perm[lo + q] : 0x7fffffff;
        __syncwarp();
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int q = lane; q < P / 2; q += 32) {
                    const int x = 2 * stride * (q / stride) + (q % stride);
                    const int y = x + stride;
                    const bool asc = (x & size) == 0;
                    const int vx = b[x], vy = b[y];
                    if ((vx > vy) == asc) {
                        b[x] = vy;
                        b[y] = vx;
                    }
                }
                __syncwarp();
            }
        }
        for (int q = lane; q < n; q += 32) perm[lo + q] = b[q];
        return;
    }
    // long segment: rank sort through scratch (ids are distinct)
    for (int64_t q = lo + lane; q < hi; q += 32) tmp[q] = perm[q];
    __syncwarp();
    for (int64_t q = lo + lane; q < hi; q += 32) {
        const int v = tmp[q];
        int64_t rank = 0;
        for (int64_t r = lo; r < hi; ++r) rank += tmp[r] < v;
        perm[lo + rank] = v;
    }
}

// First position in [lo, hi) of sorted keys with key >= v (or > v when upper).
__device__ __forceinline__ int64_t bound32(const int32_t *__restrict__ keys, int64_t lo, int64_t hi, int v,
                                           bool upper) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int k = keys[mid];
        if (k < v || (upper && k == v)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Destination order of a symmetric graph ((i, j, t) present iff (j, i, -t) is, as for a
// cutoff graph: the canonical distance is sign-symmetric).  j's in-edges are the
// reverses of its out-edges, so dst_ptr = src_ptr, and for the run of j's out-edges to
// atom i (positions [rlo, rhi), offsets ascending) the reversed edges (i, j, -t) form
// the run of i's out-edges to j in the opposite order: out-edge p of the run maps to
// edge s_ij + (rhi - 1 - p) and to in-list position rlo + (rhi - 1 - p).
__global__ void __launch_bounds__(256) dst_perm_symmetric_kernel(int N, const int64_t *__restrict__ src_ptr,
                                                                 const int32_t *__restrict__ dst,
                                                                 const int64_t *__restrict__ E_dev, int64_t capacity,
                                                                 int32_t *__restrict__ perm,
                                                                 int64_t *__restrict__ dst_ptr,
                                                                 mg_device_status_t *status) {
    const int64_t E = *E_dev;
    if (E > capacity) return;
    if (reinterpret_cast<const Status *>(status)->code == MG_ERR_TIMEOUT) return;  // offsets not valid
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= N) return;
    const int64_t lo = src_ptr[j], hi = src_ptr[j + 1];
    if (lane_id() == 0) {
        dst_ptr[j] = lo;
        if (j == N - 1) dst_ptr[N] = hi;
    }
    if (lo < 0 || hi > E) {  // never for a graph built here
        if (lane_id() == 0) set_error(status, MG_ERR_INTERNAL, -1);
        return;
    }
    for (int64_t p = lo + lane_id(); p < hi; p += 32) {
        const int i = dst[p];
        if (i < 0 || i >= N) {  // never for a graph built here
            set_error(status, MG_ERR_INTERNAL, -1);
            continue;
        }
        const int64_t rlo = bound32(dst, lo, hi, i, false);
        const int64_t rhi = bound32(dst, lo, hi, i, true);
        const int64_t ilo = src_ptr[i], ihi = src_ptr[i + 1];
        if (ilo < 0 || ihi > E || ihi < ilo) {  // never for a graph built here
            set_error(status, MG_ERR_INTERNAL, -1);
            continue;
        }
        const int64_t sij = bound32(dst, ilo, ihi, j, false);
        if (p == rlo) {  // the reverse run must have the same length
            const int64_t len = rhi - rlo;
            const bool ok = sij + len <= ihi && dst[sij + len - 1] == j && (sij + len == ihi || dst[sij + len] != j);
            if (!ok) set_error(status, MG_ERR_INTERNAL, -1);
        }
        perm[rlo + (rhi - 1 - p)] = (int32_t)(sij + (rhi - 1 - p));
    }
}

cudaError_t launch_dst_perm_symmetric(const BuildArgs &a, const Work &, cudaStream_t s) {
    if (a.N <= 0) return cudaSuccess;
    dst_perm_symmetric_kernel<<<(a.N + 7) / 8, 256, 0, s>>>(a.N, a.src_ptr, a.g.dst, a.g.edge_ptr + a.B, a.g.capacity,
                                                          a.g.perm_dst, a.g.dst_ptr, a.g.status);
    return cudaGetLastError();
}

cudaError_t launch_dst_sort(const BuildArgs &a, const Work &w, cudaStream_t s, int *launches) {
    const mg_graph_t &g = a.g;
    const int64_t *E_dev = g.edge_ptr + a.B;
    const int grid = 4 * num_sms();
    cudaMemsetAsync(w.cnt, 0, sizeof(int32_t) * (size_t)(a.N > 0 ? a.N : 1), s);
    dst_hist_kernel<<<grid, 256, 0, s>>>(g.dst, E_dev, g.capacity, w.cnt);
    ScanArgs sa{a.N, w.cnt, g.dst_ptr};
    cudaError_t e = launch_scan(sa, w, s);
    if (e) return e;
    cudaMemsetAsync(w.cursor, 0, sizeof(int32_t) * (size_t)(a.N > 0 ? a.N : 1), s);
    dst_scatter_kernel<<<grid, 256, 0, s>>>(g.dst, E_dev, g.capacity, g.dst_ptr, w.cursor, g.perm_dst);
    if (a.N > 0) dst_segsort_kernel<<<(a.N + 3) / 4, 128, 0, s>>>(a.N, g.dst_ptr, E_dev, g.capacity, g.perm_dst, w.sort_tmp);
    if (launches) *launches += 6;
    return cudaGetLastError();
}

}  // namespace mg
