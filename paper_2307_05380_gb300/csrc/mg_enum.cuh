// Warp-per-source-atom enumeration of periodic-image candidates (j, t) within a radius.
//
// The paper searches the torus by expanding the evaluated area of periodic images until
// it covers the search radius (Sec. 2.2, Alg. 1).  Here the evaluated area is computed
// directly from interplanar spacings: every image with |v| < rho satisfies
// |x_j,k - x_i,k + t_k| <= rho ||L^-1[:, k]|| = rho / d_k, so each pair (i, j) gets an exact
// per-axis offset box; each (t0, t1) row of that box is further trimmed to the chord of
// the sphere along L_2.  The warp walks the candidates 32 at a time through flattening
// levels (target atoms -> rows -> candidates), finding owners with a warp binary search
// over inclusive prefix counts, so that each step evaluates exactly 32 candidates.
//
// Target atoms come from one of two drivers:
//   all pairs  j = 0 .. n-1 in order, so lane order is canonical order (j, t0, t1, t2);
//   cell list  the structure's atoms binned by fractional coordinate (frac(x) * n_k per
//              axis, bins at least half the radius wide); a source visits only the bins
//              its reach interval [frac(x_i) - R_k, frac(x_i) + R_k] touches on each axis
//              (every bin at most once, also under wrap-around).  Bins only select
//              targets: offsets still come from the exact per-pair box on the unwrapped
//              coordinates, so every image within reach is found exactly once.
#pragma once

#include "mg_device.cuh"

namespace mg {

// Per-source constants a warp keeps in registers.
struct Source {
    float L[9];
    float invd[3];
    float inv_L2n2, L2norm;  // 1 / |L_2|^2 and |L_2|
    float xi0, xi1, xi2;
    float3 pi;
    int i_loc;   // local index of the source atom within its structure
    int begin;   // global row of the structure's first atom
    int n;       // atoms in the structure
    int nb[3];   // bins per axis (nb[0] == 0: all-pairs structure)
    int bin_base;
    int ax;      // lattice axis enumerated innermost (L, invd and xi are in the order (p0, p1, ax))
};

// With `permute`, an all-pairs structure whose record names another innermost axis is
// enumerated in the axis order (p0, p1, ax): its rows along the shortest direction hold
// more candidates each, so a skewed cell has fewer rows.  The offsets a visitor sees
// are then in that order (to_lattice_order maps them back).
__device__ __forceinline__ void load_source(Source &S, const StructRec *__restrict__ recs, int s,
                                            const float *__restrict__ frac,
                                            const float4 *__restrict__ pos, int i, bool permute = false) {
    const StructRec &R = recs[s];
    const int ax = (permute && R.nb[0] == 0 && (R.ax == 0 || R.ax == 1)) ? R.ax : 2;
    const int p0 = ax == 0 ? 1 : 0, p1 = ax == 2 ? 1 : 2;
    S.ax = ax;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        S.L[q] = R.L[3 * p0 + q];
        S.L[3 + q] = R.L[3 * p1 + q];
        S.L[6 + q] = R.L[3 * ax + q];
    }
    S.invd[0] = R.invd[p0];
    S.invd[1] = R.invd[p1];
    S.invd[2] = R.invd[ax];
#pragma unroll
    for (int k = 0; k < 3; ++k) S.nb[k] = R.nb[k];
    S.bin_base = R.bin_base;
    if (ax == 2) {
        S.inv_L2n2 = 1.0f / R.L2norm2;
        S.L2norm = R.L2norm;
    } else {
        const float n2 = S.L[6] * S.L[6] + S.L[7] * S.L[7] + S.L[8] * S.L[8];
        S.inv_L2n2 = 1.0f / n2;
        S.L2norm = sqrtf(n2);
    }
    S.begin = R.atom_begin;
    S.n = R.n_atoms;
    S.i_loc = i - S.begin;
    S.xi0 = frac[3 * (int64_t)i + p0];
    S.xi1 = frac[3 * (int64_t)i + p1];
    S.xi2 = frac[3 * (int64_t)i + ax];
    float4 p = pos[i];
    S.pi = make_float3(p.x, p.y, p.z);
}

// Cell list of the batch (device pointers in the workspace).
struct Cells {
    const int64_t *__restrict__ start;   // [bins + 1] first slot of each bin (global)
    const float4 *__restrict__ fx;       // [slots] fractional coordinates, .w = local index bits
    const float4 *__restrict__ p;        // [slots] FP32 Cartesian positions
};

// Row-level values a visitor may fetch from the row's owner lane (shuffle source ow).
struct RowRegs {
    int j;   // local target index
    int t0, t1;
};

// Row trimming: the (t0, t1) rows of a target's box are the lattice points of a
// parallelogram around the ellipse in which the sphere projects along L_2; a row holds
// candidates only if its line b + t2 L_2 passes within the radius.  With u, w the parts
// of L_0, L_1 orthogonal to L_2 and c that of the target offset, row (t0, t1) qualifies
// iff |c + t0 u + t1 w| < rho: for each t0 an interval of t1, found in closed form.
// Each target lane keeps, in a per-warp shared-memory area, the inclusive prefix of its
// rows per t0 (bytes) and each interval's first t1 (offset from the box, 4 bits), for
// boxes of at most TRIM_T0 x TRIM_T1 rows; larger boxes keep all their rows.  Pays where
// a warp's scan is a latency chain (the one-pass build); where the scan is issue-bound
// (the staged build, KNN) the table costs more instructions than the rows it saves.
constexpr int TRIM_T0 = 12, TRIM_T1 = 15;
constexpr int TRIM_STRIDE = 20;  // bytes per lane: 12 prefixes, 6 bytes of start nibbles (5 words: no bank conflicts)
struct Trim {
    float u[3], w[3];  // L_0 and L_1 minus their components along L_2
    float inv_ww;      // 1 / |w|^2
    float mu;          // widening of each t1 interval (t1 units)
    bool ok;           // usable (w not degenerate)
};

__device__ __forceinline__ Trim make_trim(const Source &S, float rho) {
    Trim T;
    const float *L = S.L;
    const float d0 = (L[0] * L[6] + L[1] * L[7] + L[2] * L[8]) * S.inv_L2n2;
    const float d1 = (L[3] * L[6] + L[4] * L[7] + L[5] * L[8]) * S.inv_L2n2;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T.u[k] = __fmaf_rn(-d0, L[6 + k], L[k]);
        T.w[k] = __fmaf_rn(-d1, L[6 + k], L[3 + k]);
    }
    const float ww = T.w[0] * T.w[0] + T.w[1] * T.w[1] + T.w[2] * T.w[2];
    const float l1 = L[3] * L[3] + L[4] * L[4] + L[5] * L[5];
    T.ok = ww > 1e-6f * l1 && isfinite(ww);
    T.inv_ww = T.ok ? 1.0f / ww : 0.f;
    T.mu = T.ok ? 1e-3f * (1.0f + rho * sqrtf(T.inv_ww)) : 0.f;
    return T;
}

// Wrapped fractional coordinate in [0, 1).
__device__ __forceinline__ float wrap01(float x) {
    float w = __fsub_rn(x, floorf(x));
    return w < 1.0f ? w : 0.0f;
}

// Bin of a wrapped coordinate along an axis with n bins.
__device__ __forceinline__ int bin_of(float w, int n) {
    return min(max((int)floorf(__fmul_rn(w, (float)n)), 0), n - 1);
}

// Levels 2 and 3 for the 32 target atoms held by the lanes (jl valid where vj; xj the
// target's fractional coordinates, pj its FP32 Cartesian position).  With `single`
// (reach below half a cell on every axis) a target has at most one image in reach, so
// each lane tests its own candidate directly and the flattening levels are skipped.
template <class Visit>
__device__ __forceinline__ void visit_targets(const Source &S, const float Rk[3], float rho2p, float rho1, float mu0,
                                              bool single, int jl, bool vj, float4 xj, float4 pj,
                                              const Trim &T, unsigned char *trim, Visit &visit) {
    const int lane = lane_id();
    int lo[3], nn[3];
    float3 a = make_float3(0.f, 0.f, 0.f);
    if (vj) {
        const float dx[3] = {__fsub_rn(xj.x, S.xi0), __fsub_rn(xj.y, S.xi1), __fsub_rn(xj.z, S.xi2)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float m = 1e-5f * (1.0f + fabsf(dx[k]) + Rk[k]);
            lo[k] = (int)ceilf(-Rk[k] - dx[k] - m);
            const int hi = (int)floorf(Rk[k] - dx[k] + m);
            nn[k] = max(0, hi - lo[k] + 1);
        }
        a = make_float3(__fsub_rn(pj.x, S.pi.x), __fsub_rn(pj.y, S.pi.y), __fsub_rn(pj.z, S.pi.z));
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = 0;
            nn[k] = 0;
        }
    }
    if (single) {
        // same operation order as the general path: b = a + t0 L0 + t1 L1, v = b + t2 L2
        const bool has = vj && nn[0] > 0 && nn[1] > 0 && nn[2] > 0;
        const float ft0 = (float)lo[0], ft1 = (float)lo[1], ft2 = (float)lo[2];
        const float bx = __fmaf_rn(ft1, S.L[3], __fmaf_rn(ft0, S.L[0], a.x));
        const float by = __fmaf_rn(ft1, S.L[4], __fmaf_rn(ft0, S.L[1], a.y));
        const float bz = __fmaf_rn(ft1, S.L[5], __fmaf_rn(ft0, S.L[2], a.z));
        const float vx = __fmaf_rn(ft2, S.L[6], bx);
        const float vy = __fmaf_rn(ft2, S.L[7], by);
        const float vz = __fmaf_rn(ft2, S.L[8], bz);
        const float d2 = __fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx)));
        RowRegs rr;
        rr.j = jl;
        rr.t0 = lo[0];
        rr.t1 = lo[1];
        const bool self = jl == S.i_loc && lo[0] == 0 && lo[1] == 0 && lo[2] == 0;
        visit(has, d2, self, lane, lo[2], rr);
        return;
    }
    int rows = (nn[2] > 0) ? nn[0] * nn[1] : 0;
    int trimmed = 0;
    if (trim) {
        __syncwarp();  // every lane is done with the previous targets' tables
        unsigned char *mine = trim + TRIM_STRIDE * lane;
        if (T.ok && rows > 0 && nn[0] <= TRIM_T0 && nn[1] <= TRIM_T1) {
            // c = the target offset minus its component along L_2
            const float al = (a.x * S.L[6] + a.y * S.L[7] + a.z * S.L[8]) * S.inv_L2n2;
            const float c0 = __fmaf_rn(-al, S.L[6], a.x), c1 = __fmaf_rn(-al, S.L[7], a.y),
                        c2 = __fmaf_rn(-al, S.L[8], a.z);
            int pre = 0;
            for (int r = 0; r < nn[0]; ++r) {
                const float ft0 = (float)(lo[0] + r);
                const float q0 = __fmaf_rn(ft0, T.u[0], c0), q1 = __fmaf_rn(ft0, T.u[1], c1),
                            q2 = __fmaf_rn(ft0, T.u[2], c2);
                // closest point of the line q + t1 w to the source: perpendicular p = q + m w
                const float m = -(q0 * T.w[0] + q1 * T.w[1] + q2 * T.w[2]) * T.inv_ww;
                const float p0 = __fmaf_rn(m, T.w[0], q0), p1 = __fmaf_rn(m, T.w[1], q1),
                            p2 = __fmaf_rn(m, T.w[2], q2);
                const float perp2 = __fmaf_rn(p2, p2, __fmaf_rn(p1, p1, __fmul_rn(p0, p0)));
                const float q2n = __fmaf_rn(q2, q2, __fmaf_rn(q1, q1, __fmul_rn(q0, q0)));
                int s1 = 0, cnt = nn[1];
                // the same error analysis as the chord below: FP32 errors stay far inside the
                // radius margin and mu while |q| and |m w| are at most 50 rho
                if (q2n <= 2500.0f * rho2p && fabsf(m) * fabsf(m) <= 2500.0f * rho2p * T.inv_ww) {
                    const float hsq = (rho2p - perp2) * T.inv_ww;
                    if (hsq < 0.0f) {
                        cnt = 0;
                    } else {
                        const float h = hsq > 0.0f ? hsq * rsqrtf(hsq) : 0.0f;
                        const float mu = T.mu + 6e-7f * fabsf(m);
                        const int l1 = max(lo[1], (int)ceilf(m - h - mu));
                        const int h1 = min(lo[1] + nn[1] - 1, (int)floorf(m + h + mu));
                        cnt = max(0, h1 - l1 + 1);
                        s1 = cnt > 0 ? l1 - lo[1] : 0;
                    }
                }
                pre += cnt;
                mine[r] = (unsigned char)pre;
                if (r & 1) mine[TRIM_T0 + (r >> 1)] |= (unsigned char)(s1 << 4);
                else mine[TRIM_T0 + (r >> 1)] = (unsigned char)s1;
            }
            for (int r = nn[0]; r < TRIM_T0; ++r) mine[r] = 0xff;  // keeps the prefixes monotone
            rows = pre;
            trimmed = 1;
        }
        __syncwarp();  // tables visible to the row lanes
    }
    const int incl = warp_incl_scan(rows);
    const int total = __shfl_sync(FULL, incl, 31);
    const int excl = incl - rows;

    for (int rb = 0; rb < total; rb += 32) {
        const int q = rb + lane;
        const bool vr = q < total;
        const int ow = warp_owner(incl, vr ? q : total - 1);
        const int o_excl = __shfl_sync(FULL, excl, ow);
        const int o_n1 = __shfl_sync(FULL, nn[1], ow);
        const int o_lo0 = __shfl_sync(FULL, lo[0], ow);
        const int o_lo1 = __shfl_sync(FULL, lo[1], ow);
        const int o_lo2 = __shfl_sync(FULL, lo[2], ow);
        const int o_n2 = __shfl_sync(FULL, nn[2], ow);
        const float ax = __shfl_sync(FULL, a.x, ow);
        const float ay = __shfl_sync(FULL, a.y, ow);
        const float az = __shfl_sync(FULL, a.z, ow);
        RowRegs rr;
        rr.j = __shfl_sync(FULL, jl, ow);
        const int rem = vr ? q - o_excl : 0;
        if (__shfl_sync(FULL, trimmed, ow)) {
            // the owner's trimmed rows: the t0 whose prefix first exceeds rem, then t1
            const unsigned char *tab = trim + TRIM_STRIDE * ow;
            int r = 0;
#pragma unroll
            for (int st = 8; st >= 1; st >>= 1) {
                const int idx = r + st - 1;  // entries past the table count as full
                if ((idx < TRIM_T0 ? (int)tab[idx] : 0xff) <= rem) r += st;
            }
            const int before = r > 0 ? (int)tab[r - 1] : 0;
            const int nib = (int)tab[TRIM_T0 + (r >> 1)];
            rr.t0 = o_lo0 + r;
            rr.t1 = o_lo1 + ((r & 1) ? (nib >> 4) : (nib & 15)) + (rem - before);
        } else {
            // rem / n1 from an approximate quotient, corrected to the exact integer one
            const int n1 = max(o_n1, 1);
            int d0 = (int)__fdividef((float)rem, (float)n1);
            while (d0 * n1 > rem) --d0;
            while ((d0 + 1) * n1 <= rem) ++d0;
            rr.t0 = o_lo0 + d0;
            rr.t1 = o_lo1 + (rem - d0 * o_n1);
        }
        // row base b = a + t0 L0 + t1 L1
        const float ft0 = (float)rr.t0, ft1 = (float)rr.t1;
        const float bx = __fmaf_rn(ft1, S.L[3], __fmaf_rn(ft0, S.L[0], ax));
        const float by = __fmaf_rn(ft1, S.L[4], __fmaf_rn(ft0, S.L[1], ay));
        const float bz = __fmaf_rn(ft1, S.L[5], __fmaf_rn(ft0, S.L[2], az));
        // chord of the sphere along L_2: t2 in t2c +- w, widened by mu.  The FP32
        // errors here (approximate reciprocal and square root included) stay below
        // 1e-5 rho / |L_2| + 6e-7 |t2c| while |b| + |t2c| |L_2| <= 100 rho, far inside mu.
        int c_lo = o_lo2, c_hi = o_lo2 + o_n2 - 1;
        {
            const float bl = __fmaf_rn(bz, S.L[8], __fmaf_rn(by, S.L[7], __fmul_rn(bx, S.L[6])));
            const float t2c = -bl * S.inv_L2n2;
            const float px = __fmaf_rn(t2c, S.L[6], bx);
            const float py = __fmaf_rn(t2c, S.L[7], by);
            const float pz = __fmaf_rn(t2c, S.L[8], bz);
            const float perp2 = __fmaf_rn(pz, pz, __fmaf_rn(py, py, __fmul_rn(px, px)));
            const float b2 = __fmaf_rn(bz, bz, __fmaf_rn(by, by, __fmul_rn(bx, bx)));
            if (b2 <= 2500.0f * rho2p && fabsf(t2c) * S.L2norm <= 50.0f * rho1) {  // error analysis holds
                const float wsq = (rho2p - perp2) * S.inv_L2n2;
                if (wsq < 0.0f) {
                    c_hi = c_lo - 1;
                } else {
                    const float w = wsq > 0.0f ? wsq * rsqrtf(wsq) : 0.0f;
                    const float mu = mu0 + 6e-7f * fabsf(t2c);
                    c_lo = max(c_lo, (int)ceilf(t2c - w - mu));
                    c_hi = min(c_hi, (int)floorf(t2c + w + mu));
                }
            }
        }
        const int clen = vr ? max(0, c_hi - c_lo + 1) : 0;
        const bool row_self = (rr.j == S.i_loc) && rr.t0 == 0 && rr.t1 == 0;
        const int incl2 = warp_incl_scan(clen);
        const int total2 = __shfl_sync(FULL, incl2, 31);
        const int excl2 = incl2 - clen;

        for (int cb = 0; cb < total2; cb += 32) {
            const int c = cb + lane;
            const bool vc = c < total2;
            const int ow2 = warp_owner(incl2, vc ? c : total2 - 1);
            const int e2 = __shfl_sync(FULL, excl2, ow2);
            const int clo = __shfl_sync(FULL, c_lo, ow2);
            const float cbx = __shfl_sync(FULL, bx, ow2);
            const float cby = __shfl_sync(FULL, by, ow2);
            const float cbz = __shfl_sync(FULL, bz, ow2);
            const bool cself = __shfl_sync(FULL, row_self ? 1 : 0, ow2) != 0;
            const int t2 = clo + (c - e2);
            const float ft2 = (float)t2;
            const float vx = __fmaf_rn(ft2, S.L[6], cbx);
            const float vy = __fmaf_rn(ft2, S.L[7], cby);
            const float vz = __fmaf_rn(ft2, S.L[8], cbz);
            const float d2 = __fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx)));
            visit(vc, d2, cself && t2 == 0, ow2, t2, rr);
        }
    }
}

// Visit all candidates with |v| < rho (a superset: box and chord are widened by safety
// margins; the caller classifies by distance).  For each chunk of 32 candidates every
// lane of the warp calls
//     visit(valid, d2, is_self, owner_lane, t2, rows)
// where d2 is the FP32 squared distance, is_self marks (i, i, 0), owner_lane is the lane
// whose `rows` hold this candidate's j, t0, t1 (fetch them with __shfl_sync), t2 the
// last offset component.  All calls are warp-uniform.  With use_cells, targets come from
// the cell list (any order of j); otherwise in ascending j (canonical order).
template <class Visit>
__device__ __forceinline__ void for_each_candidate(const Source &S, const float *__restrict__ frac,
                                                   const float4 *__restrict__ pos, const Cells &cells,
                                                   bool use_cells, float rho, unsigned char *trim, Visit &&visit) {
    const int lane = lane_id();
    const Trim T = make_trim(S, rho);
    float Rk[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) Rk[k] = rho * S.invd[k];
    const float rho2p = rho * rho * 1.0002f;
    const float rho1 = rho * 1.0001f;  // >= sqrt(rho2p)
    const float mu0 = 1e-3f * (1.0f + rho / S.L2norm);
    const bool single = fmaxf(Rk[0], fmaxf(Rk[1], Rk[2])) < 0.49f;

    if (!use_cells || S.nb[0] == 0) {
        const int p0 = S.ax == 0 ? 1 : 0, p1 = S.ax == 2 ? 1 : 2;  // the source's axis order
        for (int jb = 0; jb < S.n; jb += 32) {
            const int jl = jb + lane;
            const bool vj = jl < S.n;
            float4 xj = make_float4(0.f, 0.f, 0.f, 0.f), pj = xj;
            if (vj) {
                const int64_t row = (int64_t)S.begin + jl;
                xj = make_float4(frac[3 * row + p0], frac[3 * row + p1], frac[3 * row + S.ax], 0.f);
                pj = pos[row];
            }
            visit_targets(S, Rk, rho2p, rho1, mu0, single, jl, vj, xj, pj, T, trim, visit);
        }
        return;
    }
    // bins touched by the reach interval on each axis (each bin once)
    int blo[3], bcnt[3];
    {
        const float xw[3] = {wrap01(S.xi0), wrap01(S.xi1), wrap01(S.xi2)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int nk = S.nb[k];
            const float m = 1e-5f * (1.0f + Rk[k]);
            const int lo = (int)floorf((xw[k] - Rk[k] - m) * (float)nk);
            const int hi = (int)floorf((xw[k] + Rk[k] + m) * (float)nk);
            if (hi - lo + 1 >= nk) {
                blo[k] = 0;
                bcnt[k] = nk;
            } else {
                blo[k] = lo;
                bcnt[k] = hi - lo + 1;
            }
        }
    }
    const int nbins = bcnt[0] * bcnt[1] * bcnt[2];
    for (int bb = 0; bb < nbins; bb += 32) {
        const int q = bb + lane;
        const bool vb = q < nbins;
        int64_t st = 0;
        int cnt = 0;
        if (vb) {
            const int c2 = q % bcnt[2];
            const int c1 = (q / bcnt[2]) % bcnt[1];
            const int c0 = q / (bcnt[2] * bcnt[1]);
            const int b0 = ((blo[0] + c0) % S.nb[0] + S.nb[0]) % S.nb[0];
            const int b1 = ((blo[1] + c1) % S.nb[1] + S.nb[1]) % S.nb[1];
            const int b2 = ((blo[2] + c2) % S.nb[2] + S.nb[2]) % S.nb[2];
            const int64_t g = (int64_t)S.bin_base + (b0 * S.nb[1] + b1) * S.nb[2] + b2;
            st = cells.start[g];
            cnt = (int)(cells.start[g + 1] - st);
        }
        const int incl = warp_incl_scan(cnt);
        const int total = __shfl_sync(FULL, incl, 31);
        const int excl = incl - cnt;
        for (int ab = 0; ab < total; ab += 32) {
            const int q2 = ab + lane;
            const bool va = q2 < total;
            const int ow = warp_owner(incl, va ? q2 : total - 1);
            const int64_t ost = __shfl_sync(FULL, st, ow);
            const int oex = __shfl_sync(FULL, excl, ow);
            float4 xj = make_float4(0.f, 0.f, 0.f, 0.f), pj = xj;
            if (va) {
                xj = cells.fx[ost + (q2 - oex)];
                pj = cells.p[ost + (q2 - oex)];
            }
            visit_targets(S, Rk, rho2p, rho1, mu0, single, va ? __float_as_int(xj.w) : 0, va, xj, pj, T, trim, visit);
        }
    }
}

}  // namespace mg
