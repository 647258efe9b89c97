/*
 * FP64 CPU oracle for periodic cutoff and k-nearest-neighbour multigraphs of crystals.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg load this file's library.  It shares no code with the CUDA path.
 * It is plain and slow on purpose: brute force over an oversized box of cell offsets,
 * written so that it can be checked against the paper by eye.
 *
 * Definitions followed (Sec. 2.1):
 *   Def. 1  a material is (rho, x, z): a lattice and fractional coordinates.  Here the
 *           lattice is stored as L = rho^T, row r = lattice vector r, so that an edge
 *           vector is the row vector v = (x_j - x_i + t) L.
 *   Def. 3  the cutoff graph: Gamma_1 = {(i, j, t) : ||rho (x_j - x_i + t)|| < c_i}.
 *           Readings: the inequality is strict; (i, i, 0) is not an edge; images of an
 *           atom itself, (i, i, t != 0), are edges; x may lie outside [0, 1) and is never
 *           wrapped, so t is relative to the x given.
 *   Sec. 2.1 (after Def. 3) the KNN graph is the special case where c_i is the distance
 *           of the k-th nearest image of atom i.  Reading: exactly k edges per atom, ties
 *           broken by (d2, j, t) ascending, lexicographically, with t signed.  With
 *           keep_ties, Alg. 2's filter instead: every image whose d2 is <= the k-th d2.
 *   Def. 3  with one cutoff per atom (oracle_cutoff_atoms): the source's own c_i decides.
 *
 * The distance that decides membership and ranking is the canonical FP64 one, written
 * out below (canon_d2): every operation rounded to nearest, no fused multiply-add
 * (compile with -ffp-contract=off), inputs are the caller's values promoted to double.
 *
 * Box: for a pair (i, j) every edge has |dx_k + t_k| <= r ||L^-1[:, k]|| <= r ||L^-1||_F
 * (dx = x_j - x_i), so with the per-pair centre c = -round(dx) every edge lies in
 * c + [-Bx, Bx]^3 with Bx = ceil(r ||L^-1||_F) + 1.  Edges are produced in canonical order
 * (src, dst, tx, ty, tz) by the loop order itself.  As a self-check, an edge on the box
 * face |t_k - c_k| = Bx is reported as an error (the bound makes it impossible).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- edge buffer */

typedef struct {
    int64_t n, cap;
    int32_t *src, *dst, *off;
    double *d2;
} obuf_t;

void *oracle_buf_new(void) { return calloc(1, sizeof(obuf_t)); }

void oracle_buf_free(void *p) {
    obuf_t *b = (obuf_t *)p;
    if (!b) return;
    free(b->src); free(b->dst); free(b->off); free(b->d2);
    free(b);
}

int64_t oracle_buf_size(void *p) { return ((obuf_t *)p)->n; }

void oracle_buf_copy(void *p, int32_t *src, int32_t *dst, int32_t *off, double *d2) {
    obuf_t *b = (obuf_t *)p;
    if (src) memcpy(src, b->src, sizeof(int32_t) * b->n);
    if (dst) memcpy(dst, b->dst, sizeof(int32_t) * b->n);
    if (off) memcpy(off, b->off, sizeof(int32_t) * 3 * b->n);
    if (d2) memcpy(d2, b->d2, sizeof(double) * b->n);
}

static int push(obuf_t *b, int32_t s, int32_t d, const int t[3], double d2) {
    if (b->n == b->cap) {
        int64_t nc = b->cap ? 2 * b->cap : 1024;
        int32_t *ns = realloc(b->src, sizeof(int32_t) * nc);
        if (!ns) return -1;
        b->src = ns;
        int32_t *nd = realloc(b->dst, sizeof(int32_t) * nc);
        if (!nd) return -1;
        b->dst = nd;
        int32_t *no = realloc(b->off, sizeof(int32_t) * 3 * nc);
        if (!no) return -1;
        b->off = no;
        double *n2 = realloc(b->d2, sizeof(double) * nc);
        if (!n2) return -1;
        b->d2 = n2;
        b->cap = nc;
    }
    b->src[b->n] = s;
    b->dst[b->n] = d;
    b->off[3 * b->n + 0] = t[0];
    b->off[3 * b->n + 1] = t[1];
    b->off[3 * b->n + 2] = t[2];
    b->d2[b->n] = d2;
    b->n++;
    return 0;
}

/* ---------------------------------------------------------------- geometry */

/* Inverse of a 3x3 matrix by cofactors; returns the determinant (0 if singular). */
static double inverse3(const double L[9], double Li[9]) {
    double c00 = L[4] * L[8] - L[5] * L[7];
    double c01 = L[5] * L[6] - L[3] * L[8];
    double c02 = L[3] * L[7] - L[4] * L[6];
    double det = L[0] * c00 + L[1] * c01 + L[2] * c02;
    if (det == 0.0 || !isfinite(det)) return 0.0;
    Li[0] = c00 / det;
    Li[1] = (L[2] * L[7] - L[1] * L[8]) / det;
    Li[2] = (L[1] * L[5] - L[2] * L[4]) / det;
    Li[3] = c01 / det;
    Li[4] = (L[0] * L[8] - L[2] * L[6]) / det;
    Li[5] = (L[2] * L[3] - L[0] * L[5]) / det;
    Li[6] = c02 / det;
    Li[7] = (L[1] * L[6] - L[0] * L[7]) / det;
    Li[8] = (L[0] * L[4] - L[1] * L[3]) / det;
    return det;
}

static double frobenius(const double M[9]) {
    double s = 0.0;
    for (int q = 0; q < 9; ++q) s += M[q] * M[q];
    return sqrt(s);
}

/* Canonical FP64 distance of edge (i, j, t):
 *   df_c = (x_j[c] - x_i[c]) + t_c
 *   v_c  = ((df_0 L_0c + df_1 L_1c) + df_2 L_2c)
 *   d2   = ((v_0^2 + v_1^2) + v_2^2)
 * each operation rounded to nearest, evaluated left to right. */
static double canon_d2(const double L[9], const double *xi, const double *xj, const int t[3],
                       double v[3]) {
    double df0 = (xj[0] - xi[0]) + (double)t[0];
    double df1 = (xj[1] - xi[1]) + (double)t[1];
    double df2 = (xj[2] - xi[2]) + (double)t[2];
    double v0 = ((df0 * L[0]) + (df1 * L[3])) + (df2 * L[6]);
    double v1 = ((df0 * L[1]) + (df1 * L[4])) + (df2 * L[7]);
    double v2 = ((df0 * L[2]) + (df1 * L[5])) + (df2 * L[8]);
    if (v) { v[0] = v0; v[1] = v1; v[2] = v2; }
    return ((v0 * v0) + (v1 * v1)) + (v2 * v2);
}

static int valid_structure(const double L[9], const double *x, int n) {
    for (int q = 0; q < 9; ++q)
        if (!isfinite(L[q])) return 0;
    for (int q = 0; q < 3 * n; ++q)
        if (!isfinite(x[q])) return 0;
    return 1;
}

/* ---------------------------------------------------------------- cutoff graph */

/* Edges of source atom i (local index) of one structure, appended in canonical order.
 * row0 is the global row of the structure's first atom.  extra widens the box (the
 * result must not change).  Returns 0, -3 if the self-check failed, -1 on OOM. */
static int cutoff_atom(const double L[9], const double *x, int n, int i, double r, int extra,
                       int32_t row0, obuf_t *out) {
    double Li[9];
    if (inverse3(L, Li) == 0.0) return -2;
    int Bx = (int)ceil(r * frobenius(Li)) + 1 + extra;
    double rr = r * r;
    for (int j = 0; j < n; ++j) {
        int c[3];
        for (int k = 0; k < 3; ++k) c[k] = -(int)llround(x[3 * j + k] - x[3 * i + k]);
        int t[3];
        for (t[0] = c[0] - Bx; t[0] <= c[0] + Bx; ++t[0])
            for (t[1] = c[1] - Bx; t[1] <= c[1] + Bx; ++t[1])
                for (t[2] = c[2] - Bx; t[2] <= c[2] + Bx; ++t[2]) {
                    if (j == i && t[0] == 0 && t[1] == 0 && t[2] == 0) continue;
                    double d2 = canon_d2(L, x + 3 * i, x + 3 * j, t, NULL);
                    if (d2 < rr) {
                        for (int k = 0; k < 3; ++k)
                            if (abs(t[k] - c[k]) == Bx) return -3;
                        if (push(out, row0 + i, row0 + j, t, d2)) return -1;
                    }
                }
    }
    return 0;
}

static void atom_structure(int B, const int32_t *atom_ptr, int32_t *owner) {
    for (int s = 0; s < B; ++s)
        for (int32_t a = atom_ptr[s]; a < atom_ptr[s + 1]; ++a) owner[a] = s;
}

/* Cutoff graph of a batch.  lattice [B][9] row-major (row = lattice vector), frac
 * [N][3], cutoff [B] per-structure radii.  sources: ascending global rows to build
 * (NULL: every atom).  Returns 0, or a negative code: -1 out of memory, -2 singular
 * or non-finite structure, -3 box self-check failed, -4 bad arguments. */
int oracle_cutoff(int B, const int32_t *atom_ptr, const double *lattice, const double *frac,
                  const double *cutoff, int extra, const int32_t *sources, int64_t n_sources,
                  void *buf) {
    obuf_t *out = (obuf_t *)buf;
    int32_t N = atom_ptr[B];
    int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    if (!owner) return -1;
    atom_structure(B, atom_ptr, owner);
    int64_t count = sources ? n_sources : N;
    int rc = 0;
    for (int64_t q = 0; q < count && rc == 0; ++q) {
        int32_t a = sources ? sources[q] : (int32_t)q;
        if (a < 0 || a >= N) { rc = -4; break; }
        int s = owner[a];
        const double *L = lattice + 9 * s;
        const double *x = frac + 3 * (int64_t)atom_ptr[s];
        int n = atom_ptr[s + 1] - atom_ptr[s];
        if (!valid_structure(L, x, n) || !(cutoff[s] > 0.0)) { rc = -2; break; }
        rc = cutoff_atom(L, x, n, a - atom_ptr[s], cutoff[s], extra, atom_ptr[s], out);
    }
    free(owner);
    return rc;
}

/* Cutoff graph with one radius per atom (Def. 3 in full: the condition of edge (i, j, t)
 * uses the source's own c_i, so the graph need not be symmetric).  radius [N] holds
 * c_i for every global atom row; other arguments and return codes as oracle_cutoff. */
int oracle_cutoff_atoms(int B, const int32_t *atom_ptr, const double *lattice, const double *frac,
                        const double *radius, int extra, const int32_t *sources, int64_t n_sources,
                        void *buf) {
    obuf_t *out = (obuf_t *)buf;
    int32_t N = atom_ptr[B];
    int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    if (!owner) return -1;
    atom_structure(B, atom_ptr, owner);
    int64_t count = sources ? n_sources : N;
    int rc = 0;
    for (int64_t q = 0; q < count && rc == 0; ++q) {
        int32_t a = sources ? sources[q] : (int32_t)q;
        if (a < 0 || a >= N) { rc = -4; break; }
        int s = owner[a];
        const double *L = lattice + 9 * s;
        const double *x = frac + 3 * (int64_t)atom_ptr[s];
        int n = atom_ptr[s + 1] - atom_ptr[s];
        if (!valid_structure(L, x, n) || !(radius[a] > 0.0) || !isfinite(radius[a])) { rc = -2; break; }
        rc = cutoff_atom(L, x, n, a - atom_ptr[s], radius[a], extra, atom_ptr[s], out);
    }
    free(owner);
    return rc;
}

/* ---------------------------------------------------------------- KNN graph */

typedef struct { double d2; int32_t j; int t[3]; } cand_t;

/* Lexicographic order on (d2, j, t0, t1, t2). */
static int cand_less(const cand_t *a, const cand_t *b) {
    if (a->d2 != b->d2) return a->d2 < b->d2;
    if (a->j != b->j) return a->j < b->j;
    for (int k = 0; k < 3; ++k)
        if (a->t[k] != b->t[k]) return a->t[k] < b->t[k];
    return 0;
}

/* Lexicographic order on (j, t0, t1, t2): the canonical output order. */
static int jt_cmp(const void *pa, const void *pb) {
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    for (int k = 0; k < 3; ++k)
        if (a->t[k] != b->t[k]) return a->t[k] < b->t[k] ? -1 : 1;
    return 0;
}

/* The k nearest images of atom i, by brute force in a box that grows until it provably
 * holds every image at distance <= the k-th one:
 *   1. gather every (j, t) != (i, 0) in c + [-Bx, Bx]^3 and keep the k smallest by
 *      (d2, j, t);
 *   2. with D the k-th d2, any image with d2 <= D lies within ceil(sqrt(D) ||L^-1||_F) + 1
 *      of the centre; if that exceeds Bx, enlarge Bx and repeat.
 * The k kept are appended in canonical order (j, t). */
static int knn_atom(const double L[9], const double *x, int n, int i, int kk, int extra, int keep_ties,
                    int32_t row0, obuf_t *out) {
    double Li[9];
    if (inverse3(L, Li) == 0.0) return -2;
    double F = frobenius(Li);
    cand_t *best = (cand_t *)malloc(sizeof(cand_t) * (size_t)kk);
    if (!best) return -1;
    int Bx = 1;
    for (;;) {
        int m = 0; /* number kept, best[0..m) ascending */
        for (int j = 0; j < n; ++j) {
            int c[3];
            for (int k = 0; k < 3; ++k) c[k] = -(int)llround(x[3 * j + k] - x[3 * i + k]);
            cand_t cd;
            cd.j = j;
            for (cd.t[0] = c[0] - Bx; cd.t[0] <= c[0] + Bx; ++cd.t[0])
                for (cd.t[1] = c[1] - Bx; cd.t[1] <= c[1] + Bx; ++cd.t[1])
                    for (cd.t[2] = c[2] - Bx; cd.t[2] <= c[2] + Bx; ++cd.t[2]) {
                        if (j == i && cd.t[0] == 0 && cd.t[1] == 0 && cd.t[2] == 0) continue;
                        cd.d2 = canon_d2(L, x + 3 * i, x + 3 * j, cd.t, NULL);
                        if (m == kk && !cand_less(&cd, &best[kk - 1])) continue;
                        int p = (m < kk) ? m++ : kk - 1; /* insertion into the sorted list */
                        while (p > 0 && cand_less(&cd, &best[p - 1])) {
                            best[p] = best[p - 1];
                            --p;
                        }
                        best[p] = cd;
                    }
        }
        if (m < kk) { Bx *= 2; continue; }
        int need = (int)ceil(sqrt(best[kk - 1].d2) * F * (1.0 + 1e-12)) + 1 + extra;
        if (need > Bx) { Bx = need; continue; }
        break;
    }
    if (keep_ties) {
        /* Alg. 2's filter: every image with d2 <= D, the k-th d2 (the box holds them all) */
        double D = best[kk - 1].d2;
        free(best);
        int cap = kk, m = 0;
        cand_t *all = (cand_t *)malloc(sizeof(cand_t) * (size_t)cap);
        if (!all) return -1;
        for (int j = 0; j < n; ++j) {
            int c[3];
            for (int k = 0; k < 3; ++k) c[k] = -(int)llround(x[3 * j + k] - x[3 * i + k]);
            cand_t cd;
            cd.j = j;
            for (cd.t[0] = c[0] - Bx; cd.t[0] <= c[0] + Bx; ++cd.t[0])
                for (cd.t[1] = c[1] - Bx; cd.t[1] <= c[1] + Bx; ++cd.t[1])
                    for (cd.t[2] = c[2] - Bx; cd.t[2] <= c[2] + Bx; ++cd.t[2]) {
                        if (j == i && cd.t[0] == 0 && cd.t[1] == 0 && cd.t[2] == 0) continue;
                        cd.d2 = canon_d2(L, x + 3 * i, x + 3 * j, cd.t, NULL);
                        if (!(cd.d2 <= D)) continue;
                        if (m == cap) {
                            cand_t *na = (cand_t *)realloc(all, sizeof(cand_t) * (size_t)(2 * cap));
                            if (!na) { free(all); return -1; }
                            all = na;
                            cap *= 2;
                        }
                        all[m++] = cd;
                    }
        }
        qsort(all, (size_t)m, sizeof(cand_t), jt_cmp);
        int rc = 0;
        for (int q = 0; q < m && rc == 0; ++q) rc = push(out, row0 + i, row0 + all[q].j, all[q].t, all[q].d2);
        free(all);
        return rc;
    }
    qsort(best, (size_t)kk, sizeof(cand_t), jt_cmp);
    int rc = 0;
    for (int q = 0; q < kk && rc == 0; ++q) rc = push(out, row0 + i, row0 + best[q].j, best[q].t, best[q].d2);
    free(best);
    return rc;
}

/* KNN graph of a batch: exactly k edges per source atom, canonical order (keep_ties 0),
 * or every image at distance <= the k-th one (keep_ties 1, Alg. 2's filter).  Same
 * arguments and return codes as oracle_cutoff, with k in place of the cutoffs. */
int oracle_knn(int B, const int32_t *atom_ptr, const double *lattice, const double *frac, int k,
               int keep_ties, int extra, const int32_t *sources, int64_t n_sources, void *buf) {
    obuf_t *out = (obuf_t *)buf;
    if (k <= 0) return -4;
    int32_t N = atom_ptr[B];
    int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    if (!owner) return -1;
    atom_structure(B, atom_ptr, owner);
    int64_t count = sources ? n_sources : N;
    int rc = 0;
    for (int64_t q = 0; q < count && rc == 0; ++q) {
        int32_t a = sources ? sources[q] : (int32_t)q;
        if (a < 0 || a >= N) { rc = -4; break; }
        int s = owner[a];
        const double *L = lattice + 9 * s;
        const double *x = frac + 3 * (int64_t)atom_ptr[s];
        int n = atom_ptr[s + 1] - atom_ptr[s];
        if (!valid_structure(L, x, n)) { rc = -2; break; }
        rc = knn_atom(L, x, n, a - atom_ptr[s], k, extra, keep_ties, atom_ptr[s], out);
    }
    free(owner);
    return rc;
}

/* ---------------------------------------------------------------- edge vectors */

/* For a fixed edge list: vec = (x_dst - x_src + t) L (canonical FP64 evaluation) and
 * len = sqrt(d2).  Returns 0, or -4 if an edge's endpoints are in different structures. */
int oracle_edge_vectors(int B, const int32_t *atom_ptr, const double *lattice, const double *frac,
                        int64_t E, const int32_t *src, const int32_t *dst, const int32_t *off,
                        double *vec, double *len) {
    int32_t N = atom_ptr[B];
    int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    if (!owner) return -1;
    atom_structure(B, atom_ptr, owner);
    int rc = 0;
    for (int64_t e = 0; e < E; ++e) {
        int s = owner[src[e]];
        if (owner[dst[e]] != s) { rc = -4; break; }
        int t[3] = {off[3 * e], off[3 * e + 1], off[3 * e + 2]};
        double v[3];
        double d2 = canon_d2(lattice + 9 * s, frac + 3 * (int64_t)src[e], frac + 3 * (int64_t)dst[e], t, v);
        vec[3 * e + 0] = v[0];
        vec[3 * e + 1] = v[1];
        vec[3 * e + 2] = v[2];
        len[e] = sqrt(d2);
    }
    free(owner);
    return rc;
}

/* Analytic gradient of a loss through vec and len, edge set held fixed.
 * With g_e = dLoss/dvec_e + dLoss/dlen_e * vec_e / len_e (len_e > 0) and
 * v_e = (x_j - x_i + t) L:
 *   dLoss/dx_j += g_e L^T,  dLoss/dx_i -= g_e L^T,  dLoss/dL += (x_j - x_i + t)^T g_e.
 * grad_vec or grad_len may be NULL (zero).  Outputs are overwritten. */
int oracle_edge_grad(int B, const int32_t *atom_ptr, const double *lattice, const double *frac,
                     int64_t E, const int32_t *src, const int32_t *dst, const int32_t *off,
                     const double *grad_vec, const double *grad_len, double *grad_frac,
                     double *grad_lattice) {
    int32_t N = atom_ptr[B];
    int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    if (!owner) return -1;
    atom_structure(B, atom_ptr, owner);
    memset(grad_frac, 0, sizeof(double) * 3 * (size_t)N);
    memset(grad_lattice, 0, sizeof(double) * 9 * (size_t)B);
    int rc = 0;
    for (int64_t e = 0; e < E; ++e) {
        int s = owner[src[e]];
        if (owner[dst[e]] != s) { rc = -4; break; }
        const double *L = lattice + 9 * s;
        const double *xi = frac + 3 * (int64_t)src[e];
        const double *xj = frac + 3 * (int64_t)dst[e];
        double df[3], v[3];
        for (int c = 0; c < 3; ++c) df[c] = (xj[c] - xi[c]) + (double)off[3 * e + c];
        for (int c = 0; c < 3; ++c) v[c] = df[0] * L[c] + df[1] * L[3 + c] + df[2] * L[6 + c];
        double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double g[3];
        for (int c = 0; c < 3; ++c) {
            g[c] = grad_vec ? grad_vec[3 * e + c] : 0.0;
            if (grad_len && l > 0.0) g[c] += grad_len[e] * v[c] / l;
        }
        for (int k = 0; k < 3; ++k) {
            double h = g[0] * L[3 * k + 0] + g[1] * L[3 * k + 1] + g[2] * L[3 * k + 2];
            grad_frac[3 * (int64_t)dst[e] + k] += h;
            grad_frac[3 * (int64_t)src[e] + k] -= h;
            for (int c = 0; c < 3; ++c) grad_lattice[9 * s + 3 * k + c] += df[k] * g[c];
        }
    }
    free(owner);
    return rc;
}
