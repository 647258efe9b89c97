/*
 * Seeded synthetic crystal batches (inputs only).
 *
 * This file draws lattices, atom counts and fractional coordinates shaped like the
 * structures the paper benchmarks on (Sec. 3: Materials Project structures with at
 * most 64 atoms, batches of 256).  It holds none of the graph method's arithmetic:
 * its only geometry is a minimum-separation rejection test used while placing atoms,
 * written with a deliberately loose image box.  Both the CUDA path and the FP64
 * oracle consume what it writes; neither links it.
 *
 * Random numbers: xoshiro256** seeded through splitmix64 (Blackman & Vigna, 2018),
 * one independent stream per (seed, purpose, structure index).  Uniform doubles use
 * the top 53 bits.  Normals use the Box-Muller transform.
 *
 * Compile with -ffp-contract=off so that x86_64 and aarch64 give the same values up
 * to the libm functions (log, exp, sin, cos) used by the samplers.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------ RNG */

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

/* Independent stream for (seed, purpose, index). */
static void rng_init(rng_t *r, uint64_t seed, uint64_t purpose, uint64_t index) {
    uint64_t x = seed ^ (purpose * 0xD1B54A32D192ED03ull) ^ (index * 0x8CB92BA72F3D8DD7ull);
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static double u01(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static double uab(rng_t *r, double a, double b) { return a + (b - a) * u01(r); }
static int uint_incl(rng_t *r, int a, int b) { /* uniform integer in [a, b] */
    return a + (int)(u01(r) * (double)(b - a + 1));
}
/* log-uniform integer in [a, b]: floor(exp(U[ln a, ln(b+1)))) */
static int loguni_int(rng_t *r, int a, int b) {
    int v = (int)floor(exp(uab(r, log((double)a), log((double)b + 1.0))));
    if (v < a) v = a;
    if (v > b) v = b;
    return v;
}
static double normal(rng_t *r) {
    double u1 = u01(r), u2 = u01(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * PI * u2);
}

/* ------------------------------------------------------------- geometry */

/* Lattice rows from cell parameters: a along x, b in the xy-plane. Returns volume, or
 * -1 when the angles do not close. */
static double lattice_from_params(double a, double b, double c, double al, double be,
                                  double ga, double L[9]) {
    double ca = cos(al), cb = cos(be), cg = cos(ga), sg = sin(ga);
    double cx = cb;
    double cy = (ca - cb * cg) / sg;
    double cz2 = 1.0 - cx * cx - cy * cy;
    if (cz2 <= 1e-12) return -1.0;
    double cz = sqrt(cz2);
    L[0] = a;      L[1] = 0.0;    L[2] = 0.0;
    L[3] = b * cg; L[4] = b * sg; L[5] = 0.0;
    L[6] = c * cx; L[7] = c * cy; L[8] = c * cz;
    return a * b * c * sg * cz;
}

static double inv_frobenius(const double L[9]) {
    double c00 = L[4] * L[8] - L[5] * L[7], c01 = L[5] * L[6] - L[3] * L[8], c02 = L[3] * L[7] - L[4] * L[6];
    double c10 = L[2] * L[7] - L[1] * L[8], c11 = L[0] * L[8] - L[2] * L[6], c12 = L[1] * L[6] - L[0] * L[7];
    double c20 = L[1] * L[5] - L[2] * L[4], c21 = L[2] * L[3] - L[0] * L[5], c22 = L[0] * L[4] - L[1] * L[3];
    double det = L[0] * c00 + L[1] * c01 + L[2] * c02;
    double s = c00 * c00 + c01 * c01 + c02 * c02 + c10 * c10 + c11 * c11 + c12 * c12 + c20 * c20 +
               c21 * c21 + c22 * c22;
    return sqrt(s) / fabs(det);
}

/* Is any periodic image of (x_j - x_i) closer than s?  Loose box: every image within s
 * has |dx_k + t_k| <= s * ||L^-1||_F. */
static int too_close(const double L[9], double F, const double *xi, const double *xj, double s,
                     int skip_zero) {
    double d[3];
    int lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        d[k] = xj[k] - xi[k];
        double R = s * F;
        lo[k] = (int)ceil(-R - d[k]) - 1;
        hi[k] = (int)floor(R - d[k]) + 1;
    }
    double s2 = s * s;
    for (int t0 = lo[0]; t0 <= hi[0]; ++t0)
        for (int t1 = lo[1]; t1 <= hi[1]; ++t1)
            for (int t2 = lo[2]; t2 <= hi[2]; ++t2) {
                if (skip_zero && t0 == 0 && t1 == 0 && t2 == 0) continue;
                double f0 = d[0] + t0, f1 = d[1] + t1, f2 = d[2] + t2;
                double v0 = f0 * L[0] + f1 * L[3] + f2 * L[6];
                double v1 = f0 * L[1] + f1 * L[4] + f2 * L[7];
                double v2 = f0 * L[2] + f1 * L[5] + f2 * L[8];
                if (v0 * v0 + v1 * v1 + v2 * v2 < s2) return 1;
            }
    return 0;
}

/* ------------------------------------------------------------- configs */

#define DEG (PI / 180.0)

typedef struct {
    double len_lo, len_hi, ang_lo, ang_hi, min_sep;
    int skew; /* 1: this cell is a skewed cell (one angle U[25,40] deg, one length U[12,30]) */
} cell_recipe_t;

static void recipe_for(int cfg, rng_t *r, cell_recipe_t *rc) {
    memset(rc, 0, sizeof(*rc));
    switch (cfg) {
    case 1: rc->len_lo = 3.0; rc->len_hi = 8.0; rc->ang_lo = 60; rc->ang_hi = 120; rc->min_sep = 1.0; break;
    case 5: rc->len_lo = 3.0; rc->len_hi = 6.0; rc->ang_lo = 70; rc->ang_hi = 110; rc->min_sep = 0.9; break;
    case 3:
        rc->len_lo = 2.5; rc->len_hi = 12.0; rc->ang_lo = 50; rc->ang_hi = 130; rc->min_sep = 0.9;
        rc->skew = (u01(r) < 0.10);
        break;
    default: /* 2 and 4 */
        rc->len_lo = 2.5; rc->len_hi = 12.0; rc->ang_lo = 50; rc->ang_hi = 130; rc->min_sep = 0.9; break;
    }
}

/* Draw a cell for n atoms; returns 0 on success. */
static int draw_cell(rng_t *r, const cell_recipe_t *rc, int n, double L[9]) {
    for (int attempt = 0; attempt < 100000; ++attempt) {
        double len[3], ang[3];
        for (int k = 0; k < 3; ++k) len[k] = uab(r, rc->len_lo, rc->len_hi);
        for (int k = 0; k < 3; ++k) ang[k] = uab(r, rc->ang_lo, rc->ang_hi);
        if (rc->skew) {
            int ka = uint_incl(r, 0, 2), kl = uint_incl(r, 0, 2);
            ang[ka] = uab(r, 25.0, 40.0);
            len[kl] = uab(r, 12.0, 30.0);
        }
        double V = lattice_from_params(len[0], len[1], len[2], ang[0] * DEG, ang[1] * DEG,
                                       ang[2] * DEG, L);
        if (V <= 0.0 || V < 0.3 * len[0] * len[1] * len[2]) continue;
        if (V < 5.0 * n) { /* isotropic rescale to 5 A^3 per atom */
            double sc = cbrt(5.0 * n / V);
            for (int q = 0; q < 9; ++q) L[q] *= sc;
        }
        double F = inv_frobenius(L);
        double zero[3] = {0, 0, 0};
        if (too_close(L, F, zero, zero, rc->min_sep, 1)) continue; /* short lattice vector */
        return 0;
    }
    return -1;
}

/* Place n atoms with minimum separation; returns 0 on success, -1 after 1000 failed
 * tries for one atom (caller redraws the cell). */
static int place_atoms(rng_t *r, const double L[9], int n, double s, double *x) {
    double F = inv_frobenius(L);
    for (int a = 0; a < n; ++a) {
        int ok = 0;
        for (int tries = 0; tries < 1000 && !ok; ++tries) {
            for (int k = 0; k < 3; ++k) x[3 * a + k] = u01(r);
            ok = 1;
            for (int b = 0; b < a && ok; ++b)
                if (too_close(L, F, x + 3 * b, x + 3 * a, s, 0)) ok = 0;
        }
        if (!ok) return -1;
    }
    return 0;
}

/* Atom counts for cfg; returns total atoms. */
int64_t synth_counts(int cfg, uint64_t seed, int B, int32_t *counts) {
    int64_t tot = 0;
    for (int s = 0; s < B; ++s) {
        rng_t r;
        rng_init(&r, seed, 1, (uint64_t)s);
        int n;
        switch (cfg) {
        case 1: n = uint_incl(&r, 4, 16); break;
        case 2: n = loguni_int(&r, 1, 64); break;
        case 3: {
            double u = u01(&r);
            if (u < 0.70) n = loguni_int(&r, 1, 32);
            else if (u < 0.95) n = loguni_int(&r, 33, 128);
            else n = loguni_int(&r, 129, 400);
            break;
        }
        case 4: n = uint_incl(&r, 8, 64); break;
        case 5: { int m = uint_incl(&r, 6, 14); n = 8 * m * m * m; break; }
        default: return -1;
        }
        counts[s] = n;
        tot += n;
    }
    return tot;
}

/* Fill lattices [B][3][3] (row r = lattice vector r) and fractional coordinates for the
 * structures [s_begin, s_end) of a batch whose atom rows are given by atom_ptr.
 * Returns 0, or -(s+1) if structure s could not be generated. */
int synth_fill(int cfg, uint64_t seed, int s_begin, int s_end, const int32_t *atom_ptr,
               float *lattice, float *frac) {
    for (int s = s_begin; s < s_end; ++s) {
        rng_t r;
        rng_init(&r, seed, 2, (uint64_t)s);
        int n = atom_ptr[s + 1] - atom_ptr[s];
        double L[9];
        if (cfg == 5) {
            /* random 8-atom base cell tiled m x m x m, then Gaussian Cartesian noise */
            int m = 1;
            while (8 * m * m * m < n) ++m;
            if (8 * m * m * m != n) return -(s + 1);
            cell_recipe_t rc;
            recipe_for(cfg, &r, &rc);
            double Lb[9], xb[24];
            int done = 0;
            for (int attempt = 0; attempt < 1000 && !done; ++attempt) {
                if (draw_cell(&r, &rc, 8, Lb)) return -(s + 1);
                if (place_atoms(&r, Lb, 8, rc.min_sep, xb) == 0) done = 1;
            }
            if (!done) return -(s + 1);
            for (int q = 0; q < 9; ++q) L[q] = Lb[q] * m;
            /* inverse of L for Cartesian -> fractional noise */
            double c00 = L[4] * L[8] - L[5] * L[7], c01 = L[5] * L[6] - L[3] * L[8], c02 = L[3] * L[7] - L[4] * L[6];
            double c10 = L[2] * L[7] - L[1] * L[8], c11 = L[0] * L[8] - L[2] * L[6], c12 = L[1] * L[6] - L[0] * L[7];
            double c20 = L[1] * L[5] - L[2] * L[4], c21 = L[2] * L[3] - L[0] * L[5], c22 = L[0] * L[4] - L[1] * L[3];
            double det = L[0] * c00 + L[1] * c01 + L[2] * c02;
            /* row-vector convention: f = v * Linv, Linv[k][c] = cofactor[c][k] / det */
            double Li[9] = {c00 / det, c10 / det, c20 / det, c01 / det, c11 / det, c21 / det,
                            c02 / det, c12 / det, c22 / det};
            int64_t row = atom_ptr[s];
            for (int a0 = 0; a0 < m; ++a0)
                for (int a1 = 0; a1 < m; ++a1)
                    for (int a2 = 0; a2 < m; ++a2)
                        for (int b = 0; b < 8; ++b) {
                            double v[3] = {0.05 * normal(&r), 0.05 * normal(&r), 0.05 * normal(&r)};
                            double f[3];
                            for (int k = 0; k < 3; ++k)
                                f[k] = v[0] * Li[0 * 3 + k] + v[1] * Li[1 * 3 + k] + v[2] * Li[2 * 3 + k];
                            double xf0 = (xb[3 * b + 0] + a0) / m + f[0];
                            double xf1 = (xb[3 * b + 1] + a1) / m + f[1];
                            double xf2 = (xb[3 * b + 2] + a2) / m + f[2];
                            xf0 -= floor(xf0); xf1 -= floor(xf1); xf2 -= floor(xf2);
                            if (xf0 >= 1.0) xf0 = 0.0;
                            if (xf1 >= 1.0) xf1 = 0.0;
                            if (xf2 >= 1.0) xf2 = 0.0;
                            frac[3 * row + 0] = (float)xf0;
                            frac[3 * row + 1] = (float)xf1;
                            frac[3 * row + 2] = (float)xf2;
                            ++row;
                        }
        } else {
            cell_recipe_t rc;
            recipe_for(cfg, &r, &rc);
            double *x = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
            int done = 0;
            for (int attempt = 0; attempt < 1000 && !done; ++attempt) {
                if (draw_cell(&r, &rc, n, L)) break;
                if (place_atoms(&r, L, n, rc.min_sep, x) == 0) done = 1;
            }
            if (!done) { free(x); return -(s + 1); }
            for (int a = 0; a < n; ++a)
                for (int k = 0; k < 3; ++k) {
                    float v = (float)x[3 * a + k];
                    if (v >= 1.0f) v = 0.0f; /* keep [0, 1) after rounding */
                    frac[3 * ((int64_t)atom_ptr[s] + a) + k] = v;
                }
            free(x);
        }
        for (int q = 0; q < 9; ++q) lattice[9 * s + q] = (float)L[q];
    }
    return 0;
}

/* n standard normal draws scaled by sigma, stream (seed, purpose). */
void synth_normal(uint64_t seed, uint64_t purpose, int64_t n, double sigma, float *out) {
    const int64_t chunk = 1 << 16;
    for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        rng_t r;
        rng_init(&r, seed, 100 + purpose, (uint64_t)(c0 / chunk));
        int64_t c1 = c0 + chunk < n ? c0 + chunk : n;
        for (int64_t q = c0; q < c1; ++q) out[q] = (float)(sigma * normal(&r));
    }
}

/* Generative-loop perturbation (workload of the differentiation config): every
 * fractional coordinate moves by N(0, sigma_x) and every lattice is strained,
 * L <- L (I + eps) with eps symmetric, entries N(0, sigma_eps). */
void synth_perturb(uint64_t seed, uint64_t step, int B, const int32_t *atom_ptr, double sigma_x,
                   double sigma_eps, float *lattice, float *frac) {
    for (int s = 0; s < B; ++s) {
        rng_t r;
        rng_init(&r, seed, 1000 + step, (uint64_t)s);
        double e[9];
        for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b) {
                double v = sigma_eps * normal(&r);
                e[3 * a + b] = v;
                e[3 * b + a] = v;
            }
        double L[9], Ln[9];
        for (int q = 0; q < 9; ++q) L[q] = lattice[9 * s + q];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) {
                double acc = L[3 * a + c];
                for (int b = 0; b < 3; ++b) acc += L[3 * a + b] * e[3 * b + c];
                Ln[3 * a + c] = acc;
            }
        for (int q = 0; q < 9; ++q) lattice[9 * s + q] = (float)Ln[q];
        for (int64_t row = atom_ptr[s]; row < atom_ptr[s + 1]; ++row)
            for (int k = 0; k < 3; ++k) frac[3 * row + k] = (float)(frac[3 * row + k] + sigma_x * normal(&r));
    }
}
