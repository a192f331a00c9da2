/*
 * oracle.c -- FP64 CPU oracle of the direct-volume-rendering hot path.
 *
 * TEST INFRASTRUCTURE. This is the plain, slow, direct statement of what the
 * renderer computes, written from the paper (Beckley, "Decentralized Direct
 * Volume Rendering: A Browser-Native GPU Architecture for MRI Digital Twins",
 * arXiv 2605.19737): global min-max normalisation (Sec. 2.2, Eq. 1), the
 * central-difference gradient (Sec. 2.3, Eq. 2), the Hessian and directional
 * curvature (Sec. 2.3, Eq. 3), morphologically modulated opacity (Sec. 2.4,
 * Eq. 4), front-to-back emission-absorption compositing (Sec. 2.4, Eqs. 5-6)
 * and the multi-scale Hessian vesselness stage that Sec. 1 names (read as the
 * bright-vessel measure of Frangi et al., MICCAI 1998). Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg load it. It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Readings of passages the paper leaves open (each one is also a test pin):
 *   - volume index (i,j,k) -> (k*ny + j)*nx + i, x fastest; voxel (i,j,k) has
 *     its centre at ((i+.5)sx, (j+.5)sy, (k+.5)sz) mm; u = p/s - 0.5;
 *   - indices outside [0, N-1] are clamped (clamp-to-edge) in every stencil;
 *   - the field at a sample is the trilinear interpolation of the voxel-wise
 *     intensity, gradient and Hessian (the voxel-wise operators of Sec. 2.3
 *     evaluated at the sample), with u clamped to [0, N-1] per axis;
 *   - kappa = g^T H g / |g|^2 (Eq. 3 with g-hat = g/|g|), 0 when |g| = 0;
 *   - w(kappa) = clamp(1 + gamma kappa / kappa_ref, 0, w_max);
 *   - the sample colour is the transfer-function RGB, optionally lit by a
 *     two-sided Phong headlight rgb (ka + kd d) + ks d^16, d = |g-hat . dir|;
 *   - samples at t_k = t_near + (k + 1/2) dt for every t_k < t_far, no jitter
 *     (the deterministic, non-progressive rendering of Sec. 1 and Sec. 4);
 *   - early termination after the first sample with A >= et_threshold;
 *   - optional step-size opacity correction alpha' = 1 - (1 - alpha)^(dt/dt_ref)
 *     (off unless opacity_ref_step > 0: the paper composites Eqs. 5-6 as printed).
 * Parity pins: closed forms (homogeneous slab, linear ramp, quadratics), a
 * second brute-force field built from hat functions, library eigen-solvers,
 * brute-force convolution, invariants; see tests/test_oracle_*.py. The
 * brick min/max quantisation is this project's own definition (the paper has
 * no bricks); it is pinned by a brute-force conservativeness check.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int tf_mode;   /* 0: 1D over I_norm; 1: 2D over (I_norm, |g|/gmax); 2: 2D over (I_norm, V) */
    int tf_w, tf_h;
    int grad_mod;  /* e_g in {0, 1}: include the |g|/|g|max factor of Eq. 4 */
    int shading;   /* Phong headlight on/off */
    double gamma, kappa_ref, w_max;
    double ka, kd, ks;
    double opacity_scale, et_threshold, step_vox;
    double opacity_ref_step; /* mm; > 0: opacity corrected to this reference step, 0: Eqs. 5-6 as printed */
} or_params;

typedef struct {
    int n[3];
    double s[3];
    const double *In;  /* normalised intensity */
    const double *g;   /* 3 per voxel */
    const double *H;   /* 6 per voxel: xx yy zz xy xz yz */
    const double *V;   /* vesselness or NULL */
    double gmax;
    const uint8_t *brick_empty; /* NULL or one byte per brick */
    int bcells;                 /* cells per brick edge (4, 8 or 16) */
    int nb[3];
    const uint8_t *v_amb; /* NULL or 1 per voxel where V sits on an eigenvalue tie */
} or_vol;

#define OR_FLAG_COUNT 1u
#define OR_FLAG_ET 2u
#define OR_FLAG_BRICK 4u
#define OR_FLAG_VAMB 8u /* a sample interpolated V from a tie voxel (vesselness transfer function) */
#define OR_FLAG_KINK 16u /* a sample within rounding of a non-differentiable point (gradients only) */

static inline int64_t vidx(const int *n, int i, int j, int k) {
    return ((int64_t)k * n[1] + j) * n[0] + i;
}
static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static inline double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------------------------ Eq. 1 */

/* Global extrema of the raw intensities (Sec. 2.2, Eq. 1). */
void or_minmax(const double *raw, int64_t n, double *out2) {
    double lo = raw[0], hi = raw[0];
    for (int64_t i = 1; i < n; ++i) {
        if (raw[i] < lo) lo = raw[i];
        if (raw[i] > hi) hi = raw[i];
    }
    out2[0] = lo;
    out2[1] = hi;
}

/* I_norm = (I_raw - I_min) / (I_max - I_min)  (Sec. 2.2, Eq. 1). */
void or_normalize(const double *raw, int64_t n, double imin, double imax, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = (raw[i] - imin) / (imax - imin);
}

/* ------------------------------------------- Eq. 2 and the Hessian (Sec. 2.3) */

/* Voxel-wise central-difference gradient (Eq. 2, h = one voxel, divided by the
 * spacing in mm) and second/mixed central differences (the Hessian of Sec. 2.3),
 * with clamp-to-edge indices. H is stored xx yy zz xy xz yz. */
void or_voxel_derivatives(const double *In, const int *n, const double *s, double *g, double *H) {
    int64_t total = (int64_t)n[0] * n[1] * n[2];
    (void)total;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                int im = clampi(i - 1, 0, n[0] - 1), ip = clampi(i + 1, 0, n[0] - 1);
                int jm = clampi(j - 1, 0, n[1] - 1), jp = clampi(j + 1, 0, n[1] - 1);
                int km = clampi(k - 1, 0, n[2] - 1), kp = clampi(k + 1, 0, n[2] - 1);
                int64_t v = vidx(n, i, j, k);
                double c = In[v];
                g[3 * v + 0] = (In[vidx(n, ip, j, k)] - In[vidx(n, im, j, k)]) / (2.0 * s[0]);
                g[3 * v + 1] = (In[vidx(n, i, jp, k)] - In[vidx(n, i, jm, k)]) / (2.0 * s[1]);
                g[3 * v + 2] = (In[vidx(n, i, j, kp)] - In[vidx(n, i, j, km)]) / (2.0 * s[2]);
                H[6 * v + 0] = (In[vidx(n, ip, j, k)] - 2.0 * c + In[vidx(n, im, j, k)]) / (s[0] * s[0]);
                H[6 * v + 1] = (In[vidx(n, i, jp, k)] - 2.0 * c + In[vidx(n, i, jm, k)]) / (s[1] * s[1]);
                H[6 * v + 2] = (In[vidx(n, i, j, kp)] - 2.0 * c + In[vidx(n, i, j, km)]) / (s[2] * s[2]);
                H[6 * v + 3] = (In[vidx(n, ip, jp, k)] - In[vidx(n, ip, jm, k)] - In[vidx(n, im, jp, k)] +
                                In[vidx(n, im, jm, k)]) / (4.0 * s[0] * s[1]);
                H[6 * v + 4] = (In[vidx(n, ip, j, kp)] - In[vidx(n, ip, j, km)] - In[vidx(n, im, j, kp)] +
                                In[vidx(n, im, j, km)]) / (4.0 * s[0] * s[2]);
                H[6 * v + 5] = (In[vidx(n, i, jp, kp)] - In[vidx(n, i, jp, km)] - In[vidx(n, i, jm, kp)] +
                                In[vidx(n, i, jm, km)]) / (4.0 * s[1] * s[2]);
            }
}

/* |grad I|_max of Eq. 4: the largest voxel-wise gradient magnitude. */
double or_gmax(const double *g, int64_t nvox) {
    double m = 0.0;
    for (int64_t v = 0; v < nvox; ++v) {
        double a = sqrt(g[3 * v] * g[3 * v] + g[3 * v + 1] * g[3 * v + 1] + g[3 * v + 2] * g[3 * v + 2]);
        if (a > m) m = a;
    }
    return m;
}

/* ------------------------------------------------------- the sample field */

/* Clamped cell coordinates of continuous voxel coordinate u on an axis of n voxels:
 * u_c = clamp(u, 0, n-1); i0 = min(floor(u_c), n-2); f = u_c - i0. */
static inline void cell_of(double u, int n, int *i0, double *f) {
    double uc = clampd(u, 0.0, (double)(n - 1));
    int i = (int)floor(uc);
    if (i > n - 2) i = n - 2;
    *i0 = i;
    *f = uc - (double)i;
}

/* Trilinear interpolation of I_norm, the voxel gradient, the voxel Hessian and
 * (if present) V at world point p. out = I, gx gy gz, Hxx Hyy Hzz Hxy Hxz Hyz, V. */
static void field_at(const or_vol *v, const double p[3], double out[11]) {
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) cell_of(p[a] / v->s[a] - 0.5, v->n[a], &i0[a], &f[a]);
    for (int q = 0; q < 11; ++q) out[q] = 0.0;
    for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        int64_t id = vidx(v->n, i0[0] + dx, i0[1] + dy, i0[2] + dz);
        out[0] += w * v->In[id];
        for (int q = 0; q < 3; ++q) out[1 + q] += w * v->g[3 * id + q];
        for (int q = 0; q < 6; ++q) out[4 + q] += w * v->H[6 * id + q];
        if (v->V) out[10] += w * v->V[id];
    }
}

void or_field_at(const double *In, const double *g, const double *H, const double *V, const int *n,
                 const double *s, const double *p, double *out11) {
    or_vol v;
    memset(&v, 0, sizeof v);
    for (int a = 0; a < 3; ++a) {
        v.n[a] = n[a];
        v.s[a] = s[a];
    }
    v.In = In;
    v.g = g;
    v.H = H;
    v.V = V;
    field_at(&v, p, out11);
}

/* Second, independent statement of the same field for pinning: the
 * clamp-extended piecewise-linear intensity F(u) = sum_v I_n[v] tent(u-v)
 * summed over ALL voxels, and its derivatives taken as central differences of F
 * with h = one voxel around the clamped coordinate. out = I, g3, H6. */
static double brute_F(const double *In, const int *n, double ux, double uy, double uz) {
    ux = clampd(ux, 0.0, n[0] - 1.0);
    uy = clampd(uy, 0.0, n[1] - 1.0);
    uz = clampd(uz, 0.0, n[2] - 1.0);
    double acc = 0.0;
    for (int k = 0; k < n[2]; ++k) {
        double wz = 1.0 - fabs(uz - k);
        if (wz <= 0.0) continue;
        for (int j = 0; j < n[1]; ++j) {
            double wy = 1.0 - fabs(uy - j);
            if (wy <= 0.0) continue;
            for (int i = 0; i < n[0]; ++i) {
                double wx = 1.0 - fabs(ux - i);
                if (wx <= 0.0) continue;
                acc += wx * wy * wz * In[vidx(n, i, j, k)];
            }
        }
    }
    return acc;
}

void or_field_brute(const double *In, const int *n, const double *s, const double *p, double *out10) {
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = clampd(p[a] / s[a] - 0.5, 0.0, n[a] - 1.0);
#define F(dx, dy, dz) brute_F(In, n, u[0] + (dx), u[1] + (dy), u[2] + (dz))
    double c = F(0, 0, 0);
    out10[0] = c;
    out10[1] = (F(1, 0, 0) - F(-1, 0, 0)) / (2.0 * s[0]);
    out10[2] = (F(0, 1, 0) - F(0, -1, 0)) / (2.0 * s[1]);
    out10[3] = (F(0, 0, 1) - F(0, 0, -1)) / (2.0 * s[2]);
    out10[4] = (F(1, 0, 0) - 2.0 * c + F(-1, 0, 0)) / (s[0] * s[0]);
    out10[5] = (F(0, 1, 0) - 2.0 * c + F(0, -1, 0)) / (s[1] * s[1]);
    out10[6] = (F(0, 0, 1) - 2.0 * c + F(0, 0, -1)) / (s[2] * s[2]);
    out10[7] = (F(1, 1, 0) - F(1, -1, 0) - F(-1, 1, 0) + F(-1, -1, 0)) / (4.0 * s[0] * s[1]);
    out10[8] = (F(1, 0, 1) - F(1, 0, -1) - F(-1, 0, 1) + F(-1, 0, -1)) / (4.0 * s[0] * s[2]);
    out10[9] = (F(0, 1, 1) - F(0, 1, -1) - F(0, -1, 1) + F(0, -1, -1)) / (4.0 * s[1] * s[2]);
#undef F
}

/* Directional curvature kappa = g-hat^T H g-hat (Eq. 3) and, for tests only, the
 * isosurface mean curvature (tr H - kappa) / (2 |g|). out2 = kappa, kappa_mean. */
void or_curvature(const double *g, const double *H, double *out2) {
    double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    if (gg == 0.0) {
        out2[0] = 0.0;
        out2[1] = 0.0;
        return;
    }
    double Hg0 = H[0] * g[0] + H[3] * g[1] + H[4] * g[2];
    double Hg1 = H[3] * g[0] + H[1] * g[1] + H[5] * g[2];
    double Hg2 = H[4] * g[0] + H[5] * g[1] + H[2] * g[2];
    double kappa = (g[0] * Hg0 + g[1] * Hg1 + g[2] * Hg2) / gg;
    out2[0] = kappa;
    out2[1] = (H[0] + H[1] + H[2] - kappa) / (2.0 * sqrt(gg));
}

/* ------------------------------------------------------ transfer function */

/* Piecewise-linear lookup: x in I_norm over w entries, y over h entries (h = 1: 1D). */
static void tf_sample(const double *tf, int w, int h, double x, double y, double rgba[4]) {
    double xs = clampd(x, 0.0, 1.0) * (w - 1);
    int j = (int)floor(xs);
    if (j > w - 2) j = w - 2;
    double t = xs - j;
    if (h == 1) {
        for (int c = 0; c < 4; ++c) rgba[c] = (1.0 - t) * tf[4 * j + c] + t * tf[4 * (j + 1) + c];
        return;
    }
    double ys = clampd(y, 0.0, 1.0) * (h - 1);
    int k = (int)floor(ys);
    if (k > h - 2) k = h - 2;
    double q = ys - k;
    for (int c = 0; c < 4; ++c) {
        double lo = (1.0 - t) * tf[4 * (k * w + j) + c] + t * tf[4 * (k * w + j + 1) + c];
        double hi = (1.0 - t) * tf[4 * ((k + 1) * w + j) + c] + t * tf[4 * ((k + 1) * w + j + 1) + c];
        rgba[c] = (1.0 - q) * lo + q * hi;
    }
}

void or_tf_sample(const double *tf, int w, int h, double x, double y, double *rgba) { tf_sample(tf, w, h, x, y, rgba); }

/* --------------------------------------------------- per-sample optics */

/* Distance of x to the nearest integer. */
static double frac_dist(double x) { return fabs(x - floor(x + 0.5)); }

/* Largest magnitudes over the 8 corners of the cell that field_at interpolates at p:
 * intensity M, gradient norm G, Hessian entry Hm, second channel Vm. They bound the
 * float32 rounding of the interpolated values (kink flags below). */
static void corner_maxima(const or_vol *v, const double p[3], double *M, double *G, double *Hm, double *Vm) {
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) cell_of(p[a] / v->s[a] - 0.5, v->n[a], &i0[a], &f[a]);
    *M = *G = *Hm = *Vm = 0.0;
    for (int c = 0; c < 8; ++c) {
        int64_t id = vidx(v->n, i0[0] + (c & 1), i0[1] + ((c >> 1) & 1), i0[2] + ((c >> 2) & 1));
        const double *g = v->g + 3 * id, *H = v->H + 6 * id;
        *M = fmax(*M, fabs(v->In[id]));
        *G = fmax(*G, sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
        for (int q = 0; q < 6; ++q) *Hm = fmax(*Hm, fabs(H[q]));
        if (v->V) *Vm = fmax(*Vm, fabs(v->V[id]));
    }
}

/* Does the piecewise-linear table bend at knot jn along the intensity axis in row k,
 * i.e. do the slopes on its two sides differ in some channel? Outside [0, w-1] the
 * lookup is clamped (flat), so an end knot bends where the slope next to it is
 * non-zero. Along the second axis likewise with the roles swapped (column j). */
static int tf_bends_x(const double *tf, int w, int k, int jn) {
    const double *r = tf + 4 * (size_t)k * w;
    for (int c = 0; c < 4; ++c) {
        double left = jn > 0 ? r[4 * jn + c] - r[4 * (jn - 1) + c] : 0.0;
        double right = jn < w - 1 ? r[4 * (jn + 1) + c] - r[4 * jn + c] : 0.0;
        if (left != right) return 1;
    }
    return 0;
}

static int tf_bends_y(const double *tf, int w, int h, int j, int kn) {
    for (int c = 0; c < 4; ++c) {
        double below = kn > 0 ? tf[4 * (kn * w + j) + c] - tf[4 * ((kn - 1) * w + j) + c] : 0.0;
        double above = kn < h - 1 ? tf[4 * ((kn + 1) * w + j) + c] - tf[4 * (kn * w + j) + c] : 0.0;
        if (below != above) return 1;
    }
    return 0;
}

/* Opacity (Eq. 4) and colour of one sample at world point p seen along unit dir.
 * kink (may be NULL) is set to 1 when the sample sits within float32 rounding of a
 * point where the opacity or colour is not differentiable in the voxels: a knot or
 * end of the transfer function where the table bends, the clamps of w(kappa), of
 * |grad I|/gmax or of alpha at 1 (each window a worst-case float32 rounding bound
 * of that quantity at this sample), or a vanishing gradient (|grad I| < 1e-4 gmax)
 * where kappa and the shading normal are undefined. There a float32 evaluation may
 * take the other one-sided derivative. */
static void sample_optics_k(const or_vol *v, const or_params *P, const double *tf, const double p[3],
                            const double dir[3], double *alpha, double col[3], int *kink) {
    double fld[11];
    field_at(v, p, fld);
    const double *g = fld + 1, *H = fld + 4;
    double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    double gmag = sqrt(gg);
    double kappa = 0.0, ghat[3] = {0.0, 0.0, 0.0};
    if (gg > 0.0) {
        double km[2];
        or_curvature(g, H, km);
        kappa = km[0];
        for (int a = 0; a < 3; ++a) ghat[a] = g[a] / gmag;
    }
    double gn = v->gmax > 0.0 ? gmag / v->gmax : 0.0;
    double y = 0.0;
    if (P->tf_mode == 1) y = gn;
    if (P->tf_mode == 2) y = fld[10];
    double rgba[4];
    tf_sample(tf, P->tf_w, P->tf_h, fld[0], y, rgba);
    double mg = P->grad_mod ? (gn < 1.0 ? gn : 1.0) : 1.0;
    double winner = 1.0 + P->gamma * kappa / P->kappa_ref;
    double w = clampd(winner, 0.0, P->w_max);
    double raw = P->opacity_scale * rgba[3] * mg * w;
    *alpha = clampd(raw, 0.0, 1.0);
    if (kink) {
        /* Windows: how far float32 evaluation of the same sample can move each
         * quantity, from worst-case rounding bounds (u = 2^-24 per IEEE operation;
         * the interpolated values are sums of 8 products with rounded trilinear
         * weights, the voxel-wise derivatives are rounded differences of the same
         * float32 voxels, the sample position is good to 2e-7 voxel: 32.32 fixed
         * point over up to ~1600 samples per ray). A knot counts
         * only where the table actually bends; exact zeros and ends (I = 0 or 1) are
         * exact in float32 too and are not flagged. */
        const double u = 5.9604644775390625e-8;
        double M, G, Hm, Vm;
        corner_maxima(v, p, &M, &G, &Hm, &Vm);
        const double smin = fmin(v->s[0], fmin(v->s[1], v->s[2]));
        const int w_ = P->tf_w, h_ = P->tf_h;
        const double xs = clampd(fld[0], 0.0, 1.0) * (w_ - 1);
        const double wx = (w_ - 1) * u * (12.0 * fabs(fld[0]) + 4.0 * M);
        double ys = 0.0, wy = 0.0;
        if (h_ > 1) {
            ys = clampd(y, 0.0, 1.0) * (h_ - 1);
            wy = P->tf_mode == 1 ? (h_ - 1) * (40.0 * u * (v->gmax > 0.0 ? G / v->gmax : 0.0) + 3.0 * u * gn)
                                 : (h_ - 1) * 10.0 * u * Vm;
        }
        const int jl = (int)fmin(floor(xs), w_ - 2), kl = h_ > 1 ? (int)fmin(floor(ys), h_ - 2) : 0;
        int k = 0;
        if (fld[0] != 0.0 && fld[0] != 1.0 && frac_dist(xs) < wx) {
            const int jn = (int)floor(xs + 0.5);
            k |= tf_bends_x(tf, w_, kl, jn) || (h_ > 1 && tf_bends_x(tf, w_, kl + 1, jn));
        }
        if (h_ > 1 && y != 0.0 && y != 1.0 && frac_dist(ys) < wy) {
            const int kn = (int)floor(ys + 0.5);
            k |= tf_bends_y(tf, w_, h_, jl, kn) || tf_bends_y(tf, w_, h_, jl + 1, kn);
        }
        /* |g|/gmax; kappa (its voxel Hessians are rounded second differences, and the
         * gradient's rounding enters through dkappa/dg = 2 (H g - kappa g) / |g|^2) */
        const double dgn = 40.0 * u * (v->gmax > 0.0 ? G / v->gmax : 0.0) + 3.0 * u * gn;
        double dwin = 0.0;
        if (P->gamma != 0.0 && gg > 0.0) {
            const double dk = 24.0 * u * M / (smin * smin) + 42.0 * u * Hm +
                              50.0 * u * (3.0 * Hm + fabs(kappa)) * G / gmag + 8.0 * u * fabs(kappa);
            dwin = fabs(P->gamma / P->kappa_ref) * dk + 2.0 * u;
            k |= fabs(winner) < dwin || fabs(winner - P->w_max) < dwin;
        }
        if (P->grad_mod) k |= fabs(gn - 1.0) < dgn;
        { /* alpha's clamp at 1: raw moves with the looked-up opacity and both factors */
            const double *T = tf + 4 * (size_t)kl * w_;
            double sx = fabs(T[4 * (jl + 1) + 3] - T[4 * jl + 3]), sy = 0.0;
            if (h_ > 1) {
                const double *T1 = T + 4 * (size_t)w_;
                sx = fmax(sx, fabs(T1[4 * (jl + 1) + 3] - T1[4 * jl + 3]));
                sy = fmax(fabs(T1[4 * jl + 3] - T[4 * jl + 3]), fabs(T1[4 * (jl + 1) + 3] - T[4 * (jl + 1) + 3]));
            }
            const double dca = sx * wx + sy * wy + 4.0 * u * fabs(rgba[3]);
            const double dmg = P->grad_mod ? dgn : 0.0;
            const double draw = P->opacity_scale * (dca * mg * w + fabs(rgba[3]) * (dmg * w + mg * dwin)) +
                                4.0 * u * fabs(raw);
            k |= fabs(raw - 1.0) < draw;
        }
        /* a vanishing gradient: kappa and the shading normal are undefined at g = 0 and
         * ill-conditioned next to it (a conditioning guard, not a rounding bound) */
        if (P->shading || P->gamma != 0.0 || P->grad_mod || P->tf_mode == 1) k |= gn > 0.0 && gn < 1e-4;
        *kink = k;
    }
    if (P->opacity_ref_step > 0.0) { /* alpha' = 1 - (1 - alpha)^(dt / dt_ref) */
        double dt = P->step_vox * fmin(v->s[0], fmin(v->s[1], v->s[2]));
        *alpha = 1.0 - pow(1.0 - *alpha, dt / P->opacity_ref_step);
    }
    if (P->shading) {
        double d = fabs(ghat[0] * dir[0] + ghat[1] * dir[1] + ghat[2] * dir[2]);
        double d2 = d * d, d4 = d2 * d2, d8 = d4 * d4, d16 = d8 * d8;
        for (int c = 0; c < 3; ++c) col[c] = rgba[c] * (P->ka + P->kd * d) + P->ks * d16;
    } else {
        for (int c = 0; c < 3; ++c) col[c] = rgba[c];
    }
}

static void sample_optics(const or_vol *v, const or_params *P, const double *tf, const double p[3],
                          const double dir[3], double *alpha, double col[3]) {
    sample_optics_k(v, P, tf, p, dir, alpha, col, NULL);
}

/* ------------------------------------------------------------ ray setup */

/* Ray through the centre of pixel (i, j) (row 0 at the top): direction
 * normalize(fwd + a right + b up), a = 2(i+1/2)/W - 1, b = 1 - 2(j+1/2)/H; slab
 * intersection with the box [0, N s]; t_near = max(t0, 0). Returns 0 on a miss. */
static int ray_setup(const or_vol *v, const double *cam, int W, int H, int i, int j, double o[3], double d[3],
                     double *tn, double *tf) {
    double a = 2.0 * (i + 0.5) / W - 1.0;
    double b = 1.0 - 2.0 * (j + 0.5) / H;
    for (int q = 0; q < 3; ++q) {
        o[q] = cam[q];
        d[q] = cam[3 + q] + a * cam[6 + q] + b * cam[9 + q];
    }
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int q = 0; q < 3; ++q) d[q] = d[q] / len;
    double t0 = -INFINITY, t1 = INFINITY;
    for (int q = 0; q < 3; ++q) {
        double hi = v->n[q] * v->s[q];
        if (d[q] == 0.0) {
            if (o[q] < 0.0 || o[q] > hi) return 0;
            continue;
        }
        double ta = (0.0 - o[q]) / d[q], tb = (hi - o[q]) / d[q];
        double lo_t = ta < tb ? ta : tb, hi_t = ta < tb ? tb : ta;
        if (lo_t > t0) t0 = lo_t;
        if (hi_t < t1) t1 = hi_t;
    }
    *tn = t0 > 0.0 ? t0 : 0.0;
    *tf = t1;
    return *tn < *tf;
}

/* Brick of the cell that holds a sample: floor(i0 / B) per axis, B = bcells. */
static inline int64_t brick_of(const or_vol *v, const double p[3], int *near_face) {
    int b[3];
    *near_face = 0;
    for (int a = 0; a < 3; ++a) {
        double uc = clampd(p[a] / v->s[a] - 0.5, 0.0, (double)(v->n[a] - 1));
        int i0;
        double f;
        cell_of(p[a] / v->s[a] - 0.5, v->n[a], &i0, &f);
        b[a] = i0 / v->bcells;
        double m = floor(uc / v->bcells + 0.5) * v->bcells; /* nearest multiple of B */
        if (fabs(uc - m) < 1e-4 && m > 0.0 && m <= v->n[a] - 2) *near_face = 1;
    }
    return ((int64_t)b[2] * v->nb[1] + b[1]) * v->nb[0] + b[0];
}

/* Front-to-back emission-absorption march of one ray (Eqs. 5-6), no shortcuts:
 * every sample t_k < t_far is evaluated in order until the first k with
 * A >= et. n_adjust (-1, 0, +1) drops or adds the last sample (alternative
 * outcomes of an ambiguous sample count). */
static void march(const or_vol *v, const or_params *P, const double *tf, const double o[3], const double d[3],
                  double tn, double tfar, double et, int n_adjust, double rgba[4], int64_t *dense,
                  int64_t *evaluated, unsigned *flags) {
    double dt = P->step_vox * fmin(v->s[0], fmin(v->s[1], v->s[2]));
    int64_t ns = 0;
    while (tn + (ns + 0.5) * dt < tfar) ++ns;
    if (flags) {
        if (ns > 0 && fabs(tfar - (tn + (ns - 0.5) * dt)) < 1e-6 * dt) *flags |= OR_FLAG_COUNT;
        if (fabs((tn + (ns + 0.5) * dt) - tfar) < 1e-6 * dt) *flags |= OR_FLAG_COUNT;
    }
    ns += n_adjust;
    double C[3] = {0.0, 0.0, 0.0}, A = 0.0;
    int64_t nd = 0, ne = 0;
    for (int64_t k = 0; k < ns; ++k) {
        double t = tn + (k + 0.5) * dt;
        double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        ++nd;
        if (v->brick_empty) {
            int near_face;
            int64_t bi = brick_of(v, p, &near_face);
            if (!v->brick_empty[bi]) ++ne;
            if (near_face && flags) *flags |= OR_FLAG_BRICK;
        } else {
            ++ne;
        }
        double alpha, c[3];
        int kink = 0;
        sample_optics_k(v, P, tf, p, d, &alpha, c, flags ? &kink : NULL);
        if (kink) *flags |= OR_FLAG_KINK;
        if (flags && v->v_amb && P->tf_mode == 2) {
            int i0[3];
            double f[3];
            for (int a = 0; a < 3; ++a) cell_of(p[a] / v->s[a] - 0.5, v->n[a], &i0[a], &f[a]);
            for (int cc = 0; cc < 8; ++cc) {
                int dx = cc & 1, dy = (cc >> 1) & 1, dz = (cc >> 2) & 1;
                double wt = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                if (wt > 0.0 && v->v_amb[vidx(v->n, i0[0] + dx, i0[1] + dy, i0[2] + dz)]) *flags |= OR_FLAG_VAMB;
            }
        }
        for (int q = 0; q < 3; ++q) C[q] = C[q] + (1.0 - A) * c[q] * alpha;  /* Eq. 5 */
        A = A + (1.0 - A) * alpha;                                          /* Eq. 6 */
        if (flags && fabs(A - P->et_threshold) < 1e-5) *flags |= OR_FLAG_ET;
        if (A >= et) break;
    }
    rgba[0] = C[0];
    rgba[1] = C[1];
    rgba[2] = C[2];
    rgba[3] = A;
    if (dense) *dense = nd;
    if (evaluated) *evaluated = ne;
}

static void make_vol(or_vol *v, const double *In, const double *V, const int *n, const double *s) {
    memset(v, 0, sizeof *v);
    v->bcells = 8;
    for (int a = 0; a < 3; ++a) {
        v->n[a] = n[a];
        v->s[a] = s[a];
        v->nb[a] = (n[a] - 1 + 7) / 8;
    }
    v->In = In;
    v->V = V;
}

/* Render n_cams images of W x H premultiplied RGBA (row 0 = top, background 0).
 *   In: normalised volume; V: vesselness or NULL; v_amb: NULL or the tie mask of
 *   or_frangi (rays that interpolate V from a tie voxel get OR_FLAG_VAMB);
 *   gmax <= 0: computed here;
 *   brick_empty: NULL or the empty-brick flags of bricks of brick_cells^3 cells
 *     (only the evaluated counter and the brick-face tie flag use them);
 *   rgba_lo / rgba_hi (nullable): the outcomes with et -/+ 1e-5 and with one
 *     sample less / more when the count is ambiguous -- every ray whose flags are
 *     non-zero has these alternatives filled, the rest are copies of rgba;
 *   pix_stride > 1 renders only pixels with i % stride == 0 and j % stride == 0.
 * Returns the number of OpenMP threads used. */
int or_render(const double *In, const double *V, const uint8_t *v_amb, const int *n, const double *s,
              const or_params *P, const float *tf32, const uint8_t *brick_empty, int brick_cells, double gmax_in,
              const float *cams, int n_cams,
              int W, int H, int pix_stride, double *rgba, double *rgba_lo, double *rgba_hi, int64_t *dense,
              int64_t *evaluated, uint8_t *flags_out) {
    or_vol v;
    make_vol(&v, In, V, n, s);
    v.bcells = brick_cells;
    for (int a = 0; a < 3; ++a) v.nb[a] = (n[a] - 1 + brick_cells - 1) / brick_cells;
    int64_t nvox = (int64_t)n[0] * n[1] * n[2];
    double *g = (double *)malloc(sizeof(double) * 3 * nvox);
    double *Hs = (double *)malloc(sizeof(double) * 6 * nvox);
    or_voxel_derivatives(In, n, s, g, Hs);
    v.g = g;
    v.H = Hs;
    v.gmax = gmax_in > 0.0 ? gmax_in : or_gmax(g, nvox);
    v.brick_empty = brick_empty;
    v.v_amb = v_amb;
    int ntf = P->tf_w * P->tf_h * 4;
    double *tf = (double *)malloc(sizeof(double) * ntf);
    for (int q = 0; q < ntf; ++q) tf[q] = (double)tf32[q];
    int stride = pix_stride > 1 ? pix_stride : 1;
    int threads = 1;
#ifdef _OPENMP
    threads = omp_get_max_threads();
#endif
    for (int ci = 0; ci < n_cams; ++ci) {
        double cam[12];
        for (int q = 0; q < 12; ++q) cam[q] = (double)cams[12 * ci + q];
#pragma omp parallel for schedule(dynamic, 1)
        for (int j = 0; j < H; ++j) {
            if (j % stride) continue;
            for (int i = 0; i < W; i += stride) {
                int64_t pix = ((int64_t)ci * H + j) * W + i;
                double o[3], d[3], tn, tfar, out[4] = {0, 0, 0, 0};
                int64_t nd = 0, ne = 0;
                unsigned fl = 0;
                int hit = ray_setup(&v, cam, W, H, i, j, o, d, &tn, &tfar);
                if (hit) march(&v, P, tf, o, d, tn, tfar, P->et_threshold, 0, out, &nd, &ne, &fl);
                for (int q = 0; q < 4; ++q) rgba[4 * pix + q] = out[q];
                if (dense) dense[pix] = nd;
                if (evaluated) evaluated[pix] = ne;
                if (flags_out) flags_out[pix] = (uint8_t)fl;
                if (rgba_lo || rgba_hi) {
                    double lo[4], hi[4];
                    for (int q = 0; q < 4; ++q) lo[q] = hi[q] = out[q];
                    if (hit && (fl & (OR_FLAG_ET | OR_FLAG_COUNT))) {
                        int adj_lo = 0, adj_hi = 0;
                        if (fl & OR_FLAG_COUNT) {
                            adj_lo = -1;
                            adj_hi = +1;
                        }
                        march(&v, P, tf, o, d, tn, tfar, P->et_threshold - 1e-5, adj_lo, lo, NULL, NULL, NULL);
                        march(&v, P, tf, o, d, tn, tfar, P->et_threshold + 1e-5, adj_hi, hi, NULL, NULL, NULL);
                    }
                    for (int q = 0; q < 4; ++q) {
                        if (rgba_lo) rgba_lo[4 * pix + q] = lo[q];
                        if (rgba_hi) rgba_hi[4 * pix + q] = hi[q];
                    }
                }
            }
        }
    }
    free(tf);
    free(g);
    free(Hs);
    return threads;
}

/* Brute-force render for pinning (small volumes only): the field is the hat-function
 * sum with finite-difference derivatives (or_field_brute); every sample before t_far
 * is composited without early termination while the per-sample opacity and colour
 * are kept, and early termination is applied afterwards by cutting the list at the
 * first sample where the running A reaches et. Tests compare it with or_render. */
int or_render_brute(const double *In, const int *n, const double *s, const or_params *P, const float *tf32,
                    double gmax, const float *cams, int n_cams, int W, int H, double *rgba) {
    or_vol v;
    make_vol(&v, In, NULL, n, s);
    v.gmax = gmax;
    int ntf = P->tf_w * P->tf_h * 4;
    double *tf = (double *)malloc(sizeof(double) * ntf);
    for (int q = 0; q < ntf; ++q) tf[q] = (double)tf32[q];
    double dt = P->step_vox * fmin(s[0], fmin(s[1], s[2]));
    for (int ci = 0; ci < n_cams; ++ci) {
        double cam[12];
        for (int q = 0; q < 12; ++q) cam[q] = (double)cams[12 * ci + q];
        for (int j = 0; j < H; ++j)
            for (int i = 0; i < W; ++i) {
                int64_t pix = ((int64_t)ci * H + j) * W + i;
                double o[3], d[3], tn, tfar;
                double *out = rgba + 4 * pix;
                out[0] = out[1] = out[2] = out[3] = 0.0;
                if (!ray_setup(&v, cam, W, H, i, j, o, d, &tn, &tfar)) continue;
                int64_t cap = 16, ns = 0;
                double *al = (double *)malloc(sizeof(double) * cap), *cl = (double *)malloc(sizeof(double) * 3 * cap);
                for (int64_t k = 0; tn + (k + 0.5) * dt < tfar; ++k) {
                    double t = tn + (k + 0.5) * dt;
                    double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
                    double f10[10];
                    or_field_brute(In, n, s, p, f10);
                    double *g = f10 + 1, *Hh = f10 + 4;
                    double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2], gm = sqrt(gg);
                    double kappa = 0.0, gh[3] = {0, 0, 0};
                    if (gg > 0.0) {
                        double km[2];
                        or_curvature(g, Hh, km);
                        kappa = km[0];
                        for (int a = 0; a < 3; ++a) gh[a] = g[a] / gm;
                    }
                    double gn = gmax > 0.0 ? gm / gmax : 0.0, c4[4];
                    tf_sample(tf, P->tf_w, P->tf_h, f10[0], P->tf_mode == 1 ? gn : 0.0, c4);
                    double mg = P->grad_mod ? fmin(gn, 1.0) : 1.0;
                    double w = clampd(1.0 + P->gamma * kappa / P->kappa_ref, 0.0, P->w_max);
                    if (ns == cap) {
                        cap *= 2;
                        al = (double *)realloc(al, sizeof(double) * cap);
                        cl = (double *)realloc(cl, sizeof(double) * 3 * cap);
                    }
                    al[ns] = clampd(P->opacity_scale * c4[3] * mg * w, 0.0, 1.0);
                    if (P->opacity_ref_step > 0.0) al[ns] = 1.0 - pow(1.0 - al[ns], dt / P->opacity_ref_step);
                    double dd = fabs(gh[0] * d[0] + gh[1] * d[1] + gh[2] * d[2]);
                    for (int c = 0; c < 3; ++c)
                        cl[3 * ns + c] = P->shading ? c4[c] * (P->ka + P->kd * dd) + P->ks * pow(dd, 16.0) : c4[c];
                    ++ns;
                }
                double A = 0.0, C[3] = {0, 0, 0};
                for (int64_t k = 0; k < ns; ++k) {
                    for (int c = 0; c < 3; ++c) C[c] += (1.0 - A) * cl[3 * k + c] * al[k];
                    A += (1.0 - A) * al[k];
                    if (A >= P->et_threshold) break;
                }
                out[0] = C[0];
                out[1] = C[1];
                out[2] = C[2];
                out[3] = A;
                free(al);
                free(cl);
            }
    }
    free(tf);
    return 1;
}

/* -------------------------------------- brick min/max grid and skipping */

/* Per brick of B^3 cells (B = 4, 8 or 16), the min and max of the normalised
 * intensity over its corner voxels [Bb, min(Bb+B, N-1)] per axis, quantised to 16 bits as
 * qlo = floor(min * 65535), qhi = ceil(max * 65535). The normalisation and the
 * quantisation are taken in IEEE float32 with round-to-nearest, one operation at
 * a time (d = x - imin; r = d / (imax - imin); r * 65535), because these floats
 * decide integers that must match the kernel's bit for bit; codes are clamped to
 * [0, 65535]. raw holds float32 or uint16 values; grid is [nbz][nby][nbx][2]. */
void or_brick_minmax_q(const float *raw, const int *n, float imin, float imax, int B, uint16_t *grid) {
    int nb[3];
    for (int a = 0; a < 3; ++a) nb[a] = (n[a] - 1 + B - 1) / B;
    volatile float range = imax - imin;
    for (int bz = 0; bz < nb[2]; ++bz)
        for (int by = 0; by < nb[1]; ++by)
            for (int bx = 0; bx < nb[0]; ++bx) {
                float lo = INFINITY, hi = -INFINITY;
                for (int k = B * bz; k <= B * bz + B && k < n[2]; ++k)
                    for (int j = B * by; j <= B * by + B && j < n[1]; ++j)
                        for (int i = B * bx; i <= B * bx + B && i < n[0]; ++i) {
                            volatile float d = raw[vidx(n, i, j, k)] - imin;
                            volatile float r = d / range;
                            if (r < lo) lo = r;
                            if (r > hi) hi = r;
                        }
                volatile float ql = lo * 65535.0f, qh = hi * 65535.0f;
                int64_t b = ((int64_t)bz * nb[1] + by) * nb[0] + bx;
                grid[2 * b + 0] = (uint16_t)fminf(fmaxf(floorf(ql), 0.0f), 65535.0f);
                grid[2 * b + 1] = (uint16_t)fminf(fmaxf(ceilf(qh), 0.0f), 65535.0f);
            }
}

/* A brick is empty when every transfer-function opacity entry it can reach is
 * exactly zero: intensity entries j in [floor(qlo*255/65535) - 1,
 * ceil(qhi*255/65535) + 1] (clamped to [0, w-1]; one entry of margin on each side
 * absorbs float rounding of the interpolated sample), every row of a 2D table.
 * Integer arithmetic only. Implements the transfer-function clipping of Sec. 2.2
 * as empty-space skipping. */
void or_classify(const uint16_t *grid, int64_t nbricks, const float *tf, int w, int h, uint8_t *empty) {
    for (int64_t b = 0; b < nbricks; ++b) {
        int64_t ql = grid[2 * b], qh = grid[2 * b + 1];
        int64_t jl = (ql * (w - 1)) / 65535 - 1;
        int64_t jh = (qh * (w - 1) + 65534) / 65535 + 1;
        if (jl < 0) jl = 0;
        if (jh > w - 1) jh = w - 1;
        int e = 1;
        for (int r = 0; r < h && e; ++r)
            for (int64_t j = jl; j <= jh; ++j)
                if (tf[4 * ((int64_t)r * w + j) + 3] != 0.0f) {
                    e = 0;
                    break;
                }
        empty[b] = (uint8_t)e;
    }
}

/* --------------------------------------- multi-scale Hessian vesselness */

/* Separable Gaussian smoothing with sampled, normalised weights exp(-x^2/2 sigma^2)
 * on [-R, R], R = ceil(4 sigma) voxels, clamp-to-edge, along x then y then z. */
void or_gauss_smooth(const double *in, const int *n, double sigma, double *out) {
    int R = (int)ceil(4.0 * sigma);
    double *w = (double *)malloc(sizeof(double) * (2 * R + 1)), sum = 0.0;
    for (int i = -R; i <= R; ++i) sum += (w[i + R] = exp(-(double)i * i / (2.0 * sigma * sigma)));
    for (int i = 0; i <= 2 * R; ++i) w[i] /= sum;
    int64_t nv = (int64_t)n[0] * n[1] * n[2];
    double *a = (double *)malloc(sizeof(double) * nv), *b = (double *)malloc(sizeof(double) * nv);
    const double *src = in;
    for (int axis = 0; axis < 3; ++axis) {
        double *dst = axis == 0 ? a : (axis == 1 ? b : out);
#pragma omp parallel for schedule(static)
        for (int k = 0; k < n[2]; ++k)
            for (int j = 0; j < n[1]; ++j)
                for (int i = 0; i < n[0]; ++i) {
                    double acc = 0.0;
                    for (int t = -R; t <= R; ++t) {
                        int ii = i, jj = j, kk = k;
                        if (axis == 0) ii = clampi(i + t, 0, n[0] - 1);
                        if (axis == 1) jj = clampi(j + t, 0, n[1] - 1);
                        if (axis == 2) kk = clampi(k + t, 0, n[2] - 1);
                        acc += w[t + R] * src[vidx(n, ii, jj, kk)];
                    }
                    dst[vidx(n, i, j, k)] = acc;
                }
        src = dst;
    }
    free(w);
    free(a);
    free(b);
}

/* Eigenvalues of the symmetric 3x3 matrix H6 (xx yy zz xy xz yz) by cyclic Jacobi
 * rotations, sorted by |lambda| ascending (ties by lambda ascending). */
void or_eig3_jacobi(const double *H6, double *lam) {
    double a[3][3] = {{H6[0], H6[3], H6[4]}, {H6[3], H6[1], H6[5]}, {H6[4], H6[5], H6[2]}};
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        double scale = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2] + 2.0 * off;
        if (off <= 1e-300 || off <= 1e-32 * scale) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 3; ++k) { /* A <- A J (columns p, q) */
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - sn * akq;
                    a[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) { /* A <- J^T A (rows p, q) */
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - sn * aqk;
                    a[q][k] = sn * apk + c * aqk;
                }
            }
    }
    double l[3] = {a[0][0], a[1][1], a[2][2]};
    for (int i = 0; i < 3; ++i) /* insertion sort by (|l|, l) */
        for (int j = i + 1; j < 3; ++j) {
            int swap = fabs(l[j]) < fabs(l[i]) || (fabs(l[j]) == fabs(l[i]) && l[j] < l[i]);
            if (swap) {
                double tmp = l[i];
                l[i] = l[j];
                l[j] = tmp;
            }
        }
    lam[0] = l[0];
    lam[1] = l[1];
    lam[2] = l[2];
}

/* Frangi bright-vessel response of sorted eigenvalues (|l1| <= |l2| <= |l3|):
 * 0 if l2 > 0 or l3 > 0, else (1 - e^{-Ra^2/2a^2}) e^{-Rb^2/2b^2} (1 - e^{-S^2/2c^2})
 * with Ra = |l2|/|l3|, Rb = |l1|/sqrt|l2 l3|, S = ||l||. */
double or_frangi_response(const double *l, double alpha, double beta, double c) {
    if (l[1] > 0.0 || l[2] > 0.0 || l[1] == 0.0 || l[2] == 0.0 || c <= 0.0) return 0.0;
    double Ra = fabs(l[1]) / fabs(l[2]);
    double Rb = fabs(l[0]) / sqrt(fabs(l[1] * l[2]));
    double S = sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    return (1.0 - exp(-Ra * Ra / (2.0 * alpha * alpha))) * exp(-Rb * Rb / (2.0 * beta * beta)) *
           (1.0 - exp(-S * S / (2.0 * c * c)));
}

/* Multi-scale vesselness of the normalised volume (Sec. 1; Frangi et al. 1998):
 * for each sigma (voxels) the Gaussian-smoothed volume's Hessian (the stencils of
 * Sec. 2.3 in voxel units) times sigma^2, its sorted eigenvalues, c = 0.5 max_v S
 * over the volume, V_sigma by or_frangi_response; V = max over sigma.
 *   smax (nullable): per-scale max S; amb (nullable): 1 where a scale has a
 *   near-tie |l1| ~ |l2| (within 1e-4 |l3|) of opposite signs whose other order
 *   changes that scale's response by more than 5e-5 (the response jumps there). */
void or_frangi(const double *In, const int *n, const double *sigmas, int ns, double alpha, double beta,
               double *V, double *smax, uint8_t *amb) {
    int64_t nv = (int64_t)n[0] * n[1] * n[2];
    double *sm = (double *)malloc(sizeof(double) * nv);
    double *lam = (double *)malloc(sizeof(double) * 3 * nv);
    for (int64_t v = 0; v < nv; ++v) V[v] = 0.0;
    if (amb)
        for (int64_t v = 0; v < nv; ++v) amb[v] = 0;
    for (int si = 0; si < ns; ++si) {
        double sg = sigmas[si], s2 = sg * sg, mx = 0.0;
        or_gauss_smooth(In, n, sg, sm);
#pragma omp parallel for schedule(static) reduction(max : mx)
        for (int k = 0; k < n[2]; ++k)
            for (int j = 0; j < n[1]; ++j)
                for (int i = 0; i < n[0]; ++i) {
                    int im = clampi(i - 1, 0, n[0] - 1), ip = clampi(i + 1, 0, n[0] - 1);
                    int jm = clampi(j - 1, 0, n[1] - 1), jp = clampi(j + 1, 0, n[1] - 1);
                    int km = clampi(k - 1, 0, n[2] - 1), kp = clampi(k + 1, 0, n[2] - 1);
                    int64_t v = vidx(n, i, j, k);
                    double c = sm[v], H6[6];
                    H6[0] = s2 * (sm[vidx(n, ip, j, k)] - 2.0 * c + sm[vidx(n, im, j, k)]);
                    H6[1] = s2 * (sm[vidx(n, i, jp, k)] - 2.0 * c + sm[vidx(n, i, jm, k)]);
                    H6[2] = s2 * (sm[vidx(n, i, j, kp)] - 2.0 * c + sm[vidx(n, i, j, km)]);
                    H6[3] = s2 * (sm[vidx(n, ip, jp, k)] - sm[vidx(n, ip, jm, k)] - sm[vidx(n, im, jp, k)] +
                                  sm[vidx(n, im, jm, k)]) / 4.0;
                    H6[4] = s2 * (sm[vidx(n, ip, j, kp)] - sm[vidx(n, ip, j, km)] - sm[vidx(n, im, j, kp)] +
                                  sm[vidx(n, im, j, km)]) / 4.0;
                    H6[5] = s2 * (sm[vidx(n, i, jp, kp)] - sm[vidx(n, i, jp, km)] - sm[vidx(n, i, jm, kp)] +
                                  sm[vidx(n, i, jm, km)]) / 4.0;
                    or_eig3_jacobi(H6, lam + 3 * v);
                    const double *l = lam + 3 * v;
                    double S = sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
                    if (S > mx) mx = S;
                }
        if (smax) smax[si] = mx;
        double cc = 0.5 * mx;
#pragma omp parallel for schedule(static)
        for (int64_t v = 0; v < nv; ++v) {
            const double *l = lam + 3 * v;
            double r = or_frangi_response(l, alpha, beta, cc);
            if (r > V[v]) V[v] = r;
            if (amb && (l[0] > 0.0) != (l[1] > 0.0) && fabs(fabs(l[1]) - fabs(l[0])) < 1e-4 * fabs(l[2])) {
                /* the other order of the tied pair is equally valid; flag only if it matters */
                double alt[3] = {l[1], l[0], l[2]};
                if (fabs(or_frangi_response(alt, alpha, beta, cc) - r) > 5e-5) amb[v] = 1;
            }
        }
    }
    free(sm);
    free(lam);
}

/* Opacity and colour (Eq. 4 and the sample colour) at m world points, each seen
 * along the unit direction dir; out is [m][4] = alpha, r, g, b. Test helper. */
void or_sample_points(const double *In, const double *V, const int *n, const double *s, const or_params *P,
                      const float *tf32, double gmax, const double *pts, int64_t m, const double *dir,
                      double *out) {
    or_vol v;
    make_vol(&v, In, V, n, s);
    int64_t nvox = (int64_t)n[0] * n[1] * n[2];
    double *g = (double *)malloc(sizeof(double) * 3 * nvox);
    double *Hs = (double *)malloc(sizeof(double) * 6 * nvox);
    or_voxel_derivatives(In, n, s, g, Hs);
    v.g = g;
    v.H = Hs;
    v.gmax = gmax > 0.0 ? gmax : or_gmax(g, nvox);
    int ntf = P->tf_w * P->tf_h * 4;
    double *tf = (double *)malloc(sizeof(double) * ntf);
    for (int q = 0; q < ntf; ++q) tf[q] = (double)tf32[q];
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < m; ++q) {
        double a, c[3];
        sample_optics(&v, P, tf, pts + 3 * q, dir, &a, c);
        out[4 * q] = a;
        out[4 * q + 1] = c[0];
        out[4 * q + 2] = c[1];
        out[4 * q + 3] = c[2];
    }
    free(tf);
    free(g);
    free(Hs);
}

/* ------------------------------------------------------------ gradients */

/* Everything the adjoint of one sample needs, evaluated in FP64 at world point p. */
typedef struct {
    int i0[3];
    double f[3];
    double fld[11];   /* I, g3, H6 (xx yy zz xy xz yz), V */
    double gmag, gg, kappa, ghat[3], gn, y, rgba[4];
    int tj, tk;       /* transfer-function cell */
    double tt, tq;    /* its fractions */
    int clamp_x, clamp_y; /* 1 when the lookup coordinate lies inside [0, 1] */
    double mg, w_inner, w, raw, alpha0, alpha, d, dot, c[3];
} or_srec;

static void sample_record(const or_vol *v, const or_params *P, const double *tf, const double p[3],
                          const double dir[3], or_srec *s) {
    memset(s, 0, sizeof *s);
    for (int a = 0; a < 3; ++a) cell_of(p[a] / v->s[a] - 0.5, v->n[a], &s->i0[a], &s->f[a]);
    field_at(v, p, s->fld);
    const double *g = s->fld + 1, *H = s->fld + 4;
    s->gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    s->gmag = sqrt(s->gg);
    if (s->gg > 0.0) {
        double km[2];
        or_curvature(g, H, km);
        s->kappa = km[0];
        for (int a = 0; a < 3; ++a) s->ghat[a] = g[a] / s->gmag;
    }
    s->gn = v->gmax > 0.0 ? s->gmag / v->gmax : 0.0;
    s->y = P->tf_mode == 1 ? s->gn : (P->tf_mode == 2 ? s->fld[10] : 0.0);
    double I = s->fld[0];
    s->clamp_x = I >= 0.0 && I <= 1.0;
    double xs = clampd(I, 0.0, 1.0) * (P->tf_w - 1);
    s->tj = (int)floor(xs);
    if (s->tj > P->tf_w - 2) s->tj = P->tf_w - 2;
    s->tt = xs - s->tj;
    if (P->tf_h > 1) {
        s->clamp_y = s->y >= 0.0 && s->y <= 1.0;
        double ys = clampd(s->y, 0.0, 1.0) * (P->tf_h - 1);
        s->tk = (int)floor(ys);
        if (s->tk > P->tf_h - 2) s->tk = P->tf_h - 2;
        s->tq = ys - s->tk;
    }
    tf_sample(tf, P->tf_w, P->tf_h, I, s->y, s->rgba);
    s->mg = P->grad_mod ? (s->gn < 1.0 ? s->gn : 1.0) : 1.0;
    s->w_inner = 1.0 + P->gamma * s->kappa / P->kappa_ref;
    s->w = clampd(s->w_inner, 0.0, P->w_max);
    s->raw = P->opacity_scale * s->rgba[3] * s->mg * s->w;
    s->alpha0 = clampd(s->raw, 0.0, 1.0);
    s->alpha = s->alpha0;
    if (P->opacity_ref_step > 0.0) {
        double dt = P->step_vox * fmin(v->s[0], fmin(v->s[1], v->s[2]));
        s->alpha = 1.0 - pow(1.0 - s->alpha0, dt / P->opacity_ref_step);
    }
    s->dot = s->ghat[0] * dir[0] + s->ghat[1] * dir[1] + s->ghat[2] * dir[2];
    s->d = fabs(s->dot);
    double d16 = pow(s->d, 16.0);
    for (int q = 0; q < 3; ++q)
        s->c[q] = P->shading ? s->rgba[q] * (P->ka + P->kd * s->d) + P->ks * d16 : s->rgba[q];
}

/* Chain dL/dalpha and dL/dc of one sample back to the transfer-function entries,
 * the uniforms (gamma, ka, kd, ks, opacity_scale) and the per-voxel adjoints of the
 * interpolated fields (I_norm, gradient, Hessian), following Eq. 4, the lookup,
 * the shading, Eq. 3 and the trilinear weights; clamps pass gradient only on
 * their identity branch, |x| has derivative sign(x) (0 at 0). */
static void sample_adjoint(const or_vol *v, const or_params *P, const double *tf, const or_srec *s,
                           const double dir[3], double da, const double dc[3], double *dtf, double *dpar,
                           double *aI, double *ag, double *aH) {
    (void)tf;
    const double *g = s->fld + 1, *H = s->fld + 4;
    double drgba[4] = {0, 0, 0, 0}, dd = 0.0;
    /* colour */
    double d15 = pow(s->d, 15.0), d16 = d15 * s->d;
    for (int q = 0; q < 3; ++q) {
        if (P->shading) {
            drgba[q] += dc[q] * (P->ka + P->kd * s->d);
            dpar[1] += dc[q] * s->rgba[q];
            dpar[2] += dc[q] * s->rgba[q] * s->d;
            dpar[3] += dc[q] * d16;
            dd += dc[q] * (s->rgba[q] * P->kd + 16.0 * P->ks * d15);
        } else {
            drgba[q] += dc[q];
        }
    }
    /* opacity correction, then Eq. 4 */
    if (P->opacity_ref_step > 0.0) {
        double dt = P->step_vox * fmin(v->s[0], fmin(v->s[1], v->s[2]));
        double r = dt / P->opacity_ref_step;
        da = s->alpha0 < 1.0 ? da * r * pow(1.0 - s->alpha0, r - 1.0) : 0.0;
    }
    double draw = (s->raw >= 0.0 && s->raw <= 1.0) ? da : 0.0;
    dpar[4] += draw * s->rgba[3] * s->mg * s->w;
    drgba[3] += draw * P->opacity_scale * s->mg * s->w;
    double dmg = draw * P->opacity_scale * s->rgba[3] * s->w;
    double dw = draw * P->opacity_scale * s->rgba[3] * s->mg;
    double dwi = (s->w_inner >= 0.0 && s->w_inner <= P->w_max) ? dw : 0.0;
    dpar[0] += dwi * s->kappa / P->kappa_ref;
    double dkappa = dwi * P->gamma / P->kappa_ref;
    double dgn = 0.0;
    if (P->grad_mod && s->gn < 1.0) dgn += dmg;
    /* transfer-function lookup */
    double dI = 0.0, dy = 0.0;
    int w = P->tf_w;
    if (P->tf_h == 1) {
        for (int c = 0; c < 4; ++c) {
            dtf[4 * s->tj + c] += (1.0 - s->tt) * drgba[c];
            dtf[4 * (s->tj + 1) + c] += s->tt * drgba[c];
            if (s->clamp_x) dI += drgba[c] * (tf[4 * (s->tj + 1) + c] - tf[4 * s->tj + c]) * (w - 1);
        }
    } else {
        int j = s->tj, k = s->tk;
        double t = s->tt, q = s->tq;
        for (int c = 0; c < 4; ++c) {
            double T00 = tf[4 * (k * w + j) + c], T01 = tf[4 * (k * w + j + 1) + c];
            double T10 = tf[4 * ((k + 1) * w + j) + c], T11 = tf[4 * ((k + 1) * w + j + 1) + c];
            dtf[4 * (k * w + j) + c] += (1.0 - q) * (1.0 - t) * drgba[c];
            dtf[4 * (k * w + j + 1) + c] += (1.0 - q) * t * drgba[c];
            dtf[4 * ((k + 1) * w + j) + c] += q * (1.0 - t) * drgba[c];
            dtf[4 * ((k + 1) * w + j + 1) + c] += q * t * drgba[c];
            if (s->clamp_x) dI += drgba[c] * ((1.0 - q) * (T01 - T00) + q * (T11 - T10)) * (w - 1);
            if (s->clamp_y) dy += drgba[c] * ((1.0 - t) * (T10 - T00) + t * (T11 - T01)) * (P->tf_h - 1);
        }
        if (P->tf_mode == 1) dgn += dy; /* mode 2: V is a constant of the volume */
    }
    /* shading direction d = |g-hat . dir| and curvature kappa = g^T H g / |g|^2 */
    double dgv[3] = {0, 0, 0}, dHv[6] = {0, 0, 0, 0, 0, 0};
    if (s->gg > 0.0) {
        double sgn = s->dot > 0.0 ? 1.0 : (s->dot < 0.0 ? -1.0 : 0.0);
        double dghat[3];
        for (int a = 0; a < 3; ++a) dghat[a] = P->shading ? dd * sgn * dir[a] : 0.0;
        double proj = dghat[0] * s->ghat[0] + dghat[1] * s->ghat[1] + dghat[2] * s->ghat[2];
        for (int a = 0; a < 3; ++a) dgv[a] += (dghat[a] - proj * s->ghat[a]) / s->gmag;
        for (int a = 0; a < 3; ++a) dgv[a] += dgn * s->ghat[a] / (v->gmax > 0.0 ? v->gmax : 1.0) * (v->gmax > 0.0);
        double Hg[3] = {H[0] * g[0] + H[3] * g[1] + H[4] * g[2], H[3] * g[0] + H[1] * g[1] + H[5] * g[2],
                        H[4] * g[0] + H[5] * g[1] + H[2] * g[2]};
        for (int a = 0; a < 3; ++a) dgv[a] += dkappa * (2.0 * Hg[a] - 2.0 * s->kappa * g[a]) / s->gg;
        dHv[0] += dkappa * g[0] * g[0] / s->gg;
        dHv[1] += dkappa * g[1] * g[1] / s->gg;
        dHv[2] += dkappa * g[2] * g[2] / s->gg;
        dHv[3] += dkappa * 2.0 * g[0] * g[1] / s->gg;
        dHv[4] += dkappa * 2.0 * g[0] * g[2] / s->gg;
        dHv[5] += dkappa * 2.0 * g[1] * g[2] / s->gg;
    }
    /* trilinear weights onto the voxel fields */
    for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy2 = (c >> 1) & 1, dz = (c >> 2) & 1;
        double wt = (dx ? s->f[0] : 1.0 - s->f[0]) * (dy2 ? s->f[1] : 1.0 - s->f[1]) * (dz ? s->f[2] : 1.0 - s->f[2]);
        int64_t id = vidx(v->n, s->i0[0] + dx, s->i0[1] + dy2, s->i0[2] + dz);
        aI[id] += wt * dI;
        for (int q = 0; q < 3; ++q) ag[3 * id + q] += wt * dgv[q];
        for (int q = 0; q < 6; ++q) aH[6 * id + q] += wt * dHv[q];
    }
}

/* Transpose of the voxel stencils of Eq. 2 and Sec. 2.3 (clamp-to-edge): add the
 * adjoints of the voxel gradient and Hessian into the adjoint of I_norm. */
static void stencil_adjoint(const int *n, const double *s, const double *ag, const double *aH, double *dIn) {
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                int im = clampi(i - 1, 0, n[0] - 1), ip = clampi(i + 1, 0, n[0] - 1);
                int jm = clampi(j - 1, 0, n[1] - 1), jp = clampi(j + 1, 0, n[1] - 1);
                int km = clampi(k - 1, 0, n[2] - 1), kp = clampi(k + 1, 0, n[2] - 1);
                int64_t v = vidx(n, i, j, k);
                const double *G = ag + 3 * v, *Hh = aH + 6 * v;
                dIn[vidx(n, ip, j, k)] += G[0] / (2.0 * s[0]);
                dIn[vidx(n, im, j, k)] -= G[0] / (2.0 * s[0]);
                dIn[vidx(n, i, jp, k)] += G[1] / (2.0 * s[1]);
                dIn[vidx(n, i, jm, k)] -= G[1] / (2.0 * s[1]);
                dIn[vidx(n, i, j, kp)] += G[2] / (2.0 * s[2]);
                dIn[vidx(n, i, j, km)] -= G[2] / (2.0 * s[2]);
                double hx = Hh[0] / (s[0] * s[0]), hy = Hh[1] / (s[1] * s[1]), hz = Hh[2] / (s[2] * s[2]);
                dIn[vidx(n, ip, j, k)] += hx;
                dIn[v] -= 2.0 * hx;
                dIn[vidx(n, im, j, k)] += hx;
                dIn[vidx(n, i, jp, k)] += hy;
                dIn[v] -= 2.0 * hy;
                dIn[vidx(n, i, jm, k)] += hy;
                dIn[vidx(n, i, j, kp)] += hz;
                dIn[v] -= 2.0 * hz;
                dIn[vidx(n, i, j, km)] += hz;
                double hxy = Hh[3] / (4.0 * s[0] * s[1]), hxz = Hh[4] / (4.0 * s[0] * s[2]);
                double hyz = Hh[5] / (4.0 * s[1] * s[2]);
                dIn[vidx(n, ip, jp, k)] += hxy;
                dIn[vidx(n, ip, jm, k)] -= hxy;
                dIn[vidx(n, im, jp, k)] -= hxy;
                dIn[vidx(n, im, jm, k)] += hxy;
                dIn[vidx(n, ip, j, kp)] += hxz;
                dIn[vidx(n, ip, j, km)] -= hxz;
                dIn[vidx(n, im, j, kp)] -= hxz;
                dIn[vidx(n, im, j, km)] += hxz;
                dIn[vidx(n, i, jp, kp)] += hyz;
                dIn[vidx(n, i, jp, km)] -= hyz;
                dIn[vidx(n, i, jm, kp)] -= hyz;
                dIn[vidx(n, i, jm, km)] += hyz;
            }
}

/* Gradient of L = sum_pixels <dL/dRGBA, RGBA> (any loss through its image
 * gradient dl_drgba) with respect to the transfer-function entries (dtf, same
 * layout as tf), the uniforms dpar = (gamma, ka, kd, ks, opacity_scale) and the
 * normalised voxel intensities (dIn, may be NULL). The stopping sample of every
 * ray is the forward one (a fixed index); I_min, I_max, |grad I|_max (gmax) and V
 * are constants. Compositing adjoint (Eqs. 5-6): with T_k = prod_{j<k}(1 - a_j),
 * dC/da_k = T_k (c_k - R_{k+1}), R_{k+1} the colour composited from k+1 onwards,
 * dA/da_k = T_k prod_{j>k}(1 - a_j), dC/dc_k = T_k a_k. Serial (plain and slow). */
void or_render_grad(const double *In, const double *V, const int *n, const double *s, const or_params *P,
                    const float *tf32, double gmax, const float *cams, int n_cams, int W, int H,
                    const double *dl_drgba, double *dtf, double *dpar, double *dIn) {
    or_vol v;
    make_vol(&v, In, V, n, s);
    int64_t nvox = (int64_t)n[0] * n[1] * n[2];
    double *g = (double *)malloc(sizeof(double) * 3 * nvox), *Hs = (double *)malloc(sizeof(double) * 6 * nvox);
    or_voxel_derivatives(In, n, s, g, Hs);
    v.g = g;
    v.H = Hs;
    v.gmax = gmax > 0.0 ? gmax : or_gmax(g, nvox);
    int ntf = P->tf_w * P->tf_h * 4;
    double *tf = (double *)malloc(sizeof(double) * ntf);
    for (int q = 0; q < ntf; ++q) tf[q] = (double)tf32[q];
    for (int q = 0; q < ntf; ++q) dtf[q] = 0.0;
    for (int q = 0; q < 5; ++q) dpar[q] = 0.0;
    double *aI = (double *)calloc(nvox, sizeof(double));
    double *ag = (double *)calloc(3 * nvox, sizeof(double));
    double *aH = (double *)calloc(6 * nvox, sizeof(double));
    double dt = P->step_vox * fmin(s[0], fmin(s[1], s[2]));
    int64_t cap = 64;
    double *al = (double *)malloc(sizeof(double) * cap), *cl = (double *)malloc(sizeof(double) * 3 * cap);
    for (int ci = 0; ci < n_cams; ++ci) {
        double cam[12];
        for (int q = 0; q < 12; ++q) cam[q] = (double)cams[12 * ci + q];
        for (int j = 0; j < H; ++j)
            for (int i = 0; i < W; ++i) {
                int64_t pix = ((int64_t)ci * H + j) * W + i;
                const double *dl = dl_drgba + 4 * pix;
                /* every term of a ray's gradient carries a factor of its dl: a ray with
                 * dl = 0 adds exactly zero and is not marched */
                if (dl[0] == 0.0 && dl[1] == 0.0 && dl[2] == 0.0 && dl[3] == 0.0) continue;
                double o[3], d[3], tn, tfar;
                if (!ray_setup(&v, cam, W, H, i, j, o, d, &tn, &tfar)) continue;
                /* forward: the processed samples and their (alpha, colour) */
                int64_t ns = 0;
                double A = 0.0;
                for (int64_t k = 0; tn + (k + 0.5) * dt < tfar; ++k) {
                    double t = tn + (k + 0.5) * dt, p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
                    or_srec sr;
                    sample_record(&v, P, tf, p, d, &sr);
                    if (ns == cap) {
                        cap *= 2;
                        al = (double *)realloc(al, sizeof(double) * cap);
                        cl = (double *)realloc(cl, sizeof(double) * 3 * cap);
                    }
                    al[ns] = sr.alpha;
                    for (int q = 0; q < 3; ++q) cl[3 * ns + q] = sr.c[q];
                    ++ns;
                    A = A + (1.0 - A) * sr.alpha;
                    if (A >= P->et_threshold) break;
                }
                /* reverse: R_{k+1}, prod_{j>k}(1 - a_j), T_k from the forward prefix products */
                double *T = (double *)malloc(sizeof(double) * (ns + 1));
                T[0] = 1.0;
                for (int64_t k = 0; k < ns; ++k) T[k + 1] = T[k] * (1.0 - al[k]);
                double R[3] = {0, 0, 0}, Pk = 1.0;
                for (int64_t k = ns - 1; k >= 0; --k) {
                    double da = T[k] * (dl[0] * (cl[3 * k] - R[0]) + dl[1] * (cl[3 * k + 1] - R[1]) +
                                        dl[2] * (cl[3 * k + 2] - R[2]) + dl[3] * Pk);
                    double dc[3] = {T[k] * al[k] * dl[0], T[k] * al[k] * dl[1], T[k] * al[k] * dl[2]};
                    double t = tn + (k + 0.5) * dt, p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
                    or_srec sr;
                    sample_record(&v, P, tf, p, d, &sr);
                    sample_adjoint(&v, P, tf, &sr, d, da, dc, dtf, dpar, aI, ag, aH);
                    for (int q = 0; q < 3; ++q) R[q] = al[k] * cl[3 * k + q] + (1.0 - al[k]) * R[q];
                    Pk *= (1.0 - al[k]);
                }
                free(T);
            }
    }
    if (dIn) {
        for (int64_t q = 0; q < nvox; ++q) dIn[q] = aI[q];
        stencil_adjoint(n, s, ag, aH, dIn);
    }
    free(al);
    free(cl);
    free(aI);
    free(ag);
    free(aH);
    free(tf);
    free(g);
    free(Hs);
}

/* ------------------------------------------- 256-bin histogram and tissue peaks */

/* 256-bin density of I_norm (Sec. 2.2): bin j = min(floor(I_norm * 256), 255), with
 * I_norm formed in float32 exactly as for the brick grid (the bin is an integer
 * decision that must match the kernel's bit for bit). raw: float32 or uint16 values. */
void or_histogram256(const float *raw, int64_t n, float imin, float imax, uint64_t *hist) {
    volatile float range = imax - imin;
    for (int j = 0; j < 256; ++j) hist[j] = 0;
    for (int64_t i = 0; i < n; ++i) {
        volatile float d = raw[i] - imin;
        volatile float r = d / range;
        volatile float x = r * 256.0f;
        int j = (int)x;
        if (j > 255) j = 255;
        if (j < 0) j = 0;
        hist[j] += 1;
    }
}

/* Tri-modal peak extraction (Sec. 2.2, Tables 1-2; the paper names the result,
 * not the procedure). Reading: smooth the histogram with the binomial kernel
 * [1 4 6 4 1] (integer weights, clamp-to-edge, no division); a bin j in
 * [lo, hi] is a peak if s[j] > s[j-1] and s[j] >= s[j+1]; keep the three peaks
 * with the largest s (ties to the lower bin) and return their bins in ascending
 * order in peaks[0..2]. Returns the number of peaks found (<= 3); smoothed
 * (nullable, 256 entries) receives s. Integer arithmetic only. */
int or_tissue_peaks(const uint64_t *hist, int lo, int hi, int *peaks, uint64_t *smoothed) {
    static const int w[5] = {1, 4, 6, 4, 1};
    uint64_t s[256];
    for (int j = 0; j < 256; ++j) {
        uint64_t acc = 0;
        for (int t = -2; t <= 2; ++t) acc += (uint64_t)w[t + 2] * hist[clampi(j + t, 0, 255)];
        s[j] = acc;
        if (smoothed) smoothed[j] = acc;
    }
    if (lo < 1) lo = 1;
    if (hi > 254) hi = 254;
    int best[3] = {-1, -1, -1};
    for (int j = lo; j <= hi; ++j) {
        if (!(s[j] > s[j - 1] && s[j] >= s[j + 1])) continue;
        /* insert into the top three by (s descending, j ascending) */
        for (int q = 0; q < 3; ++q) {
            if (best[q] < 0 || s[j] > s[best[q]]) {
                for (int r = 2; r > q; --r) best[r] = best[r - 1];
                best[q] = j;
                break;
            }
        }
    }
    int cnt = 0;
    for (int q = 0; q < 3; ++q)
        if (best[q] >= 0) peaks[cnt++] = best[q];
    for (int a = 0; a < cnt; ++a) /* ascending bins */
        for (int b = a + 1; b < cnt; ++b)
            if (peaks[b] < peaks[a]) {
                int t = peaks[a];
                peaks[a] = peaks[b];
                peaks[b] = t;
            }
    for (int q = cnt; q < 3; ++q) peaks[q] = -1;
    return cnt;
}

/* ------------------------------------------------------ optional pre-filters */

/* 3x3x3 median of the normalised volume with clamp-to-edge neighbours: the
 * optional median pass Sec. 5.3 proposes against impulsive artefacts. The
 * median of 27 values is the 14th smallest (an order statistic: exact). */
static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void or_median3(const double *in, const int *n, double *out) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                double w[27];
                int m = 0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx)
                            w[m++] = in[vidx(n, clampi(i + dx, 0, n[0] - 1), clampi(j + dy, 0, n[1] - 1),
                                              clampi(k + dz, 0, n[2] - 1))];
                qsort(w, 27, sizeof(double), cmp_double);
                out[vidx(n, i, j, k)] = w[13];
            }
}
