/*
 * FP64 brute-force oracle of sparse-voxel rasterization (SVRaster,
 * arXiv 2412.04459).  TEST INFRASTRUCTURE ONLY: it is linked by the tests,
 * by the smoke check and by the CPU-baseline leg of the benchmark, never by
 * the product path.  It shares no code with the CUDA library.
 *
 * What it computes, for every requested pixel:
 *   - the pixel ray (Sec. 3.1.2 "Rendering pixels"): OpenCV pinhole, pixel
 *     centres at +0.5, camera-space direction ((x+.5-cx)/fx, (y+.5-cy)/fy, 1)
 *     rotated to world by R^T, origin -R^T t.  The camera-space z component of
 *     the direction is 1, so ray distances t are camera z-depths;
 *   - the intersection of that ray with EVERY voxel (ray-AABB of Sec. A.2,
 *     valid = (a <= b) and (a > 0)); no tiles, no sorting keys;
 *   - the hits sorted exactly by entry distance a (ties: exit b, voxel id);
 *   - front-to-back alpha compositing, Eq. (alpha_blend), with the voxel
 *     alpha of Eq. (vox_alpha) / Eq. (supp_alpha_comp): K evenly spaced
 *     samples (Eq. K_samp_pts), trilinear interpolation of the 8 raw corner
 *     densities (Eq. interp) followed by explin (Eq. explin); the view
 *     dependent colour of Eq. (vox_color), degree-3 SH evaluated once per
 *     voxel toward normalize(centre - ray origin); the voxel depth of
 *     Sec. A.4 composited as D = sum_i T_i d_i; early termination after the
 *     voxel that leaves T < t_stop (Sec. 3.1.2);
 *   - the analytic gradient of sum(g_rgb * C + g_depth * D + g_alpha * A)
 *     with respect to the raw grid-point densities and the SH coefficients
 *     (Sec. A.2 alpha gradient, Sec. A.4 depth gradient), written in the
 *     alpha form with suffix sums;
 *   - on request (the _ex entry points): the normal image N = sum_i T_i
 *     alpha_i n_i with the voxel normal n of Eq. (vox_normal), the
 *     normalised gradient of the trilinear density field at the voxel
 *     centre in the closed form of Eq. (interp_grad), and its gradient
 *     (Eq. interp_grad_grad through the normalisation); per voxel the
 *     maximum blending weight max T_i alpha_i (pruning, Sec. 3.2.2) and the
 *     subdivision priority sum |alpha_i dL/dalpha_i| (Eq. priority); the
 *     distortion loss of each ray (Sec. 3.2.3, the loss of Mip-NeRF 360),
 *     L = sum_i sum_j w_i w_j |m_i - m_j| + 1/3 sum_i w_i^2 delta_i over its
 *     composited voxels, w_i = T_i alpha_i, m_i = (a_i + b_i) / 2 and
 *     delta_i = b_i - a_i in ray distance t (camera depth), and its gradient.
 *
 * Voxel geometry: size v_s = w_s 2^-l (Eq. vox_coord); the centre is the
 * caller's value (the lattice check lives in the Python part of the oracle).
 * Outputs: C (+ T_final * bg), D, A = 1 - T_final.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OC_PI 3.14159265358979323846

typedef struct {
    double fx, fy, cx, cy;
    double R[9]; /* row-major world-to-camera rotation */
    double t[3];
    int32_t width, height;
} oc_camera;

typedef struct {
    int32_t K;
    double t_stop;
    double bg[3];
} oc_params;

typedef struct {
    double world_size;
    int64_t n_vox;
    const double *centre;     /* [N][3] */
    const uint8_t *level;     /* [N] */
    const int32_t *corner_idx;/* [N][8] */
    const double *grid;       /* [Pts] */
    const double *sh;         /* [N][16][3] */
} oc_scene;

/* ---------------------------------------------------------------- explin */

/* Eq. (explin). */
double oc_explin(double x) {
    if (x > 1.1) return x;
    return exp(x / 1.1 - 1.0 + log(1.1));
}

/* d explin / dx: 1 on the linear branch, explin(x) / 1.1 on the exponential one. */
double oc_explin_grad(double x) {
    if (x > 1.1) return 1.0;
    return exp(x / 1.1 - 1.0 + log(1.1)) / 1.1;
}

/* ------------------------------------------------------ spherical harmonics */

static double fact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* Associated Legendre function P_l^m(x), m >= 0, without the Condon-Shortley
 * phase: P_m^m = (2m-1)!! (1-x^2)^(m/2), P_{m+1}^m = x (2m+1) P_m^m,
 * (l-m) P_l^m = x (2l-1) P_{l-1}^m - (l+m-1) P_{l-2}^m. */
static double legendre(int l, int m, double x) {
    double s = sqrt(fmax(0.0, (1.0 - x) * (1.0 + x)));
    double pmm = 1.0;
    for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * s;
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double pl = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pl = (x * (2.0 * ll - 1.0) * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pm1;
        pm1 = pl;
    }
    return pl;
}

/* Real orthonormal SH of degree 0..3 at a direction, index l*l + l + m:
 *   m = 0: K_l^0 P_l^0(cos th)
 *   m > 0: sqrt(2) K_l^m cos(m phi) P_l^m(cos th)
 *   m < 0: sqrt(2) K_l^|m| sin(|m| phi) P_l^|m|(cos th)
 * with K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), th measured from +z and
 * phi = atan2(y, x).  The direction is normalised here. */
void oc_sh_basis(const double dir[3], double Y[16]) {
    double r = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    double x = dir[0] / r, y = dir[1] / r, z = dir[2] / r;
    double phi = atan2(y, x);
    for (int l = 0; l <= 3; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * OC_PI) * fact(l - am) / fact(l + am));
            double P = legendre(l, am, z);
            double v;
            if (m == 0) v = K * P;
            else if (m > 0) v = sqrt(2.0) * K * cos(am * phi) * P;
            else v = sqrt(2.0) * K * sin(am * phi) * P;
            Y[l * l + l + m] = v;
        }
    }
}

/* ------------------------------------------------------------------ rays */

void oc_pixel_ray(const oc_camera *c, double px, double py, double ro[3], double rd[3]) {
    double d[3] = {(px + 0.5 - c->cx) / c->fx, (py + 0.5 - c->cy) / c->fy, 1.0};
    for (int i = 0; i < 3; ++i) {
        rd[i] = c->R[0 * 3 + i] * d[0] + c->R[1 * 3 + i] * d[1] + c->R[2 * 3 + i] * d[2];
        ro[i] = -(c->R[0 * 3 + i] * c->t[0] + c->R[1 * 3 + i] * c->t[1] + c->R[2 * 3 + i] * c->t[2]);
    }
}

/* Ray-AABB intersection of Sec. A.2: per axis the two slab distances,
 * a = max over axes of the smaller, b = min over axes of the larger,
 * valid = (a <= b) and (a > 0). */
int oc_ray_aabb(const double c[3], double s, const double ro[3], const double rd[3],
                double *a, double *b) {
    double amax = -INFINITY, bmin = INFINITY;
    for (int i = 0; i < 3; ++i) {
        double c0 = (c[i] - 0.5 * s - ro[i]) / rd[i];
        double c1 = (c[i] + 0.5 * s - ro[i]) / rd[i];
        amax = fmax(amax, fmin(c0, c1));
        bmin = fmin(bmin, fmax(c0, c1));
    }
    *a = amax;
    *b = bmin;
    return (amax <= bmin) && (amax > 0.0);
}

/* Condition number of the segment length b - a of a valid hit with respect
 * to relative perturbations of the numbers that define it: a = (P - r_o)_i /
 * r_d,i on the entry plane's axis i and b = (Q - r_o)_j / r_d,j on the exit
 * plane's axis j move by (|P_i| + |r_o,i|) / |r_d,i| + |a| (and likewise b) per
 * unit relative change of the plane coordinate, the origin and the direction
 * component; their sum over the length.  Large for a ray that grazes the
 * voxel, or crosses a plane nearly parallel to it. */
static double segment_condition(const double c[3], double s, const double ro[3], const double rd[3],
                                double a, double b) {
    int ia = -1, ib = -1;
    double amax = -INFINITY, bmin = INFINITY, pa = 0.0, pb = 0.0;
    for (int i = 0; i < 3; ++i) {
        double lo = c[i] - 0.5 * s, hi = c[i] + 0.5 * s;
        double c0 = (lo - ro[i]) / rd[i], c1 = (hi - ro[i]) / rd[i];
        double near = fmin(c0, c1), far = fmax(c0, c1);
        if (near > amax) {
            amax = near;
            ia = i;
            pa = c0 < c1 ? lo : hi;
        }
        if (far < bmin) {
            bmin = far;
            ib = i;
            pb = c0 < c1 ? hi : lo;
        }
    }
    if (ia < 0 || ib < 0 || !(b > a)) return 0.0;
    double da = (fabs(pa) + fabs(ro[ia])) / fabs(rd[ia]) + fabs(a);
    double db = (fabs(pb) + fabs(ro[ib])) / fabs(rd[ib]) + fabs(b);
    return (da + db) / (b - a);
}

/* Trilinear weights of Eq. (interp) for local coordinate q, corner order
 * V_000, V_001, ..., V_111 (subscript = x, y, z bits, x most significant). */
static void trilinear_weights(const double q[3], double w[8]) {
    for (int c = 0; c < 8; ++c) {
        double wx = (c >> 2) & 1 ? q[0] : 1.0 - q[0];
        double wy = (c >> 1) & 1 ? q[1] : 1.0 - q[1];
        double wz = c & 1 ? q[2] : 1.0 - q[2];
        w[c] = wx * wy * wz;
    }
}

/* Trilinear interpolation of Eq. (interp) of 8 corner values at q. */
double oc_trilinear(const double V[8], const double q[3]) {
    double w[8], acc = 0.0;
    trilinear_weights(q, w);
    for (int c = 0; c < 8; ++c) acc += w[c] * V[c];
    return acc;
}

/* Gradient of the trilinear field with respect to the local coordinate at
 * the voxel centre q = (0.5, 0.5, 0.5), Eq. (interp_grad): along each axis a
 * quarter of (sum of the four corners on the far face) - (sum of the four on
 * the near face); corner c has bit 2 = x, bit 1 = y, bit 0 = z. */
void oc_interp_grad_centre(const double V[8], double g[3]) {
    for (int ax = 0; ax < 3; ++ax) {
        const int bit = 2 - ax;
        double far = 0.0, near = 0.0;
        for (int c = 0; c < 8; ++c) {
            if ((c >> bit) & 1) far += V[c];
            else near += V[c];
        }
        g[ax] = 0.25 * (far - near);
    }
}

/* Voxel normal of Eq. (vox_normal): normalize(gradient at the centre); the
 * zero vector where the gradient vanishes.  Also returns the gradient. */
static void voxel_normal(const oc_scene *S, int64_t v, double n[3], double g[3]) {
    const int32_t *ci = S->corner_idx + 8 * v;
    double V[8];
    for (int c = 0; c < 8; ++c) V[c] = S->grid[ci[c]];
    oc_interp_grad_centre(V, g);
    double len = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    for (int ax = 0; ax < 3; ++ax) n[ax] = len > 0.0 ? g[ax] / len : 0.0;
}

/* max(*p, x) stored atomically, for x >= 0 (non-negative doubles order like
 * their bit patterns). */
static void atomic_max_nonneg(double *p, double x) {
    int64_t *q = (int64_t *)p;
    int64_t want;
    memcpy(&want, &x, sizeof(want));
    int64_t cur = __atomic_load_n(q, __ATOMIC_RELAXED);
    while (cur < want && !__atomic_compare_exchange_n(q, &cur, want, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
    }
}

/* -------------------------------------------------------------- per pixel */

typedef struct {
    double a, b;
    int64_t v;
} oc_hit;

static int hit_cmp(const void *pa, const void *pb) {
    const oc_hit *x = (const oc_hit *)pa, *y = (const oc_hit *)pb;
    if (x->a < y->a) return -1;
    if (x->a > y->a) return 1;
    if (x->b < y->b) return -1;
    if (x->b > y->b) return 1;
    return (x->v > y->v) - (x->v < y->v);
}

typedef struct {
    oc_hit *hits;
    int64_t cap;
    /* per composited hit */
    double *alpha, *T, *d, *col, *pre, *ell;
    double *nrm;   /* [3] voxel normal n of each hit, when normals are rendered */
    double *cdist; /* dL_dist / dw_i of each hit, for the backward */
    double *gvec;  /* [3] unnormalised gradient of Eq. (interp_grad) of each hit */
    int64_t pcap;
} oc_scratch;

static void scratch_free(oc_scratch *s) {
    free(s->hits); free(s->alpha); free(s->T); free(s->d); free(s->col); free(s->pre); free(s->ell);
    free(s->nrm); free(s->gvec); free(s->cdist);
    memset(s, 0, sizeof(*s));
}

static int scratch_hits(oc_scratch *s, int64_t n) {
    if (n <= s->cap) return 0;
    int64_t c = s->cap ? s->cap : 256;
    while (c < n) c *= 2;
    oc_hit *h = (oc_hit *)realloc(s->hits, (size_t)c * sizeof(oc_hit));
    if (!h) return -1;
    s->hits = h;
    s->cap = c;
    return 0;
}

static int scratch_comp(oc_scratch *s, int64_t n) {
    if (n <= s->pcap) return 0;
    int64_t c = s->pcap ? s->pcap : 256;
    while (c < n) c *= 2;
    double **arrs[] = {&s->alpha, &s->T, &s->d, &s->ell};
    for (int i = 0; i < 4; ++i) {
        double *p = (double *)realloc(*arrs[i], (size_t)c * sizeof(double));
        if (!p) return -1;
        *arrs[i] = p;
    }
    double *p = (double *)realloc(s->col, (size_t)c * 3 * sizeof(double));
    if (!p) return -1;
    s->col = p;
    p = (double *)realloc(s->pre, (size_t)c * 3 * sizeof(double));
    if (!p) return -1;
    s->pre = p;
    p = (double *)realloc(s->nrm, (size_t)c * 3 * sizeof(double));
    if (!p) return -1;
    s->nrm = p;
    p = (double *)realloc(s->gvec, (size_t)c * 3 * sizeof(double));
    if (!p) return -1;
    s->gvec = p;
    p = (double *)realloc(s->cdist, (size_t)c * sizeof(double));
    if (!p) return -1;
    s->cdist = p;
    s->pcap = c;
    return 0;
}

/* All valid hits of one ray, sorted by entry distance. */
static int64_t gather_hits(const oc_scene *S, const double ro[3], const double rd[3], oc_scratch *s) {
    int64_t n = 0;
    for (int64_t v = 0; v < S->n_vox; ++v) {
        double vs = ldexp(S->world_size, -(int)S->level[v]);
        double a, b;
        if (oc_ray_aabb(S->centre + 3 * v, vs, ro, rd, &a, &b)) {
            if (scratch_hits(s, n + 1)) return -1;
            s->hits[n].a = a;
            s->hits[n].b = b;
            s->hits[n].v = v;
            ++n;
        }
    }
    qsort(s->hits, (size_t)n, sizeof(oc_hit), hit_cmp);
    return n;
}

/* Samples of one ray segment (Eq. K_samp_pts): depths t_k, interpolated raw
 * densities v_k, trilinear weights w_k. */
static void segment_samples(const oc_scene *S, int64_t v, int K, double a, double b,
                            const double ro[3], const double rd[3],
                            double *t, double *val, double (*w)[8]) {
    double vs = ldexp(S->world_size, -(int)S->level[v]);
    const double *c = S->centre + 3 * v;
    const int32_t *ci = S->corner_idx + 8 * v;
    for (int k = 1; k <= K; ++k) {
        double tk = a + (k - 0.5) / K * (b - a);
        double q[3];
        for (int i = 0; i < 3; ++i) {
            double p = ro[i] + tk * rd[i];
            q[i] = (p - (c[i] - 0.5 * vs)) / vs;
        }
        double ww[8];
        trilinear_weights(q, ww);
        double sum = 0.0;
        for (int j = 0; j < 8; ++j) sum += ww[j] * S->grid[ci[j]];
        t[k - 1] = tk;
        val[k - 1] = sum;
        if (w)
            for (int j = 0; j < 8; ++j) w[k - 1][j] = ww[j];
    }
}

/* View-dependent colour, Eq. (vox_color): pre-clamp and clamped values. */
static void voxel_colour(const oc_scene *S, int64_t v, const double ro[3], double pre[3], double col[3]) {
    const double *c = S->centre + 3 * v;
    double dir[3] = {c[0] - ro[0], c[1] - ro[1], c[2] - ro[2]};
    double Y[16];
    oc_sh_basis(dir, Y);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int n = 0; n < 16; ++n) acc += Y[n] * S->sh[48 * v + 3 * n + ch];
        pre[ch] = acc;
        col[ch] = acc > 0.0 ? acc : 0.0;
    }
}

typedef struct {
    double rgb[3], depth, alpha, t_final;
    double normal[3];  /* N = sum_i T_i alpha_i n_i (when normals are rendered) */
    double dist;       /* distortion loss of the ray */
    int32_t n_comp;
    int64_t term_vox;  /* voxel whose compositing stopped the ray, or -1 */
    double stop_margin; /* min over composited voxels of |T after it / t_stop - 1| (HUGE_VAL: none) */
} oc_pixel_out;

#define OC_KMAX 8

/* Distortion loss of the n composited hits of s (weights w_i = T_i alpha_i,
 * interval midpoints m_i and lengths delta_i in ray distance), by its
 * definition: every ordered pair and every interval on its own. */
static double distortion(const oc_scratch *s, int32_t n) {
    double L = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        double wi = s->T[i] * s->alpha[i], mi = 0.5 * (s->hits[i].a + s->hits[i].b);
        for (int32_t j = 0; j < n; ++j) {
            double wj = s->T[j] * s->alpha[j], mj = 0.5 * (s->hits[j].a + s->hits[j].b);
            L += wi * wj * fabs(mi - mj);
        }
        L += wi * wi * (s->hits[i].b - s->hits[i].a) / 3.0;
    }
    return L;
}

/* dL_dist / dw_k for every composited hit k, into s->cdist:
 * 2 sum_j w_j |m_k - m_j| + 2/3 w_k delta_k. */
static void distortion_grad_w(const oc_scratch *s, int32_t n) {
    for (int32_t k = 0; k < n; ++k) {
        double mk = 0.5 * (s->hits[k].a + s->hits[k].b), acc = 0.0;
        for (int32_t j = 0; j < n; ++j) {
            double wj = s->T[j] * s->alpha[j], mj = 0.5 * (s->hits[j].a + s->hits[j].b);
            acc += wj * fabs(mk - mj);
        }
        s->cdist[k] = 2.0 * acc + 2.0 / 3.0 * s->T[k] * s->alpha[k] * (s->hits[k].b - s->hits[k].a);
    }
}

/* Front-to-back compositing of one pixel; fills the per-hit arrays of s.
 * with_normals: also composite the voxel normals; max_weight (may be NULL):
 * per voxel, the largest blending weight T_i alpha_i seen. */
static int composite(const oc_scene *S, const oc_params *P, const double ro[3], const double rd[3],
                     oc_scratch *s, int64_t n_hits, oc_pixel_out *o, int with_normals, double *max_weight) {
    const int K = P->K;
    double rdn = sqrt(rd[0] * rd[0] + rd[1] * rd[1] + rd[2] * rd[2]);
    double T = 1.0, C[3] = {0, 0, 0}, D = 0.0, Nrm[3] = {0, 0, 0};
    int32_t n = 0;
    o->term_vox = -1;
    o->stop_margin = HUGE_VAL;
    if (scratch_comp(s, n_hits > 0 ? n_hits : 1)) return -1;
    for (int64_t i = 0; i < n_hits; ++i) {
        int64_t v = s->hits[i].v;
        double a = s->hits[i].a, b = s->hits[i].b;
        double ell = (b - a) * rdn;
        double t[OC_KMAX], val[OC_KMAX];
        segment_samples(S, v, K, a, b, ro, rd, t, val, NULL);
        double sum = 0.0;
        for (int k = 0; k < K; ++k) sum += oc_explin(val[k]);
        double alpha = 1.0 - exp(-ell / K * sum);
        /* voxel depth of Sec. A.4 */
        double d = 0.0, prod = 1.0;
        for (int k = 0; k < K; ++k) {
            double ak = 1.0 - exp(-ell / K * oc_explin(val[k]));
            d += prod * ak * t[k];
            prod *= 1.0 - ak;
        }
        double pre[3], col[3];
        voxel_colour(S, v, ro, pre, col);
        for (int ch = 0; ch < 3; ++ch) C[ch] += T * alpha * col[ch];
        D += T * d;
        if (with_normals) {
            voxel_normal(S, v, s->nrm + 3 * n, s->gvec + 3 * n);
            for (int ax = 0; ax < 3; ++ax) Nrm[ax] += T * alpha * s->nrm[3 * n + ax];
        }
        if (max_weight) atomic_max_nonneg(max_weight + v, T * alpha);
        s->alpha[n] = alpha;
        s->T[n] = T;
        s->d[n] = d;
        s->ell[n] = ell;
        for (int ch = 0; ch < 3; ++ch) {
            s->col[3 * n + ch] = col[ch];
            s->pre[3 * n + ch] = pre[ch];
        }
        ++n;
        T = T * (1.0 - alpha);
        if (P->t_stop > 0.0) {
            double m = fabs(T / P->t_stop - 1.0);
            if (m < o->stop_margin) o->stop_margin = m;
        }
        if (T < P->t_stop) {
            o->term_vox = v;
            break;
        }
    }
    for (int ch = 0; ch < 3; ++ch) o->rgb[ch] = C[ch] + T * P->bg[ch];
    for (int ax = 0; ax < 3; ++ax) o->normal[ax] = Nrm[ax];
    o->dist = distortion(s, n);
    o->depth = D;
    o->alpha = 1.0 - T;
    o->t_final = T;
    o->n_comp = n;
    return 0;
}

/* Analytic backward of one pixel (alpha form).  With T_i the transmittance in
 * front of hit i, S_i = prod_{j>i} (1 - alpha_j) and the suffix sums
 *   RC_i = alpha_{i+1} c_{i+1} + (1 - alpha_{i+1}) RC_{i+1},  RC_last = bg,
 *   RD_i = d_{i+1} + (1 - alpha_{i+1}) RD_{i+1},              RD_last = 0,
 * the partials are dC/dalpha_i = T_i (c_i - RC_i), dD/dalpha_i (through the
 * transmittance) = -T_i RD_i, dA/dalpha_i = T_i S_i, dD/dd_i = T_i and
 * dC/dc_i = T_i alpha_i.  Each voxel alpha is 1 - prod_k (1 - alpha_ik),
 * alpha_ik = 1 - exp(-(l/K) explin(v_ik)), so
 *   dalpha_i/dalpha_ik = prod_{j != k} (1 - alpha_ij),
 *   dd_i/dalpha_ik = P_k t_k - sum_{m>k} prod_{j<m, j != k}(1 - alpha_ij) alpha_im t_m
 *     (the K <= 3 cases are the closed forms of Sec. A.4),
 *   dalpha_ik/dv_ik = (1 - alpha_ik) (l/K) explin'(v_ik),
 *   dv_ik/dV_c = trilinear weight of corner c,
 *   dc/dsh[n][ch] = Y_n(dir) if the pre-clamp channel is > 0, else 0.
 * d_grid_abs / d_sh_abs (may be NULL) accumulate the absolute value of every
 * term added to d_grid / d_sh: the magnitude of an element's contributions,
 * which bounds how much of it the rounding of a lower-precision sum can
 * change when the contributions cancel.  d_grid_seg / d_sh_seg (may be NULL)
 * accumulate each term's absolute value times the condition number of the
 * hit's segment length l = (b - a)|r_d| (segment_condition): every term of a
 * hit is proportional to l for a grazing hit, so a renderer that rounds the
 * planes, the origin and the direction to precision u has a relative error of
 * order u times this factor in those terms. */
static void add_term(double *acc, double *acc_abs, double *acc_seg, int64_t i, double add, double kappa) {
#pragma omp atomic
    acc[i] += add;
    if (acc_abs) {
#pragma omp atomic
        acc_abs[i] += fabs(add);
    }
    if (acc_seg) {
#pragma omp atomic
        acc_seg[i] += fabs(add) * kappa;
    }
}

/* With normals (g_normal != NULL, the normals composited by the forward):
 * dN/dalpha_i = T_i (n_i - RN_i) with RN_i = alpha_{i+1} n_{i+1} + (1 -
 * alpha_{i+1}) RN_{i+1}, RN_last = 0, joins dL/dalpha_i; dL/dn_i = T_i
 * alpha_i g_normal passes the normalisation, dL/dgrad = (dL/dn - n (n .
 * dL/dn)) / |grad|, and reaches corner c through Eq. (interp_grad_grad):
 * dgrad/dV_c = 0.25 (2 x_c - 1, 2 y_c - 1, 2 z_c - 1).  priority (may be
 * NULL) accumulates |alpha_i dL/dalpha_i| per voxel (Eq. priority) and
 * priority_seg (may be NULL) the same terms times the segment condition. */
static void pixel_backward(const oc_scene *S, const oc_params *P, const double ro[3], const double rd[3],
                           const oc_scratch *s, const oc_pixel_out *o, const double g_rgb[3],
                           double g_depth, double g_alpha, const double *g_normal, double g_dist,
                           double *d_grid, double *d_sh,
                           double *d_grid_abs, double *d_sh_abs, double *d_grid_seg, double *d_sh_seg,
                           double *priority, double *priority_seg) {
    const int K = P->K;
    int32_t n = o->n_comp;
    double RC[3] = {P->bg[0], P->bg[1], P->bg[2]};
    double RN[3] = {0.0, 0.0, 0.0};
    double RD = 0.0, Sfx = 1.0, RW = 0.0;
    /* the distortion loss depends on the weights w_j = T_j alpha_j only, so
     * it enters dL/dalpha_i like a colour c_j = dL_dist/dw_j with no
     * background: T_i (c_i - RW_i), RW_i = alpha_{i+1} c_{i+1} + (1 -
     * alpha_{i+1}) RW_{i+1} */
    if (g_dist != 0.0) distortion_grad_w(s, n);
    for (int32_t i = n - 1; i >= 0; --i) {
        int64_t v = s->hits[i].v;
        double a = s->hits[i].a, b = s->hits[i].b;
        double Ti = s->T[i], al = s->alpha[i], ell = s->ell[i];
        const double *c = s->col + 3 * i;
        const double *pre = s->pre + 3 * i;
        double kappa = segment_condition(S->centre + 3 * v, ldexp(S->world_size, -(int)S->level[v]), ro, rd, a, b);
        double g = 0.0;
        for (int ch = 0; ch < 3; ++ch) g += g_rgb[ch] * Ti * (c[ch] - RC[ch]);
        g += g_depth * (-Ti * RD);
        g += g_alpha * Ti * Sfx;
        const double *nv = g_normal ? s->nrm + 3 * i : NULL;
        if (g_normal)
            for (int ax = 0; ax < 3; ++ax) g += g_normal[ax] * Ti * (nv[ax] - RN[ax]);
        if (g_dist != 0.0) g += g_dist * Ti * (s->cdist[i] - RW);
        if (priority) {
#pragma omp atomic
            priority[v] += fabs(al * g);
        }
        if (priority_seg) {
#pragma omp atomic
            priority_seg[v] += fabs(al * g) * kappa;
        }

        double t[OC_KMAX], val[OC_KMAX], w[OC_KMAX][8], ak[OC_KMAX];
        segment_samples(S, v, K, a, b, ro, rd, t, val, w);
        for (int k = 0; k < K; ++k) ak[k] = 1.0 - exp(-ell / K * oc_explin(val[k]));
        for (int k = 0; k < K; ++k) {
            double da_dak = 1.0;
            for (int j = 0; j < K; ++j)
                if (j != k) da_dak *= 1.0 - ak[j];
            double Pk = 1.0;
            for (int j = 0; j < k; ++j) Pk *= 1.0 - ak[j];
            double dd_dak = Pk * t[k];
            for (int m = k + 1; m < K; ++m) {
                double pm = 1.0;
                for (int j = 0; j < m; ++j)
                    if (j != k) pm *= 1.0 - ak[j];
                dd_dak -= pm * ak[m] * t[m];
            }
            double gk = g * da_dak + g_depth * Ti * dd_dak;
            double gv = gk * (1.0 - ak[k]) * (ell / K) * oc_explin_grad(val[k]);
            const int32_t *ci = S->corner_idx + 8 * v;
            for (int j = 0; j < 8; ++j) add_term(d_grid, d_grid_abs, d_grid_seg, ci[j], gv * w[k][j], kappa);
        }
        /* normal */
        if (g_normal) {
            const double *gv = s->gvec + 3 * i;
            double len = sqrt(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]);
            if (len > 0.0) {
                double dn[3], dot = 0.0, dg[3];
                for (int ax = 0; ax < 3; ++ax) {
                    dn[ax] = g_normal[ax] * Ti * al;
                    dot += dn[ax] * nv[ax];
                }
                for (int ax = 0; ax < 3; ++ax) dg[ax] = (dn[ax] - nv[ax] * dot) / len;
                const int32_t *ci = S->corner_idx + 8 * v;
                for (int c = 0; c < 8; ++c) {
                    double add = 0.0;
                    for (int ax = 0; ax < 3; ++ax) add += dg[ax] * 0.25 * (2.0 * ((c >> (2 - ax)) & 1) - 1.0);
                    add_term(d_grid, d_grid_abs, d_grid_seg, ci[c], add, kappa);
                }
            }
        }
        /* colour */
        {
            const double *cc = S->centre + 3 * v;
            double dir[3] = {cc[0] - ro[0], cc[1] - ro[1], cc[2] - ro[2]};
            double Y[16];
            oc_sh_basis(dir, Y);
            for (int ch = 0; ch < 3; ++ch) {
                if (!(pre[ch] > 0.0)) continue;
                double dc = g_rgb[ch] * Ti * al;
                for (int m = 0; m < 16; ++m) add_term(d_sh, d_sh_abs, d_sh_seg, 48 * v + 3 * m + ch, Y[m] * dc, kappa);
            }
        }
        /* suffix sums for the next (nearer) hit */
        for (int ch = 0; ch < 3; ++ch) RC[ch] = al * c[ch] + (1.0 - al) * RC[ch];
        if (g_normal)
            for (int ax = 0; ax < 3; ++ax) RN[ax] = al * nv[ax] + (1.0 - al) * RN[ax];
        if (g_dist != 0.0) RW = al * s->cdist[i] + (1.0 - al) * RW;
        RD = s->d[i] + (1.0 - al) * RD;
        Sfx *= 1.0 - al;
    }
}

/* ------------------------------------------------------------- exported */

static void pixel_xy(const oc_camera *cam, int64_t n_px, const int32_t *px_xy, int64_t p, int *x, int *y) {
    (void)n_px;
    if (px_xy) {
        *x = px_xy[2 * p];
        *y = px_xy[2 * p + 1];
    } else {
        *x = (int)(p % cam->width);
        *y = (int)(p / cam->width);
    }
}

/* Forward render of n_px pixels (px_xy = NULL: every pixel, row-major).
 * Per pixel: rgb[3], depth, alpha, t_final, number of composited hits, the
 * terminating voxel (-1 if none) and the stop margin: the smallest relative
 * distance |T / t_stop - 1| of the transmittance after a composited voxel from
 * the stop threshold (HUGE_VAL if t_stop = 0 or nothing was composited), which
 * says how close the pixel came to another termination decision.  normal
 * (may be NULL): [n_px][3] composited voxel normals; max_weight (may be NULL):
 * [N], raised to the largest T_i alpha_i of each voxel over these pixels;
 * dist (may be NULL): [n_px] distortion loss of each pixel's ray.
 * Returns 0, or -1 on allocation failure. */
int oc_render_ex(double world_size, int64_t n_vox, const double *centre, const uint8_t *level,
                 const int32_t *corner_idx, const double *grid, const double *sh,
                 const oc_camera *cam, const oc_params *P, int64_t n_px, const int32_t *px_xy,
                 double *rgb, double *depth, double *alpha, double *t_final, int32_t *n_comp,
                 int64_t *term_vox, double *stop_margin, double *normal, double *max_weight, double *dist,
                 int n_threads) {
    oc_scene S = {world_size, n_vox, centre, level, corner_idx, grid, sh};
    if (P->K < 1 || P->K > OC_KMAX) return -2;
    int err = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        oc_scratch s;
        memset(&s, 0, sizeof(s));
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < n_px; ++p) {
            int x, y;
            pixel_xy(cam, n_px, px_xy, p, &x, &y);
            double ro[3], rd[3];
            oc_pixel_ray(cam, x, y, ro, rd);
            int64_t nh = gather_hits(&S, ro, rd, &s);
            oc_pixel_out o;
            if (nh < 0 || composite(&S, P, ro, rd, &s, nh, &o, normal != NULL, max_weight)) {
#pragma omp atomic write
                err = -1;
                continue;
            }
            for (int ch = 0; ch < 3; ++ch) rgb[3 * p + ch] = o.rgb[ch];
            depth[p] = o.depth;
            alpha[p] = o.alpha;
            t_final[p] = o.t_final;
            if (n_comp) n_comp[p] = o.n_comp;
            if (term_vox) term_vox[p] = o.term_vox;
            if (stop_margin) stop_margin[p] = o.stop_margin;
            if (normal)
                for (int ax = 0; ax < 3; ++ax) normal[3 * p + ax] = o.normal[ax];
            if (dist) dist[p] = o.dist;
        }
        scratch_free(&s);
    }
    return err;
}

int oc_render(double world_size, int64_t n_vox, const double *centre, const uint8_t *level,
              const int32_t *corner_idx, const double *grid, const double *sh,
              const oc_camera *cam, const oc_params *P, int64_t n_px, const int32_t *px_xy,
              double *rgb, double *depth, double *alpha, double *t_final, int32_t *n_comp,
              int64_t *term_vox, double *stop_margin, int n_threads) {
    return oc_render_ex(world_size, n_vox, centre, level, corner_idx, grid, sh, cam, P, n_px, px_xy, rgb, depth,
                        alpha, t_final, n_comp, term_vox, stop_margin, NULL, NULL, NULL, n_threads);
}

/* Gradient of sum_p (g_rgb[p] . C_p + g_depth[p] D_p + g_alpha[p] A_p) with
 * respect to grid (accumulated into d_grid[Pts]) and sh (accumulated into
 * d_sh[N][48]).  Same pixel convention as oc_render.  g_normal (may be NULL):
 * [n_px][3] upstream gradient of the normal image, which adds
 * sum_p g_normal[p] . N_p to the objective; g_dist (may be NULL): [n_px],
 * adds sum_p g_dist[p] L_dist,p; priority (may be NULL): [N],
 * accumulates the subdivision priority of Eq. (priority). */
int oc_render_grad_ex(double world_size, int64_t n_vox, const double *centre, const uint8_t *level,
                      const int32_t *corner_idx, const double *grid, const double *sh,
                      const oc_camera *cam, const oc_params *P, int64_t n_px, const int32_t *px_xy,
                      const double *g_rgb, const double *g_depth, const double *g_alpha, const double *g_normal,
                      const double *g_dist,
                      double *d_grid, double *d_sh, double *d_grid_abs, double *d_sh_abs,
                      double *d_grid_seg, double *d_sh_seg, double *priority, double *priority_seg,
                      int n_threads) {
    oc_scene S = {world_size, n_vox, centre, level, corner_idx, grid, sh};
    if (P->K < 1 || P->K > OC_KMAX) return -2;
    int err = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        oc_scratch s;
        memset(&s, 0, sizeof(s));
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < n_px; ++p) {
            int x, y;
            pixel_xy(cam, n_px, px_xy, p, &x, &y);
            double ro[3], rd[3];
            oc_pixel_ray(cam, x, y, ro, rd);
            int64_t nh = gather_hits(&S, ro, rd, &s);
            oc_pixel_out o;
            if (nh < 0 || composite(&S, P, ro, rd, &s, nh, &o, g_normal != NULL, NULL)) {
#pragma omp atomic write
                err = -1;
                continue;
            }
            pixel_backward(&S, P, ro, rd, &s, &o, g_rgb + 3 * p, g_depth[p], g_alpha[p],
                           g_normal ? g_normal + 3 * p : NULL, g_dist ? g_dist[p] : 0.0, d_grid, d_sh, d_grid_abs,
                           d_sh_abs, d_grid_seg,
                           d_sh_seg, priority, priority_seg);
        }
        scratch_free(&s);
    }
    return err;
}

int oc_render_grad(double world_size, int64_t n_vox, const double *centre, const uint8_t *level,
                   const int32_t *corner_idx, const double *grid, const double *sh,
                   const oc_camera *cam, const oc_params *P, int64_t n_px, const int32_t *px_xy,
                   const double *g_rgb, const double *g_depth, const double *g_alpha,
                   double *d_grid, double *d_sh, double *d_grid_abs, double *d_sh_abs,
                   double *d_grid_seg, double *d_sh_seg, int n_threads) {
    return oc_render_grad_ex(world_size, n_vox, centre, level, corner_idx, grid, sh, cam, P, n_px, px_xy, g_rgb,
                             g_depth, g_alpha, NULL, NULL, d_grid, d_sh, d_grid_abs, d_sh_abs, d_grid_seg,
                             d_sh_seg, NULL, NULL, n_threads);
}

/* Sorted hit list of an arbitrary ray (for order checks): writes up to cap
 * (a, b, voxel) triples and returns the number of hits (may exceed cap). */
int64_t oc_ray_hits(double world_size, int64_t n_vox, const double *centre, const uint8_t *level,
                    const double ro[3], const double rd[3], int64_t cap, double *a_out,
                    double *b_out, int64_t *v_out) {
    oc_scene S = {world_size, n_vox, centre, level, NULL, NULL, NULL};
    oc_scratch s;
    memset(&s, 0, sizeof(s));
    int64_t n = gather_hits(&S, ro, rd, &s);
    for (int64_t i = 0; i < n && i < cap; ++i) {
        a_out[i] = s.hits[i].a;
        b_out[i] = s.hits[i].b;
        v_out[i] = s.hits[i].v;
    }
    scratch_free(&s);
    return n;
}
