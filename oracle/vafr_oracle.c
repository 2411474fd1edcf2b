/*
 * vafr_oracle.c -- plain, slow FP64 CPU oracle of the VaFR ray-casting hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg load this library.  The product
 * (the CUDA library) never calls it, and the two share no code, header, table
 * or constant generator.
 *
 * Method: "Visual Acuity Consistent Foveated Rendering towards Retinal
 * Resolution" (Zhang, Gai, Li; arXiv 2503.23410).  Equation numbers follow the
 * paper's order of display equations:
 *   Eq. 2  linear MAR model  omega(e) = m e + omega0,  f = 1/omega   (Sec. 3.2.1)
 *   Eq. 3  r = tan(e)/c_r = |(x,y) - (x0,y0)|, trig in degrees      (Sec. 3.2.1)
 *   Eq. 4  du/de = 2 f(e)
 *   Eq. 5  u(e) = 2 ln(m e + omega0)/m + c0
 *   Eq. 6  tangential rate = radial rate,  r dtheta/dv = dr/du
 *   Eq. 7  de/dr = c_r cos^2(e) 180/pi
 *   Eq. 8  v(e, theta) = theta sin(2e)/(m e + omega0)
 *   Eq. 9  l(e) = v(e, 360 deg)                        (shading height)
 *   Eq. 10 e = (exp((u - c0) m/2) - omega0)/m           (Sec. 3.2.3)
 *   Eq. 11 x = r cos(v/l(e) 360) + x0, y = r sin(v/l(e) 360) + y0
 *   Eq. 12 the four-segment form of Eqs. 5 and 8        (Sec. 3.3)
 *   Eq. 13 SR(e) = f(e) = (1/2) du/de                   (Sec. 4.1)
 * Ray-casting pipeline: Sec. 6.1 (one ray per LP texel, closest-hit shading,
 * miss shading, inverse mapping to the display; GT = one ray per pixel).
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes): integration constants c_i fixed by u(0) = 0 and continuity at the
 * pivots; texel (c, j) sits at u = c + 0.5 and angle (j + 0.5) 360/n_c with
 * n_c = max(1, floor(l(e_c) + 0.5)); the angle is atan2 in display pixel
 * coordinates (y down) wrapped to [0, 360); eccentricity is clamped to e_max
 * in reconstruction; reconstruction is bilinear in (u, angle) with per-column
 * angular wrap; Lambert shading with ambient 0.1 and a sky gradient on miss;
 * two-sided watertight triangle test, closest t > 0, equal t -> lowest id.
 * The LBVH part (30-bit Morton codes, sort, Karras radix tree, bounds) is not
 * in the paper; it follows Karras 2012 "Maximizing Parallelism in the
 * Construction of BVHs, Octrees, and k-d Trees".
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (contraction off so
 * the FP32 Morton quantisation is one IEEE op at a time on every host).
 */

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_PIVOTS 9
#define OR_DEG (M_PI / 180.0)

/* ------------------------------------------------------------------------- */
/* Acuity model and the segmented log-polar mapping (Eqs. 2, 5, 8-10, 12)     */

typedef struct {
    int    n_seg;                 /* pivots - 1                               */
    double E[OR_MAX_PIVOTS];      /* pivot eccentricities (deg)               */
    double f[OR_MAX_PIVOTS];      /* acuity at the pivots (cycles/deg)        */
    double m[OR_MAX_PIVOTS];      /* MAR slope of segment i (Eq. 2)           */
    double w0[OR_MAX_PIVOTS];     /* MAR intercept omega_i of segment i       */
    double c[OR_MAX_PIVOTS];      /* integration constant c_i (Eq. 12)        */
    int    aniso;                 /* 0: Delta(e) = 1 (isotropic, Eq. 8)       */
    double delta[OR_MAX_PIVOTS];  /* Delta at the pivots (Eq. 19)             */
} or_acuity;

/* u on segment i in the paper's literal form 2 ln(m_i e + w_i)/m_i + c_i,
 * or its m -> 0 limit 2 e / w_i + c_i (constant acuity on the segment). */
static double seg_u(const or_acuity* a, int i, double e) {
    if (a->m[i] == 0.0) return 2.0 * e / a->w0[i] + a->c[i];
    return 2.0 * log(a->m[i] * e + a->w0[i]) / a->m[i] + a->c[i];
}

/* Segment table from the pivots (Eq. 12, Sec. 3.3): MAR omega = 1/f is taken
 * piecewise linear through the pivots (E_k, 1/f_k); c_1 makes u(0) = 0 and
 * each later c_i makes u continuous at E_{i-1}.  Returns 0 or -1 on bad input. */
int or_acuity_init(or_acuity* a, const double* E, const double* f, int n_piv) {
    if (n_piv < 2 || n_piv > OR_MAX_PIVOTS) return -1;
    memset(a, 0, sizeof(*a));
    a->n_seg = n_piv - 1;
    for (int k = 0; k < n_piv; ++k) {
        if (!(f[k] > 0.0)) return -1;
        if (k > 0 && !(E[k] > E[k - 1])) return -1;
        a->E[k] = E[k];
        a->f[k] = f[k];
    }
    if (E[0] != 0.0) return -1;
    for (int i = 0; i < a->n_seg; ++i) {
        double w_lo = 1.0 / f[i], w_hi = 1.0 / f[i + 1];
        a->m[i] = (w_hi - w_lo) / (E[i + 1] - E[i]);
        a->w0[i] = w_lo - a->m[i] * E[i];
    }
    /* u(0) = 0 on segment 0; continuity at every inner pivot. */
    a->c[0] = 0.0;
    a->c[0] = -seg_u(a, 0, 0.0);
    for (int i = 1; i < a->n_seg; ++i) {
        double u_end = seg_u(a, i - 1, E[i]);
        a->c[i] = 0.0;
        a->c[i] = u_end - seg_u(a, i, E[i]);
    }
    return 0;
}

/* Segment holding eccentricity e: [E_i, E_{i+1}); beyond the last pivot the
 * last segment's formula is extended. */
static int seg_of_e(const or_acuity* a, double e) {
    for (int i = 0; i < a->n_seg - 1; ++i)
        if (e < a->E[i + 1]) return i;
    return a->n_seg - 1;
}

/* MAR omega(e) (deg/cycle), Eq. 2 per segment. */
double or_omega(const or_acuity* a, double e) {
    int i = seg_of_e(a, e);
    return a->m[i] * e + a->w0[i];
}

/* Acuity f(e) = 1/omega(e) (cycles/deg), Eq. 2. */
double or_acuity_f(const or_acuity* a, double e) { return 1.0 / or_omega(a, e); }

/* LP horizontal coordinate u(e), Eqs. 5 / 12. */
double or_u_of_e(const or_acuity* a, double e) { return seg_u(a, seg_of_e(a, e), e); }

/* Inverse, Eq. 10 per segment: e = (exp((u - c_i) m_i / 2) - omega_i) / m_i. */
double or_e_of_u(const or_acuity* a, double u) {
    int i = a->n_seg - 1;
    for (int k = 0; k < a->n_seg - 1; ++k) {
        if (u < seg_u(a, k, a->E[k + 1])) { i = k; break; }
    }
    if (a->m[i] == 0.0) return (u - a->c[i]) * a->w0[i] / 2.0;
    return (exp((u - a->c[i]) * a->m[i] / 2.0) - a->w0[i]) / a->m[i];
}

/* v(e, theta) = theta sin(2e)/(m e + omega), Eq. 8 / 12 (theta in degrees). */
double or_v_of_e_theta(const or_acuity* a, double e, double theta_deg) {
    return theta_deg * sin(2.0 * e * OR_DEG) / or_omega(a, e);
}

/* Shading height l(e) = v(e, 360 deg), Eq. 9. */
double or_l_of_e(const or_acuity* a, double e) { return or_v_of_e_theta(a, e, 360.0); }

/* Anisotropic acuity (Sec. 9, Eq. 19): the tangential shading rate is Delta(e)
 * times the radial one, v(e, theta) = Delta(e) theta sin(2e)/(m e + omega).
 * The paper leaves Delta's form open; here it is piecewise linear in e
 * through (E_k, delta_k) and constant past the last pivot.  Returns -1 unless
 * every delta_k > 0. */
int or_acuity_set_delta(or_acuity* a, const double* delta) {
    for (int k = 0; k <= a->n_seg; ++k)
        if (!(delta[k] > 0.0)) return -1;
    for (int k = 0; k <= a->n_seg; ++k) a->delta[k] = delta[k];
    a->aniso = 1;
    return 0;
}

double or_delta(const or_acuity* a, double e) {
    if (!a->aniso) return 1.0;
    if (e >= a->E[a->n_seg]) return a->delta[a->n_seg];
    int i = 0;
    while (i + 1 < a->n_seg && e >= a->E[i + 1]) ++i;
    double s = (e - a->E[i]) / (a->E[i + 1] - a->E[i]);
    return a->delta[i] + s * (a->delta[i + 1] - a->delta[i]);
}

/* Texels per column before rounding: Delta(e) l(e) (Eq. 19 at theta = 360). */
double or_l_delta_of_e(const or_acuity* a, double e) { return or_delta(a, e) * or_l_of_e(a, e); }

/* Vectorised helpers for the Python side. */
void or_eval(const or_acuity* a, int what, const double* in, double* out, int64_t n) {
    for (int64_t k = 0; k < n; ++k) {
        switch (what) {
            case 0: out[k] = or_u_of_e(a, in[k]); break;
            case 1: out[k] = or_e_of_u(a, in[k]); break;
            case 2: out[k] = or_l_of_e(a, in[k]); break;
            case 3: out[k] = or_acuity_f(a, in[k]); break;
            case 4: out[k] = or_delta(a, in[k]); break;
            default: out[k] = NAN;
        }
    }
}

int64_t or_sizeof_acuity(void) { return (int64_t)sizeof(or_acuity); }

void or_acuity_get(const or_acuity* a, double* m, double* w0, double* c) {
    for (int i = 0; i < a->n_seg; ++i) { m[i] = a->m[i]; w0[i] = a->w0[i]; c[i] = a->c[i]; }
}

/* ------------------------------------------------------------------------- */
/* Discrete LP layout (Sec. 3.2.2): columns at u = c + 0.5 for c + 0.5 < u(e_max);
 * column c holds n_c = max(1, round(Delta(e_c) l(e_c))) texels at angles
 * (j+0.5) 360/n_c (Delta = 1 unless the acuity is anisotropic, Sec. 9).
 * Texels are stored column after column: texel (c, j) at offset_c + j.
 * Returns the column count, or -1 if it would exceed cap. */
int or_lp_layout(const or_acuity* a, double e_max, int cap,
                 double* e_col, int32_t* n_col, int64_t* off_col, int64_t* total) {
    double u_max = or_u_of_e(a, e_max);
    int C = 0;
    while ((double)C + 0.5 < u_max) ++C;
    if (C > cap) return -1;
    int64_t acc = 0;
    for (int c = 0; c < C; ++c) {
        double e = or_e_of_u(a, (double)c + 0.5);
        double l = or_l_delta_of_e(a, e);
        int32_t n = (int32_t)floor(l + 0.5);
        if (n < 1) n = 1;
        e_col[c] = e;
        n_col[c] = n;
        off_col[c] = acc;
        acc += n;
    }
    *total = acc;
    return C;
}

/* ------------------------------------------------------------------------- */
/* Views: pinhole camera, pose [R | t] camera -> world (x right, y up, z fwd). */

typedef struct {
    double width, height;   /* display size in pixels                        */
    double fov_v_deg;       /* vertical field of view                        */
    double x0, y0;          /* gaze point (display pixels, y down)           */
    double pose[12];        /* row-major 3x4                                 */
} or_view;

/* c_r (Sec. 3.2.1): film height / focal length / display height in pixels. */
static double view_cr(const or_view* v) {
    return 2.0 * tan(0.5 * v->fov_v_deg * OR_DEG) / v->height;
}

/* Primary ray through display point (x, y) (continuous pixel coordinates). */
static void view_ray(const or_view* v, double x, double y, double o[3], double d[3]) {
    double cr = view_cr(v);
    double dc[3] = {cr * (x - 0.5 * v->width), cr * (0.5 * v->height - y), 1.0};
    for (int k = 0; k < 3; ++k) {
        d[k] = v->pose[4 * k + 0] * dc[0] + v->pose[4 * k + 1] * dc[1] + v->pose[4 * k + 2] * dc[2];
        o[k] = v->pose[4 * k + 3];
    }
}

/* Screen point of LP texel (c, j) by the inverse mapping (Eqs. 3, 10, 11):
 * e_c from the layout, r = tan(e_c)/c_r, angle = (j + 0.5)/n_c * 360 deg. */
static void texel_screen_point(const or_view* v, double e_c, int32_t n_c, int64_t j,
                               double* x, double* y) {
    double r = tan(e_c * OR_DEG) / view_cr(v);
    double ang = ((double)j + 0.5) / (double)n_c * 360.0;
    *x = r * cos(ang * OR_DEG) + v->x0;
    *y = r * sin(ang * OR_DEG) + v->y0;
}

/* Rays for a list of LP texels given by global texel index (Sec. 6.1). */
void or_lp_rays(const or_view* v, const double* e_col, const int32_t* n_col,
                const int64_t* off_col, int n_cols, const int64_t* texels, int64_t n,
                double* orig, double* dir, double* screen_xy) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        int64_t t = texels[k];
        int lo = 0, hi = n_cols - 1;           /* column with off_col[c] <= t */
        while (lo < hi) {
            int mid = (lo + hi + 1) / 2;
            if (off_col[mid] <= t) lo = mid; else hi = mid - 1;
        }
        double x, y;
        texel_screen_point(v, e_col[lo], n_col[lo], t - off_col[lo], &x, &y);
        view_ray(v, x, y, orig + 3 * k, dir + 3 * k);
        if (screen_xy) { screen_xy[2 * k] = x; screen_xy[2 * k + 1] = y; }
    }
}

/* Rays through display pixel centres (x + 0.5, y + 0.5), pixel id = y W + x. */
void or_pixel_rays(const or_view* v, const int64_t* pix, int64_t n, double* orig, double* dir) {
    int64_t W = (int64_t)v->width;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double x = (double)(pix[k] % W) + 0.5, y = (double)(pix[k] / W) + 0.5;
        view_ray(v, x, y, orig + 3 * k, dir + 3 * k);
    }
}

/* ------------------------------------------------------------------------- */
/* Watertight ray / triangle test (Woop, Benthin, Wald 2013, JCGT 2(1)),
 * two-sided, in FP64.  Hit iff all edge functions share a sign (zero counts
 * as inside, so a ray through a shared edge hits both neighbours), the
 * determinant is non-zero and t > 0. */

typedef struct { int kx, ky, kz; double Sx, Sy, Sz; double o[3]; } or_wray;

static void wray_init(or_wray* r, const double o[3], const double d[3]) {
    double ax = fabs(d[0]), ay = fabs(d[1]), az = fabs(d[2]);
    int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (d[kz] < 0.0) { int s = kx; kx = ky; ky = s; }
    r->kx = kx; r->ky = ky; r->kz = kz;
    r->Sx = d[kx] / d[kz];
    r->Sy = d[ky] / d[kz];
    r->Sz = 1.0 / d[kz];
    r->o[0] = o[0]; r->o[1] = o[1]; r->o[2] = o[2];
}

/* Vertices in lexicographic (x, y, z) order: the two-sided test and the hit
 * rule do not depend on vertex order, so evaluating every triangle in one
 * canonical order makes identical triangles tie exactly in FP64 as well. */
static void canonical_vertices(const float* tri, const float* v[3]) {
    v[0] = tri; v[1] = tri + 3; v[2] = tri + 6;
    for (int pass = 0; pass < 3; ++pass) {
        int i = pass == 1 ? 1 : 0, j = i + 1;
        const float* a = v[i];
        const float* b = v[j];
        int b_first = b[0] < a[0] || (b[0] == a[0] && (b[1] < a[1] || (b[1] == a[1] && b[2] < a[2])));
        if (b_first) { v[i] = b; v[j] = a; }
    }
}

static int wray_hit(const or_wray* r, const float* tri, double* t_out) {
    const float* v[3];
    canonical_vertices(tri, v);
    double A[3], B[3], C[3];
    for (int k = 0; k < 3; ++k) {
        A[k] = (double)v[0][k] - r->o[k];
        B[k] = (double)v[1][k] - r->o[k];
        C[k] = (double)v[2][k] - r->o[k];
    }
    double Ax = A[r->kx] - r->Sx * A[r->kz], Ay = A[r->ky] - r->Sy * A[r->kz];
    double Bx = B[r->kx] - r->Sx * B[r->kz], By = B[r->ky] - r->Sy * B[r->kz];
    double Cx = C[r->kx] - r->Sx * C[r->kz], Cy = C[r->ky] - r->Sy * C[r->kz];
    double U = Cx * By - Cy * Bx;
    double V = Ax * Cy - Ay * Cx;
    double W = Bx * Ay - By * Ax;
    if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0)) return 0;
    double det = U + V + W;
    if (det == 0.0) return 0;
    double Az = r->Sz * A[r->kz], Bz = r->Sz * B[r->kz], Cz = r->Sz * C[r->kz];
    double T = U * Az + V * Bz + W * Cz;
    double t = T / det;
    if (!(t > 0.0)) return 0;
    *t_out = t;
    return 1;
}

/* Signed distance-like margin of the ray from the triangle's boundary in the
 * sheared 2-D frame: min over edges of (edge function / edge length), signed
 * so that > 0 means inside.  Used by tests to classify edge ties. */
double or_edge_margin(const double* o, const double* d, const float* tri) {
    or_wray r;
    wray_init(&r, o, d);
    double P[3][2];
    for (int v = 0; v < 3; ++v) {
        double a[3];
        for (int k = 0; k < 3; ++k) a[k] = (double)tri[3 * v + k] - o[k];
        P[v][0] = a[r.kx] - r.Sx * a[r.kz];
        P[v][1] = a[r.ky] - r.Sy * a[r.kz];
    }
    double area = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[1][1] - P[0][1]) * (P[2][0] - P[0][0]);
    double sgn = area >= 0.0 ? 1.0 : -1.0;
    double best = INFINITY;
    for (int e = 0; e < 3; ++e) {
        const double* p = P[e];
        const double* q = P[(e + 1) % 3];
        double ex = q[0] - p[0], ey = q[1] - p[1];
        double len = sqrt(ex * ex + ey * ey);
        double fn = (ex * (0.0 - p[1]) - ey * (0.0 - p[0])) * sgn;
        double dist = len > 0.0 ? fn / len : -INFINITY;
        if (dist < best) best = dist;
    }
    return best;
}

/* Closest hit by brute force over all triangles: closest t > 0, equal t ->
 * lowest triangle id (loop in id order, strict comparison).  -1 on a miss. */
void or_cast_brute(const float* tris, int64_t n_tris, const double* orig, const double* dir,
                   int64_t n_rays, int32_t* hit_id, double* hit_t) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n_rays; ++k) {
        or_wray r;
        wray_init(&r, orig + 3 * k, dir + 3 * k);
        int32_t best = -1;
        double bt = INFINITY;
        for (int64_t i = 0; i < n_tris; ++i) {
            double t;
            if (wray_hit(&r, tris + 9 * i, &t) && t < bt) { bt = t; best = (int32_t)i; }
        }
        hit_id[k] = best;
        hit_t[k] = best >= 0 ? bt : INFINITY;
    }
}

/* t of a ray against one given triangle (INFINITY if no hit). */
void or_ray_tri_t(const float* tris, const int32_t* ids, const double* orig, const double* dir,
                  int64_t n, double* t_out) {
    for (int64_t k = 0; k < n; ++k) {
        or_wray r;
        double t;
        wray_init(&r, orig + 3 * k, dir + 3 * k);
        t_out[k] = (ids[k] >= 0 && wray_hit(&r, tris + 9 * (int64_t)ids[k], &t)) ? t : INFINITY;
    }
}

/* ------------------------------------------------------------------------- */
/* CPU BVH (object-median split, FP64 padded boxes).  Speeds up large scenes;
 * its result equals brute force exactly because boxes are conservative and
 * triangles use the same test and tie rule. */

typedef struct {
    double lo[3], hi[3];
    int32_t left, right;      /* children (internal) or -1                   */
    int32_t first, count;     /* triangle range in `order` for leaves         */
} or_bnode;

typedef struct {
    const float* tris;
    int64_t n_tris;
    int32_t* order;
    or_bnode* nodes;
    int32_t n_nodes;
    double* cen;
} or_bvh;

static void tri_box(const float* t, double lo[3], double hi[3]) {
    for (int k = 0; k < 3; ++k) {
        double a = t[k], b = t[3 + k], c = t[6 + k];
        lo[k] = fmin(a, fmin(b, c));
        hi[k] = fmax(a, fmax(b, c));
    }
}

static const double* g_sort_cen;
static int g_sort_axis;
static int cmp_cen(const void* pa, const void* pb) {
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    double ca = g_sort_cen[3 * a + g_sort_axis], cb = g_sort_cen[3 * b + g_sort_axis];
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return (a > b) - (a < b);
}

static int32_t bvh_build_rec(or_bvh* b, int32_t first, int32_t count) {
    int32_t id = b->n_nodes++;
    or_bnode* nd = &b->nodes[id];
    for (int k = 0; k < 3; ++k) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t i = first; i < first + count; ++i) {
        double lo[3], hi[3];
        int32_t t = b->order[i];
        tri_box(b->tris + 9 * (int64_t)t, lo, hi);
        for (int k = 0; k < 3; ++k) {
            nd->lo[k] = fmin(nd->lo[k], lo[k]);
            nd->hi[k] = fmax(nd->hi[k], hi[k]);
            clo[k] = fmin(clo[k], b->cen[3 * t + k]);
            chi[k] = fmax(chi[k], b->cen[3 * t + k]);
        }
    }
    for (int k = 0; k < 3; ++k) {          /* pad so FP64 slab tests stay conservative */
        double pad = 1e-9 * (1.0 + fabs(nd->lo[k]) + fabs(nd->hi[k]));
        nd->lo[k] -= pad;
        nd->hi[k] += pad;
    }
    if (count <= 4) {
        nd->left = nd->right = -1;
        nd->first = first;
        nd->count = count;
        return id;
    }
    int axis = 0;
    for (int k = 1; k < 3; ++k)
        if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
    g_sort_cen = b->cen;
    g_sort_axis = axis;
    qsort(b->order + first, (size_t)count, sizeof(int32_t), cmp_cen);
    int32_t half = count / 2;
    int32_t l = bvh_build_rec(b, first, half);
    int32_t r = bvh_build_rec(b, first + half, count - half);
    nd = &b->nodes[id];
    nd->left = l;
    nd->right = r;
    nd->first = -1;
    nd->count = 0;
    return id;
}

void* or_bvh_build(const float* tris, int64_t n_tris) {
    or_bvh* b = (or_bvh*)calloc(1, sizeof(or_bvh));
    b->tris = tris;
    b->n_tris = n_tris;
    b->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_tris > 0 ? n_tris : 1));
    b->nodes = (or_bnode*)malloc(sizeof(or_bnode) * (size_t)(2 * n_tris + 1));
    b->cen = (double*)malloc(sizeof(double) * 3 * (size_t)(n_tris > 0 ? n_tris : 1));
    for (int64_t i = 0; i < n_tris; ++i) {
        b->order[i] = (int32_t)i;
        for (int k = 0; k < 3; ++k)
            b->cen[3 * i + k] = ((double)tris[9 * i + k] + tris[9 * i + 3 + k] + tris[9 * i + 6 + k]) / 3.0;
    }
    if (n_tris > 0) bvh_build_rec(b, 0, (int32_t)n_tris);
    free(b->cen);
    b->cen = NULL;
    return b;
}

void or_bvh_free(void* p) {
    or_bvh* b = (or_bvh*)p;
    if (!b) return;
    free(b->order);
    free(b->nodes);
    free(b);
}

static int box_enter(const or_bnode* nd, const double o[3], const double inv[3], double tmax) {
    double t0 = 0.0, t1 = tmax;
    for (int k = 0; k < 3; ++k) {
        double a = (nd->lo[k] - o[k]) * inv[k], c = (nd->hi[k] - o[k]) * inv[k];
        if (isnan(a) || isnan(c)) {                 /* ray parallel, origin on the slab */
            if (o[k] < nd->lo[k] || o[k] > nd->hi[k]) return 0;
            continue;
        }
        double lo = fmin(a, c), hi = fmax(a, c);
        if (lo > t0) t0 = lo;
        if (hi < t1) t1 = hi;
    }
    return t0 <= t1 * (1.0 + 1e-12);
}

/* Closest hit of one ray through the CPU BVH, ignoring triangle `skip` (-1:
 * none); returns the id or -1 and the distance in *t_out. */
static int32_t bvh_closest(const or_bvh* b, const double o[3], const double d[3], int32_t skip,
                           double* t_out) {
    or_wray r;
    wray_init(&r, o, d);
    double inv[3] = {1.0 / d[0], 1.0 / d[1], 1.0 / d[2]};
    int32_t best = -1;
    double bt = INFINITY;
    int32_t stack[128];
    int sp = 0;
    if (b->n_tris > 0) stack[sp++] = 0;
    while (sp > 0) {
        const or_bnode* nd = &b->nodes[stack[--sp]];
        if (!box_enter(nd, o, inv, bt)) continue;
        if (nd->left < 0) {
            for (int32_t i = nd->first; i < nd->first + nd->count; ++i) {
                int32_t tid = b->order[i];
                double t;
                if (tid != skip && wray_hit(&r, b->tris + 9 * (int64_t)tid, &t) &&
                    (t < bt || (t == bt && tid < best))) {
                    bt = t;
                    best = tid;
                }
            }
        } else if (sp + 2 <= 128) {
            stack[sp++] = nd->right;
            stack[sp++] = nd->left;
        }
    }
    *t_out = best >= 0 ? bt : INFINITY;
    return best;
}

void or_cast_bvh(void* p, const double* orig, const double* dir, int64_t n_rays,
                 int32_t* hit_id, double* hit_t) {
    const or_bvh* b = (const or_bvh*)p;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n_rays; ++k)
        hit_id[k] = bvh_closest(b, orig + 3 * k, dir + 3 * k, -1, hit_t + k);
}

/* ------------------------------------------------------------------------- */
/* Shading (Sec. 6.1: closest-hit and miss shaders; the paper does not print
 * its shading code).  Lambert with a directional light and ambient k_a
 * (plus any point lights, or_shade_points):
 *   rgb = albedo (k_a + (1 - k_a) max(0, n . (-L))),
 * n = geometric unit normal turned to face the ray origin; a miss returns the
 * sky gradient lerp((1,1,1), (0.5,0.7,1.0), (dhat_y + 1)/2).  Alpha = 1. */

#define OR_KA 0.1

/* Point lights (the deferred pipeline's scenes carry many lights, Sec. 5.2):
 * each adds albedo * rgb_k * max(0, n . l_k) / |x_k - p|^2 at hit point p,
 * l_k the unit vector to the light; no shadows. */
void or_shade_points(const float* tris, const float* albedo, const double* orig, const double* dir,
                     const int32_t* hit_id, const double* hit_t, int64_t n, int n_pl, const double* pl_pos,
                     const double* pl_rgb, double* rgba) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        if (hit_id[k] < 0 || n_pl <= 0) continue;
        const double* d = dir + 3 * k;
        const float* t = tris + 9 * (int64_t)hit_id[k];
        double e1[3], e2[3], nrm[3], p[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = (double)t[3 + a] - t[a];
            e2[a] = (double)t[6 + a] - t[a];
            p[a] = orig[3 * k + a] + hit_t[k] * d[a];
        }
        nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double nl = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        for (int a = 0; a < 3; ++a) nrm[a] /= nl;
        if (nrm[0] * d[0] + nrm[1] * d[1] + nrm[2] * d[2] > 0.0)
            for (int a = 0; a < 3; ++a) nrm[a] = -nrm[a];
        const float* al = albedo + 3 * (int64_t)hit_id[k];
        for (int q = 0; q < n_pl; ++q) {
            double l[3], d2 = 0.0;
            for (int a = 0; a < 3; ++a) { l[a] = pl_pos[3 * q + a] - p[a]; d2 += l[a] * l[a]; }
            double cosl = (nrm[0] * l[0] + nrm[1] * l[1] + nrm[2] * l[2]) / sqrt(d2);
            if (cosl <= 0.0) continue;
            for (int a = 0; a < 3; ++a) rgba[4 * k + a] += al[a] * pl_rgb[3 * q + a] * cosl / d2;
        }
    }
}

void or_shade(const float* tris, const float* albedo, const double* light_dir,
              const double* dir, const int32_t* hit_id, int64_t n, double* rgba) {
    double L[3] = {light_dir[0], light_dir[1], light_dir[2]};
    double ln = sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
    for (int k = 0; k < 3; ++k) L[k] /= ln;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        const double* d = dir + 3 * k;
        double* out = rgba + 4 * k;
        if (hit_id[k] < 0) {
            double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double s = 0.5 * (d[1] / dl + 1.0);
            out[0] = (1.0 - s) * 1.0 + s * 0.5;
            out[1] = (1.0 - s) * 1.0 + s * 0.7;
            out[2] = (1.0 - s) * 1.0 + s * 1.0;
            out[3] = 1.0;
            continue;
        }
        const float* t = tris + 9 * (int64_t)hit_id[k];
        double e1[3], e2[3], nrm[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = (double)t[3 + a] - t[a];
            e2[a] = (double)t[6 + a] - t[a];
        }
        nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double nl = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        for (int a = 0; a < 3; ++a) nrm[a] /= nl;
        if (nrm[0] * d[0] + nrm[1] * d[1] + nrm[2] * d[2] > 0.0)
            for (int a = 0; a < 3; ++a) nrm[a] = -nrm[a];
        double lam = -(nrm[0] * L[0] + nrm[1] * L[1] + nrm[2] * L[2]);
        if (lam < 0.0) lam = 0.0;
        double s = OR_KA + (1.0 - OR_KA) * lam;
        const float* al = albedo + 3 * (int64_t)hit_id[k];
        out[0] = al[0] * s;
        out[1] = al[1] * s;
        out[2] = al[2] * s;
        out[3] = 1.0;
    }
}

/* |n_hat . d_hat| of the hit triangle (grazing-ray classifier for tests). */
void or_grazing(const float* tris, const double* dir, const int32_t* hit_id, int64_t n, double* out) {
    for (int64_t k = 0; k < n; ++k) {
        if (hit_id[k] < 0) { out[k] = 1.0; continue; }
        const float* t = tris + 9 * (int64_t)hit_id[k];
        const double* d = dir + 3 * k;
        double e1[3], e2[3], nrm[3];
        for (int a = 0; a < 3; ++a) { e1[a] = (double)t[3 + a] - t[a]; e2[a] = (double)t[6 + a] - t[a]; }
        nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double nl = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        out[k] = fabs(nrm[0] * d[0] + nrm[1] * d[1] + nrm[2] * d[2]) / (nl * dl);
    }
}

/* ------------------------------------------------------------------------- */
/* Reconstruction (Sec. 3.4 inverse-mapping pass; Eqs. 3, 5/12 forward map).
 * For a display point (x, y): r = |(x,y) - (x0,y0)|, e = atan(c_r r) (deg,
 * clamped to e_max), u = u(e), angle = atan2(y - y0, x - x0) in [0, 360).
 * Bilinear filter: columns floor(u - 0.5) and +1 (clamped to [0, C-1]); in
 * each column rows floor(angle n_c/360 - 0.5) and +1, wrapped modulo n_c. */

static void column_sample(const double* lp, int nch, int64_t off, int32_t n, double ang,
                          double* acc, double w) {
    double v = ang / 360.0 * (double)n - 0.5;
    double j0f = floor(v);
    double wv = v - j0f;
    int64_t j0 = (int64_t)j0f;
    int64_t j1 = j0 + 1;
    j0 = ((j0 % n) + n) % n;
    j1 = ((j1 % n) + n) % n;
    for (int ch = 0; ch < nch; ++ch)
        acc[ch] += w * ((1.0 - wv) * lp[(off + j0) * nch + ch] + wv * lp[(off + j1) * nch + ch]);
}

void or_reconstruct_points(const or_acuity* a, double e_max, const or_view* v,
                           const int32_t* n_col, const int64_t* off_col, int n_cols,
                           const double* lp, int nch, const double* pts, int64_t n, double* out) {
    double cr = view_cr(v);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double dx = pts[2 * k] - v->x0, dy = pts[2 * k + 1] - v->y0;
        double r = sqrt(dx * dx + dy * dy);
        double e = atan(cr * r) / OR_DEG;
        if (e > e_max) e = e_max;
        double u = or_u_of_e(a, e);
        double ang = atan2(dy, dx) / OR_DEG;
        if (ang < 0.0) ang += 360.0;
        double uf = u - 0.5;
        if (uf < 0.0) uf = 0.0;
        if (uf > (double)(n_cols - 1)) uf = (double)(n_cols - 1);
        int c0 = (int)floor(uf);
        double wu = uf - c0;
        int c1 = c0 + 1 < n_cols ? c0 + 1 : n_cols - 1;
        double acc[8] = {0};
        column_sample(lp, nch, off_col[c0], n_col[c0], ang, acc, 1.0 - wu);
        column_sample(lp, nch, off_col[c1], n_col[c1], ang, acc, wu);
        for (int ch = 0; ch < nch; ++ch) out[k * nch + ch] = acc[ch];
    }
}

/* ------------------------------------------------------------------------- */
/* LBVH reference (Karras 2012).  Morton codes from the centroid sum
 * s = (v0 + v1) + v2 in FP32, quantised on a cubic grid spanning the largest
 * extent of the scene's s-bounds, one IEEE FP32 op at a time:
 *   ext = max over axes of (hi - lo),  q = min((uint)((s - lo)/ext * 1024), 1023)
 * (q = 0 for every axis when ext = 0); 10 bits per axis interleaved x-major
 * (x bit b -> code bit 3b+2, y -> 3b+1, z -> 3b).  A cubic grid splits long
 * axes before short ones (a terrain is not cut along its thin height axis
 * as often as along its extent). */

static uint32_t spread10(uint32_t q) {
    uint32_t out = 0;
    for (int b = 0; b < 10; ++b) out |= ((q >> b) & 1u) << (3 * b);
    return out;
}

void or_morton(const float* tris, int64_t n, uint32_t* codes) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float* s = (float*)malloc(sizeof(float) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            volatile float a = tris[9 * i + k] + tris[9 * i + 3 + k];
            float v = a + tris[9 * i + 6 + k];
            s[3 * i + k] = v;
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    volatile float ext = 0.0f;
    for (int k = 0; k < 3; ++k) {
        volatile float e = hi[k] - lo[k];
        if (e > ext) ext = e;
    }
    for (int64_t i = 0; i < n; ++i) {
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            if (!(ext > 0.0f)) { q[k] = 0; continue; }
            volatile float num = s[3 * i + k] - lo[k];
            volatile float t = num / ext;
            volatile float sc = t * 1024.0f;
            uint32_t qi = (uint32_t)sc;
            q[k] = qi > 1023u ? 1023u : qi;
        }
        codes[i] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    }
    free(s);
}

/* Sort by (code, id): qsort with a total order on the pair. */
static const uint32_t* g_codes;
static int cmp_code(const void* pa, const void* pb) {
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    if (g_codes[a] != g_codes[b]) return g_codes[a] < g_codes[b] ? -1 : 1;
    return (a > b) - (a < b);
}

/* Key of sorted position i: code in the high word, position in the low word,
 * so equal codes still give distinct keys (Karras 2012, Sec. 4). */
static uint64_t rkey(const uint32_t* sc, int64_t i) { return ((uint64_t)sc[i] << 32) | (uint64_t)i; }

static int hibit64(uint64_t x) { int b = 63; while (!((x >> b) & 1u)) --b; return b; }

/* Top-down binary radix tree over sorted keys.  Range [f, l] (f < l) splits
 * at the highest bit where keys f and l differ: the left child takes the keys
 * with that bit 0.  Node numbering (Karras 2012): the root is internal node 0;
 * a child covering [a, b] is leaf a when a == b, else internal node gamma for
 * the left child and gamma + 1 for the right child, gamma the split.
 * child refs: >= 0 internal node, < 0 leaf ~k (k = sorted position). */
static void radix_rec(const uint32_t* sc, int64_t f, int64_t l, int32_t node,
                      int32_t* child, int32_t* parent_of_node, int32_t* range) {
    uint64_t kf = rkey(sc, f), kl = rkey(sc, l);
    int b = hibit64(kf ^ kl);
    int64_t lo = f, hi = l;                  /* last index with bit b == 0 */
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if ((rkey(sc, mid) >> b) & 1u) hi = mid - 1; else lo = mid;
    }
    int64_t g = lo;
    range[2 * node] = (int32_t)f;
    range[2 * node + 1] = (int32_t)l;
    int32_t L = (g == f) ? ~(int32_t)g : (int32_t)g;
    int32_t R = (g + 1 == l) ? ~(int32_t)(g + 1) : (int32_t)(g + 1);
    child[2 * node] = L;
    child[2 * node + 1] = R;
    if (L >= 0) { parent_of_node[L] = node; radix_rec(sc, f, g, L, child, parent_of_node, range); }
    if (R >= 0) { parent_of_node[R] = node; radix_rec(sc, g + 1, l, R, child, parent_of_node, range); }
}

/* Full LBVH reference: codes (input order), sorted ids, child refs of the
 * n - 1 internal nodes, per-internal-node and per-leaf FP32 bounds
 * (lo xyz, hi xyz).  Returns 0 or -1. */
int or_lbvh(const float* tris, int64_t n, uint32_t* codes, int32_t* sorted_ids,
            int32_t* child, float* node_box, float* leaf_box, int32_t* range) {
    if (n <= 0) return 0;
    or_morton(tris, n, codes);
    for (int64_t i = 0; i < n; ++i) sorted_ids[i] = (int32_t)i;
    g_codes = codes;
    qsort(sorted_ids, (size_t)n, sizeof(int32_t), cmp_code);
    uint32_t* sc = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) sc[i] = codes[sorted_ids[i]];
    for (int64_t i = 0; i < n; ++i) {
        const float* t = tris + 9 * (int64_t)sorted_ids[i];
        for (int k = 0; k < 3; ++k) {
            float a = t[k], b = t[3 + k], c = t[6 + k];
            float lo = a < b ? a : b; lo = lo < c ? lo : c;
            float hi = a > b ? a : b; hi = hi > c ? hi : c;
            leaf_box[6 * i + k] = lo;
            leaf_box[6 * i + 3 + k] = hi;
        }
    }
    if (n == 1) { free(sc); return 0; }
    int32_t* par = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    par[0] = -1;
    radix_rec(sc, 0, n - 1, 0, child, par, range);
    /* bounds: an internal node's box is the union of its children's boxes;
     * evaluate children first (post-order by descending range size works). */
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n - 1));
    int32_t* stk = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n - 1));
    int64_t no = 0, sp = 0;
    stk[sp++] = 0;
    while (sp > 0) {                          /* pre-order; reversed = children first */
        int32_t v = stk[--sp];
        order[no++] = v;
        for (int s = 0; s < 2; ++s)
            if (child[2 * v + s] >= 0) stk[sp++] = child[2 * v + s];
    }
    for (int64_t q = no - 1; q >= 0; --q) {
        int32_t v = order[q];
        float* box = node_box + 6 * (int64_t)v;
        for (int k = 0; k < 3; ++k) { box[k] = INFINITY; box[3 + k] = -INFINITY; }
        for (int s = 0; s < 2; ++s) {
            int32_t ch = child[2 * v + s];
            const float* cb = ch >= 0 ? node_box + 6 * (int64_t)ch : leaf_box + 6 * (int64_t)(~ch);
            for (int k = 0; k < 3; ++k) {
                if (cb[k] < box[k]) box[k] = cb[k];
                if (cb[3 + k] > box[3 + k]) box[3 + k] = cb[3 + k];
            }
        }
    }
    free(order);
    free(stk);
    free(par);
    free(sc);
    return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Anti-aliasing inside the LP buffer (Sec. 3.4 "internal anti-aliasing";
 * Sec. 7 ablation).  The paper runs FXAA (Lottes 2009) on the LP buffer and
 * gives no parameters.  This is that method on the LP grid, in its steps:
 *
 *  grid      texel (c, j); along the angle its neighbours are (c, j -+ 1)
 *            modulo n_c; across the radius, column c' = c -+ 1 (clamped to
 *            [0, C-1]) contributes the texel whose angular interval holds the
 *            angle of (c, j): j' = floor((2j + 1) n_c' / (2 n_c)).
 *  luma      0.299 R + 0.587 G + 0.114 B.
 *  1 skip    contrast range of {M, N, S, E, W} below max(1/12, max / 6): the
 *            texel is copied (N/S = j +- 1, E/W = c +- 1).
 *  2 axis    second differences across the angle (kA) and across the radius
 *            (kR) from the 3 x 3 neighbourhood; kR >= kA means the luma
 *            changes across columns: the edge runs along the angle and the
 *            blend steps one column, otherwise the reverse.
 *  3 side    the blend neighbour is the one with the larger luma step
 *            (positive side on a tie); the edge's mid-line luma is their
 *            mean, its threshold a quarter of the step.
 *  4 search  walk along the edge both ways, up to 12 unit steps, averaging
 *            the luma of the texel on the walk and of its partner across the
 *            edge; an end is where that mean leaves the mid-line by the
 *            threshold (a walk that finds none ends at 12).
 *  5 offset  from the nearer end d and both ends' sum D: 1/2 - d/D, applied
 *            only when the luma at that end lies on the other side of the
 *            mid-line than the texel (ties: the positive end).
 *  6 subpix  a = |mean of the 3 x 3 (edges weight 2, corners 1) - M| / range,
 *            (3 - 2a) a^2 squared, times 3/4.
 *  7 blend   texel + max(offset, subpix) (neighbour - texel), all channels.
 * Luma and every comparison are in FP32 with the operation order written
 * here, so a kernel that rounds the same way takes the same branches; the
 * offsets and the blend are FP64. */

#define OR_FXAA_STEPS 12

typedef struct {
    const int32_t* n;
    const int64_t* off;
    int C;
    const double* lp;
    int nch;
} or_lpgrid;

/* Texel of column c2 (clamped to [0, C-1]) at the angle of texel (c, j),
 * then moved dj rows within that column (modulo its count). */
static int64_t lp_at(const or_lpgrid* g, int c, int64_t j, int c2, int64_t dj) {
    if (c2 < 0) c2 = 0;
    if (c2 > g->C - 1) c2 = g->C - 1;
    int64_t n = g->n[c], n2 = g->n[c2];
    int64_t j2 = c2 == c ? j : ((2 * j + 1) * n2) / (2 * n);
    j2 = ((j2 + dj) % n2 + n2) % n2;
    return g->off[c2] + j2;
}

static float lp_luma(const or_lpgrid* g, int64_t t) {
    const double* p = g->lp + t * g->nch;
    float y = 0.299f * (float)p[0];
    y = y + 0.587f * (float)p[1];
    y = y + 0.114f * (float)p[2];
    return y;
}

void or_lp_neighbor(const int32_t* n_col, const int64_t* off_col, int C, int c, int64_t j, int c2,
                    int64_t dj, int64_t* out) {
    or_lpgrid g = {n_col, off_col, C, NULL, 0};
    *out = lp_at(&g, c, j, c2, dj);
}

void or_fxaa_lp(const int32_t* n_col, const int64_t* off_col, int C, const double* lp, int nch,
                double* out) {
    const or_lpgrid g = {n_col, off_col, C, lp, nch};
    #pragma omp parallel for schedule(dynamic, 4)
    for (int c = 0; c < C; ++c) {
        for (int64_t j = 0; j < n_col[c]; ++j) {
            const int64_t tM = off_col[c] + j;
            for (int ch = 0; ch < nch; ++ch) out[tM * nch + ch] = lp[tM * nch + ch];
            const float M = lp_luma(&g, tM);
            const float N = lp_luma(&g, lp_at(&g, c, j, c, 1)), S = lp_luma(&g, lp_at(&g, c, j, c, -1));
            const float E = lp_luma(&g, lp_at(&g, c, j, c + 1, 0)), W = lp_luma(&g, lp_at(&g, c, j, c - 1, 0));
            /* 1 skip */
            const float lo = fminf(M, fminf(fminf(N, S), fminf(E, W)));
            const float hi = fmaxf(M, fmaxf(fmaxf(N, S), fmaxf(E, W)));
            const float range = hi - lo;
            if (range < fmaxf(1.0f / 12.0f, hi * (1.0f / 6.0f))) continue;
            const float NE = lp_luma(&g, lp_at(&g, c, j, c + 1, 1)), SE = lp_luma(&g, lp_at(&g, c, j, c + 1, -1));
            const float NW = lp_luma(&g, lp_at(&g, c, j, c - 1, 1)), SW = lp_luma(&g, lp_at(&g, c, j, c - 1, -1));
            /* 2 axis */
            const float kA = 2.0f * fabsf((N + S) - 2.0f * M) + fabsf((NE + SE) - 2.0f * E) + fabsf((NW + SW) - 2.0f * W);
            const float kR = 2.0f * fabsf((E + W) - 2.0f * M) + fabsf((NE + NW) - 2.0f * N) + fabsf((SE + SW) - 2.0f * S);
            const int across_cols = kR >= kA;
            /* 3 side */
            const float Ln = across_cols ? W : S, Lp = across_cols ? E : N;
            const float gn = fabsf(Ln - M), gp = fabsf(Lp - M);
            const int pos = gp >= gn;
            const float avg = 0.5f * (M + (pos ? Lp : Ln));
            const float thr = 0.25f * fmaxf(gn, gp);
            const int side = pos ? 1 : -1;
            /* 4 search */
            int dist[2];
            float end[2];
            for (int d = 0; d < 2; ++d) {
                const int sgn = d ? 1 : -1;
                dist[d] = OR_FXAA_STEPS;
                end[d] = 0.0f;
                for (int k = 1; k <= OR_FXAA_STEPS; ++k) {
                    int64_t ta, tb;
                    if (across_cols) {               /* walk rows of column c */
                        ta = lp_at(&g, c, j, c, sgn * k);
                        tb = lp_at(&g, c, ta - off_col[c], c + side, 0);
                    } else {                         /* walk columns at the angle of (c, j) */
                        int ck = c + sgn * k;
                        if (ck < 0) ck = 0;
                        if (ck > C - 1) ck = C - 1;
                        ta = lp_at(&g, c, j, ck, 0);
                        tb = lp_at(&g, ck, ta - off_col[ck], ck, side);
                    }
                    const float s = 0.5f * (lp_luma(&g, ta) + lp_luma(&g, tb));
                    end[d] = s;
                    if (fabsf(s - avg) >= thr) { dist[d] = k; break; }
                }
            }
            /* 5 offset */
            const int near_neg = dist[0] < dist[1];
            const int dn = near_neg ? dist[0] : dist[1];
            const float lend = near_neg ? end[0] : end[1];
            const int good = ((lend - avg) < 0.0f) != ((M - avg) < 0.0f);
            const double off_edge = good ? 0.5 - (double)dn / (double)(dist[0] + dist[1]) : 0.0;
            /* 6 subpix */
            const double l3 = (2.0 * ((double)N + (double)S + (double)E + (double)W) +
                               ((double)NE + (double)NW + (double)SE + (double)SW)) / 12.0;
            double a = fabs(l3 - (double)M) / (double)range;
            if (a > 1.0) a = 1.0;
            const double b = (3.0 - 2.0 * a) * a * a;
            const double sub = b * b * 0.75;
            /* 7 blend */
            const double w = off_edge > sub ? off_edge : sub;
            const int64_t tS = across_cols ? lp_at(&g, c, j, c + side, 0) : lp_at(&g, c, j, c, side);
            for (int ch = 0; ch < nch; ++ch) {
                const double m = lp[tM * nch + ch], q = lp[tS * nch + ch];
                out[tM * nch + ch] = m + w * (q - m);
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Path tracing into the LP buffer (Sec. 8): the paper renders the LP texels
 * with the Path Tracing SDK at 1 sample per texel with next-event estimation,
 * Russian roulette off, up to 3 diffuse bounces.  Here every surface is
 * Lambertian (the scene's albedo) and the lights are the scene's directional
 * light (radiance scale 1, as the ray-casting shading) and the sky gradient
 * (what an escaping ray sees).  Per LP texel, with throughput beta = 1:
 *   segment k = 0 .. D: closest hit of the ray, ignoring the triangle it
 *     leaves (-1 for the primary ray; a planar triangle cannot be hit again);
 *     a miss adds beta * sky(d) and ends the path;
 *     rays leaving a surface start at p + delta n with delta = 1e-5 max(1,
 *     max_i |p_i|) (so coplanar neighbours of the hit triangle lie behind
 *     them) and also ignore the hit triangle;
 *     at a hit with albedo rho and normal n facing the ray: when
 *     cos = n . (-L) > 0 a shadow ray (p, -L), again ignoring the hit
 *     triangle, decides visibility and a visible light adds beta rho cos;
 *     unless k = D, the next direction is cosine-distributed about n
 *     (r = sqrt(u1), phi = 2 pi u2, z = sqrt(1 - u1), in the orthonormal
 *     basis of Duff et al. 2017), and beta *= rho (BRDF rho/pi times cos
 *     over the pdf cos/pi).
 * Random numbers: u = top 24 bits of a counter hash / 2^24, the hash being
 * SplitMix64's output function (Steele, Lea, Flood 2014) applied to seed,
 * texel index, and 2 k + dim in turn.
 * Outputs: rgba per texel and a signature per texel: the hit id of each
 * segment (-1 miss, -2 not traced) and a mask: bit k = segment k's shadow
 * ray saw the light, bit 16 + k = a shadow ray was cast there. */

static uint64_t sm64_mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double or_pt_uniform(uint64_t seed, uint64_t texel, int k, int dim) {
    uint64_t h = sm64_mix(sm64_mix(sm64_mix(seed) ^ texel) ^ (uint64_t)(2 * k + dim));
    return (double)(h >> 40) * (1.0 / 16777216.0);
}

static void sky_rgb(const double d[3], double out[3]) {
    double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double s = 0.5 * (d[1] / dl + 1.0);
    out[0] = (1.0 - s) * 1.0 + s * 0.5;
    out[1] = (1.0 - s) * 1.0 + s * 0.7;
    out[2] = (1.0 - s) * 1.0 + s * 1.0;
}

void or_path_trace(void* bvh, const float* albedo, const double* light_dir, const double* orig,
                   const double* dir, const int64_t* texel_ids, int64_t n, uint64_t seed, int D,
                   double* rgba, int32_t* sig, double* seg) {
    const or_bvh* b = (const or_bvh*)bvh;
    double L[3] = {light_dir[0], light_dir[1], light_dir[2]};
    double ln = sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
    for (int k = 0; k < 3; ++k) L[k] /= ln;
    const double toL[3] = {-L[0], -L[1], -L[2]};
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < n; ++q) {
        int32_t* sg = sig + q * (D + 2);
        for (int k = 0; k <= D; ++k) sg[k] = -2;
        sg[D + 1] = 0;
        double o[3] = {orig[3 * q], orig[3 * q + 1], orig[3 * q + 2]};
        double d[3] = {dir[3 * q], dir[3 * q + 1], dir[3 * q + 2]};
        double beta[3] = {1.0, 1.0, 1.0}, acc[3] = {0.0, 0.0, 0.0};
        int32_t skip = -1;
        for (int k = 0; k <= D; ++k) {
            if (seg) for (int a = 0; a < 3; ++a) { seg[(q * (D + 1) + k) * 6 + a] = o[a]; seg[(q * (D + 1) + k) * 6 + 3 + a] = d[a]; }
            double t;
            const int32_t id = bvh_closest(b, o, d, skip, &t);
            sg[k] = id;
            if (id < 0) {
                double sky[3];
                sky_rgb(d, sky);
                for (int a = 0; a < 3; ++a) acc[a] += beta[a] * sky[a];
                break;
            }
            const float* tr = b->tris + 9 * (int64_t)id;
            double e1[3], e2[3], nrm[3], p[3];
            for (int a = 0; a < 3; ++a) {
                e1[a] = (double)tr[3 + a] - tr[a];
                e2[a] = (double)tr[6 + a] - tr[a];
                p[a] = o[a] + t * d[a];
            }
            nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
            nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
            nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
            double nl = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
            for (int a = 0; a < 3; ++a) nrm[a] /= nl;
            if (nrm[0] * d[0] + nrm[1] * d[1] + nrm[2] * d[2] > 0.0)
                for (int a = 0; a < 3; ++a) nrm[a] = -nrm[a];
            const float* rho = albedo + 3 * (int64_t)id;
            const double pm = fmax(1.0, fmax(fabs(p[0]), fmax(fabs(p[1]), fabs(p[2]))));
            for (int a = 0; a < 3; ++a) p[a] += 1e-5 * pm * nrm[a];
            const double cosl = nrm[0] * toL[0] + nrm[1] * toL[1] + nrm[2] * toL[2];
            if (cosl > 0.0) {
                double ts;
                sg[D + 1] |= 1 << (16 + k);
                if (bvh_closest(b, p, toL, id, &ts) < 0) {
                    sg[D + 1] |= 1 << k;
                    for (int a = 0; a < 3; ++a) acc[a] += beta[a] * rho[a] * cosl;
                }
            }
            if (k == D) break;
            const double u1 = or_pt_uniform(seed, (uint64_t)texel_ids[q], k, 0);
            const double u2 = or_pt_uniform(seed, (uint64_t)texel_ids[q], k, 1);
            const double r = sqrt(u1), phi = 2.0 * M_PI * u2;
            const double lx = r * cos(phi), ly = r * sin(phi), lz = sqrt(fmax(0.0, 1.0 - u1));
            const double sgn = copysign(1.0, nrm[2]);
            const double aa = -1.0 / (sgn + nrm[2]);
            const double bb = nrm[0] * nrm[1] * aa;
            const double t1[3] = {1.0 + sgn * nrm[0] * nrm[0] * aa, sgn * bb, -sgn * nrm[0]};
            const double t2[3] = {bb, sgn + nrm[1] * nrm[1] * aa, -nrm[1]};
            for (int a = 0; a < 3; ++a) {
                d[a] = lx * t1[a] + ly * t2[a] + lz * nrm[a];
                o[a] = p[a];
                beta[a] *= rho[a];
            }
            skip = id;
        }
        rgba[4 * q] = acc[0];
        rgba[4 * q + 1] = acc[1];
        rgba[4 * q + 2] = acc[2];
        rgba[4 * q + 3] = 1.0;
    }
}

/* ------------------------------------------------------------------------- */
/* VaFR_Rep (Sec. 5.1): the right eye's LP buffer by forward grid warping of
 * the left eye's LP buffer (after Wissmann et al. 2020, but directly from the
 * LP buffer), disocclusions re-rendered.  The paper names the method only;
 * the steps here:
 *  vertices  every left texel's hit point P = o + t d (t from the left cast;
 *            a miss is a point at infinity in direction d), seen from the
 *            right eye: camera coordinates, then the right eye's forward map
 *            (Eq. 3 with its own gaze, e clamped to e_max, Eq. 12):
 *            U = u(e) - 1/2 (texel column c sits at U = c), F = angle / 360
 *            (texel j of column c sits at F = (j + 1/2)/n_c); depth =
 *            distance to the right eye (1e30 for points at infinity).
 *  mesh      the strip between columns c and c+1 (rings of n and n' texels
 *            at angles (j + 1/2)/n) is zipped: walking both rings by angle
 *            (ring c first on equal angles), each step of ring c from a_j to
 *            a_j+1 makes the triangle (a_j, a_j+1, b_k) with b_k the last
 *            ring-(c+1) vertex before a_j+1, k = max{k : (2k+1) n <
 *            (2j+3) n'}, and each step of ring c+1 from b_k to b_k+1 makes
 *            (b_k, b_k+1, a_j), j = max{j : (2j+1) n' <= (2k+3) n} (indices
 *            modulo the ring sizes); the triangles tile the strip.  Texel t
 *            owns triangle 2 t (its step towards column c+1) and 2 t + 1 (its
 *            step as the outer ring of the strip towards c-1).
 *  reject    a triangle with a vertex behind the right eye, mixing hits and
 *            misses, whose largest finite depth exceeds 1.1 x its smallest
 *            (it would stretch over a depth discontinuity), or spanning more
 *            than 64 columns or (after unwrapping) a quarter turn: such
 *            slivers only arise around a polar centre and are left to the
 *            hole pass.
 *  raster    in the (U, F) plane; a triangle spanning more than half a turn
 *            in F is unwrapped (+1 on its low vertices) and drawn at F and
 *            F - 1.  Column c covers [min, max] of the triangle's edge
 *            crossings of U = c; its rows j with (j + 1/2)/n_c inside are
 *            covered (boundaries included).  Depth and colour are
 *            interpolated barycentrically in (U, F); the nearest depth wins,
 *            ties to the lower triangle id.
 *  holes     right texels no triangle covers are ray cast like any texel.
 * Here: right rgba and winning triangle (-1 = hole) per right texel. */

#define OR_REP_DEPTH_RATIO 1.1
#define OR_REP_MAX_U_SPAN 64.0
#define OR_REP_MAX_F_SPAN 0.25

typedef struct { double U, F, z; int ok, inf; } or_rvert;

static void rep_vertex(const or_acuity* a, double e_max, const or_view* vl, const or_view* vr,
                       double e_c, int32_t n_c, int64_t j, double t, or_rvert* out) {
    double x, y, o[3], d[3];
    texel_screen_point(vl, e_c, n_c, j, &x, &y);
    view_ray(vl, x, y, o, d);
    double P[3];
    out->inf = !(t < INFINITY);
    for (int k = 0; k < 3; ++k) P[k] = out->inf ? d[k] : o[k] + t * d[k] - vr->pose[4 * k + 3];
    /* camera coordinates of the right eye: R^T P (pose columns are the camera axes) */
    double pc[3];
    for (int k = 0; k < 3; ++k)
        pc[k] = vr->pose[k] * P[0] + vr->pose[4 + k] * P[1] + vr->pose[8 + k] * P[2];
    out->ok = pc[2] > 0.0;
    if (!out->ok) return;
    double cr = view_cr(vr);
    double sx = 0.5 * vr->width + pc[0] / pc[2] / cr, sy = 0.5 * vr->height - pc[1] / pc[2] / cr;
    double dx = sx - vr->x0, dy = sy - vr->y0;
    double e = atan(cr * sqrt(dx * dx + dy * dy)) / OR_DEG;
    if (e > e_max) e = e_max;
    out->U = or_u_of_e(a, e) - 0.5;
    double ang = atan2(dy, dx) / OR_DEG;
    if (ang < 0.0) ang += 360.0;
    out->F = ang / 360.0;
    out->z = out->inf ? 1e30 : sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
}

/* barycentric weights of (u, f) in triangle v; returns 0 if degenerate */
static int rep_bary(const or_rvert* v[3], const double F3[3], double u, double f, double w[3]) {
    double x1 = v[1]->U - v[0]->U, y1 = F3[1] - F3[0];
    double x2 = v[2]->U - v[0]->U, y2 = F3[2] - F3[0];
    double det = x1 * y2 - x2 * y1;
    if (det == 0.0) return 0;
    double px = u - v[0]->U, py = f - F3[0];
    w[1] = (px * y2 - x2 * py) / det;
    w[2] = (x1 * py - px * y1) / det;
    w[0] = 1.0 - w[1] - w[2];
    return 1;
}

/* Triangle s of texel (c, j): s = 0 its segment's fan triangle towards
 * column c+1, s = 1 towards column c-1.  Returns 0 if it does not exist. */
static int rep_triangle(const int32_t* n_col, const int64_t* off_col, int C, int c, int64_t j, int s,
                        int64_t tv[3]) {
    const int c2 = s == 0 ? c + 1 : c - 1;
    if (c2 < 0 || c2 >= C) return 0;
    const int64_t n = n_col[c], n2 = n_col[c2];
    int64_t k;
    if (s == 0) {          /* ring c is the inner ring: k = max{k : (2k+1) n < (2j+3) n2} */
        const int64_t w = ((2 * j + 3) * n2 + n - 1) / n - 2;
        k = w >= 0 ? w / 2 : -1;
    } else {               /* ring c is the outer ring: k = max{k : (2k+1) n <= (2j+3) n2} */
        const int64_t q = ((2 * j + 3) * n2) / n;
        k = q >= 1 ? (q - 1) / 2 : -1;
    }
    k = ((k % n2) + n2) % n2;
    tv[0] = off_col[c] + j;
    tv[1] = off_col[c] + (j + 1) % n;
    tv[2] = off_col[c2] + k;
    return 1;
}

static void rep_raster(const or_rvert* V, const int64_t tv[3], int32_t tid, const int32_t* n_col,
                       const int64_t* off_col, int C, double* zbest, int32_t* right_tri) {
    const or_rvert* v[3] = {&V[tv[0]], &V[tv[1]], &V[tv[2]]};
    if (!v[0]->ok || !v[1]->ok || !v[2]->ok) return;
    int ninf = v[0]->inf + v[1]->inf + v[2]->inf;
    if (ninf != 0 && ninf != 3) return;
    double zlo = fmin(v[0]->z, fmin(v[1]->z, v[2]->z)), zhi = fmax(v[0]->z, fmax(v[1]->z, v[2]->z));
    if (ninf == 0 && zhi > OR_REP_DEPTH_RATIO * zlo) return;
    double ulo = fmin(v[0]->U, fmin(v[1]->U, v[2]->U)), uhi = fmax(v[0]->U, fmax(v[1]->U, v[2]->U));
    if (uhi - ulo > OR_REP_MAX_U_SPAN) return;
    double F3[3] = {v[0]->F, v[1]->F, v[2]->F};
    double flo = fmin(F3[0], fmin(F3[1], F3[2])), fhi = fmax(F3[0], fmax(F3[1], F3[2]));
    int copies = 1;
    if (fhi - flo > 0.5) {
        for (int q = 0; q < 3; ++q) if (F3[q] < 0.5) F3[q] += 1.0;
        copies = 2;
        flo = fmin(F3[0], fmin(F3[1], F3[2]));
        fhi = fmax(F3[0], fmax(F3[1], F3[2]));
    }
    if (fhi - flo > OR_REP_MAX_F_SPAN) return;
    int c0 = (int)ceil(ulo), c1 = (int)floor(uhi);
    if (c0 < 0) c0 = 0;
    if (c1 > C - 1) c1 = C - 1;
    for (int cr = c0; cr <= c1; ++cr) {
        double lo = INFINITY, hi = -INFINITY;
        for (int e = 0; e < 3; ++e) {
            int p = e, q = (e + 1) % 3;
            double up = v[p]->U - cr, uq = v[q]->U - cr;
            if (up * uq > 0.0) continue;
            if (v[p]->U == v[q]->U) {
                lo = fmin(lo, fmin(F3[p], F3[q]));
                hi = fmax(hi, fmax(F3[p], F3[q]));
                continue;
            }
            double f = F3[p] + (cr - v[p]->U) / (v[q]->U - v[p]->U) * (F3[q] - F3[p]);
            lo = fmin(lo, f);
            hi = fmax(hi, f);
        }
        if (!(lo <= hi)) continue;
        for (int cp = 0; cp < copies; ++cp) {
            double sh = cp ? -1.0 : 0.0;
            int64_t n = n_col[cr];
            int64_t j0 = (int64_t)ceil((lo + sh) * n - 0.5), j1 = (int64_t)floor((hi + sh) * n - 0.5);
            if (j0 < 0) j0 = 0;
            if (j1 > n - 1) j1 = n - 1;
            for (int64_t jj = j0; jj <= j1; ++jj) {
                double f = ((double)jj + 0.5) / (double)n - sh, w[3];
                if (!rep_bary(v, F3, (double)cr, f, w)) continue;
                double z = w[0] * v[0]->z + w[1] * v[1]->z + w[2] * v[2]->z;
                int64_t k = off_col[cr] + jj;
                if (z < zbest[k] || (z == zbest[k] && tid < right_tri[k])) {
                    zbest[k] = z;
                    right_tri[k] = tid;
                }
            }
        }
    }
}

/* Test support for the warp's parity check: for query q, warped triangle
 * q_tid[q] (numbered as right_tri) and right texel q_tex[q] (column order),
 * out[10 q + ...] = the quantities the raster decides on, so that a test can
 * tell a decision taken within rounding of its threshold from a genuine
 * difference:
 *   0 exists (1/0)      1 all vertices in front of the right eye (1/0)
 *   2 smallest camera depth of the vertices over their distance (> 0 in front)
 *   3 vertices at infinity (0..3)   4 zhi / zlo (finite vertices, else 0)
 *   5 U span            6 F span before unwrapping   7 F span after
 *   8 coverage margin of the texel centre: its signed distance to the
 *     triangle (> 0 inside) in the plane of (U in columns, F in rows of the
 *     texel's column), the smaller distance to an edge line
 *   9 interpolated depth at the texel centre (inf if not computable). */
void or_rep_probe(const or_acuity* a, double e_max, const double* e_col, const int32_t* n_col,
                  const int64_t* off_col, int C, int64_t n_tex, const or_view* vl, const or_view* vr,
                  const double* left_t, int64_t n_q, const int32_t* q_tid, const int64_t* q_tex,
                  double* out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n_q; ++q) {
        double* o = out + 10 * q;
        for (int i = 0; i < 10; ++i) o[i] = 0.0;
        o[9] = INFINITY;
        const int32_t tid = q_tid[q];
        if (tid < 0 || (int64_t)tid / 2 >= n_tex) continue;
        const int64_t ia = tid / 2;
        const int s = tid % 2;
        int c = 0;
        { int lo = 0, hi = C - 1; while (lo < hi) { int mid = (lo + hi + 1) / 2; if (off_col[mid] <= ia) lo = mid; else hi = mid - 1; } c = lo; }
        int64_t tv[3];
        if (!rep_triangle(n_col, off_col, C, c, ia - off_col[c], s, tv)) continue;
        o[0] = 1.0;
        or_rvert V[3];
        double zmin = INFINITY;
        for (int v = 0; v < 3; ++v) {
            int cv = 0;
            { int lo = 0, hi = C - 1; while (lo < hi) { int mid = (lo + hi + 1) / 2; if (off_col[mid] <= tv[v]) lo = mid; else hi = mid - 1; } cv = lo; }
            rep_vertex(a, e_max, vl, vr, e_col[cv], n_col[cv], tv[v] - off_col[cv], left_t[tv[v]], &V[v]);
            /* camera depth of the vertex in the right eye over its distance */
            double x, y, oo[3], d[3], P[3], pc2 = 0.0, len = 0.0;
            texel_screen_point(vl, e_col[cv], n_col[cv], tv[v] - off_col[cv], &x, &y);
            view_ray(vl, x, y, oo, d);
            const int inf = !(left_t[tv[v]] < INFINITY);
            for (int k = 0; k < 3; ++k) P[k] = inf ? d[k] : oo[k] + left_t[tv[v]] * d[k] - vr->pose[4 * k + 3];
            for (int k = 0; k < 3; ++k) { pc2 += vr->pose[8 + k] * P[k]; len += P[k] * P[k]; }
            const double r = pc2 / sqrt(len);
            if (r < zmin) zmin = r;
        }
        o[1] = (V[0].ok && V[1].ok && V[2].ok) ? 1.0 : 0.0;
        o[2] = zmin;
        const int ninf = V[0].inf + V[1].inf + V[2].inf;
        o[3] = ninf;
        if (!o[1]) continue;
        if (ninf == 0) {
            double zlo = fmin(V[0].z, fmin(V[1].z, V[2].z)), zhi = fmax(V[0].z, fmax(V[1].z, V[2].z));
            o[4] = zhi / zlo;
        }
        double ulo = fmin(V[0].U, fmin(V[1].U, V[2].U)), uhi = fmax(V[0].U, fmax(V[1].U, V[2].U));
        o[5] = uhi - ulo;
        double F3[3] = {V[0].F, V[1].F, V[2].F};
        double flo = fmin(F3[0], fmin(F3[1], F3[2])), fhi = fmax(F3[0], fmax(F3[1], F3[2]));
        o[6] = fhi - flo;
        if (fhi - flo > 0.5) {
            for (int k = 0; k < 3; ++k) if (F3[k] < 0.5) F3[k] += 1.0;
            flo = fmin(F3[0], fmin(F3[1], F3[2]));
            fhi = fmax(F3[0], fmax(F3[1], F3[2]));
        }
        o[7] = fhi - flo;
        /* the texel's column and row */
        const int64_t k = q_tex[q];
        int cr = 0;
        { int lo = 0, hi = C - 1; while (lo < hi) { int mid = (lo + hi + 1) / 2; if (off_col[mid] <= k) lo = mid; else hi = mid - 1; } cr = lo; }
        const int64_t n = n_col[cr], jj = k - off_col[cr];
        /* signed distance of the centre (cr, f n) to the triangle (U, F n): the
         * smaller distance to an edge line, > 0 inside; the unwrapped triangle
         * is drawn at F and F - 1, so the centre is also tried at f + 1 */
        const double fc = ((double)jj + 0.5) / (double)n;
        const double area = (V[1].U - V[0].U) * (F3[2] - F3[0]) - (V[2].U - V[0].U) * (F3[1] - F3[0]);
        const double orient = area >= 0.0 ? 1.0 : -1.0;
        double best = -INFINITY;
        for (int cp = 0; cp < 2; ++cp) {
            const double px = (double)cr, py = (fc + cp) * (double)n;
            double m = INFINITY;
            for (int e = 0; e < 3; ++e) {
                const int p0 = e, p1 = (e + 1) % 3;
                const double ex = V[p1].U - V[p0].U, ey = (F3[p1] - F3[p0]) * (double)n;
                const double len = sqrt(ex * ex + ey * ey);
                const double dist = len > 0.0 ? orient * (ex * (py - F3[p0] * (double)n) - ey * (px - V[p0].U)) / len
                                              : -INFINITY;
                if (dist < m) m = dist;
            }
            if (m > best) best = m;
        }
        o[8] = best;
        const or_rvert* vp[3] = {&V[0], &V[1], &V[2]};
        double w[3];
        const double f = fc;
        if (!rep_bary(vp, F3, (double)cr, f, w) || w[0] < -0.25 || w[1] < -0.25 || w[2] < -0.25)
            if (!rep_bary(vp, F3, (double)cr, f + 1.0, w)) continue;
        o[9] = w[0] * V[0].z + w[1] * V[1].z + w[2] * V[2].z;
    }
}

void or_reproject_lp(const or_acuity* a, double e_max, const double* e_col, const int32_t* n_col,
                     const int64_t* off_col, int C, int64_t n_tex, const or_view* vl, const or_view* vr,
                     const double* left_t, const double* left_rgba, double* right_rgba,
                     int32_t* right_tri) {
    or_rvert* V = (or_rvert*)malloc(sizeof(or_rvert) * (size_t)n_tex);
    double* zbest = (double*)malloc(sizeof(double) * (size_t)n_tex);
#pragma omp parallel for schedule(dynamic, 4)
    for (int c = 0; c < C; ++c)
        for (int64_t j = 0; j < n_col[c]; ++j)
            rep_vertex(a, e_max, vl, vr, e_col[c], n_col[c], j, left_t[off_col[c] + j], &V[off_col[c] + j]);
    for (int64_t k = 0; k < n_tex; ++k) { zbest[k] = INFINITY; right_tri[k] = -1; }
    /* serial raster: the z-test with its id tie rule is order-independent */
    for (int c = 0; c < C; ++c) {
        for (int64_t j = 0; j < n_col[c]; ++j) {
            for (int s = 0; s < 2; ++s) {
                int64_t tv[3];
                if (!rep_triangle(n_col, off_col, C, c, j, s, tv)) continue;
                const int32_t tid = (int32_t)(2 * (off_col[c] + j) + s);
                rep_raster(V, tv, tid, n_col, off_col, C, zbest, right_tri);
            }
        }
    }
    /* resolve: colours of the winning triangles */
#pragma omp parallel for schedule(dynamic, 4)
    for (int cr = 0; cr < C; ++cr) {
        for (int64_t jj = 0; jj < n_col[cr]; ++jj) {
            int64_t k = off_col[cr] + jj;
            for (int ch = 0; ch < 4; ++ch) right_rgba[4 * k + ch] = 0.0;
            int32_t tid = right_tri[k];
            if (tid < 0) continue;
            int64_t ia = tid / 2;
            int s = tid % 2;
            int c = 0;
            { int lo = 0, hi = C - 1; while (lo < hi) { int mid = (lo + hi + 1) / 2; if (off_col[mid] <= ia) lo = mid; else hi = mid - 1; } c = lo; }
            int64_t tv[3];
            rep_triangle(n_col, off_col, C, c, ia - off_col[c], s, tv);
            const or_rvert* v[3] = {&V[tv[0]], &V[tv[1]], &V[tv[2]]};
            double F3[3] = {v[0]->F, v[1]->F, v[2]->F};
            double flo = fmin(F3[0], fmin(F3[1], F3[2])), fhi = fmax(F3[0], fmax(F3[1], F3[2]));
            if (fhi - flo > 0.5) for (int q = 0; q < 3; ++q) if (F3[q] < 0.5) F3[q] += 1.0;
            double f = ((double)jj + 0.5) / (double)n_col[cr], w[3];
            if (!rep_bary(v, F3, (double)cr, f, w) || w[0] < -0.25 || w[1] < -0.25 || w[2] < -0.25)
                rep_bary(v, F3, (double)cr, f + 1.0, w);
            for (int ch = 0; ch < 4; ++ch)
                right_rgba[4 * k + ch] = w[0] * left_rgba[4 * tv[0] + ch] + w[1] * left_rgba[4 * tv[1] + ch] +
                                         w[2] * left_rgba[4 * tv[2] + ch];
        }
    }
    free(V);
    free(zbest);
}
