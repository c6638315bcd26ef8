/*
 * FP64 CPU oracle for the RIS field path of "Ray Tracing Algorithm for Reconfigurable Intelligent
 * Surfaces" (arXiv 2402.13034).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or call this file; only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark do. It shares no code, header or
 * constant table with the CUDA library.
 *
 * What it computes, per receiver point r, written out as the plain definition (no factoring):
 *
 *   E(r) = E_LOS(r) + E_env(r) + sum_m Gamma_m sum_{p in Tx-leg paths of m} sum_{q in Rx-leg paths of m} e_mpq(r)
 *
 *   e_mpq = sqrt(2 eta0 Pt Gt Ft(theta_t))                       (Eq. 4, launch field towards element m)
 *         * sqrt(G F(theta_in) F(theta_out) dy dz / (4 pi))       (Eq. 5-7, F_RIS = F_in F_out)
 *         * R_p R_q * exp(-j k (L_p + L_q)) / L_p                  (Eq. 7 phase/spreading, Fresnel per bounce)
 *         * sqrt(Gr Fr(theta_r)) * lambda / (4 pi L_q)             (Eq. 8, field at the Rx)
 *   P(r) = |E(r)|^2 / (2 eta0)                                     (Eq. 10), superposition Eq. 9.
 *
 * Paths (Sec. II-B): the direct legs Tx->e_m and e_m->Rx are checked for occlusion per element
 * (one ray per element, Sec. IV-A); reflected legs are found by the image method over sequences
 * of planar faces of length <= 2, validated ONCE between the RIS centre and the Rx (and between
 * the Tx and the RIS centre on the Tx leg) with explicit reflection points; each element then takes
 * each accepted sequence through the image method (its own mirrored images, the leg length being
 * the image-to-destination distance), without re-validation.
 * Fresnel reflection (Collin) is applied at every bounce with eps_c = eps_r - j sigma/(omega eps0).
 *
 * Readings of points the paper leaves open (scalar field, e^{+j omega t} convention, element gain
 * default G = 4 pi dy dz / lambda^2, TE Fresnel by default, unfolded leg length in Eq. 7/8, patterns
 * clamped to the front hemisphere, LOS always on, Tx->Rx specular "environment" paths behind a
 * flag) are listed in the design notes of the repository.
 *
 * Every geometric decision also reports whether it lies within AMB_TOL of flipping ("ambiguous");
 * comparisons against another implementation exclude those decisions.
 *
 * Vector mode (the polarisation extension that Sec. II-A names for Eq. 6 without giving a model): each
 * term keeps every scalar factor above except the Fresnel products and is multiplied by a polarisation
 * factor built from the real segment directions of its path:
 *   launch     e = unit(P(d0) a_t), P(k) = I - k k^T, a_t the Tx polarisation axis, d0 the departure
 *   bounce     e <- R_TE (e.s) s + R_TM (e.p_in) p_out, s = unit(k_in x n), p = s x k  (both Fresnel
 *              coefficients, complex permittivity as above; at normal incidence e <- R_TE e)
 *   RIS        e <- P(k_out) (e - 2 (e.n) n): the incident field with its normal component reversed
 *              (tangential components kept), restricted to the outgoing wavefront
 *   reception  received = unit(P(k_arr) a_r) . e ; the field vector E3 = sum of the terms' e (Eq. 8's
 *              amplitude included); zero where a projected axis vanishes.
 * With every field TE and co-polarised the received value equals the scalar model's.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_C0 299792458.0
#define OR_ETA0 (120.0 * OR_PI)       /* Eq. 1: eta0 = 120 pi ohm */
#define OR_EPS0 8.8541878128e-12
#define OR_SEG_EPS 1e-4               /* occluder hits closer than this to a segment end are ignored */

/* Half-width of the band in which a geometric decision counts as ambiguous (metres). */
static double AMB_TOL = 1e-8;

enum { PAT_ISO = 0, PAT_COS_POW = 1, PAT_MONOPOLE_QW = 2 };

/* --------------------------------------------------------------------------------------------
 * Problem description passed from Python (mirrors a ctypes.Structure).
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    const float* verts; int64_t n_verts;
    const int32_t* tris; const int32_t* face_id; const int32_t* mat_id; int64_t n_tris;
    const float* mats; int32_t n_mat;
    const float* elem_uv; int32_t M;
    float center[3], t1[3], t2[3];
    float dy, dz, elem_gain; int32_t host_face;
    float tx_pos[3]; float tx_orient[9]; float tx_power, tx_gain; int32_t tx_pattern;
    float rx_orient[9]; float rx_gain; int32_t rx_pattern;
    double freq;
    int32_t max_order_tx, max_order_rx, env_paths, fresnel_tm;
    int32_t strict_elements;   /* 1: validate each element's reflected legs at the element itself */
    int32_t vector_pol;        /* 1: vector field with polarisation (TE and TM per bounce) */
    float tx_pol[3], rx_pol[3];  /* polarisation axes of the Tx and Rx antennas (global) */
} or_problem;

typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 vf(const float* p) { return mk(p[0], p[1], p[2]); }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double norm(v3 a) { return sqrt(dot(a, a)); }
static v3 unit(v3 a) { return scl(a, 1.0 / norm(a)); }

typedef struct {
    or_problem P;
    int F;                    /* number of faces */
    v3* V;                    /* vertices */
    v3* fn; double* fd;       /* face plane: fn . x = fd, unit normal (from the face's first triangle) */
    int* fmat;                /* face material */
    int* ftri_start; int* ftri;   /* CSR list of triangles per face */
    unsigned char* edge_inner;    /* [T*3] edge opposite vertex i shared with another triangle of the same face */
    double* tbox;             /* [T*6] triangle AABB */
    v3 c, t1, t2, n;          /* RIS frame; n = unit(t1 x t2) */
    v3* e;                    /* element centres e_m = c + a t1 + b t2 */
    v3 tx, tx_z, rx_z;        /* Tx position, antenna boresights (unit local z axes) */
    v3 tx_pol, rx_pol;        /* unit polarisation axes (vector mode) */
    double lam, k, G, omega;
} or_ctx;

/* ---------------------------------------------------------------------------------------------
 * Antenna and element patterns (Sec. III-B, III-C). cos_t = cos(theta) from the pattern's axis.
 * ------------------------------------------------------------------------------------------- */
double or_pattern(int pattern, double gain, double cos_t)
{
    if (pattern == PAT_ISO) return 1.0;
    if (pattern == PAT_COS_POW) {             /* F(theta) = cos(theta)^(G/2 - 1), G linear */
        if (cos_t <= 0.0) return 0.0;
        return pow(cos_t, gain / 2.0 - 1.0);
    }
    if (pattern == PAT_MONOPOLE_QW) {         /* ((cos(kh cos t) - cos(kh)) / sin t)^2, h = lambda/4 */
        double s2 = 1.0 - cos_t * cos_t;
        if (s2 <= 0.0) return 0.0;            /* limit at the axis is 0 */
        double kh = 2.0 * OR_PI * 0.25;       /* 2 pi h / lambda with h = lambda/4 */
        double v = (cos(kh * cos_t) - cos(kh)) / sqrt(s2);
        return v * v;
    }
    return 0.0;
}

static double elem_pattern(double cos_t) { return cos_t > 0.0 ? cos_t : 0.0; }  /* F = cos(theta) */

/* Fresnel reflection coefficient at incidence cos(theta_i), TE (perpendicular) or TM. */
void or_fresnel(double cos_i, double eps_r, double sigma, double freq, int tm, double* re, double* im)
{
    double complex eps = eps_r - I * sigma / (2.0 * OR_PI * freq * OR_EPS0);
    double s2 = 1.0 - cos_i * cos_i;
    double complex root = csqrt(eps - s2);
    double complex R;
    if (!tm) R = (cos_i - root) / (cos_i + root);
    else R = (eps * cos_i - root) / (eps * cos_i + root);
    *re = creal(R);
    *im = cimag(R);
}

static double complex fresnel_c(const or_ctx* C, double cos_i, int face)
{
    int m = C->fmat[face];
    double re, im;
    or_fresnel(cos_i, C->P.mats[2 * m], C->P.mats[2 * m + 1], C->P.freq, C->P.fresnel_tm, &re, &im);
    return re + I * im;
}

/* --------------------------------------------------------------------------------------------
 * Set-up
 * ------------------------------------------------------------------------------------------ */
void or_destroy(or_ctx* C)
{
    if (!C) return;
    free(C->V); free(C->fn); free(C->fd); free(C->fmat); free(C->ftri_start); free(C->ftri);
    free(C->edge_inner); free(C->tbox); free(C->e);
    free(C);
}

static int same_pos(v3 a, v3 b) { return a.x == b.x && a.y == b.y && a.z == b.z; }

or_ctx* or_create(const or_problem* P)
{
    or_ctx* C = (or_ctx*)calloc(1, sizeof(or_ctx));
    C->P = *P;
    int64_t T = P->n_tris;
    C->V = (v3*)malloc(sizeof(v3) * (P->n_verts > 0 ? P->n_verts : 1));
    for (int64_t i = 0; i < P->n_verts; ++i) C->V[i] = vf(P->verts + 3 * i);
    int F = 0;
    for (int64_t t = 0; t < T; ++t) if (P->face_id[t] + 1 > F) F = P->face_id[t] + 1;
    C->F = F;
    C->fn = (v3*)calloc(F > 0 ? F : 1, sizeof(v3));
    C->fd = (double*)calloc(F > 0 ? F : 1, sizeof(double));
    C->fmat = (int*)calloc(F > 0 ? F : 1, sizeof(int));
    C->ftri_start = (int*)calloc(F + 1, sizeof(int));
    C->ftri = (int*)calloc(T > 0 ? T : 1, sizeof(int));
    int* seen = (int*)calloc(F > 0 ? F : 1, sizeof(int));
    for (int64_t t = 0; t < T; ++t) C->ftri_start[P->face_id[t] + 1]++;
    for (int f = 0; f < F; ++f) C->ftri_start[f + 1] += C->ftri_start[f];
    int* fill = (int*)calloc(F > 0 ? F : 1, sizeof(int));
    for (int64_t t = 0; t < T; ++t) {
        int f = P->face_id[t];
        C->ftri[C->ftri_start[f] + fill[f]++] = (int)t;
        if (!seen[f]) {                       /* plane from the face's first triangle */
            const int32_t* tv = P->tris + 3 * t;
            v3 a = C->V[tv[0]], b = C->V[tv[1]], c = C->V[tv[2]];
            v3 nn = unit(cross(sub(b, a), sub(c, a)));
            C->fn[f] = nn;
            C->fd[f] = dot(nn, a);
            C->fmat[f] = P->mat_id[t];
            seen[f] = 1;
        }
    }
    free(seen); free(fill);
    /* inner edges: edge (opposite vertex i) whose two end positions also form an edge of another
       triangle of the same face - crossing it does not leave the face */
    C->edge_inner = (unsigned char*)calloc(T > 0 ? 3 * T : 1, 1);
    for (int64_t t = 0; t < T; ++t) {
        const int32_t* tv = P->tris + 3 * t;
        int f = P->face_id[t];
        for (int i = 0; i < 3; ++i) {
            v3 a = C->V[tv[(i + 1) % 3]], b = C->V[tv[(i + 2) % 3]];
            for (int j = C->ftri_start[f]; j < C->ftri_start[f + 1]; ++j) {
                int u = C->ftri[j];
                if (u == t) continue;
                const int32_t* uv = P->tris + 3 * u;
                for (int k = 0; k < 3; ++k) {
                    v3 p = C->V[uv[k]], q = C->V[uv[(k + 1) % 3]];
                    if ((same_pos(a, p) && same_pos(b, q)) || (same_pos(a, q) && same_pos(b, p)))
                        C->edge_inner[3 * t + i] = 1;
                }
            }
        }
    }
    C->tbox = (double*)malloc(sizeof(double) * 6 * (T > 0 ? T : 1));
    for (int64_t t = 0; t < T; ++t) {
        const int32_t* tv = P->tris + 3 * t;
        v3 a = C->V[tv[0]], b = C->V[tv[1]], c = C->V[tv[2]];
        double* bx = C->tbox + 6 * t;
        bx[0] = fmin(a.x, fmin(b.x, c.x)); bx[1] = fmin(a.y, fmin(b.y, c.y)); bx[2] = fmin(a.z, fmin(b.z, c.z));
        bx[3] = fmax(a.x, fmax(b.x, c.x)); bx[4] = fmax(a.y, fmax(b.y, c.y)); bx[5] = fmax(a.z, fmax(b.z, c.z));
    }
    C->c = vf(P->center); C->t1 = vf(P->t1); C->t2 = vf(P->t2);
    C->n = unit(cross(C->t1, C->t2));
    C->e = (v3*)malloc(sizeof(v3) * (P->M > 0 ? P->M : 1));
    for (int m = 0; m < P->M; ++m)
        C->e[m] = add(C->c, add(scl(C->t1, P->elem_uv[2 * m]), scl(C->t2, P->elem_uv[2 * m + 1])));
    C->tx = vf(P->tx_pos);
    C->tx_z = unit(vf(P->tx_orient + 6));
    C->rx_z = unit(vf(P->rx_orient + 6));
    C->tx_pol = norm(vf(P->tx_pol)) > 0 ? unit(vf(P->tx_pol)) : mk(0, 0, 0);
    C->rx_pol = norm(vf(P->rx_pol)) > 0 ? unit(vf(P->rx_pol)) : mk(0, 0, 0);
    C->lam = OR_C0 / P->freq;
    C->k = 2.0 * OR_PI / C->lam;
    C->omega = 2.0 * OR_PI * P->freq;
    C->G = P->elem_gain > 0 ? (double)P->elem_gain : 4.0 * OR_PI * (double)P->dy * (double)P->dz / (C->lam * C->lam);
    return C;
}

void or_set_amb_tol(double tol) { AMB_TOL = tol; }
int or_n_faces(const or_ctx* C) { return C->F; }

/* --------------------------------------------------------------------------------------------
 * Geometry primitives
 * ------------------------------------------------------------------------------------------ */
static v3 mirror(const or_ctx* C, v3 p, int f)
{
    double s = dot(C->fn[f], p) - C->fd[f];
    return sub(p, scl(C->fn[f], 2.0 * s));
}

static double sdist(const or_ctx* C, v3 p, int f) { return dot(C->fn[f], p) - C->fd[f]; }

/* Barycentric containment of a point q lying on triangle t's plane. Returns the signed distances
   (metres, in the plane) from q to each edge; positive inside. */
static void tri_edge_dist(const or_ctx* C, int t, v3 q, double d[3])
{
    const int32_t* tv = C->P.tris + 3 * t;
    v3 a = C->V[tv[0]], b = C->V[tv[1]], c = C->V[tv[2]];
    v3 nrm = cross(sub(b, a), sub(c, a));
    double area2 = norm(nrm);
    v3 nu = scl(nrm, 1.0 / area2);
    v3 P3[3] = {a, b, c};
    for (int i = 0; i < 3; ++i) {
        v3 p = P3[(i + 1) % 3], r = P3[(i + 2) % 3];
        /* signed area of (p, r, q) relative to the triangle, times the height over edge p-r */
        double sub_area2 = dot(cross(sub(r, p), sub(q, p)), nu);
        d[i] = sub_area2 / norm(sub(r, p));
    }
}

/* Is q inside face f (any of its triangles, inclusive)? *amb set if the answer changes when the
   outer boundary moves by +-AMB_TOL (inner diagonals do not count as boundary). */
static int in_face(const or_ctx* C, int f, v3 q, double tol, int* amb)
{
    int inside = 0, in_grow = 0, in_shrink = 0;
    for (int j = C->ftri_start[f]; j < C->ftri_start[f + 1]; ++j) {
        int t = C->ftri[j];
        double d[3];
        tri_edge_dist(C, t, q, d);
        int a = 1, g = 1, s = 1;
        for (int i = 0; i < 3; ++i) {
            if (d[i] < 0.0) a = 0;
            if (d[i] < -tol) g = 0;
            if (!C->edge_inner[3 * t + i] && d[i] < tol) s = 0;
            if (C->edge_inner[3 * t + i] && d[i] < 0.0) s = 0;
        }
        inside |= a; in_grow |= g; in_shrink |= s;
    }
    if (in_grow != in_shrink) *amb = 1;
    return inside;
}

/* Does segment a->b pass through any triangle (faces ign0, ign1 skipped) at a distance in
   [SEG_EPS, len - SEG_EPS] from a? Brute force over all triangles with an exact AABB prefilter. */
static int seg_blocked(const or_ctx* C, v3 a, v3 b, int ign0, int ign1, int* amb)
{
    v3 dir = sub(b, a);
    double len = norm(dir);
    double lo[3] = {fmin(a.x, b.x), fmin(a.y, b.y), fmin(a.z, b.z)};
    double hi[3] = {fmax(a.x, b.x), fmax(a.y, b.y), fmax(a.z, b.z)};
    int blocked = 0;
    for (int64_t t = 0; t < C->P.n_tris; ++t) {
        int f = C->P.face_id[t];
        if (f == ign0 || f == ign1) continue;
        const double* bx = C->tbox + 6 * t;
        const double pad = 1e-6;
        if (bx[0] > hi[0] + pad || bx[3] < lo[0] - pad || bx[1] > hi[1] + pad || bx[4] < lo[1] - pad ||
            bx[2] > hi[2] + pad || bx[5] < lo[2] - pad)
            continue;
        const int32_t* tv = C->P.tris + 3 * t;
        v3 v0 = C->V[tv[0]], v1 = C->V[tv[1]], v2 = C->V[tv[2]];
        v3 nrm = cross(sub(v1, v0), sub(v2, v0));
        double nn = norm(nrm);
        double den = dot(nrm, dir);
        double num = dot(nrm, sub(v0, a));
        if (fabs(den) <= 1e-12 * nn * len) {
            /* segment parallel to the plane: it can only touch the triangle if it lies in it */
            if (fabs(num) / nn < AMB_TOL) *amb = 1;
            continue;
        }
        double s = num / den;            /* plane hit at a + s*dir */
        double dist = s * len;           /* distance from a along the segment */
        v3 q = add(a, scl(dir, s));
        double d[3];
        tri_edge_dist(C, (int)t, q, d);
        int inside = d[0] >= 0.0 && d[1] >= 0.0 && d[2] >= 0.0;
        int in_range = dist >= OR_SEG_EPS && dist <= len - OR_SEG_EPS;
        /* conditioning of the hit point along the plane: 1/|sin(angle to plane)| */
        double sin_a = fabs(den) / (nn * len);
        double tol_in = AMB_TOL / sin_a;
        int grow = d[0] >= -tol_in && d[1] >= -tol_in && d[2] >= -tol_in;
        int shrink = 1;
        for (int i = 0; i < 3; ++i)
            if (d[i] < (C->edge_inner[3 * t + i] ? -tol_in : tol_in)) shrink = 0;
        int near_end = fabs(dist - OR_SEG_EPS) < AMB_TOL || fabs(dist - (len - OR_SEG_EPS)) < AMB_TOL;
        int range_grow = dist >= OR_SEG_EPS - AMB_TOL && dist <= len - OR_SEG_EPS + AMB_TOL;
        if (inside && in_range) blocked = 1;
        if ((grow && range_grow) && (!shrink || near_end)) {
            /* a hit that would appear or vanish under a perturbation of AMB_TOL; it only makes the
               decision ambiguous if no robust hit exists - resolved after the loop */
            *amb |= 2;
        }
        if (shrink && in_range && !near_end) *amb |= 4;   /* a robust hit */
    }
    return blocked;
}

/* Resolve the ambiguity bits of seg_blocked: ambiguous only when some hit is marginal and no hit is robust. */
static int seg_amb(int bits) { return (bits & 2) && !(bits & 4); }

/* Occlusion of one segment. The decision is ambiguous when some hit (or a segment lying in a
   triangle's plane) is marginal and no hit is robust: a robust hit blocks under any perturbation. */
static int blocked_decision(const or_ctx* C, v3 a, v3 b, int ign0, int ign1, int* amb)
{
    int bits = 0;
    int r = seg_blocked(C, a, b, ign0, ign1, &bits);
    if (((bits & 1) || seg_amb(bits)) && !(bits & 4)) *amb = 1;
    return r;
}

/* --------------------------------------------------------------------------------------------
 * Image method (Sec. II-B): validate a face sequence between src and dst.
 * pts_out receives src, P_1..P_k, dst. Returns 1 if the path is geometrically valid and unblocked.
 * ------------------------------------------------------------------------------------------ */
/* Each condition below is classified as passing, failing robustly (it fails under every perturbation
   of AMB_TOL) or marginal. The path is valid when every condition passes; the decision is ambiguous
   when some condition is marginal and none fails robustly (a robust failure rejects the sequence
   whatever the marginal ones do). */
static int validate_seq(const or_ctx* C, v3 src, int src_face, v3 dst, int dst_face,
                        const int* seq, int k, int* amb, v3* pts)
{
    v3 img[3];
    img[0] = src;
    for (int j = 1; j <= k; ++j) img[j] = mirror(C, img[j - 1], seq[j - 1]);
    pts[0] = src;
    pts[k + 1] = dst;
    v3 y = dst;
    int ok = 1, marg = 0, rfail = 0;
    double cond = 1.0;                      /* growth of the point error along the back-trace */
    for (int j = k; j >= 1; --j) {          /* back-trace from dst towards the images */
        int f = seq[j - 1];
        v3 d = sub(img[j], y);
        double den = dot(C->fn[f], d);
        if (den == 0.0) return 0;
        double t = (C->fd[f] - dot(C->fn[f], y)) / den;
        v3 p = add(y, scl(d, t));
        pts[j] = p;
        cond *= norm(d) / fabs(den);
        if (!(t > 0.0 && t < 1.0)) {        /* the plane does not separate y from the image */
            ok = 0;
            double gap = (t <= 0.0 ? -t : t - 1.0) * norm(d);   /* distance to the boundary case */
            if (gap > AMB_TOL * cond) rfail = 1; else marg = 1;
        }
        int a = 0;
        int in = in_face(C, f, p, AMB_TOL * cond, &a);
        if (!in) ok = 0;
        if (a) marg = 1; else if (!in) rfail = 1;
        y = p;
    }
    for (int j = 1; j <= k; ++j) {          /* both neighbours strictly on the same side of each plane */
        int f = seq[j - 1];
        double s1 = sdist(C, pts[j - 1], f), s2 = sdist(C, pts[j + 1], f);
        int near = fabs(s1) < AMB_TOL || fabs(s2) < AMB_TOL;
        if (!(s1 * s2 > 0.0)) {
            ok = 0;
            if (!near) rfail = 1;
        }
        if (near) marg = 1;
    }
    for (int j = 0; j <= k && !rfail; ++j) {   /* every real segment unblocked */
        int i0 = j == 0 ? src_face : seq[j - 1];
        int i1 = j == k ? dst_face : seq[j];
        int a = 0;
        int b = blocked_decision(C, pts[j], pts[j + 1], i0, i1, &a);
        if (b) ok = 0;
        if (a) marg = 1; else if (b) rfail = 1;
    }
    if (marg && !rfail) *amb = 1;
    return ok;
}

/* Sequence enumeration: id f for (f); id F + f1*F + f2 for (f1, f2). Consecutive faces must not
   share a plane. first_excl / last_excl: faces whose plane contains the RIS centre may not be the
   first (Rx leg) or last (Tx leg) bounce. */
static int coplanar(const or_ctx* C, int a, int b)
{
    v3 x = cross(C->fn[a], C->fn[b]);
    if (norm(x) > 1e-9) return 0;
    double s = dot(C->fn[a], C->fn[b]) > 0 ? 1.0 : -1.0;
    return fabs(C->fd[a] - s * C->fd[b]) < 1e-9;
}

static int contains_centre(const or_ctx* C, int f) { return fabs(sdist(C, C->c, f)) < 1e-6; }
static int contains_pt(const or_ctx* C, int f, v3 p) { return fabs(sdist(C, p, f)) < 1e-6; }

static int decode_seq(const or_ctx* C, int64_t id, int* seq)
{
    if (id < C->F) { seq[0] = (int)id; return 1; }
    int64_t r = id - C->F;
    seq[0] = (int)(r / C->F);
    seq[1] = (int)(r % C->F);
    return 2;
}

/* mode 0: Tx leg (src Tx, dst RIS centre), 1: Rx leg (src RIS centre), 2: environment (Tx -> Rx) */
static int seq_allowed(const or_ctx* C, const int* seq, int k, int mode)
{
    for (int j = 1; j < k; ++j)
        if (seq[j] == seq[j - 1] || coplanar(C, seq[j], seq[j - 1])) return 0;
    if (mode == 0 && contains_centre(C, seq[k - 1])) return 0;
    if (mode == 1 && contains_centre(C, seq[0])) return 0;
    return 1;
}

/* The same rule for the legs of one element validated at the element itself (strict mode): the
   bounce next to the element may not lie on a plane through the element. */
static int seq_allowed_at(const or_ctx* C, const int* seq, int k, int tx_leg, v3 e)
{
    for (int j = 1; j < k; ++j)
        if (seq[j] == seq[j - 1] || coplanar(C, seq[j], seq[j - 1])) return 0;
    return !contains_pt(C, tx_leg ? seq[k - 1] : seq[0], e);
}

/* --------------------------------------------------------------------------------------------
 * Path sets
 * ------------------------------------------------------------------------------------------ */
/* Tx leg: valid reflected sequences (ids ascending) and per-element direct visibility.
   Per-decision ambiguity (each output may be NULL): vis_amb[m] for the element's direct ray,
   amb_ids / *n_amb (capacity amb_cap) the sequences whose validity is ambiguous, *n_dec the number
   of decisions taken (elements plus allowed sequences). */
int or_tx_leg(const or_ctx* C, int64_t* seq_out, int64_t cap, int64_t* n_seq, uint8_t* vis_out,
              int32_t* amb_out, uint8_t* vis_amb, int64_t* amb_ids, int64_t amb_cap, int64_t* n_amb,
              int64_t* n_dec)
{
    int amb = 0;
    int64_t n = 0, na = 0, nd = 0;
    int F = C->F, hf = C->P.host_face;
    for (int m = 0; m < C->P.M; ++m) {
        int a = 0;
        vis_out[m] = !blocked_decision(C, C->tx, C->e[m], -1, hf, &a);
        if (vis_amb) vis_amb[m] = (uint8_t)(a != 0);
        amb |= a;
        ++nd;
    }
    int64_t n_ids = C->P.max_order_tx >= 2 ? (int64_t)F + (int64_t)F * F : (C->P.max_order_tx >= 1 ? F : 0);
    /* every sequence decided independently (in parallel), then listed in ascending id order;
       state: bit 0 allowed, bit 1 valid, bit 2 ambiguous */
    uint8_t* state = (uint8_t*)calloc(n_ids > 0 ? (size_t)n_ids : 1, 1);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t id = 0; id < n_ids; ++id) {
        int seq[2];
        int k = decode_seq(C, id, seq);
        if (!seq_allowed(C, seq, k, 0)) continue;
        v3 pts[4];
        int a = 0;
        int ok = validate_seq(C, C->tx, -1, C->c, hf, seq, k, &a, pts);
        state[id] = (uint8_t)(1 | (ok ? 2 : 0) | (a ? 4 : 0));
    }
    for (int64_t id = 0; id < n_ids; ++id) {
        if (!(state[id] & 1)) continue;
        ++nd;
        if (state[id] & 2) {
            if (n < cap) seq_out[n] = id;
            ++n;
        }
        if (state[id] & 4) {
            if (amb_ids && na < amb_cap) amb_ids[na] = id;
            ++na;
            amb = 1;
        }
    }
    free(state);
    *n_seq = n;
    *amb_out = amb;
    if (n_amb) *n_amb = na;
    if (n_dec) *n_dec = nd;
    return 0;
}

/* Per receiver: valid Rx-leg sequences (from the RIS centre), environment sequences (Tx -> Rx),
   LOS visibility, per-element direct visibility bits and an ambiguity flag (any decision of this
   receiver ambiguous). Per-decision ambiguity (each output may be NULL): los_amb[i]; vis_amb bits
   [n_rx][W] like vis_bits; amb_out_ids [n_rx][amb_cap] the Rx-leg (id) and environment (id | 2^62)
   sequences whose validity is ambiguous, n_amb[i] their number; n_dec[i] the decisions taken for
   the receiver (LOS, M elements, every allowed Rx-leg and environment sequence). */
int or_rx_paths(const or_ctx* C, const float* rx_xyz, int64_t n_rx, int64_t* seq_out, int32_t cap,
                int32_t* n_seq, int64_t* env_out, int32_t env_cap, int32_t* n_env, uint8_t* los,
                uint32_t* vis_bits, int32_t* amb_out, uint8_t* los_amb, uint32_t* vis_amb,
                int64_t* amb_out_ids, int32_t amb_cap, int32_t* n_amb, int64_t* n_dec)
{
    int F = C->F, hf = C->P.host_face, M = C->P.M;
    int W = (M + 31) / 32;
    int64_t n_ids = C->P.max_order_rx >= 2 ? (int64_t)F + (int64_t)F * F : (C->P.max_order_rx >= 1 ? F : 0);
    const int64_t env_tag = (int64_t)1 << 62;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n_rx; ++i) {
        v3 r = vf(rx_xyz + 3 * i);
        int amb = 0, a = 0, na = 0;
        int64_t nd = 1 + M;
        los[i] = !blocked_decision(C, C->tx, r, -1, -1, &a);
        if (los_amb) los_amb[i] = (uint8_t)(a != 0);
        amb |= a;
        for (int w = 0; w < W; ++w) {
            vis_bits[i * W + w] = 0;
            if (vis_amb) vis_amb[i * W + w] = 0;
        }
        for (int m = 0; m < M; ++m) {
            a = 0;
            if (!blocked_decision(C, C->e[m], r, hf, -1, &a)) vis_bits[i * W + m / 32] |= 1u << (m % 32);
            if (a && vis_amb) vis_amb[i * W + m / 32] |= 1u << (m % 32);
            amb |= a;
        }
        int n = 0, ne = 0;
        for (int64_t id = 0; id < n_ids; ++id) {
            int seq[2];
            int k = decode_seq(C, id, seq);
            v3 pts[4];
            if (seq_allowed(C, seq, k, 1)) {
                a = 0;
                ++nd;
                if (validate_seq(C, C->c, hf, r, -1, seq, k, &a, pts)) {
                    if (n < cap) seq_out[i * cap + n] = id;
                    ++n;
                }
                if (a) {
                    if (amb_out_ids && na < amb_cap) amb_out_ids[i * amb_cap + na] = id;
                    ++na;
                }
                amb |= a;
            }
            if (C->P.env_paths && seq_allowed(C, seq, k, 2)) {
                a = 0;
                ++nd;
                if (validate_seq(C, C->tx, -1, r, -1, seq, k, &a, pts)) {
                    if (ne < env_cap) env_out[i * env_cap + ne] = id;
                    ++ne;
                }
                if (a) {
                    if (amb_out_ids && na < amb_cap) amb_out_ids[i * amb_cap + na] = id | env_tag;
                    ++na;
                }
                amb |= a;
            }
        }
        n_seq[i] = n;
        n_env[i] = ne;
        amb_out[i] = amb;
        if (n_amb) n_amb[i] = na;
        if (n_dec) n_dec[i] = nd;
    }
    return 0;
}

/* --------------------------------------------------------------------------------------------
 * Field (Eq. 4 - Eq. 10)
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    double L;            /* total unfolded length */
    v3 dep;              /* unit direction leaving the first point */
    v3 arr_back;         /* unit direction from the last point back towards the previous one */
    double complex R;    /* product of Fresnel coefficients */
    v3 dir[3];           /* directions of the real segments, dir[0] = dep, dir[k] = -arr_back */
    int k, seq[2];       /* bounce faces in propagation order */
} leg_t;

/* A leg by the image method (Sec. II-B): the source is mirrored across the faces of the sequence
   in propagation order; the leg length is the distance from the last image to the destination, and
   the direction of every real segment follows from the straight unfolded line by undoing the
   mirrors one face at a time (last face first). For a sequence validated at the RIS centre this is
   applied to every element as is, whether or not that element's own reflection points fall inside
   the segment (the element is not re-validated). */
static leg_t leg_by_images(const or_ctx* C, v3 src, v3 dst, const int* seq, int k)
{
    leg_t g;
    v3 img = src;
    for (int j = 0; j < k; ++j) img = mirror(C, img, seq[j]);
    v3 d = sub(dst, img);
    g.L = norm(d);
    d = scl(d, 1.0 / g.L);
    v3 dir[3];                 /* dir[j]: direction of real segment j (0 = leaving the source) */
    dir[k] = d;
    for (int j = k; j >= 1; --j) {
        v3 n = C->fn[seq[j - 1]];
        dir[j - 1] = sub(dir[j], scl(n, 2.0 * dot(n, dir[j])));
    }
    g.dep = dir[0];
    g.arr_back = scl(dir[k], -1.0);
    g.k = k;
    for (int j = 0; j <= k; ++j) g.dir[j] = dir[j];
    for (int j = 0; j < k; ++j) g.seq[j] = seq[j];
    g.R = 1.0;
    for (int j = 1; j <= k; ++j)
        g.R *= fresnel_c(C, fabs(dot(dir[j - 1], C->fn[seq[j - 1]])), seq[j - 1]);
    return g;
}

/* Tx -> ... -> Rx without the RIS (LOS when k = 0): Eq. 4 launch field and Eq. 8 reception. */
static double complex direct_term(const or_ctx* C, const leg_t* g)
{
    const or_problem* P = &C->P;
    double Ft = or_pattern(P->tx_pattern, P->tx_gain, dot(g->dep, C->tx_z));
    double Fr = or_pattern(P->rx_pattern, P->rx_gain, dot(g->arr_back, C->rx_z));
    double amp = sqrt(2.0 * OR_ETA0 * P->tx_power * P->tx_gain * Ft) * sqrt(P->rx_gain * Fr) *
                 C->lam / (4.0 * OR_PI * g->L);
    return amp * g->R * cexp(-I * C->k * g->L);
}

/* One RIS term e_mpq without Gamma_m (Eq. 4, Eq. 7, Eq. 8). */
static double complex ris_term(const or_ctx* C, const leg_t* gt, const leg_t* gr)
{
    const or_problem* P = &C->P;
    double Ft = or_pattern(P->tx_pattern, P->tx_gain, dot(gt->dep, C->tx_z));
    double Fin = elem_pattern(dot(gt->arr_back, C->n));
    double Fout = elem_pattern(dot(gr->dep, C->n));
    double Fr = or_pattern(P->rx_pattern, P->rx_gain, dot(gr->arr_back, C->rx_z));
    double Et = sqrt(2.0 * OR_ETA0 * P->tx_power * P->tx_gain * Ft);                    /* Eq. 4 */
    double ris = sqrt(C->G * Fin * Fout * (double)P->dy * (double)P->dz / (4.0 * OR_PI)) / gt->L; /* Eq. 7 */
    double rx = sqrt(P->rx_gain * Fr) * C->lam / (4.0 * OR_PI * gr->L);                 /* Eq. 8 */
    return Et * ris * rx * gt->R * gr->R * cexp(-I * C->k * (gt->L + gr->L));
}

/* ---------------------------------------------------------------------------------------------
 * Vector mode (polarisation factors as described in the file header)
 * ------------------------------------------------------------------------------------------- */
typedef struct { double complex x, y, z; } cv3;

static cv3 cv_real(v3 a) { cv3 r = {a.x, a.y, a.z}; return r; }
static cv3 cv_scale(cv3 a, double complex s) { cv3 r = {a.x * s, a.y * s, a.z * s}; return r; }
static cv3 cv_add(cv3 a, cv3 b) { cv3 r = {a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
static double complex cv_dot(cv3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }   /* bilinear */
static double cv_norm(cv3 a) { return sqrt(cabs(a.x) * cabs(a.x) + cabs(a.y) * cabs(a.y) + cabs(a.z) * cabs(a.z)); }

/* unit(P(k) a): the field direction of an antenna with polarisation axis a for propagation direction k
   (zero when a lies along k) */
static v3 pol_dir(v3 a, v3 k)
{
    v3 p = sub(a, scl(k, dot(a, k)));
    double l = norm(p);
    return l > 1e-12 ? scl(p, 1.0 / l) : mk(0, 0, 0);
}

/* One bounce on face f of a field e travelling along kin, leaving along kout: TE part along
   s = unit(kin x n) scaled by R_TE, TM part from p_in = s x kin to p_out = s x kout scaled by R_TM. */
static cv3 bounce_vec(const or_ctx* C, cv3 e, v3 kin, v3 kout, int f)
{
    const v3 n = C->fn[f];
    const double ci = fabs(dot(kin, n));
    const int m = C->fmat[f];
    double re, im;
    or_fresnel(ci, C->P.mats[2 * m], C->P.mats[2 * m + 1], C->P.freq, 0, &re, &im);
    const double complex rte = re + I * im;
    or_fresnel(ci, C->P.mats[2 * m], C->P.mats[2 * m + 1], C->P.freq, 1, &re, &im);
    const double complex rtm = re + I * im;
    v3 s = cross(kin, n);
    const double ls = norm(s);
    if (ls < 1e-12) return cv_scale(e, rte);        /* normal incidence: R_TM = -R_TE, p_out = -p_in */
    s = scl(s, 1.0 / ls);
    const v3 pin = cross(s, kin), pout = cross(s, kout);
    return cv_add(cv_scale(cv_real(s), rte * cv_dot(e, s)), cv_scale(cv_real(pout), rtm * cv_dot(e, pin)));
}

/* the bounces of a leg in propagation order */
static cv3 leg_vec(const or_ctx* C, const leg_t* g, cv3 e)
{
    for (int j = 1; j <= g->k; ++j) e = bounce_vec(C, e, g->dir[j - 1], g->dir[j], g->seq[j - 1]);
    return e;
}

/* Vector mode, Tx -> ... -> Rx without the RIS: the received value; *E3 the field vector. */
static double complex direct_term_vec(const or_ctx* C, const leg_t* g, cv3* E3)
{
    const or_problem* P = &C->P;
    double Ft = or_pattern(P->tx_pattern, P->tx_gain, dot(g->dep, C->tx_z));
    double Fr = or_pattern(P->rx_pattern, P->rx_gain, dot(g->arr_back, C->rx_z));
    double amp = sqrt(2.0 * OR_ETA0 * P->tx_power * P->tx_gain * Ft) * sqrt(P->rx_gain * Fr) *
                 C->lam / (4.0 * OR_PI * g->L);
    const double complex a = amp * cexp(-I * C->k * g->L);
    const cv3 e = leg_vec(C, g, cv_real(pol_dir(C->tx_pol, g->dep)));
    *E3 = cv_scale(e, a);
    return a * cv_dot(e, pol_dir(C->rx_pol, g->dir[g->k]));
}

/* Vector mode, one RIS term e_mpq without Gamma_m: the received value; *E3 the field vector. */
static double complex ris_term_vec(const or_ctx* C, const leg_t* gt, const leg_t* gr, cv3* E3)
{
    const or_problem* P = &C->P;
    double Ft = or_pattern(P->tx_pattern, P->tx_gain, dot(gt->dep, C->tx_z));
    double Fin = elem_pattern(dot(gt->arr_back, C->n));
    double Fout = elem_pattern(dot(gr->dep, C->n));
    double Fr = or_pattern(P->rx_pattern, P->rx_gain, dot(gr->arr_back, C->rx_z));
    double Et = sqrt(2.0 * OR_ETA0 * P->tx_power * P->tx_gain * Ft);                    /* Eq. 4 */
    double ris = sqrt(C->G * Fin * Fout * (double)P->dy * (double)P->dz / (4.0 * OR_PI)) / gt->L; /* Eq. 7 */
    double rx = sqrt(P->rx_gain * Fr) * C->lam / (4.0 * OR_PI * gr->L);                 /* Eq. 8 */
    const double complex a = Et * ris * rx * cexp(-I * C->k * (gt->L + gr->L));
    cv3 e = leg_vec(C, gt, cv_real(pol_dir(C->tx_pol, gt->dep)));
    e = cv_add(e, cv_scale(cv_real(C->n), -2.0 * cv_dot(e, C->n)));      /* normal component reversed */
    const v3 ko = gr->dir[0];
    e = cv_add(e, cv_scale(cv_real(ko), -cv_dot(e, ko)));                 /* outgoing wavefront */
    e = leg_vec(C, gr, e);
    *E3 = cv_scale(e, a);
    return a * cv_dot(e, pol_dir(C->rx_pol, gr->dir[gr->k]));
}

/* For each receiver: E0 = E_LOS + E_env, S0 = |E_LOS| + sum |env terms|, the channel row
   A[m] = sum_p sum_q e_mpq (so E = E0 + sum_m Gamma_m A[m]), SA[m] = sum_p sum_q |e_mpq| and an
   ambiguity flag covering every decision this receiver depends on (Tx-leg ones included). */
static int field_impl(const or_ctx* C, const float* rx_xyz, int64_t n_rx, double* E0, double* S0, double* A,
                      double* SA, int32_t* amb_out, double* E03, double* S03, double* A3, double* SA3)
{
    const int vec = C->P.vector_pol != 0;
    int F = C->F, hf = C->P.host_face, M = C->P.M;
    /* Tx leg (shared by all receivers) */
    int64_t cap = 1 << 20;
    int64_t* tx_ids = (int64_t*)malloc(sizeof(int64_t) * cap);
    uint8_t* tx_vis = (uint8_t*)malloc(M > 0 ? M : 1);
    int64_t n_tx = 0;
    int32_t tx_amb = 0;
    or_tx_leg(C, tx_ids, cap, &n_tx, tx_vis, &tx_amb, NULL, NULL, 0, NULL, NULL);
    if (n_tx > cap) n_tx = cap;
    int64_t n_ids = C->P.max_order_rx >= 2 ? (int64_t)F + (int64_t)F * F : (C->P.max_order_rx >= 1 ? F : 0);
    /* strict mode: every element's own valid Tx-leg sequences */
    const int strict = C->P.strict_elements != 0;
    int64_t n_tx_ids = C->P.max_order_tx >= 2 ? (int64_t)F + (int64_t)F * F : (C->P.max_order_tx >= 1 ? F : 0);
    int64_t* stx_ids = NULL;
    int64_t* stx_n = NULL;
    int* stx_amb = NULL;
    if (strict) {
        stx_ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M > 0 ? M : 1) * (size_t)(n_tx_ids > 0 ? n_tx_ids : 1));
        stx_n = (int64_t*)calloc(M > 0 ? M : 1, sizeof(int64_t));
        stx_amb = (int*)calloc(M > 0 ? M : 1, sizeof(int));
#pragma omp parallel for schedule(dynamic, 1)
        for (int m = 0; m < M; ++m) {
            for (int64_t id = 0; id < n_tx_ids; ++id) {
                int seq[2];
                int k = decode_seq(C, id, seq);
                v3 pts[4];
                if (seq_allowed_at(C, seq, k, 1, C->e[m]) &&
                    validate_seq(C, C->tx, -1, C->e[m], hf, seq, k, &stx_amb[m], pts))
                    stx_ids[(int64_t)m * n_tx_ids + stx_n[m]++] = id;
            }
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n_rx; ++i) {
        v3 r = vf(rx_xyz + 3 * i);
        int amb = tx_amb;
        double complex e0 = 0.0;
        double s0 = 0.0, s03 = 0.0;
        cv3 e03 = {0.0, 0.0, 0.0}, t3;
        /* LOS (Friis form of Eq. 4 + Eq. 8) */
        if (!blocked_decision(C, C->tx, r, -1, -1, &amb)) {
            leg_t g = leg_by_images(C, C->tx, r, NULL, 0);
            double complex v = vec ? direct_term_vec(C, &g, &t3) : direct_term(C, &g);
            e0 += v;
            s0 += cabs(v);
            if (vec) {
                e03 = cv_add(e03, t3);
                s03 += cv_norm(t3);
            }
        }
        /* valid Rx-leg sequences (validated once at the RIS centre) and environment paths */
        int64_t* rx_ids = (int64_t*)malloc(sizeof(int64_t) * (n_ids > 0 ? n_ids : 1));
        int n_q = 0;
        for (int64_t id = 0; id < n_ids; ++id) {
            int seq[2];
            int k = decode_seq(C, id, seq);
            v3 pts[4];
            if (seq_allowed(C, seq, k, 1) && validate_seq(C, C->c, hf, r, -1, seq, k, &amb, pts))
                rx_ids[n_q++] = id;
            if (C->P.env_paths && seq_allowed(C, seq, k, 2) && validate_seq(C, C->tx, -1, r, -1, seq, k, &amb, pts)) {
                leg_t g = leg_by_images(C, C->tx, r, seq, k);
                double complex v = vec ? direct_term_vec(C, &g, &t3) : direct_term(C, &g);
                e0 += v;
                s0 += cabs(v);
                if (vec) {
                    e03 = cv_add(e03, t3);
                    s03 += cv_norm(t3);
                }
            }
        }
        int64_t* m_rx = strict ? (int64_t*)malloc(sizeof(int64_t) * (n_ids > 0 ? n_ids : 1)) : NULL;
        for (int m = 0; m < M; ++m) {
            double complex a = 0.0;
            double sa = 0.0, sa3 = 0.0;
            cv3 a3 = {0.0, 0.0, 0.0};
            int rx_direct = !blocked_decision(C, C->e[m], r, hf, -1, &amb);
            /* the element's reflected legs: validated once at the RIS centre (Sec. II-B), or, in strict
               mode, between the element itself and each end */
            const int64_t* mt_ids = tx_ids;
            int64_t mt_n = n_tx;
            const int64_t* mr_ids = rx_ids;
            int mr_n = n_q;
            if (strict) {
                mt_ids = stx_ids + (int64_t)m * n_tx_ids;
                mt_n = stx_n[m];
                amb |= stx_amb[m];
                mr_n = 0;
                for (int64_t id = 0; id < n_ids; ++id) {
                    int seq[2];
                    int k = decode_seq(C, id, seq);
                    v3 pts[4];
                    if (seq_allowed_at(C, seq, k, 0, C->e[m]) && validate_seq(C, C->e[m], hf, r, -1, seq, k, &amb, pts))
                        m_rx[mr_n++] = id;
                }
                mr_ids = m_rx;
            }
            for (int64_t p = -1; p < mt_n; ++p) {           /* p = -1: direct Tx -> e_m */
                int tseq[2], tk = 0;
                if (p < 0) {
                    if (!tx_vis[m]) continue;
                } else {
                    tk = decode_seq(C, mt_ids[p], tseq);
                }
                leg_t gt = leg_by_images(C, C->tx, C->e[m], tseq, tk);
                for (int q = -1; q < mr_n; ++q) {           /* q = -1: direct e_m -> Rx */
                    int rseq[2], rk = 0;
                    if (q < 0) {
                        if (!rx_direct) continue;
                    } else {
                        rk = decode_seq(C, mr_ids[q], rseq);
                    }
                    leg_t gr = leg_by_images(C, C->e[m], r, rseq, rk);
                    double complex v = vec ? ris_term_vec(C, &gt, &gr, &t3) : ris_term(C, &gt, &gr);
                    a += v;
                    sa += cabs(v);
                    if (vec) {
                        a3 = cv_add(a3, t3);
                        sa3 += cv_norm(t3);
                    }
                }
            }
            A[(i * M + m) * 2] = creal(a);
            A[(i * M + m) * 2 + 1] = cimag(a);
            SA[i * M + m] = sa;
            if (A3) {
                double complex c3[3] = {a3.x, a3.y, a3.z};
                for (int j = 0; j < 3; ++j) {
                    A3[((i * M + m) * 3 + j) * 2] = creal(c3[j]);
                    A3[((i * M + m) * 3 + j) * 2 + 1] = cimag(c3[j]);
                }
                SA3[i * M + m] = sa3;
            }
        }
        free(m_rx);
        free(rx_ids);
        E0[2 * i] = creal(e0);
        E0[2 * i + 1] = cimag(e0);
        S0[i] = s0;
        if (E03) {
            double complex c3[3] = {e03.x, e03.y, e03.z};
            for (int j = 0; j < 3; ++j) {
                E03[(i * 3 + j) * 2] = creal(c3[j]);
                E03[(i * 3 + j) * 2 + 1] = cimag(c3[j]);
            }
            S03[i] = s03;
        }
        amb_out[i] = amb;
    }
    free(tx_ids);
    free(tx_vis);
    free(stx_ids);
    free(stx_n);
    free(stx_amb);
    return 0;
}

int or_field(const or_ctx* C, const float* rx_xyz, int64_t n_rx, double* E0, double* S0, double* A,
             double* SA, int32_t* amb_out, int32_t max_paths)
{
    (void)max_paths;
    return field_impl(C, rx_xyz, n_rx, E0, S0, A, SA, amb_out, NULL, NULL, NULL, NULL);
}

/* Vector mode: or_field's outputs (the received values) and the field vectors E03 [n][3], A3 [n][M][3]
   (complex, as interleaved pairs) with their incoherent magnitudes S03, SA3 (sums of term norms). */
int or_field_vec(const or_ctx* C, const float* rx_xyz, int64_t n_rx, double* E0, double* S0, double* A, double* SA,
                 int32_t* amb_out, double* E03, double* S03, double* A3, double* SA3)
{
    if (!C->P.vector_pol) return -1;
    return field_impl(C, rx_xyz, n_rx, E0, S0, A, SA, amb_out, E03, S03, A3, SA3);
}

/* Strict mode's path sets of element m (its reflected legs validated at the element itself):
   valid Tx-leg ids (ascending) with per-decision ambiguity, and per receiver its valid Rx-leg ids with
   the ambiguous ones; n_dec counts the decisions. Layout as or_tx_leg / or_rx_paths. */
int or_element_paths(const or_ctx* C, int m, const float* rx_xyz, int64_t n_rx, int64_t* tx_out, int64_t tx_cap,
                     int64_t* n_tx, int64_t* tx_amb_ids, int64_t tx_amb_cap, int64_t* n_tx_amb, int64_t* seq_out,
                     int32_t cap, int32_t* n_seq, int64_t* amb_ids, int32_t amb_cap, int32_t* n_amb, int64_t* n_dec)
{
    int F = C->F, hf = C->P.host_face;
    v3 e = C->e[m];
    int64_t n_tx_ids = C->P.max_order_tx >= 2 ? (int64_t)F + (int64_t)F * F : (C->P.max_order_tx >= 1 ? F : 0);
    int64_t n = 0, na = 0, nd = 0;
    for (int64_t id = 0; id < n_tx_ids; ++id) {
        int seq[2];
        int k = decode_seq(C, id, seq);
        if (!seq_allowed_at(C, seq, k, 1, e)) continue;
        v3 pts[4];
        int a = 0;
        ++nd;
        if (validate_seq(C, C->tx, -1, e, hf, seq, k, &a, pts)) {
            if (n < tx_cap) tx_out[n] = id;
            ++n;
        }
        if (a) {
            if (na < tx_amb_cap) tx_amb_ids[na] = id;
            ++na;
        }
    }
    *n_tx = n;
    *n_tx_amb = na;
    int64_t n_ids = C->P.max_order_rx >= 2 ? (int64_t)F + (int64_t)F * F : (C->P.max_order_rx >= 1 ? F : 0);
    int64_t nd_rx = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nd_rx)
    for (int64_t i = 0; i < n_rx; ++i) {
        v3 r = vf(rx_xyz + 3 * i);
        int nq = 0, nqa = 0;
        for (int64_t id = 0; id < n_ids; ++id) {
            int seq[2];
            int k = decode_seq(C, id, seq);
            if (!seq_allowed_at(C, seq, k, 0, e)) continue;
            v3 pts[4];
            int a = 0;
            ++nd_rx;
            if (validate_seq(C, e, hf, r, -1, seq, k, &a, pts)) {
                if (nq < cap) seq_out[i * cap + nq] = id;
                ++nq;
            }
            if (a) {
                if (nqa < amb_cap) amb_ids[i * amb_cap + nqa] = id;
                ++nqa;
            }
        }
        n_seq[i] = nq;
        n_amb[i] = nqa;
    }
    *n_dec = nd + nd_rx;
    return 0;
}

/* Channel impulse response of the RIS part (Sec. II-B: every multipath component through the RIS),
   per receiver: one tap per pair (Rx-leg path q, Tx-leg path p) in the order q = direct, then the
   valid Rx-leg sequences by ascending id; within q, p = direct, then the valid Tx-leg sequences by
   ascending id. The tap's amplitude is sum_m Gamma_m e_mpq (the plain triple sum restricted to one
   (p, q); a direct leg counts only the elements it reaches unblocked), its delay the travel time of
   the path through the RIS centre, (|T_p - c| + |I_q - c|) / c0 with T_p, I_q the image-method end
   points. gamma [M] interleaved (re, im); outputs [n_rx][cap]: amp (re, im), sabs (sum_m |Gamma_m e_mpq|,
   the tap's incoherent magnitude), delay (s), p_id and q_id
   (-1 for a direct leg); count[n_rx] (may exceed cap: then only cap taps are written). */
int or_cir(const or_ctx* C, const float* rx_xyz, int64_t n_rx, const double* gamma, int32_t cap, double* amp,
           double* sabs, double* delay, int64_t* p_id, int64_t* q_id, int32_t* count)
{
    if (C->P.vector_pol) return -1;           /* taps of the scalar model only */
    int F = C->F, hf = C->P.host_face, M = C->P.M;
    int64_t tcap = 1 << 20;
    int64_t* tx_ids = (int64_t*)malloc(sizeof(int64_t) * tcap);
    uint8_t* tx_vis = (uint8_t*)malloc(M > 0 ? M : 1);
    int64_t n_tx = 0;
    int32_t tx_amb = 0;
    or_tx_leg(C, tx_ids, tcap, &n_tx, tx_vis, &tx_amb, NULL, NULL, 0, NULL, NULL);
    if (n_tx > tcap) n_tx = tcap;
    int64_t n_ids = C->P.max_order_rx >= 2 ? (int64_t)F + (int64_t)F * F : (C->P.max_order_rx >= 1 ? F : 0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n_rx; ++i) {
        v3 r = vf(rx_xyz + 3 * i);
        int amb = 0;
        int64_t* rx_ids = (int64_t*)malloc(sizeof(int64_t) * (n_ids > 0 ? n_ids : 1));
        int n_q = 0;
        for (int64_t id = 0; id < n_ids; ++id) {
            int seq[2];
            int k = decode_seq(C, id, seq);
            v3 pts[4];
            if (seq_allowed(C, seq, k, 1) && validate_seq(C, C->c, hf, r, -1, seq, k, &amb, pts)) rx_ids[n_q++] = id;
        }
        uint8_t* rx_direct = (uint8_t*)malloc(M > 0 ? M : 1);
        for (int m = 0; m < M; ++m) rx_direct[m] = !blocked_decision(C, C->e[m], r, hf, -1, &amb);
        int nt = 0;
        for (int q = -1; q < n_q; ++q) {
            int rseq[2], rk = 0;
            if (q >= 0) rk = decode_seq(C, rx_ids[q], rseq);
            double Lq = leg_by_images(C, C->c, r, rseq, rk).L;
            for (int64_t p = -1; p < n_tx; ++p) {
                int tseq[2], tk = 0;
                if (p >= 0) tk = decode_seq(C, tx_ids[p], tseq);
                double Lp = leg_by_images(C, C->tx, C->c, tseq, tk).L;
                double complex a = 0.0;
                double sa = 0.0;
                for (int m = 0; m < M; ++m) {
                    if (p < 0 && !tx_vis[m]) continue;
                    if (q < 0 && !rx_direct[m]) continue;
                    leg_t gt = leg_by_images(C, C->tx, C->e[m], tseq, tk);
                    leg_t gr = leg_by_images(C, C->e[m], r, rseq, rk);
                    double complex g = gamma[2 * m] + I * gamma[2 * m + 1];
                    double complex v = g * ris_term(C, &gt, &gr);
                    a += v;
                    sa += cabs(v);
                }
                if (nt < cap) {
                    int64_t o = i * cap + nt;
                    amp[2 * o] = creal(a);
                    amp[2 * o + 1] = cimag(a);
                    sabs[o] = sa;
                    delay[o] = (Lp + Lq) / OR_C0;
                    p_id[o] = p < 0 ? -1 : tx_ids[p];
                    q_id[o] = q < 0 ? -1 : rx_ids[q];
                }
                ++nt;
            }
        }
        count[i] = nt;
        free(rx_direct);
        free(rx_ids);
    }
    free(tx_ids);
    free(tx_vis);
    return 0;
}

/* Element positions as the oracle sees them (for tests of the frame convention). */
void or_element_positions(const or_ctx* C, double* out)
{
    for (int m = 0; m < C->P.M; ++m) {
        out[3 * m] = C->e[m].x; out[3 * m + 1] = C->e[m].y; out[3 * m + 2] = C->e[m].z;
    }
}

/* Single-segment occlusion query (tests). Returns blocked; *amb receives the ambiguity flag. */
int or_segment_blocked(const or_ctx* C, const double* a, const double* b, int ign0, int ign1, int32_t* amb)
{
    int am = 0;
    int r = blocked_decision(C, mk(a[0], a[1], a[2]), mk(b[0], b[1], b[2]), ign0, ign1, &am);
    *amb = am;
    return r;
}

/* Single-sequence validation query (tests): pts receives src, P_1..P_k, dst (double[3*(k+2)]). */
int or_validate(const or_ctx* C, const double* src, int src_face, const double* dst, int dst_face,
                int64_t id, int32_t* amb, double* pts_out)
{
    int seq[2];
    int k = decode_seq(C, id, seq);
    v3 pts[4];
    int am = 0;
    int ok = validate_seq(C, mk(src[0], src[1], src[2]), src_face, mk(dst[0], dst[1], dst[2]), dst_face,
                          seq, k, &am, pts);
    for (int j = 0; j < k + 2; ++j) {
        pts_out[3 * j] = pts[j].x; pts_out[3 * j + 1] = pts[j].y; pts_out[3 * j + 2] = pts[j].z;
    }
    *amb = am;
    return ok;
}
