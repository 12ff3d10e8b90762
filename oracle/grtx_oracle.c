/*
 * grtx_oracle.c -- plain, slow FP64 CPU reference for GRTX-style Gaussian ray tracing.
 *
 * TEST INFRASTRUCTURE ONLY. The library's product path never calls, links or loads this
 * file; only the test-suite, the smoke check and the benchmark's CPU-baseline leg do. It
 * shares no code, header, table or helper with the CUDA implementation.
 *
 * Every floating-point quantity is double precision unless a function says otherwise
 * (the Morton-code quantiser works in FP32 on purpose: that integer decision is taken in
 * the precision of the kernel under test).
 *
 * What is computed and where the paper defines it:
 *   - Gaussian parameters: mean mu, covariance Sigma = R S^2 R^T from a rotation quaternion
 *     and scales, opacity o, SH colour coefficients (Sec. II-B).
 *   - Max-response depth t_alpha = (mu - r_o)^T Sigma^-1 r_d / (r_d^T Sigma^-1 r_d) and
 *     alpha = o * G(r_o + t_alpha r_d)  (Sec. III-A, Eq. t-max-resp).
 *   - View-dependent colour from SH coefficients and the ray direction (Sec. III-A).
 *   - Front-to-back alpha compositing C = sum_i alpha_i c_i prod_{j<i} (1 - alpha_j)
 *     (Sec. II-B, Eq. volume-render) with early ray termination once the accumulated
 *     opacity passes a threshold (Sec. III-A, Sec. III-C Observation II).
 *   - The unit-sphere view of a Gaussian after a per-instance ray transform (Sec. IV-A).
 *   - Multi-round k-buffer tracing (Sec. III-A), the any-hit/raygen round loop with an
 *     eviction buffer and traversal checkpointing (Sec. IV-B, Listing 1, walkthrough).
 *   - LBVH building blocks (Morton codes, binary radix tree, bottom-up bounds); the paper
 *     names a BVH (Sec. II-A) but builds it with a third-party builder, so these follow the
 *     textbook definitions of a Morton order and a binary radix tree.
 *   - The analytic gradient of the composite (the paper has no backward pass; this is the
 *     derivative of Eq. volume-render and Eq. t-max-resp).
 *
 * Readings where the paper is silent (stated once here, used throughout):
 *   - Hits are sorted by the key (t_alpha, id), lexicographically.
 *   - A Gaussian is hit iff alpha >= alpha_min and t_near < t_alpha <= t_far; Gaussians
 *     with o <= alpha_min are never hit. The ellipsoid of Sec. IV-A is the set where the
 *     response reaches alpha_min, so its radius is kappa = sqrt(2 ln(o / alpha_min)).
 *   - alpha is clamped at alpha_max before compositing; compositing stops right after
 *     the Gaussian that takes T below T_min.
 *   - Colour c = max(0, sum_k Y_k(dir) f_k + 0.5) with real spherical harmonics without
 *     the Condon-Shortley phase, evaluated at the normalised ray direction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------------------ */
/* Scene: raw parameters and the per-Gaussian quantities derived from them (Sec. II-B). */
/* ------------------------------------------------------------------------------------ */

typedef struct og_scene {
    int n, sh_degree, n_coef;
    double alpha_min;
    double *mu;     /* n*3 mean                                                        */
    double *s;      /* n*3 scales s = exp(log_scale)                                   */
    double *q;      /* n*4 normalised quaternion (w,x,y,z)                             */
    double *qnorm;  /* n norm of the raw quaternion                                    */
    double *R;      /* n*9 rotation, row-major; column j is local axis j in world      */
    double *P;      /* n*9 Sigma^-1 = R S^-2 R^T, row-major                            */
    double *o;      /* n opacity = sigmoid(logit)                                      */
    double *kappa;  /* n ellipsoid radius in Mahalanobis units (0 when not valid)      */
    double *A;      /* n*12 rows of [A|b]: x_unit = A x + b maps the ellipsoid to |x|<=1 */
    double *aabb;   /* n*6 world AABB of the ellipsoid (lo xyz, hi xyz)                */
    int *valid;     /* n: o > alpha_min                                                */
    double *sh;     /* n*n_coef*3 SH coefficients, coefficient-major per Gaussian      */
} og_scene;

/* Rotation matrix of a unit quaternion (w,x,y,z); the standard active-rotation form. */
static void og_quat_to_R(const double qn[4], double R[9])
{
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

OG_API void og_scene_free(og_scene *S)
{
    if (!S) return;
    free(S->mu); free(S->s); free(S->q); free(S->qnorm); free(S->R); free(S->P); free(S->o);
    free(S->kappa); free(S->A); free(S->aabb); free(S->valid); free(S->sh);
    free(S);
}

/* Activation and derived geometry (Sec. II-B; unit sphere of Sec. IV-A). */
OG_API og_scene *og_scene_create(int n, int sh_degree, const double *means, const double *log_scales,
                                 const double *quats, const double *logits, const double *sh,
                                 double alpha_min)
{
    og_scene *S = (og_scene *)calloc(1, sizeof(og_scene));
    if (!S) return NULL;
    S->n = n; S->sh_degree = sh_degree; S->n_coef = (sh_degree + 1) * (sh_degree + 1);
    S->alpha_min = alpha_min;
    size_t nn = (size_t)(n > 0 ? n : 1);
    S->mu = malloc(nn * 3 * sizeof(double)); S->s = malloc(nn * 3 * sizeof(double));
    S->q = malloc(nn * 4 * sizeof(double));  S->qnorm = malloc(nn * sizeof(double));
    S->R = malloc(nn * 9 * sizeof(double));
    S->P = malloc(nn * 9 * sizeof(double));  S->o = malloc(nn * sizeof(double));
    S->kappa = malloc(nn * sizeof(double));  S->A = malloc(nn * 12 * sizeof(double));
    S->aabb = malloc(nn * 6 * sizeof(double)); S->valid = malloc(nn * sizeof(int));
    S->sh = malloc(nn * (size_t)S->n_coef * 3 * sizeof(double));
    if (!S->mu || !S->s || !S->q || !S->qnorm || !S->R || !S->P || !S->o || !S->kappa || !S->A || !S->aabb ||
        !S->valid || !S->sh) { og_scene_free(S); return NULL; }
    memcpy(S->sh, sh, (size_t)n * S->n_coef * 3 * sizeof(double));
    for (int i = 0; i < n; ++i) {
        double *mu = S->mu + 3 * i, *s = S->s + 3 * i, *q = S->q + 4 * i, *R = S->R + 9 * i;
        double *P = S->P + 9 * i, *A = S->A + 12 * i, *bb = S->aabb + 6 * i;
        for (int a = 0; a < 3; ++a) { mu[a] = means[3 * i + a]; s[a] = exp(log_scales[3 * i + a]); }
        double qq = 0;
        for (int a = 0; a < 4; ++a) qq += quats[4 * i + a] * quats[4 * i + a];
        double qn = sqrt(qq);
        S->qnorm[i] = qn;
        for (int a = 0; a < 4; ++a) q[a] = quats[4 * i + a] / qn;
        og_quat_to_R(q, R);
        S->o[i] = 1.0 / (1.0 + exp(-logits[i]));
        /* Sigma^-1 = R diag(1/s^2) R^T */
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0;
                for (int m = 0; m < 3; ++m) acc += R[3 * r + m] * R[3 * c + m] / (s[m] * s[m]);
                P[3 * r + c] = acc;
            }
        S->valid[i] = S->o[i] > alpha_min;
        double kap = S->valid[i] ? sqrt(2.0 * log(S->o[i] / alpha_min)) : 0.0;
        S->kappa[i] = kap;
        /* unit-sphere transform: x_unit = diag(1/(kappa s)) R^T (x - mu) */
        for (int j = 0; j < 4 * 3; ++j) A[j] = 0.0;
        if (S->valid[i]) {
            for (int j = 0; j < 3; ++j) {
                double bj = 0;
                for (int a = 0; a < 3; ++a) {
                    A[4 * j + a] = R[3 * a + j] / (kap * s[j]);
                    bj -= A[4 * j + a] * mu[a];
                }
                A[4 * j + 3] = bj;
            }
        }
        /* AABB of {x : (x-mu)^T Sigma^-1 (x-mu) <= kappa^2}: half extent kappa sqrt(Sigma_aa) */
        for (int a = 0; a < 3; ++a) {
            double var = 0;
            for (int m = 0; m < 3; ++m) var += R[3 * a + m] * R[3 * a + m] * s[m] * s[m];
            double h = kap * sqrt(var);
            bb[a] = mu[a] - h;
            bb[3 + a] = mu[a] + h;
        }
    }
    return S;
}

OG_API void og_scene_export(const og_scene *S, double *o, double *s, double *R, double *P,
                            double *kappa, double *A, double *aabb, int *valid)
{
    size_t n = (size_t)S->n;
    if (o) memcpy(o, S->o, n * sizeof(double));
    if (s) memcpy(s, S->s, n * 3 * sizeof(double));
    if (R) memcpy(R, S->R, n * 9 * sizeof(double));
    if (P) memcpy(P, S->P, n * 9 * sizeof(double));
    if (kappa) memcpy(kappa, S->kappa, n * sizeof(double));
    if (A) memcpy(A, S->A, n * 12 * sizeof(double));
    if (aabb) memcpy(aabb, S->aabb, n * 6 * sizeof(double));
    if (valid) memcpy(valid, S->valid, n * sizeof(int));
}

/* ------------------------------------------------------------------------------------ */
/* Ray / Gaussian response (Sec. III-A, Eq. t-max-resp).                                 */
/* ------------------------------------------------------------------------------------ */

/* t_alpha, squared Mahalanobis distance d2 at t_alpha, and alpha = o exp(-d2/2). */
static void og_response(const og_scene *S, int i, const double ro[3], const double rd[3],
                        double *t_alpha, double *d2, double *alpha)
{
    const double *P = S->P + 9 * i, *mu = S->mu + 3 * i;
    double Pd[3], num = 0, den = 0;
    for (int r = 0; r < 3; ++r) Pd[r] = P[3 * r] * rd[0] + P[3 * r + 1] * rd[1] + P[3 * r + 2] * rd[2];
    for (int r = 0; r < 3; ++r) { num += (mu[r] - ro[r]) * Pd[r]; den += rd[r] * Pd[r]; }
    double t = num / den;
    double e[3];
    for (int r = 0; r < 3; ++r) e[r] = ro[r] + t * rd[r] - mu[r];
    double q = 0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) q += e[r] * P[3 * r + c] * e[c];
    *t_alpha = t;
    *d2 = q;
    *alpha = S->o[i] * exp(-0.5 * q);
}

/* The same ray/Gaussian pair seen through the unit-sphere transform of Sec. IV-A:
 * o_l = A r_o + b, d_l = A r_d; closest approach of the local line to the origin. */
OG_API void og_unit_sphere_test(const og_scene *S, int i, const double ro[3], const double rd[3],
                                double *t_alpha, double *D2)
{
    const double *A = S->A + 12 * i;
    double ol[3], dl[3];
    for (int j = 0; j < 3; ++j) {
        ol[j] = A[4 * j] * ro[0] + A[4 * j + 1] * ro[1] + A[4 * j + 2] * ro[2] + A[4 * j + 3];
        dl[j] = A[4 * j] * rd[0] + A[4 * j + 1] * rd[1] + A[4 * j + 2] * rd[2];
    }
    double a = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
    double b = ol[0] * dl[0] + ol[1] * dl[1] + ol[2] * dl[2];
    double t = -b / a;
    double p[3];
    for (int j = 0; j < 3; ++j) p[j] = ol[j] + t * dl[j];
    *t_alpha = t;
    *D2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
}

OG_API void og_response_one(const og_scene *S, int i, const double ro[3], const double rd[3],
                            double out[3])
{
    og_response(S, i, ro, rd, &out[0], &out[1], &out[2]);
}

/* ------------------------------------------------------------------------------------ */
/* Spherical harmonics (real basis, degree <= 3, no Condon-Shortley phase).              */
/* Index k = l*l + l + m. Normalisation constants are evaluated from their closed forms. */
/* ------------------------------------------------------------------------------------ */

OG_API void og_sh_basis(int degree, const double dir[3], double *Y)
{
    const double pi = 3.14159265358979323846;
    double x = dir[0], y = dir[1], z = dir[2];
    Y[0] = 0.5 * sqrt(1.0 / pi);
    if (degree < 1) return;
    double c1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = c1 * y; Y[2] = c1 * z; Y[3] = c1 * x;
    if (degree < 2) return;
    double c2a = 0.5 * sqrt(15.0 / pi), c2b = 0.25 * sqrt(5.0 / pi), c2c = 0.25 * sqrt(15.0 / pi);
    Y[4] = c2a * x * y;
    Y[5] = c2a * y * z;
    Y[6] = c2b * (3.0 * z * z - 1.0);
    Y[7] = c2a * x * z;
    Y[8] = c2c * (x * x - y * y);
    if (degree < 3) return;
    double c3a = 0.25 * sqrt(35.0 / (2.0 * pi)), c3b = 0.5 * sqrt(105.0 / pi);
    double c3c = 0.25 * sqrt(21.0 / (2.0 * pi)), c3d = 0.25 * sqrt(7.0 / pi);
    double c3e = 0.25 * sqrt(105.0 / pi);
    Y[9] = c3a * y * (3.0 * x * x - y * y);
    Y[10] = c3b * x * y * z;
    Y[11] = c3c * y * (5.0 * z * z - 1.0);
    Y[12] = c3d * z * (5.0 * z * z - 3.0);
    Y[13] = c3c * x * (5.0 * z * z - 1.0);
    Y[14] = c3e * z * (x * x - y * y);
    Y[15] = c3a * x * (x * x - 3.0 * y * y);
}

/* Colour of Gaussian i seen along unit direction dir; raw[ch] is the value before the clamp. */
static void og_color(const og_scene *S, int i, const double dir[3], double c[3], double raw[3])
{
    double Y[16];
    og_sh_basis(S->sh_degree, dir, Y);
    const double *f = S->sh + (size_t)i * S->n_coef * 3;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0;
        for (int k = 0; k < S->n_coef; ++k) acc += Y[k] * f[3 * k + ch];
        raw[ch] = acc + 0.5;
        c[ch] = raw[ch] > 0 ? raw[ch] : 0.0;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Cameras (ray generation). The paper fixes no camera convention; these are the        */
/* conventions of this implementation: pixel centres at (i+1/2, j+1/2), row 0 at top.   */
/* ------------------------------------------------------------------------------------ */

typedef struct og_camera {
    int type;            /* 0 pinhole, 1 equidistant fisheye                               */
    int width, height;
    double pos[3], right[3], up[3], forward[3];   /* orthonormal camera basis in world    */
    double fov;          /* pinhole: vertical field of view; fisheye: theta at half width  */
    double t_near, t_far;
} og_camera;

OG_API void og_camera_rays(const og_camera *cam, double *origins, double *dirs, double *tnear,
                           double *tfar)
{
    int W = cam->width, H = cam->height;
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            size_t r = (size_t)py * W + px;
            double d[3];
            if (cam->type == 0) {
                double th = tan(0.5 * cam->fov), aspect = (double)W / (double)H;
                double u = (2.0 * (px + 0.5) / W - 1.0) * th * aspect;
                double v = (1.0 - 2.0 * (py + 0.5) / H) * th;
                for (int a = 0; a < 3; ++a) d[a] = cam->forward[a] + u * cam->right[a] + v * cam->up[a];
            } else {
                double f = (0.5 * W) / cam->fov;
                double dx = px + 0.5 - 0.5 * W, dy = 0.5 * H - (py + 0.5);
                double rr = sqrt(dx * dx + dy * dy), th = rr / f;
                double cp = rr > 0 ? dx / rr : 1.0, sp = rr > 0 ? dy / rr : 0.0;
                for (int a = 0; a < 3; ++a)
                    d[a] = sin(th) * cp * cam->right[a] + sin(th) * sp * cam->up[a] + cos(th) * cam->forward[a];
            }
            double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int a = 0; a < 3; ++a) { origins[3 * r + a] = cam->pos[a]; dirs[3 * r + a] = d[a] / nd; }
            tnear[r] = cam->t_near;
            tfar[r] = cam->t_far;
        }
}

/* ------------------------------------------------------------------------------------ */
/* Definition mode: brute force over every Gaussian, sort, composite.                   */
/* ------------------------------------------------------------------------------------ */

typedef struct og_params {
    double alpha_min, T_min, alpha_max;
    double bg[3];
} og_params;

typedef struct og_hit { double t; int id; double alpha; } og_hit;

static int og_hit_cmp(const void *a, const void *b)
{
    const og_hit *x = (const og_hit *)a, *y = (const og_hit *)b;
    if (x->t < y->t) return -1;
    if (x->t > y->t) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Key order (t, id), lexicographic. */
static int og_key_less(double t1, int i1, double t2, int i2)
{
    return t1 < t2 || (t1 == t2 && i1 < i2);
}

/* Composite hits[0..nh) front to back (Eq. volume-render) with the alpha clamp and early
 * termination. Writes rgb + T to out[4]; returns the number of Gaussians blended. */
static int og_composite(const og_scene *S, const og_params *p, const double rd[3],
                        const og_hit *hits, int nh, double out[4], int *ids_out, int ids_cap)
{
    double dir[3], nd = sqrt(rd[0] * rd[0] + rd[1] * rd[1] + rd[2] * rd[2]);
    for (int a = 0; a < 3; ++a) dir[a] = rd[a] / nd;
    double C[3] = {0, 0, 0}, T = 1.0;
    int nb = 0;
    for (int h = 0; h < nh; ++h) {
        double a = hits[h].alpha < p->alpha_max ? hits[h].alpha : p->alpha_max;
        double c[3], raw[3];
        og_color(S, hits[h].id, dir, c, raw);
        for (int ch = 0; ch < 3; ++ch) C[ch] += T * a * c[ch];
        T *= (1.0 - a);
        if (ids_out && nb < ids_cap) ids_out[nb] = hits[h].id;
        ++nb;
        if (T < p->T_min) break;
    }
    for (int ch = 0; ch < 3; ++ch) out[ch] = C[ch] + T * p->bg[ch];
    out[3] = T;
    return nb;
}

/* All hits of one ray, sorted by (t_alpha, id). Returns the count; *hits is malloc'd. */
static int og_ray_hits(const og_scene *S, const og_params *p, const double ro[3], const double rd[3],
                       double tn, double tf, og_hit **hits_out)
{
    int cap = 64, nh = 0;
    og_hit *hits = (og_hit *)malloc(cap * sizeof(og_hit));
    for (int i = 0; i < S->n; ++i) {
        if (!S->valid[i]) continue;
        double t, d2, al;
        og_response(S, i, ro, rd, &t, &d2, &al);
        if (al >= p->alpha_min && t > tn && t <= tf) {
            if (nh == cap) { cap *= 2; hits = (og_hit *)realloc(hits, cap * sizeof(og_hit)); }
            hits[nh].t = t; hits[nh].id = i; hits[nh].alpha = al; ++nh;
        }
    }
    qsort(hits, nh, sizeof(og_hit), og_hit_cmp);
    *hits_out = hits;
    return nh;
}

/* Render n_rays rays. out: n_rays*4 (rgb, T). n_blend (optional): Gaussians blended per ray.
 * ids (optional): the first ids_cap blended ids of each ray, in blend order. */
OG_API void og_render(const og_scene *S, const og_params *p, int n_rays, const double *origins,
                      const double *dirs, const double *tnear, const double *tfar, double *out,
                      int *n_blend, int *ids, int ids_cap, int *n_hits_total)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < n_rays; ++r) {
        og_hit *hits;
        int nh = og_ray_hits(S, p, origins + 3 * r, dirs + 3 * r, tnear[r], tfar[r], &hits);
        int nb = og_composite(S, p, dirs + 3 * r, hits, nh, out + 4 * r,
                              ids ? ids + (size_t)r * ids_cap : NULL, ids_cap);
        if (n_blend) n_blend[r] = nb;
        if (n_hits_total) n_hits_total[r] = nh;
        free(hits);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Multi-level instancing (Sec. VI "Support for Dynamic and Multi-Object Scenes"): a     */
/* world of placed objects, each a Gaussian scene under an affine object-to-world map.   */
/* ------------------------------------------------------------------------------------ */

typedef struct og_whit { double t; int id; double alpha; int inst, g; } og_whit;

static int og_whit_cmp(const void *a, const void *b)
{
    const og_whit *x = (const og_whit *)a, *y = (const og_whit *)b;
    if (x->t < y->t) return -1;
    if (x->t > y->t) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Inverse of the 3x3 matrix m (row-major) by cofactors; returns the determinant. */
static double og_inv3(const double m[9], double inv[9])
{
    double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
    double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    inv[0] = c00 / det;
    inv[1] = (m[2] * m[7] - m[1] * m[8]) / det;
    inv[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    inv[3] = c01 / det;
    inv[4] = (m[0] * m[8] - m[2] * m[6]) / det;
    inv[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    inv[6] = c02 / det;
    inv[7] = (m[1] * m[6] - m[0] * m[7]) / det;
    inv[8] = (m[0] * m[4] - m[1] * m[3]) / det;
    return det;
}

/* Render through a world of n_inst instances: instance i places scenes[inst_scene[i]] with
 * the object-to-world map x_w = L x_o + c, M[12 i ..] = rows (L_r0 | c_0), (L_r1 | c_1),
 * (L_r2 | c_2). Per ray, by the definition: every Gaussian g of every instance is met along
 * the ray mapped into the object's frame, o_o = L^-1 (o - c), d_o = L^-1 d (an affine map, so
 * t is the world t); it is hit when its response reaches alpha_min with t_near < t <= t_far.
 * Hits are ordered by (t, world id), world id = (the n of the scenes of instances 0..i-1) +
 * g, and composited front to back with the colour seen along the object-frame direction
 * d_o / |d_o|. Outputs as og_render, ids in world ids. */
OG_API void og_world_render(og_scene *const *scenes, int n_inst, const int *inst_scene, const double *M,
                            const og_params *p, int n_rays, const double *origins, const double *dirs,
                            const double *tnear, const double *tfar, double *out, int *n_blend, int *ids,
                            int ids_cap, int *n_hits_total)
{
    double *Li = (double *)malloc(sizeof(double) * 9 * (n_inst > 0 ? n_inst : 1));
    int *id_base = (int *)malloc(sizeof(int) * (n_inst > 0 ? n_inst : 1));
    int base = 0;
    for (int i = 0; i < n_inst; ++i) {
        const double *m = M + 12 * i;
        double L[9] = {m[0], m[1], m[2], m[4], m[5], m[6], m[8], m[9], m[10]};
        og_inv3(L, Li + 9 * i);
        id_base[i] = base;
        base += scenes[inst_scene[i]]->n;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < n_rays; ++r) {
        const double *ro = origins + 3 * r, *rd = dirs + 3 * r;
        int cap = 64, nh = 0;
        og_whit *hits = (og_whit *)malloc(cap * sizeof(og_whit));
        double *dob = (double *)malloc(sizeof(double) * 3 * (n_inst > 0 ? n_inst : 1));
        for (int i = 0; i < n_inst; ++i) {
            const og_scene *S = scenes[inst_scene[i]];
            const double *m = M + 12 * i, *A = Li + 9 * i;
            double v[3] = {ro[0] - m[3], ro[1] - m[7], ro[2] - m[11]}, oo[3], od[3];
            for (int a = 0; a < 3; ++a) {
                oo[a] = A[3 * a] * v[0] + A[3 * a + 1] * v[1] + A[3 * a + 2] * v[2];
                od[a] = A[3 * a] * rd[0] + A[3 * a + 1] * rd[1] + A[3 * a + 2] * rd[2];
            }
            double nd = sqrt(od[0] * od[0] + od[1] * od[1] + od[2] * od[2]);
            for (int a = 0; a < 3; ++a) dob[3 * i + a] = od[a] / nd;
            for (int g = 0; g < S->n; ++g) {
                if (!S->valid[g]) continue;
                double t, d2, al;
                og_response(S, g, oo, od, &t, &d2, &al);
                if (al >= p->alpha_min && t > tnear[r] && t <= tfar[r]) {
                    if (nh == cap) { cap *= 2; hits = (og_whit *)realloc(hits, cap * sizeof(og_whit)); }
                    hits[nh].t = t; hits[nh].id = id_base[i] + g; hits[nh].alpha = al;
                    hits[nh].inst = i; hits[nh].g = g;
                    ++nh;
                }
            }
        }
        qsort(hits, nh, sizeof(og_whit), og_whit_cmp);
        double C[3] = {0, 0, 0}, T = 1.0;
        int nb = 0;
        for (int h = 0; h < nh; ++h) {
            double a = hits[h].alpha < p->alpha_max ? hits[h].alpha : p->alpha_max;
            double c[3], raw[3];
            og_color(scenes[inst_scene[hits[h].inst]], hits[h].g, dob + 3 * hits[h].inst, c, raw);
            for (int ch = 0; ch < 3; ++ch) C[ch] += T * a * c[ch];
            T *= (1.0 - a);
            if (ids && nb < ids_cap) ids[(size_t)r * ids_cap + nb] = hits[h].id;
            ++nb;
            if (T < p->T_min) break;
        }
        for (int ch = 0; ch < 3; ++ch) out[4 * r + ch] = C[ch] + T * p->bg[ch];
        out[4 * r + 3] = T;
        if (n_blend) n_blend[r] = nb;
        if (n_hits_total) n_hits_total[r] = nh;
        free(dob);
        free(hits);
    }
    free(Li);
    free(id_base);
}

OG_API int og_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* k-buffer insertion (Sec. III-A; any-hit shader of Listing 1).                         */
/* ------------------------------------------------------------------------------------ */

/* Insert (t,id) into the ascending k-buffer kt/kid holding *cnt <= k entries. When the
 * buffer was already full, the larger of {new entry, old farthest entry} is rejected: it is
 * returned through rej_t/rej_id and the function returns 1. Otherwise it returns 0. */
OG_API int og_kbuf_insert(double *kt, int *kid, int *cnt, int k, double t, int id, double *rej_t,
                          int *rej_id)
{
    int n = *cnt, rejected = 0;
    if (n == k) {
        if (!og_key_less(t, id, kt[k - 1], kid[k - 1])) { *rej_t = t; *rej_id = id; return 1; }
        *rej_t = kt[k - 1]; *rej_id = kid[k - 1];
        rejected = 1;
        n = k - 1;
    }
    int pos = n;
    while (pos > 0 && og_key_less(t, id, kt[pos - 1], kid[pos - 1])) {
        kt[pos] = kt[pos - 1]; kid[pos] = kid[pos - 1]; --pos;
    }
    kt[pos] = t; kid[pos] = id;
    *cnt = n + 1;
    return rejected;
}

/* ------------------------------------------------------------------------------------ */
/* A BVH over Gaussian AABBs for the round simulator: top-down median split, one        */
/* Gaussian per leaf (the instance-per-leaf tree of Sec. IV-A). Any valid BVH gives the  */
/* same image; this one exists only so the round loop has a tree to traverse.            */
/* ------------------------------------------------------------------------------------ */

typedef struct og_node { double lo[3], hi[3]; int left, right, leaf; } og_node;
typedef struct og_bvh { int n_nodes, root; og_node *nodes; } og_bvh;

static const og_scene *g_sort_scene;
static int g_sort_axis;
static int og_centroid_cmp(const void *a, const void *b)
{
    int i = *(const int *)a, j = *(const int *)b;
    const double *ba = g_sort_scene->aabb + 6 * i, *bb = g_sort_scene->aabb + 6 * j;
    double ca = ba[g_sort_axis] + ba[3 + g_sort_axis], cb = bb[g_sort_axis] + bb[3 + g_sort_axis];
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return (i > j) - (i < j);
}

static int og_bvh_rec(og_bvh *B, const og_scene *S, int *idx, int cnt)
{
    int me = B->n_nodes++;
    og_node *nd = &B->nodes[me];
    for (int a = 0; a < 3; ++a) { nd->lo[a] = INFINITY; nd->hi[a] = -INFINITY; }
    for (int j = 0; j < cnt; ++j) {
        const double *bb = S->aabb + 6 * idx[j];
        for (int a = 0; a < 3; ++a) {
            if (bb[a] < nd->lo[a]) nd->lo[a] = bb[a];
            if (bb[3 + a] > nd->hi[a]) nd->hi[a] = bb[3 + a];
        }
    }
    if (cnt == 1) { nd->leaf = idx[0]; nd->left = nd->right = -1; return me; }
    nd->leaf = -1;
    int axis = 0;
    double ext = -1;
    for (int a = 0; a < 3; ++a)
        if (nd->hi[a] - nd->lo[a] > ext) { ext = nd->hi[a] - nd->lo[a]; axis = a; }
    g_sort_scene = S; g_sort_axis = axis;
    qsort(idx, cnt, sizeof(int), og_centroid_cmp);
    int half = cnt / 2;
    int l = og_bvh_rec(B, S, idx, half);
    int r = og_bvh_rec(B, S, idx + half, cnt - half);
    B->nodes[me].left = l;
    B->nodes[me].right = r;
    return me;
}

OG_API og_bvh *og_bvh_build(const og_scene *S)
{
    og_bvh *B = (og_bvh *)calloc(1, sizeof(og_bvh));
    int nv = 0;
    int *idx = (int *)malloc((size_t)(S->n > 0 ? S->n : 1) * sizeof(int));
    for (int i = 0; i < S->n; ++i)
        if (S->valid[i]) idx[nv++] = i;
    B->nodes = (og_node *)calloc((size_t)(2 * nv + 1), sizeof(og_node));
    B->root = nv > 0 ? og_bvh_rec(B, S, idx, nv) : -1;
    free(idx);
    return B;
}

OG_API void og_bvh_free(og_bvh *B)
{
    if (!B) return;
    free(B->nodes);
    free(B);
}

OG_API int og_bvh_num_nodes(const og_bvh *B) { return B->n_nodes; }

/* Entry/exit of the ray with an AABB, clipped to [tn, tf]. Returns 0 on a miss. */
static int og_slab(const double lo[3], const double hi[3], const double ro[3], const double rd[3],
                   double tn, double tf, double *t0, double *t1)
{
    double a0 = tn, a1 = tf;
    for (int a = 0; a < 3; ++a) {
        double inv = 1.0 / rd[a];
        double ta = (lo[a] - ro[a]) * inv, tb = (hi[a] - ro[a]) * inv;
        double mn = fmin(ta, tb), mx = fmax(ta, tb);
        a0 = fmax(a0, mn);
        a1 = fmin(a1, mx);
    }
    *t0 = a0; *t1 = a1;
    return a0 <= a1;
}

/* ------------------------------------------------------------------------------------ */
/* Round mode: the multi-round k-buffer loop (Sec. III-A) with the raygen / any-hit      */
/* shaders of Listing 1, the eviction buffer and checkpointed traversal (Sec. IV-B).     */
/* ------------------------------------------------------------------------------------ */

typedef struct og_round_cfg {
    int k;            /* k-buffer size, >= 1                                               */
    int checkpoint;   /* 1: resume from checkpointed nodes + eviction buffer (Sec. IV-B);  */
                      /* 0: restart from the root every round with t_min = last blended   */
    int ckpt_cap;     /* checkpoint entries per round (< 0: unbounded)                    */
    int evict_cap;    /* eviction entries (< 0: unbounded)                                */
} og_round_cfg;

typedef struct og_round_stats {
    long long nodes, leaves, rounds, ckpt_writes, evictions, fallbacks, unique_nodes;
} og_round_stats;

typedef struct og_entry { double t; int ref; } og_entry;   /* node (or leaf) ref + entry t */
typedef struct og_list { og_entry *e; int n, cap; } og_list;

static void og_push(og_list *L, double t, int ref)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 64;
        L->e = (og_entry *)realloc(L->e, (size_t)L->cap * sizeof(og_entry));
    }
    L->e[L->n].t = t; L->e[L->n].ref = ref; ++L->n;
}

typedef struct og_ray_state {
    double *kt; int *kid; int cnt;          /* k-buffer                                       */
    og_hit *ev; int nev, evcap;             /* eviction buffer (t, id, alpha)                 */
    og_list src, dst, stack;                /* checkpoint ping-pong lists and traversal stack */
    unsigned char *seen;                    /* visited-node flags for the unique count        */
} og_ray_state;

/* Append a rejected hit to the eviction buffer (Listing 1, any-hit shader). Returns 1 when
 * the capacity is exceeded. */
static int og_evict(og_ray_state *st, const og_round_cfg *cfg, double t, int id)
{
    if (cfg->evict_cap >= 0 && st->nev >= cfg->evict_cap) return 1;
    if (st->nev == st->evcap) {
        st->evcap = st->evcap ? 2 * st->evcap : 64;
        st->ev = (og_hit *)realloc(st->ev, (size_t)st->evcap * sizeof(og_hit));
    }
    st->ev[st->nev].t = t; st->ev[st->nev].id = id; st->ev[st->nev].alpha = 0;
    st->nev++;
    return 0;
}

/* One traversal round over the interval (L, t_max] (Sec. III-A). With checkpoint = 1 the
 * round starts from the checkpoint source list and writes nodes that fail the t_max test to
 * the destination list, and rejected hits go to the eviction buffer (Sec. IV-B). With
 * checkpoint = 0 it starts from the root and simply culls (the restart baseline).
 * Returns 0 on success, 1 if a checkpoint or eviction capacity was exceeded. */
static int og_trace_round(const og_scene *S, const og_bvh *B, const og_params *p,
                          const og_round_cfg *cfg, og_ray_state *st, const double ro[3],
                          const double rd[3], double tn, double tf, double L_t, int L_id,
                          int checkpoint, og_round_stats *stats)
{
    int k = cfg->k;
    double tmax = st->cnt == k ? st->kt[k - 1] : INFINITY;
    og_list *work = &st->stack;
    work->n = 0;
    st->dst.n = 0;
    int n_roots = 0;
    if (checkpoint) {
        n_roots = st->src.n;
    } else {
        double t0, t1;
        const og_node *rt = &B->nodes[B->root];
        if (og_slab(rt->lo, rt->hi, ro, rd, tn, tf, &t0, &t1) && !(t1 < L_t)) og_push(work, t0, B->root);
    }
    int ri = 0;
    for (;;) {
        if (work->n == 0) {
            if (ri >= n_roots) break;
            og_push(work, st->src.e[ri].t, st->src.e[ri].ref);
            ++ri;
        }
        og_entry cur = work->e[--work->n];
        if (cur.t > tmax) {            /* fails the t_max test */
            if (checkpoint) {
                if (cfg->ckpt_cap >= 0 && st->dst.n >= cfg->ckpt_cap) return 1;
                og_push(&st->dst, cur.t, cur.ref);
                stats->ckpt_writes++;
            }
            continue;
        }
        const og_node *nd = &B->nodes[cur.ref];
        if (st->seen && !st->seen[cur.ref]) { st->seen[cur.ref] = 1; stats->unique_nodes++; }
        if (nd->leaf >= 0) {
            stats->leaves++;
            int g = nd->leaf;
            double t, d2, al;
            og_response(S, g, ro, rd, &t, &d2, &al);
            if (!(al >= p->alpha_min && t > tn && t <= tf)) continue;
            if (!og_key_less(L_t, L_id, t, g)) continue;      /* key <= L: blended already */
            double rt_; int rid;
            if (og_kbuf_insert(st->kt, st->kid, &st->cnt, k, t, g, &rt_, &rid) && checkpoint) {
                if (og_evict(st, cfg, rt_, rid)) return 1;
                stats->evictions++;
            }
            if (st->cnt == k) tmax = st->kt[k - 1];    /* tight t_max: the farthest kept key */
            continue;
        }
        stats->nodes++;
        /* internal node: test both children; the nearer child is traversed first */
        double e0, x0, e1, x1;
        const og_node *c0 = &B->nodes[nd->left], *c1 = &B->nodes[nd->right];
        int h0 = og_slab(c0->lo, c0->hi, ro, rd, tn, tf, &e0, &x0) && !(x0 < L_t);
        int h1 = og_slab(c1->lo, c1->hi, ro, rd, tn, tf, &e1, &x1) && !(x1 < L_t);
        if (h0 && h1) {
            if (e0 <= e1) { og_push(work, e1, nd->right); og_push(work, e0, nd->left); }
            else { og_push(work, e0, nd->left); og_push(work, e1, nd->right); }
        } else if (h0) {
            og_push(work, e0, nd->left);
        } else if (h1) {
            og_push(work, e1, nd->right);
        }
    }
    return 0;
}

/* Render with the multi-round loop of Listing 1 (raygen shader): before each round the
 * closest evicted hits move into the k-buffer, a traversal round runs, the k-buffer is
 * blended in order with per-Gaussian early termination, and the loop stops when the
 * k-buffer was not filled. Overflow of a capacity makes the ray redo that round from the
 * root and finish in restart mode, which is always correct. Outputs as og_render; stats
 * (optional) are summed over rays. */
OG_API void og_render_rounds(const og_scene *S, const og_bvh *B, const og_params *p,
                             const og_round_cfg *cfg, int n_rays, const double *origins,
                             const double *dirs, const double *tnear, const double *tfar,
                             double *out, int *n_blend, og_round_stats *stats_out, int count_unique)
{
    og_round_stats total;
    memset(&total, 0, sizeof(total));
#pragma omp parallel
    {
        og_round_stats st_loc;
        memset(&st_loc, 0, sizeof(st_loc));
        og_ray_state st;
        memset(&st, 0, sizeof(st));
        int k = cfg->k;
        st.kt = (double *)malloc((size_t)k * sizeof(double));
        st.kid = (int *)malloc((size_t)k * sizeof(int));
        if (count_unique) st.seen = (unsigned char *)malloc((size_t)(B->n_nodes > 0 ? B->n_nodes : 1));
#pragma omp for schedule(dynamic, 4)
        for (int r = 0; r < n_rays; ++r) {
            const double *ro = origins + 3 * r, *rd = dirs + 3 * r;
            double tn = tnear[r], tf = tfar[r];
            double dir[3], nd = sqrt(rd[0] * rd[0] + rd[1] * rd[1] + rd[2] * rd[2]);
            for (int a = 0; a < 3; ++a) dir[a] = rd[a] / nd;
            double C[3] = {0, 0, 0}, T = 1.0;
            int nb = 0, done = (B->root < 0);
            int checkpoint = cfg->checkpoint;
            double L_t = tn; int L_id = -1;          /* every key must exceed (t_near, -1) */
            st.nev = 0; st.src.n = 0; st.dst.n = 0;
            if (st.seen) memset(st.seen, 0, (size_t)B->n_nodes);
            if (!done && checkpoint) {
                double t0, t1;
                const og_node *rt = &B->nodes[B->root];
                if (og_slab(rt->lo, rt->hi, ro, rd, tn, tf, &t0, &t1)) og_push(&st.src, t0, B->root);
            }
            while (!done) {
                st_loc.rounds++;
                /* move the closest evicted hits into the k-buffer; the rest stay evicted */
                st.cnt = 0;
                if (checkpoint) {
                    int w = 0;
                    for (int e = 0; e < st.nev; ++e) {
                        double rt_; int rid;
                        if (og_kbuf_insert(st.kt, st.kid, &st.cnt, k, st.ev[e].t, st.ev[e].id, &rt_, &rid)) {
                            st.ev[w].t = rt_; st.ev[w].id = rid; ++w;
                        }
                    }
                    st.nev = w;
                }
                if (og_trace_round(S, B, p, cfg, &st, ro, rd, tn, tf, L_t, L_id, checkpoint, &st_loc)) {
                    st_loc.fallbacks++;
                    checkpoint = 0;
                    st.cnt = 0; st.nev = 0;
                    og_trace_round(S, B, p, cfg, &st, ro, rd, tn, tf, L_t, L_id, 0, &st_loc);
                }
                /* blend the k-buffer in order; stop right after T drops below T_min */
                for (int j = 0; j < st.cnt; ++j) {
                    double t, d2, al;
                    og_response(S, st.kid[j], ro, rd, &t, &d2, &al);
                    double a = al < p->alpha_max ? al : p->alpha_max;
                    double c[3], raw[3];
                    og_color(S, st.kid[j], dir, c, raw);
                    for (int ch = 0; ch < 3; ++ch) C[ch] += T * a * c[ch];
                    T *= (1.0 - a);
                    ++nb;
                    if (T < p->T_min) { done = 1; break; }
                }
                if (done || st.cnt < k) break;
                L_t = st.kt[k - 1]; L_id = st.kid[k - 1];
                if (checkpoint) { og_list tmp = st.src; st.src = st.dst; st.dst = tmp; }
            }
            for (int ch = 0; ch < 3; ++ch) out[4 * r + ch] = C[ch] + T * p->bg[ch];
            out[4 * r + 3] = T;
            if (n_blend) n_blend[r] = nb;
        }
        free(st.kt); free(st.kid); free(st.ev); free(st.src.e); free(st.dst.e); free(st.stack.e);
        free(st.seen);
#pragma omp critical
        {
            total.nodes += st_loc.nodes; total.leaves += st_loc.leaves; total.rounds += st_loc.rounds;
            total.ckpt_writes += st_loc.ckpt_writes; total.evictions += st_loc.evictions;
            total.fallbacks += st_loc.fallbacks; total.unique_nodes += st_loc.unique_nodes;
        }
    }
    if (stats_out) *stats_out = total;
}

/* ------------------------------------------------------------------------------------ */
/* Analytic gradient of the rendered image (derivative of Eq. volume-render and of       */
/* alpha = o G(r_o + t_alpha r_d) of Eq. t-max-resp). The hit set, their order and the   */
/* termination index are piecewise constant in the parameters and are not differentiated.*/
/* ------------------------------------------------------------------------------------ */

typedef struct og_grads {
    double *means, *log_scales, *quats, *logits, *sh;   /* shapes of the raw parameters */
} og_grads;

/* dR/dq for the quaternion (w,x,y,z): dR[m][e] = d R_e / d q_m, R_e row-major. */
static void og_dR_dq(const double qn[4], double dR[4][9])
{
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    double Dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    double Dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    double Dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    memcpy(dR[0], Dw, sizeof(Dw)); memcpy(dR[1], Dx, sizeof(Dx));
    memcpy(dR[2], Dy, sizeof(Dy)); memcpy(dR[3], Dz, sizeof(Dz));
}

static void og_atomic_add(double *p, double v)
{
#pragma omp atomic
    *p += v;
}

/* dL_drgbT: n_rays*4 upstream gradient w.r.t. (r, g, b, T) of each output pixel.
 * Gradients are accumulated (+=) into g, which the caller zeroes.
 * gabs (may be NULL): the same shapes, receiving for every gradient element the sum of the
 * magnitudes of the terms that element is summed from, each term taken with the magnitudes
 * of the quantities it is formed from (|dL/dC|, T, alpha, colours, the partial composites
 * C_<=j and C_final that the opacity derivative subtracts, |dL/dT|). It is the scale of a
 * first-order rounding-error bound for a lower-precision evaluation of the same sums: an
 * element whose terms cancel can only be known to about eps * gabs, not eps * |g|.
 * A term decided at a kink -- a colour channel whose SH sum + 0.5 lies within OG_KINK_MARGIN
 * of the clamp at 0, or an alpha within OG_KINK_MARGIN of alpha_max -- may be present in a
 * lower-precision evaluation and absent here (or the reverse); gabs is +inf for every
 * element such a term feeds, whether or not this evaluation includes it. */
#define OG_KINK_MARGIN 1e-5
OG_API void og_backward(const og_scene *S, const og_params *p, int n_rays, const double *origins,
                        const double *dirs, const double *tnear, const double *tfar,
                        const double *dL_drgbT, const og_grads *g, const og_grads *gabs)
{
    int K = S->n_coef;
#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < n_rays; ++r) {
        const double *ro = origins + 3 * r, *rd = dirs + 3 * r;
        og_hit *hits;
        int nh = og_ray_hits(S, p, ro, rd, tnear[r], tfar[r], &hits);
        double dir[3], nd = sqrt(rd[0] * rd[0] + rd[1] * rd[1] + rd[2] * rd[2]);
        for (int a = 0; a < 3; ++a) dir[a] = rd[a] / nd;
        /* forward pass, keeping what the backward needs */
        double *Tb = (double *)malloc((size_t)(nh + 1) * sizeof(double));
        double *col = (double *)malloc((size_t)(nh + 1) * 3 * sizeof(double));
        double *raw = (double *)malloc((size_t)(nh + 1) * 3 * sizeof(double));
        double C[3] = {0, 0, 0}, T = 1.0;
        int m = 0;
        for (int h = 0; h < nh; ++h) {
            double a = hits[h].alpha < p->alpha_max ? hits[h].alpha : p->alpha_max;
            og_color(S, hits[h].id, dir, col + 3 * h, raw + 3 * h);
            Tb[h] = T;
            for (int ch = 0; ch < 3; ++ch) C[ch] += T * a * col[3 * h + ch];
            T *= (1.0 - a);
            m = h + 1;
            if (T < p->T_min) break;
        }
        const double *gout = dL_drgbT + 4 * r;
        double dLdT = gout[3];
        for (int ch = 0; ch < 3; ++ch) dLdT += p->bg[ch] * gout[ch];   /* out = C + T bg */
        double Sacc[3] = {0, 0, 0};   /* colour contributed by the hits behind the current one */
        for (int h = m - 1; h >= 0; --h) {
            int i = hits[h].id;
            double al = hits[h].alpha;
            int clamped = !(al < p->alpha_max);
            double a = clamped ? p->alpha_max : al;
            /* colour: dC/dc = T_before a; c = max(0, raw) */
            double Y[16];
            og_sh_basis(S->sh_degree, dir, Y);
            for (int ch = 0; ch < 3; ++ch) {
                if (gabs && fabs(raw[3 * h + ch]) < OG_KINK_MARGIN)
                    for (int kk = 0; kk < K; ++kk) og_atomic_add(&gabs->sh[((size_t)i * K + kk) * 3 + ch], INFINITY);
                if (!(raw[3 * h + ch] > 0)) continue;
                double dc = gout[ch] * Tb[h] * a;
                for (int kk = 0; kk < K; ++kk) {
                    og_atomic_add(&g->sh[((size_t)i * K + kk) * 3 + ch], dc * Y[kk]);
                    if (gabs) og_atomic_add(&gabs->sh[((size_t)i * K + kk) * 3 + ch], fabs(dc * Y[kk]));
                }
            }
            /* opacity of this hit */
            double dLda = -dLdT * T / (1.0 - a);
            for (int ch = 0; ch < 3; ++ch)
                dLda += gout[ch] * (Tb[h] * col[3 * h + ch] - Sacc[ch] / (1.0 - a));
            /* magnitude of the same expression's pieces: the colour behind this hit is formed
             * as C_final - C_<=h, so its scale is |C_final| + |C_<=h| */
            double dLda_abs = fabs(dLdT) * T / (1.0 - a);
            for (int ch = 0; ch < 3; ++ch) {
                double upto = C[ch] - Sacc[ch];                  /* C_<=h */
                dLda_abs += fabs(gout[ch]) * (Tb[h] * fabs(col[3 * h + ch]) +
                                              (fabs(C[ch]) + fabs(upto)) / (1.0 - a));
            }
            for (int ch = 0; ch < 3; ++ch) Sacc[ch] += Tb[h] * a * col[3 * h + ch];
            if (gabs && fabs(al - p->alpha_max) < OG_KINK_MARGIN) {
                og_atomic_add(&gabs->logits[i], INFINITY);
                for (int a2 = 0; a2 < 3; ++a2) {
                    og_atomic_add(&gabs->means[3 * i + a2], INFINITY);
                    og_atomic_add(&gabs->log_scales[3 * i + a2], INFINITY);
                }
                for (int mm = 0; mm < 4; ++mm) og_atomic_add(&gabs->quats[4 * i + mm], INFINITY);
            }
            if (clamped) continue;
            /* alpha = o exp(-d2/2), d2 = min_t (x(t)-mu)^T Sigma^-1 (x(t)-mu); by the
             * envelope theorem d(d2) = partial derivative at fixed t = t_alpha. */
            double t, d2, al2;
            og_response(S, i, ro, rd, &t, &d2, &al2);
            double o = S->o[i];
            double G = exp(-0.5 * d2);
            og_atomic_add(&g->logits[i], dLda * G * o * (1.0 - o));
            double dLdd2 = dLda * (-0.5 * al2);
            const double *mu = S->mu + 3 * i, *P = S->P + 9 * i, *R = S->R + 9 * i, *s = S->s + 3 * i;
            double e[3];
            for (int a2 = 0; a2 < 3; ++a2) e[a2] = ro[a2] + t * rd[a2] - mu[a2];
            for (int a2 = 0; a2 < 3; ++a2) {
                double Pe = P[3 * a2] * e[0] + P[3 * a2 + 1] * e[1] + P[3 * a2 + 2] * e[2];
                og_atomic_add(&g->means[3 * i + a2], dLdd2 * (-2.0 * Pe));
            }
            double dRm[9];
            for (int j = 0; j < 3; ++j) {
                double pj = R[j] * e[0] + R[3 + j] * e[1] + R[6 + j] * e[2];   /* r_j . e */
                double inv2 = 1.0 / (s[j] * s[j]);
                og_atomic_add(&g->log_scales[3 * i + j], dLdd2 * (-2.0 * pj * pj * inv2));
                for (int a2 = 0; a2 < 3; ++a2) dRm[3 * a2 + j] = dLdd2 * 2.0 * pj * e[a2] * inv2;
            }
            double dR[4][9], dqn[4];
            og_dR_dq(S->q + 4 * i, dR);
            for (int mm = 0; mm < 4; ++mm) {
                double acc = 0;
                for (int ee = 0; ee < 9; ++ee) acc += dR[mm][ee] * dRm[ee];
                dqn[mm] = acc;
            }
            const double *qn = S->q + 4 * i;
            double dot = qn[0] * dqn[0] + qn[1] * dqn[1] + qn[2] * dqn[2] + qn[3] * dqn[3];
            for (int mm = 0; mm < 4; ++mm)
                og_atomic_add(&g->quats[4 * i + mm], (dqn[mm] - qn[mm] * dot) / S->qnorm[i]);
            if (gabs) {
                /* the same chain with every factor and partial sum taken by magnitude */
                double sc = dLda_abs * 0.5 * al2;                /* |dL/d d2| scale */
                og_atomic_add(&gabs->logits[i], dLda_abs * G * o * (1.0 - o));
                double ae[3];
                for (int a2 = 0; a2 < 3; ++a2) ae[a2] = fabs(e[a2]);
                for (int a2 = 0; a2 < 3; ++a2) {
                    double Pa = fabs(P[3 * a2]) * ae[0] + fabs(P[3 * a2 + 1]) * ae[1] + fabs(P[3 * a2 + 2]) * ae[2];
                    og_atomic_add(&gabs->means[3 * i + a2], 2.0 * sc * Pa);
                }
                double aRm[9];
                for (int j = 0; j < 3; ++j) {
                    double pa = fabs(R[j]) * ae[0] + fabs(R[3 + j]) * ae[1] + fabs(R[6 + j]) * ae[2];
                    double inv2 = 1.0 / (s[j] * s[j]);
                    og_atomic_add(&gabs->log_scales[3 * i + j], 2.0 * sc * pa * pa * inv2);
                    for (int a2 = 0; a2 < 3; ++a2) aRm[3 * a2 + j] = 2.0 * sc * pa * ae[a2] * inv2;
                }
                double aq[4], adot = 0;
                for (int mm = 0; mm < 4; ++mm) {
                    double acc = 0;
                    for (int ee = 0; ee < 9; ++ee) acc += fabs(dR[mm][ee]) * aRm[ee];
                    aq[mm] = acc;
                    adot += fabs(qn[mm]) * acc;
                }
                for (int mm = 0; mm < 4; ++mm)
                    og_atomic_add(&gabs->quats[4 * i + mm], (aq[mm] + fabs(qn[mm]) * adot) / S->qnorm[i]);
            }
        }
        free(Tb); free(col); free(raw); free(hits);
    }
}

/* ------------------------------------------------------------------------------------ */
/* LBVH building blocks: Morton order, binary radix tree, bottom-up bounds.              */
/* ------------------------------------------------------------------------------------ */

/* Bounds of the AABB centroids, FP32 (min/max are exact). bounds: lo xyz, hi xyz. */
OG_API void og_centroid_bounds(int n, const float *aabb, float *bounds)
{
    for (int a = 0; a < 3; ++a) { bounds[a] = INFINITY; bounds[3 + a] = -INFINITY; }
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            float c = 0.5f * (aabb[6 * i + a] + aabb[6 * i + 3 + a]);
            if (c < bounds[a]) bounds[a] = c;
            if (c > bounds[3 + a]) bounds[3 + a] = c;
        }
}

/* 63-bit Morton code of each AABB centroid: each coordinate is quantised to 21 bits over
 * the bounds, in FP32 (the precision of the kernel under test), then the bits are
 * interleaved x, y, z from the most significant triple down. */
OG_API void og_morton63(int n, const float *aabb, const float *bounds, uint64_t *codes)
{
    for (int i = 0; i < n; ++i) {
        uint32_t qv[3];
        for (int a = 0; a < 3; ++a) {
            float c = 0.5f * (aabb[6 * i + a] + aabb[6 * i + 3 + a]);
            float ext = bounds[3 + a] - bounds[a];
            float scale = ext > 0.0f ? 2097152.0f / ext : 0.0f;
            float u = (c - bounds[a]) * scale;
            qv[a] = u <= 0.0f ? 0u : (u >= 2097151.0f ? 2097151u : (uint32_t)u);
        }
        uint64_t code = 0;
        for (int b = 0; b < 21; ++b) {
            code |= (uint64_t)((qv[0] >> b) & 1u) << (3 * b + 2);
            code |= (uint64_t)((qv[1] >> b) & 1u) << (3 * b + 1);
            code |= (uint64_t)((qv[2] >> b) & 1u) << (3 * b);
        }
        codes[i] = code;
    }
}

/* Size-aware 64-bit Morton code (extended Morton codes for LBVH construction, Vinkler,
 * Bittner and Havran, HPG 2017): the AABB diagonal length is a fourth coordinate, on the
 * grid of the positions at half their resolution. Per box, in FP32:
 *   q_a = floor((c_a - lo_a) * (2^16 / (hi_a - lo_a))), clamped to [0, 2^16 - 1], for the
 *         centroid c (0 on an axis of zero extent);
 *   q_s = floor(diag * (2^15 / E)), clamped to [0, 2^16 - 2], diag = sqrt((ex^2 + ey^2) + ez^2)
 *         of the box extents and E the largest extent of the bounds (0 when E == 0).
 * Bit b of (x, y, z, s) goes to bit 4b + (3, 2, 1, 0). The clamp of q_s below 2^16 - 1 keeps
 * every code below 2^64 - 1, which marks empty boxes. */
OG_API void og_morton_sized64(int n, const float *aabb, const float *bounds, uint64_t *codes)
{
    float E = 0.0f;
    for (int a = 0; a < 3; ++a) {
        float ext = bounds[3 + a] - bounds[a];
        if (ext > E) E = ext;
    }
    float scale_s = E > 0.0f ? 32768.0f / E : 0.0f;
    for (int i = 0; i < n; ++i) {
        const float *bb = aabb + 6 * i;
        uint32_t q[4];
        for (int a = 0; a < 3; ++a) {
            float c = 0.5f * (bb[a] + bb[3 + a]);
            float ext = bounds[3 + a] - bounds[a];
            float scale = ext > 0.0f ? 65536.0f / ext : 0.0f;
            float u = (c - bounds[a]) * scale;
            q[a] = u <= 0.0f ? 0u : (u >= 65535.0f ? 65535u : (uint32_t)u);
        }
        float ex = bb[3] - bb[0], ey = bb[4] - bb[1], ez = bb[5] - bb[2];
        float d2 = ex * ex;
        d2 = d2 + ey * ey;
        d2 = d2 + ez * ez;
        float us = sqrtf(d2) * scale_s;
        q[3] = us <= 0.0f ? 0u : (us >= 65534.0f ? 65534u : (uint32_t)us);
        uint64_t code = 0;
        for (int b = 0; b < 16; ++b)
            for (int a = 0; a < 4; ++a)
                code |= (uint64_t)((q[a] >> b) & 1u) << (4 * b + 3 - a);
        codes[i] = code;
    }
}

/* Length of the common prefix of sorted keys i and j, with the index appended to break
 * ties between equal codes; -1 outside the array. */
static int og_prefix(const uint64_t *k, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    if (k[i] != k[j]) {
        uint64_t x = k[i] ^ k[j];
        int c = 0;
        while (!(x & (1ull << 63))) { x <<= 1; ++c; }
        return c;
    }
    uint32_t x = (uint32_t)i ^ (uint32_t)j;
    if (x == 0) return 96;
    int c = 0;
    while (!(x & 0x80000000u)) { x <<= 1; ++c; }
    return 64 + c;
}

#define OG_LEAF 0x80000000u

/* The binary radix tree over keys[first..last] (Karras-style numbering: the root is node
 * 0; a range [a,b] split at g has children [a,g] and [g+1,b], an internal child being
 * numbered by the end of its range next to the split, a one-key child being leaf g or g+1). */
static void og_radix_rec(const uint64_t *keys, int n, int first, int last, int id, uint32_t *left,
                         uint32_t *right)
{
    int common = og_prefix(keys, n, first, last);
    int g = first;
    while (g + 1 < last && og_prefix(keys, n, first, g + 1) > common) ++g;
    left[id] = (g == first) ? (OG_LEAF | (uint32_t)g) : (uint32_t)g;
    right[id] = (g + 1 == last) ? (OG_LEAF | (uint32_t)(g + 1)) : (uint32_t)(g + 1);
    if (g != first) og_radix_rec(keys, n, first, g, g, left, right);
    if (g + 1 != last) og_radix_rec(keys, n, g + 1, last, g + 1, left, right);
}

OG_API void og_radix_tree(int n, const uint64_t *sorted_keys, uint32_t *left, uint32_t *right)
{
    if (n >= 2) og_radix_rec(sorted_keys, n, 0, n - 1, 0, left, right);
}

static void og_refit_rec(uint32_t ref, const uint32_t *left, const uint32_t *right,
                         const float *leaf_aabb, float *node_aabb, float out[6])
{
    if (ref & OG_LEAF) {
        memcpy(out, leaf_aabb + 6 * (size_t)(ref & ~OG_LEAF), 6 * sizeof(float));
        return;
    }
    float a[6], b[6];
    og_refit_rec(left[ref], left, right, leaf_aabb, node_aabb, a);
    og_refit_rec(right[ref], left, right, leaf_aabb, node_aabb, b);
    for (int c = 0; c < 3; ++c) {
        out[c] = a[c] < b[c] ? a[c] : b[c];
        out[3 + c] = a[3 + c] > b[3 + c] ? a[3 + c] : b[3 + c];
    }
    memcpy(node_aabb + 6 * (size_t)ref, out, 6 * sizeof(float));
}

/* Bounds of every internal node = union of its children's bounds (FP32, exact). */
OG_API void og_refit(int n, const uint32_t *left, const uint32_t *right, const float *leaf_aabb,
                     float *node_aabb)
{
    float root[6];
    if (n >= 2) og_refit_rec(0u, left, right, leaf_aabb, node_aabb, root);
}

/* Locally-ordered clustering (PLOC: Meister and Bittner, "Parallel Locally-Ordered
 * Clustering for Bounding Volume Hierarchy Construction", IEEE TVCG 2018) over n >= 2 boxes in
 * Morton order. Clusters start as the leaves. Each iteration, every cluster i picks its
 * nearest neighbour among clusters i-r..i+r: the one whose union with it has the smallest
 * surface area 2 (ex ey + ey ez + ez ex) (FP32, in that order), ties to the lower index;
 * every mutual pair (i, j), i < j, merges into a new internal node (left = cluster i,
 * right = cluster j) that takes cluster i's place, nodes numbered in order of creation by
 * increasing i; the surviving clusters keep their order. Iterations repeat until one cluster
 * remains (the globally closest pair is always mutual, so every iteration merges). Output:
 * internal node created k-th is numbered n - 2 - k (the root is 0); left/right hold
 * internal numbers or (0x80000000 | leaf index). Returns the number of iterations. */
static float og_ploc_area(const float *a, const float *b)
{
    float e0 = fmaxf(a[3], b[3]) - fminf(a[0], b[0]);
    float e1 = fmaxf(a[4], b[4]) - fminf(a[1], b[1]);
    float e2 = fmaxf(a[5], b[5]) - fminf(a[2], b[2]);
    float s = e0 * e1;
    s = s + e1 * e2;
    s = s + e2 * e0;
    return 2.0f * s;
}

OG_API int og_ploc(int n, const float *aabb, int radius, uint32_t *left, uint32_t *right)
{
    float *cb = (float *)malloc(sizeof(float) * 6 * n), *cb2 = (float *)malloc(sizeof(float) * 6 * n);
    uint32_t *id = (uint32_t *)malloc(sizeof(uint32_t) * n), *id2 = (uint32_t *)malloc(sizeof(uint32_t) * n);
    uint32_t *lc = (uint32_t *)malloc(sizeof(uint32_t) * n), *rc = (uint32_t *)malloc(sizeof(uint32_t) * n);
    int *nn = (int *)malloc(sizeof(int) * n);
    memcpy(cb, aabb, sizeof(float) * 6 * n);
    for (int i = 0; i < n; ++i) id[i] = OG_LEAF | (uint32_t)i;
    int m = n, created = 0, iters = 0;
    while (m > 1) {
        ++iters;
        for (int i = 0; i < m; ++i) {
            float best = INFINITY;
            int bj = -1;
            int lo = i - radius < 0 ? 0 : i - radius, hi = i + radius > m - 1 ? m - 1 : i + radius;
            for (int j = lo; j <= hi; ++j) {
                if (j == i) continue;
                float a = og_ploc_area(cb + 6 * i, cb + 6 * j);
                if (a < best) { best = a; bj = j; }           /* ascending j: ties keep the lower */
            }
            nn[i] = bj;
        }
        int w = 0;
        for (int i = 0; i < m; ++i) {
            int j = nn[i];
            if (nn[j] == i && j < i) continue;                /* merged into cluster j */
            if (nn[j] == i) {
                lc[created] = id[i];
                rc[created] = id[j];
                for (int c = 0; c < 3; ++c) {
                    cb2[6 * w + c] = fminf(cb[6 * i + c], cb[6 * j + c]);
                    cb2[6 * w + 3 + c] = fmaxf(cb[6 * i + 3 + c], cb[6 * j + 3 + c]);
                }
                id2[w] = (uint32_t)created++;
            } else {
                memcpy(cb2 + 6 * w, cb + 6 * i, sizeof(float) * 6);
                id2[w] = id[i];
            }
            ++w;
        }
        float *tf = cb; cb = cb2; cb2 = tf;
        uint32_t *ti = id; id = id2; id2 = ti;
        m = w;
    }
    for (int k = 0; k < n - 1; ++k) {
        uint32_t L = lc[k], R = rc[k];
        left[n - 2 - k] = (L & OG_LEAF) ? L : (uint32_t)(n - 2) - L;
        right[n - 2 - k] = (R & OG_LEAF) ? R : (uint32_t)(n - 2) - R;
    }
    free(cb); free(cb2); free(id); free(id2); free(lc); free(rc); free(nn);
    return iters;
}

/* ------------------------------------------------------------------------------------ */
/* One bounce off a rectangular planar mirror (Sec. VI "GRTX-HW on Secondary Rays").     */
/* ------------------------------------------------------------------------------------ */

typedef struct og_mirror {
    double center[3], normal[3], axis_u[3], axis_v[3];
    double half_u, half_v, t_near_secondary;
} og_mirror;

/* Primary rays of cam with t_far clipped where they hit the mirror, and one reflected ray per
 * such primary (origin at the hit point, direction d - 2 (d.n) n, t in (t_near_secondary, inf)).
 * Secondaries are listed in pixel order; returns their number. */
OG_API int og_mirror_rays(const og_camera *cam, const og_mirror *m, double *po, double *pd, double *ptn,
                          double *ptf, double *so, double *sd, double *stn, double *stf, int *spix)
{
    og_camera_rays(cam, po, pd, ptn, ptf);
    int n = cam->width * cam->height, ns = 0;
    for (int p = 0; p < n; ++p) {
        const double *o = po + 3 * p, *d = pd + 3 * p;
        double den = 0, num = 0;
        for (int a = 0; a < 3; ++a) { den += d[a] * m->normal[a]; num += (m->center[a] - o[a]) * m->normal[a]; }
        if (den == 0.0) continue;
        double t = num / den;
        if (!(t > ptn[p] && t < ptf[p])) continue;
        double q[3], du = 0, dv = 0;
        for (int a = 0; a < 3; ++a) q[a] = o[a] + t * d[a];
        for (int a = 0; a < 3; ++a) {
            du += (q[a] - m->center[a]) * m->axis_u[a];
            dv += (q[a] - m->center[a]) * m->axis_v[a];
        }
        if (fabs(du) > m->half_u || fabs(dv) > m->half_v) continue;
        ptf[p] = t;
        for (int a = 0; a < 3; ++a) {
            so[3 * ns + a] = q[a];
            sd[3 * ns + a] = d[a] - 2.0 * den * m->normal[a];
        }
        stn[ns] = m->t_near_secondary;
        stf[ns] = INFINITY;
        spix[ns] = p;
        ++ns;
    }
    return ns;
}

/* A solid glass ball (Sec. VI "GRTX-HW on Secondary Rays": a spherical glass object placed in
 * the scene for refractions): centre, radius, index of refraction, t_near of its rays. */
typedef struct og_glass {
    double center[3], radius, ior, t_near_secondary;
} og_glass;

/* Snell refraction of unit direction I at a surface with unit normal N facing against I
 * (N.I < 0) from index n1 into n2, eta = n1 / n2: T = eta I + (eta cos_i - cos_t) N with
 * cos_i = -N.I and cos_t = sqrt(1 - eta^2 (1 - cos_i^2)) (clamped at 0). */
static void og_refract(const double I[3], const double Nf[3], double eta, double T[3])
{
    double ci = -(I[0] * Nf[0] + I[1] * Nf[1] + I[2] * Nf[2]);
    double k = 1.0 - eta * eta * (1.0 - ci * ci);
    double ct = k > 0.0 ? sqrt(k) : 0.0;
    for (int a = 0; a < 3; ++a) T[a] = eta * I[a] + (eta * ci - ct) * Nf[a];
}

/* Entry distance of the ray o + t d into the ball (t in units of |d|), or -1 when the ray
 * misses it, only grazes it, or starts inside it. */
static double og_glass_entry(const og_glass *gl, const double *o, const double *d)
{
    double oc[3], a = 0, b = 0, cc = 0;
    for (int q = 0; q < 3; ++q) {
        oc[q] = o[q] - gl->center[q];
        a += d[q] * d[q];
        b += oc[q] * d[q];
        cc += oc[q] * oc[q];
    }
    cc -= gl->radius * gl->radius;
    if (cc <= 0.0 || a == 0.0) return -1.0;
    double disc = b * b - a * cc;
    if (disc <= 0.0) return -1.0;
    return (-b - sqrt(disc)) / a;
}

/* The nearest of n_mirrors mirrors and n_glass glass balls along each primary ray of cam
 * (within its (t_near, t_far)) clips the primary there and spawns one secondary ray:
 *  - a mirror reflects it as in og_mirror_rays;
 *  - a glass ball refracts it into the ball at the entry point p1 (air index 1), carries it
 *    straight to the far side p2 = p1 + t2 v, t2 = -2 v.(p1 - c), refracts it out into the
 *    air, and the secondary starts at p2 with that direction. The ball's inside is empty
 *    space (nothing is rendered along the chord), there is no Fresnel reflection, and a
 *    camera inside a ball sees no ball.
 * Secondaries are listed in pixel order; returns their number. */
OG_API int og_secondary_rays(const og_camera *cam, const og_mirror *mirrors, int n_mirrors, const og_glass *glass,
                             int n_glass, double *po, double *pd, double *ptn, double *ptf, double *so, double *sd,
                             double *stn, double *stf, int *spix)
{
    og_camera_rays(cam, po, pd, ptn, ptf);
    int n = cam->width * cam->height, ns = 0;
    for (int p = 0; p < n; ++p) {
        const double *o = po + 3 * p, *d = pd + 3 * p;
        double t_best = ptf[p];
        int kind = 0, which = -1;
        for (int i = 0; i < n_mirrors; ++i) {
            const og_mirror *m = mirrors + i;
            double den = 0, num = 0;
            for (int a = 0; a < 3; ++a) { den += d[a] * m->normal[a]; num += (m->center[a] - o[a]) * m->normal[a]; }
            if (den == 0.0) continue;
            double t = num / den;
            if (!(t > ptn[p] && t < t_best)) continue;
            double du = 0, dv = 0;
            for (int a = 0; a < 3; ++a) {
                double qa = o[a] + t * d[a] - m->center[a];
                du += qa * m->axis_u[a];
                dv += qa * m->axis_v[a];
            }
            if (fabs(du) > m->half_u || fabs(dv) > m->half_v) continue;
            t_best = t; kind = 1; which = i;
        }
        for (int i = 0; i < n_glass; ++i) {
            double t = og_glass_entry(glass + i, o, d);
            if (!(t > ptn[p] && t < t_best)) continue;
            t_best = t; kind = 2; which = i;
        }
        if (kind == 0) continue;
        ptf[p] = t_best;
        double q[3];
        for (int a = 0; a < 3; ++a) q[a] = o[a] + t_best * d[a];
        if (kind == 1) {
            const og_mirror *m = mirrors + which;
            double den = 0;
            for (int a = 0; a < 3; ++a) den += d[a] * m->normal[a];
            for (int a = 0; a < 3; ++a) {
                so[3 * ns + a] = q[a];
                sd[3 * ns + a] = d[a] - 2.0 * den * m->normal[a];
            }
            stn[ns] = m->t_near_secondary;
        } else {
            const og_glass *gl = glass + which;
            double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double u[3], n1[3], v[3], p2[3], n2[3], w[3];
            for (int a = 0; a < 3; ++a) {
                u[a] = d[a] / len;
                n1[a] = (q[a] - gl->center[a]) / gl->radius;
            }
            og_refract(u, n1, 1.0 / gl->ior, v);
            double vl = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]), vp = 0;
            for (int a = 0; a < 3; ++a) { v[a] /= vl; vp += v[a] * (q[a] - gl->center[a]); }
            double t2 = -2.0 * vp;
            for (int a = 0; a < 3; ++a) {
                p2[a] = q[a] + t2 * v[a];
                n2[a] = -(p2[a] - gl->center[a]) / gl->radius;     /* inward: faces against v */
            }
            og_refract(v, n2, gl->ior, w);
            double wl = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            for (int a = 0; a < 3; ++a) {
                so[3 * ns + a] = p2[a];
                sd[3 * ns + a] = w[a] / wl;
            }
            stn[ns] = gl->t_near_secondary;
        }
        stf[ns] = INFINITY;
        spix[ns] = p;
        ++ns;
    }
    return ns;
}

/* Continue Eq. volume-render past the mirror: the primary pixel (C + T bg, T) becomes
 * (C + T C2, T T2) with (C2, T2) the secondary ray's pixel rendered against the same bg. */
OG_API void og_composite_bounce(double *rgbT, const double *sec_rgbT, const int *spix, int n_sec, const double bg[3])
{
    for (int j = 0; j < n_sec; ++j) {
        double *a = rgbT + 4 * spix[j];
        const double *b = sec_rgbT + 4 * j;
        double T = a[3];
        for (int c = 0; c < 3; ++c) a[c] = (a[c] - T * bg[c]) + T * b[c];
        a[3] = T * b[3];
    }
}
