/*
 * bt_oracle.c -- plain FP64 CPU oracle for BundleTrack's online pose-graph
 * optimisation (Sec. IV-D, Eq. 1-3).
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file's library.  It is written to be read
 * against the paper, not to be fast: every energy term is visited one by one,
 * every Jacobian is the full 12-column derivative with respect to both node
 * poses, and the normal equations are a dense 6N x 6N matrix.
 *
 * Readings of the paper that this file fixes (each one a parameter or a
 * convention, shared with the CUDA library through its documented interface,
 * not through code):
 *   - T_i maps object to camera i; the graph energy depends on the poses only
 *     through T_i and T_j of each edge (Eq. 1-3).
 *   - Eq. 1 sums over ordered pairs i != j.  Dense terms E_g(i,j) and E_g(j,i)
 *     differ (the source frame changes).  A correspondence set C_ij serves
 *     both E_f(i,j) and E_f(j,i), which are equal, so the sparse energy of an
 *     unordered pair enters with weight 2 * lambda_1.
 *   - rho is the Huber loss (Sec. IV-D): rho(r) = r^2/2 for |r| <= delta,
 *     delta (|r| - delta/2) beyond.  The IRLS weight is rho'(r)/r.  For the
 *     vector residual of Eq. 2 the weight comes from its norm and multiplies
 *     all three rows.
 *   - Projective association (Eq. 3): nearest pixel of the projection, target
 *     pixel must be masked with a depth and a normal, then the point-pair
 *     distance and normal-angle gates.  The association is frozen while the
 *     Jacobian is formed (no derivative of the depth lookup) and recomputed
 *     at the start of every iteration.
 *   - The accept/reject decision of the association produces integers (pixel
 *     indices, keep/drop).  It is taken in IEEE single precision (the
 *     precision of the GPU's residual pass; the paper fixes none) straight
 *     from the definition: each operation of the formula rounded on its
 *     own, in the order written, no fused multiply-add.  A GPU kernel may
 *     order and fuse its operations otherwise, so its decision may differ
 *     from this one for a pixel lying within single-precision rounding of
 *     a decision boundary (the half-pixel edge of the nearest pixel, the
 *     image edge, the distance gate, the angle gate).  orc_associate_classify
 *     evaluates every pixel in FP64 and lists the outcomes that such
 *     rounding admits.  Residuals, Jacobians, weights and everything after
 *     are FP64.
 *   - Gauss-Newton step: solve H dxi = -g exactly (Cholesky, no damping) over
 *     the nodes not flagged fixed (the gauge: frame I_0 is held constant),
 *     then T_i <- exp(dxi_i) T_i.
 */
#include "bt_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* FP64 rigid-transform helpers (4x4 row-major)                              */
/* ------------------------------------------------------------------------ */

static void pose_inv(const double T[16], double out[16])
{
    /* [R t; 0 1]^-1 = [R^T  -R^T t; 0 1] */
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) out[r * 4 + c] = T[c * 4 + r];
        out[r * 4 + 3] = -((T[0 * 4 + r] * T[3] + T[1 * 4 + r] * T[7]) + T[2 * 4 + r] * T[11]);
    }
    out[12] = out[13] = out[14] = 0.0;
    out[15] = 1.0;
}

static void pose_mul(const double A[16], const double B[16], double C[16])
{
    double tmp[16];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 4; ++c) {
            double s = (A[r * 4 + 0] * B[0 * 4 + c] + A[r * 4 + 1] * B[1 * 4 + c]) + A[r * 4 + 2] * B[2 * 4 + c];
            if (c == 3) s += A[r * 4 + 3];
            tmp[r * 4 + c] = s;
        }
    }
    tmp[12] = tmp[13] = tmp[14] = 0.0;
    tmp[15] = 1.0;
    memcpy(C, tmp, sizeof(tmp));
}

static void apply(const double T[16], const double p[3], double out[3])
{
    for (int r = 0; r < 3; ++r)
        out[r] = T[r * 4 + 0] * p[0] + T[r * 4 + 1] * p[1] + T[r * 4 + 2] * p[2] + T[r * 4 + 3];
}

static void rotate_t(const double T[16], const double v[3], double out[3])
{
    /* R^T v */
    for (int r = 0; r < 3; ++r)
        out[r] = T[0 * 4 + r] * v[0] + T[1 * 4 + r] * v[1] + T[2 * 4 + r] * v[2];
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------ */
/* Huber M-estimator (Sec. IV-D: "Huber loss is used")                      */
/* ------------------------------------------------------------------------ */

double orc_huber_rho(double r, double delta)
{
    double a = fabs(r);
    return a <= delta ? 0.5 * r * r : delta * (a - 0.5 * delta);
}

double orc_huber_weight(double r, double delta)
{
    double a = fabs(r);
    return a <= delta ? 1.0 : delta / a;
}

/* ------------------------------------------------------------------------ */
/* SE(3) exponential / logarithm, xi = (v, w): translation first (Sec. IV-D) */
/* R = I + A [w]x + B [w]x^2, t = (I + B [w]x + C [w]x^2) v with            */
/* A = sin(th)/th, B = (1-cos th)/th^2, C = (th - sin th)/th^3.              */
/* ------------------------------------------------------------------------ */

static void exp_coeffs(double th, double* A, double* B, double* C)
{
    double t2 = th * th;
    if (th < 1e-4) {
        *A = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
        *B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        *C = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
    } else {
        double s = sin(th), c = cos(th);
        *A = s / th;
        *B = (1.0 - c) / t2;
        *C = (th - s) / (t2 * th);
    }
}

void orc_se3_exp(const double xi[6], double T[16])
{
    const double* v = xi;
    const double* w = xi + 3;
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double A, B, C;
    exp_coeffs(th, &A, &B, &C);
    double W[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    double W2[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            W2[r * 3 + c] = W[r * 3 + 0] * W[0 * 3 + c] + W[r * 3 + 1] * W[1 * 3 + c] + W[r * 3 + 2] * W[2 * 3 + c];
    double V[9];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            double id = (r == c) ? 1.0 : 0.0;
            T[r * 4 + c] = id + A * W[r * 3 + c] + B * W2[r * 3 + c];
            V[r * 3 + c] = id + B * W[r * 3 + c] + C * W2[r * 3 + c];
        }
    }
    for (int r = 0; r < 3; ++r) T[r * 4 + 3] = V[r * 3 + 0] * v[0] + V[r * 3 + 1] * v[1] + V[r * 3 + 2] * v[2];
    T[12] = T[13] = T[14] = 0.0;
    T[15] = 1.0;
}

void orc_se3_log(const double T[16], double xi[6])
{
    double tr = T[0] + T[5] + T[10];
    double c = 0.5 * (tr - 1.0);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double th = acos(c);
    double k = (th < 1e-4) ? 0.5 + th * th / 12.0 : 0.5 * th / sin(th);
    double w[3] = {k * (T[9] - T[6]), k * (T[2] - T[8]), k * (T[4] - T[1])};
    double A, B, C;
    exp_coeffs(th, &A, &B, &C);
    /* V^-1 = I - [w]x/2 + (1/th^2)(1 - A/(2B)) [w]x^2 */
    double D = (th < 1e-4) ? 1.0 / 12.0 + th * th / 720.0 : (1.0 - A / (2.0 * B)) / (th * th);
    double W[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    double t[3] = {T[3], T[7], T[11]};
    for (int r = 0; r < 3; ++r) {
        double s = t[r];
        for (int q = 0; q < 3; ++q) {
            double w2 = W[r * 3 + 0] * W[0 * 3 + q] + W[r * 3 + 1] * W[1 * 3 + q] + W[r * 3 + 2] * W[2 * 3 + q];
            s += (-0.5 * W[r * 3 + q] + D * w2) * t[q];
        }
        xi[r] = s;
    }
    xi[3] = w[0];
    xi[4] = w[1];
    xi[5] = w[2];
}

/* ------------------------------------------------------------------------ */
/* Cholesky factorisation and solve (textbook, lower triangular)            */
/* ------------------------------------------------------------------------ */

int orc_cholesky_solve(int n, double* A, double* b)
{
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
        if (!(d > 0.0)) return -1;
        double l = sqrt(d);
        A[j * n + j] = l;
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = s / l;
        }
    }
    for (int i = 0; i < n; ++i) { /* L y = b */
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= A[i * n + k] * b[k];
        b[i] = s / A[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) { /* L^T x = y */
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= A[k * n + i] * b[k];
        b[i] = s / A[i * n + i];
    }
    return 0;
}

/* Conjugate gradients with the diagonal preconditioner M = diag(A) (the
 * inner solver of Sec. IV-D), textbook form: r = b - A x, z = M^-1 r,
 * p = z; alpha = r.z / p.Ap, x += alpha p, r -= alpha Ap, beta = r'.z' / r.z,
 * p = z' + beta p. */
int orc_pcg_solve(int n, const double* A, double* b, int max_iters, double rel_tol, int* iters)
{
    double* x = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int status = 0, it = 0;
    if (!x || !r || !z || !p || !q) status = -2;
    double bb = 0.0, rz = 0.0;
    for (int i = 0; i < n && status == 0; ++i) {
        if (!(A[i * n + i] > 0.0)) status = -1;
        r[i] = b[i];
        bb += b[i] * b[i];
    }
    for (int i = 0; i < n && status == 0; ++i) {
        z[i] = r[i] / A[i * n + i];
        p[i] = z[i];
        rz += r[i] * z[i];
    }
    double rr = bb;
    while (status == 0 && it < max_iters && rr > rel_tol * rel_tol * bb) {
        double pq = 0.0;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += A[i * n + j] * p[j];
            q[i] = s;
            pq += p[i] * s;
        }
        if (!(pq > 0.0)) { status = -1; break; }
        const double alpha = rz / pq;
        rr = 0.0;
        for (int i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            rr += r[i] * r[i];
        }
        double rz_new = 0.0;
        for (int i = 0; i < n; ++i) {
            z[i] = r[i] / A[i * n + i];
            rz_new += r[i] * z[i];
        }
        const double beta = rz_new / rz;
        rz = rz_new;
        for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        ++it;
    }
    if (status == 0) memcpy(b, x, sizeof(double) * (size_t)n);
    if (iters) *iters = it;
    free(x); free(r); free(z); free(p); free(q);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Projective data association (Eq. 3 and the gating sentence after it)     */
/* ------------------------------------------------------------------------ */

/* A pixel takes part (as source or as target) when it is masked, has a
 * positive finite depth and a finite normal. */
static int pixel_valid(const orc_frame* f, long pix)
{
    if (!f->mask[pix]) return 0;
    float z = f->depth[pix];
    if (!(z > 0.0f) || !isfinite(z)) return 0;
    const float* n = f->normals + 3 * pix;
    return isfinite(n[0]) && isfinite(n[1]) && isfinite(n[2]);
}

/* The decision for one source pixel (u, v) of frame i, taken in IEEE single
 * precision -- the precision of the GPU's residual pass; the paper fixes
 * none -- straight from the definition, every operation rounded on its own
 * in the order written (the library is compiled without contraction):
 *   p  = pi_D^-1(u, v)                      back-projection in camera i
 *   q  = B p, B = T_j T_i^-1                p seen from camera j
 *   u' = floor(pi(q) + 1/2)                 nearest pixel of the projection
 *   t  = pi_D^-1(u')                        the looked-up target point
 *   keep if q_z > 0, u' inside the image, u' valid, |t - q| <= d_max and
 *   n_i . R_B^T n_j >= cos(theta_max)       (unit normals: the angle gate)
 * |t - q| equals |T_i T_j^-1 t - p| of Eq. 3 (a rigid motion keeps
 * distances) and n_i . R_B^T n_j the cosine of the angle between n_i and the
 * target normal brought into camera i.  Bf: B rounded to single, row-major
 * 3x4.  Returns the target pixel, or -1. */
static long decide_f32(const orc_frame* fi, const orc_frame* fj, const float Bf[12], float dmax, float cmin,
                       int u, int v)
{
    const long pix = (long)v * fi->width + u;
    const float z = fi->depth[pix];
    const float p[3] = {((float)u - fi->cx) * z / fi->fx, ((float)v - fi->cy) * z / fi->fy, z};
    float q[3];
    for (int r = 0; r < 3; ++r) q[r] = Bf[4 * r] * p[0] + Bf[4 * r + 1] * p[1] + Bf[4 * r + 2] * p[2] + Bf[4 * r + 3];
    if (!(q[2] > 0.0f)) return -1;
    const float fu = floorf(fj->fx * q[0] / q[2] + fj->cx + 0.5f);
    const float fv = floorf(fj->fy * q[1] / q[2] + fj->cy + 0.5f);
    if (!(fu >= 0.0f && fu < (float)fj->width && fv >= 0.0f && fv < (float)fj->height)) return -1;
    const int iu = (int)fu, iv = (int)fv;
    const long tp = (long)iv * fj->width + iu;
    if (!pixel_valid(fj, tp)) return -1;
    const float zt = fj->depth[tp];
    const float t[3] = {((float)iu - fj->cx) * zt / fj->fx, ((float)iv - fj->cy) * zt / fj->fy, zt};
    const float d[3] = {t[0] - q[0], t[1] - q[1], t[2] - q[2]};
    if (!(sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) <= dmax)) return -1;
    const float* ni = fi->normals + 3 * pix;
    const float* nj = fj->normals + 3 * tp;
    float nb[3]; /* R_B^T n_j: the target normal in camera i */
    for (int r = 0; r < 3; ++r) nb[r] = Bf[r] * nj[0] + Bf[4 + r] * nj[1] + Bf[8 + r] * nj[2];
    if (!(ni[0] * nb[0] + ni[1] * nb[1] + ni[2] * nb[2] >= cmin)) return -1;
    return tp;
}

static void pair_transforms(const double Ti[16], const double Tj[16], double B[16], double A[16], float Bf[12])
{
    double Tiinv[16], Tjinv[16];
    pose_inv(Ti, Tiinv);
    pose_inv(Tj, Tjinv);
    pose_mul(Tj, Tiinv, B); /* camera i -> camera j */
    pose_mul(Ti, Tjinv, A); /* camera j -> camera i */
    for (int k = 0; k < 12; ++k) Bf[k] = (float)B[k];
}

int orc_associate(const orc_frame* fi, const orc_frame* fj, const double Ti[16],
                  const double Tj[16], const orc_params* prm,
                  int32_t* src_pix, int32_t* tgt_pix, int cap)
{
    double B[16], A[16];
    float Bf[12];
    pair_transforms(Ti, Tj, B, A, Bf);
    const float dmax = (float)prm->dense_max_dist;
    const float cmin = (float)cos(prm->dense_max_normal_deg * ORC_PI / 180.0);
    int n = 0;
    for (int v = 0; v < fi->height; ++v) {
        for (int u = 0; u < fi->width; ++u) {
            long pix = (long)v * fi->width + u;
            if (!pixel_valid(fi, pix)) continue;
            long tp = decide_f32(fi, fj, Bf, dmax, cmin, u, v);
            if (tp < 0) continue;
            if (n < cap) {
                src_pix[n] = (int32_t)pix;
                tgt_pix[n] = (int32_t)tp;
            }
            ++n;
        }
    }
    return n;
}

/* FP64 gate quantities of source point p (camera i, normal ni) against
 * target pixel tp of frame j: distance |A t - p| of the pair, cosine of the
 * angle between ni and R_A n_j, and the point-to-plane residual
 * r = ni . (A t - p) of Eq. 3.  Returns 0 when tp cannot be a target. */
static int target_terms(const orc_frame* fj, const double A[16], long tp, const double p[3], const double ni[3],
                        double* d, double* c, double* r)
{
    if (!pixel_valid(fj, tp)) return 0;
    const int iu = (int)(tp % fj->width), iv = (int)(tp / fj->width);
    const double zt = fj->depth[tp];
    const double t[3] = {((double)iu - fj->cx) * zt / fj->fx, ((double)iv - fj->cy) * zt / fj->fy, zt};
    double ti[3], nr[3];
    apply(A, t, ti);
    const double nj[3] = {fj->normals[3 * tp], fj->normals[3 * tp + 1], fj->normals[3 * tp + 2]};
    for (int k = 0; k < 3; ++k) nr[k] = A[k * 4 + 0] * nj[0] + A[k * 4 + 1] * nj[1] + A[k * 4 + 2] * nj[2];
    const double e[3] = {ti[0] - p[0], ti[1] - p[1], ti[2] - p[2]};
    *d = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    *c = ni[0] * nr[0] + ni[1] * nr[1] + ni[2] * nr[2];
    *r = ni[0] * e[0] + ni[1] * e[1] + ni[2] * e[2];
    return 1;
}

/* Admissible outcomes of every decision (see the header).  Error model of a
 * single-precision evaluation: unit roundoff u = 2^-24, every input and
 * intermediate carrying at most K = 16 roundings of its own magnitude
 * (the back-projection, the rounding of B, a three-term sum, a reciprocal
 * or divide, a product and a sum -- about six -- with a factor of more than
 * two to spare, for any order or fusion of the operations):
 *   q_r      : dq_r = 2 K u (|B_r0 p_0| + |B_r1 p_1| + |B_r2 p_2| + |B_r3|)
 *   u' edge  : e_u  = (f_x dq_0 + |u^ - c_x| dq_2) / q_2 + K u (|u^| + 1)
 *   distance : e_d  = dq_0 + dq_1 + dq_2 + K u (|t|_1 + d_max)
 *   cosine   : e_c  = 8 K u
 * where u^ = pi(q) + 1/2 in FP64.  Every nearest-pixel candidate within
 * e_u of u^ on each axis is examined; a candidate whose distance or cosine
 * lies within e_d / e_c of its gate may be kept or dropped. */
int orc_associate_classify(const orc_frame* fi, const orc_frame* fj, const double Ti[16],
                           const double Tj[16], const orc_params* prm, int32_t* src_pix,
                           int32_t* nominal, int32_t* alt, double* slack, int cap)
{
    double B[16], A[16];
    float Bf[12];
    pair_transforms(Ti, Tj, B, A, Bf);
    const float dmax_f = (float)prm->dense_max_dist;
    const double cmin = cos(prm->dense_max_normal_deg * ORC_PI / 180.0);
    const float cmin_f = (float)cmin;
    const double dmax = prm->dense_max_dist, hub = prm->huber_dense;
    const double K = 16.0, u32 = ldexp(1.0, -24);
    int n = 0;
    for (int v = 0; v < fi->height; ++v) {
        for (int u = 0; u < fi->width; ++u) {
            const long pix = (long)v * fi->width + u;
            if (!pixel_valid(fi, pix)) continue;
            const long nom = decide_f32(fi, fj, Bf, dmax_f, cmin_f, u, v);
            /* admissible outcomes: up to four candidate pixels and "dropped" */
            long adm[5];
            double arho[5];
            int na = 0;
            int reject_ok = 0;
            const double z = fi->depth[pix];
            const double p[3] = {((double)u - fi->cx) * z / fi->fx, ((double)v - fi->cy) * z / fi->fy, z};
            const double ni[3] = {fi->normals[3 * pix], fi->normals[3 * pix + 1], fi->normals[3 * pix + 2]};
            double q[3], dq[3];
            for (int r = 0; r < 3; ++r) {
                q[r] = B[4 * r] * p[0] + B[4 * r + 1] * p[1] + B[4 * r + 2] * p[2] + B[4 * r + 3];
                dq[r] = 2.0 * K * u32 * (fabs(B[4 * r] * p[0]) + fabs(B[4 * r + 1] * p[1]) +
                                         fabs(B[4 * r + 2] * p[2]) + fabs(B[4 * r + 3]));
            }
            if (!(q[2] > dq[2])) {
                /* behind (or within rounding of) camera j: only a projection
                 * far outside the image could come out, i.e. dropped */
                reject_ok = 1;
            }
            if (q[2] > 0.0) {
                const double uh = fj->fx * q[0] / q[2] + fj->cx + 0.5;
                const double vh = fj->fy * q[1] / q[2] + fj->cy + 0.5;
                const double eu = (fj->fx * dq[0] + fabs(uh - 0.5 - fj->cx) * dq[2]) / q[2] + K * u32 * (fabs(uh) + 1.0);
                const double ev = (fj->fy * dq[1] + fabs(vh - 0.5 - fj->cy) * dq[2]) / q[2] + K * u32 * (fabs(vh) + 1.0);
                const double cu[2] = {floor(uh - eu), floor(uh + eu)};
                const double cv[2] = {floor(vh - ev), floor(vh + ev)};
                for (int a = 0; a < 2; ++a) {
                    if (a == 1 && cu[1] == cu[0]) continue;
                    for (int b = 0; b < 2; ++b) {
                        if (b == 1 && cv[1] == cv[0]) continue;
                        if (!(cu[a] >= 0.0 && cu[a] < fj->width && cv[b] >= 0.0 && cv[b] < fj->height)) {
                            reject_ok = 1;
                            continue;
                        }
                        const long tp = (long)cv[b] * fj->width + (long)cu[a];
                        double d, c, r;
                        if (!target_terms(fj, A, tp, p, ni, &d, &c, &r)) {
                            reject_ok = 1;
                            continue;
                        }
                        const int iu = (int)(tp % fj->width), iv = (int)(tp / fj->width);
                        const double zt = fj->depth[tp];
                        const double tl1 = fabs(((double)iu - fj->cx) * zt / fj->fx) +
                                           fabs(((double)iv - fj->cy) * zt / fj->fy) + zt;
                        const double ed = dq[0] + dq[1] + dq[2] + K * u32 * (tl1 + dmax);
                        const double ec = 8.0 * K * u32;
                        const int fail = d > dmax + ed || c < cmin - ec;
                        const int pass = d <= dmax - ed && c >= cmin + ec;
                        if (!fail) {
                            adm[na] = tp;
                            arho[na] = orc_huber_rho(r, hub);
                            ++na;
                        }
                        if (!pass) reject_ok = 1;
                    }
                }
            }
            if (reject_ok) {
                adm[na] = -1;
                arho[na] = 0.0;
                ++na;
            }
            /* the single-precision decision must itself be admissible; if it
             * is not, report it as its own (inconsistent) outcome with an
             * infinite slack so that every test sees the failure */
            double rho_nom = NAN;
            for (int k = 0; k < na; ++k)
                if (adm[k] == nom) rho_nom = arho[k];
            if (n < cap) {
                src_pix[n] = (int32_t)pix;
                nominal[n] = (int32_t)nom;
                int m = 0;
                double s = 0.0;
                for (int k = 0; k < na; ++k) {
                    if (adm[k] == nom) continue;
                    if (m < 4) alt[4 * n + m++] = (int32_t)adm[k];
                    const double ds = fabs(arho[k] - rho_nom);
                    if (!(ds <= s)) s = ds; /* NaN (inconsistent nominal) propagates */
                }
                for (; m < 4; ++m) alt[4 * n + m] = -2;
                slack[n] = isnan(rho_nom) ? INFINITY : s;
            }
            ++n;
        }
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Residuals and Jacobians                                                  */
/* ------------------------------------------------------------------------ */

void orc_dense_terms(const orc_frame* fi, const orc_frame* fj, const double Ti[16],
                     const double Tj[16], const int32_t* src_pix, const int32_t* tgt_pix,
                     int n, double* r, double* J)
{
    /* A = T_i T_j^-1 maps camera j to camera i */
    double Tjinv[16], A[16];
    pose_inv(Tj, Tjinv);
    pose_mul(Ti, Tjinv, A);
    for (int k = 0; k < n; ++k) {
        long sp = src_pix[k], tp = tgt_pix[k];
        int u = (int)(sp % fi->width), v = (int)(sp / fi->width);
        int iu = (int)(tp % fj->width), iv = (int)(tp / fj->width);
        double z = fi->depth[sp], zt = fj->depth[tp];
        double p[3] = {((double)u - fi->cx) * z / fi->fx, ((double)v - fi->cy) * z / fi->fy, z};
        double q[3] = {((double)iu - fj->cx) * zt / fj->fx, ((double)iv - fj->cy) * zt / fj->fy, zt};
        double ni[3] = {fi->normals[3 * sp], fi->normals[3 * sp + 1], fi->normals[3 * sp + 2]};
        double qi[3];
        apply(A, q, qi); /* T_i T_j^-1 pi_D^-1(.) */
        r[k] = ni[0] * (qi[0] - p[0]) + ni[1] * (qi[1] - p[1]) + ni[2] * (qi[2] - p[2]);
        /* d r / d delta_i = n_i^T [I | -[A q]x] = (n_i, (A q) x n_i) */
        double* Jk = J + 12 * k;
        double c1[3];
        cross3(qi, ni, c1);
        Jk[0] = ni[0]; Jk[1] = ni[1]; Jk[2] = ni[2];
        Jk[3] = c1[0]; Jk[4] = c1[1]; Jk[5] = c1[2];
        /* d r / d delta_j = -n_i^T R_A [I | -[q]x] = (-m, m x q), m = R_A^T n_i */
        double mv[3], c2[3];
        rotate_t(A, ni, mv);
        cross3(mv, q, c2);
        Jk[6] = -mv[0]; Jk[7] = -mv[1]; Jk[8] = -mv[2];
        Jk[9] = c2[0]; Jk[10] = c2[1]; Jk[11] = c2[2];
    }
}

void orc_sparse_terms(const orc_match_set* m, const double Ti[16], const double Tj[16],
                      double* e, double* J)
{
    double Tiinv[16], Tjinv[16];
    pose_inv(Ti, Tiinv);
    pose_inv(Tj, Tjinv);
    for (int k = 0; k < m->count; ++k) {
        double pm[3] = {m->pts_i[3 * k], m->pts_i[3 * k + 1], m->pts_i[3 * k + 2]};
        double pn[3] = {m->pts_j[3 * k], m->pts_j[3 * k + 1], m->pts_j[3 * k + 2]};
        double a[3], b[3];
        apply(Tiinv, pm, a);
        apply(Tjinv, pn, b);
        for (int r = 0; r < 3; ++r) e[3 * k + r] = a[r] - b[r];
        /* (exp(d) T)^-1 p = T^-1 exp(-d) p ~ T^-1 p - R^T (v - [p]x w):
         *   d e / d delta_i = -R_i^T [I | -[p_m]x]
         *   d e / d delta_j = +R_j^T [I | -[p_n]x]                      */
        double Pm[9] = {0, -pm[2], pm[1], pm[2], 0, -pm[0], -pm[1], pm[0], 0};
        double Pn[9] = {0, -pn[2], pn[1], pn[2], 0, -pn[0], -pn[1], pn[0], 0};
        double* Jk = J + 36 * k;
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) {
                double RiT = Ti[c * 4 + r], RjT = Tj[c * 4 + r];
                double RiTP = 0.0, RjTP = 0.0; /* (R^T [p]x)[r][c] */
                for (int q = 0; q < 3; ++q) {
                    RiTP += Ti[q * 4 + r] * Pm[q * 3 + c];
                    RjTP += Tj[q * 4 + r] * Pn[q * 3 + c];
                }
                Jk[r * 12 + c] = -RiT;
                Jk[r * 12 + 3 + c] = RiTP;
                Jk[r * 12 + 6 + c] = RjT;
                Jk[r * 12 + 9 + c] = -RjTP;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Normal equations of Eq. 1 (IRLS Gauss-Newton, Sec. IV-D)                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    const orc_frame* frames;
    int n_frames;
    const double* poses;
    const orc_match_set* sets;
    int n_sets;
    const orc_params* prm;
    int n_threads, tid;
    int want_system;  /* 0: energy only */
    /* frozen association (NULL: associate): lists per ordered pair
     * k = i (N-1) + (j < i ? j : j - 1) */
    const int32_t* const* fz_src;
    const int32_t* const* fz_tgt;
    const int32_t* fz_n;
    double* H;        /* 6N x 6N (thread private) */
    double* g;        /* 6N */
    double e_dense, e_sparse;
    long n_dense, n_sparse;
    int failed;
} work_t;

static void add_terms(work_t* w, int ni, int nj, int rows, const double* J, const double* res, double wgt)
{
    /* H += wgt J^T J and g += wgt J^T res for a (rows x 12) Jacobian whose
     * columns 0-5 belong to node ni and 6-11 to node nj. */
    const int n6 = 6 * w->n_frames;
    int col[12];
    for (int c = 0; c < 6; ++c) {
        col[c] = 6 * ni + c;
        col[6 + c] = 6 * nj + c;
    }
    for (int a = 0; a < 12; ++a) {
        double ga = 0.0;
        for (int r = 0; r < rows; ++r) ga += J[r * 12 + a] * res[r];
        w->g[col[a]] += wgt * ga;
        for (int b = 0; b < 12; ++b) {
            double hab = 0.0;
            for (int r = 0; r < rows; ++r) hab += J[r * 12 + a] * J[r * 12 + b];
            w->H[(long)col[a] * n6 + col[b]] += wgt * hab;
        }
    }
}

static void* worker(void* arg)
{
    work_t* w = (work_t*)arg;
    const int N = w->n_frames;
    const orc_params* prm = w->prm;
    long n_dense_items = (long)N * (N - 1);
    long n_items = n_dense_items + w->n_sets;
    for (long it = w->tid; it < n_items; it += w->n_threads) {
        if (it < n_dense_items) {
            /* ordered pair (i -> j): E_g(i, j) of Eq. 3, weight lambda_2 */
            int i = (int)(it / (N - 1));
            int jj = (int)(it % (N - 1));
            int j = jj < i ? jj : jj + 1;
            const orc_frame* fi = &w->frames[i];
            const orc_frame* fj = &w->frames[j];
            const double* Ti = w->poses + 16 * i;
            const double* Tj = w->poses + 16 * j;
            int cap = fi->width * fi->height;
            int n;
            int32_t* sp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
            int32_t* tp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
            if (!sp || !tp) { free(sp); free(tp); w->failed = 1; continue; }
            if (w->fz_src) {
                n = w->fz_n[it];
                if (n < 0 || n > cap) { free(sp); free(tp); w->failed = 1; continue; }
                for (int k = 0; k < n; ++k) {
                    sp[k] = w->fz_src[it][k];
                    tp[k] = w->fz_tgt[it][k];
                    if (sp[k] < 0 || sp[k] >= cap || tp[k] < 0 || tp[k] >= fj->width * fj->height) w->failed = 1;
                }
                if (w->failed) { free(sp); free(tp); continue; }
            } else {
                n = orc_associate(fi, fj, Ti, Tj, prm, sp, tp, cap);
            }
            double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
            double* J = (double*)malloc(sizeof(double) * 12 * (size_t)(n > 0 ? n : 1));
            if (!r || !J) { free(sp); free(tp); free(r); free(J); w->failed = 1; continue; }
            orc_dense_terms(fi, fj, Ti, Tj, sp, tp, n, r, J);
            for (int k = 0; k < n; ++k) {
                w->e_dense += prm->lambda_dense * orc_huber_rho(r[k], prm->huber_dense);
                if (w->want_system)
                    add_terms(w, i, j, 1, J + 12 * k, r + k,
                              prm->lambda_dense * orc_huber_weight(r[k], prm->huber_dense));
            }
            w->n_dense += n;
            free(sp); free(tp); free(r); free(J);
        } else {
            /* unordered pair: E_f(i, j) + E_f(j, i) of Eq. 2, weight 2 lambda_1 */
            const orc_match_set* m = &w->sets[it - n_dense_items];
            if (m->count <= 0) continue;
            if (m->i < 0 || m->i >= N || m->j < 0 || m->j >= N || m->i == m->j) { w->failed = 1; continue; }
            double* e = (double*)malloc(sizeof(double) * 3 * (size_t)m->count);
            double* J = (double*)malloc(sizeof(double) * 36 * (size_t)m->count);
            if (!e || !J) { free(e); free(J); w->failed = 1; continue; }
            orc_sparse_terms(m, w->poses + 16 * m->i, w->poses + 16 * m->j, e, J);
            const double lam = 2.0 * prm->lambda_sparse;
            for (int k = 0; k < m->count; ++k) {
                const double* ek = e + 3 * k;
                double ne = sqrt(ek[0] * ek[0] + ek[1] * ek[1] + ek[2] * ek[2]);
                w->e_sparse += lam * orc_huber_rho(ne, prm->huber_sparse);
                if (w->want_system)
                    add_terms(w, m->i, m->j, 3, J + 36 * k, ek, lam * orc_huber_weight(ne, prm->huber_sparse));
            }
            w->n_sparse += m->count;
            free(e); free(J);
        }
    }
    return NULL;
}

static int run_workers(const orc_frame* frames, int n_frames, const double* poses,
                       const orc_match_set* sets, int n_sets, const orc_params* prm,
                       int n_threads, int want_system, double* H, double* g, double out[5],
                       const int32_t* const* fz_src, const int32_t* const* fz_tgt, const int32_t* fz_n)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    const long n6 = 6L * n_frames;
    work_t* ws = (work_t*)calloc((size_t)n_threads, sizeof(work_t));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!ws || !th) { free(ws); free(th); return -1; }
    int failed = 0;
    for (int t = 0; t < n_threads; ++t) {
        work_t* w = &ws[t];
        w->frames = frames; w->n_frames = n_frames; w->poses = poses;
        w->sets = sets; w->n_sets = n_sets; w->prm = prm;
        w->n_threads = n_threads; w->tid = t; w->want_system = want_system;
        w->fz_src = fz_src; w->fz_tgt = fz_tgt; w->fz_n = fz_n;
        if (want_system) {
            w->H = (double*)calloc((size_t)(n6 * n6), sizeof(double));
            w->g = (double*)calloc((size_t)n6, sizeof(double));
            if (!w->H || !w->g) failed = 1;
        }
    }
    if (!failed) {
        int started = 0;
        for (int t = 1; t < n_threads; ++t) {
            if (pthread_create(&th[t], NULL, worker, &ws[t]) != 0) { failed = 1; break; }
            started = t;
        }
        worker(&ws[0]);
        for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    }
    /* combine the per-thread sums in thread order (deterministic) */
    double ed = 0.0, es = 0.0;
    long nd = 0, ns = 0;
    if (want_system && !failed) {
        memset(H, 0, sizeof(double) * (size_t)(n6 * n6));
        memset(g, 0, sizeof(double) * (size_t)n6);
    }
    for (int t = 0; t < n_threads; ++t) {
        work_t* w = &ws[t];
        failed |= w->failed;
        ed += w->e_dense; es += w->e_sparse;
        nd += w->n_dense; ns += w->n_sparse;
        if (want_system && !failed) {
            for (long k = 0; k < n6 * n6; ++k) H[k] += w->H[k];
            for (long k = 0; k < n6; ++k) g[k] += w->g[k];
        }
        free(w->H); free(w->g);
    }
    free(ws); free(th);
    out[0] = ed + es; out[1] = ed; out[2] = es; out[3] = (double)nd; out[4] = (double)ns;
    return failed ? -1 : 0;
}

void orc_energy(const orc_frame* frames, int n_frames, const double* poses,
                const orc_match_set* sets, int n_sets, const orc_params* prm,
                int n_threads, double out[5])
{
    if (run_workers(frames, n_frames, poses, sets, n_sets, prm, n_threads, 0, NULL, NULL, out, NULL, NULL, NULL) != 0)
        out[0] = out[1] = out[2] = NAN;
}

long orc_normal_equations(const orc_frame* frames, int n_frames, const double* poses,
                          const orc_match_set* sets, int n_sets, const orc_params* prm,
                          int n_threads, double* H, double* g, double* energy)
{
    double out[5];
    if (run_workers(frames, n_frames, poses, sets, n_sets, prm, n_threads, 1, H, g, out, NULL, NULL, NULL) != 0) {
        *energy = NAN;
        return -1;
    }
    *energy = out[0];
    return (long)out[3];
}

long orc_normal_equations_frozen(const orc_frame* frames, int n_frames, const double* poses,
                                 const orc_match_set* sets, int n_sets, const orc_params* prm,
                                 const int32_t* const* src_pix, const int32_t* const* tgt_pix,
                                 const int32_t* counts, int n_threads, double* H, double* g, double* energy)
{
    double out[5];
    if (run_workers(frames, n_frames, poses, sets, n_sets, prm, n_threads, 1, H, g, out, src_pix, tgt_pix,
                    counts) != 0) {
        *energy = NAN;
        return -1;
    }
    *energy = out[0];
    return (long)out[3];
}

/* ------------------------------------------------------------------------ */
/* Gauss-Newton loop (Sec. IV-D)                                            */
/* ------------------------------------------------------------------------ */

int orc_solve(const orc_frame* frames, int n_frames, double* poses, const int32_t* fixed,
              const orc_match_set* sets, int n_sets, const orc_params* prm, int iters,
              int n_threads, double* cost_per_iter, double* cost_final)
{
    const int N = n_frames;
    const long n6 = 6L * N;
    int nfree = 0;
    int* freeidx = (int*)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    double* poses0 = (double*)malloc(sizeof(double) * 16 * (size_t)(N > 0 ? N : 1));
    double* H = (double*)malloc(sizeof(double) * (size_t)(n6 * n6 > 0 ? n6 * n6 : 1));
    double* g = (double*)malloc(sizeof(double) * (size_t)(n6 > 0 ? n6 : 1));
    if (!freeidx || !poses0 || !H || !g) { free(freeidx); free(poses0); free(H); free(g); return -2; }
    memcpy(poses0, poses, sizeof(double) * 16 * (size_t)N);
    for (int i = 0; i < N; ++i)
        if (!fixed[i]) freeidx[nfree++] = i;
    const int m = 6 * nfree;
    double* Hf = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m * m : 1));
    double* b = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int status = 0;
    for (int it = 0; it < iters && status == 0; ++it) {
        double E;
        if (orc_normal_equations(frames, N, poses, sets, n_sets, prm, n_threads, H, g, &E) < 0) {
            status = -2;
            break;
        }
        if (cost_per_iter) cost_per_iter[it] = E;
        if (m == 0) continue;
        /* gauge: drop the rows and columns of fixed nodes */
        for (int a = 0; a < nfree; ++a)
            for (int ra = 0; ra < 6; ++ra) {
                long row = 6L * freeidx[a] + ra;
                b[6 * a + ra] = -g[row];
                for (int c = 0; c < nfree; ++c)
                    for (int rc = 0; rc < 6; ++rc)
                        Hf[(6 * a + ra) * m + 6 * c + rc] = H[row * n6 + 6L * freeidx[c] + rc];
            }
        if ((prm->solver == 1 ? orc_pcg_solve(m, Hf, b, prm->pcg_max_iters, prm->pcg_tol, NULL)
                              : orc_cholesky_solve(m, Hf, b)) != 0) {
            status = -1;
            break;
        }
        /* T_i <- exp(dxi_i) T_i */
        for (int a = 0; a < nfree; ++a) {
            double E6[16];
            double* T = poses + 16 * freeidx[a];
            orc_se3_exp(b + 6 * a, E6);
            pose_mul(E6, T, T);
        }
    }
    if (status != 0) {
        memcpy(poses, poses0, sizeof(double) * 16 * (size_t)N);
    } else if (cost_final) {
        double out[5];
        orc_energy(frames, N, poses, sets, n_sets, prm, n_threads, out);
        *cost_final = out[0];
    }
    free(freeidx); free(poses0); free(H); free(g); free(Hf); free(b);
    return status;
}
