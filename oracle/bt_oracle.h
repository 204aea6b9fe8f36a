/*
 * bt_oracle.h -- plain FP64 CPU oracle for BundleTrack's pose-graph
 * optimisation (Wen & Bekris, IROS 2021, Sec. IV-D, Eq. 1-3).
 *
 * TEST INFRASTRUCTURE.  This library is the slow, obviously-correct
 * statement of what the CUDA path computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header or constant with the CUDA library.
 *
 * Conventions (the same ones the library's public interface documents):
 *   pose T_i: 4x4 row-major double, object -> camera i (Sec. III: the object
 *             pose in the camera frame);
 *   tangent perturbation delta = (v, w): three translation then three
 *             rotation parameters (Sec. IV-D), applied on the left,
 *             T <- exp(delta) T;
 *   pinhole:  u = fx X/Z + cx, v = fy Y/Z + cy, pixel centres at integers;
 *   depth:    metres, <= 0 or non-finite = no measurement;
 *   normals:  camera frame, per pixel, non-finite = no normal.
 */
#ifndef BT_ORACLE_H
#define BT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    const float* depth;     /* H*W */
    const float* normals;   /* H*W*3 */
    const uint8_t* mask;    /* H*W, nonzero = object */
    float fx, fy, cx, cy;
    int32_t width, height;
} orc_frame;

/* Feature correspondences C_ij (Eq. 2): pts_i[k] in camera i matches
 * pts_j[k] in camera j.  One set per unordered node pair. */
typedef struct {
    int32_t i, j;
    int32_t count;
    const float* pts_i;     /* count*3 */
    const float* pts_j;     /* count*3 */
} orc_match_set;

typedef struct {
    double huber_sparse;          /* Huber threshold of E_f (metres) */
    double huber_dense;           /* Huber threshold of E_g (metres) */
    double dense_max_dist;        /* association gate: point-pair distance */
    double dense_max_normal_deg;  /* association gate: normal angle */
    double lambda_sparse;         /* lambda_1 of Eq. 1 */
    double lambda_dense;          /* lambda_2 of Eq. 1 */
    int32_t solver;               /* 0: Cholesky, 1: PCG with Jacobi preconditioner */
    int32_t pcg_max_iters;        /* PCG: iteration limit */
    double pcg_tol;               /* PCG: stop when |r| <= pcg_tol |b| */
} orc_params;

/* Huber M-estimator rho and its IRLS weight rho'(r)/r. */
double orc_huber_rho(double r, double delta);
double orc_huber_weight(double r, double delta);

/* SE(3) exponential of xi = (v, w) (closed form), written to T (4x4). */
void orc_se3_exp(const double xi[6], double T[16]);
/* SE(3) logarithm (inverse of orc_se3_exp for rotation angles < pi). */
void orc_se3_log(const double T[16], double xi[6]);

/* Solve A x = b for symmetric positive-definite A (n x n, row-major, both
 * overwritten; x returned in b).  Returns 0, or -1 if A is not positive
 * definite. */
int orc_cholesky_solve(int n, double* A, double* b);

/* Solve A x = b for symmetric positive-definite A (n x n, row-major, not
 * modified) by the conjugate-gradient method with the diagonal (Jacobi)
 * preconditioner, from x = 0, until |b - A x| <= rel_tol |b| or max_iters
 * iterations; x returned in b, the iteration count in *iters (may be NULL).
 * Returns 0, or -1 if a diagonal entry or a curvature p^T A p is not
 * positive. */
int orc_pcg_solve(int n, const double* A, double* b, int max_iters, double rel_tol, int* iters);

/* Projective data association of Eq. 3 for the ordered pair (i -> j): every
 * valid masked pixel of frame i is projected into frame j, rounded to the
 * nearest pixel, and kept if that pixel is valid and passes the distance and
 * normal-angle gates.  Writes up to `cap` (source pixel, target pixel)
 * indices in increasing source-pixel order and returns the number kept.  The
 * accept/reject decision is taken in IEEE single precision, straight from
 * the definition (see the source for the formula and its order). */
int orc_associate(const orc_frame* fi, const orc_frame* fj, const double Ti[16],
                  const double Tj[16], const orc_params* prm,
                  int32_t* src_pix, int32_t* tgt_pix, int cap);

/* Classification of the association decisions of the ordered pair (i -> j)
 * against single-precision rounding.  For every valid masked pixel of frame
 * i (increasing pixel order; k-th entry), evaluated in FP64:
 *   src_pix[k]     the source pixel;
 *   nominal[k]     orc_associate's decision: target pixel, or -1 (dropped);
 *   alt[4k..4k+3]  the other outcomes that a single-precision evaluation
 *                  may reach -- a neighbouring nearest pixel when the
 *                  projection lies within rounding of a half-pixel edge, or
 *                  -1 when a gate or the image edge is within rounding --
 *                  padded with -2;
 *   slack[k]       max |rho(outcome) - rho(nominal)| (Huber cost of Eq. 3,
 *                  rho = 0 when dropped) over those outcomes; +inf when the
 *                  single-precision decision is itself not admissible.
 * The rounding bound is stated in the source.  Returns the number of valid
 * source pixels (entries beyond cap are counted, not written). */
int orc_associate_classify(const orc_frame* fi, const orc_frame* fj, const double Ti[16],
                           const double Tj[16], const orc_params* prm, int32_t* src_pix,
                           int32_t* nominal, int32_t* alt, double* slack, int cap);

/* Dense point-to-plane residual of Eq. 3 for a frozen association, with its
 * Jacobian with respect to left perturbations of T_i (columns 0-5) and T_j
 * (columns 6-11).  r: n, J: n*12. */
void orc_dense_terms(const orc_frame* fi, const orc_frame* fj, const double Ti[16],
                     const double Tj[16], const int32_t* src_pix, const int32_t* tgt_pix,
                     int n, double* r, double* J);

/* Sparse residual e = T_i^-1 p_m - T_j^-1 p_n of Eq. 2 for every pair of a
 * match set, with its 3x12 Jacobian (left perturbations of T_i, then T_j).
 * e: count*3, J: count*36 (row-major 3x12 per pair). */
void orc_sparse_terms(const orc_match_set* m, const double Ti[16], const double Tj[16],
                      double* e, double* J);

/* Total energy of Eq. 1 at the given poses (association recomputed).
 * out[0] = E, out[1] = dense part, out[2] = sparse part,
 * out[3] = accepted dense associations, out[4] = sparse pairs. */
void orc_energy(const orc_frame* frames, int n_frames, const double* poses,
                const orc_match_set* sets, int n_sets, const orc_params* prm,
                int n_threads, double out[5]);

/* Gauss-Newton normal equations over all 6N parameters (no gauge applied):
 * H (6N x 6N) = sum lambda w J^T J, g (6N) = sum lambda w J^T r, and the
 * energy at the same poses.  Returns the accepted dense association count. */
long orc_normal_equations(const orc_frame* frames, int n_frames, const double* poses,
                          const orc_match_set* sets, int n_sets, const orc_params* prm,
                          int n_threads, double* H, double* g, double* energy);

/* orc_normal_equations with a given association instead of Eq. 3's
 * (protocol: the same terms of an association computed elsewhere).
 * src_pix[k], tgt_pix[k], counts[k]: the accepted pairs of the ordered pair
 * k = i (N-1) + (j < i ? j : j - 1).  Returns the number of dense terms, or
 * -1 on a pixel index out of range. */
long orc_normal_equations_frozen(const orc_frame* frames, int n_frames, const double* poses,
                                 const orc_match_set* sets, int n_sets, const orc_params* prm,
                                 const int32_t* const* src_pix, const int32_t* const* tgt_pix,
                                 const int32_t* counts, int n_threads, double* H, double* g, double* energy);

/* Iteratively re-weighted Gauss-Newton (Sec. IV-D): `iters` iterations of
 * associate -> normal equations -> Cholesky (or, with prm->solver == 1, the
 * paper's preconditioned conjugate gradients) -> T_i <- exp(dxi_i) T_i for the
 * nodes with fixed[i] == 0, then the energy at the final poses.
 * cost_per_iter[k] = E before iteration k.  Returns 0, or -1 (poses
 * restored to their input values) if a system is not positive definite. */
int orc_solve(const orc_frame* frames, int n_frames, double* poses, const int32_t* fixed,
              const orc_match_set* sets, int n_sets, const orc_params* prm, int iters,
              int n_threads, double* cost_per_iter, double* cost_final);

#ifdef __cplusplus
}
#endif
#endif
