/*
 * bt.h -- C interface of the GB300 pose-graph library (libbt.so).
 *
 * The library implements the online pose-graph optimisation of BundleTrack
 * (Wen & Bekris, IROS 2021, Sec. IV-D): for the current frame and the
 * keyframes retrieved from the memory pool it minimises Eq. 1,
 *
 *     E = sum_{i != j} ( lambda_1 E_f(i,j) + lambda_2 E_g(i,j) ),
 *
 * where E_f (Eq. 2) is a Huber-robust point-to-point cost over sparse feature
 * correspondences and E_g (Eq. 3) a Huber-robust point-to-plane cost over the
 * dense projective association of every masked pixel, by iteratively
 * re-weighted Gauss-Newton on se(3) with the first frame held fixed.
 *
 * Conventions used by every call:
 *   - pose: 4x4 row-major double, maps OBJECT coordinates to CAMERA
 *     coordinates of that frame (the node poses of Sec. IV-D: the object's
 *     pose expressed in each camera); the last row must be 0 0 0 1;
 *   - pixel (u, v): u = column, v = row, pixel centres at integer coordinates;
 *     pinhole model u = fx X/Z + cx, v = fy Y/Z + cy;
 *   - depth: metres along the optical axis, row-major H x W float; values
 *     <= 0 or non-finite mean "no measurement";
 *   - normals: camera frame, row-major H x W x 3 float, non-finite = none;
 *   - mask: row-major H x W uint8, nonzero = object (Sec. IV-A).
 * A pixel takes part in the dense term (as source or as target) when it is
 * masked, has a positive finite depth and a finite normal.
 *
 * Memory and threading:
 *   - every call enqueues its GPU work on the stream given at creation
 *     (a cudaStream_t passed as void*, NULL = the legacy default stream);
 *   - input buffers stay owned by the caller and are copied (host) or read
 *     (device) before the call returns, so they may be freed afterwards;
 *   - output buffers are caller-allocated host memory;
 *   - calls that return data to the host synchronise that stream;
 *   - one graph may be used by one host thread at a time;
 *   - no call aborts or throws: every failure is a negative status
 *     (BT_ERR_*) and bt_last_error() gives a message for the calling thread.
 */
#ifndef BT_H
#define BT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define BT_OK 0
#define BT_ERR_INVALID (-1)   /* bad argument, size or state of an argument */
#define BT_ERR_CUDA (-2)      /* a CUDA call failed (message has the detail) */
#define BT_ERR_OOM (-3)       /* device or host allocation failed */
#define BT_ERR_SINGULAR (-4)  /* normal equations not positive definite */
#define BT_ERR_TIMEOUT (-5)   /* a bounded device-side wait ran out */
#define BT_ERR_STATE (-6)     /* call not valid in the graph's current state */

/* memory kinds of input pointers */
#define BT_HOST 0
#define BT_DEVICE 1

/* storage precision of the per-pixel point/normal maps (arithmetic is FP32
 * for the residual pass and FP64 for the solve in every case).  BT_BF16 and
 * BT_FP16 store normals and the in-plane point coordinates directly and depth
 * as an offset from the frame's mean valid depth, 8 bytes per target pixel
 * and 16 per source pixel instead of 16 and 32 (not in the paper). */
#define BT_FP32 0
#define BT_BF16 1
#define BT_FP16 2

#define BT_MAX_NODES 24          /* nodes in one solve (6*(N-1) <= 138 unknowns) */
#define BT_MAX_REPORT_ITERS 64

typedef struct bt_graph bt_graph;   /* opaque; created and freed by the library */

typedef struct {
    float fx, fy, cx, cy;   /* pinhole intrinsics, pixels */
    int32_t width, height;  /* image size, pixels (>= 1) */
} bt_intrinsics;

/* Method constants.  bt_config_default() fills the values this library uses
 * when the paper leaves a constant unstated:
 *   huber_sparse = huber_dense = 0.005 m   (Huber thresholds of Eq. 2 / Eq. 3)
 *   dense_max_dist = 0.02 m                (association gate on point-pair distance)
 *   dense_max_normal_deg = 45              (association gate on normal angle)
 *   lambda_sparse = lambda_dense = 1       (lambda_1, lambda_2 of Eq. 1)
 *   precision = BT_FP32, max_frames = 0 (no limit on stored frames),
 *   solver = BT_SOLVER_CHOLESKY, pcg_max_iters = 500, pcg_tol = 1e-10.
 * precision selects the storage of the per-pixel maps (BT_FP32 / BT_BF16 /
 * BT_FP16); it is fixed for the graph's lifetime.  solver selects how each
 * Gauss-Newton system H dx = -g is solved: BT_SOLVER_CHOLESKY, an exact FP64
 * LDL^T factorisation, or BT_SOLVER_PCG, the paper's conjugate gradients
 * with the diagonal (Jacobi) preconditioner (Sec. IV-D), in FP64 from
 * dx = 0 until |H dx + g| <= pcg_tol |g| or pcg_max_iters iterations. */
#define BT_SOLVER_CHOLESKY 0
#define BT_SOLVER_PCG 1
typedef struct {
    double huber_sparse;
    double huber_dense;
    double dense_max_dist;
    double dense_max_normal_deg;
    double lambda_sparse;
    double lambda_dense;
    int32_t precision;
    int32_t max_frames;
    int32_t solver;
    int32_t pcg_max_iters;
    double pcg_tol;
} bt_config;

/* Correspondences between a frame being added and an already stored frame
 * (the set C_ij of Eq. 2; the paper caches it per pair, Sec. IV-D). */
typedef struct {
    int32_t other_frame;     /* id returned by an earlier bt_add_frame */
    int32_t count;           /* number of pairs, >= 0 */
    const float* pts_self;   /* count x 3, camera frame of the new frame */
    const float* pts_other;  /* count x 3, camera frame of other_frame */
} bt_matches;

typedef struct {
    int32_t iters_run;        /* Gauss-Newton iterations executed */
    int32_t status;           /* BT_OK or the error the solve ended with */
    int32_t used_warmstart;   /* reserved, 0 */
    int32_t fell_back;        /* reserved, 0 */
    double cost_init;         /* E (Eq. 1) at the starting poses */
    double cost_final;        /* E at the returned poses (association recomputed) */
    double dense_cost_final;  /* lambda_2 part of cost_final */
    double sparse_cost_final; /* lambda_1 part of cost_final */
    double cost_per_iter[BT_MAX_REPORT_ITERS]; /* E before iteration k */
    int64_t dense_inliers;    /* accepted dense associations at the final poses */
    int64_t dense_pixel_pairs;/* sum over ordered pairs of source pixels, x iters */
} bt_solve_report;

/* Fills *cfg with the defaults above.  Never fails. */
void bt_config_default(bt_config* cfg);

/* Creates an empty graph (Sec. IV-D, G = {V, E}).  cfg may be NULL (defaults).
 * cuda_stream: cudaStream_t as void* (NULL = legacy default stream); the
 * caller keeps ownership and must keep it alive until bt_graph_destroy.
 * Returns BT_OK and *out, or BT_ERR_INVALID (bad cfg / out NULL),
 * BT_ERR_CUDA, BT_ERR_OOM. */
int bt_graph_create(const bt_config* cfg, void* cuda_stream, bt_graph** out);

/* Frees the graph and all device memory it owns (synchronises its stream).
 * NULL is ignored. */
void bt_graph_destroy(bt_graph* g);

/* Adds one RGB-D observation I_tau (Sec. III) with its mask M_tau and normal
 * map, builds its device point/normal maps and its list of dense source
 * pixels, and stores its initial pose.  The new frame joins the active node
 * set at the end.  fixed != 0 holds the pose constant (the gauge: frame I_0,
 * Sec. IV-D).  matches (n_matches entries, may be NULL when 0) add the
 * correspondence sets between this frame and earlier frames.
 *   depth:   H x W float;  normals: H x W x 3 float;  mask: H x W uint8;
 *   mem_kind: BT_HOST (pageable or pinned host memory) or BT_DEVICE (device
 *   pointers on this GPU) -- it applies to depth, normals, mask and the
 *   match point arrays; intrinsics and pose_init are always host memory.
 * On success *frame_id_out (may be NULL) receives the new frame's id.
 * Errors: BT_ERR_INVALID (NULL required pointer, size <= 0, unknown
 * other_frame, negative count, more than max_frames frames),
 * BT_ERR_CUDA, BT_ERR_OOM.  On error the graph is unchanged. */
int bt_add_frame(bt_graph* g, const float* depth, const float* normals, const uint8_t* mask,
                 const bt_intrinsics* intrinsics, const double pose_init[16], int32_t fixed,
                 const bt_matches* matches, int32_t n_matches, int32_t mem_kind,
                 int32_t* frame_id_out);

/* Sets (replaces) the correspondence set between two stored frames:
 * pts_a[k] (camera frame of frame_a) matches pts_b[k] (camera frame of
 * frame_b); count x 3 floats each, in memory of kind mem_kind.  count == 0
 * removes the set.  Errors: BT_ERR_INVALID, BT_ERR_CUDA, BT_ERR_OOM. */
int bt_set_matches(bt_graph* g, int32_t frame_a, int32_t frame_b, int32_t count,
                   const float* pts_a, const float* pts_b, int32_t mem_kind);

/* Removes a stored frame (and every correspondence set that involves it)
 * and frees its device memory; it also leaves the active set.
 * Errors: BT_ERR_INVALID (unknown id). */
int bt_remove_frame(bt_graph* g, int32_t frame_id);

/* Chooses which stored frames form the pose graph of the next solve, in node
 * order (the keyframes selected for the current frame, Sec. IV-C), n >= 1,
 * no repeats, n <= BT_MAX_NODES.  Until called, the active set is every frame
 * in the order added.  Errors: BT_ERR_INVALID. */
int bt_set_active(bt_graph* g, const int32_t* frame_ids, int32_t n);

/* Number of active nodes, or a negative status. */
int bt_num_active(const bt_graph* g);

/* Replaces / reads the poses of the active nodes (n_active x 16 doubles,
 * host, node order).  Errors: BT_ERR_INVALID. */
int bt_set_poses(bt_graph* g, const double* poses);
int bt_get_poses(const bt_graph* g, double* poses);

/* Runs `iters` (0..BT_MAX_REPORT_ITERS) Gauss-Newton iterations of Sec.
 * IV-D over the active nodes -- per iteration: dense association and
 * point-to-plane residuals for every ordered pair, Huber point-to-point
 * residuals for every correspondence set, reduction into 6x6 blocks,
 * assembly of the normal equations over the non-fixed nodes, FP64 Cholesky
 * solve, FP64 se(3) update -- then evaluates E at the final poses.  The new
 * poses are stored in the graph (the memory write-back of Sec. IV-D) and, if
 * poses_out != NULL, copied to it (n_active x 16 doubles, host).  rep may be
 * NULL.  Synchronises the stream.
 * Errors: BT_ERR_INVALID (iters out of range, no active nodes, more than
 * BT_MAX_NODES), BT_ERR_SINGULAR (a system was not positive definite: poses
 * are left as they were before the call), BT_ERR_CUDA, BT_ERR_OOM. */
int bt_solve(bt_graph* g, int32_t iters, double* poses_out, bt_solve_report* rep);

/* Evaluates Eq. 1 at the stored poses of the active nodes (association
 * recomputed), without changing them.  cost_out[0] = E, [1] = dense part,
 * [2] = sparse part (host, 3 doubles); dense_inliers may be NULL.
 * Synchronises the stream.  Errors: BT_ERR_INVALID, BT_ERR_CUDA. */
int bt_eval_cost(bt_graph* g, double* cost_out, int64_t* dense_inliers);

/* ---------------------------------------------------------------- batches
 * Many independent pose graphs solved together (not in the paper: the
 * throughput form of the same optimisation).  Each Gauss-Newton iteration of
 * the whole batch is three launches -- the residual pass over every graph's
 * tiles and correspondence sets, the FP64 pair reduction over every graph's
 * node pairs, and one solve CTA per graph -- and the iterations are captured
 * once as a CUDA graph and replayed.  The residual pass's CTA shape (threads
 * x source pixels per thread, i.e. the tile size of the first reduction
 * stage) is chosen by timing each candidate on the batch itself
 * (autotuning) unless fixed with bt_batch_set_shape. */
typedef struct bt_batch bt_batch;

/* Creates an empty batch working on cuda_stream (NULL: the batch creates and
 * owns a non-blocking stream; the legacy default stream cannot be captured).
 * Errors: BT_ERR_INVALID, BT_ERR_CUDA, BT_ERR_OOM. */
int bt_batch_create(void* cuda_stream, bt_batch** out);
void bt_batch_destroy(bt_batch* b);

/* Adds a graph (not owned: it must outlive the batch and must not be solved
 * through bt_solve while a batch solve is running).  Its active node set and
 * stored poses at the time of each bt_batch_solve are what is solved.
 * Every graph of a batch must use the same storage precision.
 * Errors: BT_ERR_INVALID (NULL, already added, no or too many active nodes,
 * different precision). */
int bt_batch_add(bt_batch* b, bt_graph* g);

/* Number of graphs, or a negative status. */
int bt_batch_size(const bt_batch* b);

/* Residual-pass CTA shapes the autotuner chooses from (threads x source
 * pixels per thread: 128x4, 128x2, 256x4, 64x4, 64x8, 32x16). */
#define BT_NUM_SHAPES 6
/* The shape of the single-graph solve (bt_solve, bt_eval_cost): 256 x 4,
 * 1024-pixel tiles.  A batch fixed to this shape reproduces bt_solve bit for
 * bit. */
#define BT_SINGLE_GRAPH_SHAPE 2

/* Fixes the residual CTA shape (0 .. BT_NUM_SHAPES-1) or re-enables
 * autotuning (-1, the default).  Errors: BT_ERR_INVALID. */
int bt_batch_set_shape(bt_batch* b, int32_t shape);

/* The shape in use and the autotuner's measured time per shape
 * (BT_NUM_SHAPES doubles, microseconds of one full residual pass; 0 where
 * not measured).  Either
 * pointer may be NULL.  Errors: BT_ERR_INVALID. */
int bt_batch_tuning(const bt_batch* b, int32_t* shape_out, double* us_per_shape);

/* Solves every graph of the batch from its stored poses with `iters`
 * Gauss-Newton iterations (the same algorithm as bt_solve) and writes the
 * results back into the graphs.  reps: NULL or bt_batch_size() reports in the
 * order graphs were added.  Synchronises the batch stream.
 * Errors: BT_ERR_INVALID, BT_ERR_SINGULAR (the affected graphs keep their
 * poses, the others are updated), BT_ERR_CUDA, BT_ERR_OOM. */
int bt_batch_solve(bt_batch* b, int32_t iters, bt_solve_report* reps);

/* ---------------------------------------------------------- warm start
 * Learned initialisation of all nodes of a pose graph (not in the paper: it
 * takes the place of the coarse pose from sparse matches, RANSAC and a
 * closed-form fit, of Sec. IV-B).  For every correspondence set (edge i -> j,
 * points p in camera i, q in camera j, initial relative pose
 * M0 = T_j T_i^-1) a set network predicts an increment D of the edge's
 * relative pose, M = D M0:
 *   features  x = ((M0 p - c) / 0.1 m, (q - M0 p) / 0.01 m), c = mean of q
 *   network   x -> 128 -> 256 (ReLU, shared over the set) -> max over the
 *             set -> 128 (ReLU) -> 6 = (omega / 0.1 rad, u / 0.01 m)
 *   increment D(x) = exp(omega) (x - c) + c + u
 * with BF16 weight copies of an FP32 master vector and FP32 sums.  The node
 * poses then follow from one FP64 linear least-squares relative-pose
 * averaging solve: each free node is first anchored on its edge to the
 * lowest-indexed fixed node, then left increments d_i minimise
 *   sum over edges |d_j - Ad(M_ij) d_i - log(D_ij M0_ij M_ij^-1)|^2_W,
 *   W = diag(1/0.01^2 x3, 1/0.1^2 x3) on (v, omega),
 * by Cholesky, and T_i <- exp(d_i) T_i.  Training (mean of 1/2 |y - y*|^2
 * over a minibatch, Adam with beta = (0.9, 0.999), eps = 1e-8) runs on a
 * device-resident set of samples whose labels y* come from the poses a solve
 * converged to.  Parameters: BT_WS_NUM_PARAMS floats in the order
 * W1[128][6], b1[128], W2[256][128], b2[256], W3[128][256], b3[128],
 * W4[6][128], b4[6] (row = output unit). */
#define BT_WS_NUM_PARAMS 67590
typedef struct bt_warmstart bt_warmstart;

/* Creates a warm start working on cuda_stream (NULL: it creates and owns a
 * non-blocking stream).  Parameters must be set before use.
 * Errors: BT_ERR_INVALID, BT_ERR_CUDA, BT_ERR_OOM. */
int bt_warmstart_create(void* cuda_stream, bt_warmstart** out);
void bt_warmstart_destroy(bt_warmstart* ws);
/* BT_WS_NUM_PARAMS (for bindings that check their layout). */
int32_t bt_warmstart_num_params(void);

/* Sets the FP32 master parameters (host or device array of
 * BT_WS_NUM_PARAMS) and refreshes the BF16 copies; clears the Adam moments
 * and step count.  Errors: BT_ERR_INVALID (NULL, non-finite), BT_ERR_CUDA. */
int bt_warmstart_set_params(bt_warmstart* ws, const float* params, int32_t mem_kind);
/* Copies the FP32 master parameters out.  Errors: BT_ERR_INVALID, BT_ERR_STATE
 * (no parameters set), BT_ERR_CUDA. */
int bt_warmstart_get_params(const bt_warmstart* ws, float* params, int32_t mem_kind);

/* Training state for a checkpoint: the Adam first and second moments
 * (BT_WS_NUM_PARAMS floats each, host or device) and the number of steps
 * taken.  A training run resumed from get_params + get_adam (set_params,
 * then set_adam) continues exactly as the uninterrupted run would.
 * set_params clears this state.  Errors: BT_ERR_INVALID (NULL, negative
 * step, non-finite or negative second moment), BT_ERR_STATE (no
 * parameters set), BT_ERR_CUDA. */
int bt_warmstart_get_adam(const bt_warmstart* ws, float* m, float* v, int32_t* step, int32_t mem_kind);
int bt_warmstart_set_adam(bt_warmstart* ws, const float* m, const float* v, int32_t step, int32_t mem_kind);

/* Appends one training sample: count > 0 point pairs (pts_i in camera i,
 * pts_j in camera j: count x 3 float, host or device), the initial poses of
 * the two frames (4x4 row-major; M0 = T_j T_i^-1) and, optionally, the poses
 * a solve converged to (both NULL: label 0).  The data is copied.
 * Errors: BT_ERR_INVALID, BT_ERR_CUDA, BT_ERR_OOM. */
int bt_warmstart_add_set(bt_warmstart* ws, const float* pts_i, const float* pts_j, int32_t count,
                         const double* pose_i, const double* pose_j, const double* label_i, const double* label_j,
                         int32_t mem_kind);
/* Appends one sample per non-empty correspondence set between active nodes
 * of g (in the order of its edges: pairs of frame ids in increasing order),
 * with initial and label poses given per active node (N x 4x4 host arrays,
 * active order; poses_label may be NULL).  Point data is copied on the
 * device.  Errors: BT_ERR_INVALID, BT_ERR_CUDA, BT_ERR_OOM. */
int bt_warmstart_add_graph(bt_warmstart* ws, bt_graph* g, const double* poses_init, const double* poses_label);
/* Number of stored samples, or a negative status. */
int32_t bt_warmstart_num_samples(const bt_warmstart* ws);
/* Drops every stored sample (device memory is kept for reuse). */
int bt_warmstart_clear_samples(bt_warmstart* ws);
/* The centre c (3 floats) and label y* (6 floats) of sample id; either
 * pointer may be NULL.  Errors: BT_ERR_INVALID, BT_ERR_CUDA. */
int bt_warmstart_get_sample(const bt_warmstart* ws, int32_t id, float* centre, float* label);

/* The calls below that run the network report BT_ERR_TIMEOUT when one of
 * the forward pass's bounded waits on the tensor cores ran out (1 s, see
 * bt_debug_tensor_wait_ns); the outputs of that pass are discarded and the
 * CUDA context stays usable.  bt_warmstart_train_step without loss_out does
 * not synchronise: such a timeout is reported by the next call that does.
 *
 * Network outputs (n x 6 floats, host) for samples ids[0..n) (host array).
 * Errors: BT_ERR_INVALID (id out of range), BT_ERR_STATE, BT_ERR_TIMEOUT,
 * BT_ERR_CUDA. */
int bt_warmstart_predict(bt_warmstart* ws, const int32_t* ids, int32_t n, float* y_out);
/* Gradient (BT_WS_NUM_PARAMS floats, host; may be NULL) and value (may be
 * NULL) of the mean loss over samples ids[0..n), without an update. */
int bt_warmstart_gradient(bt_warmstart* ws, const int32_t* ids, int32_t n, float* grad_out, double* loss_out);
/* One Adam step with learning rate lr on the mean loss over samples
 * ids[0..n).  loss_out: NULL (no synchronisation) or the loss before the step. */
int bt_warmstart_train_step(bt_warmstart* ws, const int32_t* ids, int32_t n, float lr, double* loss_out);

/* Replaces the stored poses of g's free active nodes by the warm start
 * computed from its correspondence sets at its stored poses (fixed nodes are
 * kept).  Errors: BT_ERR_INVALID, BT_ERR_STATE, BT_ERR_SINGULAR (a free node
 * without correspondences; poses unchanged), BT_ERR_TIMEOUT (poses
 * unchanged), BT_ERR_CUDA, BT_ERR_OOM. */
int bt_warmstart_apply(bt_warmstart* ws, bt_graph* g);
/* The same for every graph of a batch, in one launch per kernel; status_out:
 * NULL or bt_batch_size() statuses.  Graphs that fail keep their poses. */
int bt_warmstart_apply_batch(bt_warmstart* ws, bt_batch* b, int32_t* status_out);

/* Warm-started batch solve with the plain solve as fallback: applies the
 * warm start to every graph of b, runs `iters` Gauss-Newton iterations of the
 * batch (bt_batch_solve), and re-solves with `fallback_iters` plain
 * iterations (bt_solve, from the poses stored before the call) every graph
 * whose solve failed or that fails the acceptance rule:
 *   ref_costs != NULL (the plain solve's final costs, one per graph in batch
 *     order): the final cost exceeds (1 + tol) * ref_costs[k];
 *   ref_costs == NULL (a rule that needs no plain solve): the last
 *     warm-started iteration changed the cost by more than tol times the
 *     final cost, |E_{iters-1} - E_iters| > tol E_iters -- the iterations had
 *     not converged (with iters == 0 only failures fall back).
 * reps: NULL or bt_batch_size() reports with used_warmstart / fell_back set.
 * Synchronises the batch stream.
 * Errors: BT_ERR_INVALID, BT_ERR_STATE, BT_ERR_SINGULAR, BT_ERR_TIMEOUT (every
 * graph keeps the poses it had before the call), BT_ERR_CUDA, BT_ERR_OOM. */
int bt_batch_solve_warm(bt_batch* b, bt_warmstart* ws, int32_t iters, int32_t fallback_iters,
                        const double* ref_costs, double tol, bt_solve_report* reps);

/* ------------------------------------------------- coarse registration
 * Sec. IV-B: RANSAC over 3-point samples of a correspondence set, each
 * hypothesis the closed-form least-squares rigid fit (Arun et al.; computed
 * in quaternion form), an inlier a pair with |R p + t - q| < inlier_dist
 * (the paper uses 5 mm; its normal-angle gate needs normals, which
 * correspondence sets do not carry).  The result is the sample with the
 * most inliers (ties: the earlier sample), refitted on its inliers when
 * refine != 0 (the paper keeps the best sample's fit).  Sample h draws its
 * indices from the counter-based SplitMix64 generator: value(c) =
 * mix(seed + (c + 1) * 0x9E3779B97F4A7C15) for c = 16 h, 16 h + 1, ...,
 * index = value % count, the first three distinct indices.  Inlier tests are
 * evaluated in single precision with a fixed operation order. */

/* Relative pose of one correspondence set: rel_out (4x4 row-major) maps
 * camera i to camera j, q ~ rel_out p (pts_i, pts_j: count x 3 floats, host
 * or device); inliers_out (may be NULL) gets the inlier count.  With fewer
 * than 3 points or only degenerate samples rel_out is the identity and the
 * count 0.  Enqueued on cuda_stream and synchronised.
 * Errors: BT_ERR_INVALID, BT_ERR_CUDA, BT_ERR_OOM. */
int bt_ransac(const float* pts_i, const float* pts_j, int32_t count, int32_t mem_kind, int32_t hypotheses,
              uint64_t seed, double inlier_dist, int32_t refine, double* rel_out, int32_t* inliers_out,
              void* cuda_stream);

/* Coarse initialisation of a graph's free active nodes, as the paper
 * initialises a new frame from the previous one: each free node j with a
 * correspondence set to a fixed node f (the lowest-indexed such f) gets
 * T_j = M T_f with M = T_j T_f^-1 estimated by bt_ransac on that set (all
 * sets in one launch); other nodes keep their poses.
 * Errors: BT_ERR_INVALID, BT_ERR_CUDA, BT_ERR_OOM. */
int bt_ransac_init(bt_graph* g, int32_t hypotheses, uint64_t seed, double inlier_dist, int32_t refine);

/* --------------------------------------------- memory pool (host only)
 * Keyframe selection of Sec. IV-C and pool augmentation of Sec. IV-E.  Both
 * read the rotation blocks of 4x4 row-major poses (host arrays) and do no
 * GPU work.  The distance of two keyframes is the geodesic distance of their
 * rotations, arccos((tr(R_a^T R_b) - 1) / 2). */

/* Greedy minimum-H-subgraph selection: starts from pool entry 0 (I_0) and
 * repeatedly adds the pool entry with the smallest summed distance to the
 * current frame and to every entry selected so far (ties: the earlier entry),
 * until min(K, n_pool) entries are selected.  Writes their pool indices in
 * selection order to out[0 .. count) and returns count, or a negative status
 * (BT_ERR_INVALID: negative size, NULL, non-finite pose). */
int32_t bt_select_keyframes(const double* pool_poses, int32_t n_pool, const double* pose_current, int32_t K,
                            int32_t* out);

/* Pool augmentation rule: 1 when the current frame's distance to every pool
 * entry exceeds min_deg degrees (the paper uses 10), else 0; a negative
 * status on bad arguments. */
int32_t bt_is_novel_view(const double* pool_poses, int32_t n_pool, const double* pose_current, double min_deg);

/* ------------------------------------------------------------ diagnostics
 * Intermediate results of a Gauss-Newton iteration of bt_solve at the stored
 * poses of the active nodes, computed by the solve's own kernels, so that an
 * independent implementation can be compared with them value by value.  No
 * paper counterpart; the stored poses are not changed. */

/* The dense association of the ordered pair (src_node -> dst_node), both
 * indices in the active node order (Eq. 3 and the gating sentence after it,
 * Sec. IV-D): for every valid masked pixel of src_node, in increasing pixel
 * order, the pixel v * width + u of dst_node that the residual pass
 * associates it with, or -1 when it is dropped (projection behind the
 * camera or outside the image, invalid target pixel, distance gate, angle
 * gate).  tgt_out: host array of cap entries, or NULL to query the count
 * only; *count_out (may be NULL) receives the number of valid source
 * pixels, also when cap is too small.  Synchronises the stream.
 * Errors: BT_ERR_INVALID (NULL graph, node out of range, src_node ==
 * dst_node, cap smaller than the count), BT_ERR_CUDA, BT_ERR_OOM. */
int bt_debug_associate(bt_graph* g, int32_t src_node, int32_t dst_node, int32_t* tgt_out, int32_t cap,
                       int32_t* count_out);

/* The normal equations H dx = -g of one Gauss-Newton iteration at the stored
 * poses (Sec. IV-D), exactly as bt_solve assembles them before its FP64
 * factorisation: n = 6 x (free active nodes) unknowns, right perturbations
 * T_i <- T_i exp(dx_i), dx_i = (v, w) (translation first), free nodes in
 * active order.  H_out: n x n row-major, symmetric; g_out: n; both host.
 * cost_out (4 doubles, may be NULL): E of Eq. 1, its dense part, its sparse
 * part and the number of accepted dense associations at those poses.
 * *n_out (may be NULL) receives n, also when n_cap < n.  Synchronises the
 * stream.  Errors: BT_ERR_INVALID (NULL graph or output, n_cap < n, no free
 * node), BT_ERR_CUDA, BT_ERR_OOM. */
int bt_debug_normal_equations(bt_graph* g, double* H_out, double* g_out, int32_t n_cap, int32_t* n_out,
                              double* cost_out);

/* Makes the library's next n device or pinned host allocations fail as if
 * memory were exhausted -- the calls that needed them return BT_ERR_OOM and
 * leave their objects as they were -- so that a caller can exercise its
 * out-of-memory handling without exhausting a GPU; n = 0 cancels.  Process
 * wide (every thread and graph).  Returns the number of injected failures
 * that were still pending.  Allocations the device-memory cache can serve
 * from idle blocks are not allocations and do not consume one. */
int32_t bt_debug_fail_allocations(int32_t n);

/* Sets the bound (nanoseconds of the GPU's global timer) of the warm-start
 * forward pass's waits for its tensor-core contractions, for the launches
 * that follow; ns < 0 restores the default of 1 s, and ns = 0 makes the first
 * wait give up at once, so that a caller can exercise the BT_ERR_TIMEOUT
 * path (the kernel still lets the contraction in flight finish before it
 * frees its tensor memory).  Process wide.  Returns the previous bound. */
int64_t bt_debug_tensor_wait_ns(int64_t ns);

/* Profiling counters of one graph (the tracing facility; no paper
 * counterpart).  Launch counts are always kept; kernel durations are summed
 * from CUDA events recorded on the graph's stream around each launch of the
 * residual and reduce kernels of the timed solves (every solve, or every
 * k-th: see bt_profile_enable); the pixel-pair and correspondence counts
 * below cover the same timed launches. */
typedef struct {
    int64_t prep_launches;      /* frame-preparation kernels (3 per frame) */
    int64_t xform_launches;     /* transform kernels: always 0 (a solve's first
                                 * transforms are formed on the host, the later
                                 * ones by the update in the reduce kernel);
                                 * kept so that the layout does not change */
    int64_t residual_launches;  /* residual pass launches (dense + sparse) */
    int64_t reduce_launches;    /* reduce / assemble / solve launches */
    double residual_ms;         /* summed event time of timed residual launches */
    double reduce_ms;           /* summed event time of timed reduce launches */
    int64_t timed_residual_launches;
    int64_t timed_reduce_launches;
    int64_t dense_pixel_pairs;  /* source-pixel x target pairs of timed residual launches */
    int64_t sparse_pairs;       /* correspondences of timed residual launches */
    /* SM clock cycles of the solve stage (the last CTA of each Gauss-Newton
     * iteration): [0] gathering the pair blocks and assembling H, g;
     * [1] Cholesky factorisation with the forward substitution; [2] back
     * substitution; [3] pose update and single-precision transforms */
    int64_t solve_phase_cycles[4];
} bt_profile;

/* Enables (on > 0) or disables (on == 0) event timing and resets every
 * counter.  With on = k the events time every k-th bt_solve / bt_eval_cost
 * from here on (the first included): recording events between the kernels
 * of a solve costs host time and breaks the programmatic launch overlap of
 * the timed solves, so sampling keeps the untimed ones at full speed.
 * Errors: BT_ERR_INVALID (on < 0), BT_ERR_CUDA. */
int bt_profile_enable(bt_graph* g, int32_t on);

/* Copies the counters to *out (host).  Errors: BT_ERR_INVALID. */
int bt_profile_read(const bt_graph* g, bt_profile* out);

/* Device memory cache (no paper counterpart).  Frames and correspondence
 * sets live in blocks of a per-graph pool; a destroyed graph hands its
 * blocks to a process-wide cache of idle blocks, from which later graphs
 * take blocks of the same size class before allocating, so a series of
 * graphs reuses device memory instead of allocating and freeing it (cudaFree
 * synchronises the device).  Thread-safe.
 *
 * bt_device_cache_bytes: bytes of idle cached blocks.
 * bt_device_cache_trim: frees the idle blocks above 64 KiB (the smaller
 * ones share 2 MiB slabs that stay until the process exits) and returns the
 * bytes freed. */
int64_t bt_device_cache_bytes(void);
int64_t bt_device_cache_trim(void);

/* Dense energy of one frame pair without allocating device memory.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory at the time they need the number: code that
 * runs inside a framework owning all device memory through its own caching
 * allocator (a cudaMalloc there fragments the pool or is forbidden), real-time
 * loops where cudaMalloc/cudaFree would synchronise the device and stall
 * other streams, and embedders working under a fixed device-memory budget.
 *
 * It computes the dense part of bt_eval_cost (cost_out[1]) for a graph made
 * of these two frames, straight from the caller's buffers, with the same
 * association decisions, gates and Huber loss as the residual pass.
 *   depth_x, normals_x, mask_x: DEVICE pointers (H x W, H x W x 3, H x W);
 *   Kx, pose_x, cfg: host memory (cfg may be NULL for the defaults);
 *   out: DEVICE pointer to 2 doubles, receives the energy and the number of
 *        accepted associations (as a double);
 *   cuda_stream: cudaStream_t as void* (NULL = legacy default stream).
 * The work is enqueued on the stream and the call returns without waiting.
 * Scratch: a library-owned static device array of 512 KiB + 256 B, held by
 * every GPU that loads the library until the process exits; each frame may
 * have at most 16,777,216 pixels (sides <= 32767), larger frames are rejected
 * with BT_ERR_INVALID and a message.  All calls share that array: calls
 * whose GPU work overlaps (on different streams or from different threads)
 * race and must be serialised by the caller.  The first call on a device
 * looks up the array's device address with that device current; make that
 * first call before any stream capture.
 * Errors: BT_ERR_INVALID, BT_ERR_CUDA; bt_noalloc_last_error() has the text. */
int bt_pair_dense_energy_noalloc(const float* depth_a, const float* normals_a, const uint8_t* mask_a,
                                 const bt_intrinsics* Ka, const double pose_a[16],
                                 const float* depth_b, const float* normals_b, const uint8_t* mask_b,
                                 const bt_intrinsics* Kb, const double pose_b[16], const bt_config* cfg,
                                 double* out, void* cuda_stream);

/* Message of the last bt_pair_dense_energy_noalloc failure on the calling
 * thread ("" if none). */
const char* bt_noalloc_last_error(void);

/* Text for a status code (static storage). */
const char* bt_status_str(int status);

/* Message describing the last failure on the calling thread ("" if none). */
const char* bt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
