// bt_ws.h -- device layout and kernel entry points of the learned warm start.
//
// The warm start replaces the coarse initialisation from sparse matches
// (Sec. IV-B) for every node of a pose graph at once: a set network on each
// correspondence set predicts the increment of that edge's relative pose,
// and an FP64 relative-pose averaging solve turns the edge increments into
// node poses, which Gauss-Newton (Sec. IV-D) then refines.
//
// Network (shared over the points of a set, max-pool over the set):
//   x (6) -> 128 -> 256 (ReLU after each) -> max over the set -> 128 (ReLU) -> 6
// Parameters: one flat FP32 vector (the master copy trained by Adam) in the
// order W1 [128][6], b1, W2 [256][128], b2, W3 [128][256], b3, W4 [6][128], b4
// (row = output unit); BF16 copies of the four weight matrices are what the
// kernels read.  Inputs of the 128 -> 256 contraction are rounded to BF16,
// every sum is FP32.
#pragma once

#include "bt_internal.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace bt {
namespace ws {

constexpr int kIn = 6, kH1 = 128, kH2 = 256, kH3 = 128, kOut = 6;
constexpr int oW1 = 0, ob1 = oW1 + kH1 * kIn, oW2 = ob1 + kH1, ob2 = oW2 + kH2 * kH1, oW3 = ob2 + kH2,
              ob3 = oW3 + kH3 * kH2, oW4 = ob3 + kH3, ob4 = oW4 + kOut * kH3, kNumParams = ob4 + kOut;
constexpr int bW1 = 0, bW2 = bW1 + kH1 * kIn, bW3 = bW2 + kH2 * kH1, bW4 = bW3 + kH3 * kH2,
              kNumBf16 = bW4 + kOut * kH3;
static_assert(kNumParams == 67590, "parameter layout");

// Feature and output scales: x = ((p' - c) / 0.1 m, (q - p') / 0.01 m),
// y = (omega / 0.1 rad, u / 0.01 m).
constexpr float kInvSP = 10.0f, kInvSR = 100.0f;
constexpr double kSW = 0.1, kSU = 0.01;

// One correspondence set (edge i -> j): p in camera i, q in camera j.
struct Sample {
    const float* p;     // [n][3]
    const float* q;     // [n][3]
    int n;
    int pad;
    float m[12];        // M0 = T_j T_i^-1 at the initial poses, float 3x4 row-major
    float c[4];         // centre of the set: mean of q (c[3] unused)
    float ystar[6];     // training label
    float pad2[2];
};

// Where the prep kernel finds the poses of a sample (3x4 row-major FP64):
// M0 = Tj0 Ti0^-1 and, when Ti1 is not null, the label from M = Tj1 Ti1^-1.
struct PrepItem {
    int sample;
    int pad;
    const double* Ti0;
    const double* Tj0;
    const double* Ti1;
    const double* Tj1;
};

struct Net {
    float* master;              // [kNumParams]
    __nv_bfloat16* wb;          // [kNumBf16]
    float* m;                   // Adam first moments
    float* v;                   // Adam second moments
    int* fault;                 // set to 1 when a bounded wait of the forward pass ran out (mapped host word)
    long long wait_ns;          // bound of the forward pass's waits on the tensor cores (<= 0: give up at once)
};

// What the backward pass needs of one set's forward pass.
struct Cache {
    float g[kH2];       // max-pooled features
    int r[kH2];         // row holding each channel's maximum
    float z3[kH3];      // head pre-activations
    float y[kOut];
    float pad[2];
};

// One graph of an averaging launch.
struct AvgGraph {
    int N, n_edges, n_free, pad;
    const NodeDev* nodes;       // free_idx < 0: fixed
    const EdgeDev* edges;       // (i, j), count
    const float* y;             // [n_edges][6] network outputs
    const Sample* smp;          // [n_edges] (centres)
    double* pose;               // [N][12] in: initial poses, out: warm-start poses
    double* scratch;            // [n_edges][kAvgScratch]
    int* status;                // 0 ok, 1 singular (poses left unchanged)
};

cudaError_t launch_prep(Sample* smp, const PrepItem* items, int n, cudaStream_t s);
cudaError_t launch_to_bf16(Net net, cudaStream_t s);
// Forward over sets ids[0..n) (ids may be null: sets 0..n); y_out [n][6];
// cache (training) [n] or null.
cudaError_t launch_forward(Net net, const Sample* smp, const int* ids, int n, float* y_out, Cache* cache,
                           cudaStream_t s);
size_t forward_smem_bytes();
// Per-set gradients of the mean loss 1/2 |y - y*|^2 into G [n][kNumParams],
// per-set losses into loss_per [n].
cudaError_t launch_backward(Net net, const Sample* smp, const int* ids, int n, const Cache* cache, float* G,
                            float* loss_per, cudaStream_t s);
// grad = sum over sets of G (fixed order), loss = sum of loss_per (FP64).
cudaError_t launch_reduce(const float* G, const float* loss_per, int n, float* grad, double* loss,
                          cudaStream_t s);
// Adam step: c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t).
cudaError_t launch_adam(Net net, const float* grad, float lr, float beta1, float beta2, float eps, float c1,
                        float c2, cudaStream_t s);
// Scratch doubles per edge of an averaging launch: the increment D [12], the
// residual e [6], the adjoint A [36], P = A^T W A (lower triangle) [21],
// A^T W e [6], padding.
constexpr int kAvgScratch = 88;
cudaError_t launch_average(const AvgGraph* graphs, int n_graphs, int max_free, cudaStream_t s);
size_t average_smem_bytes(int max_free, int max_N);
// Rebases sample point pointers after the point pool moved.
cudaError_t launch_rebase(Sample* smp, int n, const float* old_p, const float* new_p, const float* old_q,
                          const float* new_q, cudaStream_t s);

}  // namespace ws
}  // namespace bt
