// bt_warmstart.cu -- kernels of the learned warm start (see bt_ws.h): sample
// preparation, the set network's forward and backward passes, the gradient
// reduction, Adam, and the FP64 relative-pose averaging solve that turns the
// predicted edge increments into node poses for Gauss-Newton (Sec. IV-D).
//
// Forward pass: a persistent CTA per SM keeps the BF16 W2 (in the tensor
// cores' core-matrix layout) and W3 in shared memory and walks its sets in
// chunks of 128 points.  Layer 1 (K = 6) runs on the FP32 pipes and is
// rounded to BF16 into one of two shared-memory tiles; the 128 x 256 x 128
// contraction of layer 2 runs on the fifth-generation tensor cores
// (tcgen05.mma, BF16 in, FP32 accumulators in tensor memory, issued by one
// thread, completion signalled on an mbarrier).  While the tensor cores work
// on chunk c, the CUDA cores compute layer 1 of chunk c+1 into the other
// tile, and then read chunk c's accumulators (tcgen05.ld) for bias, ReLU and
// a running per-channel maximum (with the row that holds it, first row on
// ties); two accumulators in tensor memory let chunk c+1's contraction run
// during that read-out.  Then the 256 -> 128 -> 6 head.  Every wait on the
// tensor cores is bounded (globaltimer); a wait that runs out sets the
// network's fault word, drains the contraction in flight, frees the tensor
// memory and ends the kernel, and the host reports BT_ERR_TIMEOUT.
// Backward pass: only the rows that hold a channel's maximum receive
// gradient, so layer 1 and layer 2 gradients are outer products over at most
// 256 rows, recomputed from the inputs with the forward pass's arithmetic.
#include "bt_ldlt.h"
#include "bt_ws.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace bt {
namespace ws {

namespace {

constexpr int kFwdThreads = 256;
constexpr int kChunk = 128;     // points per layer-2 tile: the M of one tensor-core contraction
constexpr int kLd3 = 258;       // padded row length (BF16) of the layer-3 weights (odd word stride)

__device__ __forceinline__ float bf2f(__nv_bfloat16 b) { return __bfloat162float(b); }

// Features of one point pair (p in camera i, q in camera j: v = px py pz qx
// qy qz), FP32 with a fixed operation order (the backward pass recomputes
// them bit for bit).
__device__ __forceinline__ void features_from(const float v[6], const float* m, const float* c, float x[6])
{
    const float px = v[0], py = v[1], pz = v[2];
    const float qx = v[3], qy = v[4], qz = v[5];
    const float ux = __fmaf_rn(m[0], px, __fmaf_rn(m[1], py, __fmaf_rn(m[2], pz, m[3])));
    const float uy = __fmaf_rn(m[4], px, __fmaf_rn(m[5], py, __fmaf_rn(m[6], pz, m[7])));
    const float uz = __fmaf_rn(m[8], px, __fmaf_rn(m[9], py, __fmaf_rn(m[10], pz, m[11])));
    x[0] = __fmul_rn(__fsub_rn(ux, c[0]), kInvSP);
    x[1] = __fmul_rn(__fsub_rn(uy, c[1]), kInvSP);
    x[2] = __fmul_rn(__fsub_rn(uz, c[2]), kInvSP);
    x[3] = __fmul_rn(__fsub_rn(qx, ux), kInvSR);
    x[4] = __fmul_rn(__fsub_rn(qy, uy), kInvSR);
    x[5] = __fmul_rn(__fsub_rn(qz, uz), kInvSR);
}

// Point pair k of a set (zeros when k >= n).
__device__ __forceinline__ void load_pair(const float* __restrict__ p, const float* __restrict__ q, int k, int n,
                                          float v[6])
{
    if (k < n) {
        v[0] = p[3 * k];
        v[1] = p[3 * k + 1];
        v[2] = p[3 * k + 2];
        v[3] = q[3 * k];
        v[4] = q[3 * k + 1];
        v[5] = q[3 * k + 2];
    } else {
#pragma unroll
        for (int e = 0; e < 6; ++e) v[e] = 0.f;
    }
}

// Features of point k of a set.
__device__ __forceinline__ void point_features(const float* __restrict__ p, const float* __restrict__ q,
                                               const float* m, const float* c, int k, float x[6])
{
    float v[6];
    load_pair(p, q, k, k + 1, v);
    features_from(v, m, c, x);
}

// Offset (floats) of layer-1 unit u's packed weights in the forward kernel's
// shared memory: 8 floats a unit, each block of 32 units skewed by 16 bytes,
// so that the four threads of a row, which take the blocks u / 32 = 0..3,
// read four different bank groups.
__device__ __forceinline__ int w1_at(int u) { return u * 8 + (u >> 5) * 4; }

// z1_unit with the unit's weights and bias packed as w[0..5], w[6] = bias
// (two 16-byte shared-memory loads); the same operations in the same order.
__device__ __forceinline__ float z1_unit8(const float* w8, const float x[6])
{
    const float4 a = *reinterpret_cast<const float4*>(w8);
    const float4 b = *reinterpret_cast<const float4*>(w8 + 4);
    float z = b.z;
    z = __fmaf_rn(a.x, x[0], z);
    z = __fmaf_rn(a.y, x[1], z);
    z = __fmaf_rn(a.z, x[2], z);
    z = __fmaf_rn(a.w, x[3], z);
    z = __fmaf_rn(b.x, x[4], z);
    z = __fmaf_rn(b.y, x[5], z);
    return z;
}

// Layer-1 pre-activation of one unit (weights w[6], bias b), fixed order.
__device__ __forceinline__ float z1_unit(const float* w, float b, const float x[6])
{
    float a = b;
#pragma unroll
    for (int k = 0; k < 6; ++k) a = __fmaf_rn(w[k], x[k], a);
    return a;
}

// ---------------------------------------------------------------------------
// Fifth-generation tensor cores (PTX ISA: tcgen05 instructions, shared-memory
// matrix descriptors, instruction descriptor of kind::f16)
// ---------------------------------------------------------------------------

// Both operands of the layer-2 contraction are K-major BF16 with K = 128,
// stored without swizzling as core matrices of 8 rows x 16 bytes (8 values of
// K): element (row, k) at core_off(row, k).  In the matrix descriptor the
// leading-dimension offset is the distance between core matrices that follow
// each other along K, the stride-dimension offset the distance between
// neighbouring groups of 8 rows.
constexpr uint32_t kCoreK = 128;                    // bytes from one core matrix to the next along K
constexpr uint32_t kCoreRows = (kH1 / 8) * kCoreK;  // 2048: bytes from one group of 8 rows to the next
constexpr uint32_t kH1TileBytes = kChunk * kH1 * 2; // one BF16 [128][128] tile of layer-1 outputs
__host__ __device__ constexpr uint32_t core_off(int row, int k)
{
    return (uint32_t)(row >> 3) * kCoreRows + (uint32_t)(k >> 3) * kCoreK + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// Matrix descriptor: start address >> 4 (bits 0-13), leading-dimension byte
// offset >> 4 (16-29), stride-dimension byte offset >> 4 (32-45), the fixed
// value 1 in bits 46-48, base offset 0, no swizzling.
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kCoreK >> 4) << 16) |
           ((uint64_t)(kCoreRows >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kH2 >> 3) << 17) |
                            ((uint32_t)(kChunk >> 4) << 24);
static_assert(kChunk == 128 && kH2 % 16 == 0 && kH2 <= 256, "shape of one kind::f16 contraction (M = 128)");

constexpr int kTmemCols = 2 * kH2;                 // two FP32 [128][256] accumulators
constexpr long long kTensorWaitNs = 1000000000LL;  // default bound of a wait on the tensor cores (1 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// D[128][256] (tensor memory at d_tmem) = A[128][128] . B[256][128]^T, A and B
// K-major in shared memory: eight K = 16 steps, the first overwriting D; the
// completion of all eight arrives on the mbarrier at `bar`.  One thread.
__device__ __forceinline__ void issue_layer2(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, uint32_t bar)
{
#pragma unroll
    for (int k = 0; k < kH1 / 16; ++k) {
        const uint64_t ad = mat_desc(a_saddr + 2 * kCoreK * k), bd = mat_desc(b_saddr + 2 * kCoreK * k);
        asm volatile(
            "{\n\t.reg .pred acc;\n\tsetp.ne.b32 acc, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, acc;\n\t}"
            ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"((uint32_t)(k > 0))
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Waits until phase `parity` of the mbarrier at `bar` has completed, for at
// most limit_ns of the global timer; limit_ns <= 0 gives up without polling.
__device__ __forceinline__ bool wait_tensor(uint32_t bar, uint32_t parity, long long limit_ns)
{
    if (limit_ns <= 0) return false;
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((long long)(global_ns() - t0) > limit_ns) return false;
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Eight 16-lane x 256-bit blocks of tensor memory from taddr on (columns
// taddr + 8j .. + 8j + 7 for block j), waited for: lane l of the warp gets
// v[4j], v[4j+1] = row (l / 4), columns 8j + 2 (l % 4) + {0, 1}, and
// v[4j+2], v[4j+3] = row (l / 4) + 8, the same columns.
__device__ __forceinline__ void tmem_load_16x256b_x8(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

// Layer 1 of one row of a chunk, 64 of the 128 units (half 0 or 1): ReLU,
// rounded to BF16, written as eight 16-byte core-matrix rows of the tile.
__device__ __forceinline__ void layer1_half_row(unsigned char* tile, const float* sW1, const float x[6], int row,
                                                int half)
{
    unsigned char* dst = tile + core_off(row, half * 64);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int u = half * 64 + 8 * j + 2 * e;
            const float h0 = fmaxf(z1_unit8(sW1 + w1_at(u), x), 0.f);
            const float h1 = fmaxf(z1_unit8(sW1 + w1_at(u + 1), x), 0.f);
            __nv_bfloat162 b = __floats2bfloat162_rn(h0, h1);
            w[e] = *reinterpret_cast<uint32_t*>(&b);
        }
        *reinterpret_cast<uint4*>(dst + j * kCoreK) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Shared-memory layout of the forward kernel (byte offsets).
struct Fwd {
    static constexpr size_t W2 = 0;                                          // bf16 [256][128], core_off layout
    static constexpr size_t H1 = W2 + 2 * (size_t)kH2 * kH1;                 // 2 x bf16 [128][128], core_off layout
    static constexpr size_t W3 = H1 + 2 * (size_t)kH1TileBytes;              // bf16 [128][kLd3]
    static constexpr size_t W1 = W3 + ((2 * (size_t)kH3 * kLd3 + 15) / 16) * 16;   // float [128][8] + skew (w1_at)
    static constexpr size_t B2 = W1 + 4 * ((size_t)kH1 * 8 + 16);            // float [256]
    static constexpr size_t B3 = B2 + 4 * (size_t)kH2;                       // float [128]
    static constexpr size_t W4 = B3 + 4 * (size_t)kH3;                       // float [6][128]
    static constexpr size_t B4 = W4 + 4 * (size_t)kOut * kH3;                // float [8]
    static constexpr size_t G = B4 + 32;                                     // float [256]
    static constexpr size_t R = G + 4 * (size_t)kH2;                         // int [256]
    static constexpr size_t RV = R + 4 * (size_t)kH2;                        // float [4][256]
    static constexpr size_t RI = RV + 16 * (size_t)kH2;                      // int [4][256]
    static constexpr size_t H3 = RI + 16 * (size_t)kH2;                      // float [128]
    static constexpr size_t Z3 = H3 + 4 * (size_t)kH3;                       // float [128]
    static constexpr size_t MC = Z3 + 4 * (size_t)kH3;                       // float [16]: m[12], c[3]
    static constexpr size_t BAR = MC + 64;                                   // two mbarriers (u64)
    static constexpr size_t TM = BAR + 16;                                   // tensor-memory base address
    static constexpr size_t Total = TM + 16;
};
static_assert(Fwd::H1 % 16 == 0 && Fwd::W3 % 16 == 0 && Fwd::W1 % 16 == 0 && Fwd::BAR % 8 == 0, "alignment");
static_assert(Fwd::Total <= 227 * 1024, "shared memory of one CTA");
static_assert(Fwd::Total > 114 * 1024, "one CTA per SM: the two accumulators take all of its tensor memory");
static_assert(kFwdThreads == 2 * kH3 && kFwdThreads == kH2, "head mapping: two threads per layer-3 unit");
static_assert(kFwdThreads == 2 * kChunk, "layer 1: two threads per row of a chunk");

template <bool kTrain>
__global__ void __launch_bounds__(kFwdThreads, 1)
    forward_kernel(Net net, const Sample* __restrict__ smp, const int* __restrict__ ids, int n_sets,
                   float* __restrict__ y_out, Cache* __restrict__ cache)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __nv_bfloat16* sW3 = reinterpret_cast<__nv_bfloat16*>(sm + Fwd::W3);    // layer 3: [unit][kLd3]
    float* sW1 = reinterpret_cast<float*>(sm + Fwd::W1);     // unit u at w1_at(u): weights [0..5], bias [6]
    float* sB2 = reinterpret_cast<float*>(sm + Fwd::B2);
    float* sB3 = reinterpret_cast<float*>(sm + Fwd::B3);
    float* sW4 = reinterpret_cast<float*>(sm + Fwd::W4);
    float* sB4 = reinterpret_cast<float*>(sm + Fwd::B4);
    float* sG = reinterpret_cast<float*>(sm + Fwd::G);
    int* sR = reinterpret_cast<int*>(sm + Fwd::R);
    float* sRV = reinterpret_cast<float*>(sm + Fwd::RV);
    int* sRI = reinterpret_cast<int*>(sm + Fwd::RI);
    float* sH3 = reinterpret_cast<float*>(sm + Fwd::H3);
    float* sZ3 = reinterpret_cast<float*>(sm + Fwd::Z3);
    float* sMC = reinterpret_cast<float*>(sm + Fwd::MC);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // stage the weights once per CTA; W2 as 16-byte core-matrix rows
    for (int k = tid; k < kH2 * kH1 / 8; k += kFwdThreads) {
        const int row = k >> 4, k8 = (k & 15) * 8;
        *reinterpret_cast<uint4*>(sm + Fwd::W2 + core_off(row, k8)) =
            *reinterpret_cast<const uint4*>(net.wb + bW2 + row * kH1 + k8);
    }
    for (int k = tid; k < kH3 * kH2 / 2; k += kFwdThreads) {   // bf16 pairs, rows padded to kLd3
        const int o = k / (kH2 / 2), c2 = (k % (kH2 / 2)) * 2;
        *reinterpret_cast<uint32_t*>(sW3 + o * kLd3 + c2) =
            *reinterpret_cast<const uint32_t*>(net.wb + bW3 + o * kH2 + c2);
    }
    for (int k = tid; k < kH1 * 8; k += kFwdThreads) {
        const int u = k >> 3, e = k & 7;
        sW1[w1_at(u) + e] = e < kIn ? bf2f(net.wb[bW1 + u * kIn + e]) : (e == kIn ? net.master[ob1 + u] : 0.f);
    }
    for (int k = tid; k < kOut * kH3; k += kFwdThreads) sW4[k] = bf2f(net.wb[bW4 + k]);
    for (int k = tid; k < kH2; k += kFwdThreads) sB2[k] = net.master[ob2 + k];
    for (int k = tid; k < kH3; k += kFwdThreads) sB3[k] = net.master[ob3 + k];
    if (tid < kOut) sB4[tid] = net.master[ob4 + tid];

    const uint32_t bar0 = smem_u32(sm + Fwd::BAR);    // mbarrier of accumulator b at bar0 + 8 b
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sm + Fwd::TM)),
                     "r"((uint32_t)kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the tensor cores read W2 and the layer-1 tiles through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + Fwd::TM);
    const uint32_t w2_s = smem_u32(sm + Fwd::W2), h1_s = smem_u32(sm + Fwd::H1);
    unsigned char* const h1_tile = sm + Fwd::H1;

    // read-out: warp w takes the tensor-memory lanes (rows of a chunk)
    // 32 (w % 4) .. + 31 and the columns 128 (w / 4) .. + 127; a lane holds
    // 32 of those columns (idx: column 128 cw + 8 (idx / 2) + 2 (lane % 4) + idx % 2)
    const int qr = warp & 3, cw = warp >> 2;
    float b2[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) b2[k] = sB2[128 * cw + 8 * (k >> 1) + 2 * (lane & 3) + (k & 1)];
    const int lrow = tid >> 1, lhalf = tid & 1;   // layer 1: thread = (row of the chunk, half of the 128 units)
    uint32_t cc = 0;                              // chunks this CTA has contracted so far
    bool fault = false;
    for (int s = blockIdx.x; s < n_sets; s += gridDim.x) {
        const int sid = ids ? ids[s] : s;
        const Sample* S = smp + sid;
        const int n = S->n;
        if (tid < 12) sMC[tid] = S->m[tid];
        else if (tid < 15) sMC[tid] = S->c[tid - 12];
        __syncthreads();      // weights staged (first set), sMC ready, previous set's head done
        if (n <= 0) {         // empty set: no prediction
            if (tid < kOut) y_out[(size_t)s * kOut + tid] = 0.f;
            continue;
        }
        const float* P = S->p;
        const float* Q = S->q;
        // running maxima of the thread's 32 columns (ReLU outputs are >= 0);
        // training also keeps the row that holds each (first row on ties)
        float best[32];
        int bestr[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            best[k] = kTrain ? -1.f : 0.f;
            bestr[k] = 0;
        }
        const int nch = (n + kChunk - 1) / kChunk;
        float pq[6];                             // the point pair of this thread's row of a chunk
        load_pair(P, Q, lrow, n, pq);
        {
            float x[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (lrow < n) features_from(pq, sMC, sMC + 12, x);
            layer1_half_row(h1_tile + (cc & 1) * kH1TileBytes, sW1, x, lrow, lhalf);
        }
        load_pair(P, Q, kChunk + lrow, n, pq);   // in flight during the first contraction
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) issue_layer2(tmem + (cc & 1) * kH2, h1_s + (cc & 1) * kH1TileBytes, w2_s, bar0 + 8 * (cc & 1));
        for (int c = 0; c < nch; ++c, ++cc) {
            const uint32_t b = cc & 1;
            if (c + 1 < nch) {   // layer 1 of the next chunk while the tensor cores work on this one
                const int gr = (c + 1) * kChunk + lrow;
                float x[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (gr < n) features_from(pq, sMC, sMC + 12, x);
                layer1_half_row(h1_tile + (b ^ 1) * kH1TileBytes, sW1, x, lrow, lhalf);
                load_pair(P, Q, (c + 2) * kChunk + lrow, n, pq);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            const bool done = wait_tensor(bar0 + 8 * b, (cc >> 1) & 1, net.wait_ns);
            tc_fence_before();
            if (__syncthreads_or(!done)) {
                // give the contraction in flight time to finish before the
                // tensor memory is freed, then end the kernel
                wait_tensor(bar0 + 8 * b, (cc >> 1) & 1, kTensorWaitNs);
                fault = true;
                break;
            }
            tc_fence_after();
            if (c + 1 < nch && tid == 0)
                issue_layer2(tmem + (b ^ 1) * kH2, h1_s + (b ^ 1) * kH1TileBytes, w2_s, bar0 + 8 * (b ^ 1));
            // bias, ReLU and the running maximum of chunk c; rows in increasing order
            const uint32_t tacc = tmem + b * kH2 + 128 * cw;
#pragma unroll
            for (int lh = 0; lh < 2; ++lh) {
                const int rb = c * kChunk + 32 * qr + 16 * lh;
                if (rb >= n) break;   // the same for the whole warp
                const int ra = rb + (lane >> 2), rc = ra + 8;
                const bool va = ra < n, vc = rc < n;
#pragma unroll
                for (int cq = 0; cq < 2; ++cq) {
                    uint32_t v[32];
                    tmem_load_16x256b_x8(tacc + ((uint32_t)(32 * qr + 16 * lh) << 16) + 64 * cq, v);
#pragma unroll
                    for (int g = 0; g < 8; ++g)
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int k = 2 * (8 * cq + g) + e;
                            if constexpr (kTrain) {
                                const float za = fmaxf(__uint_as_float(v[4 * g + e]) + b2[k], 0.f);
                                if (va && za > best[k]) {
                                    best[k] = za;
                                    bestr[k] = ra;
                                }
                                const float zc = fmaxf(__uint_as_float(v[4 * g + 2 + e]) + b2[k], 0.f);
                                if (vc && zc > best[k]) {
                                    best[k] = zc;
                                    bestr[k] = rc;
                                }
                            } else {   // max(0, max_rows z) = max_rows relu(z): one maximum an element
                                if (va) best[k] = fmaxf(best[k], __uint_as_float(v[4 * g + e]) + b2[k]);
                                if (vc) best[k] = fmaxf(best[k], __uint_as_float(v[4 * g + 2 + e]) + b2[k]);
                            }
                        }
                }
            }
            tc_fence_before();
        }
        if (fault) break;
        // combine the 8 lanes of each column, then the four row quarters
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            float v = best[k];
            int r = bestr[k];
#pragma unroll
            for (int off = 4; off < 32; off <<= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, v, off);
                if constexpr (kTrain) {
                    const int orr = __shfl_xor_sync(0xffffffffu, r, off);
                    if (ov > v || (ov == v && orr < r)) {
                        v = ov;
                        r = orr;
                    }
                } else {
                    v = fmaxf(v, ov);
                }
            }
            if (lane < 4) {
                const int col = 128 * cw + 8 * (k >> 1) + 2 * lane + (k & 1);
                sRV[qr * kH2 + col] = v;
                if (kTrain) sRI[qr * kH2 + col] = r;
            }
        }
        __syncthreads();
        {
            float v = sRV[tid];
            int r = kTrain ? sRI[tid] : 0;
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                const float v1 = sRV[q * kH2 + tid];
                if constexpr (kTrain) {
                    const int r1 = sRI[q * kH2 + tid];
                    if (v1 > v || (v1 == v && r1 < r)) {
                        v = v1;
                        r = r1;
                    }
                } else {
                    v = fmaxf(v, v1);
                }
            }
            sG[tid] = v;
            sR[tid] = r;
        }
        __syncthreads();
        {   // head layer 3: unit tid % 128, input half tid / 128; the odd row
            // stride kLd3 / 2 words puts the 32 units of a warp in 32 banks
            const int o = tid & (kH3 - 1), half = tid >> 7;
            const __nv_bfloat16* w = sW3 + o * kLd3 + half * 128;
            const float* g = sG + half * 128;
            float a = 0.f;
#pragma unroll 8
            for (int k = 0; k < 128; ++k) a = __fmaf_rn(bf2f(w[k]), g[k], a);
            sRV[tid] = a;      // the max-pool scratch is free again
        }
        __syncthreads();
        if (tid < kH3) {
            const float z = sB3[tid] + (sRV[tid] + sRV[kH3 + tid]);
            sZ3[tid] = z;
            sH3[tid] = fmaxf(z, 0.f);
        }
        __syncthreads();
        if (warp < kOut) {   // head layer 4: one warp per output
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) a = __fmaf_rn(sW4[warp * kH3 + lane + 32 * i], sH3[lane + 32 * i], a);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
            const float y = sB4[warp] + a;
            if (lane == 0) {
                y_out[(size_t)s * kOut + warp] = y;
                if (kTrain) cache[s].y[warp] = y;
            }
        }
        if (kTrain) {
            cache[s].g[tid] = sG[tid];
            cache[s].r[tid] = sR[tid];
            if (tid < kH3) cache[s].z3[tid] = sZ3[tid];
        }
    }
    if (fault && tid == 0) {
        *reinterpret_cast<volatile int*>(net.fault) = 1;
        __threadfence_system();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTmemCols)
                     : "memory");
    }
}

template <bool kTrain>
struct ForwardAttr {
    static void set()
    {
        static const bool done = [] {      // once per process, thread-safe
            cudaFuncSetAttribute(forward_kernel<kTrain>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Fwd::Total);
            return true;
        }();
        (void)done;
    }
};

int num_sms()
{
    static const int n = [] {             // once per process, thread-safe
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

// ---------------------------------------------------------------------------
// Backward pass: one CTA per set of the minibatch
// ---------------------------------------------------------------------------

constexpr int kBwdThreads = 256;

__global__ void __launch_bounds__(kBwdThreads)
    backward_kernel(Net net, const Sample* __restrict__ smp, const int* __restrict__ ids, int n_sets,
                    const Cache* __restrict__ cache, float inv_n, float* __restrict__ G,
                    float* __restrict__ loss_per)
{
    __shared__ float sW1[kH1 * kIn], sB1[kH1];
    __shared__ float sg[kH2], sdz2[kH2], sdz3[kH3], sh3[kH3], sz3[kH3], sdy[8], sMC[16];
    __shared__ int sr[kH2];
    __shared__ float sxr[kH2 * kIn];
    __shared__ float spart[2][kH1][7];
    const int s = blockIdx.x, tid = threadIdx.x;
    const int sid = ids ? ids[s] : s;
    const Sample* S = smp + sid;
    const Cache* C = cache + s;
    float* Gs = G + (size_t)s * kNumParams;
    const int n = S->n;
    if (n <= 0) {
        for (int k = tid; k < kNumParams; k += kBwdThreads) Gs[k] = 0.f;
        if (tid == 0) loss_per[s] = 0.f;
        return;
    }
    for (int k = tid; k < kH1 * kIn; k += kBwdThreads) sW1[k] = bf2f(net.wb[bW1 + k]);
    if (tid < kH1) sB1[tid] = net.master[ob1 + tid];
    sg[tid] = C->g[tid];
    sr[tid] = C->r[tid];
    if (tid < kH3) {
        sz3[tid] = C->z3[tid];
        sh3[tid] = fmaxf(C->z3[tid], 0.f);
    }
    if (tid < 12) sMC[tid] = S->m[tid];
    else if (tid < 15) sMC[tid] = S->c[tid - 12];
    if (tid < kOut) sdy[tid] = (C->y[tid] - S->ystar[tid]);
    __syncthreads();
    if (tid == 0) {
        float l = 0.f;
        for (int m = 0; m < kOut; ++m) l = __fmaf_rn(sdy[m], sdy[m], l);
        loss_per[s] = 0.5f * l * inv_n;
    }
    __syncthreads();
    if (tid < kOut) sdy[tid] *= inv_n;
    __syncthreads();
    // layer 4
    for (int k = tid; k < kOut * kH3; k += kBwdThreads) Gs[oW4 + k] = sdy[k / kH3] * sh3[k % kH3];
    if (tid < kOut) Gs[ob4 + tid] = sdy[tid];
    if (tid < kH3) {
        float a = 0.f;
        for (int m = 0; m < kOut; ++m) a = __fmaf_rn(bf2f(net.wb[bW4 + m * kH3 + tid]), sdy[m], a);
        const float d = sz3[tid] > 0.f ? a : 0.f;
        sdz3[tid] = d;
        Gs[ob3 + tid] = d;
    }
    __syncthreads();
    // layer 3: dW3 = dz3 g^T, dg = W3^T dz3
    for (int k = tid; k < kH3 * kH2; k += kBwdThreads) Gs[oW3 + k] = sdz3[k >> 8] * sg[k & 255];
    {
        float a = 0.f;
        for (int o = 0; o < kH3; ++o) a = __fmaf_rn(bf2f(net.wb[bW3 + o * kH2 + tid]), sdz3[o], a);
        const float d = sg[tid] > 0.f ? a : 0.f;     // ReLU' at the row holding the maximum
        sdz2[tid] = d;
        Gs[ob2 + tid] = d;
        float x[6];
        point_features(S->p, S->q, sMC, sMC + 12, sr[tid], x);
#pragma unroll
        for (int k = 0; k < 6; ++k) sxr[tid * kIn + k] = x[k];
    }
    __syncthreads();
    // layer 2: dW2[c][j] = dz2[c] * bf16(relu(z1(row r_c, unit j)))
    for (int k = tid; k < kH2 * kH1; k += kBwdThreads) {
        const int c = k >> 7, j = k & 127;
        const float z = z1_unit(sW1 + j * kIn, sB1[j], sxr + c * kIn);
        const float h = __bfloat162float(__float2bfloat16_rn(fmaxf(z, 0.f)));
        Gs[oW2 + k] = sdz2[c] * h;
    }
    // layer 1: dW1[j][k] = sum_c dz2[c] W2[c][j] [z1(r_c, j) > 0] x(r_c)[k]
    {
        const int j = tid & 127, half = tid >> 7;
        float a[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int c = half * 128; c < half * 128 + 128; ++c) {
            const float d = sdz2[c];
            if (d == 0.f) continue;
            const float z = z1_unit(sW1 + j * kIn, sB1[j], sxr + c * kIn);
            if (z > 0.f) {
                const float w = d * bf2f(net.wb[bW2 + c * kH1 + j]);
#pragma unroll
                for (int k = 0; k < 6; ++k) a[k] = __fmaf_rn(w, sxr[c * kIn + k], a[k]);
                a[6] += w;
            }
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) spart[half][j][k] = a[k];
    }
    __syncthreads();
    if (tid < kH1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) Gs[oW1 + tid * kIn + k] = spart[0][tid][k] + spart[1][tid][k];
        Gs[ob1 + tid] = spart[0][tid][6] + spart[1][tid][6];
    }
}

__global__ void reduce_kernel(const float* __restrict__ G, const float* __restrict__ loss_per, int n,
                              float* __restrict__ grad, double* __restrict__ loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kNumParams) {
        float a = 0.f;
        for (int s = 0; s < n; ++s) a += G[(size_t)s * kNumParams + p];
        grad[p] = a;
    }
    if (p == 0) {
        double l = 0.0;
        for (int s = 0; s < n; ++s) l += (double)loss_per[s];
        *loss = l;
    }
}

__device__ __forceinline__ int bf16_index(int p)
{
    if (p < ob1) return bW1 + (p - oW1);
    if (p >= oW2 && p < ob2) return bW2 + (p - oW2);
    if (p >= oW3 && p < ob3) return bW3 + (p - oW3);
    if (p >= oW4 && p < ob4) return bW4 + (p - oW4);
    return -1;
}

__global__ void adam_kernel(Net net, const float* __restrict__ grad, float lr, float beta1, float beta2,
                            float eps, float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNumParams) return;
    const float g = grad[p];
    const float m = beta1 * net.m[p] + (1.f - beta1) * g;
    const float v = beta2 * net.v[p] + (1.f - beta2) * g * g;
    net.m[p] = m;
    net.v[p] = v;
    const float w = net.master[p] - lr * (m * c1) / (sqrtf(v * c2) + eps);
    net.master[p] = w;
    const int b = bf16_index(p);
    if (b >= 0) net.wb[b] = __float2bfloat16_rn(w);
}

__global__ void to_bf16_kernel(Net net)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNumParams) return;
    const int b = bf16_index(p);
    if (b >= 0) net.wb[b] = __float2bfloat16_rn(net.master[p]);
}

// ---------------------------------------------------------------------------
// FP64 rigid-motion helpers (3x4 row-major [R | t]); twists ordered (v, omega)
// ---------------------------------------------------------------------------

__device__ void pose_mul(const double* A, const double* B, double* C)
{
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 4; ++c) {
            double s = A[r * 4 + 0] * B[0 * 4 + c] + A[r * 4 + 1] * B[1 * 4 + c] + A[r * 4 + 2] * B[2 * 4 + c];
            if (c == 3) s += A[r * 4 + 3];
            C[r * 4 + c] = s;
        }
    }
}

__device__ void pose_inv(const double* A, double* C)
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) C[r * 4 + c] = A[c * 4 + r];
    for (int r = 0; r < 3; ++r)
        C[r * 4 + 3] = -(A[0 * 4 + r] * A[3] + A[1 * 4 + r] * A[7] + A[2 * 4 + r] * A[11]);
}

// Rodrigues coefficients: A = sin t / t, B = (1 - cos t) / t^2, C = (1 - A) / t^2.
__device__ void rodrigues_coeffs(double th, double& A, double& B, double& C)
{
    const double t2 = th * th;
    if (th < 1e-4) {
        A = 1.0 - t2 / 6.0;
        B = 0.5 - t2 / 24.0;
        C = 1.0 / 6.0 - t2 / 120.0;
    } else {
        const double s = sin(th), c = cos(th);
        A = s / th;
        B = (1.0 - c) / t2;
        C = (1.0 - A) / t2;
    }
}

// T = exp(xi) for xi = (v, w): R = I + A [w]x + B [w]x^2, t = (I + B [w]x + C [w]x^2) v.
__device__ void se3_exp(const double* xi, double* T)
{
    const double* v = xi;
    const double* w = xi + 3;
    const double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double A, B, C;
    rodrigues_coeffs(th, A, B, C);
    const double W[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    double W2[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            W2[r * 3 + c] = W[r * 3 + 0] * W[0 * 3 + c] + W[r * 3 + 1] * W[1 * 3 + c] + W[r * 3 + 2] * W[2 * 3 + c];
    for (int r = 0; r < 3; ++r) {
        double t = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double id = r == c ? 1.0 : 0.0;
            T[r * 4 + c] = id + A * W[r * 3 + c] + B * W2[r * 3 + c];
            t += (id + B * W[r * 3 + c] + C * W2[r * 3 + c]) * v[c];
        }
        T[r * 4 + 3] = t;
    }
}

// w = log(R) of the rotation block of a 3x4 pose.
__device__ void so3_log(const double* T, double* w, double& th)
{
    double c = 0.5 * (T[0] + T[5] + T[10] - 1.0);
    c = c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c);
    th = acos(c);
    const double k = th < 1e-4 ? 0.5 + th * th / 12.0 : 0.5 * th / sin(th);
    w[0] = k * (T[9] - T[6]);
    w[1] = k * (T[2] - T[8]);
    w[2] = k * (T[4] - T[1]);
}

// xi = log(T): w = log(R), v = V^-1 t with V^-1 = I - [w]x / 2 + D [w]x^2,
// D = (1 - A / (2 B)) / t^2.
__device__ void se3_log(const double* T, double* xi)
{
    double w[3], th;
    so3_log(T, w, th);
    double A, B, C;
    rodrigues_coeffs(th, A, B, C);
    const double D = th < 1e-4 ? 1.0 / 12.0 + th * th / 720.0 : (1.0 - A / (2.0 * B)) / (th * th);
    const double W[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    for (int r = 0; r < 3; ++r) {
        double v = 0.0;
        for (int c = 0; c < 3; ++c) {
            double w2 = W[r * 3 + 0] * W[0 * 3 + c] + W[r * 3 + 1] * W[1 * 3 + c] + W[r * 3 + 2] * W[2 * 3 + c];
            v += ((r == c ? 1.0 : 0.0) - 0.5 * W[r * 3 + c] + D * w2) * T[c * 4 + 3];
        }
        xi[r] = v;
        xi[3 + r] = w[r];
    }
}

// The increment D of an edge from its output y and centre c:
// D(x) = R (x - c) + c + u, R = exp(omega).
__device__ void increment_from_output(const float* y, const float* c, double* D)
{
    double xi[6] = {0.0, 0.0, 0.0, y[0] * kSW, y[1] * kSW, y[2] * kSW};
    se3_exp(xi, D);
    for (int r = 0; r < 3; ++r) {
        const double Rc = D[r * 4 + 0] * c[0] + D[r * 4 + 1] * c[1] + D[r * 4 + 2] * c[2];
        D[r * 4 + 3] = (double)c[r] + y[3 + r] * kSU - Rc;
    }
}

// ---------------------------------------------------------------------------
// Sample preparation: centre, M0 (float) and label, one warp per item
// ---------------------------------------------------------------------------

__global__ void prep_kernel(Sample* __restrict__ smp, const PrepItem* __restrict__ items, int n_items)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= n_items) return;
    const PrepItem it = items[w];
    Sample* S = smp + it.sample;
    const int n = S->n;
    const float* q = S->q;
    // the centre: compensated FP32 sums per lane, combined in FP64 (a warp's
    // FP64 instruction, a conversion included, holds its DP unit as long as
    // a full one whatever the active lanes, so the per-point work stays off it)
    float s3[3] = {0.f, 0.f, 0.f}, k3[3] = {0.f, 0.f, 0.f};
    for (int k = lane; k < n; k += 32)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float y = q[3 * k + d] - k3[d];
            const float t = s3[d] + y;
            k3[d] = (t - s3[d]) - y;
            s3[d] = t;
        }
    double sx = (double)s3[0] - (double)k3[0], sy = (double)s3[1] - (double)k3[1],
           sz = (double)s3[2] - (double)k3[2];
    for (int off = 16; off > 0; off >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, off);
        sy += __shfl_xor_sync(0xffffffffu, sy, off);
        sz += __shfl_xor_sync(0xffffffffu, sz, off);
    }
    // M0 = T_j T_i^-1 one entry a lane (lanes 0-11, the operations of
    // pose_inv and pose_mul), the centre on lanes 12-14
    if (lane < 12) {
        const int r = lane >> 2, cc = lane & 3;
        const double* Ti = it.Ti0;
        const double* Tj = it.Tj0;
        double v;
        if (cc < 3) {
            v = Tj[r * 4 + 0] * Ti[cc * 4 + 0] + Tj[r * 4 + 1] * Ti[cc * 4 + 1] + Tj[r * 4 + 2] * Ti[cc * 4 + 2];
        } else {
            double iv[3];
            for (int k = 0; k < 3; ++k) iv[k] = -(Ti[0 * 4 + k] * Ti[3] + Ti[1 * 4 + k] * Ti[7] + Ti[2 * 4 + k] * Ti[11]);
            v = Tj[r * 4 + 0] * iv[0] + Tj[r * 4 + 1] * iv[1] + Tj[r * 4 + 2] * iv[2];
            v += Tj[r * 4 + 3];
        }
        S->m[lane] = (float)v;
    } else if (lane < 15) {
        const double sd = lane == 12 ? sx : lane == 13 ? sy : sz;
        S->c[lane - 12] = (float)(n > 0 ? sd / n : 0.0);
    } else if (lane == 15) {
        S->c[3] = 0.f;
    } else if (lane < 22 && !it.Ti1) {
        S->ystar[lane - 16] = 0.f;
    }
    if (lane != 0 || !it.Ti1) return;
    // training label (one lane): the increment from M0 to the converged M
    const double c[3] = {n > 0 ? sx / n : 0.0, n > 0 ? sy / n : 0.0, n > 0 ? sz / n : 0.0};
    double inv[12], M0[12];
    pose_inv(it.Ti0, inv);
    pose_mul(it.Tj0, inv, M0);
    {
        double M[12], M0inv[12], D[12], w[3], th;
        pose_inv(it.Ti1, inv);
        pose_mul(it.Tj1, inv, M);
        pose_inv(M0, M0inv);
        pose_mul(M, M0inv, D);
        so3_log(D, w, th);
        for (int r = 0; r < 3; ++r) {
            const double Rc = D[r * 4 + 0] * c[0] + D[r * 4 + 1] * c[1] + D[r * 4 + 2] * c[2];
            S->ystar[r] = (float)(w[r] / kSW);
            S->ystar[3 + r] = (float)((D[r * 4 + 3] + Rc - c[r]) / kSU);
        }
    }
}

__global__ void rebase_kernel(Sample* __restrict__ smp, int n, const float* old_p, const float* new_p,
                              const float* old_q, const float* new_q)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    smp[k].p = new_p + (smp[k].p - old_p);
    smp[k].q = new_q + (smp[k].q - old_q);
}

// ---------------------------------------------------------------------------
// Relative-pose averaging, one CTA per graph (FP64)
// ---------------------------------------------------------------------------

constexpr int kAvgThreads = 256;
constexpr int kScr = kAvgScratch;   // scratch doubles per edge (bt_ws.h)
constexpr int kScrP = 54;           // P = A^T W A, lower triangle (21)
constexpr int kScrG = 75;           // A^T W e (6)
static_assert(kScrG + 6 <= kScr, "averaging scratch per edge");

// Row and column of entry q (0..20) of a 6x6 lower triangle, row by row.
__device__ __forceinline__ void tri_rc(int q, int& r, int& c)
{
    r = 0;
    while ((r + 1) * (r + 2) / 2 <= q) ++r;
    c = q - r * (r + 1) / 2;
}

__global__ void __launch_bounds__(kAvgThreads) average_kernel(const AvgGraph* __restrict__ graphs)
{
    extern __shared__ double asm_[];
    __shared__ int s_sing;
    const AvgGraph G = graphs[blockIdx.x];
    const int N = G.N, E = G.n_edges, nf = G.n_free, n = 6 * nf, ld = n + 1;
    const int tid = threadIdx.x;
    double* sT0 = asm_;                      // [N][12]
    double* sT = sT0 + 12 * N;               // [N][12]
    double* H = sT + 12 * N;                 // [n][ld]
    double* b = H + (size_t)n * ld;          // [n]
    LdltScratch sc;                          // the solve's scratch (bt_ldlt.h)
    sc.rD = b + n;                           // [n]
    sc.colb = sc.rD + n;                     // [2n]
    sc.part = sc.colb + 2 * n;               // [256]
    int* eof = reinterpret_cast<int*>(sc.part + 256);   // [N][N]
    int* freenode = eof + N * N;             // [nf]
    sc.tab = freenode + nf;                  // [n (n + 1) / 2]
    const double Wd[6] = {1.0 / (kSU * kSU), 1.0 / (kSU * kSU), 1.0 / (kSU * kSU),
                          1.0 / (kSW * kSW), 1.0 / (kSW * kSW), 1.0 / (kSW * kSW)};
    if (tid == 0) s_sing = 0;
    for (int k = tid; k < 12 * N; k += kAvgThreads) sT0[k] = sT[k] = G.pose[k];
    for (int k = tid; k < N * N; k += kAvgThreads) eof[k] = -1;
    for (int k = tid; k < N; k += kAvgThreads)
        if (G.nodes[k].free_idx >= 0) freenode[G.nodes[k].free_idx] = k;
    __syncthreads();
    for (int e = tid; e < E; e += kAvgThreads) {
        const EdgeDev ed = G.edges[e];
        if (G.smp[e].n > 0) {
            eof[ed.i * N + ed.j] = e;
            eof[ed.j * N + ed.i] = e;
            increment_from_output(G.y + (size_t)e * kOut, G.smp[e].c, G.scratch + (size_t)e * kScr);
        }
    }
    __syncthreads();
    // 1. anchor every free node on its edge to the lowest fixed node
    for (int j = tid; j < N; j += kAvgThreads) {
        if (G.nodes[j].free_idx < 0) continue;
        for (int f = 0; f < N; ++f) {
            if (G.nodes[f].free_idx >= 0) continue;
            const int e = eof[f * N + j];
            if (e < 0) continue;
            const double* D = G.scratch + (size_t)e * kScr;
            double out[12];
            if (G.edges[e].i == f) {                       // D predicts T_j T_f^-1
                pose_mul(D, sT0 + 12 * j, out);
            } else {                                       // D predicts T_f T_j^-1
                double a[12], bq[12], Dinv[12], fi[12];
                pose_inv(sT0 + 12 * f, fi);
                pose_mul(sT0 + 12 * j, fi, a);
                pose_inv(D, Dinv);
                pose_mul(a, Dinv, bq);
                pose_mul(bq, sT0 + 12 * f, out);
            }
            for (int k = 0; k < 12; ++k) sT[12 * j + k] = out[k];
            break;
        }
    }
    __syncthreads();
    // 2. per edge: e = log(D M0 M^-1) and A = Ad(M) at the anchored poses
    for (int e = tid; e < E; e += kAvgThreads) {
        if (G.smp[e].n <= 0) continue;
        const int i = G.edges[e].i, j = G.edges[e].j;
        double* scr = G.scratch + (size_t)e * kScr;
        double inv[12], M0[12], M[12], Minv[12], t1[12], t2[12];
        pose_inv(sT0 + 12 * i, inv);
        pose_mul(sT0 + 12 * j, inv, M0);
        pose_inv(sT + 12 * i, inv);
        pose_mul(sT + 12 * j, inv, M);
        pose_inv(M, Minv);
        pose_mul(scr, M0, t1);
        pose_mul(t1, Minv, t2);
        se3_log(t2, scr + 12);
        double* A = scr + 18;
        const double tx[9] = {0.0, -M[11], M[7], M[11], 0.0, -M[3], -M[7], M[3], 0.0};
        for (int r = 0; r < 6; ++r)
            for (int c = 0; c < 6; ++c) A[r * 6 + c] = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                A[r * 6 + c] = M[r * 4 + c];
                A[(r + 3) * 6 + (c + 3)] = M[r * 4 + c];
                A[r * 6 + (c + 3)] = tx[r * 3 + 0] * M[0 * 4 + c] + tx[r * 3 + 1] * M[1 * 4 + c] +
                                     tx[r * 3 + 2] * M[2 * 4 + c];
            }
    }
    __syncthreads();
    // 3. normal equations over the free nodes (lower triangle) and right-hand
    // side.  The edge (i, j) has Jacobians J_i = -A, J_j = I on its
    // residual e (weights W): its i-side diagonal block A^T W A and its
    // gradient term A^T W e are formed once per edge, with the lanes packed
    // over (edge, entry) -- a warp's FP64 instruction takes its DP unit as
    // long whether 6 or 32 lanes are active -- then summed per node.
    for (int idx = tid; idx < E * 27; idx += kAvgThreads) {
        const int e = idx / 27, q = idx % 27;
        if (G.smp[e].n <= 0) continue;
        double* scr = G.scratch + (size_t)e * kScr;
        const double* A = scr + 18;
        double v = 0.0;
        if (q < 21) {
            int al, be;
            tri_rc(q, al, be);
            for (int g = 0; g < 6; ++g) v += A[g * 6 + al] * Wd[g] * A[g * 6 + be];
            scr[kScrP + q] = v;
        } else {
            const int al = q - 21;
            for (int g = 0; g < 6; ++g) v += A[g * 6 + al] * Wd[g] * scr[12 + g];
            scr[kScrG + al] = v;
        }
    }
    __syncthreads();
    // diagonal blocks: free node a's edges, A^T W A where a is the i side, W
    // where it is the j side
    for (int idx = tid; idx < nf * 21; idx += kAvgThreads) {
        const int f = idx / 21;
        int al, be;
        tri_rc(idx % 21, al, be);
        const int a = freenode[f];
        double v = 0.0;
        for (int m = 0; m < N; ++m) {
            const int e = m == a ? -1 : eof[a * N + m];
            if (e < 0) continue;
            if (G.edges[e].j == a) v += al == be ? Wd[al] : 0.0;
            else v += G.scratch[(size_t)e * kScr + kScrP + idx % 21];
        }
        H[(6 * f + al) * ld + 6 * f + be] = v;
    }
    // off-diagonal blocks: -A^T W (a = i) or -W A (a = j) of the edge between
    for (int idx = tid; idx < n * n; idx += kAvgThreads) {
        const int r = idx / n, c = idx % n;
        if (c > r || r / 6 == c / 6) continue;
        const int a = freenode[r / 6], al = r % 6, bn = freenode[c / 6], be = c % 6;
        double v = 0.0;
        const int e = eof[a * N + bn];
        if (e >= 0) {
            const double* A = G.scratch + (size_t)e * kScr + 18;
            if (G.edges[e].i == a) v = -A[be * 6 + al] * Wd[be];      // J_a = -A, J_b = I
            else v = -Wd[al] * A[al * 6 + be];                        // J_a = I, J_b = -A
        }
        H[r * ld + c] = v;
    }
    for (int r = tid; r < n; r += kAvgThreads) {
        const int a = freenode[r / 6], al = r % 6;
        double v = 0.0;
        for (int m = 0; m < N; ++m) {
            const int e = m == a ? -1 : eof[a * N + m];
            if (e < 0) continue;
            const double* scr = G.scratch + (size_t)e * kScr;
            if (G.edges[e].j == a) v += Wd[al] * scr[12 + al];
            else v -= scr[kScrG + al];
        }
        b[r] = v;
    }
    __syncthreads();
    // 4-5. H d = b by LDL^T with a one-column look-ahead (bt_ldlt.h); a
    // pivot that is not positive, or a solution that is not finite, leaves
    // the poses as they were
    if (n > 0) {
        unsigned long long t_unused;
        ldlt_solve(H, ld, n, b, sc, &s_sing, t_unused);
        for (int i = tid; i < n; i += kAvgThreads)
            if (!isfinite(b[i])) s_sing = 1;
        __syncthreads();
    }
    if (s_sing) {
        if (tid == 0) *G.status = 1;
        return;
    }
    // 6. T_j <- exp(d_j) T_j for the free nodes
    for (int j = tid; j < N; j += kAvgThreads) {
        const int f = G.nodes[j].free_idx;
        if (f < 0) continue;
        double E6[12], out[12];
        se3_exp(b + 6 * f, E6);
        pose_mul(E6, sT + 12 * j, out);
        for (int k = 0; k < 12; ++k) G.pose[12 * j + k] = out[k];
    }
    if (tid == 0) *G.status = 0;
}

}  // namespace

cudaError_t launch_prep(Sample* smp, const PrepItem* items, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    prep_kernel<<<(n + 7) / 8, 256, 0, s>>>(smp, items, n);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(Net net, cudaStream_t s)
{
    to_bf16_kernel<<<(kNumParams + 255) / 256, 256, 0, s>>>(net);
    return cudaGetLastError();
}

size_t forward_smem_bytes() { return Fwd::Total; }

cudaError_t launch_forward(Net net, const Sample* smp, const int* ids, int n, float* y_out, Cache* cache,
                           cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int grid = n < num_sms() ? n : num_sms();
    if (cache) {
        ForwardAttr<true>::set();
        forward_kernel<true><<<grid, kFwdThreads, Fwd::Total, s>>>(net, smp, ids, n, y_out, cache);
    } else {
        ForwardAttr<false>::set();
        forward_kernel<false><<<grid, kFwdThreads, Fwd::Total, s>>>(net, smp, ids, n, y_out, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_backward(Net net, const Sample* smp, const int* ids, int n, const Cache* cache, float* G,
                            float* loss_per, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    backward_kernel<<<n, kBwdThreads, 0, s>>>(net, smp, ids, n, cache, 1.0f / (float)n, G, loss_per);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const float* G, const float* loss_per, int n, float* grad, double* loss,
                          cudaStream_t s)
{
    reduce_kernel<<<(kNumParams + 255) / 256, 256, 0, s>>>(G, loss_per, n, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(Net net, const float* grad, float lr, float beta1, float beta2, float eps, float c1,
                        float c2, cudaStream_t s)
{
    adam_kernel<<<(kNumParams + 255) / 256, 256, 0, s>>>(net, grad, lr, beta1, beta2, eps, c1, c2);
    return cudaGetLastError();
}

size_t average_smem_bytes(int max_free, int max_N)
{
    const size_t n = 6 * (size_t)max_free;
    return sizeof(double) * (24 * (size_t)max_N + n * (n + 1) + 4 * n + 256) +
           sizeof(int) * ((size_t)max_N * max_N + max_free + n * (n + 1) / 2) + 16;
}

cudaError_t launch_average(const AvgGraph* graphs, int n_graphs, int max_free, cudaStream_t s)
{
    if (n_graphs <= 0) return cudaSuccess;
    const size_t smem = average_smem_bytes(max_free, kMaxNodes);
    static const bool attr = [] {         // once per process, thread-safe
        cudaFuncSetAttribute(average_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)average_smem_bytes(kMaxNodes - 1, kMaxNodes));
        return true;
    }();
    (void)attr;
    average_kernel<<<n_graphs, kAvgThreads, smem, s>>>(graphs);
    return cudaGetLastError();
}

cudaError_t launch_rebase(Sample* smp, int n, const float* old_p, const float* new_p, const float* old_q,
                          const float* new_q, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    rebase_kernel<<<(n + 255) / 256, 256, 0, s>>>(smp, n, old_p, new_p, old_q, new_q);
    return cudaGetLastError();
}

}  // namespace ws
}  // namespace bt
