// bt_warmstart.cu -- kernels of the learned warm start (see bt_ws.h): sample
// preparation, the set network's forward and backward passes, the gradient
// reduction, Adam, and the FP64 relative-pose averaging solve that turns the
// predicted edge increments into node poses for Gauss-Newton (Sec. IV-D).
//
// Forward pass: a persistent CTA per SM keeps the BF16 W2 (padded rows, for
// conflict-free ldmatrix) and W3 in shared memory and walks its sets in
// chunks of 64 points: layer 1 (K = 6) on the FP32 pipes, rounded to BF16
// into shared memory; the 64 x 256 x 128 contraction of layer 2 on the tensor
// cores (mma.sync m16n8k16, BF16 in, FP32 accumulate, 8 warps of 32 x 64
// tiles); bias, ReLU and a running per-channel maximum (with the row that
// holds it, first row on ties) in registers; then the 256 -> 128 -> 6 head.
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
constexpr int kChunk = 64;      // points per layer-2 tile
constexpr int kLd = 136;        // padded row length (BF16) of W2 and the h1 tile in shared memory
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

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* ptr)
{
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(ptr));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory layout of the forward kernel (byte offsets).
struct Fwd {
    static constexpr size_t W2 = 0;                                          // bf16 [256][kLd]
    static constexpr size_t H1 = W2 + 2 * (size_t)kH2 * kLd;                 // bf16 [64][kLd]
    static constexpr size_t W3 = H1 + 2 * (size_t)kChunk * kLd;              // bf16 [128][kLd3]
    static constexpr size_t W1 = W3 + ((2 * (size_t)kH3 * kLd3 + 15) / 16) * 16;   // float [128][8] + skew (w1_at)
    static constexpr size_t B2 = W1 + 4 * ((size_t)kH1 * 8 + 16);            // float [256]
    static constexpr size_t B3 = B2 + 4 * (size_t)kH2;                       // float [128]
    static constexpr size_t W4 = B3 + 4 * (size_t)kH3;                       // float [6][128]
    static constexpr size_t B4 = W4 + 4 * (size_t)kOut * kH3;                // float [8]
    static constexpr size_t G = B4 + 32;                                     // float [256]
    static constexpr size_t R = G + 4 * (size_t)kH2;                         // int [256]
    static constexpr size_t RV = R + 4 * (size_t)kH2;                        // float [2][256]
    static constexpr size_t RI = RV + 8 * (size_t)kH2;                       // int [2][256]
    static constexpr size_t H3 = RI + 8 * (size_t)kH2;                       // float [128]
    static constexpr size_t Z3 = H3 + 4 * (size_t)kH3;                       // float [128]
    static constexpr size_t MC = Z3 + 4 * (size_t)kH3;                       // float [16]: m[12], c[3]
    static constexpr size_t Total = MC + 64;
};
static_assert(Fwd::H1 % 16 == 0 && Fwd::W3 % 16 == 0 && Fwd::W1 % 16 == 0, "alignment");
static_assert(kFwdThreads == 2 * kH3 && kFwdThreads == kH2, "head mapping: two threads per layer-3 unit");

template <bool kTrain>
__global__ void __launch_bounds__(kFwdThreads, 1)
    forward_kernel(Net net, const Sample* __restrict__ smp, const int* __restrict__ ids, int n_sets,
                   float* __restrict__ y_out, Cache* __restrict__ cache)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __nv_bfloat16* sW2 = reinterpret_cast<__nv_bfloat16*>(sm + Fwd::W2);
    __nv_bfloat16* sH1 = reinterpret_cast<__nv_bfloat16*>(sm + Fwd::H1);
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
    // stage the weights once per CTA
    for (int k = tid; k < kH2 * kH1 / 8; k += kFwdThreads) {
        const int row = k >> 4, c8 = (k & 15) * 8;
        *reinterpret_cast<uint4*>(sW2 + row * kLd + c8) =
            *reinterpret_cast<const uint4*>(net.wb + bW2 + row * kH1 + c8);
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

    const int wm = warp & 1, wn = warp >> 1;     // warp tile: rows wm*32 .. +32, columns wn*64 .. +64
    __syncthreads();
    float b2[16];                                // layer-2 bias of the thread's 16 columns
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) b2[2 * nt + e] = sB2[wn * 64 + nt * 8 + 2 * (lane & 3) + e];
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
        float best[16];
        int bestr[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            best[k] = -1.f;
            bestr[k] = 0;
        }
        const int lrow = tid >> 2, q4 = tid & 3;  // layer 1: thread = (row, quarter of the 128 units)
        float pq[6];                             // the point pair of this thread's row of the chunk
        load_pair(P, Q, lrow, n, pq);
        for (int r0 = 0; r0 < n; r0 += kChunk) {
            {
                const int gr = r0 + lrow;
                float x[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (gr < n) features_from(pq, sMC, sMC + 12, x);
                uint32_t packed[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int u = q4 * 32 + 2 * k;
                    const float h0 = fmaxf(z1_unit8(sW1 + w1_at(u), x), 0.f);
                    const float h1 = fmaxf(z1_unit8(sW1 + w1_at(u + 1), x), 0.f);
                    __nv_bfloat162 b2 = __floats2bfloat162_rn(h0, h1);
                    packed[k] = *reinterpret_cast<uint32_t*>(&b2);
                }
                uint4* dst = reinterpret_cast<uint4*>(sH1 + lrow * kLd + q4 * 32);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    dst[k] = make_uint4(packed[4 * k], packed[4 * k + 1], packed[4 * k + 2], packed[4 * k + 3]);
            }
            __syncthreads();
            // the next chunk's point pair: the loads are in flight during layer 2
            load_pair(P, Q, r0 + kChunk + lrow, n, pq);
            float acc[2][8][4];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
#pragma unroll
            for (int k0 = 0; k0 < kH1; k0 += 16) {
                uint32_t a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
                    ldsm_x4(a[mt], sH1 + (wm * 32 + mt * 16 + (lane & 15)) * kLd + k0 + (lane >> 4) * 8);
#pragma unroll
                for (int np = 0; np < 4; ++np) {
                    uint32_t b[4];
                    ldsm_x4(b, sW2 + (wn * 64 + np * 16 + (lane & 7) + ((lane >> 4) << 3)) * kLd + k0 +
                                   ((lane >> 3) & 1) * 8);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma_bf16(acc[mt][2 * np], a[mt], b[0], b[1]);
                        mma_bf16(acc[mt][2 * np + 1], a[mt], b[2], b[3]);
                    }
                }
            }
            // bias, ReLU, running maximum; rows visited in increasing order
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int row = r0 + wm * 32 + mt * 16 + (lane >> 2) + 8 * h;
                    if (row < n) {
#pragma unroll
                        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const float v = fmaxf(acc[mt][nt][2 * h + e] + b2[2 * nt + e], 0.f);
                                if (v > best[2 * nt + e]) {
                                    best[2 * nt + e] = v;
                                    bestr[2 * nt + e] = row;
                                }
                            }
                    }
                }
            __syncthreads();   // the next chunk overwrites sH1
        }
        // combine the 8 lanes of each column, then the two row halves
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float v = best[k];
            int r = bestr[k];
#pragma unroll
            for (int off = 4; off < 32; off <<= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, v, off);
                const int orr = __shfl_xor_sync(0xffffffffu, r, off);
                if (ov > v || (ov == v && orr < r)) {
                    v = ov;
                    r = orr;
                }
            }
            if (lane < 4) {
                const int col = wn * 64 + (k >> 1) * 8 + 2 * lane + (k & 1);
                sRV[wm * kH2 + col] = v;
                sRI[wm * kH2 + col] = r;
            }
        }
        __syncthreads();
        {
            float v = sRV[tid];
            int r = sRI[tid];
            const float v1 = sRV[kH2 + tid];
            const int r1 = sRI[kH2 + tid];
            if (v1 > v || (v1 == v && r1 < r)) {
                v = v1;
                r = r1;
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
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int k = lane; k < n; k += 32) {
        sx += q[3 * k];
        sy += q[3 * k + 1];
        sz += q[3 * k + 2];
    }
    for (int off = 16; off > 0; off >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, off);
        sy += __shfl_xor_sync(0xffffffffu, sy, off);
        sz += __shfl_xor_sync(0xffffffffu, sz, off);
    }
    if (lane != 0) return;
    const double c[3] = {n > 0 ? sx / n : 0.0, n > 0 ? sy / n : 0.0, n > 0 ? sz / n : 0.0};
    double inv[12], M0[12];
    pose_inv(it.Ti0, inv);
    pose_mul(it.Tj0, inv, M0);
    for (int k = 0; k < 12; ++k) S->m[k] = (float)M0[k];
    for (int k = 0; k < 3; ++k) S->c[k] = (float)c[k];
    S->c[3] = 0.f;
    if (it.Ti1) {
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
    } else {
        for (int k = 0; k < 6; ++k) S->ystar[k] = 0.f;
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
constexpr int kScr = 64;        // scratch doubles per edge: D [12], e [6], A [36]

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
    // 3. normal equations over the free nodes (lower triangle) and right-hand side
    for (int idx = tid; idx < n * n; idx += kAvgThreads) {
        const int r = idx / n, c = idx % n;
        if (c > r) continue;
        const int a = freenode[r / 6], al = r % 6, bn = freenode[c / 6], be = c % 6;
        double v = 0.0;
        if (a == bn) {
            for (int m = 0; m < N; ++m) {
                const int e = m == a ? -1 : eof[a * N + m];
                if (e < 0) continue;
                if (G.edges[e].j == a) {
                    v += al == be ? Wd[al] : 0.0;
                } else {
                    const double* A = G.scratch + (size_t)e * kScr + 18;
                    for (int g = 0; g < 6; ++g) v += A[g * 6 + al] * Wd[g] * A[g * 6 + be];
                }
            }
        } else {
            const int e = eof[a * N + bn];
            if (e >= 0) {
                const double* A = G.scratch + (size_t)e * kScr + 18;
                if (G.edges[e].i == a) v = -A[be * 6 + al] * Wd[be];      // J_a = -A, J_b = I
                else v = -Wd[al] * A[al * 6 + be];                        // J_a = I, J_b = -A
            }
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
            if (G.edges[e].j == a) {
                v += Wd[al] * scr[12 + al];
            } else {
                for (int g = 0; g < 6; ++g) v -= scr[18 + g * 6 + al] * Wd[g] * scr[12 + g];
            }
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
