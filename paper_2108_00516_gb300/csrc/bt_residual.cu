// bt_residual.cu -- sm_103a kernels of the pose-graph hot path (BundleTrack,
// Sec. IV-D, Eq. 1-3): frame preparation and the residual pass.
//
//   prep_*          frame preparation: per-pixel target map (z, n) and the
//                   compacted list of valid masked source pixels (pi_D^-1).
//   residual_kernel one launch per Gauss-Newton iteration: CTAs [0, E) take
//                   one correspondence set each (Eq. 2), CTAs [E, E+T) stage
//                   one tile of source pixels in shared memory and loop over
//                   every target node (Eq. 3): association, gates,
//                   point-to-plane residual, Jacobian, Huber weight, and a
//                   deterministic reduction of the 21 + 6 unique J^T W J /
//                   J^T W r terms per (tile, target).
//
// The reduction into FP64 blocks, the solve and the update are in bt_solve.cu.
//
// Perturbations.  The library solves for right perturbations,
// T_i <- T_i exp(d_i) with d = (v, w).  This is a linear change of tangent
// coordinates (d_left = Ad_{T_i} d_right) of the left-perturbation system,
// so every Gauss-Newton iterate is the same pose as with left perturbations;
// it lets a dense pair (i -> j) contribute one block K' to (i,i), (j,j) and
// -K' to (i,j), (j,i).
//
// Association decision.  Keep / drop and the looked-up pixel are integers
// decided in single precision by the device functions of bt_assoc.cuh (fused
// multiply-adds, the hardware reciprocal, packed FP32x2 arithmetic).  Another
// single-precision evaluation -- or the exact one -- can differ from it only
// for pixels within rounding of a half-pixel edge, the image edge or a gate;
// bt_debug_associate exports the decisions so that they can be checked pixel
// by pixel.  Residual values, Jacobians and weights are FP32 as well.
#include "bt_internal.h"
#include "bt_assoc.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

namespace bt {

// ---------------------------------------------------------------------------
// K0: frame preparation
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool pixel_valid(const float* depth, const float* normals,
                                            const uint8_t* mask, int pix, float& z, float3& n)
{
    if (!mask[pix]) return false;
    z = depth[pix];
    if (!(z > 0.f) || !isfinite(z)) return false;
    n = make_float3(normals[3 * pix], normals[3 * pix + 1], normals[3 * pix + 2]);
    return isfinite(n.x) && isfinite(n.y) && isfinite(n.z);
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* total, int* sm /* >= 33 */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int w = lane < nw ? sm[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) sm[lane] = w;       // inclusive warp totals
        if (lane == nw - 1) sm[32] = w;
    }
    __syncthreads();
    const int before = warp > 0 ? sm[warp - 1] : 0;
    *total = sm[32];
    return before + x - v;
}

// 16-bit storage helpers (BF16 / FP16 as raw bits)
template <int P>
__device__ __forceinline__ unsigned short to16(float x)
{
    if constexpr (P == 1) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    else return __half_as_ushort(__float2half_rn(x));
}
template <int P>
__device__ __forceinline__ float from16(unsigned short b)
{
    if constexpr (P == 1) return __bfloat162float(__ushort_as_bfloat16(b));
    else return __half2float(__ushort_as_half(b));
}
template <int P>
__device__ __forceinline__ unsigned short nan16()
{
    return P == 1 ? (unsigned short)0x7FC0 : (unsigned short)0x7E00;
}

size_t prep_scratch_bytes(int HW)
{
    const size_t nblk = (HW + kPrepPix - 1) / kPrepPix;
    return (nblk + 1) * (sizeof(int) + sizeof(double)) + 16;
}

// Validity, count and depth sum of each block of kPrepPix pixels.
__global__ void __launch_bounds__(kThreads) prep_count_kernel(
    const float* __restrict__ depth, const float* __restrict__ normals,
    const uint8_t* __restrict__ mask, int HW, int* __restrict__ blockcnt, double* __restrict__ blocksum)
{
    __shared__ int sm[33];
    __shared__ double sz[kThreads / 32];
    const int base = blockIdx.x * kPrepPix + threadIdx.x * kPixPerThread;
    int c = 0;
    float zs = 0.f;
#pragma unroll
    for (int k = 0; k < kPixPerThread; ++k) {
        const int pix = base + k;
        if (pix < HW) {
            float z;
            float3 n;
            if (pixel_valid(depth, normals, mask, pix, z, n)) {
                ++c;
                zs += z;
            }
        }
    }
    int total;
    block_exclusive_scan(c, &total, sm);
    double dz = zs;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) dz += __shfl_xor_sync(0xffffffffu, dz, o);
    if ((threadIdx.x & 31) == 0) sz[threadIdx.x >> 5] = dz;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += sz[w];
        blockcnt[blockIdx.x] = total;
        blocksum[blockIdx.x] = t;
    }
}

// Exclusive scan of the block counts; M and the reference depth (mean valid
// depth, used by the 16-bit encodings).
__global__ void prep_scan_kernel(int* __restrict__ blockcnt, const double* __restrict__ blocksum, int nblk,
                                 int* __restrict__ out2, int* __restrict__ host_out2)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int s = 0;
        double z = 0.0;
        for (int b = 0; b < nblk; ++b) {
            const int c = blockcnt[b];
            blockcnt[b] = s;
            s += c;
            z += blocksum[b];
        }
        out2[0] = s;
        out2[1] = __float_as_int(s > 0 ? (float)(z / s) : 0.f);
        if (host_out2) {      // the host's read-back slot (mapped pinned memory)
            host_out2[0] = out2[0];
            host_out2[1] = out2[1];
        }
    }
}

// Target map of every pixel and the compacted source list of the valid ones.
template <int P>
__global__ void __launch_bounds__(kThreads) prep_write_kernel(
    const float* __restrict__ depth, const float* __restrict__ normals,
    const uint8_t* __restrict__ mask, int W, int HW, float cx, float cy, float ifx, float ify,
    const int* __restrict__ blockoff, const int* __restrict__ out2, void* __restrict__ tgt_v,
    void* __restrict__ src_p_v, void* __restrict__ src_n_v)
{
    __shared__ int sm[33];
    const int base = blockIdx.x * kPrepPix + threadIdx.x * kPixPerThread;
    const float zref = P == 0 ? 0.f : __int_as_float(out2[1]);
    bool ok[kPixPerThread];
    float zz[kPixPerThread];
    float3 nn[kPixPerThread];
    int c = 0;
#pragma unroll
    for (int k = 0; k < kPixPerThread; ++k) {
        const int pix = base + k;
        ok[k] = pix < HW && pixel_valid(depth, normals, mask, pix, zz[k], nn[k]);
        c += ok[k];
        if (pix < HW) {
            if constexpr (P == 0) {
                reinterpret_cast<float4*>(tgt_v)[pix] =
                    ok[k] ? make_float4(zz[k], nn[k].x, nn[k].y, nn[k].z) : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                ushort4 t;
                t.x = ok[k] ? to16<P>(zz[k] - zref) : nan16<P>();
                t.y = ok[k] ? to16<P>(nn[k].x) : (unsigned short)0;
                t.z = ok[k] ? to16<P>(nn[k].y) : (unsigned short)0;
                t.w = ok[k] ? to16<P>(nn[k].z) : (unsigned short)0;
                reinterpret_cast<ushort4*>(tgt_v)[pix] = t;
            }
        }
    }
    int total;
    int off = blockoff[blockIdx.x] + block_exclusive_scan(c, &total, sm);
#pragma unroll
    for (int k = 0; k < kPixPerThread; ++k) {
        if (!ok[k]) continue;
        const int pix = base + k;
        const int u = pix % W, v = pix / W;
        const float z = zz[k];
        // pi_D^-1(x): (u - cx) z / fx, (v - cy) z / fy, z
        const float px = ((float)u - cx) * z * ifx;
        const float py = ((float)v - cy) * z * ify;
        if constexpr (P == 0) {
            reinterpret_cast<float4*>(src_p_v)[off] = make_float4(px, py, z, 0.f);
            reinterpret_cast<float4*>(src_n_v)[off] = make_float4(nn[k].x, nn[k].y, nn[k].z, 0.f);
        } else {
            reinterpret_cast<ushort4*>(src_p_v)[off] = make_ushort4(to16<P>(px), to16<P>(py), to16<P>(z - zref), 0);
            reinterpret_cast<ushort4*>(src_n_v)[off] =
                make_ushort4(to16<P>(nn[k].x), to16<P>(nn[k].y), to16<P>(nn[k].z), 0);
        }
        ++off;
    }
}

cudaError_t launch_prep(const float* depth, const float* normals, const uint8_t* mask, int W, int H, float cx,
                        float cy, float ifx, float ify, int precision, void* tgt, void* src_p, void* src_n,
                        void* block_scratch, int* out2, int* host_out2, cudaStream_t s)
{
    const int HW = W * H;
    const int nblk = (HW + kPrepPix - 1) / kPrepPix;
    int* blockcnt = static_cast<int*>(block_scratch);
    double* blocksum = reinterpret_cast<double*>(
        (reinterpret_cast<uintptr_t>(blockcnt + nblk + 1) + 15) & ~static_cast<uintptr_t>(15));
    prep_count_kernel<<<nblk, kThreads, 0, s>>>(depth, normals, mask, HW, blockcnt, blocksum);
    prep_scan_kernel<<<1, 32, 0, s>>>(blockcnt, blocksum, nblk, out2, host_out2);
    if (precision == 1)
        prep_write_kernel<1><<<nblk, kThreads, 0, s>>>(depth, normals, mask, W, HW, cx, cy, ifx, ify, blockcnt, out2,
                                                       tgt, src_p, src_n);
    else if (precision == 2)
        prep_write_kernel<2><<<nblk, kThreads, 0, s>>>(depth, normals, mask, W, HW, cx, cy, ifx, ify, blockcnt, out2,
                                                       tgt, src_p, src_n);
    else
        prep_write_kernel<0><<<nblk, kThreads, 0, s>>>(depth, normals, mask, W, HW, cx, cy, ifx, ify, blockcnt, out2,
                                                       tgt, src_p, src_n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Residual pass
// ---------------------------------------------------------------------------

// Per-target constants of a tile, staged in shared memory by the CTA.
struct PairConst {
    PairK k;
    const void* tgt;
    float zref;                          // target frame's reference depth (16-bit maps)
};

__device__ __forceinline__ void fill_pair_const(const SolveArgs& a, int i, int j, PairConst& c)
{
    const NodeDev Nj = a.nodes[j];
    c.k = make_pair_k(a.xf + (size_t)(i * a.N + j) * 12, Nj.fx, Nj.fy, Nj.cx, Nj.cy, Nj.ifx, Nj.ify, Nj.W, Nj.H);
    c.tgt = Nj.tgt;
    c.zref = Nj.zref;
}

// Target-map gather: (z, nx, ny, nz) as FP32 whatever the storage.
template <int P>
__device__ __forceinline__ float4 load_target(const void* tgt, size_t idx, float zref)
{
    if constexpr (P == 0) {
        return __ldg(reinterpret_cast<const float4*>(tgt) + idx);
    } else {
        const ushort4 v = __ldg(reinterpret_cast<const ushort4*>(tgt) + idx);
        return make_float4(zref + from16<P>(v.x), from16<P>(v.y), from16<P>(v.z), from16<P>(v.w));
    }
}

template <int P>
__device__ __forceinline__ void load_source(const NodeDev& Ni, int idx, float4& p, float4& n)
{
    if constexpr (P == 0) {
        p = __ldg(reinterpret_cast<const float4*>(Ni.src_p) + idx);
        n = __ldg(reinterpret_cast<const float4*>(Ni.src_n) + idx);
    } else {
        const ushort4 a = __ldg(reinterpret_cast<const ushort4*>(Ni.src_p) + idx);
        const ushort4 b = __ldg(reinterpret_cast<const ushort4*>(Ni.src_n) + idx);
        p = make_float4(from16<P>(a.x), from16<P>(a.y), Ni.zref + from16<P>(a.z), 0.f);
        n = make_float4(from16<P>(b.x), from16<P>(b.y), from16<P>(b.z), 0.f);
    }
}

// Warp reduce-scatter of 32 values: afterwards lane l holds the warp total of
// value l (recursive halving, 31 shuffles instead of 5 x 32).
__device__ __forceinline__ float warp_transpose_reduce(float (&v)[kDenseVals], int lane)
{
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const bool upper = (lane & step) != 0;
#pragma unroll
        for (int k = 0; k < step; ++k) {
            const float send = upper ? v[k] : v[k + step];
            const float keep = upper ? v[k + step] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, step);
        }
    }
    return v[0];
}

size_t residual_smem_bytes(int N, int shape)
{
    const int nt = N > 1 ? N - 1 : 1;
    return 2 * sizeof(float4) * shape_tile(shape) + sizeof(PairConst) * kMaxNodes +
           sizeof(float) * (size_t)nt * (kShapeThreads[shape] / 32) * kDenseVals;
}

// acc[0..20] += w J J^T (upper triangle, row-major), acc[21..26] += w J r,
// acc[27] += rho, acc[28] += 1, two entries per packed FP32x2 FMA: rows
// (0,1), (2,3), (4,5) of one column share the broadcast J_b.
__device__ __forceinline__ void accumulate_pair(float (&acc)[kDenseVals], float2 J01, float2 J23, float2 J45, float w,
                                                float r, float rho)
{
    const float2 ww = make_float2(w, w);
    const float2 w01 = __fmul2_rn(J01, ww), w23 = __fmul2_rn(J23, ww), w45 = __fmul2_rn(J45, ww);
    const float J[6] = {J01.x, J01.y, J23.x, J23.y, J45.x, J45.y};
    auto f2 = [&](int lo, int hi, float2 a, float b) {
        const float2 s = __ffma2_rn(a, make_float2(b, b), make_float2(acc[lo], acc[hi]));
        acc[lo] = s.x;
        acc[hi] = s.y;
    };
    // upper-triangle index of (a, b), b >= a: (0,b) = b, (1,b) = 5 + b,
    // (2,b) = 9 + b, (3,b) = 12 + b, (4,b) = 14 + b, (5,5) = 20
    acc[0] = fmaf(w01.x, J[0], acc[0]);
#pragma unroll
    for (int b = 1; b < 6; ++b) f2(b, 5 + b, w01, J[b]);
    acc[11] = fmaf(w23.x, J[2], acc[11]);
#pragma unroll
    for (int b = 3; b < 6; ++b) f2(9 + b, 12 + b, w23, J[b]);
    acc[18] = fmaf(w45.x, J[4], acc[18]);
    f2(19, 20, w45, J[5]);
    f2(21, 22, w01, r);
    f2(23, 24, w23, r);
    f2(25, 26, w45, r);
    const float2 s = __fadd2_rn(make_float2(acc[27], acc[28]), make_float2(rho, 1.f));
    acc[27] = s.x;
    acc[28] = s.y;
}

// Pixels per thread whose target gathers are issued together, and resident
// threads per SM the residual kernels are compiled for, by storage precision
// (FP32: six 128-thread CTAs, at most 80 registers a thread; 16-bit: five).
#ifndef BT_RES_BATCH_F32
#define BT_RES_BATCH_F32 2
#endif
#ifndef BT_RES_THREADS_F32
#define BT_RES_THREADS_F32 768
#endif
constexpr int residual_batch(int P) { return P == 0 ? BT_RES_BATCH_F32 : 4; }
constexpr int residual_threads_per_sm(int P) { return P == 0 ? BT_RES_THREADS_F32 : 640; }
// The FP32 cost-only pass (no Jacobian, two sums a pixel) fits in 64
// registers without spills: 1024 resident threads a SM, more warps to hide
// the gathers (the 16-bit decodes would spill there).
constexpr int residual_threads_per_sm(int P, bool full) { return full || P != 0 ? residual_threads_per_sm(P) : 1024; }

// One tile of kT x kB source pixels of node i against every other node j.
// The work of the tile is (N-1) x kW units -- unit (jj, c) = target jj, chunk
// c of 32 x kB consecutive tile pixels -- in target-major order, and warp w
// takes the N-1 consecutive units [w (N-1), (w+1) (N-1)).  A warp keeps its
// 21 + 6 + 2 sums in registers while its units stay on one target and
// reduces them across its lanes (a 31-shuffle reduce-scatter) only when the
// target changes: about (N-1)/kW + 1 reductions per warp instead of N-1.
// Per unit each lane takes its kB pixels in batches that go through three
// phases -- projection and bounds, the target gathers of the batch (all in
// flight together), then gates, residual, Jacobian and accumulation.  The
// warp totals are parked in shared memory; one barrier at the end, then the
// (N-1) x 32 block sums of the tile are written to dpart[tile][jj] (each
// the sum, in warp order, of the warps that covered that target).
template <bool kFull, int kT, int kB, int P>
__device__ void dense_tile(const SolveArgs& a, int tile, unsigned char* dsm)
{
    constexpr int kW = kT / 32;
    constexpr int kTile = kT * kB;
    constexpr int kUnit = 32 * kB;
    constexpr int kBatch = kB < residual_batch(P) ? kB : residual_batch(P);
    constexpr int kBatches = kB / kBatch;
    static_assert(kBatch * kBatches == kB, "pixels per thread: 1 or even");
    const int N = a.N;
    const int i = a.tile_node[tile];
    const NodeDev Ni = a.nodes[i];
    const int base = (tile - Ni.tile0) * kTile;
    const int nvalid = min(kTile, Ni.M - base);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4* sp = reinterpret_cast<float4*>(dsm);
    float4* sn = sp + kTile;
    PairConst* pc = reinterpret_cast<PairConst*>(sn + kTile);
    float* red = reinterpret_cast<float*>(pc + kMaxNodes);   // [N-1][kW][32]
    for (int s = threadIdx.x; s < kTile; s += kT) {
        float4 pp = make_float4(0.f, 0.f, 0.f, 0.f), nn = pp;
        if (s < nvalid) load_source<P>(Ni, base + s, pp, nn);
        sp[s] = pp;
        sn[s] = nn;
    }
    // the source tile is frame data; the transforms below were written by
    // the predecessor (the previous update), so the wait goes here
    pdl_wait_and_release();
    if (threadIdx.x < N && threadIdx.x != i) fill_pair_const(a, i, threadIdx.x, pc[threadIdx.x]);
    __syncthreads();
    const float dmax2 = a.dmax2, cmin = a.cmin, hub = a.huber_dense;
    const int M1 = N - 1;
    int u = warp * M1;
    const int u_end = u + M1;
    while (u < u_end) {
        const int jj = u / kW;
        const int j = jj < i ? jj : jj + 1;
        const int u_stop = min(u_end, (jj + 1) * kW);
        const PairK& K = pc[j].k;
        const void* tgt = pc[j].tgt;
        const float zref = pc[j].zref;
        float acc[kDenseVals];
#pragma unroll
        for (int k = 0; k < kDenseVals; ++k) acc[k] = 0.f;
        for (; u < u_stop; ++u) {
            const int c0 = (u - jj * kW) * kUnit;
            if (c0 >= nvalid) continue;     // chunk past the last valid pixel of the tile
#pragma unroll
            for (int bb = 0; bb < kBatches; ++bb) {
                // phase 1: q = M p, nearest pixel, bounds
                float2 qxy[kBatch];
                float qz[kBatch];
                int iu[kBatch], iv[kBatch];
                bool ok[kBatch];
#pragma unroll
                for (int k = 0; k < kBatch; ++k) {
                    const int s = c0 + (bb * kBatch + k) * 32 + lane;
                    const float4 p = sp[BT_CHECK_IDX(s < kTile, kChkSourceTile, a.ctrl) ? s : 0];
                    ok[k] = assoc_project(K, p.x, p.y, p.z, qxy[k], qz[k], iu[k], iv[k]) && s < nvalid &&
                            BT_CHECK_IDX((unsigned)iu[k] < (unsigned)K.W && (unsigned)iv[k] < (unsigned)K.H,
                                         kChkGather, a.ctrl);
                }
                // phase 2: the gathers of the batch in flight together
                float4 t[kBatch];
#pragma unroll
                for (int k = 0; k < kBatch; ++k)
                    t[k] = ok[k] ? load_target<P>(tgt, (size_t)iv[k] * K.W + iu[k], zref)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                // phase 3: gates, residual, Jacobian, Huber, accumulation
#pragma unroll
                for (int k = 0; k < kBatch; ++k) {
                    if (!(ok[k] && t[k].x > 0.f)) continue;
                    float2 txy, dxy;
                    float dz;
                    if (!assoc_distance(K, iu[k], iv[k], t[k].x, qxy[k], qz[k], dmax2, txy, dxy, dz))
                        continue;
                    const float4 n = sn[c0 + (bb * kBatch + k) * 32 + lane];
                    float2 nxy;
                    float nz;
                    if (!assoc_normal(K, n.x, n.y, n.z, t[k].y, t[k].z, t[k].w, cmin, nxy, nz)) continue;
                    // accepted: r = n' . (t - q), the point-to-plane distance
                    // of Eq. 3 expressed in camera j; J~ = (n', t x n')
                    const float r = assoc_residual(nxy, nz, dxy, dz);
                    const float ar = fabsf(r);
                    const bool inl = ar <= hub;
                    const float rho = inl ? 0.5f * r * r : hub * (ar - 0.5f * hub);
                    if constexpr (kFull) {
                        const float w = inl ? 1.f : hub * rcp_approx(ar);
                        const float tz = t[k].x;
                        const float2 J23 = make_float2(nz, fmaf(txy.y, nz, -tz * nxy.y));
                        const float2 J45 = make_float2(fmaf(tz, nxy.x, -txy.x * nz), fmaf(txy.x, nxy.y, -txy.y * nxy.x));
                        accumulate_pair(acc, nxy, J23, J45, w, r, rho);
                    } else {
                        const float2 s = __fadd2_rn(make_float2(acc[27], acc[28]), make_float2(rho, 1.f));
                        acc[27] = s.x;
                        acc[28] = s.y;
                    }
                }
            }
        }
        float* slot = red + ((size_t)(BT_CHECK_IDX(jj < M1 && warp < kW, kChkRedSlot, a.ctrl) ? jj : 0) * kW + warp) *
                                kDenseVals;
        if constexpr (kFull) {
            slot[lane] = warp_transpose_reduce(acc, lane);
        } else {
            float c0 = acc[27], c1 = acc[28];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                c0 += __shfl_xor_sync(0xffffffffu, c0, o);
                c1 += __shfl_xor_sync(0xffffffffu, c1, o);
            }
            if (lane == 0) {
                slot[27] = c0;
                slot[28] = c1;
            }
        }
    }
    __syncthreads();
    const int nout = M1 * kDenseVals;
    for (int o = threadIdx.x; o < nout; o += kT) {
        const int jj = o / kDenseVals, v = o % kDenseVals;
        if (!kFull && v != 27 && v != 28) continue;
        // warps that covered target jj: units [jj kW, (jj+1) kW), warp = unit / (N-1)
        const int w0 = (jj * kW) / M1, w1 = ((jj + 1) * kW - 1) / M1;
        float s = 0.f;
        if constexpr (P == 0) {
            for (int w = w0; w <= w1; ++w) s += red[((size_t)jj * kW + w) * kDenseVals + v];
        } else {
            // compensated (Kahan) sum of the warps' block sums
            float cmp = 0.f;
            for (int w = w0; w <= w1; ++w) {
                const float y = red[((size_t)jj * kW + w) * kDenseVals + v] - cmp;
                const float t2 = s + y;
                cmp = (t2 - s) - y;
                s = t2;
            }
        }
        if (BT_CHECK_IDX(tile < a.n_tiles && jj < M1, kChkOutput, a.ctrl))
            a.dpart[((size_t)tile * M1 + jj) * kDenseVals + v] = s;
    }
}

// Sparse term of one correspondence set (Eq. 2): e = T_i^-1 p_m - T_j^-1 p_n
// in the object frame, Huber weight from ||e||, and the 39 moments from which
// the right-perturbation blocks are rebuilt in FP64:
//   [0] sum w  [1..3] sum w a  [4..6] sum w b  [7..12] sum w a a^T (xx xy xz yy yz zz)
//   [13..18] sum w b b^T  [19..27] sum w b a^T (row-major)  [28..30] sum w e
//   [31..33] sum w a x e  [34..36] sum w b x e  [37] sum rho  [38] count
template <bool kFull>
__device__ void sparse_edge(const SolveArgs& a, int e)
{
    __shared__ float sred[kThreads / 32][kSparseVals];
    const EdgeDev E = a.edges[e];
    float Ti[12], Tj[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        Ti[k] = a.xinv[E.i * 12 + k];
        Tj[k] = a.xinv[E.j * 12 + k];
    }
    const float hub = a.huber_sparse;
    float acc[kSparseVals];
#pragma unroll
    for (int k = 0; k < kSparseVals; ++k) acc[k] = 0.f;
    for (int k = threadIdx.x; k < E.count; k += blockDim.x) {
        const float pmx = __ldg(E.pa + 3 * k), pmy = __ldg(E.pa + 3 * k + 1), pmz = __ldg(E.pa + 3 * k + 2);
        const float pnx = __ldg(E.pb + 3 * k), pny = __ldg(E.pb + 3 * k + 1), pnz = __ldg(E.pb + 3 * k + 2);
        const float ax = fmaf(Ti[0], pmx, fmaf(Ti[1], pmy, fmaf(Ti[2], pmz, Ti[3])));
        const float ay = fmaf(Ti[4], pmx, fmaf(Ti[5], pmy, fmaf(Ti[6], pmz, Ti[7])));
        const float az = fmaf(Ti[8], pmx, fmaf(Ti[9], pmy, fmaf(Ti[10], pmz, Ti[11])));
        const float bx = fmaf(Tj[0], pnx, fmaf(Tj[1], pny, fmaf(Tj[2], pnz, Tj[3])));
        const float by = fmaf(Tj[4], pnx, fmaf(Tj[5], pny, fmaf(Tj[6], pnz, Tj[7])));
        const float bz = fmaf(Tj[8], pnx, fmaf(Tj[9], pny, fmaf(Tj[10], pnz, Tj[11])));
        const float ex = ax - bx, ey = ay - by, ez = az - bz;
        const float ne = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
        const bool inl = ne <= hub;
        acc[37] += inl ? 0.5f * ne * ne : hub * (ne - 0.5f * hub);
        acc[38] += 1.f;
        if constexpr (kFull) {
            const float w = inl ? 1.f : hub / ne;
            const float wax = w * ax, way = w * ay, waz = w * az;
            const float wbx = w * bx, wby = w * by, wbz = w * bz;
            acc[0] += w;
            acc[1] += wax; acc[2] += way; acc[3] += waz;
            acc[4] += wbx; acc[5] += wby; acc[6] += wbz;
            acc[7] = fmaf(wax, ax, acc[7]);  acc[8] = fmaf(wax, ay, acc[8]);  acc[9] = fmaf(wax, az, acc[9]);
            acc[10] = fmaf(way, ay, acc[10]); acc[11] = fmaf(way, az, acc[11]); acc[12] = fmaf(waz, az, acc[12]);
            acc[13] = fmaf(wbx, bx, acc[13]); acc[14] = fmaf(wbx, by, acc[14]); acc[15] = fmaf(wbx, bz, acc[15]);
            acc[16] = fmaf(wby, by, acc[16]); acc[17] = fmaf(wby, bz, acc[17]); acc[18] = fmaf(wbz, bz, acc[18]);
            acc[19] = fmaf(wbx, ax, acc[19]); acc[20] = fmaf(wbx, ay, acc[20]); acc[21] = fmaf(wbx, az, acc[21]);
            acc[22] = fmaf(wby, ax, acc[22]); acc[23] = fmaf(wby, ay, acc[23]); acc[24] = fmaf(wby, az, acc[24]);
            acc[25] = fmaf(wbz, ax, acc[25]); acc[26] = fmaf(wbz, ay, acc[26]); acc[27] = fmaf(wbz, az, acc[27]);
            const float wex = w * ex, wey = w * ey, wez = w * ez;
            acc[28] += wex; acc[29] += wey; acc[30] += wez;
            acc[31] = fmaf(ay, wez, fmaf(-az, wey, acc[31]));
            acc[32] = fmaf(az, wex, fmaf(-ax, wez, acc[32]));
            acc[33] = fmaf(ax, wey, fmaf(-ay, wex, acc[33]));
            acc[34] = fmaf(by, wez, fmaf(-bz, wey, acc[34]));
            acc[35] = fmaf(bz, wex, fmaf(-bx, wez, acc[35]));
            acc[36] = fmaf(bx, wey, fmaf(-by, wex, acc[36]));
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kSparseVals; ++k) {
        if (!kFull && k < 37) continue;
        float v = acc[k];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sred[warp][k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kSparseVals; k += blockDim.x) {   // blocks of 32 threads too
        if (!kFull && k < 37) continue;
        if (!BT_CHECK_IDX(e < a.n_edges, kChkOutput, a.ctrl)) continue;
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w][k];
        a.spart[(size_t)e * kSparseVals + k] = s;
    }
}


template <bool kFull, int kT, int kB, int P>
__global__ void __launch_bounds__(kT, residual_threads_per_sm(P, kFull) / kT) residual_kernel(SolveArgs a)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    if ((int)blockIdx.x < a.n_edges) {
        pdl_wait_and_release();
        sparse_edge<kFull>(a, blockIdx.x);
    } else {
        dense_tile<kFull, kT, kB, P>(a, blockIdx.x - a.n_edges, dsm);   // waits after staging its tile
    }
}

// Batched residual pass: CTA b takes work item work[b] = (graph, item).
template <bool kFull, int kT, int kB, int P>
__global__ void __launch_bounds__(kT, residual_threads_per_sm(P, kFull) / kT) batch_residual_kernel(const SolveArgs* __restrict__ args,
                                                                       const int2* __restrict__ work)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ SolveArgs sa;
    const int2 w = work[blockIdx.x];     // the work list and arguments: written before the solve
    if (threadIdx.x == 0) sa = args[w.x];
    __syncthreads();
    if (w.y < sa.n_edges) {
        pdl_wait_and_release();
        sparse_edge<kFull>(sa, w.y);
    } else
        dense_tile<kFull, kT, kB, P>(sa, w.y - sa.n_edges, dsm);
}

// Diagnostic export of the association of the ordered pair (i -> j): one
// thread per source entry, the same decision functions and the same target
// gather as dense_tile, out[s] = target pixel or -1.
template <int P>
__global__ void __launch_bounds__(kThreads) assoc_debug_kernel(SolveArgs a, int i, int j, int* __restrict__ out)
{
    pdl_wait_and_release();
    __shared__ PairConst pc;
    if (threadIdx.x == 0) fill_pair_const(a, i, j, pc);
    __syncthreads();
    const NodeDev Ni = a.nodes[i];
    const PairK& K = pc.k;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < Ni.M; s += gridDim.x * blockDim.x) {
        float4 p, n;
        load_source<P>(Ni, s, p, n);
        float2 qxy;
        float qz;
        int iu, iv;
        int res = -1;
        if (assoc_project(K, p.x, p.y, p.z, qxy, qz, iu, iv)) {
            const float4 t = load_target<P>(pc.tgt, (size_t)iv * K.W + iu, pc.zref);
            float2 txy, dxy, nxy;
            float dz, nz;
            if (t.x > 0.f && assoc_distance(K, iu, iv, t.x, qxy, qz, a.dmax2, txy, dxy, dz) &&
                assoc_normal(K, n.x, n.y, n.z, t.y, t.z, t.w, a.cmin, nxy, nz))
                res = iv * K.W + iu;
        }
        out[s] = res;
    }
}

cudaError_t launch_assoc_debug(const SolveArgs& a, int i, int j, int M, int* out, cudaStream_t s)
{
    const int grid = std::max(1, std::min((M + kThreads - 1) / kThreads, 4096));
    if (a.precision == 1) return launch_chained(assoc_debug_kernel<1>, dim3(grid), dim3(kThreads), 0, s, a, i, j, out);
    if (a.precision == 2) return launch_chained(assoc_debug_kernel<2>, dim3(grid), dim3(kThreads), 0, s, a, i, j, out);
    return launch_chained(assoc_debug_kernel<0>, dim3(grid), dim3(kThreads), 0, s, a, i, j, out);
}

template <int S, int P>
static void set_residual_attrs_p()
{
    constexpr int kT = kShapeThreads[S], kB = kShapePix[S];
    const int mx = (int)residual_smem_bytes(kMaxNodes, S);
    cudaFuncSetAttribute(residual_kernel<true, kT, kB, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(residual_kernel<false, kT, kB, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(batch_residual_kernel<true, kT, kB, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(batch_residual_kernel<false, kT, kB, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

template <int S>
static void set_residual_attrs()
{
    set_residual_attrs_p<S, 0>();
    set_residual_attrs_p<S, 1>();
    set_residual_attrs_p<S, 2>();
}

// Once per process (a function-local static: thread-safe initialisation).
static void ensure_residual_attrs()
{
    static const bool done = [] {
        set_residual_attrs<0>();
        set_residual_attrs<1>();
        set_residual_attrs<2>();
        set_residual_attrs<3>();
        set_residual_attrs<4>();
        set_residual_attrs<5>();
        return true;
    }();
    (void)done;
}

template <int S, int P>
static cudaError_t launch_residual_shape(const SolveArgs& a, bool full, int grid, size_t smem, cudaStream_t s)
{
    constexpr int kT = kShapeThreads[S], kB = kShapePix[S];
    if (full) return launch_chained(residual_kernel<true, kT, kB, P>, dim3(grid), dim3(kT), smem, s, a);
    return launch_chained(residual_kernel<false, kT, kB, P>, dim3(grid), dim3(kT), smem, s, a);
}

template <int S>
static cudaError_t launch_residual_s(const SolveArgs& a, bool full, int grid, size_t smem, cudaStream_t s)
{
    if (a.precision == 1) return launch_residual_shape<S, 1>(a, full, grid, smem, s);
    if (a.precision == 2) return launch_residual_shape<S, 2>(a, full, grid, smem, s);
    return launch_residual_shape<S, 0>(a, full, grid, smem, s);
}

cudaError_t launch_residual(const SolveArgs& a, bool full, cudaStream_t s, int shape)
{
    ensure_residual_attrs();
    const int grid = a.n_edges + a.n_tiles;
    if (grid == 0) return cudaSuccess;
    const size_t smem = residual_smem_bytes(a.N, shape);
    switch (shape) {
    case 1: return launch_residual_s<1>(a, full, grid, smem, s);
    case 2: return launch_residual_s<2>(a, full, grid, smem, s);
    case 3: return launch_residual_s<3>(a, full, grid, smem, s);
    case 4: return launch_residual_s<4>(a, full, grid, smem, s);
    case 5: return launch_residual_s<5>(a, full, grid, smem, s);
    default: return launch_residual_s<0>(a, full, grid, smem, s);
    }
}

template <int S, int P>
static cudaError_t launch_batch_residual_shape(const SolveArgs* args, const int2* work, int n, size_t smem,
                                               bool full, cudaStream_t s)
{
    constexpr int kT = kShapeThreads[S], kB = kShapePix[S];
    if (full) return launch_chained(batch_residual_kernel<true, kT, kB, P>, dim3(n), dim3(kT), smem, s, args, work);
    return launch_chained(batch_residual_kernel<false, kT, kB, P>, dim3(n), dim3(kT), smem, s, args, work);
}

template <int S>
static cudaError_t launch_batch_residual_s(const SolveArgs* args, const int2* work, int n, size_t smem, bool full,
                                           int precision, cudaStream_t s)
{
    if (precision == 1) return launch_batch_residual_shape<S, 1>(args, work, n, smem, full, s);
    if (precision == 2) return launch_batch_residual_shape<S, 2>(args, work, n, smem, full, s);
    return launch_batch_residual_shape<S, 0>(args, work, n, smem, full, s);
}

cudaError_t launch_batch_residual(const SolveArgs* args_dev, const int2* work_res, int n_work, int max_N, bool full,
                                  int shape, int precision, cudaStream_t s)
{
    ensure_residual_attrs();
    if (n_work == 0) return cudaSuccess;
    const size_t smem = residual_smem_bytes(max_N, shape);
    switch (shape) {
    case 1: return launch_batch_residual_s<1>(args_dev, work_res, n_work, smem, full, precision, s);
    case 2: return launch_batch_residual_s<2>(args_dev, work_res, n_work, smem, full, precision, s);
    case 3: return launch_batch_residual_s<3>(args_dev, work_res, n_work, smem, full, precision, s);
    case 4: return launch_batch_residual_s<4>(args_dev, work_res, n_work, smem, full, precision, s);
    case 5: return launch_batch_residual_s<5>(args_dev, work_res, n_work, smem, full, precision, s);
    default: return launch_batch_residual_s<0>(args_dev, work_res, n_work, smem, full, precision, s);
    }
}

void prepare_residual_attributes() { ensure_residual_attrs(); }

}  // namespace bt
