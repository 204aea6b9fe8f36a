// bt_kernels.cu -- sm_103a kernels of the pose-graph hot path (BundleTrack,
// Sec. IV-D, Eq. 1-3).
//
//   prep_*          frame preparation: per-pixel target map (z, n) and the
//                   compacted list of valid masked source pixels (pi_D^-1).
//   residual_kernel one launch per Gauss-Newton iteration: CTAs [0, E) take
//                   one correspondence set each (Eq. 2), CTAs [E, E+T) one
//                   tile of 1024 source pixels each and loop over every target
//                   node (Eq. 3): association, gates, point-to-plane residual,
//                   Jacobian, Huber weight, and a deterministic block
//                   reduction of the 21 + 6 unique J^T W J / J^T W r terms.
//   reduce_kernel   one CTA per ordered pair / correspondence set turns the
//                   FP32 partials into FP64 6x6 blocks; the last CTA to finish
//                   assembles the normal equations over the free nodes, runs
//                   the FP64 Cholesky solve and the FP64 se(3) update.
//
// Perturbations.  The library solves for right perturbations,
// T_i <- T_i exp(d_i) with d = (v, w).  This is a linear change of tangent
// coordinates (d_left = Ad_{T_i} d_right) of the left-perturbation system,
// so every Gauss-Newton iterate is the same pose as with left perturbations;
// it lets a dense pair (i -> j) contribute one block K' to (i,i), (j,j) and
// -K' to (i,j), (j,i).
//
// Association decision.  Keep / drop and the looked-up pixel are integers
// decided in IEEE single precision with the operation order below and no
// contraction into FMA (__fmul_rn / __fadd_rn / __frcp_rn), so that the same
// single-precision inputs always give the same decisions as any other
// implementation that follows the same specification.  Residual values,
// Jacobians and weights use ordinary FP32 arithmetic.
#include "bt_internal.h"

#include <cuda_runtime.h>
#include <math.h>

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

__global__ void __launch_bounds__(kThreads) prep_count_kernel(
    const float* __restrict__ depth, const float* __restrict__ normals,
    const uint8_t* __restrict__ mask, int HW, float4* __restrict__ tgt, int* __restrict__ blockcnt)
{
    __shared__ int sm[33];
    const int base = blockIdx.x * kPrepPix + threadIdx.x * kPixPerThread;
    int c = 0;
#pragma unroll
    for (int k = 0; k < kPixPerThread; ++k) {
        const int pix = base + k;
        if (pix < HW) {
            float z;
            float3 n;
            const bool ok = pixel_valid(depth, normals, mask, pix, z, n);
            tgt[pix] = ok ? make_float4(z, n.x, n.y, n.z) : make_float4(0.f, 0.f, 0.f, 0.f);
            c += ok;
        }
    }
    int total;
    block_exclusive_scan(c, &total, sm);
    if (threadIdx.x == 0) blockcnt[blockIdx.x] = total;
}

__global__ void prep_scan_kernel(int* __restrict__ blockcnt, int nblk, int* __restrict__ M_out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int s = 0;
        for (int b = 0; b < nblk; ++b) {
            const int c = blockcnt[b];
            blockcnt[b] = s;
            s += c;
        }
        *M_out = s;
    }
}

__global__ void __launch_bounds__(kThreads) prep_write_kernel(
    const float* __restrict__ depth, const float* __restrict__ normals,
    const uint8_t* __restrict__ mask, int W, int HW, float cx, float cy, float ifx, float ify,
    const int* __restrict__ blockoff, float4* __restrict__ src_p, float4* __restrict__ src_n)
{
    __shared__ int sm[33];
    const int base = blockIdx.x * kPrepPix + threadIdx.x * kPixPerThread;
    bool ok[kPixPerThread];
    float zz[kPixPerThread];
    float3 nn[kPixPerThread];
    int c = 0;
#pragma unroll
    for (int k = 0; k < kPixPerThread; ++k) {
        const int pix = base + k;
        ok[k] = pix < HW && pixel_valid(depth, normals, mask, pix, zz[k], nn[k]);
        c += ok[k];
    }
    int total;
    int off = blockoff[blockIdx.x] + block_exclusive_scan(c, &total, sm);
#pragma unroll
    for (int k = 0; k < kPixPerThread; ++k) {
        if (!ok[k]) continue;
        const int pix = base + k;
        const int u = pix % W, v = pix / W;
        const float z = zz[k];
        // pi_D^-1(x): ((u - cx) z) * (1/fx), ((v - cy) z) * (1/fy), z
        const float px = __fmul_rn(__fmul_rn(__fsub_rn((float)u, cx), z), ifx);
        const float py = __fmul_rn(__fmul_rn(__fsub_rn((float)v, cy), z), ify);
        src_p[off] = make_float4(px, py, z, 0.f);
        src_n[off] = make_float4(nn[k].x, nn[k].y, nn[k].z, 0.f);
        ++off;
    }
}

cudaError_t launch_prep(const float* depth, const float* normals, const uint8_t* mask, int W, int H,
                        float cx, float cy, float ifx, float ify, float4* tgt, float4* src_p,
                        float4* src_n, int* block_scratch, int* M_dev, cudaStream_t s)
{
    const int HW = W * H;
    const int nblk = (HW + kPrepPix - 1) / kPrepPix;
    prep_count_kernel<<<nblk, kThreads, 0, s>>>(depth, normals, mask, HW, tgt, block_scratch);
    prep_scan_kernel<<<1, 32, 0, s>>>(block_scratch, nblk, M_dev);
    prep_write_kernel<<<nblk, kThreads, 0, s>>>(depth, normals, mask, W, HW, cx, cy, ifx, ify,
                                                block_scratch, src_p, src_n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 rigid-transform helpers (3x4 row-major), no FMA contraction so that the
// single-precision copies of M = T_j T_i^-1 are reproducible bit for bit.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void pose_inv_d(const double* T, double* out)
{
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c) out[r * 4 + c] = T[c * 4 + r];
        out[r * 4 + 3] = -__dadd_rn(__dadd_rn(__dmul_rn(T[0 * 4 + r], T[3]), __dmul_rn(T[1 * 4 + r], T[7])),
                                    __dmul_rn(T[2 * 4 + r], T[11]));
    }
}

__device__ __forceinline__ void pose_mul_d(const double* A, const double* B, double* C)
{
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double s = __dadd_rn(__dadd_rn(__dmul_rn(A[r * 4 + 0], B[0 * 4 + c]), __dmul_rn(A[r * 4 + 1], B[1 * 4 + c])),
                                 __dmul_rn(A[r * 4 + 2], B[2 * 4 + c]));
            if (c == 3) s = __dadd_rn(s, A[r * 4 + 3]);
            C[r * 4 + c] = s;
        }
    }
}

// Writes xf[i*N+j] = float(T_j T_i^-1) and xinv[i] = float(T_i^-1) for the
// threads' share of pairs; `pose` may be read through L1 (written by this CTA
// or by an earlier kernel).
__device__ void write_xforms(const SolveArgs& a, int tid, int nthreads)
{
    const int N = a.N;
    for (int id = tid; id < N * N; id += nthreads) {
        const int i = id / N, j = id % N;
        double Ti[12], Tj[12], Tinv[12], M[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            Ti[k] = a.pose[i * 12 + k];
            Tj[k] = a.pose[j * 12 + k];
        }
        pose_inv_d(Ti, Tinv);
        pose_mul_d(Tj, Tinv, M);
#pragma unroll
        for (int k = 0; k < 12; ++k) a.xf[id * 12 + k] = __double2float_rn(M[k]);
        if (j == 0) {
#pragma unroll
            for (int k = 0; k < 12; ++k) a.xinv[i * 12 + k] = __double2float_rn(Tinv[k]);
        }
    }
}

__global__ void xform_kernel(SolveArgs a) { write_xforms(a, threadIdx.x, blockDim.x); }

cudaError_t launch_xforms(const SolveArgs& a, cudaStream_t s)
{
    xform_kernel<<<1, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Residual pass
// ---------------------------------------------------------------------------

struct PairConst {
    float m[12];                         // camera i -> camera j (single)
    float fx, fy, cx, cy, ifx, ify, Wf, Hf;
    int W, pad;
    const float4* tgt;
};

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

// One dense pixel-pair: association (Eq. 3), gates, residual, Jacobian and the
// Huber-weighted accumulation into acc (full) or cost/count only.
template <bool kFull>
__device__ __forceinline__ void pixel_pair(const float4 p, const float4 n, const PairConst& c,
                                           float dmax2, float cmin, float hub, float (&acc)[kDenseVals])
{
    // T_j T_i^-1 p
    const float qx = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.m[0], p.x), __fmul_rn(c.m[1], p.y)), __fmul_rn(c.m[2], p.z)), c.m[3]);
    const float qy = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.m[4], p.x), __fmul_rn(c.m[5], p.y)), __fmul_rn(c.m[6], p.z)), c.m[7]);
    const float qz = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.m[8], p.x), __fmul_rn(c.m[9], p.y)), __fmul_rn(c.m[10], p.z)), c.m[11]);
    if (!(qz > 0.f)) return;
    // pi(.) and the nearest pixel
    const float rz = __frcp_rn(qz);
    const float uh = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(c.fx, qx), rz), c.cx), 0.5f);
    const float vh = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(c.fy, qy), rz), c.cy), 0.5f);
    if (!(uh >= 0.f && uh < c.Wf && vh >= 0.f && vh < c.Hf)) return;
    const int iu = (int)floorf(uh), iv = (int)floorf(vh);
    const float4 t = __ldg(c.tgt + (size_t)iv * c.W + iu);
    if (!(t.x > 0.f)) return;
    // pi_D^-1 at the looked-up pixel (camera j)
    const float tx = __fmul_rn(__fmul_rn(__fsub_rn((float)iu, c.cx), t.x), c.ifx);
    const float ty = __fmul_rn(__fmul_rn(__fsub_rn((float)iv, c.cy), t.x), c.ify);
    const float tz = t.x;
    const float dx = __fsub_rn(tx, qx), dy = __fsub_rn(ty, qy), dz = __fsub_rn(tz, qz);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    if (!(d2 <= dmax2)) return;
    // source normal in camera j, angle gate against the target normal
    const float nx = __fadd_rn(__fadd_rn(__fmul_rn(c.m[0], n.x), __fmul_rn(c.m[1], n.y)), __fmul_rn(c.m[2], n.z));
    const float ny = __fadd_rn(__fadd_rn(__fmul_rn(c.m[4], n.x), __fmul_rn(c.m[5], n.y)), __fmul_rn(c.m[6], n.z));
    const float nz = __fadd_rn(__fadd_rn(__fmul_rn(c.m[8], n.x), __fmul_rn(c.m[9], n.y)), __fmul_rn(c.m[10], n.z));
    const float cs = __fadd_rn(__fadd_rn(__fmul_rn(nx, t.y), __fmul_rn(ny, t.z)), __fmul_rn(nz, t.w));
    if (!(cs >= cmin)) return;
    // accepted: r = n_j . (q - T_j T_i^-1 p), the point-to-plane distance of Eq. 3
    // expressed in camera j; J~ = (n_j, q x n_j)
    const float r = fmaf(nx, dx, fmaf(ny, dy, nz * dz));
    const float ar = fabsf(r);
    const bool inl = ar <= hub;
    const float rho = inl ? 0.5f * r * r : hub * (ar - 0.5f * hub);
    if constexpr (kFull) {
        const float w = inl ? 1.f : hub / ar;
        const float J[6] = {nx, ny, nz, fmaf(ty, nz, -tz * ny), fmaf(tz, nx, -tx * nz), fmaf(tx, ny, -ty * nx)};
        float wJ[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) wJ[k] = w * J[k];
        int idx = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b) {
                acc[idx] = fmaf(wJ[a], J[b], acc[idx]);
                ++idx;
            }
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[21 + k] = fmaf(wJ[k], r, acc[21 + k]);
    }
    acc[27] += rho;
    acc[28] += 1.f;
}

template <bool kFull>
__device__ void dense_tile(const SolveArgs& a, int tile)
{
    __shared__ PairConst pc[kMaxNodes];
    __shared__ float red[kThreads / 32][kDenseVals];
    const int N = a.N;
    const int i = a.tile_node[tile];
    const NodeDev Ni = a.nodes[i];
    const int base = (tile - Ni.tile0) * kTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < N && threadIdx.x != i) {
        const int j = threadIdx.x;
        const NodeDev Nj = a.nodes[j];
        PairConst& c = pc[j];
#pragma unroll
        for (int k = 0; k < 12; ++k) c.m[k] = a.xf[(i * N + j) * 12 + k];
        c.fx = Nj.fx; c.fy = Nj.fy; c.cx = Nj.cx; c.cy = Nj.cy; c.ifx = Nj.ifx; c.ify = Nj.ify;
        c.Wf = (float)Nj.W; c.Hf = (float)Nj.H; c.W = Nj.W; c.tgt = Nj.tgt;
    }
    float4 P[kPixPerThread], Nn[kPixPerThread];
    bool ok[kPixPerThread];
#pragma unroll
    for (int k = 0; k < kPixPerThread; ++k) {
        const int idx = base + k * kThreads + threadIdx.x;
        ok[k] = idx < Ni.M;
        P[k] = ok[k] ? __ldg(Ni.src_p + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
        Nn[k] = ok[k] ? __ldg(Ni.src_n + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const float dmax2 = a.dmax2, cmin = a.cmin, hub = a.huber_dense;
    for (int jj = 0; jj < N - 1; ++jj) {
        const int j = jj < i ? jj : jj + 1;
        float acc[kDenseVals];
#pragma unroll
        for (int k = 0; k < kDenseVals; ++k) acc[k] = 0.f;
#pragma unroll
        for (int k = 0; k < kPixPerThread; ++k)
            if (ok[k]) pixel_pair<kFull>(P[k], Nn[k], pc[j], dmax2, cmin, hub, acc);
        float* out = a.dpart + ((size_t)tile * (N - 1) + jj) * kDenseVals;
        if constexpr (kFull) {
            const float v = warp_transpose_reduce(acc, lane);
            red[warp][lane] = v;
            __syncthreads();
            if (threadIdx.x < kDenseVals) {
                float s = 0.f;
#pragma unroll
                for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
                out[threadIdx.x] = s;
            }
            __syncthreads();
        } else {
            float c0 = acc[27], c1 = acc[28];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                c0 += __shfl_xor_sync(0xffffffffu, c0, o);
                c1 += __shfl_xor_sync(0xffffffffu, c1, o);
            }
            if (lane == 0) {
                red[warp][0] = c0;
                red[warp][1] = c1;
            }
            __syncthreads();
            if (threadIdx.x < 2) {
                float s = 0.f;
#pragma unroll
                for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
                out[27 + threadIdx.x] = s;
            }
            __syncthreads();
        }
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
    for (int k = threadIdx.x; k < E.count; k += kThreads) {
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
    if (threadIdx.x < kSparseVals && (kFull || threadIdx.x >= 37)) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) s += sred[w][threadIdx.x];
        a.spart[(size_t)e * kSparseVals + threadIdx.x] = s;
    }
}

template <bool kFull>
__global__ void __launch_bounds__(kThreads, 2) residual_kernel(SolveArgs a)
{
    if ((int)blockIdx.x < a.n_edges)
        sparse_edge<kFull>(a, blockIdx.x);
    else
        dense_tile<kFull>(a, blockIdx.x - a.n_edges);
}

cudaError_t launch_residual(const SolveArgs& a, bool full, cudaStream_t s)
{
    const int grid = a.n_edges + a.n_tiles;
    if (grid == 0) return cudaSuccess;
    if (full)
        residual_kernel<true><<<grid, kThreads, 0, s>>>(a);
    else
        residual_kernel<false><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reduce / assemble / solve / update
// ---------------------------------------------------------------------------

__device__ __forceinline__ int sym_idx(int r, int c)
{
    // index of (min, max) in the row-major upper triangle of a 6x6 matrix
    const int a = r < c ? r : c, b = r < c ? c : r;
    return a * 6 - (a * (a - 1)) / 2 + (b - a);
}

// Second stage of a dense ordered pair p = (i -> j): FP64 sum of the tile
// partials, then K' = Ad_{T_j}^T K Ad_{T_j}, g' = Ad_{T_j}^T g~ (camera-j
// left-perturbation block -> right perturbations), times lambda_2.
template <bool kFull>
__device__ void reduce_pair(const SolveArgs& a, int p, double* sm)
{
    const int N = a.N;
    const int i = p / (N - 1), jj = p % (N - 1);
    const int j = jj < i ? jj : jj + 1;
    const NodeDev Ni = a.nodes[i];
    const int v = threadIdx.x & 31, grp = threadIdx.x >> 5;
    double s = 0.0;
    if (kFull || v == 27 || v == 28)
        for (int t = Ni.tile0 + grp; t < Ni.tile0 + Ni.ntiles; t += kThreads / 32)
            s += (double)a.dpart[((size_t)t * (N - 1) + jj) * kDenseVals + v];
    sm[grp * 32 + v] = s;
    __syncthreads();
    double* tot = sm + 256;     // 32
    double* K = sm + 288;       // 36
    double* Ad = sm + 324;      // 36
    double* KA = sm + 360;      // 36
    if (threadIdx.x < 32) {
        double t = 0.0;
#pragma unroll
        for (int g = 0; g < kThreads / 32; ++g) t += sm[g * 32 + threadIdx.x];
        tot[threadIdx.x] = t;
    }
    __syncthreads();
    double* out = a.pairblk + (size_t)p * kPairBlk;
    const double lam = a.lambda_dense;
    if (!kFull) {
        if (threadIdx.x == 0) {
            out[27] = lam * tot[27];
            out[28] = tot[28];
        }
        return;
    }
    if (threadIdx.x < 36) {
        const int r = threadIdx.x / 6, c = threadIdx.x % 6;
        K[threadIdx.x] = tot[sym_idx(r, c)];
        // Ad_T = [[R, [t]x R], [0, R]] for T = T_j
        const double* T = a.pose + j * 12;
        double val;
        if (r >= 3 && c < 3) {
            val = 0.0;
        } else if (r < 3 && c < 3) {
            val = T[r * 4 + c];
        } else if (r >= 3 && c >= 3) {
            val = T[(r - 3) * 4 + (c - 3)];
        } else {
            // ([t]x R)[r][c-3]
            const double tx = T[3], ty = T[7], tz = T[11];
            const double sk[9] = {0.0, -tz, ty, tz, 0.0, -tx, -ty, tx, 0.0};
            const int cc = c - 3;
            val = sk[r * 3 + 0] * T[0 * 4 + cc] + sk[r * 3 + 1] * T[1 * 4 + cc] + sk[r * 3 + 2] * T[2 * 4 + cc];
        }
        Ad[threadIdx.x] = val;
    }
    __syncthreads();
    if (threadIdx.x < 36) {
        const int r = threadIdx.x / 6, c = threadIdx.x % 6;
        double x = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) x += K[r * 6 + k] * Ad[k * 6 + c];
        KA[threadIdx.x] = x;
    }
    __syncthreads();
    if (threadIdx.x < 36) {
        const int r = threadIdx.x / 6, c = threadIdx.x % 6;
        if (c >= r) {
            double x = 0.0;
#pragma unroll
            for (int k = 0; k < 6; ++k) x += Ad[k * 6 + r] * KA[k * 6 + c];
            out[sym_idx(r, c)] = lam * x;
        }
    } else if (threadIdx.x < 42) {
        const int r = threadIdx.x - 36;
        double x = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) x += Ad[k * 6 + r] * tot[21 + k];
        out[21 + r] = lam * x;
    } else if (threadIdx.x == 42) {
        out[27] = lam * tot[27];
        out[28] = tot[28];
    }
}

// Second stage of a correspondence set: right-perturbation blocks from the
// moments (J_i = -S(a), J_j = S(b), S(x) = [I | -[x]x]), times 2 lambda_1:
//   H_ii = [[W I, -[sa]x], [[sa]x, tr(Saa) I - Saa]]
//   H_jj = [[W I, -[sb]x], [[sb]x, tr(Sbb) I - Sbb]]
//   H_ij = -[[W I, -[sb]x], [[sa]x, tr(Sba) I - Sba]]
//   g_i = -[sum w e; sum w a x e],  g_j = [sum w e; sum w b x e]
template <bool kFull>
__device__ void reduce_edge(const SolveArgs& a, int e, double* sm)
{
    double* m = sm;   // 40
    if (threadIdx.x < kSparseVals) m[threadIdx.x] = (double)a.spart[(size_t)e * kSparseVals + threadIdx.x];
    __syncthreads();
    double* out = a.edgeblk + (size_t)e * kEdgeBlk;
    const double lam = 2.0 * a.lambda_sparse;
    if (threadIdx.x == 0) {
        out[90] = lam * m[37];
        out[91] = m[38];
    }
    if (!kFull) return;
    if (threadIdx.x < 36) {
        const int r = threadIdx.x / 6, c = threadIdx.x % 6;
        const double W = m[0];
        const double sa[3] = {m[1], m[2], m[3]}, sb[3] = {m[4], m[5], m[6]};
        // symmetric 3x3 from (xx xy xz yy yz zz)
        auto S3 = [&](int base, int rr, int cc) {
            const int lo = rr < cc ? rr : cc, hi = rr < cc ? cc : rr;
            const int id = lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
            return m[base + id];
        };
        auto skew = [&](const double* x, int rr, int cc) {
            // [x]x[rr][cc]
            if (rr == cc) return 0.0;
            if (rr == 0) return cc == 1 ? -x[2] : x[1];
            if (rr == 1) return cc == 0 ? x[2] : -x[0];
            return cc == 0 ? -x[1] : x[0];
        };
        auto block = [&](const double* s_row, const double* s_col, int mbase, bool mat_sym, int rr, int cc) {
            // [[W I, -[s_col]x], [[s_row]x, tr(S) I - S]] entry (rr, cc)
            if (rr < 3 && cc < 3) return rr == cc ? W : 0.0;
            if (rr < 3) return -skew(s_col, rr, cc - 3);
            if (cc < 3) return skew(s_row, rr - 3, cc);
            const int a3 = rr - 3, b3 = cc - 3;
            double tr, sv;
            if (mat_sym) {
                tr = S3(mbase, 0, 0) + S3(mbase, 1, 1) + S3(mbase, 2, 2);
                sv = S3(mbase, a3, b3);
            } else {
                tr = m[mbase + 0] + m[mbase + 4] + m[mbase + 8];
                sv = m[mbase + a3 * 3 + b3];
            }
            return (a3 == b3 ? tr : 0.0) - sv;
        };
        if (c >= r) {
            out[sym_idx(r, c)] = lam * block(sa, sa, 7, true, r, c);
            out[21 + sym_idx(r, c)] = lam * block(sb, sb, 13, true, r, c);
        }
        out[42 + threadIdx.x] = -lam * block(sa, sb, 19, false, r, c);
    } else if (threadIdx.x < 42) {
        const int r = threadIdx.x - 36;   // g_i = -[sum w e; sum w a x e], g_j = [sum w e; sum w b x e]
        out[78 + r] = -lam * (r < 3 ? m[28 + r] : m[31 + r - 3]);
        out[84 + r] = lam * (r < 3 ? m[28 + r] : m[34 + r - 3]);
    }
}

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// SE(3) exponential of xi = (v, w) as a 3x4 matrix (Rodrigues form with the
// V matrix; series for small angles).
__device__ void se3_exp_d(const double* xi, double* E)
{
    const double wx = xi[3], wy = xi[4], wz = xi[5];
    const double th2 = wx * wx + wy * wy + wz * wz;
    const double th = sqrt(th2);
    double A, B, C;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        double s, c;
        sincos(th, &s, &c);
        A = s / th;
        B = (1.0 - c) / th2;
        C = (th - s) / (th2 * th);
    }
    const double W[9] = {0.0, -wz, wy, wz, 0.0, -wx, -wy, wx, 0.0};
    double W2[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            W2[r * 3 + c] = W[r * 3 + 0] * W[0 * 3 + c] + W[r * 3 + 1] * W[1 * 3 + c] + W[r * 3 + 2] * W[2 * 3 + c];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        double t = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double id = r == c ? 1.0 : 0.0;
            E[r * 4 + c] = id + A * W[r * 3 + c] + B * W2[r * 3 + c];
            t += (id + B * W[r * 3 + c] + C * W2[r * 3 + c]) * xi[c];
        }
        E[r * 4 + 3] = t;
    }
}

// Last CTA: assemble H, g over the free nodes, Cholesky, solve, update.
template <bool kFull>
__device__ void final_phase(const SolveArgs& a, int iter, double* sm)
{
    const int N = a.N, P = a.n_pairs, NE = a.n_edges;
    if (threadIdx.x == 0) {
        double ed = 0.0, es = 0.0, cnt = 0.0;
        for (int p = 0; p < P; ++p) {
            ed += ldcg(a.pairblk + (size_t)p * kPairBlk + 27);
            cnt += ldcg(a.pairblk + (size_t)p * kPairBlk + 28);
        }
        for (int e = 0; e < NE; ++e) es += ldcg(a.edgeblk + (size_t)e * kEdgeBlk + 90);
        a.costs[iter * 4 + 0] = ed + es;
        a.costs[iter * 4 + 1] = ed;
        a.costs[iter * 4 + 2] = es;
        a.costs[iter * 4 + 3] = cnt;
    }
    if (!kFull) return;
    const int nf = a.n_free, n = 6 * nf;
    if (n == 0) return;
    const int status0 = *(volatile int*)&a.ctrl->status;
    if (status0 != 0) return;
    double* H = sm;                 // n*n
    double* g = H + n * n;          // n
    int* node_of = (int*)(g + n);   // nf
    int* edge_of = node_of + kMaxNodes;   // N*N
    __shared__ int s_fail;
    __shared__ double s_inv;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int f = a.nodes[k].free_idx;
        if (f >= 0) node_of[f] = k;
    }
    for (int k = threadIdx.x; k < N * N; k += blockDim.x) edge_of[k] = -1;
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
        const EdgeDev E = a.edges[e];
        edge_of[E.i * N + E.j] = e;
        edge_of[E.j * N + E.i] = e;
    }
    __syncthreads();
    auto pidx = [&](int from, int to) { return from * (N - 1) + (to < from ? to : to - 1); };
    // lower triangle of H
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int r = idx / n, c = idx % n;
        if (c > r) continue;
        const int A = node_of[r / 6], B = node_of[c / 6], rr = r % 6, cc = c % 6;
        const int s6 = sym_idx(rr, cc);
        double s = 0.0;
        if (A == B) {
            for (int k = 0; k < N; ++k) {
                if (k == A) continue;
                s += ldcg(a.pairblk + (size_t)pidx(A, k) * kPairBlk + s6);
                s += ldcg(a.pairblk + (size_t)pidx(k, A) * kPairBlk + s6);
                const int e = edge_of[A * N + k];
                if (e >= 0) {
                    const bool is_i = a.edges[e].i == A;
                    s += ldcg(a.edgeblk + (size_t)e * kEdgeBlk + (is_i ? 0 : 21) + s6);
                }
            }
        } else {
            s = -ldcg(a.pairblk + (size_t)pidx(A, B) * kPairBlk + s6) -
                ldcg(a.pairblk + (size_t)pidx(B, A) * kPairBlk + s6);
            const int e = edge_of[A * N + B];
            if (e >= 0) {
                const bool is_i = a.edges[e].i == A;
                s += ldcg(a.edgeblk + (size_t)e * kEdgeBlk + 42 + (is_i ? rr * 6 + cc : cc * 6 + rr));
            }
        }
        H[r * n + c] = s;
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const int A = node_of[r / 6], rr = r % 6;
        double s = 0.0;
        for (int k = 0; k < N; ++k) {
            if (k == A) continue;
            s += ldcg(a.pairblk + (size_t)pidx(A, k) * kPairBlk + 21 + rr);
            s -= ldcg(a.pairblk + (size_t)pidx(k, A) * kPairBlk + 21 + rr);
            const int e = edge_of[A * N + k];
            if (e >= 0) {
                const bool is_i = a.edges[e].i == A;
                s += ldcg(a.edgeblk + (size_t)e * kEdgeBlk + (is_i ? 78 : 84) + rr);
            }
        }
        g[r] = -s;   // right-hand side of H dx = -g
    }
    __syncthreads();
    // Cholesky H = L L^T (lower triangle, in place)
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double d = H[k * n + k];
            if (!(d > 0.0)) {
                s_fail = 1;
            } else {
                const double l = sqrt(d);
                H[k * n + k] = l;
                s_inv = 1.0 / l;
            }
        }
        __syncthreads();
        if (s_fail) break;
        const double inv = s_inv;
        for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) H[r * n + k] *= inv;
        __syncthreads();
        const int m = n - k - 1;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            const int r = k + 1 + t / m, c = k + 1 + t % m;
            if (c <= r) H[r * n + c] -= H[r * n + k] * H[c * n + k];
        }
        __syncthreads();
    }
    if (s_fail) {
        if (threadIdx.x == 0) a.ctrl->status = -4;
        return;
    }
    // forward / backward substitution (one warp)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int k = 0; k < n; ++k) {
            const double yk = g[k] / H[k * n + k];
            __syncwarp();
            if (lane == 0) g[k] = yk;
            for (int r = k + 1 + lane; r < n; r += 32) g[r] -= H[r * n + k] * yk;
            __syncwarp();
        }
        for (int k = n - 1; k >= 0; --k) {
            const double xk = g[k] / H[k * n + k];
            __syncwarp();
            if (lane == 0) g[k] = xk;
            for (int r = lane; r < k; r += 32) g[r] -= H[k * n + r] * xk;
            __syncwarp();
        }
    }
    __syncthreads();
    // T_A <- T_A exp(dx_A)
    if (threadIdx.x < nf) {
        const int A = node_of[threadIdx.x];
        double E[12], T[12], Tn[12];
        se3_exp_d(g + 6 * threadIdx.x, E);
#pragma unroll
        for (int k = 0; k < 12; ++k) T[k] = a.pose[A * 12 + k];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                double s = T[r * 4 + 0] * E[0 * 4 + c] + T[r * 4 + 1] * E[1 * 4 + c] + T[r * 4 + 2] * E[2 * 4 + c];
                if (c == 3) s += T[r * 4 + 3];
                Tn[r * 4 + c] = s;
            }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) a.pose[A * 12 + k] = Tn[k];
    }
    __syncthreads();
    write_xforms(a, threadIdx.x, blockDim.x);
}

template <bool kFull>
__global__ void __launch_bounds__(kThreads) reduce_kernel(SolveArgs a, int iter)
{
    extern __shared__ double sm[];
    __shared__ int s_last;
    const int b = blockIdx.x;
    if (b < a.n_pairs)
        reduce_pair<kFull>(a, b, sm);
    else if (b < a.n_pairs + a.n_edges)
        reduce_edge<kFull>(a, b - a.n_pairs, sm);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(&a.ctrl->counter, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) a.ctrl->counter = 0u;
    final_phase<kFull>(a, iter, sm);
}

size_t reduce_smem_bytes(int n_free, int N)
{
    const size_t n = 6 * (size_t)n_free;
    size_t fin = (n * n + n) * sizeof(double) + (kMaxNodes + (size_t)N * N) * sizeof(int);
    size_t ph1 = 400 * sizeof(double);
    return fin > ph1 ? fin : ph1;
}

cudaError_t launch_reduce(const SolveArgs& a, bool full, int iter, cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(reduce_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(reduce_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const int grid = a.n_pairs + a.n_edges > 0 ? a.n_pairs + a.n_edges : 1;
    const size_t smem = reduce_smem_bytes(a.n_free, a.N);
    if (full)
        reduce_kernel<true><<<grid, kThreads, smem, s>>>(a, iter);
    else
        reduce_kernel<false><<<grid, kThreads, smem, s>>>(a, iter);
    return cudaGetLastError();
}

}  // namespace bt
