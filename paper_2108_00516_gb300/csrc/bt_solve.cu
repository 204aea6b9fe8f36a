// bt_solve.cu -- sm_103a kernels of the pose-graph solve (BundleTrack, Sec. IV-D):
// single-precision transforms of the FP64 poses, the reduction of the residual
// pass's FP32 partials into FP64 6x6 blocks, the assembly of the normal
// equations, the FP64 Cholesky (LDL^T) solve and the FP64 se(3) update, for one
// graph (reduce_kernel) or a batch of graphs (batch_*_kernel).
//
//   reduce_kernel   one CTA per unordered node pair turns the FP32 partials of
//                   both directions and the pair's correspondence set into
//                   FP64 6x6 blocks; the last CTA to finish assembles the
//                   normal equations over the free nodes, runs the FP64
//                   Cholesky solve and the FP64 se(3) update.
//
// Perturbations are right perturbations, T_i <- T_i exp(d_i) (see
// bt_residual.cu for why every iterate equals the left-perturbation one).
#include "bt_internal.h"
#include "bt_ldlt.h"
#include "bt_xform.cuh"

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace bt {

// ---------------------------------------------------------------------------
// Single-precision transforms of the FP64 poses (bt_xform.cuh: double-float
// arithmetic on the FP32 pipes, the same bits the host forms for the first
// pass of a solve and for the no-alloc call).
// ---------------------------------------------------------------------------

// Writes xf[i*N+j] = T_j T_i^-1 (i != j) and xinv[i] = T_i^-1 in single
// precision with the threads of one CTA: the splits of every pose first,
// then one matrix entry per thread.  `sf` is shared scratch of
// kXfSplit * N floats.
__device__ void write_xforms(const SolveArgs& a, float* __restrict__ sf, const double* __restrict__ pose)
{
    const int N = a.N, tid = threadIdx.x, nt = blockDim.x;
    for (int id = tid; id < N * 15; id += nt) {
        const int i = id / 15;
        xf_split_entry(pose + i * 12, id - 15 * i, sf + kXfSplit * i);
    }
    __syncthreads();
    for (int id = tid; id < N * 12; id += nt) {
        const int i = id / 12;
        a.xinv[id] = xf_inv_entry(sf + kXfSplit * i, id - 12 * i);
    }
    // pairs i != j only (the residual pass never reads xf[i*N+i])
    const int M = N > 1 ? N - 1 : 0;
    for (int id = tid; id < N * M * 12; id += nt) {
        const int pr = id / 12, e = id % 12;
        const int i = pr / M, jj = pr % M, j = jj < i ? jj : jj + 1;
        a.xf[(i * N + j) * 12 + e] = xf_pair_entry(sf + kXfSplit * j, sf + kXfSplit * i, e);
    }
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

__device__ __forceinline__ int upair_index(int a, int b, int N)
{
    // a < b, lexicographic order of the unordered pairs
    return a * N - (a * (a + 1)) / 2 + (b - a - 1);
}

// Entry (r, c) of Ad_T = [[R, [t]x R], [0, R]] for a 3x4 pose T.
__device__ __forceinline__ double ad_entry(const double* T, int r, int c)
{
    if (r >= 3 && c < 3) return 0.0;
    if (r < 3 && c < 3) return T[r * 4 + c];
    if (r >= 3 && c >= 3) return T[(r - 3) * 4 + (c - 3)];
    const double tx = T[3], ty = T[7], tz = T[11];
    const int cc = c - 3;
    const double R0 = T[0 * 4 + cc], R1 = T[1 * 4 + cc], R2 = T[2 * 4 + cc];
    if (r == 0) return -tz * R1 + ty * R2;
    if (r == 1) return tz * R0 - tx * R2;
    return -ty * R0 + tx * R1;
}

// Right-perturbation blocks of a correspondence set from its moments m (see
// sparse_edge), J_i = -S(a), J_j = S(b), S(x) = [I | -[x]x]:
//   H_ii = [[W I, -[sa]x], [[sa]x, tr(Saa) I - Saa]]
//   H_jj = [[W I, -[sb]x], [[sb]x, tr(Sbb) I - Sbb]]
//   H_ij = -[[W I, -[sb]x], [[sa]x, tr(Sba) I - Sba]]
// which: 0 = ii, 1 = jj, 2 = ij.
__device__ __forceinline__ double skew_entry(const double* x, int r, int c)
{
    if (r == c) return 0.0;
    if (r == 0) return c == 1 ? -x[2] : x[1];
    if (r == 1) return c == 0 ? x[2] : -x[0];
    return c == 0 ? -x[1] : x[0];
}

__device__ double sparse_block(const double* m, int which, int r, int c)
{
    const double W = m[0];
    const double* sa = m + 1;
    const double* sb = m + 4;
    const double* s_row = which == 1 ? sb : sa;
    const double* s_col = which == 0 ? sa : sb;
    double v;
    if (r < 3 && c < 3) {
        v = r == c ? W : 0.0;
    } else if (r < 3) {
        v = -skew_entry(s_col, r, c - 3);
    } else if (c < 3) {
        v = skew_entry(s_row, r - 3, c);
    } else {
        const int a3 = r - 3, b3 = c - 3;
        double tr, sv;
        if (which == 2) {
            tr = m[19] + m[23] + m[27];
            sv = m[19 + a3 * 3 + b3];
        } else {
            const int base = which == 0 ? 7 : 13;   // (xx xy xz yy yz zz)
            tr = m[base + 0] + m[base + 3] + m[base + 5];
            const int lo = a3 < b3 ? a3 : b3, hi = a3 < b3 ? b3 : a3;
            const int id = lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
            sv = m[base + id];
        }
        v = (a3 == b3 ? tr : 0.0) - sv;
    }
    return which == 2 ? -v : v;
}

// Second stage of an unordered pair {A < B}: sums of the tile partials of both
// directions (compensated FP32, widened to FP64), K' = Ad_{T_dst}^T K Ad_{T_dst} and g' = Ad_{T_dst}^T g~ for
// each (camera-j left blocks -> right perturbations), plus the pair's
// correspondence set; written pre-combined:
//   D_A = S + H_AA, D_B = S + H_BB, O_AB = -S + H_AB, g_A = gd + g_A^s,
//   g_B = -gd + g_B^s with S = lambda_2 (K'_{A->B} + K'_{B->A}) and
//   gd = lambda_2 (g'_{A->B} - g'_{B->A}).
constexpr int kPairSmemDoubles = 1520;   // shared memory of the pair stage (doubles)

// Neumaier-compensated accumulation in FP32: s + c is the running sum with
// an error of order u^2 (u = 2^-24) per term instead of u.  On GB300 a
// warp-wide FP64 instruction holds its sub-partition's DP unit for ~64
// cycles, so long sums run on the FP32 pipes and only their results are
// widened to FP64.
__device__ __forceinline__ void comp_add(float& s, float& c, float x)
{
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

template <bool kFull>
__device__ void reduce_upair(const SolveArgs& a, int u, double* sm)
{
    const int N = a.N;
    const int2 ab = a.upairs[u];
    const int A = ab.x, B = ab.y;
    const int e = a.upair_edge[u];
    const bool has = e >= 0;
    const int tid = threadIdx.x;
    float* fs = reinterpret_cast<float*>(sm);   // [2][16][32] (s, c) pairs
    double* tot = sm + 1024;   // [2][32] tile sums of both directions
    double* Ad = sm + 1088;    // [2][36]: Ad_{T_B} for A->B, Ad_{T_A} for B->A
    double* K = sm + 1160;     // [2][36]: K, then Ad^T K Ad per direction
    double* KA = sm + 1232;    // [2][36]
    double* mo = sm + 1304;    // 40 sparse moments
    double* gt = sm + 1344;    // [2][6] Ad^T g per direction
    double* hs = sm + 1356;    // [3][36] sparse blocks (A,A), (B,B), (A,B)
    double* ps = sm + 1464;    // [2][12] T_B, T_A
    int* sfwd = reinterpret_cast<int*>(sm + 1488);
    // loads that do not depend on the tile sums go out first
    double pv = 0.0;
    float mv = 0.f;
    int ei = -1;
    if (kFull && tid < 24) pv = __ldcg(a.pose + (tid < 12 ? B : A) * 12 + tid % 12);
    if (has && tid >= 128 && tid < 128 + kSparseVals) mv = __ldcg(a.spart + (size_t)e * kSparseVals + tid - 128);
    if (kFull && has && tid == 64) ei = __ldcg(&a.edges[e].i);
    // tile sums: thread = (direction, one of 16 tile groups, 4 consecutive
    // values); each thread reads every 16th tile of its direction as float4
    // (independent loads), compensated FP32 sums, groups combined in a fixed
    // order
    const int dir = tid >> 7, v4 = tid & 7, grp = (tid >> 3) & 15;
    const int src = dir ? B : A, dst = dir ? A : B;
    const int jj = dst < src ? dst : dst - 1;
    const int tile0 = a.nodes[src].tile0, ntiles = a.nodes[src].ntiles;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    if (kFull || v4 >= 6) {
        const size_t stride = (size_t)(N - 1) * (kDenseVals / 4);
        const float4* base =
            reinterpret_cast<const float4*>(a.dpart + ((size_t)tile0 * (N - 1) + jj) * kDenseVals) + v4;
        int t = grp;
        for (; t + 112 < ntiles; t += 128) {
            float4 x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = __ldcg(base + (size_t)(t + 16 * q) * stride);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                comp_add(s[0], c[0], x[q].x);
                comp_add(s[1], c[1], x[q].y);
                comp_add(s[2], c[2], x[q].z);
                comp_add(s[3], c[3], x[q].w);
            }
        }
        float4 x[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {     // t + 112 >= ntiles: at most 7 tiles left
            const int tq = t + 16 * q;
            x[q] = tq < ntiles ? __ldcg(base + (size_t)tq * stride) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            comp_add(s[0], c[0], x[q].x);
            comp_add(s[1], c[1], x[q].y);
            comp_add(s[2], c[2], x[q].z);
            comp_add(s[3], c[3], x[q].w);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int o = ((dir * 16 + grp) * 32 + 4 * v4 + k) * 2;
        fs[o] = s[k];
        fs[o + 1] = c[k];
    }
    if (kFull && tid < 24) ps[tid] = pv;
    if (tid >= 128 && tid < 128 + kSparseVals) mo[tid - 128] = has ? (double)mv : 0.0;
    if (tid == 64) *sfwd = ei;
    __syncthreads();
    if (tid < 64) {
        const int d = tid >> 5, w = tid & 31;
        float S0 = 0.f, C0 = 0.f;
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            const int o = ((d * 16 + g) * 32 + w) * 2;
            comp_add(S0, C0, fs[o]);
            C0 += fs[o + 1];
        }
        tot[tid] = (double)S0 + (double)C0;
    }
    __syncthreads();
    double* out = a.upairblk + (size_t)u * kUPairBlk;
    const double lg = a.lambda_dense, ls = 2.0 * a.lambda_sparse;
    if (!kFull) {
        if (tid == 0) {
            out[90] = lg * (tot[27] + tot[32 + 27]);
            out[91] = has ? ls * mo[37] : 0.0;
            out[92] = tot[28] + tot[32 + 28];
        }
        return;
    }
    if (tid < 72) {
        const int d = tid / 36, q = tid % 36, r = q / 6, cc = q % 6;
        Ad[tid] = ad_entry(ps + d * 12, r, cc);
        K[tid] = tot[d * 32 + sym_idx(r, cc)];
    }
    __syncthreads();
    // the 6-term products as two independent 3-term FMA chains (a dependent
    // FP64 operation costs ~100 cycles on the critical path)
    if (tid < 72) {
        const int d = tid / 36, q = tid % 36, r = q / 6, cc = q % 6;
        const double* Kr = K + d * 36 + r * 6;
        const double* Ac = Ad + d * 36 + cc;
        const double x0 = fma(Kr[2], Ac[12], fma(Kr[1], Ac[6], Kr[0] * Ac[0]));
        const double x1 = fma(Kr[5], Ac[30], fma(Kr[4], Ac[24], Kr[3] * Ac[18]));
        KA[tid] = x0 + x1;
    }
    __syncthreads();
    // K'_d = Ad_d^T K_d Ad_d and g'_d = Ad_d^T g_d per direction (threads
    // 0-83), and the three sparse blocks (threads 128-235), side by side
    if (tid < 72) {
        const int d = tid / 36, q = tid % 36, r = q / 6, cc = q % 6;
        const double* Ar = Ad + d * 36 + r;
        const double* Bc = KA + d * 36 + cc;
        const double x0 = fma(Ar[12], Bc[12], fma(Ar[6], Bc[6], Ar[0] * Bc[0]));
        const double x1 = fma(Ar[30], Bc[30], fma(Ar[24], Bc[24], Ar[18] * Bc[18]));
        K[tid] = x0 + x1;
    } else if (tid < 84) {
        const int d = (tid - 72) / 6, r = (tid - 72) % 6;
        double g = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) g += Ad[d * 36 + k * 6 + r] * tot[d * 32 + 21 + k];
        gt[tid - 72] = g;
    } else if (tid >= 128 && tid < 128 + 108) {
        const int w = (tid - 128) / 36, q = (tid - 128) % 36, r = q / 6, cc = q % 6;
        const bool fwd = has && *sfwd == A;   // correspondence set stored as (A, B)
        double h = 0.0;
        if (has) {
            if (w == 0) h = sparse_block(mo, fwd ? 0 : 1, r, cc);
            else if (w == 1) h = sparse_block(mo, fwd ? 1 : 0, r, cc);
            else h = fwd ? sparse_block(mo, 2, r, cc) : sparse_block(mo, 2, cc, r);
        }
        hs[tid - 128] = ls * h;
    }
    __syncthreads();
    if (tid < 36) {
        const int r = tid / 6, cc = tid % 6;
        const int q = (r < cc ? r : cc) * 6 + (r < cc ? cc : r);   // S is symmetric: one rounding for both halves
        const double Sv = lg * (K[q] + K[36 + q]);
        if (cc >= r) {
            out[sym_idx(r, cc)] = Sv + hs[tid];
            out[21 + sym_idx(r, cc)] = Sv + hs[36 + tid];
        }
        out[42 + tid] = -Sv + hs[72 + tid];
    } else if (tid < 42) {
        const int r = tid - 36;
        const bool fwd = has && *sfwd == A;
        const double gdv = lg * (gt[r] - gt[6 + r]);
        // g_i = -[sum w e; sum w a x e], g_j = [sum w e; sum w b x e]
        const double gi = has ? -ls * (r < 3 ? mo[28 + r] : mo[31 + r - 3]) : 0.0;
        const double gj = has ? ls * (r < 3 ? mo[28 + r] : mo[34 + r - 3]) : 0.0;
        out[78 + r] = gdv + (fwd ? gi : gj);
        out[84 + r] = -gdv + (fwd ? gj : gi);
    } else if (tid == 42) {
        out[90] = lg * (tot[27] + tot[32 + 27]);
        out[91] = has ? ls * mo[37] : 0.0;
        out[92] = tot[28] + tot[32 + 28];
    }
}

// The SE(3) exponential of xi = (v, w) as a 3x4 matrix:
// R = I + A W + B W^2, t = (I + B W + C W^2) v = v + B (w x v) + C (w (w.v) -
// th^2 v), with W = [w]x, W^2 = w w^T - th^2 I, A = sin(th)/th,
// B = (1 - cos th)/th^2, C = (th - sin th)/th^3.  Below th = 0.1 the
// coefficients come from their Taylor series through th^8 (truncation
// < 3e-18), which keeps FP64 sincos off the critical path; above it from
// sincos.  which: 0 = A, 1 = B, 2 = C.
__device__ double se3_exp_coef(const double* xi, int which)
{
    const double th2 = fma(xi[5], xi[5], fma(xi[4], xi[4], xi[3] * xi[3]));
    if (th2 < 0.01) {
        if (which == 0)
            return 1.0 + th2 * (-1.0 / 6.0 + th2 * (1.0 / 120.0 + th2 * (-1.0 / 5040.0 + th2 * (1.0 / 362880.0))));
        if (which == 1)
            return 0.5 + th2 * (-1.0 / 24.0 + th2 * (1.0 / 720.0 + th2 * (-1.0 / 40320.0 + th2 * (1.0 / 3628800.0))));
        return 1.0 / 6.0 + th2 * (-1.0 / 120.0 + th2 * (1.0 / 5040.0 + th2 * (-1.0 / 362880.0 + th2 * (1.0 / 39916800.0))));
    }
    const double th = sqrt(th2);
    double sn, cs;
    sincos(th, &sn, &cs);
    if (which == 0) return sn / th;
    if (which == 1) return (1.0 - cs) / th2;
    return (th - sn) / (th2 * th);
}

// Entry (r, c) of exp(xi); cf = (th^2, A, B, C).  One thread per entry: a
// warp-wide FP64 instruction costs its sub-partition ~64 cycles whatever the
// number of active lanes, so the entries are spread over lanes.
__device__ double se3_exp_entry(const double* xi, const double* cf, int r, int c)
{
    const double th2 = cf[0], A = cf[1], B = cf[2], C = cf[3];
    const double* w = xi + 3;
    if (c < 3) {
        // [w]x (r, c): 0 on the diagonal, -w_k for (0,1), (1,2), (2,0), +w_k
        // for the transposed positions, k the third index
        const int k = 3 - r - c;
        const double Wrc = r == c ? 0.0 : ((r + 1) % 3 == c ? -w[k] : w[k]);
        const double W2rc = fma(w[r], w[c], r == c ? -th2 : 0.0);
        return fma(B, W2rc, fma(A, Wrc, r == c ? 1.0 : 0.0));
    }
    const int r1 = (r + 1) % 3, r2 = (r + 2) % 3;
    const double cross = fma(w[r1], xi[r2], -(w[r2] * xi[r1]));     // (w x v)_r
    const double wv = fma(w[2], xi[2], fma(w[1], xi[1], w[0] * xi[0]));
    const double inner = fma(w[r], wv, -(th2 * xi[r]));              // (W^2 v)_r
    return fma(C, inner, fma(B, cross, xi[r]));
}

// Last CTA: energies, then (full) assembly of H and g over the free nodes,
// the FP64 solve of H dx = -g (square-root-free Cholesky with a one-column
// look-ahead, bt_ldlt.h; or PCG, the paper's inner solver), and finally
// T <- T exp(dx).
// The first global reads of the last CTA, issued by every CTA of the reduce
// kernel before its pair stage: the last CTA is only known after the
// hand-off, and these values (the sticky status of earlier iterations, the
// nodes' free indices, the poses) do not change within the kernel, so their
// L2 round trip overlaps the pair stage instead of following the hand-off.
// Thread t holds pose entries t and t + blockDim.x (12 N <= 2 * 256) and the
// free index of node t.
static_assert(12 * kMaxNodes <= 2 * kThreads && kMaxNodes <= kThreads, "final_prefetch: two pose entries a thread");
struct FinalPrefetch {
    int status;
    int free_idx;
    double pose0, pose1;
};

template <bool kFull>
__device__ __forceinline__ FinalPrefetch final_prefetch(const SolveArgs& a)
{
    FinalPrefetch pf{0, -1, 0.0, 0.0};
    if (!kFull) return pf;
    const int tid = threadIdx.x, nt = blockDim.x, N = a.N;
    pf.status = __ldcg(&a.ctrl->status);
    if (tid < N) pf.free_idx = __ldcg(&a.nodes[tid].free_idx);
    if (tid < 12 * N) pf.pose0 = __ldcg(a.pose + tid);
    if (tid + nt < 12 * N) pf.pose1 = __ldcg(a.pose + tid + nt);
    return pf;
}

template <bool kFull>
__device__ void final_phase(const SolveArgs& a, int iter, double* sm, const FinalPrefetch& pf)
{
    const int N = a.N, U = a.n_upairs;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    const int nf = a.n_free, n = 6 * nf;
    const int status0 = kFull ? pf.status : 0;
    // energies of the iteration: from the staged pair blocks when a full
    // solve stages them, else straight from global memory
    const bool staged_costs = kFull && n > 0 && status0 == 0 && a.stage_blocks != 0;
    auto write_costs = [&](const double* blocks, bool shared) {
        double ed = 0.0, es = 0.0, cnt = 0.0;
        for (int u = lane; u < U; u += 32) {
            const double* o = blocks + (size_t)u * kUPairBlk;
            ed += shared ? o[90] : __ldcg(o + 90);
            es += shared ? o[91] : __ldcg(o + 91);
            cnt += shared ? o[92] : __ldcg(o + 92);
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            ed += __shfl_xor_sync(0xffffffffu, ed, off);
            es += __shfl_xor_sync(0xffffffffu, es, off);
            cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        }
        if (lane == 0) {
            a.costs[iter * 4 + 0] = ed + es;
            a.costs[iter * 4 + 1] = ed;
            a.costs[iter * 4 + 2] = es;
            a.costs[iter * 4 + 3] = cnt;
        }
    };
    if (!staged_costs && tid < 32) write_costs(a.upairblk, false);
    if (!kFull || n == 0 || status0 != 0) return;
    unsigned long long t0 = clock64();
    const int ld = n + 1;        // odd leading dimension: conflict-free FP64 rows
    double* H = sm;              // n*ld: lower triangle H, then L^T in the upper triangle
    double* y = H + n * ld;      // n
    double* rD = y + n;          // n: 1 / D_k
    double* ps = rD + n;         // 12 * N poses
    double* tinv = ps + 12 * kMaxNodes;   // 12 * N
    // tinv + 12 * kMaxNodes: [2][n] scaled columns, then the triangle index
    // table (n (n+1) / 2 ints, rounded up to whole doubles), then the staged
    // pair blocks
    const size_t tab_dbl = ((size_t)n * (n + 1) / 2 + 1) / 2;
    double* stage = tinv + 12 * kMaxNodes + 2 * n + tab_dbl;
    if (((size_t)(stage - sm)) & 1) ++stage;               // 16-byte alignment for double2
    const size_t stage_len = a.stage_blocks ? (size_t)U * kUPairBlk : 0;
    int* node_of = reinterpret_cast<int*>(stage + stage_len);
    __shared__ int s_fail;
    if (tid < N && pf.free_idx >= 0) node_of[pf.free_idx] = tid;
    if (tid < 12 * N) ps[tid] = pf.pose0;
    if (tid + nt < 12 * N) ps[tid + nt] = pf.pose1;
    if (tid == 0) s_fail = 0;
    {   // pair blocks to shared memory, up to twelve independent loads in
        // flight per thread (one round for ten nodes: each round costs an
        // L2 round trip)
        const double2* src = reinterpret_cast<const double2*>(a.upairblk);
        double2* dst = reinterpret_cast<double2*>(stage);
        const int n2 = (int)(stage_len / 2);
        for (int q0 = tid; q0 < n2; q0 += 12 * nt) {
            double2 v[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const int q = q0 + k * nt;
                if (q < n2) v[k] = __ldcg(src + q);
            }
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const int q = q0 + k * nt;
                if (q < n2) dst[q] = v[k];
            }
        }
    }
    __syncthreads();
    // (with staged blocks the energies are added up during the update, by a
    // warp that has no other work there: here their FP64 adds would hold
    // one sub-partition's DP unit beside its share of the diagonal sums)
    const int cost_warp = (nt >> 5) - 1;
    const bool staged = a.stage_blocks != 0;
    auto blk = [&](size_t q) { return staged ? stage[q] : __ldcg(a.upairblk + q); };
    // diagonal blocks and gradient: one thread per (free node, value), values
    // 0-20 the unique block entries, 21-26 the gradient entries (all the
    // warps' FP64 pipes at once rather than one warp per node)
    for (int q = tid; q < nf * 27; q += nt) {
        const int f = q / 27, v = q - 27 * f;
        const int A = node_of[f];
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < N; ++k) {
            if (k == A) continue;
            const int u = A < k ? upair_index(A, k, N) : upair_index(k, A, N);
            const size_t off = (size_t)u * kUPairBlk + (v < 21 ? (A < k ? 0 : 21) + v : (A < k ? 78 : 84) + v - 21);
            if (k & 1) s1 += blk(off); else s0 += blk(off);
        }
        const double s = s0 + s1;
        if (v < 21) {
            int r = 0, e = v;
            while (e >= 6 - r) { e -= 6 - r; ++r; }
            const int c = r + e;     // (r, c), c >= r, of the 6x6 block
            H[(6 * f + c) * ld + 6 * f + r] = s;
        } else {
            y[6 * f + v - 21] = -s;   // right-hand side of H dx = -g
        }
    }
    // off-diagonal blocks (fa > fb)
    const int nob = nf * (nf - 1) / 2;
    for (int q = tid; q < nob * 36; q += nt) {
        const int b = q / 36, e = q % 36, rr = e / 6, cc = e % 6;
        // b = fa (fa - 1) / 2 + fb with fb < fa: fa from the square root,
        // corrected by one step either way (b < 253, exact in FP32)
        int fa = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)b)) * 0.5f);
        if (fa * (fa - 1) / 2 > b) --fa;
        if (fa * (fa + 1) / 2 <= b) ++fa;
        const int fb = b - fa * (fa - 1) / 2;
        const int A = node_of[fa], B = node_of[fb];
        const int u = A < B ? upair_index(A, B, N) : upair_index(B, A, N);
        H[(6 * fa + rr) * ld + 6 * fb + cc] = blk((size_t)u * kUPairBlk + 42 + (A < B ? rr * 6 + cc : cc * 6 + rr));
    }
    __syncthreads();
    if (a.ne_out != nullptr) {
        // diagnostic export of the assembled system (symmetric H, g = -y);
        // no solve, no update
        for (int q = tid; q < n * n; q += nt) {
            const int r = q / n, c = q - r * n;
            a.ne_out[q] = r >= c ? H[r * ld + c] : H[c * ld + r];
        }
        for (int q = tid; q < n; q += nt) a.ne_out[n * n + q] = -y[q];
        if (staged_costs && warp == cost_warp) write_costs(stage, true);
        return;
    }
    unsigned long long t1 = clock64();
    double* colb = tinv + 12 * kMaxNodes;   // [2][n]
    unsigned long long t2, t3;
    if (a.solver == 1) {
        // Conjugate gradients with the diagonal preconditioner (the paper's
        // inner solver, Sec. IV-D), FP64, from dx = 0.  The matrix-vector
        // product is split over (row, column chunk) pairs so that every
        // thread has work: a warp-wide FP64 instruction costs its
        // sub-partition the same whatever the number of active lanes.
        double* xv = colb;           // dx
        double* pv = colb + n;       // search direction
        double* rv = y;              // residual, starts as -g
        double* zv = rD;             // preconditioned residual
        double* qv = tinv;           // H p
        double* part = reinterpret_cast<double*>(node_of + kMaxNodes);   // [n * C]
        double* red = part + 256;    // [8]
        const int C = nt / n > 0 ? nt / n : 1;
        const int w = (n + C - 1) / C;
        auto block_sum = [&](double v) {
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) red[warp] = v;
            __syncthreads();
            double t = 0.0;
            for (int k = 0; k < nt / 32; ++k) t += red[k];
            __syncthreads();
            return t;
        };
        double bb = 0.0, rz = 0.0;
        for (int i = tid; i < n; i += nt) {
            const double d = H[i * ld + i];
            if (!(d > 0.0)) s_fail = 1;
            xv[i] = 0.0;
            zv[i] = rv[i] / d;
            pv[i] = zv[i];
            bb += rv[i] * rv[i];
            rz += rv[i] * zv[i];
        }
        bb = block_sum(bb);
        rz = block_sum(rz);
        double rr = bb;
        for (int it = 0; !s_fail && it < a.pcg_max_iters && rr > a.pcg_tol2 * bb; ++it) {
            if (tid < n * C) {
                const int i = tid / C, c = tid % C;
                const int j1 = (c + 1) * w < n ? (c + 1) * w : n;
                double v = 0.0;
                for (int j = c * w; j < j1; ++j) v += (j <= i ? H[i * ld + j] : H[j * ld + i]) * pv[j];
                part[tid] = v;
            }
            __syncthreads();
            double pq = 0.0;
            for (int i = tid; i < n; i += nt) {
                double v = 0.0;
                for (int c = 0; c < C; ++c) v += part[i * C + c];
                qv[i] = v;
                pq += pv[i] * v;
            }
            pq = block_sum(pq);
            if (!(pq > 0.0)) {
                if (tid == 0) s_fail = 1;
                __syncthreads();
                break;
            }
            const double alpha = rz / pq;
            double rrp = 0.0, rzp = 0.0;
            for (int i = tid; i < n; i += nt) {
                xv[i] += alpha * pv[i];
                rv[i] -= alpha * qv[i];
                zv[i] = rv[i] / H[i * ld + i];
                rrp += rv[i] * rv[i];
                rzp += rv[i] * zv[i];
            }
            rr = block_sum(rrp);
            const double rz_new = block_sum(rzp);
            const double beta = rz_new / rz;
            rz = rz_new;
            for (int i = tid; i < n; i += nt) pv[i] = zv[i] + beta * pv[i];
            __syncthreads();
        }
        if (s_fail) {
            if (tid == 0) a.ctrl->status = -4;
            if (staged_costs && warp == cost_warp) write_costs(stage, true);
            return;
        }
        for (int i = tid; i < n; i += nt) y[i] = xv[i];
        __syncthreads();
        t2 = t3 = clock64();
    } else {
    // LDL^T with a one-column look-ahead, D w = z, blocked L^T dx = w
    // (bt_ldlt.h); the forward substitution of -g is carried along
    LdltScratch sc;
    sc.rD = rD;
    sc.colb = colb;
    sc.tab = reinterpret_cast<int*>(colb + 2 * n);
    sc.part = reinterpret_cast<double*>(node_of + kMaxNodes);
    // the energies are added up by the last warp while warp 0 runs the
    // first block of the back substitution alone
    ldlt_solve(H, ld, n, y, sc, &s_fail, t2, [&](int w) {
        if (staged_costs && w == cost_warp) write_costs(stage, true);
    });
    if (s_fail) {
        if (tid == 0) a.ctrl->status = -4;
        if (staged_costs && warp == cost_warp) write_costs(stage, true);
        return;
    }
    __syncthreads();
    t3 = clock64();
    }
    // T_A <- T_A exp(dx_A) in three steps: the coefficients of exp per node
    // (warps 0-2, one coefficient each, so the three FP64 chains run on
    // three sub-partitions), the entries of exp(dx_A) (one thread each), the
    // products T_A exp(dx_A) (one thread each).  The look-ahead columns, rD
    // and tinv are free now (after PCG the last warp adds up the energies
    // meanwhile; the Cholesky path has done so during its back substitution).
    {
        double* cf = rD;       // [nf][4]: th^2, A, B, C
        double* E = colb;      // [nf][12]
        double* P = tinv;      // [nf][12]
        if (warp < 3 && lane < nf) {
            const double* xi = y + 6 * lane;
            const double c = se3_exp_coef(xi, warp);
            cf[4 * lane + 1 + warp] = c;
            if (warp == 0) cf[4 * lane] = fma(xi[5], xi[5], fma(xi[4], xi[4], xi[3] * xi[3]));
        }
        if (a.solver == 1 && staged_costs && warp == cost_warp) write_costs(stage, true);
        __syncthreads();
        for (int q = tid; q < 12 * nf; q += nt) {
            // rotation entries (f, r, c < 3) first, then the translations
            int f, r, c;
            if (q < 9 * nf) {
                f = q / 9;
                const int e = q - 9 * f;
                r = e / 3;
                c = e - 3 * r;
            } else {
                const int e = q - 9 * nf;
                f = e / 3;
                r = e - 3 * f;
                c = 3;
            }
            E[f * 12 + r * 4 + c] = se3_exp_entry(y + 6 * f, cf + 4 * f, r, c);
        }
        __syncthreads();
        for (int q = tid; q < 12 * nf; q += nt) {
            const int f = q / 12, e = q % 12, r = e >> 2, c = e & 3;
            const double* T = ps + node_of[f] * 12;
            const double* Ef = E + f * 12;
            double v = T[r * 4 + 0] * Ef[0 * 4 + c] + T[r * 4 + 1] * Ef[1 * 4 + c] + T[r * 4 + 2] * Ef[2 * 4 + c];
            if (c == 3) v += T[r * 4 + 3];
            P[q] = v;
        }
        __syncthreads();
        for (int q = tid; q < 12 * nf; q += nt) ps[node_of[q / 12] * 12 + q % 12] = P[q];
    }
    __syncthreads();
    for (int q = tid; q < 12 * N; q += nt) a.pose[q] = ps[q];
    // split scratch from tinv on (32 N floats: tinv, the look-ahead columns,
    // the triangle table and the staged blocks are free now)
    write_xforms(a, reinterpret_cast<float*>(tinv), ps);
    if (tid == 0) {
        unsigned long long t4 = clock64();
        a.ctrl->clk[0] += t1 - t0;
        a.ctrl->clk[1] += t2 - t1;
        a.ctrl->clk[2] += t3 - t2;
        a.ctrl->clk[3] += t4 - t3;
    }
}

template <bool kFull>
__global__ void __launch_bounds__(kThreads, 1) reduce_kernel(SolveArgs a, int iter)
{
    extern __shared__ double sm[];
    __shared__ int s_last;
    const int b = blockIdx.x;
    // the previous update's poses and status: written before the residual
    // pass this kernel waits for, so read ahead of the wait
    const FinalPrefetch pf = final_prefetch<kFull>(a);
    pdl_wait_and_release();
    if (b < a.n_upairs) reduce_upair<kFull>(a, b, sm);
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
    final_phase<kFull>(a, iter, sm, pf);
}

static size_t reduce_smem_bytes_for(int n_free, int N, bool stage)
{
    const size_t n = 6 * (size_t)n_free;
    const size_t U = (size_t)N * (N - 1) / 2;
    const size_t sl = stage ? U * kUPairBlk : 0;
    const size_t tab_dbl = (n * (n + 1) / 2 + 1) / 2;
    // ... + the PCG scratch after node_of: 256 partial sums + 8 warp sums
    size_t fin = (n * (n + 1) + 4 * n + 24 * (size_t)kMaxNodes + tab_dbl + 1 + sl + 264) * sizeof(double) +
                 kMaxNodes * sizeof(int);
    size_t ph1 = kPairSmemDoubles * sizeof(double);
    return fin > ph1 ? fin : ph1;
}

bool reduce_stage_fits(int n_free, int N) { return reduce_smem_bytes_for(n_free, N, true) <= kReduceSmemMax; }

size_t reduce_smem_bytes(int n_free, int N)
{
    return reduce_smem_bytes_for(n_free, N, reduce_stage_fits(n_free, N));
}

cudaError_t launch_reduce(const SolveArgs& a, bool full, int iter, cudaStream_t s)
{
    static const bool attr_set = [] {      // once per process, thread-safe
        cudaFuncSetAttribute(reduce_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReduceSmemMax);
        cudaFuncSetAttribute(reduce_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReduceSmemMax);
        return true;
    }();
    (void)attr_set;
    const int grid = a.n_upairs > 0 ? a.n_upairs : 1;
    const size_t smem = reduce_smem_bytes(a.n_free, a.N);
    if (full)
        return launch_chained(reduce_kernel<true>, dim3(grid), dim3(kThreads), smem, s, a, iter);
    return launch_chained(reduce_kernel<false>, dim3(grid), dim3(kThreads), smem, s, a, iter);
}

// ---------------------------------------------------------------------------
// Batched solver kernels (one CTA per graph or per (graph, pair))
// ---------------------------------------------------------------------------

__global__ void batch_xform_kernel(const SolveArgs* __restrict__ args)
{
    pdl_wait_and_release();
    __shared__ float sf[kXfSplit * kMaxNodes];
    __shared__ SolveArgs sa;
    if (threadIdx.x == 0) sa = args[blockIdx.x];
    __syncthreads();
    write_xforms(sa, sf, sa.pose);
}

template <bool kFull>
__global__ void __launch_bounds__(kThreads) batch_pair_kernel(const SolveArgs* __restrict__ args,
                                                              const int2* __restrict__ work)
{
    pdl_wait_and_release();
    __shared__ double sm[kPairSmemDoubles];
    __shared__ SolveArgs sa;
    const int2 w = work[blockIdx.x];
    if (threadIdx.x == 0) sa = args[w.x];
    __syncthreads();
    reduce_upair<kFull>(sa, w.y, sm);
}

template <bool kFull>
__global__ void __launch_bounds__(kThreads, 1) batch_solve_kernel(const SolveArgs* __restrict__ args, int iter)
{
    pdl_wait_and_release();
    extern __shared__ double smd[];
    __shared__ SolveArgs sa;
    if (threadIdx.x == 0) sa = args[blockIdx.x];
    __syncthreads();
    final_phase<kFull>(sa, iter, smd, final_prefetch<kFull>(sa));
}

cudaError_t launch_batch_xforms(const SolveArgs* args_dev, int n_graphs, cudaStream_t s)
{
    if (n_graphs == 0) return cudaSuccess;
    return launch_chained(batch_xform_kernel, dim3(n_graphs), dim3(kThreads), 0, s, args_dev);
}

cudaError_t launch_batch_pairs(const SolveArgs* args_dev, const int2* work_pair, int n_work, bool full,
                               cudaStream_t s)
{
    if (n_work == 0) return cudaSuccess;
    if (full)
        return launch_chained(batch_pair_kernel<true>, dim3(n_work), dim3(kThreads), 0, s, args_dev, work_pair);
    return launch_chained(batch_pair_kernel<false>, dim3(n_work), dim3(kThreads), 0, s, args_dev, work_pair);
}

cudaError_t launch_batch_solve(const SolveArgs* args_dev, int n_graphs, size_t smem, bool full, int iter,
                               cudaStream_t s)
{
    static const bool attr_set = [] {      // once per process, thread-safe
        cudaFuncSetAttribute(batch_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReduceSmemMax);
        cudaFuncSetAttribute(batch_solve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReduceSmemMax);
        return true;
    }();
    (void)attr_set;
    if (n_graphs == 0) return cudaSuccess;
    if (full)
        return launch_chained(batch_solve_kernel<true>, dim3(n_graphs), dim3(kThreads), smem, s, args_dev, iter);
    return launch_chained(batch_solve_kernel<false>, dim3(n_graphs), dim3(kThreads), smem, s, args_dev, iter);
}

void prepare_launch_attributes()
{
    prepare_residual_attributes();
    cudaFuncSetAttribute(batch_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReduceSmemMax);
    cudaFuncSetAttribute(batch_solve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReduceSmemMax);
    cudaFuncSetAttribute(reduce_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReduceSmemMax);
    cudaFuncSetAttribute(reduce_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReduceSmemMax);
}

}  // namespace bt
