// bt_ldlt.h -- FP64 solve of a symmetric positive-definite system H x = y
// by one CTA of 256 threads: the square-root-free Cholesky factorisation
// H = L D L^T with a one-column look-ahead (forward substitution L z = y
// carried along), D w = z, and a blocked back substitution L^T x = w.  Used
// by the Gauss-Newton step of Sec. IV-D (bt_solve.cu) and by the learned
// warm start's relative-pose averaging (bt_warmstart.cu).
//
// On GB300 a dependent FP64 operation costs ~64 cycles and a warp-wide FP64
// instruction occupies its sub-partition's DP unit for about as long whatever
// the number of active lanes, so the solve is arranged for short dependency
// chains and for many lanes behind each FP64 instruction.
#pragma once

#include "bt_internal.h"

namespace bt {

// 1/d for a positive FP64 pivot: the hardware approximation (rcp.approx.f64,
// relative error below 1e-6 on GB300) refined by one Newton step
// r <- r + r (1 - d r), which leaves a relative error below 1e-12 (measured
// on 1M pivots spanning 1e-6 .. 1e6) -- ample for a factorisation whose
// results are compared at 1e-5, and two dependent FP64 operations shorter
// than the correctly rounded reciprocal on the column chain.
__device__ __forceinline__ double rcp_fp64(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    const double e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

// Trailing rows from which warp 4 joins the bulk update (see ldlt_solve).
#ifndef BT_LDLT_WIDE_ROWS
#define BT_LDLT_WIDE_ROWS 30
#endif
constexpr int kWideBulkRows = BT_LDLT_WIDE_ROWS;

// Largest system: 6 unknowns per free node.  The back substitution splits
// the rows above a block of 32 unknowns into min(4, 256 / r0) column chunks
// (256 threads), which needs r0 < n <= 256.
constexpr int kLdltMaxN = 6 * (kMaxNodes - 1);
static_assert(kLdltMaxN <= 256, "ldlt_solve: at most 256 unknowns for one 256-thread CTA");

// Shared-memory scratch of ldlt_solve for an n x n system.
struct LdltScratch {
    double* rD;     // [n]      1 / D_k
    double* colb;   // [2][n]   the scaled look-ahead column, double-buffered
    int* tab;       // [n (n + 1) / 2]  (row, column) of the trailing triangle
    double* part;   // [256]    partial dot products of the back substitution
};

// H: n x n (n <= kLdltMaxN) in shared memory, row-major with leading
// dimension ld, lower triangle filled; the upper triangle is overwritten with
// L^T.  y: [n] right-hand side in shared memory, overwritten with x.  *fail
// (shared memory, zero on entry) is set when a pivot is not positive; x is
// then meaningless, and the caller reads *fail after the call (the call ends
// with a barrier).  t_mid: every thread's clock after the factorisation and
// D w = z.  idle(warp): called once by each of warps 1-7 while warp 0 alone
// runs the first block of the back substitution (work the caller has for
// otherwise idle warps; it must not touch H, y or the scratch, and is not
// called when a pivot failed).  All threads of the CTA (blockDim.x == 256)
// must call it.
struct LdltNoIdle {
    __device__ void operator()(int) const {}
};

template <typename Idle = LdltNoIdle>
__device__ __forceinline__ void ldlt_solve(double* __restrict__ H, int ld, int n, double* __restrict__ y,
                                           const LdltScratch& sc, int* fail, unsigned long long& t_mid,
                                           const Idle& idle = Idle())
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    double* rD = sc.rD;
    double* colb = sc.colb;
    int* tab = sc.tab;
    // LDL^T with a one-column look-ahead, one barrier per column.  At step k
    // warp 0 prepares column k+1 -- its update by column k, the pivot
    // D_{k+1} and reciprocal, and the scaled l_{i,k+1} -- while warps
    // {1,2,3,5,6,7} (no FP64 pipe shared with warp 0) apply column k to the
    // trailing triangle of rows and columns >= k+2 and carry the forward
    // substitution.  The scaled column is double-buffered; L is stored
    // transposed in the upper triangle, L_ik at (k, i).  A failed pivot
    // (not positive) sets *fail and a zero reciprocal; the loop still runs
    // to the end (same bounds, finite or discarded values), which keeps a
    // shared-memory read and a branch off every column of the chain.
    for (int ip = tid; ip < n; ip += nt)
        for (int jp = 0; jp <= ip; ++jp) tab[ip * (ip + 1) / 2 + jp] = (ip << 16) | jp;
    if (warp == 0) {
        double r = 0.0;
        if (lane == 0) {
            const double d = H[0];
            if (!(d > 0.0)) *fail = 1; else r = rcp_fp64(d);
            rD[0] = r;
        }
        r = __shfl_sync(0xffffffffu, r, 0);
        for (int i = 1 + lane; i < n; i += 32) {
            const double l = H[i * ld] * r;
            colb[i] = l;
            H[i] = l;
        }
    }
    __syncthreads();
    // bulk warps: {1,2,3,5,6,7}, and also warp 4 while the trailing triangle
    // is large (the early columns, where the bulk update and not warp 0's
    // chain sets the pace; warp 4 shares warp 0's FP64 unit, which has slack
    // there)
    const int bt6 = (warp != 0 && warp != 4 && warp < 8) ? (warp < 4 ? warp - 1 : warp - 2) * 32 + lane : -1;
    const int bt7 = (warp != 0 && warp < 8) ? (warp - 1) * 32 + lane : -1;
    for (int k = 0; k < n - 1; ++k) {
        const double* ck = colb + (k & 1) * n;        // l_{i,k}
        double* cn = colb + ((k + 1) & 1) * n;        // l_{i,k+1}, written now
        const bool wide = n - k - 2 >= kWideBulkRows;
        const int nbulk = wide ? 7 * 32 : 6 * 32;
        const int bt = wide ? bt7 : bt6;
        const bool bulk = bt >= 0;
        if (warp == 0) {
            // column p = k + 1, rows i = p .. n-1 in slots of 32: u_i = H_ip -
            // l_ik H_pk (the pivot is u_p), then every lane forms 1 / u_p
            // itself (no divergent branch, no second broadcast) and scales
            const int p = k + 1;
            const double hpk = H[p * ld + k];         // unscaled H_{k+1,k}
            const int nq = (n - p + 31) >> 5;         // active slots (warp-uniform)
            constexpr int kRows = (kLdltMaxN + 31) / 32;
            double hv[kRows], cv[kRows], u[kRows];
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                if (q >= nq) break;
                const int i = p + lane + 32 * q;
                hv[q] = i < n ? H[i * ld + p] : 0.0;
                cv[q] = i < n ? ck[i] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                if (q >= nq) break;
                u[q] = hv[q] - cv[q] * hpk;
            }
            const double h = __shfl_sync(0xffffffffu, u[0], 0);
            // h > 0 as an integer test on the bits (positive, not NaN): no
            // FP64 compare on the chain
            const long long hb = __double_as_longlong(h);
            const bool ok = hb > 0ll && hb <= 0x7ff0000000000000ll;
            const double rp = ok ? rcp_fp64(h) : 0.0;
            if (lane == 0) {
                if (!ok) *fail = 1;
                H[p * ld + p] = h;
                rD[p] = rp;
            }
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                if (q >= nq) break;
                const int i = p + lane + 32 * q;
                if (i > p && i < n) {
                    const double l = u[q] * rp;
                    H[i * ld + p] = u[q];
                    cn[i] = l;
                    H[p * ld + i] = l;
                }
            }
        } else if (bulk) {
            const int m1 = n - k - 2, tri = m1 * (m1 + 1) / 2;
            const double zk = y[k];
            for (int i = k + 1 + bt; i < n; i += nbulk) y[i] -= ck[i] * zk;
            int t = bt;
            for (; t + nbulk < tri; t += 2 * nbulk) {
                const int e0 = tab[t], e1 = tab[t + nbulk];
                const int i0 = k + 2 + (e0 >> 16), j0 = k + 2 + (e0 & 0xffff);
                const int i1 = k + 2 + (e1 >> 16), j1 = k + 2 + (e1 & 0xffff);
                const double a0 = H[i0 * ld + j0], a1 = H[i1 * ld + j1];
                const double l0 = ck[i0], l1 = ck[i1];
                const double b0 = H[j0 * ld + k], b1 = H[j1 * ld + k];
                H[i0 * ld + j0] = a0 - l0 * b0;
                H[i1 * ld + j1] = a1 - l1 * b1;
            }
            for (; t < tri; t += nbulk) {
                const int e = tab[t];
                const int i = k + 2 + (e >> 16), j = k + 2 + (e & 0xffff);
                H[i * ld + j] -= ck[i] * H[j * ld + k];
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += nt) y[i] *= rD[i];   // D w = z
    __syncthreads();
    t_mid = clock64();
    const bool failed = *fail != 0;
    // L^T x = w, unit diagonal (L_ki is stored at (i, k)), in blocks of 32
    // unknowns from the last block up.  Warp 0 runs the chain of one block
    // with the block's values in registers, lane l holding row r0 + l: x_k
    // is broadcast from its lane with a shuffle, and the FP64 instructions
    // issued do not grow with the size of the system.  The rows above the
    // block then take the
    // block's unknowns as dot products, split into column chunks over
    // several warps (partial sums in shared memory, added per row).
    double* part = sc.part;
    for (int r0 = ((n - 1) >> 5) << 5; r0 >= 0; r0 -= 32) {
        const int r1 = min(n, r0 + 32);
        if (warp == 0) {
            const int i = r0 + lane;
            double wv = i < r1 ? y[i] : 0.0;
            int k = r1 - 1;
            // two unknowns a step: x_k is final; every lane forms
            // x_{k-1} = w_{k-1} - L_{k,k-1} x_k itself from the broadcast
            // values (the same FMA its owner would apply), so the chain is
            // one shuffle and two FMAs deep per two unknowns; each row takes
            // x_k, then x_{k-1}, exactly as in the one-at-a-time order
            for (; k > r0 + 1; k -= 2) {
                const double hk = i < k ? H[i * ld + k] : 0.0;
                const double hk1 = i < k - 1 ? H[i * ld + k - 1] : 0.0;
                const double lk = H[(k - 1) * ld + k];        // L_{k,k-1}
                const double xk = __shfl_sync(0xffffffffu, wv, k - r0);
                const double wk1 = __shfl_sync(0xffffffffu, wv, k - 1 - r0);
                const double xk1 = fma(-lk, xk, wk1);
                if (i < k) wv = fma(-hk, xk, wv);
                if (i < k - 1) wv = fma(-hk1, xk1, wv);
            }
            if (k == r0 + 1) {
                const double hk = i < k ? H[i * ld + k] : 0.0;
                const double xk = __shfl_sync(0xffffffffu, wv, k - r0);
                if (i < k) wv = fma(-hk, xk, wv);
            }
            if (i < r1) y[i] = wv;
        } else if (r0 + 32 >= n && !failed) {
            idle(warp);
        }
        __syncthreads();
        if (r0 == 0) break;
        const int chunks = min(4, 256 / r0);      // r0 <= 128: at least 2
        if (tid < chunks * r0) {
            const int i = tid % r0, c = tid / r0;
            double s0 = 0.0, s1 = 0.0;
            int k = r0 + c;
            for (; k + chunks < r1; k += 2 * chunks) {
                s0 = fma(H[i * ld + k], y[k], s0);
                s1 = fma(H[i * ld + k + chunks], y[k + chunks], s1);
            }
            if (k < r1) s0 = fma(H[i * ld + k], y[k], s0);
            part[c * r0 + i] = s0 + s1;
        }
        __syncthreads();
        for (int i = tid; i < r0; i += nt) {
            double s = part[i];
            for (int c = 1; c < chunks; ++c) s += part[c * r0 + i];
            y[i] -= s;
        }
        __syncthreads();
    }
}

}  // namespace bt
