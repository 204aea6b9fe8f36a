// bt_xform.cuh -- the single-precision pair transforms M = T_j T_i^-1 that
// the residual pass reads (camera i -> camera j), formed from the FP64 poses
// in double-float arithmetic on the FP32 pipes, and reproducible bit for bit
// on the host (the first pass of a solve, the no-alloc call).
//
// Each FP64 input x is split into x = hi + lo with hi = RN32(x) and
// lo = RN32(x - hi) (an error of 2^-48 |x| at most).  An entry
// M_rc = sum_k T_j[r][k] T_i^-1[k][c] (+ T_j[r][3] for c = 3) is then a
// double-float dot product: exact two-products of the leading parts
// (p = a b, e = fma(a, b, -p)), the cross terms in single precision, and
// Knuth's two-sum for the running sum, which keeps the translation accurate
// through the cancellation of its ~0.5 m terms; the sum is rounded once to
// single precision.  The result is within about 2^-44 of the exact entry
// before that last rounding, so it equals the FP64-formed entry rounded to
// single precision except within that distance of a rounding boundary.
//
// On GB300 every FP64 instruction, the conversions included, holds its
// sub-partition's DP unit for ~64 cycles; here only the splits (and the
// inverse's translation) use it, the products and sums run on the FP32
// pipes.  Every operation is written out (no contraction, no reassociation:
// the device uses the _rn intrinsics, the host compiles with
// -ffp-contract=off), so host and device give the same bits.
#pragma once

#include <cmath>

namespace bt {

struct DFloat {
    float h, l;
};

__host__ __device__ __forceinline__ float xf_add(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}

__host__ __device__ __forceinline__ float xf_sub(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}

__host__ __device__ __forceinline__ float xf_mul(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}

__host__ __device__ __forceinline__ float xf_fma(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}

// x = hi + lo
__host__ __device__ __forceinline__ DFloat xf_split(double x)
{
#ifdef __CUDA_ARCH__
    const float h = __double2float_rn(x);
    const float l = __double2float_rn(__dsub_rn(x, (double)h));
#else
    const float h = (float)x;
    const float l = (float)(x - (double)h);
#endif
    return DFloat{h, l};
}

// Entry k of the translation of T^-1 for a 3x4 pose T: -(R^T t)_k, FP64
// with fused multiply-adds in a fixed order.
__host__ __device__ __forceinline__ double xf_inv_translation(const double* T, int k)
{
    return -fma(T[2 * 4 + k], T[11], fma(T[1 * 4 + k], T[7], T[0 * 4 + k] * T[3]));
}

// sum_k a[k] b[k] (k < 3), plus a[3] when add_t, as a double-float dot
// product rounded once to single precision.
__host__ __device__ __forceinline__ float xf_entry(const DFloat* a, const DFloat* b, bool add_t)
{
    float sh = xf_mul(a[0].h, b[0].h);
    float sl = xf_add(xf_fma(a[0].h, b[0].h, -sh), xf_fma(a[0].h, b[0].l, xf_mul(a[0].l, b[0].h)));
    for (int k = 1; k < 3; ++k) {
        const float p = xf_mul(a[k].h, b[k].h);
        const float pe = xf_add(xf_fma(a[k].h, b[k].h, -p), xf_fma(a[k].h, b[k].l, xf_mul(a[k].l, b[k].h)));
        const float s = xf_add(sh, p);
        const float bb = xf_sub(s, sh);
        const float e = xf_add(xf_sub(sh, xf_sub(s, bb)), xf_sub(p, bb));
        sh = s;
        sl = xf_add(sl, xf_add(e, pe));
    }
    if (add_t) {
        const float s = xf_add(sh, a[3].h);
        const float bb = xf_sub(s, sh);
        const float e = xf_add(xf_sub(sh, xf_sub(s, bb)), xf_sub(a[3].h, bb));
        sh = s;
        sl = xf_add(sl, xf_add(e, a[3].l));
    }
    return xf_add(sh, sl);
}

// The splits of one pose T (entries 0-11) and of its inverse's translation
// (entries 12-14): hi at sp[k], lo at sp[16 + k] (32 floats a pose).
constexpr int kXfSplit = 32;

__host__ __device__ __forceinline__ void xf_split_entry(const double* T, int k, float* sp)
{
    const DFloat d = xf_split(k < 12 ? T[k] : xf_inv_translation(T, k - 12));
    sp[k] = d.h;
    sp[16 + k] = d.l;
}

// Entry e = 4 r + c of T_j T_i^-1 from the splits of T_j (sj) and T_i (si).
__host__ __device__ __forceinline__ float xf_pair_entry(const float* sj, const float* si, int e)
{
    const int r = e >> 2, c = e & 3;
    DFloat A[4], B[3];
    for (int k = 0; k < 4; ++k) A[k] = DFloat{sj[r * 4 + k], sj[16 + r * 4 + k]};
    for (int k = 0; k < 3; ++k) {
        // column c of T_i^-1: row c of R_i for c < 3, the inverse's translation for c = 3
        const int q = c < 3 ? c * 4 + k : 12 + k;
        B[k] = DFloat{si[q], si[16 + q]};
    }
    return xf_entry(A, B, c == 3);
}

// Entry e = 4 r + c of T_i^-1 rounded to single precision (the leading part
// of its split: the FP64 value rounded once).
__host__ __device__ __forceinline__ float xf_inv_entry(const float* si, int e)
{
    const int r = e >> 2, c = e & 3;
    return c < 3 ? si[c * 4 + r] : si[12 + r];
}

}  // namespace bt
