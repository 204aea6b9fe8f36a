// bt_assoc.cuh -- the per-pixel projective association of Eq. 3 (Sec. IV-D)
// in the form the GPU kernels evaluate it: projection of a source point into
// the target camera, nearest pixel and image bounds, then the point-pair
// distance and normal-angle gates and the point-to-plane residual.  Shared by
// the residual pass, its diagnostic export of the association and the
// no-alloc pair energy, so all three take the same decisions.
//
// Arithmetic: single precision with fused multiply-adds and the hardware
// reciprocal; pairs of coordinates go through packed FP32x2 instructions.
// A decision can therefore differ from another single-precision evaluation
// (or from the exact one) only for a pixel whose projection lies within
// rounding of a half-pixel edge or of the image edge, or whose distance or
// angle lies within rounding of its gate.
#pragma once

#include <cuda_runtime.h>

namespace bt {

// Constants of one ordered pair, source camera i -> target camera j, with
// M = T_j T_i^-1 (3x4, single precision).
struct PairK {
    float2 c0, c1, c2, c3;      // rows 0 and 1 of M by column: (M00, M10), (M01, M11), (M02, M12), (M03, M13)
    float m20, m21, m22, m23;   // row 2
    float2 f;                   // (fx, fy) of camera j
    float2 ch;                  // (cx + 1/2, cy + 1/2): nearest pixel = floor(pi(q) + 1/2)
    float2 ifc;                 // (1/fx, 1/fy)
    float2 cif;                 // (-cx/fx, -cy/fy)
    int W, H;
};

__host__ __device__ __forceinline__ PairK make_pair_k(const float* m, float fx, float fy, float cx, float cy,
                                                       float ifx, float ify, int W, int H)
{
    PairK k;
    k.c0 = make_float2(m[0], m[4]);
    k.c1 = make_float2(m[1], m[5]);
    k.c2 = make_float2(m[2], m[6]);
    k.c3 = make_float2(m[3], m[7]);
    k.m20 = m[8];
    k.m21 = m[9];
    k.m22 = m[10];
    k.m23 = m[11];
    k.f = make_float2(fx, fy);
    k.ch = make_float2(cx + 0.5f, cy + 0.5f);
    k.ifc = make_float2(ifx, ify);
    k.cif = make_float2(-cx * ifx, -cy * ify);
    k.W = W;
    k.H = H;
    return k;
}

#ifdef __CUDACC__
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// q = M p and the nearest pixel (iu, iv) of its projection.  True when
// q_z > 1e-30 m and the pixel lies in the image.  Above 1e-30 the
// reciprocal of q_z is finite, so the projected coordinates are finite and
// their floor converts exactly or saturates to a value out of range.
__device__ __forceinline__ bool assoc_project(const PairK& k, float px, float py, float pz, float2& qxy, float& qz,
                                              int& iu, int& iv)
{
    qxy = __ffma2_rn(k.c0, make_float2(px, px), k.c3);
    qxy = __ffma2_rn(k.c1, make_float2(py, py), qxy);
    qxy = __ffma2_rn(k.c2, make_float2(pz, pz), qxy);
    qz = fmaf(k.m22, pz, fmaf(k.m21, py, fmaf(k.m20, px, k.m23)));
    const float rz = rcp_approx(qz);
    const float2 uv = __ffma2_rn(__fmul2_rn(qxy, k.f), make_float2(rz, rz), k.ch);
    iu = __float2int_rd(uv.x);
    iv = __float2int_rd(uv.y);
    return qz > 1e-30f && (unsigned)iu < (unsigned)k.W && (unsigned)iv < (unsigned)k.H;
}

// Distance gate against the looked-up target pixel (iu, iv) with depth tz > 0:
// t = pi_D^-1(iu, iv) in camera j, d = t - q; true when |d|^2 <= dmax2.
__device__ __forceinline__ bool assoc_distance(const PairK& k, int iu, int iv, float tz, float2 qxy, float qz,
                                               float dmax2, float2& txy, float2& dxy, float& dz)
{
    txy = __fmul2_rn(__ffma2_rn(make_float2((float)iu, (float)iv), k.ifc, k.cif), make_float2(tz, tz));
    dxy = __ffma2_rn(qxy, make_float2(-1.f, -1.f), txy);
    dz = tz - qz;
    return fmaf(dz, dz, fmaf(dxy.y, dxy.y, dxy.x * dxy.x)) <= dmax2;
}

// Normal gate: the source normal n_s rotated into camera j (n' = R n_s)
// against the target normal (tnx, tny, tnz); true when n' . n_t >= cmin
// (unit normals: the cosine of their angle).
__device__ __forceinline__ bool assoc_normal(const PairK& k, float nsx, float nsy, float nsz, float tnx, float tny,
                                             float tnz, float cmin, float2& nxy, float& nz)
{
    nxy = __ffma2_rn(k.c2, make_float2(nsz, nsz),
                     __ffma2_rn(k.c1, make_float2(nsy, nsy), __fmul2_rn(k.c0, make_float2(nsx, nsx))));
    nz = fmaf(k.m22, nsz, fmaf(k.m21, nsy, k.m20 * nsx));
    return fmaf(nz, tnz, fmaf(nxy.y, tny, nxy.x * tnx)) >= cmin;
}

// Point-to-plane residual of Eq. 3 expressed in camera j: r = n' . (t - q).
__device__ __forceinline__ float assoc_residual(float2 nxy, float nz, float2 dxy, float dz)
{
    return fmaf(nxy.x, dxy.x, fmaf(nxy.y, dxy.y, nz * dz));
}
#endif

}  // namespace bt
