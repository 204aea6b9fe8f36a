// bt_noalloc.cu -- bt_pair_dense_energy_noalloc: the dense energy of a frame
// pair for callers that cannot allocate device memory.
//
// It is a variant of the residual pass in cost mode that reads the caller's
// raw depth / normal / mask buffers directly (no prepared target map, no
// compacted source list) and keeps its per-CTA partial sums in one
// file-scope device array instead of graph-owned scratch, so a call performs
// no cudaMalloc, cudaFree or other allocating call.
//
// Scratch: bt_noalloc_scratch, kNoAllocMaxBlocks CTA partials (2 doubles
// each) plus a completion counter, 256-byte aligned, 512 KiB + 256 B in
// total.  Every GPU that loads the library holds it until the process exits.
// Every call shares it and it keeps the last call's contents; the counter is
// cleared at the start of each call.  Calls whose GPU work overlaps (two
// streams, or two host threads) race on it.
#include "bt.h"
#include "bt_assoc.cuh"
#include "bt_xform.cuh"

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocPix = 4;                               // pixels per thread
constexpr int kNoAllocBlockPix = kNoAllocThreads * kNoAllocPix;
constexpr int kNoAllocMaxBlocks = 32768;                     // both directions together
constexpr long long kNoAllocMaxPixels = (long long)(kNoAllocMaxBlocks / 2) * kNoAllocBlockPix;  // per frame

struct NoAllocScratch {
    double partial[kNoAllocMaxBlocks][2];   // per CTA: energy, associations
    unsigned int counter;                   // CTAs finished in this call
};

static __device__ __align__(256) NoAllocScratch bt_noalloc_scratch;

thread_local std::string g_noalloc_err;

// Device address of the scratch array per device, filled on the first call
// made while that device is current.
constexpr int kMaxDevices = 64;
NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

struct Xf {
    bt::PairK kab;   // camera a -> camera b
    bt::PairK kba;   // camera b -> camera a
};

struct View {
    const float* depth;
    const float* normals;
    const uint8_t* mask;
    float fx, fy, cx, cy, ifx, ify;
    int W, H;
};

__device__ __forceinline__ bool valid_px(const View& v, int pix, float& z, float& nx, float& ny, float& nz)
{
    if (!v.mask[pix]) return false;
    z = v.depth[pix];
    if (!(z > 0.f) || !isfinite(z)) return false;
    nx = v.normals[3 * pix];
    ny = v.normals[3 * pix + 1];
    nz = v.normals[3 * pix + 2];
    return isfinite(nx) && isfinite(ny) && isfinite(nz);
}

// One direction per half of the grid: CTAs [0, nb_a) take source frame a and
// target b, CTAs [nb_a, nb_a + nb_b) the reverse.  The association decision
// and the residual are the residual pass's own device functions
// (bt_assoc.cuh); the energy is the Huber sum of the accepted point-to-plane
// residuals times lambda_2.
__global__ void __launch_bounds__(kNoAllocThreads) pair_energy_kernel(
    NoAllocScratch* scr, View va, View vb, Xf xf, int nb_a, float dmax2, float cmin, float hub, double lambda,
    double* out)
{
    __shared__ double red[kNoAllocThreads / 32][2];
    __shared__ int s_last;
    const bool rev = (int)blockIdx.x >= nb_a;
    const View& src = rev ? vb : va;
    const View& dst = rev ? va : vb;
    const bt::PairK& K = rev ? xf.kba : xf.kab;
    const int blk = rev ? blockIdx.x - nb_a : blockIdx.x;
    float e = 0.f, cnt = 0.f;
    const int HW = src.W * src.H;
#pragma unroll
    for (int k = 0; k < kNoAllocPix; ++k) {
        const int pix = blk * kNoAllocBlockPix + k * kNoAllocThreads + threadIdx.x;
        if (pix >= HW) continue;
        float z, nx, ny, nz;
        if (!valid_px(src, pix, z, nx, ny, nz)) continue;
        const int u = pix % src.W, v = pix / src.W;
        // pi_D^-1(x) as the frame preparation of the graph path computes it
        const float px = ((float)u - src.cx) * z * src.ifx;
        const float py = ((float)v - src.cy) * z * src.ify;
        float2 qxy;
        float qz;
        int iu, iv;
        if (!bt::assoc_project(K, px, py, z, qxy, qz, iu, iv)) continue;
        const int tp = iv * dst.W + iu;
        float tz, tnx, tny, tnz;
        if (!valid_px(dst, tp, tz, tnx, tny, tnz)) continue;
        float2 txy, dxy, nxy;
        float dz, nzr;
        if (!bt::assoc_distance(K, iu, iv, tz, qxy, qz, dmax2, txy, dxy, dz)) continue;
        if (!bt::assoc_normal(K, nx, ny, nz, tnx, tny, tnz, cmin, nxy, nzr)) continue;
        const float r = bt::assoc_residual(nxy, nzr, dxy, dz);
        const float ar = fabsf(r);
        e += ar <= hub ? 0.5f * r * r : hub * (ar - 0.5f * hub);
        cnt += 1.f;
    }
    double de = e, dc = cnt;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        de += __shfl_xor_sync(0xffffffffu, de, o);
        dc += __shfl_xor_sync(0xffffffffu, dc, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = de;
        red[threadIdx.x >> 5][1] = dc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < kNoAllocThreads / 32; ++w) {
            s0 += red[w][0];
            s1 += red[w][1];
        }
        scr->partial[blockIdx.x][0] = s0;
        scr->partial[blockIdx.x][1] = s1;
        __threadfence();
        const unsigned t = atomicAdd(&scr->counter, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    // last CTA: fixed-order sum of every CTA's partial (deterministic)
    __threadfence();
    if (threadIdx.x < 32) {
        double s0 = 0.0, s1 = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) {
            s0 += __ldcg(&scr->partial[b][0]);
            s1 += __ldcg(&scr->partial[b][1]);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (threadIdx.x == 0) {
            out[0] = lambda * s0;
            out[1] = s1;
            scr->counter = 0u;
        }
    }
}

int fail(int code, const std::string& msg)
{
    g_noalloc_err = msg;
    return code;
}

// M = T_dst T_src^-1 as the solve kernels form it (bt_xform.cuh: double-float
// arithmetic, the same operations in the same order) -- the same bits.
void pair_transform(const double* Tsrc, const double* Tdst, float* m)
{
    float ss[bt::kXfSplit], sd[bt::kXfSplit];
    for (int k = 0; k < 15; ++k) {
        bt::xf_split_entry(Tsrc, k, ss);
        bt::xf_split_entry(Tdst, k, sd);
    }
    for (int e = 0; e < 12; ++e) m[e] = bt::xf_pair_entry(sd, ss, e);
}

}  // namespace

extern "C" int bt_pair_dense_energy_noalloc(const float* depth_a, const float* normals_a, const uint8_t* mask_a,
                                            const bt_intrinsics* Ka, const double pose_a[16],
                                            const float* depth_b, const float* normals_b, const uint8_t* mask_b,
                                            const bt_intrinsics* Kb, const double pose_b[16], const bt_config* cfg,
                                            double* out, void* cuda_stream)
{
    g_noalloc_err.clear();
    if (!depth_a || !normals_a || !mask_a || !Ka || !pose_a || !depth_b || !normals_b || !mask_b || !Kb ||
        !pose_b || !out)
        return fail(BT_ERR_INVALID, "bt_pair_dense_energy_noalloc: NULL argument");
    for (const bt_intrinsics* K : {Ka, Kb}) {
        if (K->width < 1 || K->height < 1 || K->width > 32767 || K->height > 32767 ||
            (long long)K->width * K->height > kNoAllocMaxPixels)
            return fail(BT_ERR_INVALID, "bt_pair_dense_energy_noalloc: image larger than the fixed scratch allows "
                                        "(at most 16777216 pixels per frame, sides <= 32767)");
        if (!std::isfinite(K->fx) || !std::isfinite(K->fy) || K->fx == 0.f || K->fy == 0.f)
            return fail(BT_ERR_INVALID, "bt_pair_dense_energy_noalloc: bad intrinsics");
    }
    bt_config c;
    bt_config_default(&c);
    if (cfg) c = *cfg;
    if (!(c.huber_dense > 0.0) || !(c.dense_max_dist > 0.0) || !(c.lambda_dense >= 0.0))
        return fail(BT_ERR_INVALID, "bt_pair_dense_energy_noalloc: bad config");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(BT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(BT_ERR_INVALID, "bt_pair_dense_energy_noalloc: device index too large");
    NoAllocScratch* scr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, bt_noalloc_scratch);
            if (e != cudaSuccess)
                return fail(BT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
        }
        scr = g_scratch_ptr[dev];
    }
    auto view = [](const float* d, const float* n, const uint8_t* m, const bt_intrinsics* K) {
        View v;
        v.depth = d;
        v.normals = n;
        v.mask = m;
        v.fx = K->fx; v.fy = K->fy; v.cx = K->cx; v.cy = K->cy;
        v.ifx = 1.0f / K->fx;
        v.ify = 1.0f / K->fy;
        v.W = K->width;
        v.H = K->height;
        return v;
    };
    const View va = view(depth_a, normals_a, mask_a, Ka), vb = view(depth_b, normals_b, mask_b, Kb);
    Xf xf;
    float mab[12], mba[12];
    pair_transform(pose_a, pose_b, mab);
    pair_transform(pose_b, pose_a, mba);
    xf.kab = bt::make_pair_k(mab, vb.fx, vb.fy, vb.cx, vb.cy, vb.ifx, vb.ify, vb.W, vb.H);
    xf.kba = bt::make_pair_k(mba, va.fx, va.fy, va.cx, va.cy, va.ifx, va.ify, va.W, va.H);
    const int nb_a = (Ka->width * Ka->height + kNoAllocBlockPix - 1) / kNoAllocBlockPix;
    const int nb_b = (Kb->width * Kb->height + kNoAllocBlockPix - 1) / kNoAllocBlockPix;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the completion counter must start at zero; the last CTA of a call also
    // resets it, but a call that never ran to completion would leave it set
    e = cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return fail(BT_ERR_CUDA, std::string("clear counter: ") + cudaGetErrorString(e));
    const float dmax2 = (float)(c.dense_max_dist * c.dense_max_dist);
    const float cmin = (float)std::cos(c.dense_max_normal_deg * 3.14159265358979323846 / 180.0);
    pair_energy_kernel<<<nb_a + nb_b, kNoAllocThreads, 0, s>>>(scr, va, vb, xf, nb_a, dmax2, cmin,
                                                             (float)c.huber_dense, c.lambda_dense, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BT_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return BT_OK;
}

extern "C" const char* bt_noalloc_last_error(void) { return g_noalloc_err.c_str(); }
