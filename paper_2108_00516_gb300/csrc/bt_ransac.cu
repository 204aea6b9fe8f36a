// bt_ransac.cu -- coarse registration of Sec. IV-B on the GPU: RANSAC over
// 3-point samples of a correspondence set (p_k in camera i, q_k in camera j),
// each hypothesis the closed-form least-squares rigid fit, inliers counted
// with the distance threshold delta; the result is the hypothesis with the
// most inliers (ties: the earlier sample), optionally refitted on its
// inliers.
//
//   hypothesis_kernel  one thread per (set, sample): indices from the
//                      counter-based SplitMix64 generator (Steele, Lea, Flood
//                      2014) -- sample h uses counters 16 h, 16 h + 1, ... and
//                      keeps the first three distinct indices value % n --
//                      then the FP64 fit in quaternion form (Horn 1987: the
//                      eigenvector of the largest eigenvalue of a symmetric
//                      4x4 matrix built from the cross-covariance, here by
//                      cyclic Jacobi rotations), the same optimum as the SVD
//                      form of Arun et al. 1987.
//   score_kernel       one warp per (set, sample): the inlier test in IEEE
//                      single precision with a fixed operation order
//                      (u = ((R00 px + R01 py) + R02 pz) + tx, each product
//                      and sum rounded; (ex ex + ey ey) + ez ez < fl(delta^2)),
//                      counts by ballot.
//   select_kernel      one CTA per set: argmax, optional FP64 refit.
#include "bt_host.h"

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

using namespace bthost;

namespace {

struct RSet {
    const float* p;      // [n][3] camera i
    const float* q;      // [n][3] camera j
    int n;
    int pad;
};

// Per hypothesis: R (row-major 3x3), t, as double; valid flag separately.
constexpr int kHyp = 12;

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t counter)
{
    uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Largest-eigenvalue eigenvector of a symmetric 4x4 matrix by cyclic Jacobi
// rotations (FP64).
__device__ void top_eigenvector4(double (&A)[4][4], double (&v)[4])
{
    double V[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) V[r][c] = r == c ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 12; ++sweep) {
        double off = 0.0, dg = 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            dg += A[r][r] * A[r][r];
#pragma unroll
            for (int c = r + 1; c < 4; ++c) off += A[r][c] * A[r][c];
        }
        if (!(off > 1e-30 * dg)) break;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
#pragma unroll
            for (int q = p + 1; q < 4; ++q) {
                const double apq = A[p][q];
                if (apq == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
#pragma unroll
                for (int k = 0; k < 4; ++k) {          // A <- A J (columns p, q)
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {          // A <- J^T A (rows p, q)
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {          // V <- V J
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
        }
    }
    int best = 0;
#pragma unroll
    for (int k = 1; k < 4; ++k)
        if (A[k][k] > A[best][best]) best = k;
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = V[k][best];
}

// Rigid least-squares fit q ~ R p + t from centroids and the cross-covariance
// S_ab = sum (p - p_c)_a (q - q_c)_b (quaternion form).
__device__ void fit_from_moments(const double (&S)[3][3], const double (&pc)[3], const double (&qc)[3], double* out)
{
    const double Sxx = S[0][0], Sxy = S[0][1], Sxz = S[0][2];
    const double Syx = S[1][0], Syy = S[1][1], Syz = S[1][2];
    const double Szx = S[2][0], Szy = S[2][1], Szz = S[2][2];
    double N[4][4] = {{Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx},
                      {Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz},
                      {Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy},
                      {Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz}};
    double v[4];
    top_eigenvector4(N, v);
    const double nrm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
    const double w = v[0] / nrm, x = v[1] / nrm, y = v[2] / nrm, z = v[3] / nrm;
    const double R[9] = {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
                         2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
                         2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)};
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = R[k];
#pragma unroll
    for (int r = 0; r < 3; ++r) out[9 + r] = qc[r] - (R[3 * r] * pc[0] + R[3 * r + 1] * pc[1] + R[3 * r + 2] * pc[2]);
}

__global__ void hypothesis_kernel(const RSet* __restrict__ sets, int H, uint64_t seed, double* __restrict__ hyp,
                                  int* __restrict__ valid)
{
    const int s = blockIdx.y, h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= H) return;
    const RSet S = sets[s];
    const size_t o = (size_t)s * H + h;
    valid[o] = 0;
    if (S.n < 3) return;
    int idx[3];
    int got = 0;
    for (int c = 0; c < 16 && got < 3; ++c) {
        const int k = (int)(splitmix64(seed, 16ull * (uint64_t)h + (uint64_t)c) % (uint64_t)S.n);
        bool dup = false;
        for (int m = 0; m < got; ++m) dup |= idx[m] == k;
        if (!dup) idx[got++] = k;
    }
    if (got < 3) return;
    double p[3][3], q[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            p[m][a] = (double)S.p[3 * idx[m] + a];
            q[m][a] = (double)S.q[3 * idx[m] + a];
        }
    // collinear or coincident sample: no unique rotation
    const double ax = p[1][0] - p[0][0], ay = p[1][1] - p[0][1], az = p[1][2] - p[0][2];
    const double bx = p[2][0] - p[0][0], by = p[2][1] - p[0][1], bz = p[2][2] - p[0][2];
    const double cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
    const double cr = sqrt(cx * cx + cy * cy + cz * cz);
    const double sc = ax * ax + ay * ay + az * az + bx * bx + by * by + bz * bz;
    if (!(cr > 1e-12 * (sc > 1e-30 ? sc : 1e-30))) return;
    double pc[3], qc[3], M[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        pc[a] = (p[0][a] + p[1][a] + p[2][a]) / 3.0;
        qc[a] = (q[0][a] + q[1][a] + q[2][a]) / 3.0;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            double v = 0.0;
#pragma unroll
            for (int m = 0; m < 3; ++m) v += (p[m][a] - pc[a]) * (q[m][b] - qc[b]);
            M[a][b] = v;
        }
    fit_from_moments(M, pc, qc, hyp + o * kHyp);
    valid[o] = 1;
}

// Single-precision inlier test (fixed operation order, no contraction).
__device__ __forceinline__ bool inlier(const float (&R)[9], const float (&t)[3], const float* p, const float* q,
                                       float thr2)
{
    float e2 = 0.f;
    float e[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float u = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[3 * r], p[0]), __fmul_rn(R[3 * r + 1], p[1])),
                                            __fmul_rn(R[3 * r + 2], p[2])),
                                  t[r]);
        e[r] = __fsub_rn(u, q[r]);
    }
    e2 = __fadd_rn(__fadd_rn(__fmul_rn(e[0], e[0]), __fmul_rn(e[1], e[1])), __fmul_rn(e[2], e[2]));
    return e2 < thr2;
}

__global__ void score_kernel(const RSet* __restrict__ sets, int H, const double* __restrict__ hyp,
                             const int* __restrict__ valid, float thr2, int* __restrict__ count)
{
    const int s = blockIdx.y;
    const int h = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (h >= H) return;
    const size_t o = (size_t)s * H + h;
    if (!valid[o]) {
        if (lane == 0) count[o] = -1;
        return;
    }
    const RSet S = sets[s];
    float R[9], t[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = (float)hyp[o * kHyp + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = (float)hyp[o * kHyp + 9 + k];
    int c = 0;
    for (int k0 = 0; k0 < S.n; k0 += 32) {
        const int k = k0 + lane;
        bool in = false;
        if (k < S.n) in = inlier(R, t, S.p + 3 * k, S.q + 3 * k, thr2);
        c += __popc(__ballot_sync(0xffffffffu, in));
    }
    if (lane == 0) count[o] = c;
}

// One CTA per set: the best hypothesis (most inliers, then lowest index) and,
// with refine, the FP64 fit on its inliers.  out: [set][16]: R (9), t (3),
// inlier count, best sample index (as doubles), 2 unused.
__global__ void select_kernel(const RSet* __restrict__ sets, int H, const double* __restrict__ hyp,
                              const int* __restrict__ count, float thr2, int refine, double* __restrict__ out)
{
    __shared__ int sc[256], sh[256];
    __shared__ double red[8][16];
    const int s = blockIdx.x, tid = threadIdx.x;
    int bc = -1, bh = -1;
    for (int h = tid; h < H; h += blockDim.x) {
        const int c = count[(size_t)s * H + h];
        if (c > bc) {            // h increases: ties keep the earlier sample
            bc = c;
            bh = h;
        }
    }
    sc[tid] = bc;
    sh[tid] = bh;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (tid < w) {
            const int c2 = sc[tid + w], h2 = sh[tid + w];
            if (c2 > sc[tid] || (c2 == sc[tid] && c2 >= 0 && (sh[tid] < 0 || h2 < sh[tid]))) {
                sc[tid] = c2;
                sh[tid] = h2;
            }
        }
        __syncthreads();
    }
    const int best = sh[0], bestc = sc[0];
    double* o = out + (size_t)s * 16;
    if (best < 0 || bestc < 0) {
        if (tid == 0) {
            for (int k = 0; k < 16; ++k) o[k] = 0.0;
            o[0] = o[4] = o[8] = 1.0;
            o[12] = 0.0;
            o[13] = -1.0;
        }
        return;
    }
    const double* hb = hyp + ((size_t)s * H + best) * kHyp;
    if (!refine) {
        if (tid < 12) o[tid] = hb[tid];
        if (tid == 0) {
            o[12] = bestc;
            o[13] = best;
        }
        return;
    }
    // refit on the inliers of the best sample: FP64 moments over the inliers
    const RSet S = sets[s];
    float R[9], t[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = (float)hb[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = (float)hb[9 + k];
    double m[16];    // [0] count, [1..3] sum p, [4..6] sum q, [7..15] sum p q^T (row-major)
#pragma unroll
    for (int k = 0; k < 16; ++k) m[k] = 0.0;
    for (int k = tid; k < S.n; k += blockDim.x) {
        if (!inlier(R, t, S.p + 3 * k, S.q + 3 * k, thr2)) continue;
        const double pv[3] = {S.p[3 * k], S.p[3 * k + 1], S.p[3 * k + 2]};
        const double qv[3] = {S.q[3 * k], S.q[3 * k + 1], S.q[3 * k + 2]};
        m[0] += 1.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            m[1 + a] += pv[a];
            m[4 + a] += qv[a];
#pragma unroll
            for (int b = 0; b < 3; ++b) m[7 + 3 * a + b] += pv[a] * qv[b];
        }
    }
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        double v = m[k];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double T[16];
        for (int k = 0; k < 16; ++k) {
            T[k] = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) T[k] += red[w][k];
        }
        const double n = T[0];
        if (n >= 3.0) {
            const double pc[3] = {T[1] / n, T[2] / n, T[3] / n};
            const double qc[3] = {T[4] / n, T[5] / n, T[6] / n};
            double M[3][3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) M[a][b] = T[7 + 3 * a + b] - n * pc[a] * qc[b];
            fit_from_moments(M, pc, qc, o);
        } else {
            for (int k = 0; k < 12; ++k) o[k] = hb[k];
        }
        o[12] = bestc;
        o[13] = best;
    }
}

struct Scratch {
    DevBuf sets, hyp, valid, count, out;
};

int run_ransac(const std::vector<RSet>& sets, int H, uint64_t seed, double delta, int refine, cudaStream_t st,
               std::vector<double>& out)
{
    const int S = (int)sets.size();
    out.assign(16 * (size_t)S, 0.0);
    if (S == 0) return BT_OK;
    Scratch sc;
    auto cleanup = [&]() {
        for (DevBuf* b : {&sc.sets, &sc.hyp, &sc.valid, &sc.count, &sc.out}) b->release();
    };
    cudaError_t e = sc.sets.ensure(sizeof(RSet) * S);
    if (e == cudaSuccess) e = sc.hyp.ensure(sizeof(double) * kHyp * (size_t)S * H);
    if (e == cudaSuccess) e = sc.valid.ensure(sizeof(int) * (size_t)S * H);
    if (e == cudaSuccess) e = sc.count.ensure(sizeof(int) * (size_t)S * H);
    if (e == cudaSuccess) e = sc.out.ensure(sizeof(double) * 16 * (size_t)S);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc.sets.p, sets.data(), sizeof(RSet) * S, cudaMemcpyHostToDevice, st);
    const float thr2 = (float)(delta * delta);
    if (e == cudaSuccess) {
        hypothesis_kernel<<<dim3((H + 127) / 128, S), 128, 0, st>>>(sc.sets.as<RSet>(), H, seed, sc.hyp.as<double>(),
                                                                   sc.valid.as<int>());
        score_kernel<<<dim3((H + 7) / 8, S), 256, 0, st>>>(sc.sets.as<RSet>(), H, sc.hyp.as<double>(),
                                                          sc.valid.as<int>(), thr2, sc.count.as<int>());
        select_kernel<<<S, 256, 0, st>>>(sc.sets.as<RSet>(), H, sc.hyp.as<double>(), sc.count.as<int>(), thr2,
                                         refine, sc.out.as<double>());
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out.data(), sc.out.p, sizeof(double) * 16 * S, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "ransac");
    return BT_OK;
}

void to_pose16(const double* r, double* T)
{
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) T[4 * a + b] = r[3 * a + b];
        T[4 * a + 3] = r[9 + a];
    }
    T[12] = T[13] = T[14] = 0.0;
    T[15] = 1.0;
}

void mul44(const double* A, const double* B, double* C)
{
    double t[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += A[4 * r + k] * B[4 * k + c];
            t[4 * r + c] = s;
        }
    for (int k = 0; k < 16; ++k) C[k] = t[k];
}

void inv44(const double* A, double* C)
{
    double t[16] = {0};
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) t[4 * r + c] = A[4 * c + r];
        t[4 * r + 3] = -(A[4 * 0 + r] * A[3] + A[4 * 1 + r] * A[7] + A[4 * 2 + r] * A[11]);
    }
    t[15] = 1.0;
    for (int k = 0; k < 16; ++k) C[k] = t[k];
}

}  // namespace

extern "C" {

int bt_ransac(const float* pts_i, const float* pts_j, int32_t count, int32_t mem_kind, int32_t hypotheses,
              uint64_t seed, double inlier_dist, int32_t refine, double* rel_out, int32_t* inliers_out,
              void* cuda_stream)
{
    NvtxRange nvtx_range("bt_ransac");
    last_error().clear();
    if (!rel_out || (count > 0 && (!pts_i || !pts_j))) return fail(BT_ERR_INVALID, "bt_ransac: NULL argument");
    if (count < 0 || hypotheses < 1 || hypotheses > (1 << 20) || !(inlier_dist > 0.0) || !std::isfinite(inlier_dist))
        return fail(BT_ERR_INVALID, "bt_ransac: bad count, hypotheses or inlier_dist");
    if (mem_kind != BT_HOST && mem_kind != BT_DEVICE) return fail(BT_ERR_INVALID, "bt_ransac: mem_kind");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    float* dp = nullptr;
    float* dq = nullptr;
    const size_t bytes = sizeof(float) * 3 * (size_t)(count > 0 ? count : 1);
    if (mem_kind == BT_HOST) {
        BT_CUDA(alloc_should_fail() ? cudaErrorMemoryAllocation : cudaMalloc(&dp, bytes), "cudaMalloc(ransac points)");
        cudaError_t e = alloc_should_fail() ? cudaErrorMemoryAllocation : cudaMalloc(&dq, bytes);
        if (e == cudaSuccess && count > 0) e = cudaMemcpyAsync(dp, pts_i, bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && count > 0) e = cudaMemcpyAsync(dq, pts_j, bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            cudaFree(dp);
            cudaFree(dq);
            return cuda_fail(e, "upload ransac points");
        }
    }
    std::vector<RSet> sets(1);
    sets[0].p = mem_kind == BT_HOST ? dp : pts_i;
    sets[0].q = mem_kind == BT_HOST ? dq : pts_j;
    sets[0].n = count;
    std::vector<double> out;
    int stt = run_ransac(sets, hypotheses, seed, inlier_dist, refine, st, out);
    if (mem_kind == BT_HOST) {
        cudaFree(dp);
        cudaFree(dq);
    }
    if (stt != BT_OK) return stt;
    to_pose16(out.data(), rel_out);
    if (inliers_out) *inliers_out = (int32_t)out[12];
    return BT_OK;
}

int bt_ransac_init(bt_graph* g, int32_t hypotheses, uint64_t seed, double inlier_dist, int32_t refine)
{
    NvtxRange nvtx_range("bt_ransac_init");
    last_error().clear();
    if (!g) return fail(BT_ERR_INVALID, "bt_ransac_init: NULL graph");
    if (hypotheses < 1 || hypotheses > (1 << 20) || !(inlier_dist > 0.0) || !std::isfinite(inlier_dist))
        return fail(BT_ERR_INVALID, "bt_ransac_init: bad hypotheses or inlier_dist");
    const int N = (int)g->active.size();
    std::vector<int> ids(g->active.begin(), g->active.end());
    // anchor of each free node: its correspondence set with the lowest-indexed fixed node
    std::vector<RSet> sets;
    std::vector<int> node, anchor, fwd;
    for (int j = 0; j < N; ++j) {
        const Frame& fj = g->frames.at(ids[j]);
        if (fj.fixed) continue;
        for (int f = 0; f < N; ++f) {
            const Frame& ff = g->frames.at(ids[f]);
            if (!ff.fixed) continue;
            const int a = ids[f] < ids[j] ? ids[f] : ids[j], b = ids[f] < ids[j] ? ids[j] : ids[f];
            auto it = g->matches.find(std::make_pair(a, b));
            if (it == g->matches.end() || it->second.count <= 0) continue;
            RSet s;
            s.p = it->second.pa;      // camera of the lower frame id
            s.q = it->second.pb;
            s.n = it->second.count;
            s.pad = 0;
            sets.push_back(s);
            node.push_back(j);
            anchor.push_back(f);
            fwd.push_back(ids[f] < ids[j] ? 1 : 0);   // 1: set maps camera f -> camera j
            break;
        }
    }
    if (g->stream) BT_CUDA(cudaStreamSynchronize(g->stream), "bt_ransac_init: sync");
    std::vector<double> out;
    int st = run_ransac(sets, hypotheses, seed, inlier_dist, refine, g->stream, out);
    if (st != BT_OK) return st;
    for (size_t k = 0; k < sets.size(); ++k) {
        double M[16], Mi[16], T[16];
        to_pose16(out.data() + 16 * k, M);
        const double* Tf = g->frames.at(ids[anchor[k]]).pose;
        if (fwd[k]) {
            mul44(M, Tf, T);          // M = T_j T_f^-1
        } else {
            inv44(M, Mi);             // M = T_f T_j^-1
            mul44(Mi, Tf, T);
        }
        std::memcpy(g->frames.at(ids[node[k]]).pose, T, sizeof(double) * 16);
    }
    return BT_OK;
}

}  // extern "C"
