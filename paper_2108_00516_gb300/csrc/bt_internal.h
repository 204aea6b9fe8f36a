// bt_internal.h -- device data layout and kernel entry points of libbt.
//
// Layout in HBM (all device buffers are owned by a bt_graph):
//   per stored frame (storage precision P of the graph: FP32, BF16 or FP16)
//     tgt   [H*W]  (z, nx, ny, nz) per pixel, read by the projective gather
//                  (Eq. 3).  FP32: float4, z = 0 where the pixel cannot be a
//                  dense target (not masked / no depth / no normal), 16 B.
//                  BF16/FP16: 4 x 16 bit (z - zref, nx, ny, nz), z - zref =
//                  NaN where invalid, 8 B; zref = the frame's mean valid depth
//     src_p [M]    back-projected source points of the M valid masked pixels,
//                  increasing pixel order: float4 (px, py, pz, 0) or
//                  4 x 16 bit (px, py, pz - zref, 0)
//     src_n [M]    their normals: float4 (nx, ny, nz, 0) or 4 x 16 bit
//   per correspondence set (unordered frame pair)
//     pa, pb float[3*count]  the two camera-frame point lists of Eq. 2
//   per solve (active node set of N nodes)
//     NodeDev[N], EdgeDev[E], tile_node[T], pose double[N][12] (3x4),
//     xf PairXf[N*N] (float camera i -> camera j), xinv float[N][12] (T^-1),
//     dpart float[T][N-1][32] (per source tile and target: the 21 + 6 unique
//     J^T W J / J^T W r terms, cost, count), spart float[E][40] (sparse
//     moments), upairblk double[U][96] (per unordered node pair: its combined
//     FP64 contributions to H and g), control words.
#pragma once

#include "bt.h"

#include <cstdint>
#include <cuda_runtime.h>

namespace bt {

constexpr int kThreads = 256;                 // reduce CTAs, sparse CTAs, prep CTAs
constexpr int kPixPerThread = 4;              // prep
// Dense residual CTA shapes (threads x source pixels per thread); the tile of
// a CTA is their product.  A thread takes its pixels of one target in
// batches of up to 4 (the gathers of a batch are in flight together) and
// reduces its sums across the warp once per target, so more pixels per
// thread spread that reduction over more pixel pairs.  Shape
// BT_SINGLE_GRAPH_SHAPE (256 x 4) is the single-graph path's; the batched
// solver's autotuner picks among all of them.
constexpr int kNumShapes = 6;     // BT_NUM_SHAPES
constexpr int kSingleShape = BT_SINGLE_GRAPH_SHAPE;   // CTA shape of the single-graph solve (bt_solve)
constexpr int kShapeThreads[kNumShapes] = {128, 128, 256, 64, 64, 32};
constexpr int kShapePix[kNumShapes] = {4, 2, 4, 4, 8, 16};
constexpr int kResThreads = 128;              // sparse CTAs of the residual launch
constexpr int kMaxTile = 1024;
constexpr int kDenseVals = 32;                // 21 H + 6 g + cost + count + 3 pad
constexpr int kSparseVals = 40;               // 39 moments + pad
// per unordered pair {a < b}: [0..20] D_a (upper 6x6), [21..41] D_b, [42..77]
// O_ab (rows of a, columns of b), [78..83] g_a, [84..89] g_b, [90] dense
// cost, [91] sparse cost, [92] dense count
constexpr int kUPairBlk = 96;
constexpr int kMaxNodes = 24;
constexpr int kPrepPix = 1024;                // pixels per prep CTA (256 threads x 4)

struct NodeDev {
    const void* src_p;
    const void* src_n;
    const void* tgt;
    float zref;     // reference depth of the 16-bit encodings (0 for FP32)
    int M;          // valid source pixels
    int W, H;
    float fx, fy, cx, cy, ifx, ify;
    int tile0, ntiles;
    int free_idx;   // index among non-fixed nodes, -1 if fixed
};

struct EdgeDev {
    int i, j;       // node indices, i != j; pa lives in camera i, pb in camera j
    int count;
    const float* pa;
    const float* pb;
};

struct Control {
    unsigned int counter;   // last-block detection of the reduce kernel
    int status;             // 0 ok, -4 singular (sticky for the solve)
    unsigned checked;       // BT_CHECKED builds: bits of the index checks that failed (kChk*)
    int pad;
    // SM clock cycles spent by the last CTA, summed over the solve's
    // iterations: [0] gather + assembly, [1] factorisation (with forward
    // substitution), [2] back substitution, [3] pose update + transforms
    unsigned long long clk[4];
};

constexpr size_t kReduceSmemMax = 226 * 1024;   // of the 227 KB a CTA may opt into (1 KB left for static shared memory)

struct SolveArgs {
    int N, n_tiles, n_pairs, n_edges, n_free, n_upairs;
    int precision;          // storage precision of the per-pixel maps (BT_FP32 / BT_BF16 / BT_FP16)
    int tile;               // source pixels per dense tile (CTA shape product)
    int stage_blocks;       // 1: the last CTA copies the pair blocks to shared memory
    float dmax2, cmin, huber_dense, huber_sparse;
    double lambda_dense, lambda_sparse;
    int solver;             // BT_SOLVER_CHOLESKY / BT_SOLVER_PCG
    int pcg_max_iters;
    double pcg_tol2;        // squared relative residual tolerance of PCG
    const NodeDev* nodes;
    const EdgeDev* edges;
    const int* tile_node;
    const int2* upairs;     // [U] (a, b), a < b, lexicographic
    const int* upair_edge;  // [U] correspondence set of the pair or -1
    double* pose;       // [N][12]
    float* xf;          // [N*N][12] camera i -> camera j
    float* xinv;        // [N][12] object <- camera
    float* dpart;       // [T][N-1][32]
    float* spart;       // [E][40]
    double* upairblk;   // [U][96]
    Control* ctrl;
    double* costs;      // [iter][4]: total, dense, sparse, dense count
    double* ne_out;     // NULL, or [n*n + n]: the assembled H and g are written here instead of solving
};

// Bounds-checked build (compiled with -DBT_CHECKED: libbt_checked.so).  The
// residual pass tests every shared-memory, gather and output index it forms
// before the access; a failed test skips the access and sets a bit in the
// solve's control block, which the host reports as BT_ERR_INVALID.  Nothing
// traps.  In the normal build the tests compile to nothing.
constexpr unsigned kChkSourceTile = 1u;    // staged source pixel / normal
constexpr unsigned kChkPipeSlot = 2u;      // per-lane pipeline slot
constexpr unsigned kChkGather = 4u;        // target-map pixel
constexpr unsigned kChkRedSlot = 8u;       // per-warp reduction slot
constexpr unsigned kChkOutput = 16u;       // dpart / spart entry
#ifdef BT_CHECKED
#ifdef __CUDACC__
__device__ __forceinline__ bool index_check(bool ok, unsigned bit, Control* ctrl)
{
    if (!ok) atomicOr(&ctrl->checked, bit);
    return ok;
}
#endif
#define BT_CHECK_IDX(cond, bit, ctrl) (::bt::index_check((cond), (bit), (ctrl)))
#else
#define BT_CHECK_IDX(cond, bit, ctrl) true
#endif

// Programmatic dependent launch.  The kernels of a solve form one chain per
// stream (residual -> reduce -> residual -> ...; the batched solver's chain
// starts with its transform kernel).  Each is
// launched with programmatic stream serialisation: it may be scheduled
// while its predecessor is still running, waits (griddepcontrol.wait) before
// touching anything the predecessor writes, and at once allows its own
// successor to be scheduled (griddepcontrol.launch_dependents), so the
// launch latency of every kernel overlaps the tail of the previous one --
// for the reduce kernel, its single-CTA solve stage.  The wait covers the
// predecessor's completion and memory, and each predecessor waited for its
// own, so every earlier kernel of the chain is complete as well.  Work that
// reads only what earlier kernels (not the predecessor) wrote may run before
// the wait: the residual pass stages its source tiles (frame data) there, and
// the reduce kernel reads the poses and status of the previous update, so
// that their latency overlaps the predecessor's tail.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait_and_release()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                  Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// K0 (frame preparation) for storage precision `precision`.  All launches
// on `s`.  block_scratch must hold prep_scratch_bytes(W*H) bytes; out2[0]
// receives the valid source count (int) and out2[1] the reference depth
// (float bits).  tgt / src_p / src_n are sized for the precision.
size_t prep_scratch_bytes(int HW);
inline size_t pixel_bytes(int precision) { return precision == 0 ? 16 : 8; }
cudaError_t launch_prep(const float* depth, const float* normals, const uint8_t* mask,
                        int W, int H, float cx, float cy, float ifx, float ify, int precision,
                        void* tgt, void* src_p, void* src_n, void* block_scratch,
                        int* out2, int* host_out2, cudaStream_t s);

// One residual pass (dense tiles + sparse edges) and one reduce/solve pass.
// full = true: Gauss-Newton iteration `iter` (records E before the update);
// full = false: cost only, recorded at slot `iter`.
cudaError_t launch_residual(const SolveArgs& a, bool full, cudaStream_t s, int shape = kSingleShape);
cudaError_t launch_reduce(const SolveArgs& a, bool full, int iter, cudaStream_t s);

// Diagnostic export: target pixel (or -1) of every source entry of node i
// against node j at the current transforms (out: device, nodes[i].M ints).
cudaError_t launch_assoc_debug(const SolveArgs& a, int i, int j, int M, int* out, cudaStream_t s);

size_t reduce_smem_bytes(int n_free, int N);
bool reduce_stage_fits(int n_free, int N);
size_t residual_smem_bytes(int N, int shape);
inline int shape_tile(int shape) { return kShapeThreads[shape] * kShapePix[shape]; }

// Batched solver: one launch each per Gauss-Newton iteration over every graph.
//   work_res: (graph, item) per residual CTA, item < n_edges = correspondence
//             set, else dense tile item - n_edges
//   work_pair: (graph, unordered pair) per pair-reduction CTA
cudaError_t launch_batch_xforms(const SolveArgs* args_dev, int n_graphs, cudaStream_t s);
cudaError_t launch_batch_residual(const SolveArgs* args_dev, const int2* work_res, int n_work, int max_N,
                                  bool full, int shape, int precision, cudaStream_t s);
cudaError_t launch_batch_pairs(const SolveArgs* args_dev, const int2* work_pair, int n_work, bool full,
                               cudaStream_t s);
cudaError_t launch_batch_solve(const SolveArgs* args_dev, int n_graphs, size_t smem, bool full, int iter,
                               cudaStream_t s);
// Sets every kernel's shared-memory attribute (call before a stream capture).
void prepare_launch_attributes();
void prepare_residual_attributes();

}  // namespace bt
