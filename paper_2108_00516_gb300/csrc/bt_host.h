// bt_host.h -- host-side state of libbt shared by its translation units
// (graphs, batches, device buffers, error reporting).  Private to the library.
#pragma once

#include "bt.h"
#include "bt_internal.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

namespace bthost {

// Message of the calling thread's last failure (returned by bt_last_error).
std::string& last_error();


inline int fail(int code, const std::string& msg)
{
    last_error() = msg;
    return code;
}

inline int cuda_fail(cudaError_t e, const char* what)
{
    last_error() = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? BT_ERR_OOM : BT_ERR_CUDA;
}

#define BT_CUDA(call, what)                         \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes)
    {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = std::max<size_t>(bytes, 256);
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// Device blocks recycled within one graph: a freed buffer goes back to the
// free list of its size class and is handed out again in stream order (all
// of a graph's work runs on its stream, and batch and warm-start calls
// synchronise before returning), so a steady turnover of frames and
// correspondence sets neither allocates nor frees -- cudaFree would also
// synchronise the whole device.
struct DevPool {
    std::multimap<size_t, void*> free_blocks;
    std::vector<void*> owned;
    static size_t size_class(size_t bytes)
    {
        const size_t q = bytes <= 65536 ? 256 : 65536;
        return ((std::max<size_t>(bytes, 1) + q - 1) / q) * q;
    }
    cudaError_t get(size_t bytes, void** out)
    {
        const size_t c = size_class(bytes);
        auto it = free_blocks.find(c);
        if (it != free_blocks.end()) {
            *out = it->second;
            free_blocks.erase(it);
            return cudaSuccess;
        }
        cudaError_t e = cudaMalloc(out, c);
        if (e == cudaSuccess) owned.push_back(*out);
        else *out = nullptr;
        return e;
    }
    void put(void* p, size_t bytes)
    {
        if (p) free_blocks.emplace(size_class(bytes), p);
    }
    void release()
    {
        for (void* p : owned) cudaFree(p);
        owned.clear();
        free_blocks.clear();
    }
};

struct Frame {
    int id = -1;
    bt_intrinsics K{};
    int fixed = 0;
    double pose[16];
    void* tgt = nullptr;     // target map, element size bt::pixel_bytes(precision)
    void* src_p = nullptr;   // source points (room for every pixel; the first M are used)
    void* src_n = nullptr;   // source normals
    size_t tgt_bytes = 0, src_bytes = 0;
    float zref = 0.f;        // reference depth of the 16-bit encodings
    int M = 0;               // valid source pixels (known once `pending` is resolved)
    int* dev_m2 = nullptr;   // device (M, zref bits) written by the prep kernels
    int slot = -1;           // pinned host slot receiving dev_m2
    bool pending = false;    // M / zref not read back yet
};

struct MatchSet {
    int fa = -1, fb = -1;   // fa < fb; pa in camera fa, pb in camera fb
    int count = 0;
    float* pa = nullptr;
    float* pb = nullptr;
};


inline bool finite_pose(const double* T)
{
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(T[k])) return false;
    return T[12] == 0.0 && T[13] == 0.0 && T[14] == 0.0 && T[15] == 1.0;
}


}  // namespace bthost

struct bt_graph {
    bt_config cfg{};
    cudaStream_t stream = nullptr;
    int next_id = 0;
    std::map<int, bthost::Frame> frames;
    std::map<std::pair<int, int>, bthost::MatchSet> matches;
    std::vector<int> active;
    bool topo_dirty = true;

    // scratch for uploads and frame preparation
    bthost::DevBuf up_depth, up_normals, up_mask, prep_blk;
    bthost::DevPool pool;               // frame maps, source lists, correspondence sets
    int* pin_m2 = nullptr;              // pinned host slots [cap][2] for (M, zref) read-backs
    int pin_cap = 0;
    std::vector<int> free_slots;

    // per-solve state
    bthost::DevBuf d_nodes, d_edges, d_tile_node, d_upairs, d_upair_edge, d_pose, d_xf, d_xinv, d_dpart,
        d_spart, d_upairblk, d_ctrl, d_costs;
    bt::SolveArgs args{};
    int64_t pixels_per_pass = 0;
    int64_t sparse_per_pass = 0;
    int built_tile = 0;     // tile size the current tables were built for
    std::vector<double> pose_stage;   // host staging of poses for batched uploads

    // profiling
    bt_profile prof{};
    bool prof_on = false;
    std::vector<cudaEvent_t> events;

    ~bt_graph()
    {
        if (stream) cudaStreamSynchronize(stream);
        else cudaDeviceSynchronize();
        pool.release();
        if (pin_m2) cudaFreeHost(pin_m2);
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        for (bthost::DevBuf* b : {&up_depth, &up_normals, &up_mask, &prep_blk, &d_nodes, &d_edges, &d_tile_node,
                          &d_upairs, &d_upair_edge, &d_pose, &d_xf, &d_xinv, &d_dpart, &d_spart, &d_upairblk,
                          &d_ctrl, &d_costs})
            b->release();
    }
};

struct bt_batch {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<bt_graph*> graphs;
    int shape = -1;          // fixed CTA shape, or -1 = autotune
    int precision = -1;      // storage precision shared by every graph of the batch
    int tuned_shape = -1;    // autotuner's choice for the current graph set
    bool dirty = true;       // graph set / topology changed since the last build
    bthost::DevBuf d_args, d_work_res, d_work_pair;
    int n_work_res = 0, n_work_pair = 0, max_N = 1;
    size_t solve_smem = 0;
    int64_t pixels_per_pass = 0;
    cudaGraphExec_t exec = nullptr;
    int exec_iters = -1, exec_shape = -1;
    std::vector<double> tune_us;   // autotuner timings per shape (microseconds)

    ~bt_batch()
    {
        if (stream) cudaStreamSynchronize(stream);
        if (exec) cudaGraphExecDestroy(exec);
        d_args.release();
        d_work_res.release();
        d_work_pair.release();
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace bthost {

// Builds the graph's device tables (nodes, dense tiles of `tile` source
// pixels, correspondence sets, node pairs) for its active nodes.
int build_topology(bt_graph* g, int tile);
// Reads back (M, zref) of every frame whose preparation is still pending
// (one stream synchronisation for all of them).
int resolve_pending(bt_graph* g);
// Uploads the active nodes' stored poses, clears the control words and
// launches the float transforms of a new solve.
int upload_poses(bt_graph* g, std::vector<double>& staging);

}  // namespace bthost
