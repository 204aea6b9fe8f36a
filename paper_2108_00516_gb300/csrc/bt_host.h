// bt_host.h -- host-side state of libbt shared by its translation units
// (graphs, batches, device buffers, error reporting).  Private to the library.
#pragma once

#include "bt.h"
#include "bt_internal.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <unordered_map>
#include <vector>

namespace bthost {

// Message of the calling thread's last failure (returned by bt_last_error).
std::string& last_error();

// Allocation-failure injection (bt_debug_fail_allocations): true when the
// allocation about to be made is to fail as out of memory (consumes one
// pending failure).  Every device and pinned host allocation of the library
// asks first.
bool alloc_should_fail();

// A named NVTX range over the rest of the enclosing scope (the library's
// entry points), so that profilers can attribute GPU work to the call that
// enqueued it; costs one test of a function pointer when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};


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
        if (alloc_should_fail()) return cudaErrorMemoryAllocation;
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

// Pinned host memory that stream-ordered copies read from or write to
// asynchronously.  `mark` records an event after the last copy that uses the
// memory; `acquire` waits for that event before the memory is written again
// (or grown), so staging never races a copy still in flight.
struct PinBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool busy = false;
    cudaError_t acquire(size_t bytes)
    {
        if (busy) {
            cudaError_t e = cudaEventSynchronize(done);
            if (e != cudaSuccess) return e;
            busy = false;
        }
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        const size_t want = std::max<size_t>(bytes + bytes / 4, 4096);
        if (alloc_should_fail()) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaHostAlloc(&p, want, cudaHostAllocDefault);
        if (e == cudaSuccess) cap = want;
        else p = nullptr;
        return e;
    }
    cudaError_t mark(cudaStream_t s)
    {
        if (!done) {
            cudaError_t e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaEventRecord(done, s);
        if (e == cudaSuccess) busy = true;
        return e;
    }
    void release()
    {
        if (busy && done) cudaEventSynchronize(done);
        busy = false;
        if (done) cudaEventDestroy(done);
        done = nullptr;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
    template <class T>
    T* at(size_t off) const { return reinterpret_cast<T*>(static_cast<char*>(p) + off); }
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Makes stream `to` wait for the work already enqueued on stream `from`.
inline int order_streams(cudaStream_t from, cudaStream_t to)
{
    if (from == to) return BT_OK;
    cudaEvent_t e;
    BT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    cudaError_t r = cudaEventRecord(e, from);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(to, e, 0);
    cudaEventDestroy(e);
    BT_CUDA(r, "order streams");
    return BT_OK;
}

// One solve's state block on the device: control words, the 3x4 poses of the
// N active nodes, then the energies of every pass (4 doubles each).  A solve
// uploads the leading `upload_bytes` (cleared control words and the starting
// poses) in one copy and reads `readback_bytes(iters)` back in one copy.
struct StateLayout {
    size_t pose = 0, xf = 0, xinv = 0, costs = 0, bytes = 0;
    explicit StateLayout(int N)
    {
        pose = align_up(sizeof(bt::Control), 64);
        // the single-precision pair transforms of the first pass, formed on
        // the host and uploaded with the poses (later passes' are written by
        // the solve kernel in place)
        xf = align_up(pose + sizeof(double) * 12 * (size_t)N, 64);
        xinv = align_up(xf + sizeof(float) * 12 * (size_t)N * N, 64);
        costs = align_up(xinv + sizeof(float) * 12 * (size_t)N, 64);
        bytes = align_up(costs + sizeof(double) * 4 * (BT_MAX_REPORT_ITERS + 1), 256);
    }
    size_t upload_bytes() const { return costs; }
    size_t readback_bytes(int iters) const { return costs + sizeof(double) * 4 * (size_t)(iters + 1); }
};

// Idle device blocks shared by every graph of the process (bt_memory.cu):
// an idle block of size class `cls` on the current device, or a new one;
// and the hand-over of an idle block (its stream synchronised) to the cache.
cudaError_t cache_take(size_t cls, void** out);
void cache_give(int device, size_t cls, void* p);

// Device blocks recycled within one graph: a freed buffer goes back to the
// free list of its size class and is handed out again in stream order (all
// of a graph's work runs on its stream, and batch and warm-start calls
// synchronise before returning), so a steady turnover of frames and
// correspondence sets neither allocates nor frees -- cudaFree would also
// synchronise the whole device.  New blocks come from the process-wide
// cache, and a destroyed graph's blocks go back to it.
struct DevPool {
    std::multimap<size_t, void*> free_blocks;
    std::vector<std::pair<size_t, void*>> owned;   // (size class, block)
    int device = -1;
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
        if (device < 0) {
            cudaError_t e = cudaGetDevice(&device);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = cache_take(c, out);
        if (e == cudaSuccess) owned.emplace_back(c, *out);
        else *out = nullptr;
        return e;
    }
    void put(void* p, size_t bytes)
    {
        if (p) free_blocks.emplace(size_class(bytes), p);
    }
    // Every block back to the process-wide cache; the caller has synchronised
    // the stream that used them.
    void release()
    {
        for (auto& cb : owned) cache_give(device, cb.first, cb.second);
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
    void* mblock = nullptr;  // points of the correspondence sets given with the frame
    size_t mblock_bytes = 0;
};

struct MatchSet {
    int fa = -1, fb = -1;   // fa < fb; pa in camera fa, pb in camera fb
    int count = 0;
    float* pa = nullptr;
    float* pb = nullptr;
    bool owned = true;      // pa, pb are pool blocks of their own; else inside a frame's mblock
};

struct FramePairHash {
    size_t operator()(const std::pair<int, int>& p) const
    {
        return std::hash<uint64_t>()(((uint64_t)(uint32_t)p.first << 32) | (uint32_t)p.second);
    }
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
    std::unordered_map<int, bthost::Frame> frames;   // by frame id (looked up per node on every solve)
    // keyed by the frame pair (a < b); looked up for every node pair of each
    // solve's graph, so hashed rather than ordered
    std::unordered_map<std::pair<int, int>, bthost::MatchSet, bthost::FramePairHash> matches;
    std::unordered_map<int, std::vector<int>> partners;   // frame -> frames it has a correspondence set with
    std::vector<int> active;
    bool topo_dirty = true;

    // scratch for uploads and frame preparation
    bthost::DevBuf up_depth, up_normals, up_mask, prep_blk;
    bthost::DevPool pool;               // frame maps, source lists, correspondence sets
    int* pin_m2 = nullptr;              // pinned host slots [cap][2] for (M, zref) read-backs
    int* pin_m2_dev = nullptr;          // the same slots as the device writes them (mapped)
    int pin_cap = 0;
    std::vector<int> free_slots;

    // per-solve state: the topology tables (nodes, edges, tile owners, node
    // pairs, pair -> edge) in one device block staged through pinned memory,
    // the solve state block (StateLayout) likewise, and the work buffers
    bthost::DevBuf d_tab, d_state, d_dpart, d_spart, d_upairblk;
    bthost::DevBuf d_debug;             // outputs of the diagnostic calls
    bthost::PinBuf pin_tab, pin_state;
    bthost::PinBuf pin_match;           // staging of the correspondence sets given to bt_add_frame
    bt::SolveArgs args{};
    int64_t pixels_per_pass = 0;
    int64_t sparse_per_pass = 0;
    int built_tile = 0;     // tile size the current tables were built for
    uint64_t topo_version = 0;   // incremented by every build of the tables

    // profiling
    bt_profile prof{};
    bool prof_on = false;
    int prof_period = 1;      // event timing on every prof_period-th solve
    int64_t prof_solves = 0;  // solves since profiling was enabled
    bool prof_timed = false;  // the current solve records events
    std::vector<cudaEvent_t> events;

    ~bt_graph()
    {
        if (stream) cudaStreamSynchronize(stream);
        else cudaDeviceSynchronize();
        pool.release();
        if (pin_m2) cudaFreeHost(pin_m2);
        pin_tab.release();
        pin_state.release();
        pin_match.release();
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        for (bthost::DevBuf* b : {&up_depth, &up_normals, &up_mask, &prep_blk, &d_tab, &d_state,
                                  &d_dpart, &d_spart, &d_upairblk, &d_debug})
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
    // solve state of every graph of the batch, one StateLayout block each at
    // state_off[k]: one upload and one read-back per batched solve
    bthost::DevBuf d_state;
    bthost::PinBuf pin_state, pin_tab;
    std::vector<size_t> state_off;
    std::vector<bt::SolveArgs> h_args;   // host copy of d_args
    std::vector<uint64_t> topo_versions; // the graphs' table versions h_args was built from
    uint64_t build_id = 0;               // unique per batch_build in the process (never 0 once built)
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
        d_state.release();
        pin_state.release();
        pin_tab.release();
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace bthost {

// A correspondence set between two active nodes: i = node of m->fa, j = node
// of m->fb.
struct ActiveEdge {
    int i, j;
    const MatchSet* m;
};
// The non-empty correspondence sets among g's active nodes, ordered by their
// frame-id pair (fa, fb).  Looks up the N (N - 1) / 2 active pairs only, so
// the cost does not grow with the number of sets stored in the graph.
std::vector<ActiveEdge> active_edges(const bt_graph* g);

// Builds the graph's device tables (nodes, dense tiles of `tile` source
// pixels, correspondence sets, node pairs) for its active nodes.
int build_topology(bt_graph* g, int tile);
// Reads back (M, zref) of every frame whose preparation is still pending
// (one stream synchronisation for all of them).
int resolve_pending(bt_graph* g);
// Uploads the active nodes' stored poses and cleared control words (one
// copy from pinned staging) and launches the float transforms of a new solve.
int upload_poses(bt_graph* g);
// Writes cleared control words and the stored poses of g's active nodes into
// a state block at `blk` (host memory laid out as StateLayout).
// Cleared control words and the graph's poses into the staging block `blk`;
// with `xforms`, also the first pass's single-precision transforms.
void stage_state(const bt_graph* g, char* blk, bool xforms = false);
// Fills `rep` (when not NULL) from a state block read back after `iters`
// iterations and returns the solve's status (BT_OK or BT_ERR_SINGULAR).
int fill_report(bt_graph* g, const char* blk, int iters, bt_solve_report* rep);

// A batched solve in stages; bt_batch_solve runs them in order, the
// warm-started solve enqueues its network between the upload and the launch.
// Autotuning, tables and the captured CUDA graph (when out of date).
int batch_prepare(bt_batch* b, int iters);
// Cleared control words and the stored poses of every graph, one copy.
int batch_upload_state(bt_batch* b);
// The captured solve and the read-back of every graph's state, one copy.
int batch_launch(bt_batch* b, int iters);
// After the stream is synchronised: reports and the poses of the graphs
// that were not singular; returns BT_OK or BT_ERR_SINGULAR.
int batch_collect(bt_batch* b, int iters, bt_solve_report* reps);

}  // namespace bthost
