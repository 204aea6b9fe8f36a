// bt_warmstart_api.cu -- host runtime of the learned warm start (bt_warmstart_*
// in include/bt.h).  A bt_warmstart owns the network parameters (FP32 master
// copy, BF16 copies, Adam moments), a device-resident training set
// (correspondence sets with their initial relative poses and labels) and the
// scratch of its launches; every step runs in the kernels of bt_warmstart.cu.
#include "bt_host.h"
#include "bt_ws.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <new>
#include <vector>

using namespace bthost;
namespace W = bt::ws;

namespace {
// bound of the forward pass's waits on the tensor cores (bt_debug_tensor_wait_ns)
constexpr long long kDefaultTensorWaitNs = 1000000000LL;
std::atomic<long long> g_tensor_wait_ns{kDefaultTensorWaitNs};
}  // namespace

struct bt_warmstart {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevBuf master, wb, m, v;
    bool have_params = false;
    int adam_t = 0;
    // training set
    DevBuf pool_p, pool_q, samples, stage, items;
    int64_t n_points = 0, cap_points = 0;
    int n_samples = 0, cap_samples = 0;
    // launch scratch
    DevBuf ids, y, cache, G, loss_per, grad, loss;
    DevBuf app_samples, app_y, app_graphs, app_scratch, app_status, app_items;
    PinBuf pin_app, pin_status;   // staging of the apply tables and the per-graph status
    // fault word of the forward pass (mapped pinned host memory: the kernel
    // writes it, the host reads it after the call's synchronisation)
    int* fault_host = nullptr;
    int* fault_dev = nullptr;
    // the apply tables on the device were built for this batch build (0:
    // none); a warm-started batched solve of an unchanged batch reuses them
    uint64_t app_build = 0;
    int app_S = 0, app_max_free = 0;

    W::Net net() const
    {
        return W::Net{master.as<float>(), wb.as<__nv_bfloat16>(), m.as<float>(), v.as<float>(), fault_dev,
                      g_tensor_wait_ns.load(std::memory_order_relaxed)};
    }

    ~bt_warmstart()
    {
        if (stream) cudaStreamSynchronize(stream);
        for (DevBuf* b : {&master, &wb, &m, &v, &pool_p, &pool_q, &samples, &stage, &items, &ids, &y, &cache, &G,
                          &loss_per, &grad, &loss, &app_samples, &app_y, &app_graphs, &app_scratch, &app_status,
                          &app_items})
            b->release();
        pin_app.release();
        pin_status.release();
        if (fault_host) cudaFreeHost(fault_host);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

// Grows a device buffer to `bytes`, keeping its first `keep` bytes.
int grow(DevBuf& b, size_t bytes, size_t keep, cudaStream_t s, void** old_out = nullptr)
{
    if (old_out) *old_out = b.p;
    if (bytes <= b.cap) return BT_OK;
    void* p = nullptr;
    BT_CUDA(alloc_should_fail() ? cudaErrorMemoryAllocation : cudaMalloc(&p, bytes), "cudaMalloc(warm-start data)");
    if (keep) BT_CUDA(cudaMemcpyAsync(p, b.p, keep, cudaMemcpyDeviceToDevice, s), "copy warm-start data");
    BT_CUDA(cudaStreamSynchronize(s), "sync warm-start growth");
    if (b.p) cudaFree(b.p);
    b.p = p;
    b.cap = bytes;
    return BT_OK;
}

// Room for `add_pts` more points and `add_sets` more samples; sample point
// pointers are rebased when the pools move.
int reserve(bt_warmstart* ws, int64_t add_pts, int add_sets)
{
    cudaStream_t s = ws->stream;
    if (ws->n_points + add_pts > ws->cap_points) {
        int64_t cap = std::max<int64_t>(ws->cap_points * 2, std::max<int64_t>(ws->n_points + add_pts, 1 << 20));
        void *old_p, *old_q;
        const size_t keep = sizeof(float) * 3 * (size_t)ws->n_points;
        int st = grow(ws->pool_p, sizeof(float) * 3 * (size_t)cap, keep, s, &old_p);
        if (st != BT_OK) return st;
        st = grow(ws->pool_q, sizeof(float) * 3 * (size_t)cap, keep, s, &old_q);
        if (st != BT_OK) return st;
        if (ws->n_samples > 0 && (old_p != ws->pool_p.p || old_q != ws->pool_q.p))
            BT_CUDA(W::launch_rebase(ws->samples.as<W::Sample>(), ws->n_samples, static_cast<const float*>(old_p),
                                     ws->pool_p.as<float>(), static_cast<const float*>(old_q),
                                     ws->pool_q.as<float>(), s),
                    "launch rebase");
        ws->cap_points = cap;
    }
    if (ws->n_samples + add_sets > ws->cap_samples) {
        int cap = std::max(ws->cap_samples * 2, std::max(ws->n_samples + add_sets, 4096));
        int st = grow(ws->samples, sizeof(W::Sample) * (size_t)cap, sizeof(W::Sample) * (size_t)ws->n_samples, s);
        if (st != BT_OK) return st;
        ws->cap_samples = cap;
    }
    return BT_OK;
}

// BT_ERR_TIMEOUT when a forward pass since the last check gave up waiting on
// the tensor cores (its outputs are not valid); clears the fault word.  Call
// after the stream has been synchronised.
int take_fault(bt_warmstart* ws, const char* who)
{
    volatile int* f = ws->fault_host;
    if (*f == 0) return BT_OK;
    *f = 0;
    return fail(BT_ERR_TIMEOUT, std::string(who) +
                                    ": a wait of the network's forward pass on the tensor cores ran out; "
                                    "its outputs were discarded");
}

int check_ready(const bt_warmstart* ws, const char* who)
{
    if (!ws) return fail(BT_ERR_INVALID, std::string(who) + ": NULL warm start");
    if (!ws->have_params) return fail(BT_ERR_STATE, std::string(who) + ": parameters not set");
    return BT_OK;
}

int upload_ids(bt_warmstart* ws, const int32_t* ids, int n)
{
    for (int k = 0; k < n; ++k)
        if (ids[k] < 0 || ids[k] >= ws->n_samples) return fail(BT_ERR_INVALID, "warm start: sample id out of range");
    BT_CUDA(ws->ids.ensure(sizeof(int) * (size_t)std::max(n, 1)), "alloc ids");
    BT_CUDA(cudaMemcpyAsync(ws->ids.p, ids, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, ws->stream),
            "upload ids");
    return BT_OK;
}

// Forward (with cache), backward and reduction over the given samples:
// leaves the mean gradient in ws->grad and the mean loss in ws->loss.
int gradient_pass(bt_warmstart* ws, const int32_t* ids, int n)
{
    int st = upload_ids(ws, ids, n);
    if (st != BT_OK) return st;
    cudaStream_t s = ws->stream;
    BT_CUDA(ws->y.ensure(sizeof(float) * W::kOut * (size_t)n), "alloc y");
    BT_CUDA(ws->cache.ensure(sizeof(W::Cache) * (size_t)n), "alloc cache");
    BT_CUDA(ws->G.ensure(sizeof(float) * W::kNumParams * (size_t)n), "alloc per-set gradients");
    BT_CUDA(ws->loss_per.ensure(sizeof(float) * (size_t)n), "alloc losses");
    BT_CUDA(ws->grad.ensure(sizeof(float) * W::kNumParams), "alloc gradient");
    BT_CUDA(ws->loss.ensure(sizeof(double)), "alloc loss");
    const W::Net net = ws->net();
    const W::Sample* smp = ws->samples.as<W::Sample>();
    const int* d_ids = ws->ids.as<int>();
    BT_CUDA(W::launch_forward(net, smp, d_ids, n, ws->y.as<float>(), ws->cache.as<W::Cache>(), s), "launch forward");
    BT_CUDA(W::launch_backward(net, smp, d_ids, n, ws->cache.as<W::Cache>(), ws->G.as<float>(),
                               ws->loss_per.as<float>(), s),
            "launch backward");
    BT_CUDA(W::launch_reduce(ws->G.as<float>(), ws->loss_per.as<float>(), n, ws->grad.as<float>(),
                             ws->loss.as<double>(), s),
            "launch reduce");
    return BT_OK;
}

// Edges of a graph's active nodes in the order of its device edge table.
struct HostEdge {
    int i, j, count;
    const float* pa;
    const float* pb;
};

std::vector<HostEdge> graph_edges(const bt_graph* g)
{
    std::vector<HostEdge> out;
    for (const ActiveEdge& e : active_edges(g)) out.push_back(HostEdge{e.i, e.j, e.m->count, e.m->pa, e.m->pb});
    return out;
}

int ensure_tables(bt_graph* g)
{
    if (g->active.empty()) return fail(BT_ERR_INVALID, "warm start: graph has no active nodes");
    if (g->topo_dirty || g->built_tile == 0)
        return build_topology(g, g->built_tile > 0 ? g->built_tile : bt::shape_tile(bt::kSingleShape));
    return BT_OK;
}

// Enqueues on stream s the warm start of every graph in `gs` (one launch of
// each kernel for all of them).  pose[k] holds the device poses of graph k's
// active nodes: the network reads the starting relative poses from it and
// the averaging writes the new poses into it.  Graph k's status lands in
// app_status[k] (0 ok; 1 averaging system singular, poses left as they were).
// The graphs' tables must be current.
int launch_apply(bt_warmstart* ws, int S, int n_graphs, int max_free, cudaStream_t s);

int enqueue_apply(bt_warmstart* ws, bt_graph* const* gs, int n_graphs, double* const* pose, cudaStream_t s)
{
    ws->app_build = 0;     // the tables are rewritten below
    std::vector<W::Sample> smp;
    std::vector<W::PrepItem> items;
    std::vector<W::AvgGraph> avg;
    std::vector<int> first(n_graphs + 1, 0);
    int max_free = 0;
    for (int k = 0; k < n_graphs; ++k) {
        bt_graph* g = gs[k];
        const std::vector<HostEdge> edges = graph_edges(g);
        if ((int)edges.size() != g->args.n_edges) return fail(BT_ERR_STATE, "warm start: edge table out of date");
        first[k] = (int)smp.size();
        for (const HostEdge& e : edges) {
            W::Sample x{};
            x.p = e.pa;
            x.q = e.pb;
            x.n = e.count;
            W::PrepItem it{};
            it.sample = (int)smp.size();
            it.Ti0 = pose[k] + 12 * e.i;
            it.Tj0 = pose[k] + 12 * e.j;
            smp.push_back(x);
            items.push_back(it);
        }
        max_free = std::max(max_free, g->args.n_free);
    }
    first[n_graphs] = (int)smp.size();
    const int S = (int)smp.size();
    BT_CUDA(ws->app_samples.ensure(sizeof(W::Sample) * (size_t)std::max(S, 1)), "alloc samples");
    BT_CUDA(ws->app_items.ensure(sizeof(W::PrepItem) * (size_t)std::max(S, 1)), "alloc items");
    BT_CUDA(ws->app_y.ensure(sizeof(float) * W::kOut * (size_t)std::max(S, 1)), "alloc outputs");
    BT_CUDA(ws->app_scratch.ensure(sizeof(double) * W::kAvgScratch * (size_t)std::max(S, 1)), "alloc scratch");
    BT_CUDA(ws->app_graphs.ensure(sizeof(W::AvgGraph) * (size_t)n_graphs), "alloc graphs");
    BT_CUDA(ws->app_status.ensure(sizeof(int) * (size_t)n_graphs), "alloc status");
    for (int k = 0; k < n_graphs; ++k) {
        const bt_graph* g = gs[k];
        W::AvgGraph a{};
        a.N = g->args.N;
        a.n_edges = g->args.n_edges;
        a.n_free = g->args.n_free;
        a.nodes = g->args.nodes;
        a.edges = g->args.edges;
        a.y = ws->app_y.as<float>() + (size_t)first[k] * W::kOut;
        a.smp = ws->app_samples.as<W::Sample>() + first[k];
        a.pose = pose[k];
        a.scratch = ws->app_scratch.as<double>() + (size_t)first[k] * W::kAvgScratch;
        a.status = ws->app_status.as<int>() + k;
        avg.push_back(a);
    }
    // the three tables go up from one pinned staging block
    const size_t o_items = align_up(sizeof(W::Sample) * (size_t)S, 256),
                 o_avg = o_items + align_up(sizeof(W::PrepItem) * (size_t)S, 256),
                 bytes = o_avg + sizeof(W::AvgGraph) * (size_t)n_graphs;
    BT_CUDA(ws->pin_app.acquire(bytes), "cudaHostAlloc(warm-start staging)");
    if (S > 0) {
        std::memcpy(ws->pin_app.p, smp.data(), sizeof(W::Sample) * S);
        std::memcpy(ws->pin_app.at<char>(o_items), items.data(), sizeof(W::PrepItem) * S);
        BT_CUDA(cudaMemcpyAsync(ws->app_samples.p, ws->pin_app.p, sizeof(W::Sample) * S, cudaMemcpyHostToDevice, s),
                "upload samples");
        BT_CUDA(cudaMemcpyAsync(ws->app_items.p, ws->pin_app.at<char>(o_items), sizeof(W::PrepItem) * S,
                                cudaMemcpyHostToDevice, s),
                "upload items");
    }
    std::memcpy(ws->pin_app.at<char>(o_avg), avg.data(), sizeof(W::AvgGraph) * n_graphs);
    BT_CUDA(cudaMemcpyAsync(ws->app_graphs.p, ws->pin_app.at<char>(o_avg), sizeof(W::AvgGraph) * n_graphs,
                            cudaMemcpyHostToDevice, s),
            "upload graphs");
    BT_CUDA(ws->pin_app.mark(s), "record warm-start upload");
    ws->app_S = S;
    ws->app_max_free = max_free;
    return launch_apply(ws, S, n_graphs, max_free, s);
}

// The three launches of a warm start over the apply tables already on the
// device: relative poses and centres from the current poses, the network,
// the averaging.
int launch_apply(bt_warmstart* ws, int S, int n_graphs, int max_free, cudaStream_t s)
{
    W::Sample* d_smp = ws->app_samples.as<W::Sample>();
    BT_CUDA(W::launch_prep(d_smp, ws->app_items.as<W::PrepItem>(), S, s), "launch prep");
    BT_CUDA(W::launch_forward(ws->net(), d_smp, nullptr, S, ws->app_y.as<float>(), nullptr, s), "launch forward");
    BT_CUDA(W::launch_average(ws->app_graphs.as<W::AvgGraph>(), n_graphs, max_free, s), "launch average");
    return BT_OK;
}

// Enqueues the read-back of the per-graph status words into pinned staging.
int read_status(bt_warmstart* ws, int n_graphs, cudaStream_t s)
{
    BT_CUDA(ws->pin_status.acquire(sizeof(int) * (size_t)n_graphs), "cudaHostAlloc(status staging)");
    BT_CUDA(cudaMemcpyAsync(ws->pin_status.p, ws->app_status.p, sizeof(int) * n_graphs, cudaMemcpyDeviceToHost, s),
            "read status");
    BT_CUDA(ws->pin_status.mark(s), "record status read-back");
    return BT_OK;
}

// Predicts and applies the warm start to every graph in `gs`, then stores
// the new poses in the graphs.
int apply_graphs(bt_warmstart* ws, bt_graph* const* gs, int n_graphs, int* status_out)
{
    cudaStream_t s = ws->stream;
    std::vector<double*> pose(n_graphs);
    for (int k = 0; k < n_graphs; ++k) {
        bt_graph* g = gs[k];
        int st = ensure_tables(g);
        if (st != BT_OK) return st;
        st = order_streams(g->stream, s);
        if (st != BT_OK) return st;
        const StateLayout L((int)g->active.size());
        BT_CUDA(g->pin_state.acquire(L.bytes), "cudaHostAlloc(state staging)");
        stage_state(g, g->pin_state.at<char>(0));
        BT_CUDA(cudaMemcpyAsync(g->d_state.p, g->pin_state.p, L.upload_bytes(), cudaMemcpyHostToDevice, s),
                "upload poses");
        pose[k] = g->args.pose;
    }
    int st = enqueue_apply(ws, gs, n_graphs, pose.data(), s);
    if (st != BT_OK) return st;
    for (int k = 0; k < n_graphs; ++k) {
        bt_graph* g = gs[k];
        const StateLayout L(g->args.N);
        BT_CUDA(cudaMemcpyAsync(g->pin_state.at<char>(L.pose), g->args.pose, sizeof(double) * 12 * g->args.N,
                                cudaMemcpyDeviceToHost, s),
                "read poses");
        BT_CUDA(g->pin_state.mark(s), "record pose read-back");
    }
    st = read_status(ws, n_graphs, s);
    if (st != BT_OK) return st;
    BT_CUDA(cudaStreamSynchronize(s), "warm start: synchronize");
    ws->pin_status.busy = false;
    for (int k = 0; k < n_graphs; ++k) gs[k]->pin_state.busy = false;
    st = take_fault(ws, "warm start");
    if (st != BT_OK) {     // no graph's poses are stored
        if (status_out)
            for (int k = 0; k < n_graphs; ++k) status_out[k] = st;
        return st;
    }
    int worst = BT_OK;
    for (int k = 0; k < n_graphs; ++k) {
        bt_graph* g = gs[k];
        const int bad = ws->pin_status.at<int>(0)[k];
        if (status_out) status_out[k] = bad ? BT_ERR_SINGULAR : BT_OK;
        if (bad) {
            worst = BT_ERR_SINGULAR;
            continue;
        }
        const double* P = g->pin_state.at<double>(StateLayout(g->args.N).pose);
        for (int q = 0; q < g->args.N; ++q)
            std::memcpy(g->frames.at(g->active[q]).pose, P + 12 * (size_t)q, sizeof(double) * 12);
    }
    if (worst != BT_OK)
        return fail(worst, "warm start: averaging system not positive definite for some graph; its poses are unchanged");
    return BT_OK;
}

}  // namespace

extern "C" {

int bt_warmstart_create(void* cuda_stream, bt_warmstart** out)
{
    last_error().clear();
    if (!out) return fail(BT_ERR_INVALID, "bt_warmstart_create: NULL out");
    *out = nullptr;
    bt_warmstart* ws = new (std::nothrow) bt_warmstart();
    if (!ws) return fail(BT_ERR_OOM, "bt_warmstart_create: host allocation");
    if (cuda_stream) {
        ws->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&ws->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete ws;
            return cuda_fail(e, "bt_warmstart_create: stream");
        }
        ws->own_stream = true;
    }
    cudaError_t e = cudaSuccess;
    for (DevBuf* b : {&ws->master, &ws->m, &ws->v}) {
        if (e == cudaSuccess) e = b->ensure(sizeof(float) * W::kNumParams);
    }
    if (e == cudaSuccess) e = ws->wb.ensure(sizeof(__nv_bfloat16) * W::kNumBf16);
    if (e == cudaSuccess)
        e = alloc_should_fail() ? cudaErrorMemoryAllocation
                                : cudaHostAlloc(reinterpret_cast<void**>(&ws->fault_host), sizeof(int),
                                                cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *ws->fault_host = 0;
        e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&ws->fault_dev), ws->fault_host, 0);
    }
    if (e != cudaSuccess) {
        delete ws;
        return cuda_fail(e, "bt_warmstart_create: parameters");
    }
    *out = ws;
    return BT_OK;
}

void bt_warmstart_destroy(bt_warmstart* ws) { delete ws; }

int32_t bt_warmstart_num_params(void) { return W::kNumParams; }

int bt_warmstart_set_params(bt_warmstart* ws, const float* params, int32_t mem_kind)
{
    last_error().clear();
    if (!ws || !params) return fail(BT_ERR_INVALID, "bt_warmstart_set_params: NULL argument");
    if (mem_kind != BT_HOST && mem_kind != BT_DEVICE) return fail(BT_ERR_INVALID, "bt_warmstart_set_params: mem_kind");
    if (mem_kind == BT_HOST)
        for (int k = 0; k < W::kNumParams; ++k)
            if (!std::isfinite(params[k])) return fail(BT_ERR_INVALID, "bt_warmstart_set_params: non-finite value");
    cudaStream_t s = ws->stream;
    BT_CUDA(cudaMemcpyAsync(ws->master.p, params, sizeof(float) * W::kNumParams,
                            mem_kind == BT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s),
            "upload parameters");
    BT_CUDA(cudaMemsetAsync(ws->m.p, 0, sizeof(float) * W::kNumParams, s), "clear moments");
    BT_CUDA(cudaMemsetAsync(ws->v.p, 0, sizeof(float) * W::kNumParams, s), "clear moments");
    BT_CUDA(W::launch_to_bf16(ws->net(), s), "launch to_bf16");
    BT_CUDA(cudaStreamSynchronize(s), "bt_warmstart_set_params: synchronize");
    ws->have_params = true;
    ws->adam_t = 0;
    return BT_OK;
}

int bt_warmstart_get_adam(const bt_warmstart* ws, float* m, float* v, int32_t* step, int32_t mem_kind)
{
    last_error().clear();
    int st = check_ready(ws, "bt_warmstart_get_adam");
    if (st != BT_OK) return st;
    if (!m || !v || !step) return fail(BT_ERR_INVALID, "bt_warmstart_get_adam: NULL argument");
    if (mem_kind != BT_HOST && mem_kind != BT_DEVICE) return fail(BT_ERR_INVALID, "bt_warmstart_get_adam: mem_kind");
    const cudaMemcpyKind kind = mem_kind == BT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    BT_CUDA(cudaMemcpyAsync(m, ws->m.p, sizeof(float) * W::kNumParams, kind, ws->stream), "read moments");
    BT_CUDA(cudaMemcpyAsync(v, ws->v.p, sizeof(float) * W::kNumParams, kind, ws->stream), "read moments");
    BT_CUDA(cudaStreamSynchronize(ws->stream), "bt_warmstart_get_adam: synchronize");
    *step = ws->adam_t;
    return BT_OK;
}

int bt_warmstart_set_adam(bt_warmstart* ws, const float* m, const float* v, int32_t step, int32_t mem_kind)
{
    last_error().clear();
    int st = check_ready(ws, "bt_warmstart_set_adam");
    if (st != BT_OK) return st;
    if (!m || !v || step < 0) return fail(BT_ERR_INVALID, "bt_warmstart_set_adam: NULL argument or negative step");
    if (mem_kind != BT_HOST && mem_kind != BT_DEVICE) return fail(BT_ERR_INVALID, "bt_warmstart_set_adam: mem_kind");
    if (mem_kind == BT_HOST)
        for (int k = 0; k < W::kNumParams; ++k)
            if (!std::isfinite(m[k]) || !(v[k] >= 0.f) || !std::isfinite(v[k]))
                return fail(BT_ERR_INVALID, "bt_warmstart_set_adam: non-finite moment or negative second moment");
    const cudaMemcpyKind kind = mem_kind == BT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    BT_CUDA(cudaMemcpyAsync(ws->m.p, m, sizeof(float) * W::kNumParams, kind, ws->stream), "upload moments");
    BT_CUDA(cudaMemcpyAsync(ws->v.p, v, sizeof(float) * W::kNumParams, kind, ws->stream), "upload moments");
    BT_CUDA(cudaStreamSynchronize(ws->stream), "bt_warmstart_set_adam: synchronize");
    ws->adam_t = step;
    return BT_OK;
}

int bt_warmstart_get_params(const bt_warmstart* ws, float* params, int32_t mem_kind)
{
    last_error().clear();
    int st = check_ready(ws, "bt_warmstart_get_params");
    if (st != BT_OK) return st;
    if (!params) return fail(BT_ERR_INVALID, "bt_warmstart_get_params: NULL argument");
    BT_CUDA(cudaMemcpyAsync(params, ws->master.p, sizeof(float) * W::kNumParams,
                            mem_kind == BT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ws->stream),
            "read parameters");
    BT_CUDA(cudaStreamSynchronize(ws->stream), "bt_warmstart_get_params: synchronize");
    return BT_OK;
}

int bt_warmstart_add_set(bt_warmstart* ws, const float* pts_i, const float* pts_j, int32_t count,
                         const double* pose_i, const double* pose_j, const double* label_i, const double* label_j,
                         int32_t mem_kind)
{
    last_error().clear();
    if (!ws || !pts_i || !pts_j || !pose_i || !pose_j) return fail(BT_ERR_INVALID, "bt_warmstart_add_set: NULL argument");
    if (count <= 0) return fail(BT_ERR_INVALID, "bt_warmstart_add_set: count must be > 0");
    if (mem_kind != BT_HOST && mem_kind != BT_DEVICE) return fail(BT_ERR_INVALID, "bt_warmstart_add_set: mem_kind");
    if ((label_i == nullptr) != (label_j == nullptr))
        return fail(BT_ERR_INVALID, "bt_warmstart_add_set: give both label poses or neither");
    if (!finite_pose(pose_i) || !finite_pose(pose_j) || (label_i && (!finite_pose(label_i) || !finite_pose(label_j))))
        return fail(BT_ERR_INVALID, "bt_warmstart_add_set: bad pose");
    int st = reserve(ws, count, 1);
    if (st != BT_OK) return st;
    cudaStream_t s = ws->stream;
    const cudaMemcpyKind kind = mem_kind == BT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    float* dp = ws->pool_p.as<float>() + 3 * ws->n_points;
    float* dq = ws->pool_q.as<float>() + 3 * ws->n_points;
    BT_CUDA(cudaMemcpyAsync(dp, pts_i, sizeof(float) * 3 * (size_t)count, kind, s), "upload points");
    BT_CUDA(cudaMemcpyAsync(dq, pts_j, sizeof(float) * 3 * (size_t)count, kind, s), "upload points");
    W::Sample x{};
    x.p = dp;
    x.q = dq;
    x.n = count;
    BT_CUDA(cudaMemcpyAsync(ws->samples.as<W::Sample>() + ws->n_samples, &x, sizeof(x), cudaMemcpyHostToDevice, s),
            "upload sample");
    double stage[48];
    std::memcpy(stage, pose_i, sizeof(double) * 12);
    std::memcpy(stage + 12, pose_j, sizeof(double) * 12);
    if (label_i) {
        std::memcpy(stage + 24, label_i, sizeof(double) * 12);
        std::memcpy(stage + 36, label_j, sizeof(double) * 12);
    }
    BT_CUDA(ws->stage.ensure(sizeof(stage)), "alloc stage");
    BT_CUDA(ws->items.ensure(sizeof(W::PrepItem)), "alloc items");
    const double* d = ws->stage.as<double>();
    W::PrepItem it{ws->n_samples, 0, d, d + 12, label_i ? d + 24 : nullptr, label_i ? d + 36 : nullptr};
    BT_CUDA(cudaMemcpyAsync(ws->stage.p, stage, sizeof(stage), cudaMemcpyHostToDevice, s), "upload stage");
    BT_CUDA(cudaMemcpyAsync(ws->items.p, &it, sizeof(it), cudaMemcpyHostToDevice, s), "upload item");
    BT_CUDA(W::launch_prep(ws->samples.as<W::Sample>(), ws->items.as<W::PrepItem>(), 1, s), "launch prep");
    BT_CUDA(cudaStreamSynchronize(s), "bt_warmstart_add_set: synchronize");
    ws->n_points += count;
    ws->n_samples += 1;
    return BT_OK;
}

int bt_warmstart_add_graph(bt_warmstart* ws, bt_graph* g, const double* poses_init, const double* poses_label)
{
    last_error().clear();
    if (!ws || !g || !poses_init) return fail(BT_ERR_INVALID, "bt_warmstart_add_graph: NULL argument");
    const int N = (int)g->active.size();
    if (N < 2) return fail(BT_ERR_INVALID, "bt_warmstart_add_graph: fewer than two active nodes");
    for (int k = 0; k < N; ++k)
        if (!finite_pose(poses_init + 16 * k) || (poses_label && !finite_pose(poses_label + 16 * k)))
            return fail(BT_ERR_INVALID, "bt_warmstart_add_graph: bad pose");
    const std::vector<HostEdge> edges = graph_edges(g);
    int64_t pts = 0;
    for (const HostEdge& e : edges) pts += e.count;
    int st = reserve(ws, pts, (int)edges.size());
    if (st != BT_OK) return st;
    if (edges.empty()) return BT_OK;
    cudaStream_t s = ws->stream;
    if (g->stream != s) BT_CUDA(cudaStreamSynchronize(g->stream), "sync graph stream");
    std::vector<double> stage(24 * (size_t)N);
    for (int k = 0; k < N; ++k) {
        std::memcpy(&stage[12 * (size_t)k], poses_init + 16 * k, sizeof(double) * 12);
        if (poses_label) std::memcpy(&stage[12 * ((size_t)N + k)], poses_label + 16 * k, sizeof(double) * 12);
    }
    BT_CUDA(ws->stage.ensure(sizeof(double) * stage.size()), "alloc stage");
    BT_CUDA(ws->items.ensure(sizeof(W::PrepItem) * edges.size()), "alloc items");
    BT_CUDA(cudaMemcpyAsync(ws->stage.p, stage.data(), sizeof(double) * stage.size(), cudaMemcpyHostToDevice, s),
            "upload stage");
    const double* d0 = ws->stage.as<double>();
    const double* d1 = d0 + 12 * (size_t)N;
    std::vector<W::Sample> smp;
    std::vector<W::PrepItem> items;
    int64_t off = ws->n_points;
    for (const HostEdge& e : edges) {
        float* dp = ws->pool_p.as<float>() + 3 * off;
        float* dq = ws->pool_q.as<float>() + 3 * off;
        BT_CUDA(cudaMemcpyAsync(dp, e.pa, sizeof(float) * 3 * (size_t)e.count, cudaMemcpyDeviceToDevice, s), "copy points");
        BT_CUDA(cudaMemcpyAsync(dq, e.pb, sizeof(float) * 3 * (size_t)e.count, cudaMemcpyDeviceToDevice, s), "copy points");
        W::Sample x{};
        x.p = dp;
        x.q = dq;
        x.n = e.count;
        W::PrepItem it{ws->n_samples + (int)smp.size(), 0, d0 + 12 * e.i, d0 + 12 * e.j,
                       poses_label ? d1 + 12 * e.i : nullptr, poses_label ? d1 + 12 * e.j : nullptr};
        smp.push_back(x);
        items.push_back(it);
        off += e.count;
    }
    BT_CUDA(cudaMemcpyAsync(ws->samples.as<W::Sample>() + ws->n_samples, smp.data(), sizeof(W::Sample) * smp.size(),
                            cudaMemcpyHostToDevice, s),
            "upload samples");
    BT_CUDA(cudaMemcpyAsync(ws->items.p, items.data(), sizeof(W::PrepItem) * items.size(), cudaMemcpyHostToDevice, s),
            "upload items");
    BT_CUDA(W::launch_prep(ws->samples.as<W::Sample>(), ws->items.as<W::PrepItem>(), (int)items.size(), s),
            "launch prep");
    BT_CUDA(cudaStreamSynchronize(s), "bt_warmstart_add_graph: synchronize");
    ws->n_points = off;
    ws->n_samples += (int)smp.size();
    return BT_OK;
}

int32_t bt_warmstart_num_samples(const bt_warmstart* ws)
{
    if (!ws) return fail(BT_ERR_INVALID, "bt_warmstart_num_samples: NULL warm start");
    return ws->n_samples;
}

int bt_warmstart_clear_samples(bt_warmstart* ws)
{
    if (!ws) return fail(BT_ERR_INVALID, "bt_warmstart_clear_samples: NULL warm start");
    ws->n_samples = 0;
    ws->n_points = 0;
    return BT_OK;
}

int bt_warmstart_predict(bt_warmstart* ws, const int32_t* ids, int32_t n, float* y_out)
{
    NvtxRange nvtx_range("bt_warmstart_predict");
    last_error().clear();
    int st = check_ready(ws, "bt_warmstart_predict");
    if (st != BT_OK) return st;
    if (n < 0 || (n > 0 && (!ids || !y_out))) return fail(BT_ERR_INVALID, "bt_warmstart_predict: bad arguments");
    if (n == 0) return BT_OK;
    st = upload_ids(ws, ids, n);
    if (st != BT_OK) return st;
    BT_CUDA(ws->y.ensure(sizeof(float) * W::kOut * (size_t)n), "alloc y");
    BT_CUDA(W::launch_forward(ws->net(), ws->samples.as<W::Sample>(), ws->ids.as<int>(), n, ws->y.as<float>(),
                              nullptr, ws->stream),
            "launch forward");
    BT_CUDA(cudaMemcpyAsync(y_out, ws->y.p, sizeof(float) * W::kOut * (size_t)n, cudaMemcpyDeviceToHost, ws->stream),
            "read outputs");
    BT_CUDA(cudaStreamSynchronize(ws->stream), "bt_warmstart_predict: synchronize");
    return take_fault(ws, "bt_warmstart_predict");
}

int bt_warmstart_get_sample(const bt_warmstart* ws, int32_t id, float* centre, float* label)
{
    last_error().clear();
    if (!ws || id < 0 || id >= ws->n_samples) return fail(BT_ERR_INVALID, "bt_warmstart_get_sample: bad id");
    W::Sample x;
    BT_CUDA(cudaMemcpyAsync(&x, ws->samples.as<W::Sample>() + id, sizeof(x), cudaMemcpyDeviceToHost, ws->stream),
            "read sample");
    BT_CUDA(cudaStreamSynchronize(ws->stream), "bt_warmstart_get_sample: synchronize");
    if (centre)
        for (int k = 0; k < 3; ++k) centre[k] = x.c[k];
    if (label)
        for (int k = 0; k < 6; ++k) label[k] = x.ystar[k];
    return BT_OK;
}

int bt_warmstart_gradient(bt_warmstart* ws, const int32_t* ids, int32_t n, float* grad_out, double* loss_out)
{
    NvtxRange nvtx_range("bt_warmstart_gradient");
    last_error().clear();
    int st = check_ready(ws, "bt_warmstart_gradient");
    if (st != BT_OK) return st;
    if (n <= 0 || !ids) return fail(BT_ERR_INVALID, "bt_warmstart_gradient: bad arguments");
    st = gradient_pass(ws, ids, n);
    if (st != BT_OK) return st;
    if (grad_out)
        BT_CUDA(cudaMemcpyAsync(grad_out, ws->grad.p, sizeof(float) * W::kNumParams, cudaMemcpyDeviceToHost, ws->stream),
                "read gradient");
    if (loss_out)
        BT_CUDA(cudaMemcpyAsync(loss_out, ws->loss.p, sizeof(double), cudaMemcpyDeviceToHost, ws->stream), "read loss");
    BT_CUDA(cudaStreamSynchronize(ws->stream), "bt_warmstart_gradient: synchronize");
    return take_fault(ws, "bt_warmstart_gradient");
}

int bt_warmstart_train_step(bt_warmstart* ws, const int32_t* ids, int32_t n, float lr, double* loss_out)
{
    NvtxRange nvtx_range("bt_warmstart_train_step");
    last_error().clear();
    int st = check_ready(ws, "bt_warmstart_train_step");
    if (st != BT_OK) return st;
    if (n <= 0 || !ids || !std::isfinite(lr) || lr < 0.f)
        return fail(BT_ERR_INVALID, "bt_warmstart_train_step: bad arguments");
    st = take_fault(ws, "bt_warmstart_train_step (an earlier step)");
    if (st != BT_OK) return st;
    st = gradient_pass(ws, ids, n);
    if (st != BT_OK) return st;
    const double b1 = 0.9, b2 = 0.999;
    const int t = ws->adam_t + 1;
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, t))), c2 = (float)(1.0 / (1.0 - std::pow(b2, t)));
    BT_CUDA(W::launch_adam(ws->net(), ws->grad.as<float>(), lr, (float)b1, (float)b2, 1e-8f, c1, c2, ws->stream),
            "launch adam");
    ws->adam_t = t;
    if (loss_out) {
        BT_CUDA(cudaMemcpyAsync(loss_out, ws->loss.p, sizeof(double), cudaMemcpyDeviceToHost, ws->stream), "read loss");
        BT_CUDA(cudaStreamSynchronize(ws->stream), "bt_warmstart_train_step: synchronize");
        return take_fault(ws, "bt_warmstart_train_step");
    }
    return BT_OK;
}

int bt_warmstart_apply(bt_warmstart* ws, bt_graph* g)
{
    NvtxRange nvtx_range("bt_warmstart_apply");
    last_error().clear();
    int st = check_ready(ws, "bt_warmstart_apply");
    if (st != BT_OK) return st;
    if (!g) return fail(BT_ERR_INVALID, "bt_warmstart_apply: NULL graph");
    if ((int)g->active.size() > BT_MAX_NODES) return fail(BT_ERR_INVALID, "bt_warmstart_apply: too many active nodes");
    bt_graph* gs[1] = {g};
    return apply_graphs(ws, gs, 1, nullptr);
}

int bt_warmstart_apply_batch(bt_warmstart* ws, bt_batch* b, int32_t* status_out)
{
    NvtxRange nvtx_range("bt_warmstart_apply_batch");
    last_error().clear();
    int st = check_ready(ws, "bt_warmstart_apply_batch");
    if (st != BT_OK) return st;
    if (!b || b->graphs.empty()) return fail(BT_ERR_INVALID, "bt_warmstart_apply_batch: empty batch");
    return apply_graphs(ws, b->graphs.data(), (int)b->graphs.size(), status_out);
}

int bt_batch_solve_warm(bt_batch* b, bt_warmstart* ws, int32_t iters, int32_t fallback_iters,
                        const double* ref_costs, double tol, bt_solve_report* reps)
{
    NvtxRange nvtx_range("bt_batch_solve_warm");
    last_error().clear();
    int st = check_ready(ws, "bt_batch_solve_warm");
    if (st != BT_OK) return st;
    if (!b || b->graphs.empty()) return fail(BT_ERR_INVALID, "bt_batch_solve_warm: empty batch");
    if (iters < 0 || iters > BT_MAX_REPORT_ITERS || fallback_iters < 0 || fallback_iters > BT_MAX_REPORT_ITERS ||
        !(tol >= 0.0))
        return fail(BT_ERR_INVALID, "bt_batch_solve_warm: bad iteration counts or tolerance");
    const size_t G = b->graphs.size();
    // the stored poses are the plain start and the fallback's start
    std::vector<std::vector<double>> start(G);
    for (size_t k = 0; k < G; ++k) {
        bt_graph* g = b->graphs[k];
        start[k].resize(16 * g->active.size());
        for (size_t q = 0; q < g->active.size(); ++q)
            std::memcpy(&start[k][16 * q], g->frames.at(g->active[q]).pose, sizeof(double) * 16);
    }
    // one stream-ordered sequence: starting poses up, the network and the
    // averaging write the warm start into the batch's state block, the
    // captured solve runs from there, one read-back
    cudaStream_t s = b->stream;
    st = batch_prepare(b, iters);
    if (st != BT_OK) return st;
    for (bt_graph* g : b->graphs) {
        st = ensure_tables(g);
        if (st != BT_OK) return st;
        st = order_streams(g->stream, s);
        if (st != BT_OK) return st;
    }
    st = order_streams(ws->stream, s);
    if (st == BT_OK) st = batch_upload_state(b);
    if (st != BT_OK) return st;
    std::vector<double*> pose(G);
    for (size_t k = 0; k < G; ++k) pose[k] = b->h_args[k].pose;
    // the apply tables depend only on the batch build (edges, point sets,
    // pointers into the batch's state block): rebuilt only when it changed
    if (ws->app_build != 0 && ws->app_build == b->build_id) {
        st = launch_apply(ws, ws->app_S, (int)G, ws->app_max_free, s);
    } else {
        st = enqueue_apply(ws, b->graphs.data(), (int)G, pose.data(), s);
        if (st == BT_OK) ws->app_build = b->build_id;
    }
    if (st == BT_OK) st = read_status(ws, (int)G, s);
    if (st == BT_OK) st = batch_launch(b, iters);
    if (st != BT_OK) return st;
    BT_CUDA(cudaStreamSynchronize(s), "bt_batch_solve_warm: synchronize");
    b->pin_state.busy = false;
    ws->pin_status.busy = false;
    st = take_fault(ws, "bt_batch_solve_warm");
    if (st != BT_OK) return st;     // before any graph's poses are stored
    std::vector<int> ws_status(G, BT_OK);
    for (size_t k = 0; k < G; ++k) ws_status[k] = ws->pin_status.at<int>(0)[k] ? BT_ERR_SINGULAR : BT_OK;
    std::vector<bt_solve_report> r(G);
    batch_collect(b, iters, r.data());
    int worst = BT_OK;
    for (size_t k = 0; k < G; ++k) {
        r[k].used_warmstart = ws_status[k] == BT_OK ? 1 : 0;
        // with the plain solve's costs: worse than (1 + tol) times them; else
        // (the rule needs no plain solve) the last warm-started iteration
        // still moved the cost by more than tol of its final value, i.e. the
        // iterations did not converge
        const double e_last = r[k].cost_final;
        const bool moving = iters >= 1 && !(std::fabs(r[k].cost_per_iter[iters - 1] - e_last) <= tol * e_last);
        const bool bad = r[k].status != BT_OK ||
                         (ref_costs ? !(r[k].cost_final <= (1.0 + tol) * ref_costs[k]) : moving);
        if (bad) {
            bt_graph* g = b->graphs[k];
            for (size_t q = 0; q < g->active.size(); ++q)
                std::memcpy(g->frames.at(g->active[q]).pose, &start[k][16 * q], sizeof(double) * 16);
            bt_solve_report plain{};
            int s2 = bt_solve(g, fallback_iters, nullptr, &plain);
            if (s2 != BT_OK && s2 != BT_ERR_SINGULAR) return s2;
            plain.used_warmstart = r[k].used_warmstart;
            plain.fell_back = 1;
            r[k] = plain;
        }
        if (r[k].status != BT_OK) worst = r[k].status;
    }
    if (reps)
        for (size_t k = 0; k < G; ++k) reps[k] = r[k];
    if (worst != BT_OK) return fail(worst, "bt_batch_solve_warm: some graphs were singular; their poses are unchanged");
    return BT_OK;
}

int64_t bt_debug_tensor_wait_ns(int64_t ns)
{
    const long long v = ns < 0 ? kDefaultTensorWaitNs : (long long)ns;
    return (int64_t)g_tensor_wait_ns.exchange(v);
}

}  // extern "C"
