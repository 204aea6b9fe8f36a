// bt_debug.cu -- diagnostic entry points of libbt: the dense association of
// one ordered pair and the assembled normal equations of one Gauss-Newton
// iteration (Sec. IV-D), computed by the solve's own kernels at the stored
// poses so that an independent implementation can check them value by value.
#include "bt_host.h"

#include <cuda_runtime.h>

using namespace bthost;

namespace {

// Tables for the single-graph CTA shape, the stored poses uploaded and the
// float transforms launched (the first steps of bt_solve).
int prepare(bt_graph* g)
{
    if (g->active.empty()) return fail(BT_ERR_INVALID, "no active nodes");
    if (g->topo_dirty || g->built_tile != bt::shape_tile(bt::kSingleShape)) {
        int st = build_topology(g, bt::shape_tile(bt::kSingleShape));
        if (st != BT_OK) return st;
    }
    return upload_poses(g);
}

}  // namespace

extern "C" {

int bt_debug_associate(bt_graph* g, int32_t src_node, int32_t dst_node, int32_t* tgt_out, int32_t cap,
                       int32_t* count_out)
{
    NvtxRange nvtx_range("bt_debug_associate");
    last_error().clear();
    if (!g) return fail(BT_ERR_INVALID, "bt_debug_associate: NULL graph");
    const int N = (int)g->active.size();
    if (src_node < 0 || src_node >= N || dst_node < 0 || dst_node >= N || src_node == dst_node)
        return fail(BT_ERR_INVALID, "bt_debug_associate: node out of range");
    int st = prepare(g);
    if (st != BT_OK) return st;
    const int M = g->frames.at(g->active[src_node]).M;
    if (count_out) *count_out = M;
    if (!tgt_out) return BT_OK;     // count query
    if (cap < M) return fail(BT_ERR_INVALID, "bt_debug_associate: cap smaller than the source pixel count");
    if (M == 0) return BT_OK;
    cudaStream_t s = g->stream;
    BT_CUDA(g->d_debug.ensure(sizeof(int32_t) * (size_t)M), "bt_debug_associate: alloc");
    BT_CUDA(bt::launch_assoc_debug(g->args, src_node, dst_node, M, g->d_debug.as<int>(), s),
            "bt_debug_associate: launch");
    BT_CUDA(cudaMemcpyAsync(tgt_out, g->d_debug.p, sizeof(int32_t) * (size_t)M, cudaMemcpyDeviceToHost, s),
            "bt_debug_associate: read back");
    BT_CUDA(cudaStreamSynchronize(s), "bt_debug_associate: synchronize");
    g->pin_state.busy = false;
    return BT_OK;
}

int bt_debug_normal_equations(bt_graph* g, double* H_out, double* g_out, int32_t n_cap, int32_t* n_out,
                              double* cost_out)
{
    NvtxRange nvtx_range("bt_debug_normal_equations");
    last_error().clear();
    if (!g || !H_out || !g_out) return fail(BT_ERR_INVALID, "bt_debug_normal_equations: NULL argument");
    if (g->active.empty()) return fail(BT_ERR_INVALID, "bt_debug_normal_equations: no active nodes");
    if (g->topo_dirty || g->built_tile != bt::shape_tile(bt::kSingleShape)) {
        int st = build_topology(g, bt::shape_tile(bt::kSingleShape));
        if (st != BT_OK) return st;
    }
    const int n = 6 * g->args.n_free;
    if (n_out) *n_out = n;
    if (n == 0) return fail(BT_ERR_INVALID, "bt_debug_normal_equations: no free node");
    if (n_cap < n) return fail(BT_ERR_INVALID, "bt_debug_normal_equations: n_cap smaller than 6 x free nodes");
    int st = upload_poses(g);
    if (st != BT_OK) return st;
    cudaStream_t s = g->stream;
    const size_t vals = (size_t)n * n + n;
    BT_CUDA(g->d_debug.ensure(sizeof(double) * vals), "bt_debug_normal_equations: alloc");
    bt::SolveArgs a = g->args;
    a.ne_out = g->d_debug.as<double>();
    BT_CUDA(bt::launch_residual(a, true, s), "bt_debug_normal_equations: residual pass");
    BT_CUDA(bt::launch_reduce(a, true, 0, s), "bt_debug_normal_equations: reduce");
    const StateLayout L(a.N);
    BT_CUDA(cudaMemcpyAsync(g->pin_state.p, g->d_state.p, L.readback_bytes(0), cudaMemcpyDeviceToHost, s),
            "bt_debug_normal_equations: read state");
    BT_CUDA(cudaMemcpyAsync(H_out, a.ne_out, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost, s),
            "bt_debug_normal_equations: read H");
    BT_CUDA(cudaMemcpyAsync(g_out, a.ne_out + (size_t)n * n, sizeof(double) * n, cudaMemcpyDeviceToHost, s),
            "bt_debug_normal_equations: read g");
    BT_CUDA(cudaStreamSynchronize(s), "bt_debug_normal_equations: synchronize");
    g->pin_state.busy = false;
    const bt::Control& ctrl = *g->pin_state.at<bt::Control>(0);
    if (ctrl.status == -4) return fail(BT_ERR_SINGULAR, "bt_debug_normal_equations: solve stage failed");
    if (cost_out) {
        const double* c = g->pin_state.at<double>(L.costs);
        for (int k = 0; k < 4; ++k) cost_out[k] = c[k];
    }
    return BT_OK;
}

}  // extern "C"
