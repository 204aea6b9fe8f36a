// bt_api.cu -- host runtime behind the C interface in include/bt.h.
//
// A bt_graph owns the device copies of its frames (target map + compacted
// source pixels, built on the GPU by the prep kernels), the correspondence
// sets, and the per-solve work buffers (grow-only, so repeated solves do not
// allocate).  bt_solve uploads the poses with the single-precision
// transforms formed from them on the host, enqueues on the graph's stream
//   iters x [residual(full) -> reduce(full)]  ->  residual(cost) -> reduce(cost)
// and then one device-to-host copy of poses, costs and status.
#include "bt_host.h"
#include "bt_xform.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

using namespace bthost;

static_assert(bt::kNumShapes == BT_NUM_SHAPES, "shape count of the interface");

std::string& bthost::last_error()
{
    thread_local std::string s;
    return s;
}



namespace {

int validate_config(const bt_config& c)
{
    auto pos = [](double x) { return std::isfinite(x) && x > 0.0; };
    if (!pos(c.huber_sparse) || !pos(c.huber_dense) || !pos(c.dense_max_dist))
        return fail(BT_ERR_INVALID, "config: Huber thresholds and dense_max_dist must be finite and > 0");
    if (!std::isfinite(c.dense_max_normal_deg) || c.dense_max_normal_deg < 0.0 || c.dense_max_normal_deg > 180.0)
        return fail(BT_ERR_INVALID, "config: dense_max_normal_deg must be in [0, 180]");
    if (!std::isfinite(c.lambda_sparse) || !std::isfinite(c.lambda_dense) || c.lambda_sparse < 0.0 ||
        c.lambda_dense < 0.0)
        return fail(BT_ERR_INVALID, "config: lambdas must be finite and >= 0");
    if (c.precision != BT_FP32 && c.precision != BT_BF16 && c.precision != BT_FP16)
        return fail(BT_ERR_INVALID, "config: precision must be BT_FP32, BT_BF16 or BT_FP16");
    if (c.max_frames < 0) return fail(BT_ERR_INVALID, "config: max_frames must be >= 0");
    if (c.solver != BT_SOLVER_CHOLESKY && c.solver != BT_SOLVER_PCG)
        return fail(BT_ERR_INVALID, "config: solver must be BT_SOLVER_CHOLESKY or BT_SOLVER_PCG");
    if (c.pcg_max_iters < 0 || !std::isfinite(c.pcg_tol) || c.pcg_tol < 0.0)
        return fail(BT_ERR_INVALID, "config: pcg_max_iters must be >= 0 and pcg_tol finite and >= 0");
    return BT_OK;
}

// Copies a count x 3 point list (host or device) into a pooled device block.
int upload_points(bt_graph* g, const float* src, int count, int mem_kind, float** out)
{
    *out = nullptr;
    if (count == 0) return BT_OK;
    const size_t bytes = sizeof(float) * 3 * (size_t)count;
    void* p = nullptr;
    BT_CUDA(g->pool.get(bytes, &p), "alloc(matches)");
    cudaError_t e = cudaMemcpyAsync(p, src, bytes,
                                    mem_kind == BT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->stream);
    if (e != cudaSuccess) {
        g->pool.put(p, bytes);
        return cuda_fail(e, "cudaMemcpyAsync(matches)");
    }
    *out = static_cast<float*>(p);
    return BT_OK;
}

void drop_matches(bt_graph* g, const MatchSet& m)
{
    if (!m.owned) return;    // the points belong to a frame's block
    g->pool.put(m.pa, sizeof(float) * 3 * (size_t)m.count);
    g->pool.put(m.pb, sizeof(float) * 3 * (size_t)m.count);
}

void unlink_partners(bt_graph* g, int fa, int fb)
{
    for (int k = 0; k < 2; ++k) {
        auto it = g->partners.find(k == 0 ? fa : fb);
        if (it == g->partners.end()) continue;
        std::vector<int>& v = it->second;
        v.erase(std::remove(v.begin(), v.end(), k == 0 ? fb : fa), v.end());
        if (v.empty()) g->partners.erase(it);
    }
}

void store_matches(bt_graph* g, int fa, int fb, int count, float* pa, float* pb, bool owned);

int put_matches(bt_graph* g, int fa, int fb, int count, const float* pa, const float* pb, int mem_kind)
{
    if (fa == fb) return fail(BT_ERR_INVALID, "matches: a frame cannot match itself");
    if (!g->frames.count(fa) || !g->frames.count(fb)) return fail(BT_ERR_INVALID, "matches: unknown frame id");
    if (count < 0) return fail(BT_ERR_INVALID, "matches: negative count");
    if (count > 0 && (!pa || !pb)) return fail(BT_ERR_INVALID, "matches: NULL point array");
    if (fa > fb) {
        std::swap(fa, fb);
        std::swap(pa, pb);
    }
    float *da = nullptr, *db = nullptr;
    int st = upload_points(g, pa, count, mem_kind, &da);
    if (st != BT_OK) return st;
    st = upload_points(g, pb, count, mem_kind, &db);
    if (st != BT_OK) {
        g->pool.put(da, sizeof(float) * 3 * (size_t)count);
        return st;
    }
    store_matches(g, fa, fb, count, da, db, true);
    return BT_OK;
}

// The correspondence sets given with a new frame f.  From host memory they
// go up together: the points are packed into pinned staging and copied in
// one transfer into one block owned by f (freed with f; the sets only point
// into it).  Device-resident sets are copied one by one.
int add_frame_matches(bt_graph* g, Frame& f, const bt_matches* matches, int n, int mem_kind)
{
    if (n <= 0) return BT_OK;
    if (mem_kind != BT_HOST) {
        for (int k = 0; k < n; ++k) {
            int st = put_matches(g, f.id, matches[k].other_frame, matches[k].count, matches[k].pts_self,
                                 matches[k].pts_other, mem_kind);
            if (st != BT_OK) return st;
        }
        return BT_OK;
    }
    for (int k = 0; k < n; ++k)
        if (matches[k].other_frame == f.id) return fail(BT_ERR_INVALID, "matches: a frame cannot match itself");
    size_t total = 0;
    for (int k = 0; k < n; ++k) total += 2 * sizeof(float) * 3 * (size_t)matches[k].count;
    char* blk = nullptr;
    if (total > 0) {
        BT_CUDA(g->pin_match.acquire(total), "cudaHostAlloc(match staging)");
        size_t off = 0;
        for (int k = 0; k < n; ++k) {
            const size_t b = sizeof(float) * 3 * (size_t)matches[k].count;
            if (b == 0) continue;
            std::memcpy(g->pin_match.at<char>(off), matches[k].pts_self, b);
            std::memcpy(g->pin_match.at<char>(off + b), matches[k].pts_other, b);
            off += 2 * b;
        }
        void* p = nullptr;
        BT_CUDA(g->pool.get(total, &p), "alloc(matches)");
        f.mblock = p;
        f.mblock_bytes = total;
        BT_CUDA(cudaMemcpyAsync(p, g->pin_match.p, total, cudaMemcpyHostToDevice, g->stream), "upload matches");
        BT_CUDA(g->pin_match.mark(g->stream), "record match upload");
        blk = static_cast<char*>(p);
    }
    size_t off = 0;
    for (int k = 0; k < n; ++k) {
        const int c = matches[k].count;
        const size_t b = sizeof(float) * 3 * (size_t)c;
        float* self = c > 0 ? reinterpret_cast<float*>(blk + off) : nullptr;
        float* other = c > 0 ? reinterpret_cast<float*>(blk + off + b) : nullptr;
        off += 2 * b;
        const int fo = matches[k].other_frame;
        if (fo < f.id) store_matches(g, fo, f.id, c, other, self, false);
        else store_matches(g, f.id, fo, c, self, other, false);
    }
    return BT_OK;
}

// Stores (or, for count 0, removes) the set of the pair fa < fb whose
// points are already on the device.
void store_matches(bt_graph* g, int fa, int fb, int count, float* pa, float* pb, bool owned)
{
    MatchSet ms;
    ms.fa = fa;
    ms.fb = fb;
    ms.count = count;
    ms.pa = pa;
    ms.pb = pb;
    ms.owned = owned;
    auto key = std::make_pair(fa, fb);
    auto it = g->matches.find(key);
    if (it != g->matches.end()) {
        drop_matches(g, it->second);
        g->matches.erase(it);
        unlink_partners(g, fa, fb);
    }
    if (count > 0) {
        g->matches[key] = ms;
        g->partners[fa].push_back(fb);
        g->partners[fb].push_back(fa);
    }
    g->topo_dirty = true;
}

// Rebuilds the node / tile / edge tables of the active set and sizes the
// per-solve buffers.
}  // namespace

std::vector<ActiveEdge> bthost::active_edges(const bt_graph* g)
{
    const int N = (int)g->active.size();
    std::vector<ActiveEdge> out;
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b) {
            const int fa = g->active[a], fb = g->active[b];
            auto it = g->matches.find(std::make_pair(std::min(fa, fb), std::max(fa, fb)));
            if (it == g->matches.end() || it->second.count <= 0) continue;
            const bool fwd = fa < fb;
            out.push_back(ActiveEdge{fwd ? a : b, fwd ? b : a, &it->second});
        }
    std::sort(out.begin(), out.end(), [](const ActiveEdge& x, const ActiveEdge& y) {
        return std::make_pair(x.m->fa, x.m->fb) < std::make_pair(y.m->fa, y.m->fb);
    });
    return out;
}

int bthost::resolve_pending(bt_graph* g)
{
    // every pending frame holds one read-back slot: none is pending when all
    // slots are free (no scan over the stored frames on every solve)
    if ((int)g->free_slots.size() >= g->pin_cap) return BT_OK;
    BT_CUDA(cudaStreamSynchronize(g->stream), "read back frame preparation");
    for (auto& kv : g->frames) {
        Frame& f = kv.second;
        if (!f.pending) continue;
        f.M = g->pin_m2[2 * f.slot];
        std::memcpy(&f.zref, &g->pin_m2[2 * f.slot + 1], sizeof(float));
        g->free_slots.push_back(f.slot);
        g->pool.put(f.dev_m2, 2 * sizeof(int));
        f.dev_m2 = nullptr;
        f.slot = -1;
        f.pending = false;
    }
    return BT_OK;
}

int bthost::build_topology(bt_graph* g, int tile)
{
    int pst = resolve_pending(g);
    if (pst != BT_OK) return pst;
    const int N = (int)g->active.size();
    if (N < 1) return fail(BT_ERR_INVALID, "solve: no active nodes");
    if (N > BT_MAX_NODES) return fail(BT_ERR_INVALID, "solve: more than BT_MAX_NODES active nodes");
    std::vector<bt::NodeDev> nodes(N);
    std::vector<int> tile_node;
    {
        size_t nt = 0;
        for (int k = 0; k < N; ++k) nt += (size_t)(g->frames.at(g->active[k]).M + tile - 1) / tile;
        tile_node.reserve(nt);
    }
    int nfree = 0;
    int64_t px = 0;
    for (int k = 0; k < N; ++k) {
        const Frame& f = g->frames.at(g->active[k]);
        bt::NodeDev& d = nodes[k];
        d.src_p = f.src_p;
        d.src_n = f.src_n;
        d.tgt = f.tgt;
        d.zref = f.zref;
        d.M = f.M;
        d.W = f.K.width;
        d.H = f.K.height;
        d.fx = f.K.fx;
        d.fy = f.K.fy;
        d.cx = f.K.cx;
        d.cy = f.K.cy;
        d.ifx = 1.0f / f.K.fx;
        d.ify = 1.0f / f.K.fy;
        d.tile0 = (int)tile_node.size();
        d.ntiles = (f.M + tile - 1) / tile;
        for (int t = 0; t < d.ntiles; ++t) tile_node.push_back(k);
        d.free_idx = f.fixed ? -1 : nfree++;
        px += (int64_t)f.M * (N - 1);
    }
    std::vector<bt::EdgeDev> edges;
    for (const ActiveEdge& ae : active_edges(g)) {
        bt::EdgeDev e;
        e.i = ae.i;
        e.j = ae.j;
        e.count = ae.m->count;
        e.pa = ae.m->pa;
        e.pb = ae.m->pb;
        edges.push_back(e);
    }
    const int T = (int)tile_node.size(), P = N * (N - 1), E = (int)edges.size(), U = N * (N - 1) / 2;
    std::vector<int2> upairs;
    std::vector<int> upair_edge(std::max(U, 1), -1);
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b) upairs.push_back(make_int2(a, b));
    for (int e = 0; e < E; ++e) {
        const int a = std::min(edges[e].i, edges[e].j), b = std::max(edges[e].i, edges[e].j);
        upair_edge[a * N - a * (a + 1) / 2 + (b - a - 1)] = e;
    }
    cudaStream_t s = g->stream;
    // one device block for the tables, staged through pinned memory
    size_t off = 0;
    auto take = [&off](size_t bytes) {
        const size_t o = off;
        off = align_up(o + std::max<size_t>(bytes, 1), 256);
        return o;
    };
    const size_t o_nodes = take(sizeof(bt::NodeDev) * N), o_edges = take(sizeof(bt::EdgeDev) * E),
                 o_tiles = take(sizeof(int) * T), o_upairs = take(sizeof(int2) * U),
                 o_upair_edge = take(sizeof(int) * U), tab_bytes = off;
    BT_CUDA(g->pin_tab.acquire(tab_bytes), "cudaHostAlloc(table staging)");
    std::memcpy(g->pin_tab.at<char>(o_nodes), nodes.data(), sizeof(bt::NodeDev) * N);
    if (E > 0) std::memcpy(g->pin_tab.at<char>(o_edges), edges.data(), sizeof(bt::EdgeDev) * E);
    if (T > 0) std::memcpy(g->pin_tab.at<char>(o_tiles), tile_node.data(), sizeof(int) * T);
    if (U > 0) {
        std::memcpy(g->pin_tab.at<char>(o_upairs), upairs.data(), sizeof(int2) * U);
        std::memcpy(g->pin_tab.at<char>(o_upair_edge), upair_edge.data(), sizeof(int) * U);
    }
    BT_CUDA(g->d_tab.ensure(tab_bytes), "alloc tables");
    BT_CUDA(g->d_state.ensure(StateLayout(N).bytes), "alloc solve state");
    BT_CUDA(g->d_dpart.ensure(sizeof(float) * bt::kDenseVals * (size_t)std::max(T, 1) * std::max(N - 1, 1)),
            "alloc dpart");
    BT_CUDA(g->d_spart.ensure(sizeof(float) * bt::kSparseVals * std::max(E, 1)), "alloc spart");
    BT_CUDA(g->d_upairblk.ensure(sizeof(double) * bt::kUPairBlk * std::max(U, 1)), "alloc upairblk");
    BT_CUDA(cudaMemcpyAsync(g->d_tab.p, g->pin_tab.p, tab_bytes, cudaMemcpyHostToDevice, s), "upload tables");
    BT_CUDA(g->pin_tab.mark(s), "record table upload");
    bt::SolveArgs& a = g->args;
    a.N = N;
    a.n_tiles = T;
    a.n_pairs = P;
    a.n_edges = E;
    a.n_free = nfree;
    a.n_upairs = U;
    a.tile = tile;
    a.precision = g->cfg.precision;
    a.stage_blocks = bt::reduce_stage_fits(nfree, N) ? 1 : 0;
    const bt_config& c = g->cfg;
    a.dmax2 = (float)(c.dense_max_dist * c.dense_max_dist);
    a.cmin = (float)std::cos(c.dense_max_normal_deg * 3.14159265358979323846 / 180.0);
    a.huber_dense = (float)c.huber_dense;
    a.huber_sparse = (float)c.huber_sparse;
    a.lambda_dense = c.lambda_dense;
    a.lambda_sparse = c.lambda_sparse;
    a.solver = c.solver;
    a.pcg_max_iters = c.pcg_max_iters;
    a.pcg_tol2 = c.pcg_tol * c.pcg_tol;
    char* tab = g->d_tab.as<char>();
    a.nodes = reinterpret_cast<bt::NodeDev*>(tab + o_nodes);
    a.edges = reinterpret_cast<bt::EdgeDev*>(tab + o_edges);
    a.tile_node = reinterpret_cast<int*>(tab + o_tiles);
    a.upairs = reinterpret_cast<int2*>(tab + o_upairs);
    a.upair_edge = reinterpret_cast<int*>(tab + o_upair_edge);
    const StateLayout L(N);
    char* state = g->d_state.as<char>();
    a.ctrl = reinterpret_cast<bt::Control*>(state);
    a.pose = reinterpret_cast<double*>(state + L.pose);
    a.costs = reinterpret_cast<double*>(state + L.costs);
    a.xf = reinterpret_cast<float*>(state + L.xf);
    a.xinv = reinterpret_cast<float*>(state + L.xinv);
    a.dpart = g->d_dpart.as<float>();
    a.spart = g->d_spart.as<float>();
    a.upairblk = g->d_upairblk.as<double>();
    g->pixels_per_pass = px;
    int64_t sp = 0;
    for (const bt::EdgeDev& e : edges) sp += e.count;
    g->sparse_per_pass = sp;
    g->topo_dirty = false;
    g->topo_version++;
    g->built_tile = tile;
    return BT_OK;
}

void bthost::stage_state(const bt_graph* g, char* blk, bool xforms)
{
    const int N = (int)g->active.size();
    const StateLayout L(N);
    std::memset(blk, 0, sizeof(bt::Control));
    double* pose = reinterpret_cast<double*>(blk + L.pose);
    for (int k = 0; k < N; ++k) std::memcpy(pose + 12 * (size_t)k, g->frames.at(g->active[k]).pose, sizeof(double) * 12);
    if (!xforms) return;
    // the transforms the solve kernel forms after each update (write_xforms,
    // bt_xform.cuh), with the same operations in the same order
    float* xf = reinterpret_cast<float*>(blk + L.xf);
    float* xinv = reinterpret_cast<float*>(blk + L.xinv);
    std::vector<float> sp((size_t)bt::kXfSplit * N);
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < 15; ++k) bt::xf_split_entry(pose + 12 * (size_t)i, k, sp.data() + bt::kXfSplit * i);
    for (int i = 0; i < N; ++i)
        for (int e = 0; e < 12; ++e) xinv[12 * i + e] = bt::xf_inv_entry(sp.data() + bt::kXfSplit * i, e);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            for (int e = 0; e < 12; ++e)
                xf[((size_t)i * N + j) * 12 + e] =
                    bt::xf_pair_entry(sp.data() + bt::kXfSplit * j, sp.data() + bt::kXfSplit * i, e);
        }
}

int bthost::upload_poses(bt_graph* g)
{
    const StateLayout L((int)g->active.size());
    BT_CUDA(g->pin_state.acquire(L.bytes), "cudaHostAlloc(state staging)");
    // the poses and the first pass's transforms in one copy (no transform
    // kernel ahead of the first residual pass)
    stage_state(g, g->pin_state.at<char>(0), true);
    BT_CUDA(cudaMemcpyAsync(g->d_state.p, g->pin_state.p, L.upload_bytes(), cudaMemcpyHostToDevice, g->stream),
            "upload poses");
    BT_CUDA(g->pin_state.mark(g->stream), "record state upload");
    return BT_OK;
}

int bthost::fill_report(bt_graph* g, const char* blk, int iters, bt_solve_report* rep)
{
    const StateLayout L((int)g->active.size());
    const bt::Control& ctrl = *reinterpret_cast<const bt::Control*>(blk);
    const double* costs = reinterpret_cast<const double*>(blk + L.costs);
    if (g->prof_on)
        for (int k = 0; k < 4; ++k) g->prof.solve_phase_cycles[k] += (int64_t)ctrl.clk[k];
    const int status = ctrl.checked != 0u ? BT_ERR_INVALID : ctrl.status == -4 ? BT_ERR_SINGULAR : BT_OK;
    if (rep) {
        std::memset(rep, 0, sizeof(*rep));
        rep->iters_run = iters;
        rep->status = status;
        rep->cost_init = iters > 0 ? costs[0] : costs[4 * iters];
        rep->cost_final = costs[4 * iters + 0];
        rep->dense_cost_final = costs[4 * iters + 1];
        rep->sparse_cost_final = costs[4 * iters + 2];
        rep->dense_inliers = (int64_t)std::llround(costs[4 * iters + 3]);
        for (int k = 0; k < iters; ++k) rep->cost_per_iter[k] = costs[4 * k];
        rep->dense_pixel_pairs = g->pixels_per_pass * iters;
    }
    return status;
}

namespace {

// Makes sure 4 * passes events exist (two per residual and reduce launch).
int ensure_events(bt_graph* g, int passes)
{
    while ((int)g->events.size() < 4 * passes) {
        cudaEvent_t e;
        BT_CUDA(cudaEventCreate(&e), "cudaEventCreate");
        g->events.push_back(e);
    }
    return BT_OK;
}

// Enqueues `iters` full passes and one cost pass; with profiling on, events
// bracket every launch on the graph's stream.
int enqueue_passes(bt_graph* g, int iters, bool cost_pass, int cost_slot)
{
    cudaStream_t s = g->stream;
    const bt::SolveArgs& a = g->args;
    const int passes = iters + (cost_pass ? 1 : 0);
    g->prof_timed = g->prof_on && (g->prof_solves++ % g->prof_period) == 0;
    if (g->prof_timed) {
        int st = ensure_events(g, passes);
        if (st != BT_OK) return st;
    }
    for (int p = 0; p < passes; ++p) {
        const bool full = p < iters;
        const int slot = full ? p : cost_slot;
        if (g->prof_timed) BT_CUDA(cudaEventRecord(g->events[4 * p + 0], s), "event");
        BT_CUDA(bt::launch_residual(a, full, s), "launch residual");
        if (g->prof_timed) BT_CUDA(cudaEventRecord(g->events[4 * p + 1], s), "event");
        BT_CUDA(bt::launch_reduce(a, full, slot, s), "launch reduce");
        if (g->prof_timed) BT_CUDA(cudaEventRecord(g->events[4 * p + 2], s), "event");
        if (a.n_edges + a.n_tiles > 0) g->prof.residual_launches++;
        g->prof.reduce_launches++;
    }
    return BT_OK;
}

// After the stream has been synchronised: fold the event times in.
void collect_events(bt_graph* g, int passes)
{
    if (!g->prof_timed) return;
    for (int p = 0; p < passes; ++p) {
        float t1 = 0.f, t2 = 0.f;
        if (cudaEventElapsedTime(&t1, g->events[4 * p + 0], g->events[4 * p + 1]) == cudaSuccess &&
            g->args.n_edges + g->args.n_tiles > 0) {
            g->prof.residual_ms += t1;
            g->prof.timed_residual_launches++;
            g->prof.dense_pixel_pairs += g->pixels_per_pass;
            g->prof.sparse_pairs += g->sparse_per_pass;
        }
        if (cudaEventElapsedTime(&t2, g->events[4 * p + 1], g->events[4 * p + 2]) == cudaSuccess) {
            g->prof.reduce_ms += t2;
            g->prof.timed_reduce_launches++;
        }
    }
}

}  // namespace

extern "C" {

void bt_config_default(bt_config* cfg)
{
    if (!cfg) return;
    cfg->huber_sparse = 0.005;
    cfg->huber_dense = 0.005;
    cfg->dense_max_dist = 0.02;
    cfg->dense_max_normal_deg = 45.0;
    cfg->lambda_sparse = 1.0;
    cfg->lambda_dense = 1.0;
    cfg->precision = BT_FP32;
    cfg->max_frames = 0;
    cfg->solver = BT_SOLVER_CHOLESKY;
    cfg->pcg_max_iters = 500;
    cfg->pcg_tol = 1e-10;
}

int bt_graph_create(const bt_config* cfg, void* cuda_stream, bt_graph** out)
{
    last_error().clear();
    if (!out) return fail(BT_ERR_INVALID, "bt_graph_create: out is NULL");
    *out = nullptr;
    bt_config c;
    bt_config_default(&c);
    if (cfg) c = *cfg;
    int st = validate_config(c);
    if (st != BT_OK) return st;
    int dev = 0;
    BT_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    bt_graph* g = new (std::nothrow) bt_graph();
    if (!g) return fail(BT_ERR_OOM, "bt_graph_create: host allocation failed");
    g->cfg = c;
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    *out = g;
    return BT_OK;
}

void bt_graph_destroy(bt_graph* g) { delete g; }

int bt_add_frame(bt_graph* g, const float* depth, const float* normals, const uint8_t* mask,
                 const bt_intrinsics* K, const double pose_init[16], int32_t fixed,
                 const bt_matches* matches, int32_t n_matches, int32_t mem_kind, int32_t* frame_id_out)
{
    NvtxRange nvtx_range("bt_add_frame");
    last_error().clear();
    if (!g || !depth || !normals || !mask || !K || !pose_init)
        return fail(BT_ERR_INVALID, "bt_add_frame: NULL argument");
    if (mem_kind != BT_HOST && mem_kind != BT_DEVICE) return fail(BT_ERR_INVALID, "bt_add_frame: bad mem_kind");
    if (K->width < 1 || K->height < 1 || K->width > 32767 || K->height > 32767 ||
        (int64_t)K->width * K->height > (1 << 28))
        return fail(BT_ERR_INVALID, "bt_add_frame: image size out of range");
    if (!std::isfinite(K->fx) || !std::isfinite(K->fy) || K->fx == 0.f || K->fy == 0.f || !std::isfinite(K->cx) ||
        !std::isfinite(K->cy))
        return fail(BT_ERR_INVALID, "bt_add_frame: bad intrinsics");
    if (!finite_pose(pose_init)) return fail(BT_ERR_INVALID, "bt_add_frame: pose must be finite with last row 0 0 0 1");
    if (n_matches < 0 || (n_matches > 0 && !matches)) return fail(BT_ERR_INVALID, "bt_add_frame: bad matches");
    if (g->cfg.max_frames > 0 && (int)g->frames.size() >= g->cfg.max_frames)
        return fail(BT_ERR_INVALID, "bt_add_frame: max_frames reached");
    for (int k = 0; k < n_matches; ++k) {
        if (!g->frames.count(matches[k].other_frame)) return fail(BT_ERR_INVALID, "bt_add_frame: unknown other_frame");
        if (matches[k].count < 0 || (matches[k].count > 0 && (!matches[k].pts_self || !matches[k].pts_other)))
            return fail(BT_ERR_INVALID, "bt_add_frame: bad match set");
    }
    cudaStream_t s = g->stream;
    const int W = K->width, H = K->height, HW = W * H;
    const float *d_depth = depth, *d_normals = normals;
    const uint8_t* d_mask = mask;
    if (mem_kind == BT_HOST) {
        BT_CUDA(g->up_depth.ensure(sizeof(float) * HW), "alloc upload");
        BT_CUDA(g->up_normals.ensure(sizeof(float) * 3 * (size_t)HW), "alloc upload");
        BT_CUDA(g->up_mask.ensure((size_t)HW), "alloc upload");
        BT_CUDA(cudaMemcpyAsync(g->up_depth.p, depth, sizeof(float) * HW, cudaMemcpyHostToDevice, s), "upload depth");
        BT_CUDA(cudaMemcpyAsync(g->up_normals.p, normals, sizeof(float) * 3 * (size_t)HW, cudaMemcpyHostToDevice, s),
                "upload normals");
        BT_CUDA(cudaMemcpyAsync(g->up_mask.p, mask, (size_t)HW, cudaMemcpyHostToDevice, s), "upload mask");
        d_depth = g->up_depth.as<float>();
        d_normals = g->up_normals.as<float>();
        d_mask = g->up_mask.as<uint8_t>();
    }
    const int P = g->cfg.precision;
    const size_t pb = bt::pixel_bytes(P);
    BT_CUDA(g->prep_blk.ensure(bt::prep_scratch_bytes(HW)), "alloc prep");
    // a pinned host slot for the (M, zref) read-back, read at the next
    // topology build instead of waiting here
    if (g->free_slots.empty()) {
        int st = resolve_pending(g);       // no copy may be in flight into the old slots
        if (st != BT_OK) return st;
        const int cap = std::max(64, 2 * g->pin_cap);
        int* np = nullptr;
        BT_CUDA(alloc_should_fail() ? cudaErrorMemoryAllocation
                                    : cudaHostAlloc(reinterpret_cast<void**>(&np), sizeof(int) * 2 * (size_t)cap,
                                                    cudaHostAllocMapped),
                "cudaHostAlloc(read-back slots)");
        int* npd = nullptr;
        const cudaError_t em = cudaHostGetDevicePointer(reinterpret_cast<void**>(&npd), np, 0);
        if (em != cudaSuccess) {
            cudaFreeHost(np);
            return cuda_fail(em, "cudaHostGetDevicePointer(read-back slots)");
        }
        if (g->pin_m2) cudaFreeHost(g->pin_m2);
        g->pin_m2 = np;
        g->pin_m2_dev = npd;
        for (int k = cap - 1; k >= g->pin_cap; --k) g->free_slots.push_back(k);
        g->pin_cap = cap;
    }
    Frame f;
    f.tgt_bytes = pb * HW;
    f.src_bytes = pb * HW;
    void *t = nullptr, *sp = nullptr, *sn = nullptr, *m2 = nullptr;
    cudaError_t e = g->pool.get(f.tgt_bytes, &t);
    if (e == cudaSuccess) e = g->pool.get(f.src_bytes, &sp);
    if (e == cudaSuccess) e = g->pool.get(f.src_bytes, &sn);
    if (e == cudaSuccess) e = g->pool.get(2 * sizeof(int), &m2);
    f.tgt = t;
    f.src_p = sp;
    f.src_n = sn;
    f.dev_m2 = static_cast<int*>(m2);
    const float ifx = 1.0f / K->fx, ify = 1.0f / K->fy;
    // (M, zref) land in a mapped pinned slot, written by the preparation's
    // scan kernel itself (no separate read-back copy), read at the next
    // topology build after a stream synchronisation
    if (e == cudaSuccess) {
        f.slot = g->free_slots.back();
        g->free_slots.pop_back();
        e = bt::launch_prep(d_depth, d_normals, d_mask, W, H, K->cx, K->cy, ifx, ify, P, f.tgt, f.src_p, f.src_n,
                            g->prep_blk.p, f.dev_m2, g->pin_m2_dev + 2 * f.slot, s);
        f.pending = true;
        if (e != cudaSuccess) {
            g->free_slots.push_back(f.slot);
            f.slot = -1;
        }
    }
    g->prof.prep_launches += 3;
    if (e != cudaSuccess) {
        g->pool.put(f.tgt, f.tgt_bytes);
        g->pool.put(f.src_p, f.src_bytes);
        g->pool.put(f.src_n, f.src_bytes);
        g->pool.put(f.dev_m2, 2 * sizeof(int));
        return cuda_fail(e, "bt_add_frame: preparation");
    }
    f.id = g->next_id;
    f.K = *K;
    f.fixed = fixed ? 1 : 0;
    std::memcpy(f.pose, pose_init, sizeof(double) * 16);
    g->frames[f.id] = f;
    g->next_id++;
    int st = add_frame_matches(g, g->frames[f.id], matches, n_matches, mem_kind);
    if (st != BT_OK) {
        std::string msg = last_error();
        bt_remove_frame(g, f.id);
        g->next_id--;
        last_error() = msg;
        return st;
    }
    g->active.push_back(f.id);
    g->topo_dirty = true;
    if (frame_id_out) *frame_id_out = f.id;
    return BT_OK;
}

int bt_set_matches(bt_graph* g, int32_t frame_a, int32_t frame_b, int32_t count, const float* pts_a,
                   const float* pts_b, int32_t mem_kind)
{
    NvtxRange nvtx_range("bt_set_matches");
    last_error().clear();
    if (!g) return fail(BT_ERR_INVALID, "bt_set_matches: NULL graph");
    if (mem_kind != BT_HOST && mem_kind != BT_DEVICE) return fail(BT_ERR_INVALID, "bt_set_matches: bad mem_kind");
    return put_matches(g, frame_a, frame_b, count, pts_a, pts_b, mem_kind);
}

int bt_remove_frame(bt_graph* g, int32_t frame_id)
{
    if (!g) return fail(BT_ERR_INVALID, "bt_remove_frame: NULL graph");
    auto it = g->frames.find(frame_id);
    if (it == g->frames.end()) return fail(BT_ERR_INVALID, "bt_remove_frame: unknown frame id");
    // blocks go back to the pool: later work that reuses them is enqueued
    // after every earlier use on the same stream
    Frame& f = it->second;
    g->pool.put(f.tgt, f.tgt_bytes);
    g->pool.put(f.src_p, f.src_bytes);
    g->pool.put(f.src_n, f.src_bytes);
    if (f.pending) {
        g->pool.put(f.dev_m2, 2 * sizeof(int));
        g->free_slots.push_back(f.slot);
    }
    if (f.mblock) g->pool.put(f.mblock, f.mblock_bytes);
    g->frames.erase(it);
    auto pit = g->partners.find(frame_id);
    if (pit != g->partners.end()) {
        const std::vector<int> others = pit->second;
        for (int o : others) {
            auto m = g->matches.find(std::make_pair(std::min(o, frame_id), std::max(o, frame_id)));
            if (m != g->matches.end()) {
                drop_matches(g, m->second);
                g->matches.erase(m);
            }
            unlink_partners(g, o, frame_id);
        }
    }
    g->active.erase(std::remove(g->active.begin(), g->active.end(), frame_id), g->active.end());
    g->topo_dirty = true;
    return BT_OK;
}

int bt_set_active(bt_graph* g, const int32_t* ids, int32_t n)
{
    last_error().clear();
    if (!g || !ids) return fail(BT_ERR_INVALID, "bt_set_active: NULL argument");
    if (n < 1 || n > BT_MAX_NODES) return fail(BT_ERR_INVALID, "bt_set_active: n out of range");
    std::vector<int> v(ids, ids + n);
    for (int k = 0; k < n; ++k) {
        if (!g->frames.count(v[k])) return fail(BT_ERR_INVALID, "bt_set_active: unknown frame id");
        for (int q = 0; q < k; ++q)
            if (v[q] == v[k]) return fail(BT_ERR_INVALID, "bt_set_active: repeated frame id");
    }
    if (v != g->active) {
        g->active = v;
        g->topo_dirty = true;
    }
    return BT_OK;
}

int bt_num_active(const bt_graph* g)
{
    if (!g) return fail(BT_ERR_INVALID, "bt_num_active: NULL graph");
    return (int)g->active.size();
}

int bt_set_poses(bt_graph* g, const double* poses)
{
    last_error().clear();
    if (!g || !poses) return fail(BT_ERR_INVALID, "bt_set_poses: NULL argument");
    for (size_t k = 0; k < g->active.size(); ++k)
        if (!finite_pose(poses + 16 * k)) return fail(BT_ERR_INVALID, "bt_set_poses: bad pose");
    for (size_t k = 0; k < g->active.size(); ++k)
        std::memcpy(g->frames.at(g->active[k]).pose, poses + 16 * k, sizeof(double) * 16);
    return BT_OK;
}

int bt_get_poses(const bt_graph* g, double* poses)
{
    if (!g || !poses) return fail(BT_ERR_INVALID, "bt_get_poses: NULL argument");
    for (size_t k = 0; k < g->active.size(); ++k)
        std::memcpy(poses + 16 * k, g->frames.at(g->active[k]).pose, sizeof(double) * 16);
    return BT_OK;
}

int bt_solve(bt_graph* g, int32_t iters, double* poses_out, bt_solve_report* rep)
{
    NvtxRange nvtx_range("bt_solve");
    last_error().clear();
    if (!g) return fail(BT_ERR_INVALID, "bt_solve: NULL graph");
    if (iters < 0 || iters > BT_MAX_REPORT_ITERS) return fail(BT_ERR_INVALID, "bt_solve: iters out of range");
    if (g->active.empty()) return fail(BT_ERR_INVALID, "bt_solve: no active nodes");
    if (g->topo_dirty || g->built_tile != bt::shape_tile(bt::kSingleShape)) {
        int st = build_topology(g, bt::shape_tile(bt::kSingleShape));
        if (st != BT_OK) return st;
    }
    int st = upload_poses(g);
    if (st != BT_OK) return st;
    cudaStream_t s = g->stream;
    const bt::SolveArgs& a = g->args;
    st = enqueue_passes(g, iters, true, iters);
    if (st != BT_OK) return st;
    const int N = a.N;
    const StateLayout L(N);
    // read back into the staging the upload came from (ordered after it on s)
    BT_CUDA(cudaMemcpyAsync(g->pin_state.p, g->d_state.p, L.readback_bytes(iters), cudaMemcpyDeviceToHost, s),
            "read solve state");
    BT_CUDA(g->pin_state.mark(s), "record state read-back");
    BT_CUDA(cudaStreamSynchronize(s), "bt_solve: synchronize");
    g->pin_state.busy = false;
    collect_events(g, iters + 1);
    const char* blk = g->pin_state.at<char>(0);
    const int status = fill_report(g, blk, iters, rep);
    const double* pose = reinterpret_cast<const double*>(blk + L.pose);
    if (status == BT_ERR_INVALID)
        return fail(status, "bt_solve: an index check of the bounds-checked build failed; poses unchanged");
    if (status != BT_OK) return fail(status, "bt_solve: normal equations not positive definite; poses unchanged");
    for (int k = 0; k < N; ++k) {
        Frame& f = g->frames.at(g->active[k]);
        std::memcpy(f.pose, pose + 12 * (size_t)k, sizeof(double) * 12);
        if (poses_out) std::memcpy(poses_out + 16 * (size_t)k, f.pose, sizeof(double) * 16);
    }
    return BT_OK;
}

int bt_eval_cost(bt_graph* g, double* cost_out, int64_t* dense_inliers)
{
    NvtxRange nvtx_range("bt_eval_cost");
    last_error().clear();
    if (!g || !cost_out) return fail(BT_ERR_INVALID, "bt_eval_cost: NULL argument");
    if (g->active.empty()) return fail(BT_ERR_INVALID, "bt_eval_cost: no active nodes");
    if (g->topo_dirty || g->built_tile != bt::shape_tile(bt::kSingleShape)) {
        int st = build_topology(g, bt::shape_tile(bt::kSingleShape));
        if (st != BT_OK) return st;
    }
    int st = upload_poses(g);
    if (st != BT_OK) return st;
    cudaStream_t s = g->stream;
    st = enqueue_passes(g, 0, true, 0);
    if (st != BT_OK) return st;
    const StateLayout L(g->args.N);
    BT_CUDA(cudaMemcpyAsync(g->pin_state.p, g->d_state.p, L.readback_bytes(0), cudaMemcpyDeviceToHost, s),
            "read costs");
    BT_CUDA(g->pin_state.mark(s), "record state read-back");
    BT_CUDA(cudaStreamSynchronize(s), "bt_eval_cost: synchronize");
    g->pin_state.busy = false;
    const double* c = g->pin_state.at<double>(L.costs);
    collect_events(g, 1);
    if (g->pin_state.at<bt::Control>(0)->checked != 0u)
        return fail(BT_ERR_INVALID, "bt_eval_cost: an index check of the bounds-checked build failed");
    cost_out[0] = c[0];
    cost_out[1] = c[1];
    cost_out[2] = c[2];
    if (dense_inliers) *dense_inliers = (int64_t)std::llround(c[3]);
    return BT_OK;
}

int bt_profile_enable(bt_graph* g, int32_t on)
{
    if (!g) return fail(BT_ERR_INVALID, "bt_profile_enable: NULL graph");
    BT_CUDA(g->stream ? cudaStreamSynchronize(g->stream) : cudaDeviceSynchronize(), "bt_profile_enable: sync");
    if (on < 0) return fail(BT_ERR_INVALID, "bt_profile_enable: negative period");
    std::memset(&g->prof, 0, sizeof(g->prof));
    g->prof_on = on != 0;
    g->prof_period = on > 0 ? on : 1;
    g->prof_solves = 0;
    g->prof_timed = false;
    return BT_OK;
}

int bt_profile_read(const bt_graph* g, bt_profile* out)
{
    if (!g || !out) return fail(BT_ERR_INVALID, "bt_profile_read: NULL argument");
    *out = g->prof;
    return BT_OK;
}

const char* bt_status_str(int status)
{
    switch (status) {
    case BT_OK: return "ok";
    case BT_ERR_INVALID: return "invalid argument";
    case BT_ERR_CUDA: return "CUDA error";
    case BT_ERR_OOM: return "out of memory";
    case BT_ERR_SINGULAR: return "normal equations not positive definite";
    case BT_ERR_TIMEOUT: return "device wait timed out";
    case BT_ERR_STATE: return "invalid state";
    default: return "unknown status";
    }
}

const char* bt_last_error(void) { return last_error().c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched solver
// ---------------------------------------------------------------------------


namespace {

// (Re)builds every graph's tables for `shape` and the batch's work lists.
int batch_build(bt_batch* b, int shape)
{
    const int tile = bt::shape_tile(shape);
    std::vector<bt::SolveArgs> args;
    std::vector<int2> wres, wpair;
    b->max_N = 1;
    b->solve_smem = 0;
    b->pixels_per_pass = 0;
    for (size_t k = 0; k < b->graphs.size(); ++k) {
        bt_graph* g = b->graphs[k];
        if (g->topo_dirty || g->built_tile != tile) {
            int st = build_topology(g, tile);
            if (st != BT_OK) return st;
        }
        // the graph's tables and frames were enqueued on its own stream
        int st = order_streams(g->stream, b->stream);
        if (st != BT_OK) return st;
        const bt::SolveArgs& a = g->args;
        args.push_back(a);
        for (int e = 0; e < a.n_edges; ++e) wres.push_back(make_int2((int)k, e));
        for (int t = 0; t < a.n_tiles; ++t) wres.push_back(make_int2((int)k, a.n_edges + t));
        for (int u = 0; u < a.n_upairs; ++u) wpair.push_back(make_int2((int)k, u));
        b->max_N = std::max(b->max_N, a.N);
        b->solve_smem = std::max(b->solve_smem, bt::reduce_smem_bytes(a.n_free, a.N));
        b->pixels_per_pass += g->pixels_per_pass;
    }
    cudaStream_t s = b->stream;
    // every graph's solve state moves into one batch block (pointers in the
    // batch's copy of its arguments)
    const size_t G = b->graphs.size();
    b->state_off.assign(G + 1, 0);
    for (size_t k = 0; k < G; ++k) b->state_off[k + 1] = b->state_off[k] + StateLayout(args[k].N).bytes;
    BT_CUDA(b->d_state.ensure(b->state_off[G]), "alloc batch state");
    for (size_t k = 0; k < G; ++k) {
        const StateLayout L(args[k].N);
        char* blk = b->d_state.as<char>() + b->state_off[k];
        args[k].ctrl = reinterpret_cast<bt::Control*>(blk);
        args[k].pose = reinterpret_cast<double*>(blk + L.pose);
        args[k].costs = reinterpret_cast<double*>(blk + L.costs);
    }
    b->h_args = args;
    static std::atomic<uint64_t> next_build_id{0};
    b->build_id = ++next_build_id;
    b->topo_versions.clear();
    for (bt_graph* g : b->graphs) b->topo_versions.push_back(g->topo_version);
    const size_t n_args = std::max<size_t>(args.size(), 1), n_res = std::max<size_t>(wres.size(), 1),
                 n_pair = std::max<size_t>(wpair.size(), 1);
    BT_CUDA(b->d_args.ensure(sizeof(bt::SolveArgs) * n_args), "alloc batch args");
    BT_CUDA(b->d_work_res.ensure(sizeof(int2) * n_res), "alloc batch work");
    BT_CUDA(b->d_work_pair.ensure(sizeof(int2) * n_pair), "alloc batch work");
    const size_t o_res = align_up(sizeof(bt::SolveArgs) * n_args, 256),
                 o_pair = o_res + align_up(sizeof(int2) * n_res, 256), tab_bytes = o_pair + sizeof(int2) * n_pair;
    BT_CUDA(b->pin_tab.acquire(tab_bytes), "cudaHostAlloc(batch table staging)");
    if (!args.empty()) std::memcpy(b->pin_tab.p, args.data(), sizeof(bt::SolveArgs) * args.size());
    if (!wres.empty()) std::memcpy(b->pin_tab.at<char>(o_res), wres.data(), sizeof(int2) * wres.size());
    if (!wpair.empty()) std::memcpy(b->pin_tab.at<char>(o_pair), wpair.data(), sizeof(int2) * wpair.size());
    if (!args.empty())
        BT_CUDA(cudaMemcpyAsync(b->d_args.p, b->pin_tab.p, sizeof(bt::SolveArgs) * args.size(),
                                cudaMemcpyHostToDevice, s),
                "upload batch args");
    if (!wres.empty())
        BT_CUDA(cudaMemcpyAsync(b->d_work_res.p, b->pin_tab.at<char>(o_res), sizeof(int2) * wres.size(),
                                cudaMemcpyHostToDevice, s),
                "upload batch work");
    if (!wpair.empty())
        BT_CUDA(cudaMemcpyAsync(b->d_work_pair.p, b->pin_tab.at<char>(o_pair), sizeof(int2) * wpair.size(),
                                cudaMemcpyHostToDevice, s),
                "upload batch work");
    BT_CUDA(b->pin_tab.mark(s), "record batch table upload");
    b->n_work_res = (int)wres.size();
    b->n_work_pair = (int)wpair.size();
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->exec_shape = shape;
    return BT_OK;
}

}  // namespace

// Cleared control words and the stored poses of every graph, in one copy.
int bthost::batch_upload_state(bt_batch* b)
{
    const size_t G = b->graphs.size();
    BT_CUDA(b->pin_state.acquire(b->state_off[G]), "cudaHostAlloc(batch state staging)");
    for (size_t k = 0; k < G; ++k) stage_state(b->graphs[k], b->pin_state.at<char>(b->state_off[k]));
    const size_t bytes = b->state_off[G - 1] + StateLayout(b->h_args[G - 1].N).upload_bytes();
    BT_CUDA(cudaMemcpyAsync(b->d_state.p, b->pin_state.p, bytes, cudaMemcpyHostToDevice, b->stream),
            "upload batch poses");
    BT_CUDA(b->pin_state.mark(b->stream), "record batch state upload");
    return BT_OK;
}

namespace {

// Enqueues the whole solve (xforms, iters full passes, one cost pass).
int batch_enqueue(bt_batch* b, int iters, int shape)
{
    const bt::SolveArgs* A = b->d_args.as<bt::SolveArgs>();
    const int G = (int)b->graphs.size();
    cudaStream_t s = b->stream;
    BT_CUDA(bt::launch_batch_xforms(A, G, s), "batch xforms");
    for (int p = 0; p <= iters; ++p) {
        const bool full = p < iters;
        BT_CUDA(bt::launch_batch_residual(A, b->d_work_res.as<int2>(), b->n_work_res, b->max_N, full, shape,
                                          b->precision, s),
                "batch residual");
        BT_CUDA(bt::launch_batch_pairs(A, b->d_work_pair.as<int2>(), b->n_work_pair, full, s), "batch pairs");
        BT_CUDA(bt::launch_batch_solve(A, G, b->solve_smem, full, p, s), "batch solve");
    }
    return BT_OK;
}

// Times one full residual pass per CTA shape and keeps the fastest.
int batch_autotune(bt_batch* b)
{
    cudaEvent_t e0, e1;
    BT_CUDA(cudaEventCreate(&e0), "event");
    BT_CUDA(cudaEventCreate(&e1), "event");
    b->tune_us.assign(bt::kNumShapes, 0.0);
    int best = 0;
    double best_us = 1e300;
    for (int sh = 0; sh < bt::kNumShapes; ++sh) {
        int st = batch_build(b, sh);
        if (st == BT_OK) st = batch_upload_state(b);
        if (st != BT_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        const bt::SolveArgs* A = b->d_args.as<bt::SolveArgs>();
        BT_CUDA(bt::launch_batch_xforms(A, (int)b->graphs.size(), b->stream), "batch xforms");
        float ms = 0.f, tot = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            BT_CUDA(cudaEventRecord(e0, b->stream), "event");
            BT_CUDA(bt::launch_batch_residual(A, b->d_work_res.as<int2>(), b->n_work_res, b->max_N, true, sh,
                                              b->precision, b->stream),
                    "batch residual");
            BT_CUDA(cudaEventRecord(e1, b->stream), "event");
            BT_CUDA(cudaEventSynchronize(e1), "event sync");
            BT_CUDA(cudaEventElapsedTime(&ms, e0, e1), "event time");
            if (rep > 0) tot += ms;
        }
        const double us = 1e3 * tot / 2.0;
        b->tune_us[sh] = us;
        if (us < best_us) {
            best_us = us;
            best = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuned_shape = best;
    return BT_OK;
}

}  // namespace

int bthost::batch_prepare(bt_batch* b, int iters)
{
    bt::prepare_launch_attributes();
    bool topo_changed = b->dirty;
    for (bt_graph* g : b->graphs) topo_changed |= g->topo_dirty;
    // tables rebuilt outside the batch (a single-graph solve at another tile
    // size, e.g. the warm-started solve's fallback) moved or rewrote what the
    // batch's arguments point to
    bool moved = b->topo_versions.size() != b->graphs.size();
    for (size_t k = 0; !moved && k < b->graphs.size(); ++k) moved = b->graphs[k]->topo_version != b->topo_versions[k];
    if (topo_changed) {
        b->dirty = false;
        if (b->shape < 0) {
            int st = batch_autotune(b);
            if (st != BT_OK) return st;
        }
    }
    const int shape = b->shape >= 0 ? b->shape : (b->tuned_shape >= 0 ? b->tuned_shape : 0);
    if (topo_changed || moved || b->exec_shape != shape) {
        int st = batch_build(b, shape);
        if (st != BT_OK) return st;
    }
    if (!b->exec || b->exec_iters != iters) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t graph;
        BT_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        int st = batch_enqueue(b, iters, shape);
        cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        if (st != BT_OK) return st;
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        b->exec_iters = iters;
    }
    return BT_OK;
}

int bthost::batch_launch(bt_batch* b, int iters)
{
    const size_t G = b->graphs.size();
    BT_CUDA(cudaGraphLaunch(b->exec, b->stream), "graph launch");
    // read back into the staging the upload came from (stream order keeps
    // the two copies apart; the host reads it after synchronising)
    const size_t bytes = b->state_off[G - 1] + StateLayout(b->h_args[G - 1].N).readback_bytes(iters);
    BT_CUDA(cudaMemcpyAsync(b->pin_state.p, b->d_state.p, bytes, cudaMemcpyDeviceToHost, b->stream),
            "read batch state");
    BT_CUDA(b->pin_state.mark(b->stream), "record batch state read-back");
    return BT_OK;
}

int bthost::batch_collect(bt_batch* b, int iters, bt_solve_report* reps)
{
    int worst = BT_OK;
    for (size_t k = 0; k < b->graphs.size(); ++k) {
        bt_graph* g = b->graphs[k];
        const char* blk = b->pin_state.at<char>(b->state_off[k]);
        const StateLayout L(b->h_args[k].N);
        const int status = fill_report(g, blk, iters, reps ? &reps[k] : nullptr);
        if (status != BT_OK) {
            worst = status;
            continue;
        }
        const double* pose = reinterpret_cast<const double*>(blk + L.pose);
        for (int q = 0; q < b->h_args[k].N; ++q)
            std::memcpy(g->frames.at(g->active[q]).pose, pose + 12 * (size_t)q, sizeof(double) * 12);
    }
    return worst;
}

extern "C" {

int bt_batch_create(void* cuda_stream, bt_batch** out)
{
    last_error().clear();
    if (!out) return fail(BT_ERR_INVALID, "bt_batch_create: out is NULL");
    *out = nullptr;
    bt_batch* b = new (std::nothrow) bt_batch();
    if (!b) return fail(BT_ERR_OOM, "bt_batch_create: host allocation failed");
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return cuda_fail(e, "bt_batch_create: stream");
        }
        b->own_stream = true;
    }
    *out = b;
    return BT_OK;
}

void bt_batch_destroy(bt_batch* b) { delete b; }

int bt_batch_add(bt_batch* b, bt_graph* g)
{
    last_error().clear();
    if (!b || !g) return fail(BT_ERR_INVALID, "bt_batch_add: NULL argument");
    if (g->active.empty() || (int)g->active.size() > BT_MAX_NODES)
        return fail(BT_ERR_INVALID, "bt_batch_add: graph needs 1..BT_MAX_NODES active nodes");
    for (bt_graph* h : b->graphs)
        if (h == g) return fail(BT_ERR_INVALID, "bt_batch_add: graph already in the batch");
    if (b->precision >= 0 && g->cfg.precision != b->precision)
        return fail(BT_ERR_INVALID, "bt_batch_add: every graph of a batch must use the same storage precision");
    b->precision = g->cfg.precision;
    b->graphs.push_back(g);
    b->dirty = true;
    b->tuned_shape = -1;
    return BT_OK;
}

int bt_batch_size(const bt_batch* b)
{
    if (!b) return fail(BT_ERR_INVALID, "bt_batch_size: NULL batch");
    return (int)b->graphs.size();
}

int bt_batch_set_shape(bt_batch* b, int32_t shape)
{
    if (!b) return fail(BT_ERR_INVALID, "bt_batch_set_shape: NULL batch");
    if (shape < -1 || shape >= bt::kNumShapes) return fail(BT_ERR_INVALID, "bt_batch_set_shape: unknown shape");
    b->shape = shape;
    b->dirty = true;
    return BT_OK;
}

int bt_batch_tuning(const bt_batch* b, int32_t* shape_out, double* us_per_shape)
{
    if (!b) return fail(BT_ERR_INVALID, "bt_batch_tuning: NULL batch");
    if (shape_out) *shape_out = b->shape >= 0 ? b->shape : b->tuned_shape;
    if (us_per_shape)
        for (int k = 0; k < bt::kNumShapes; ++k)
            us_per_shape[k] = k < (int)b->tune_us.size() ? b->tune_us[k] : 0.0;
    return BT_OK;
}

int bt_batch_solve(bt_batch* b, int32_t iters, bt_solve_report* reps)
{
    NvtxRange nvtx_range("bt_batch_solve");
    last_error().clear();
    if (!b) return fail(BT_ERR_INVALID, "bt_batch_solve: NULL batch");
    if (iters < 0 || iters > BT_MAX_REPORT_ITERS) return fail(BT_ERR_INVALID, "bt_batch_solve: iters out of range");
    if (b->graphs.empty()) return fail(BT_ERR_INVALID, "bt_batch_solve: empty batch");
    int st = batch_prepare(b, iters);
    if (st == BT_OK) st = batch_upload_state(b);
    if (st == BT_OK) st = batch_launch(b, iters);
    if (st != BT_OK) return st;
    BT_CUDA(cudaStreamSynchronize(b->stream), "bt_batch_solve: synchronize");
    b->pin_state.busy = false;
    st = batch_collect(b, iters, reps);
    if (st != BT_OK) return fail(st, "bt_batch_solve: some graphs were singular; their poses are unchanged");
    return BT_OK;
}

}  // extern "C"
