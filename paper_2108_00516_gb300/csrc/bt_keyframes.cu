// bt_keyframes.cu -- memory-pool keyframe selection (Sec. IV-C) and pool
// augmentation (Sec. IV-E): host code of libbt (a few hundred rotations,
// well under a millisecond; no GPU work).
//
// The edge weight of two keyframes is the geodesic distance of their
// rotations, arccos((tr(R_a^T R_b) - 1) / 2).  The minimum H-subgraph is
// approximated greedily: start from the pool's first frame I_0 and add the
// pool frame with the smallest summed distance to the current frame and to
// every frame already selected, until K frames are selected.  Running sums
// keep the greedy loop O(n K) after the O(n) distances to the current frame.
#include "bt_host.h"

#include <cmath>
#include <vector>

using namespace bthost;

namespace {

// Rotation blocks of two row-major 4x4 poses.
double geodesic(const double* Ta, const double* Tb)
{
    double tr = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) tr += Ta[r * 4 + c] * Tb[r * 4 + c];
    double x = 0.5 * (tr - 1.0);
    x = x > 1.0 ? 1.0 : (x < -1.0 ? -1.0 : x);
    return std::acos(x);
}

bool finite16(const double* T)
{
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(T[k])) return false;
    return true;
}

}  // namespace

extern "C" {

int32_t bt_select_keyframes(const double* pool_poses, int32_t n_pool, const double* pose_current, int32_t K,
                            int32_t* out)
{
    last_error().clear();
    if (n_pool < 0 || K < 0) return fail(BT_ERR_INVALID, "bt_select_keyframes: negative size");
    if (n_pool == 0 || K == 0) return 0;
    if (!pool_poses || !pose_current || !out) return fail(BT_ERR_INVALID, "bt_select_keyframes: NULL argument");
    if (!finite16(pose_current)) return fail(BT_ERR_INVALID, "bt_select_keyframes: non-finite pose");
    for (int f = 0; f < n_pool; ++f)
        if (!finite16(pool_poses + 16 * (size_t)f)) return fail(BT_ERR_INVALID, "bt_select_keyframes: non-finite pose");
    const int want = K < n_pool ? K : n_pool;
    std::vector<double> cost(n_pool);
    std::vector<char> taken(n_pool, 0);
    // cost of a candidate: distance to the current frame plus the distances
    // to the frames selected so far (I_0 first)
    for (int f = 0; f < n_pool; ++f)
        cost[f] = geodesic(pool_poses + 16 * (size_t)f, pose_current) + geodesic(pool_poses + 16 * (size_t)f, pool_poses);
    out[0] = 0;
    taken[0] = 1;
    for (int k = 1; k < want; ++k) {
        int best = -1;
        for (int f = 0; f < n_pool; ++f)
            if (!taken[f] && (best < 0 || cost[f] < cost[best])) best = f;     // ties: the earlier entry
        out[k] = best;
        taken[best] = 1;
        for (int f = 0; f < n_pool; ++f)
            if (!taken[f]) cost[f] += geodesic(pool_poses + 16 * (size_t)f, pool_poses + 16 * (size_t)best);
    }
    return want;
}

int32_t bt_is_novel_view(const double* pool_poses, int32_t n_pool, const double* pose_current, double min_deg)
{
    last_error().clear();
    if (n_pool < 0 || !(min_deg >= 0.0)) return fail(BT_ERR_INVALID, "bt_is_novel_view: bad size or threshold");
    if (n_pool > 0 && (!pool_poses || !pose_current)) return fail(BT_ERR_INVALID, "bt_is_novel_view: NULL argument");
    const double lim = min_deg * 3.14159265358979323846 / 180.0;
    for (int f = 0; f < n_pool; ++f)
        if (!(geodesic(pool_poses + 16 * (size_t)f, pose_current) > lim)) return 0;
    return 1;
}

}  // extern "C"
