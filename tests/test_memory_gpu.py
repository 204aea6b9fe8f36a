"""Device memory: correspondence sets given with a frame (one packed upload
into a block the frame owns) against sets given one by one, and the
process-wide cache of idle device blocks behind the per-graph pools."""
import numpy as np
import pytest

import synthgen as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bt():
    from paper_2108_00516_gb300 import build as lbuild
    lbuild.build()
    from paper_2108_00516_gb300 import bt as _bt
    _bt.load()
    return _bt


def _one_by_one(bt, g):
    pg = bt.PoseGraph()
    ids = [pg.add_frame(r.depth, r.normals, r.mask, c.as_tuple(), P, bool(f))
           for r, c, P, f in zip(g.renders, g.cams, g.pose_init, g.fixed)]
    for (i, j, pi, pj) in g.matches:
        pg.set_matches(ids[j], ids[i], pj, pi)       # reversed order on purpose
    pg.frame_ids = ids
    return pg


def test_sets_with_the_frame_equal_sets_one_by_one(bt):
    g = S.tiny_graph(2)
    a = bt.graph_from_synth(g)          # sets given to bt_add_frame (packed, frame-owned)
    b = _one_by_one(bt, g)              # bt_set_matches per set (own blocks)
    Pa, ra = a.solve(5)
    Pb, rb = b.solve(5)
    assert np.array_equal(Pa, Pb) and ra["cost_final"] == rb["cost_final"]
    # drop the frame that owns the packed block of its sets, re-give one of
    # them one by one, and compare again
    for pg in (a, b):
        pg.remove_frame(pg.frame_ids[1])
        i, j, pi, pj = next(m for m in g.matches if (m[0], m[1]) == (0, 2))
        pg.set_matches(pg.frame_ids[0], pg.frame_ids[2], pi, pj)
        pg.set_poses(np.stack([g.pose_init[k] for k in (0, 2, 3)]))
    Pa, ra = a.solve(5)
    Pb, rb = b.solve(5)
    assert np.array_equal(Pa, Pb) and ra["cost_final"] == rb["cost_final"]
    a.close()
    b.close()


def test_destroyed_graphs_feed_the_cache(bt):
    g = S.tiny_graph(1)
    bt.device_cache_trim()
    base = bt.device_cache_bytes()
    pg = bt.graph_from_synth(g)
    P0, r0 = pg.solve(4)
    pg.close()
    idle = bt.device_cache_bytes()
    assert idle > base                           # the graph's blocks are idle in the cache
    pg = bt.graph_from_synth(g)                  # takes them back
    assert bt.device_cache_bytes() < idle
    P1, r1 = pg.solve(4)
    assert np.array_equal(P0, P1) and r0["cost_final"] == r1["cost_final"]
    pg.close()
    freed = bt.device_cache_trim()
    assert freed > 0 and bt.device_cache_bytes() == idle - freed


def test_injected_out_of_memory_leaves_state(bt):
    """bt_debug_fail_allocations makes the next allocation fail as if the GPU
    were out of memory: the call reports BT_ERR_OOM, the graph keeps its
    frames and poses, and the same calls succeed once the injection is used
    up, with the results of a graph that never failed."""
    g = S.tiny_graph(9)
    r, c = g.renders[0], g.cams[0]
    pg = bt.PoseGraph()
    assert bt.debug_fail_allocations(1) == 0
    with pytest.raises(bt.BTError) as e:
        pg.add_frame(r.depth, r.normals, r.mask, c.as_tuple(), g.pose_init[0], True)
    assert e.value.status == bt.BT_ERR_OOM
    assert pg.num_active == 0
    assert bt.debug_fail_allocations(0) == 0          # consumed by that call
    pg.close()
    ref = bt.graph_from_synth(g)
    P_ref, r_ref = ref.solve(3)
    ref.close()
    pg = bt.graph_from_synth(g)
    P0 = pg.get_poses()
    bt.debug_fail_allocations(1)                      # the solve's first table allocation fails
    with pytest.raises(bt.BTError) as e:
        pg.solve(3)
    assert e.value.status == bt.BT_ERR_OOM
    assert np.array_equal(pg.get_poses(), P0)
    assert bt.debug_fail_allocations(0) == 0
    P, rep = pg.solve(3)
    assert np.array_equal(P, P_ref) and rep["cost_final"] == r_ref["cost_final"]
    pg.close()
