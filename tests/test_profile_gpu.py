"""The profiling counters (bt_profile_*): launch counts of every solve, event
timings and pixel-pair counts of the sampled solves only."""
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


@pytest.mark.parametrize("every", [1, 3])
def test_sampled_event_timing(bt, every):
    g = S.tiny_graph(2)
    pg = bt.graph_from_synth(g)
    iters, solves = 4, 7
    pg.profile_enable(every)
    px = []
    for _ in range(solves):
        pg.set_poses(g.pose_init)
        _, rep = pg.solve(iters)
        px.append(rep["dense_pixel_pairs"])
    p = pg.profile_read()
    timed = len(range(0, solves, every))
    passes = iters + 1
    assert p["residual_launches"] == solves * passes and p["reduce_launches"] == solves * passes
    assert p["timed_residual_launches"] == timed * passes and p["timed_reduce_launches"] == timed * passes
    # every pass (the cost pass too) of a timed solve counts its pixel pairs
    assert p["dense_pixel_pairs"] == timed * px[0] // iters * passes
    assert p["residual_ms"] > 0 and p["reduce_ms"] > 0
    pg.profile_enable(0)
    pg.set_poses(g.pose_init)
    pg.solve(iters)
    q = pg.profile_read()
    assert q["timed_residual_launches"] == 0 and q["residual_launches"] == passes
    with pytest.raises(bt.BTError):
        pg.profile_enable(-1)
    pg.close()
