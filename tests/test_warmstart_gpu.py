"""Learned warm start on the GPU (bt_warmstart_*) against the FP64 oracle
(oracle/warmstart.py): network outputs, labels, gradients, Adam steps, a
short training run and the relative-pose averaging solve.

Tolerances.  The oracle runs the same network (BF16 weights, BF16-rounded
inputs of the 128 -> 256 contraction) in FP64; the GPU sums in FP32 and forms
M0 and the features in FP32.  Outputs therefore agree to ~1e-5 relative,
except where an FP32 layer-1 value sits within its rounding error of a BF16
rounding boundary and the two sides round one element of h1 to neighbouring
BF16 values (2^-8 relative on that element); the bounds below allow for that.
The max-pool's argmax is an integer decided in floating point: the test data
are checked to have every channel's maximum ahead of the runner-up by far
more than FP32 rounding, so both sides route the gradient to the same rows.
"""
import numpy as np
import pytest

import oracle as O
import oracle.warmstart as W
import synthgen as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bt():
    from paper_2108_00516_gb300 import build as lbuild
    lbuild.build()
    from paper_2108_00516_gb300 import bt as _bt
    _bt.load()
    return _bt


def _pose(rng, ang, tr):
    w = rng.normal(size=3)
    w *= ang / np.linalg.norm(w)
    return O.se3_exp(np.concatenate([rng.normal(size=3) * tr, w]))


def _sets(seed, sizes):
    """Synthetic correspondence sets: points of an object ~0.45 m away, q =
    M_true p + 1 mm noise with 20 % outliers, M0 = M_true perturbed."""
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        p = (rng.normal(size=(n, 3)) * [0.04, 0.04, 0.03] + [0.0, 0.0, 0.45]).astype(np.float32)
        M = _pose(rng, 0.15, 0.02)
        q = p.astype(np.float64) @ M[:3, :3].T + M[:3, 3] + rng.normal(scale=0.001, size=(n, 3))
        k = int(0.2 * n)
        q[:k] = q[rng.permutation(n)[:k]] + rng.normal(scale=0.03, size=(k, 3))
        q = q.astype(np.float32)
        M0 = _pose(rng, 0.08, 0.01) @ M
        out.append((p, q, M0, M))
    return out


def _params(seed):
    rng = np.random.default_rng(seed)
    P = S.warmstart_init(seed).astype(np.float64)
    return (P + rng.normal(scale=0.01, size=P.shape)).astype(np.float32)


# set sizes around the 128-point chunks of the forward pass
SIZES = [1, 7, 63, 64, 65, 127, 128, 129, 130, 255, 256, 257, 800]


def _loaded(bt, sets, params):
    ws = bt.WarmStart(params)
    for p, q, M0, M in sets:
        ws.add_set(p, q, np.eye(4), M0, np.eye(4), M)
    return ws


def test_forward_labels_match_oracle(bt):
    sets = _sets(1, SIZES)
    P = _params(1)
    ws = _loaded(bt, sets, P)
    y = ws.predict(range(len(sets)))
    for k, (p, q, M0, M) in enumerate(sets):
        x, c = W.features(p, q, M0)
        yo, _ = W.forward(P.astype(np.float64), x)
        assert np.all(np.abs(y[k] - yo) <= 1e-3 * (1 + np.abs(yo))), (k, y[k], yo)
        cg, lab = ws.sample(k)
        assert np.allclose(cg, c, atol=1e-6)
        lo = W.label(M0, M, c)
        assert np.allclose(lab, lo, rtol=1e-5, atol=1e-4), (lab, lo)
    errs = [np.max(np.abs(y[k] - W.forward(P.astype(np.float64), W.features(*s[:3])[0])[0]))
            for k, s in enumerate(sets)]
    assert np.median(errs) < 1e-4


def test_forward_is_set_order_invariant(bt):
    (p, q, M0, M), = _sets(2, [300])
    perm = np.random.default_rng(0).permutation(300)
    ws = _loaded(bt, [(p, q, M0, M), (p[perm], q[perm], M0, M)], _params(2))
    y = ws.predict([0, 1])
    assert np.allclose(y[0], y[1], rtol=1e-5, atol=1e-6)


def test_forward_wait_timeout_is_reported(bt):
    """A forward pass whose bounded wait on the tensor cores runs out reports
    BT_ERR_TIMEOUT (here the bound is 0: the first wait gives up at once) and
    leaves the context usable: the next pass gives the same outputs."""
    sets = _sets(3, [200, 333])
    ws = _loaded(bt, sets, _params(3))
    y0 = ws.predict([0, 1])
    prev = bt.debug_tensor_wait_ns(0)
    try:
        with pytest.raises(bt.BTError) as e:
            ws.predict([0, 1])
        assert e.value.status == bt.BT_ERR_TIMEOUT
    finally:
        bt.debug_tensor_wait_ns(-1)
    assert prev == 1_000_000_000
    assert np.array_equal(ws.predict([0, 1]), y0)


def test_training_and_inference_forward_agree(bt):
    """The training forward pass (running maxima with the row of each) and
    the inference pass (maxima only) pool the same values: the mean loss of
    bt_warmstart_gradient, formed from the training pass's outputs, equals
    the loss formed here from bt_warmstart_predict's outputs."""
    sets = _sets(4, SIZES)
    ws = _loaded(bt, sets, _params(4))
    ids = list(range(len(sets)))
    y = ws.predict(ids).astype(np.float64)
    ystar = np.array([ws.sample(k)[1] for k in ids], np.float64)
    loss_inf = float(np.mean(0.5 * np.sum((y - ystar) ** 2, axis=1)))
    loss_train, _ = ws.gradient(ids)
    assert abs(loss_train - loss_inf) <= 1e-6 * loss_inf, (loss_train, loss_inf)


def _routing_gap(P, x):
    """Smallest gap, over channels with a positive maximum, between the
    maximum of h2 and the runner-up (FP64 oracle values)."""
    L = W.unpack(P)
    h1 = W.bf16(np.maximum(x @ W.bf16(L["W1"]).T + L["b1"], 0))
    h2 = np.maximum(h1 @ W.bf16(L["W2"]).T + L["b2"], 0)
    s = np.sort(h2, axis=0)
    top, second = s[-1], s[-2] if len(x) > 1 else np.zeros(h2.shape[1])
    pos = top > 0
    return np.min((top - second)[pos] / top[pos]) if pos.any() else 1.0


def _routed_sets(seed, sizes, P, gap=2e-5):
    """Sets (seeded, deterministic) whose every channel maximum leads the
    runner-up by more than `gap` relative: FP32 accumulation over 128 terms
    moves a value by < 1e-5 relative, so both sides pick the same rows."""
    out = []
    for k, n in enumerate(sizes):
        for t in range(100):
            cand = _sets(seed * 1000 + 17 * k + t, [n])[0]
            if _routing_gap(P.astype(np.float64), W.features(*cand[:3])[0]) > gap:
                out.append(cand)
                break
        else:
            raise AssertionError("no well-separated set found")
    return out


def test_gradient_matches_oracle(bt):
    P = _params(3)
    sets = _routed_sets(3, [5, 64, 65, 130], P)
    ws = _loaded(bt, sets, P)
    xs = [W.features(p, q, M0)[0] for p, q, M0, _ in sets]
    targets = [W.label(M0, M, W.features(p, q, M0)[1]) for p, q, M0, M in sets]
    loss_g, g = ws.gradient(range(len(sets)))
    loss_o, go = W.loss_and_grad(P.astype(np.float64), xs, targets)
    assert abs(loss_g - loss_o) <= 1e-4 * loss_o
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in W.LAYERS])
    for k, (name, _) in enumerate(W.LAYERS):
        a, b = g[offs[k]:offs[k + 1]].astype(np.float64), go[offs[k]:offs[k + 1]]
        scale = np.max(np.abs(b)) + 1e-30
        assert np.max(np.abs(a - b)) <= 5e-3 * scale, (name, np.max(np.abs(a - b)), scale)
        assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b), name


def test_adam_steps_match_oracle(bt):
    P = _params(4)
    sets = _routed_sets(4, [40, 90, 70], P)
    ws = _loaded(bt, sets, P)
    xs = [W.features(p, q, M0)[0] for p, q, M0, _ in sets]
    ts = [W.label(M0, M, W.features(p, q, M0)[1]) for p, q, M0, M in sets]
    lr = 1e-3
    batches = [[0, 1], [1, 2]]
    Po, m, v = P.astype(np.float64), np.zeros(W.N_PARAMS), np.zeros(W.N_PARAMS)
    for t, ids in enumerate(batches, start=1):
        before = ws.get_params().astype(np.float64)
        ws.train_step(ids, lr)
        after = ws.get_params().astype(np.float64)
        _, go = W.loss_and_grad(Po, [xs[k] for k in ids], [ts[k] for k in ids])
        Pn, m, v = W.adam(Po, go, m, v, t, lr)
        step_g, step_o = after - before, Pn - Po
        # |m_hat| <= sqrt(v_hat) up to the mismatch of the two bias
        # corrections (a factor below 1.002 for two steps)
        assert np.max(np.abs(step_g)) <= lr * 1.002
        # where the gradient is well above FP32 noise the steps agree
        ok = np.abs(go) > 1e-3 * np.max(np.abs(go))
        assert np.max(np.abs(step_g[ok] - step_o[ok])) <= 2e-2 * lr
        Po = after       # continue from the GPU's parameters (both sides step the same state)


def test_short_training_reduces_loss(bt):
    graphs = [S.training_graph(k) for k in range(40)]
    ws = bt.WarmStart(S.warmstart_init(0))
    for g in graphs:
        pg = bt.graph_from_synth(g)
        ws.add_graph(pg, g.pose_init, g.pose_true)
        pg.close()
    n = ws.num_samples()
    assert n == sum(len(g.matches) for g in graphs)
    ids = np.arange(n)
    loss0, _ = ws.gradient(ids)
    rng = np.random.default_rng(0)
    for step in range(300):
        ws.train_step(rng.choice(n, 32, replace=False), 1e-3)
    loss1, _ = ws.gradient(ids)
    assert loss1 < 0.3 * loss0, (loss0, loss1)


def test_apply_matches_oracle_average(bt):
    g = S.tiny_graph(0)
    P = _params(5)
    ws = bt.WarmStart(P)
    pg = bt.graph_from_synth(g)
    ws.apply(pg)
    got = pg.get_poses()
    D = {}
    for (i, j, pi, pj) in g.matches:
        M0 = g.pose_init[j] @ np.linalg.inv(g.pose_init[i])
        x, c = W.features(pi, pj, M0)
        y, _ = W.forward(P.astype(np.float64), x)
        D[(i, j)] = W.increment(y, c)
    ref = W.average(list(g.pose_init), list(g.fixed), D)
    for k in range(g.n):
        rot = S.rotation_angle(got[k][:3, :3] @ ref[k][:3, :3].T)
        assert rot < 1e-4 and np.max(np.abs(got[k][:3, 3] - ref[k][:3, 3])) < 1e-5, k
    assert np.array_equal(got[0], g.pose_init[0])        # the fixed node is kept


def test_apply_batch_equals_single(bt):
    gs = [S.tiny_graph(k) for k in range(3)]
    P = _params(6)
    ws = bt.WarmStart(P)
    singles = []
    for g in gs:
        pg = bt.graph_from_synth(g)
        ws.apply(pg)
        singles.append(pg.get_poses())
    pgs = [bt.graph_from_synth(g) for g in gs]
    batch = bt.Batch()
    for pg in pgs:
        batch.add(pg)
    assert ws.apply_batch(batch) == [0, 0, 0]
    for pg, ref in zip(pgs, singles):
        assert np.array_equal(pg.get_poses(), ref)


def test_warmstart_errors(bt):
    ws = bt.WarmStart()
    g = S.tiny_graph(1)
    pg = bt.graph_from_synth(g)
    with pytest.raises(bt.BTError) as e:
        ws.apply(pg)
    assert e.value.status == bt.BT_ERR_STATE
    bad = S.warmstart_init(0)
    bad[5] = np.nan
    with pytest.raises(bt.BTError):
        ws.set_params(bad)
    ws.set_params(S.warmstart_init(0))
    with pytest.raises(bt.BTError):
        ws.add_set(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), np.eye(4), np.eye(4))
    with pytest.raises(bt.BTError):
        ws.predict([0])                       # no samples yet
    # a free node without any correspondence set: singular averaging system
    g2 = S.SynthGraph(g.cams, g.renders, g.pose_true, g.pose_init, g.fixed,
                      [m for m in g.matches if 3 not in (m[0], m[1])], g.shape)
    pg2 = bt.graph_from_synth(g2)
    with pytest.raises(bt.BTError) as e:
        ws.apply(pg2)
    assert e.value.status == bt.BT_ERR_SINGULAR
    assert np.array_equal(pg2.get_poses(), g.pose_init)


def test_largest_graph_solve_and_average(bt):
    """BT_MAX_NODES = 24 nodes (6 x 23 = 138 unknowns, the largest system of
    both FP64 solves): the Gauss-Newton solve against the oracle, the batch
    against the single graph bit for bit, and the warm start's averaging
    against the oracle's."""
    g = S.random_graph(777, bt.BT_MAX_NODES, S.TINY_CAMERA, 60, 0.2)
    pg = bt.graph_from_synth(g)
    P_gpu, rep = pg.solve(2)
    ro = O.solve(g, 2)
    assert rep["status"] == 0 and ro["status"] == 0
    assert abs(rep["cost_final"] - ro["cost_final"]) <= 1e-5 * ro["cost_final"]
    for a, b_ in zip(P_gpu, ro["poses"]):
        assert S.rotation_angle(a[:3, :3] @ b_[:3, :3].T) <= 1e-5 and np.abs(a[:3, 3] - b_[:3, 3]).max() <= 1e-6
    pb = bt.graph_from_synth(g)
    batch = bt.Batch()
    batch.add(pb)
    batch.set_shape(bt.BT_SINGLE_GRAPH_SHAPE)
    r_b = batch.solve(2)[0]
    assert r_b["cost_final"] == rep["cost_final"] and np.array_equal(pb.get_poses(), P_gpu)
    batch.close()
    P = _params(8)
    ws = bt.WarmStart(P)
    pw = bt.graph_from_synth(g)
    ws.apply(pw)
    got = pw.get_poses()
    D = {}
    for (i, j, pi, pj) in g.matches:
        M0 = g.pose_init[j] @ np.linalg.inv(g.pose_init[i])
        x, c = W.features(pi, pj, M0)
        y, _ = W.forward(P.astype(np.float64), x)
        D[(i, j)] = W.increment(y, c)
    ref = W.average(list(g.pose_init), list(g.fixed), D)
    for k in range(g.n):
        rot = S.rotation_angle(got[k][:3, :3] @ ref[k][:3, :3].T)
        assert rot < 1e-4 and np.max(np.abs(got[k][:3, 3] - ref[k][:3, 3])) < 1e-5, k
    ws.close()
    for h in (pg, pb, pw):
        h.close()


def test_training_resumes_from_checkpoint(bt):
    """Parameters + Adam state saved after 20 steps and loaded into a fresh
    warm start continue exactly as the uninterrupted run (bit for bit); a
    warm start given the parameters alone (moments cleared) takes different
    steps."""
    graphs = [S.training_graph(k) for k in range(12)]

    def fresh(params):
        ws = bt.WarmStart(params)
        for g in graphs:
            pg = bt.graph_from_synth(g)
            ws.add_graph(pg, g.pose_init, g.pose_true)
            pg.close()
        return ws

    rng = np.random.default_rng(3)
    a = fresh(S.warmstart_init(2))
    n = a.num_samples()
    batches = [rng.choice(n, 16, replace=False) for _ in range(40)]
    for ids in batches[:20]:
        a.train_step(ids, 1e-3)
    params, (m, v, t) = a.get_params(), a.get_adam()
    assert t == 20 and np.abs(m).max() > 0 and v.min() >= 0
    for ids in batches[20:]:
        a.train_step(ids, 1e-3)
    b = fresh(params)
    b.set_adam(m, v, t)
    for ids in batches[20:]:
        b.train_step(ids, 1e-3)
    assert np.array_equal(a.get_params(), b.get_params())
    assert b.get_adam()[2] == 40
    c = fresh(params)                      # moments cleared by set_params
    for ids in batches[20:]:
        c.train_step(ids, 1e-3)
    assert not np.array_equal(a.get_params(), c.get_params())
    with pytest.raises(bt.BTError):
        c.set_adam(m, -np.abs(v) - 1.0, 5)
    for w in (a, b, c):
        w.close()
