"""Trains the learned warm start (bt_warmstart_*) on seeded synthetic graphs.

Each training graph (synthgen.training_graph: 2-4 views, the object, noise,
correspondence and initialisation model of the batched workload) is solved
by the plain Gauss-Newton solver of the library (bt_solve, 10 iterations from
the perturbed initial poses); every correspondence set becomes one sample
whose label is the increment from the initial to the converged relative
pose.  Worker processes generate and solve the graphs (each with its own CUDA
context) and return only the correspondence sets and the poses; the main
process stores the samples on the device and trains with the library's own
BF16 forward / backward kernels and Adam.

    python -m paper_2108_00516_gb300.train_warmstart --graphs 100000 --epochs 20 \
        --out paper_2108_00516_gb300/weights/warmstart.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

DEFAULT_OUT = Path(__file__).resolve().parent / "weights" / "warmstart.npz"


def _label_job(args):
    """Worker: one training graph, solved by the plain GPU solver."""
    k, seed_base, iters = args
    import synthgen as S
    from paper_2108_00516_gb300 import bt
    g = S.training_graph(k, seed_base)
    pg = bt.graph_from_synth(g)
    P, rep = pg.solve(iters, raise_on_error=False)
    pg.close()
    if rep["status"] != 0:
        return None
    return g.pose_init.copy(), P, [(i, j, pi, pj) for (i, j, pi, pj) in g.matches if len(pi) > 0]


def collect(pool, ids, seed_base, iters, ws, log, what):
    t0 = time.time()
    n_graphs = n_sets = skipped = 0
    for res in pool.imap(_label_job, [(k, seed_base, iters) for k in ids], chunksize=8):
        if res is None:
            skipped += 1
            continue
        P0, P, sets = res
        for (i, j, pi, pj) in sets:
            ws.add_set(pi, pj, P0[i], P0[j], P[i], P[j])
            n_sets += 1
        n_graphs += 1
        if n_graphs % 5000 == 0:
            log(f"  {what}: {n_graphs} graphs, {n_sets} sets, {time.time() - t0:.0f} s")
    log(f"{what}: {n_graphs} graphs ({skipped} singular, skipped), {n_sets} sets in {time.time() - t0:.1f} s")
    return n_graphs, n_sets


def edge_errors(ws, ids):
    """Mean |omega - omega*| (deg) and |u - u*| (mm) of the network's edge
    increments, and the same for the zero increment (the plain start)."""
    ids = np.asarray(ids)
    y = ws.predict(ids).astype(np.float64)
    lab = np.stack([ws.sample(int(k))[1] for k in ids]).astype(np.float64)
    rot = lambda d: np.degrees(np.linalg.norm(d[:, :3], axis=1) * 0.1)
    tr = lambda d: np.linalg.norm(d[:, 3:], axis=1) * 10.0
    return dict(net_rot_deg=float(rot(y - lab).mean()), net_trans_mm=float(tr(y - lab).mean()),
                init_rot_deg=float(rot(lab).mean()), init_trans_mm=float(tr(lab).mean()))


def mean_loss(ws, ids, chunk=1024):
    tot = 0.0
    for a in range(0, len(ids), chunk):
        part = ids[a:a + chunk]
        loss, _ = ws.gradient(part)
        tot += loss * len(part)
    return tot / max(1, len(ids))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--graphs", type=int, default=100000)
    ap.add_argument("--heldout", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-min", type=float, default=2e-5)
    ap.add_argument("--label-iters", type=int, default=10)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=0)
    ap.add_argument("--out", type=str, default=str(DEFAULT_OUT))
    ap.add_argument("--checkpoint", type=str, default="",
                    help="after every epoch, save parameters, Adam state, epoch, step and RNG state here")
    ap.add_argument("--resume", type=str, default="", help="continue from a --checkpoint file")
    a = ap.parse_args(argv)
    log = lambda m: print(m, flush=True)

    from paper_2108_00516_gb300 import build as lbuild
    lbuild.build()
    import synthgen as S
    # the workers fork before this process touches CUDA; each makes its own context
    import multiprocessing as mp
    workers = a.workers or max(1, (os.cpu_count() or 2) - 1)
    pool = mp.get_context("fork").Pool(workers)
    from paper_2108_00516_gb300 import bt
    bt.load()
    ws = bt.WarmStart(S.warmstart_init(a.init_seed))
    t_start = time.time()
    n_tr_graphs, n_tr = collect(pool, range(a.graphs), S.TRAIN_SEED, a.label_iters, ws, log, "train")
    n_ho_graphs, n_ho = collect(pool, range(a.heldout), S.HELDOUT_SEED, a.label_iters, ws, log, "held-out")
    pool.close()
    pool.join()
    t_data = time.time() - t_start
    train_ids = np.arange(n_tr, dtype=np.int32)
    ho_ids = np.arange(n_tr, n_tr + n_ho, dtype=np.int32)
    rng = np.random.default_rng(a.init_seed)
    steps_per_epoch = max(1, n_tr // a.batch)
    total = steps_per_epoch * a.epochs
    history = []
    before = edge_errors(ws, ho_ids) if n_ho else {}
    log(f"held-out edge error before training: {before}")
    t0 = time.time()
    step = 0
    first_epoch = 0
    if a.resume:
        ck = np.load(a.resume)
        ws.set_params(ck["params"])
        ws.set_adam(ck["adam_m"], ck["adam_v"], int(ck["adam_t"]))
        first_epoch, step = int(ck["epoch"]), int(ck["step"])
        rng.bit_generator.state = json.loads(str(ck["rng"]))
        history = json.loads(str(ck["history"]))
        log(f"resumed from {a.resume}: epoch {first_epoch}, step {step}")
    for ep in range(first_epoch, a.epochs):
        perm = rng.permutation(n_tr).astype(np.int32)
        run = 0.0
        for s in range(steps_per_epoch):
            lr = a.lr_min + 0.5 * (a.lr - a.lr_min) * (1 + math.cos(math.pi * step / total))
            want = s % 50 == 0
            loss = ws.train_step(perm[s * a.batch:(s + 1) * a.batch], lr, want_loss=want)
            if want:
                run = loss if run == 0.0 else 0.9 * run + 0.1 * loss
            step += 1
        val = mean_loss(ws, ho_ids) if n_ho else float("nan")
        history.append(dict(epoch=ep + 1, train_loss=run, heldout_loss=val, seconds=time.time() - t0))
        if a.checkpoint:
            m, v, adam_t = ws.get_adam()
            np.savez(a.checkpoint, params=ws.get_params(), adam_m=m, adam_v=v, adam_t=adam_t, epoch=ep + 1,
                     step=step, rng=json.dumps(rng.bit_generator.state), history=json.dumps(history))
        log(f"epoch {ep + 1}: train {run:.4f}  held-out {val:.4f}  ({time.time() - t0:.1f} s)")
    t_train = time.time() - t0
    after = edge_errors(ws, ho_ids) if n_ho else {}
    log(f"held-out edge error after training: {after}")
    meta = dict(graphs=n_tr_graphs, train_sets=n_tr, heldout_graphs=n_ho_graphs, heldout_sets=n_ho,
                epochs=a.epochs, batch=a.batch, lr=a.lr, lr_min=a.lr_min, label_iters=a.label_iters,
                init_seed=a.init_seed, train_seed=S.TRAIN_SEED, heldout_seed=S.HELDOUT_SEED,
                data_seconds=round(t_data, 1), train_seconds=round(t_train, 1), steps=step,
                heldout_edge_error_before=before, heldout_edge_error_after=after, history=history)
    out = Path(a.out)
    out.parent.mkdir(parents=True, exist_ok=True)
    np.savez(out, params=ws.get_params(), meta=json.dumps(meta))
    log(f"wrote {out}")
    ws.close()


if __name__ == "__main__":
    main()
