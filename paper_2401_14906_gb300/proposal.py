"""Training and evaluation of the learned smoothing proposal (see include/sn.h).

Training data: seeded 256^3 uint16 maps (even indices Voronoi partitions with
20-93 seeds, odd ones 1-20 ellipsoids), extracted and smoothed by the plain GPU
path (16 sweeps, relaxation 0.5, constraint distance 1); every point is one
example (its features, its final offset).  The model is trained by AdamW with
the library's kernels and saved as PROPOSAL_PARAMS (float32, SN_LEARN_PARAMS
values).

Evaluation on a map: the plain smoother's offsets after `iterations` sweeps
are the reference; the proposal plus k correction sweeps is compared with them
(largest per-axis offset difference over all points, voxel units) and both are
timed with CUDA events on the same stream.

    python -m paper_2401_14906_gb300.proposal --maps 200 --epochs 4
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import sn

HERE = os.path.dirname(os.path.abspath(__file__))
PROPOSAL_PARAMS = os.path.join(HERE, "proposal_params.npy")
PROPOSAL_META = os.path.join(HERE, "proposal_params.json")


def _dev(labels):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(labels).view(
        {1: np.uint8, 2: np.int16, 4: np.int32}[labels.dtype.itemsize])).cuda()
    return t.view({1: torch.uint8, 2: torch.uint16, 4: torch.uint32}[labels.dtype.itemsize])


def he_uniform(seed):
    """Initial parameters: weights uniform in +-sqrt(6 / fan_in), zero biases (numpy PCG64, seeded)."""
    rng = np.random.default_rng(seed)
    parts = []
    for rows, cols in ((64, 32), (64, None), (64, 64), (64, None), (3, 64), (3, None)):
        if cols is None:
            parts.append(np.zeros(rows))
        else:
            parts.append(rng.uniform(-np.sqrt(6.0 / cols), np.sqrt(6.0 / cols), size=rows * cols))
    return np.concatenate(parts).astype(np.float32)


def train(n_maps=200, epochs=4, batch=4096, lr=2e-3, weight_decay=1e-4, iterations=16, relaxation=0.5,
          constraint=1.0, seed=0, log=print):
    import sn_synth
    L = sn.sn_learner_create()
    sn.sn_learner_set_params(L, he_uniform(seed))
    t0 = time.time()
    for i in range(n_maps):
        w = sn_synth.config4_train_map(i)
        m = sn.sn_extract(_dev(w.labels))
        sn.sn_smooth(m, iterations, relaxation, constraint)
        sn.sn_learner_add_examples(L, m, constraint)
        m.free()
    n = sn.sn_learner_n_examples(L)
    log(f"[proposal] {n_maps} maps, {n} examples in {time.time() - t0:.1f} s")
    losses = []
    for ep in range(epochs):
        t1 = time.time()
        loss = sn.sn_learner_train(L, 1, batch, lr * (0.5 ** (ep // 2)), weight_decay, seed=seed * 1000 + ep)
        losses.append(loss)
        log(f"[proposal] epoch {ep}: last minibatch mse {loss:.6f} ({time.time() - t1:.1f} s)")
    meta = {"maps": n_maps, "examples": n, "epochs": epochs, "batch": batch, "lr": lr,
            "weight_decay": weight_decay, "iterations": iterations, "relaxation": relaxation,
            "constraint": constraint, "seed": seed, "losses": losses}
    return L, meta


def evaluate(L, labels, spacing=(1.0, 1.0, 1.0), iterations=16, relaxation=0.5, constraint=1.0,
             corrections=(0, 2, 4), repeats=10, engines=("mma_sync",)):
    """Plain smoothing vs proposal + k corrections on one map: errors (voxels) and device times (ms)."""
    import torch
    stream = torch.cuda.current_stream()
    m = sn.sn_extract(_dev(labels), spacing)
    np_ = m.counts[0]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(repeats):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / repeats

    ms_plain = timed(lambda: sn.sn_smooth(m, iterations, relaxation, constraint))
    ref = sn.sn_mesh_device_arrays(m)["offsets"].clone()
    out = {"points": np_, "iterations": iterations, "ms_plain": ms_plain, "learned": []}
    for engine in engines:
        sn.sn_learner_set_engine(L, engine)
        for k in corrections:
            ms = timed(lambda: sn.sn_smooth_learned(m, L, k, relaxation, constraint))
            off = sn.sn_mesh_device_arrays(m)["offsets"]
            err = (off - ref).abs()
            out["learned"].append({"engine": engine, "corrections": k, "ms": ms,
                                   "speedup": ms_plain / ms if ms > 0 else None,
                                   "max_err_vox": float(err.max().item()) if np_ else 0.0,
                                   "mean_err_vox": float(err.mean().item()) if np_ else 0.0})
    sn.sn_learner_set_engine(L, "mma_sync")
    m.free()
    return out


def load_learner(path=PROPOSAL_PARAMS):
    p = np.load(path).astype(np.float32)
    L = sn.sn_learner_create()
    sn.sn_learner_set_params(L, p)
    return L


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--maps", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=PROPOSAL_PARAMS)
    ap.add_argument("--eval-dims", type=int, default=512)
    a = ap.parse_args()
    import sn_synth
    L, meta = train(a.maps, a.epochs, a.batch, a.lr, seed=a.seed)
    np.save(a.out, sn.sn_learner_get_params(L))
    w = sn_synth.config2((a.eval_dims,) * 3)
    meta["eval"] = evaluate(L, w.labels, w.spacing)
    meta["eval_map"] = f"atlas-like {a.eval_dims}^3 uint16, 93 labels"
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta["eval"]))


if __name__ == "__main__":
    main()
