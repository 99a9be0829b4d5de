"""Training and use of the learned cascade setup (orchestration only).

The arithmetic -- exact block setups that label the data, feature
extraction, the network's forward/backward passes and Adam -- runs in the
library's kernels; this module only loops over meshes and minibatches.
"""
from __future__ import annotations

import time

import torch

import paper_2606_12577_gb300 as cmg


def label_mesh(A, bs: int = 3, nu: int = 3):
    """(features, targets) of every block of the finest level of operator A,
    targets from the exact additive cascade (Algorithm 2)."""
    coeff = torch.tensor(A.coeff, dtype=torch.float64, device="cuda")
    h = cmg.setup_hierarchy(A.dim, A.n, A.offsets, coeff, block=bs, max_levels=1)
    c = cmg.setup_cascade(h, "additive", nu=nu)
    return cmg.block_features(h, 0), cmg.block_targets(c, 0)


def make_dataset(meshes, bs: int = 3, nu: int = 3, total: int | None = None):
    """Labelled blocks of every mesh (an iterable, consumed one mesh at a
    time, so meshes can stream in while earlier ones are labelled).  With
    ``total`` (the number of blocks over all meshes) the data set is
    allocated once and filled in place; otherwise the per-mesh tensors are
    concatenated."""
    Xs, Ts = [], []
    X = T = None
    pos = 0
    for A in meshes:
        Xm, Tm = label_mesh(A, bs, nu)
        if total is None:
            Xs.append(Xm)
            Ts.append(Tm)
            continue
        if X is None:
            X = torch.empty((total, Xm.shape[1]), dtype=Xm.dtype, device=Xm.device)
            T = torch.empty((total, Tm.shape[1]), dtype=Tm.dtype, device=Tm.device)
        X[pos:pos + Xm.shape[0]] = Xm
        T[pos:pos + Tm.shape[0]] = Tm
        pos += Xm.shape[0]
        del Xm, Tm
    if total is None:
        return torch.cat(Xs), torch.cat(Ts)
    return X[:pos], T[:pos]


def train(model: "cmg.MLP", X, T, steps: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
          lr_final: float = 1e-5, log_every: int = 10):
    """Adam on minibatches drawn without replacement per epoch (a random
    permutation per epoch; each batch gathers its rows, so the data set is
    never copied whole); the learning rate decays geometrically from lr to
    lr_final.  The loss is read back (one synchronisation) every
    ``log_every`` steps and at the last one; returns those losses."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    n = X.shape[0]
    batch = min(batch, n, model.max_batch)
    perm = torch.randperm(n, device="cuda", generator=g)
    pos = 0
    hist = []
    decay = (lr_final / lr) ** (1.0 / max(1, steps - 1))
    for k in range(steps):
        if pos + batch > n:
            perm = torch.randperm(n, device="cuda", generator=g)
            pos = 0
        idx = perm[pos:pos + batch]
        want = k % log_every == 0 or k == steps - 1
        loss = model.train_step(X.index_select(0, idx), T.index_select(0, idx), lr * decay ** k, with_loss=want)
        pos += batch
        if want:
            hist.append(loss)
    return hist


def setup_pair(A, model, bs: int = 3, nu: int = 3, lowp: bool = False):
    """Exact and learned cascades on the same hierarchy, with their setup
    times (ms, CUDA events on the current stream)."""
    coeff = torch.tensor(A.coeff, dtype=torch.float64, device="cuda")
    h = cmg.setup_hierarchy(A.dim, A.n, A.offsets, coeff, block=bs)
    s = torch.cuda.current_stream()
    out = {}
    for name, mdl in (("exact", None), ("learned", model)):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(s)
        c = cmg.setup_cascade(h, "additive", nu=nu, lowp=lowp, model=mdl)
        e1.record(s)
        torch.cuda.synchronize()
        out[name] = (c, e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3)
    return h, out
