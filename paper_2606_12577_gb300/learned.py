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


def make_dataset(meshes, bs: int = 3, nu: int = 3):
    Xs, Ts = [], []
    for A in meshes:
        X, T = label_mesh(A, bs, nu)
        Xs.append(X)
        Ts.append(T)
    return torch.cat(Xs), torch.cat(Ts)


def train(model: "cmg.MLP", X, T, steps: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
          lr_final: float = 1e-5, log_every: int = 10):
    """Adam on minibatches drawn without replacement per epoch (one permuted
    copy of the data per epoch, batches are contiguous slices of it); the
    learning rate decays geometrically from lr to lr_final.  The loss is read
    back (one synchronisation) every ``log_every`` steps and at the last one;
    returns those losses."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    n = X.shape[0]
    batch = min(batch, n, model.max_batch)

    def shuffled():
        perm = torch.randperm(n, device="cuda", generator=g)
        return X.index_select(0, perm).contiguous(), T.index_select(0, perm).contiguous()

    Xs, Ts = shuffled()
    pos = 0
    hist = []
    decay = (lr_final / lr) ** (1.0 / max(1, steps - 1))
    for k in range(steps):
        if pos + batch > n:
            Xs, Ts = shuffled()
            pos = 0
        want = k % log_every == 0 or k == steps - 1
        loss = model.train_step(Xs[pos:pos + batch], Ts[pos:pos + batch], lr * decay ** k, with_loss=want)
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
