"""FP64 oracle of the learned-setup network and its data -- TEST INFRASTRUCTURE.

The learned setup is not in the paper; it predicts the blocks that
Algorithm 2 computes, from each block's prescaled operator window.  This
module restates, in plain numpy:

  * the network  X -> relu(X W1^T + b1) -> relu(. W2^T + b2) -> . W3^T + b3,
    with every weight matrix rounded to BF16 (round to nearest, ties to
    even) before use, and its mean-squared-error loss;
  * the gradients of that loss w.r.t. the FP32 master parameters by
    backpropagation written out layer by layer (the rounding is treated as
    the identity, as the training kernels do);
  * the features (prescaled operator rows over the (bs+2)^2 window of a
    block) and targets (prescaled Lambda~ blocks of an oracle cascade).

Pinned in tests/test_oracle_mlp.py by central finite differences and by
the definitions of the features, targets, rounding and loss.  ``planted``
(tests only) makes one step take a known-wrong form, so that a test can show
that the pins reject it.
"""
from __future__ import annotations

import contextlib

import numpy as np

# planted mistakes (tests only): None runs every step as stated
PLANTS = ("weights_unrounded", "loss_sum", "relu_grad_open", "window_mirror", "target_unscaled")
_planted = None


@contextlib.contextmanager
def planted(name: str):
    """Inside the block one step takes the named known-wrong form."""
    global _planted
    assert name in PLANTS
    _planted = name
    try:
        yield
    finally:
        _planted = None


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (r.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def unpack(p, nin, nhid, nout):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = []
    for shape in ((nhid, nin), (nhid,), (nhid, nhid), (nhid,), (nout, nhid), (nout,)):
        n = int(np.prod(shape))
        out.append(p[o:o + n].reshape(shape))
        o += n
    return out


def _rounder(bf16):
    """Weights as used in the products: BF16-rounded FP32 masters, or exact."""
    if bf16 and _planted != "weights_unrounded":
        return lambda w: bf16_round(np.asarray(w, dtype=np.float32))
    return lambda w: np.asarray(w, dtype=np.float64)


def forward(p, X, nin, nhid, nout, bf16=True):
    W1, b1, W2, b2, W3, b3 = unpack(p, nin, nhid, nout)
    q = _rounder(bf16)
    Z1 = X @ q(W1).T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ q(W2).T + b2
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ q(W3).T + b3
    return Y, (Z1, H1, Z2, H2)


def loss_and_grad(p, X, T, nin, nhid, nout, bf16=True):
    """MSE = mean((Y - T)^2) over all entries, and its gradient (flat, same
    layout as p)."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(p, nin, nhid, nout)
    q = _rounder(bf16)
    Y, (Z1, H1, Z2, H2) = forward(p, X, nin, nhid, nout, bf16)
    n = Y.size
    E = Y - T
    if _planted == "loss_sum":
        n = 1
    loss = float(np.sum(E * E) / n)
    dY = 2.0 * E / n
    dW3 = dY.T @ H2
    db3 = dY.sum(axis=0)
    dH2 = dY @ q(W3)
    dZ2 = dH2 * (Z2 > 0) if _planted != "relu_grad_open" else dH2
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ q(W2)
    dZ1 = dH1 * (Z1 > 0)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, g


def block_features(A, bs: int) -> np.ndarray:
    """[nblocks, bs^2 (bs+2)^2]: for every block (x fastest over the block
    grid) and block node p (x fastest), the row of W A W (W = diag A^-1/2)
    over the window of nodes bs*b-1 .. bs*b+bs, zero outside the grid."""
    nx, ny, _ = A.n
    d = None
    for s, o in enumerate(A.offsets):
        if o == (0, 0, 0):
            d = A.coeff[s]
    w = 1.0 / np.sqrt(d)
    nbx, nby = -(-nx // bs), -(-ny // bs)
    win = bs + 2
    sx = -1 if _planted == "window_mirror" else 1
    F = np.zeros((nbx * nby, bs * bs * win * win))
    for by in range(nby):
        for bx in range(nbx):
            b = bx + nbx * by
            for p in range(bs * bs):
                lx, ly = p % bs, p // bs
                ix, iy = bs * bx + lx, bs * by + ly
                if ix >= nx or iy >= ny:
                    continue
                i = ix + nx * iy
                for s, (dx, dy, _) in enumerate(A.offsets):
                    jx, jy = ix + dx, iy + dy
                    if not (0 <= jx < nx and 0 <= jy < ny):
                        continue
                    j = jx + nx * jy
                    F[b, p * win * win + (lx + sx * dx + 1) + win * (ly + sx * dy + 1)] += w[i] * A.coeff[s, i] * w[j]
    return F


def block_targets(lam_blocks: np.ndarray, A, bs: int, nu: int) -> np.ndarray:
    """Prescaled blocks W^-1 Lambda_l W^-1 in the padded bs^2 x bs^2 layout
    (absent nodes zero) from an oracle cascade's Lambda ([nu][sum n_b^2],
    blocks in order, each over its present nodes)."""
    nx, ny, _ = A.n
    d = None
    for s, o in enumerate(A.offsets):
        if o == (0, 0, 0):
            d = A.coeff[s]
    nbx, nby = -(-nx // bs), -(-ny // bs)
    nm = bs * bs
    T = np.zeros((nbx * nby, nu * nm * nm))
    for l in range(nu):
        off = 0
        for by in range(nby):
            for bx in range(nbx):
                b = bx + nbx * by
                pres = []
                for p in range(nm):
                    ix, iy = bs * bx + p % bs, bs * by + p // bs
                    if ix < nx and iy < ny:
                        pres.append((p, ix + nx * iy))
                k = len(pres)
                blk = lam_blocks[l, off:off + k * k].reshape(k, k)
                off += k * k
                for a, (p, i) in enumerate(pres):
                    for c, (qq, j) in enumerate(pres):
                        sc = 1.0 if _planted == "target_unscaled" else np.sqrt(d[i] * d[j])
                        T[b, (l * nm + p) * nm + qq] = blk[a, c] * sc
    return T
