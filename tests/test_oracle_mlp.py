"""Pins of the learned-setup oracle (oracle/mlp.py) and of the workload-5
generator: backpropagation against central finite differences, BF16 rounding
against its definition, features/targets against direct definitions, and the
Q1 stencil against its closed form."""
import numpy as np
import pytest

import oracle
import problems
from oracle import mlp as om


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.001953125, 1.005859375, -3.14159, 0.0], dtype=np.float32)
    r = om.bf16_round(x)
    # BF16 keeps 7 mantissa bits: 1 + 2^-8 is a tie -> even (1.0); 1 + 2^-9 rounds down;
    # 1 + 3*2^-9 is past the midpoint -> 1 + 2^-7
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 and r[3] == 1.0078125
    assert abs(r[4] - (-3.140625)) < 1e-12 and r[5] == 0.0
    rng = np.random.default_rng(0)
    v = rng.standard_normal(1000).astype(np.float32)
    rv = om.bf16_round(v)
    assert np.all(np.abs(rv - v) <= np.abs(v) * 2.0 ** -8 + 1e-30)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    nin, nhid, nout, B = 7, 5, 4, 6
    n = nhid * nin + nhid + nhid * nhid + nhid + nout * nhid + nout
    p = rng.standard_normal(n) * 0.5
    X = rng.standard_normal((B, nin))
    T = rng.standard_normal((B, nout))
    loss, g = om.loss_and_grad(p, X, T, nin, nhid, nout, bf16=False)
    h = 1e-6
    fd = np.zeros(n)
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        fd[k] = (om.loss_and_grad(p + e, X, T, nin, nhid, nout, bf16=False)[0]
                 - om.loss_and_grad(p - e, X, T, nin, nhid, nout, bf16=False)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-9)


def test_loss_is_the_mean_squared_error():
    """At zero parameters the output is zero and the loss is mean(T^2) over
    all B x nout entries; the finite differences above cannot see a
    consistent rescaling of loss and gradient, this can."""
    rng = np.random.default_rng(2)
    nin, nhid, nout, B = 4, 3, 5, 6
    n = nhid * nin + nhid + nhid * nhid + nhid + nout * nhid + nout
    T = rng.standard_normal((B, nout))
    loss, g = om.loss_and_grad(np.zeros(n), rng.standard_normal((B, nin)), T, nin, nhid, nout)
    assert loss == pytest.approx(np.mean(T ** 2), rel=1e-15)
    # only the output bias sees the error at zero weights: d loss / d b3 = -2 mean_rows(T) / nout
    np.testing.assert_allclose(g[-nout:], -2.0 * T.sum(axis=0) / T.size, rtol=1e-14)


def test_q1_closed_form_and_structure():
    A = problems.q1_jittered(6, 1, jitter=0.0, kappa=np.ones((7, 7)))
    c = A.coeff.reshape(9, 6, 6)
    # the standard bilinear-element Laplacian stencil (1/3)[-1 -1 -1; -1 8 -1; -1 -1 -1]
    np.testing.assert_allclose(c[:, 2, 2] * 3, [-1, -1, -1, -1, 8, -1, -1, -1, -1], atol=1e-12)
    from tests import dense_ref
    A = problems.q1_jittered(8, 5)
    D = dense_ref.dense_from_stencil(A)
    assert np.abs(D - D.T).max() <= 1e-12 * np.abs(D).max()
    assert np.linalg.eigvalsh(D).min() > 0
    rs = D.sum(1).reshape(8, 8)
    assert np.abs(rs[1:-1, 1:-1]).max() <= 1e-12 * np.abs(D).max()  # constants in the kernel away from the boundary


def test_features_and_targets_definitions():
    A = problems.q1_jittered(10, 3)
    bs = 3
    F = om.block_features(A, bs)
    nbx = 4
    assert F.shape == (16, 9 * 25)
    # centre entry of each present node's row is the prescaled diagonal = 1
    win = 5
    for b in range(16):
        bx, by = b % nbx, b // nbx
        for p in range(9):
            ix, iy = 3 * bx + p % 3, 3 * by + p // 3
            v = F[b, p * 25 + (p % 3 + 1) + win * (p // 3 + 1)]
            assert (v == pytest.approx(1.0)) if (ix < 10 and iy < 10) else v == 0.0
    h = oracle.Hierarchy(A, bs=bs, max_levels=1)
    c = oracle.Cascade(h, "additive", nu=2)
    T = om.block_targets(c.lam(0), A, bs, 2)
    assert T.shape == (16, 2 * 81)
    d = A.coeff[4]
    # a full block's target equals sqrt(d_i d_j) Lambda_ij
    lam = c.lam(0)
    blk0 = lam[0, :81].reshape(9, 9)
    idx = [0, 1, 2, 10, 11, 12, 20, 21, 22]
    np.testing.assert_allclose(T[0, :81].reshape(9, 9), blk0 * np.sqrt(np.outer(d[idx], d[idx])), rtol=1e-13)


def _dense_prescaled(A):
    from tests import dense_ref
    D = dense_ref.dense_from_stencil(A)
    w = 1.0 / np.sqrt(np.diag(D))
    return w[:, None] * D * w[None, :]


@pytest.mark.parametrize("n,bs", [(10, 3), (9, 2)])
def test_features_are_the_prescaled_rows_over_every_window(n, bs):
    """Every entry of the features against the definition read off the dense
    prescaled operator W A W (built independently of the stencil walk): block
    node p's row over the (bs+2)^2 window of nodes bs*b - 1 .. bs*b + bs,
    zero outside the grid and for absent nodes of edge blocks."""
    A = problems.q1_jittered(n, 7)
    At = _dense_prescaled(A)
    F = om.block_features(A, bs)
    nb1 = -(-n // bs)
    win = bs + 2
    ref = np.zeros_like(F)
    for by in range(nb1):
        for bx in range(nb1):
            for p in range(bs * bs):
                ix, iy = bs * bx + p % bs, bs * by + p // bs
                if ix >= n or iy >= n:
                    continue
                for v in range(win):
                    for u in range(win):
                        jx, jy = bs * bx - 1 + u, bs * by - 1 + v
                        if 0 <= jx < n and 0 <= jy < n:
                            ref[bx + nb1 * by, p * win * win + u + win * v] = At[ix + n * iy, jx + n * jy]
    np.testing.assert_allclose(F, ref, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("n,bs", [(10, 3), (9, 2)])
def test_targets_are_the_prescaled_blocks_of_every_block(n, bs):
    """Every block's target, edge blocks included, against the dense
    block-diagonal Lambda_l of the oracle's cascade: W^-1 Lambda_l W^-1 on
    the present nodes, zero on the absent ones."""
    from tests import dense_ref
    A = problems.q1_jittered(n, 9)
    nu = 2
    h = oracle.Hierarchy(A, bs=bs, max_levels=1)
    c = oracle.Cascade(h, "additive", nu=nu)
    T = om.block_targets(c.lam(0), A, bs, nu)
    blocks, _ = dense_ref.block_partition(A.n, 2, bs)
    lam = c.lam(0)
    offs = np.cumsum([0] + [len(r) ** 2 for r in blocks])
    d = np.diag(dense_ref.dense_from_stencil(A))
    nb1 = -(-n // bs)
    nm = bs * bs
    for l in range(nu):
        L = np.zeros((A.N, A.N))
        for b, rows in enumerate(blocks):
            L[np.ix_(rows, rows)] = lam[l, offs[b]:offs[b + 1]].reshape(len(rows), len(rows))
        Lt = np.sqrt(d)[:, None] * L * np.sqrt(d)[None, :]
        for by in range(nb1):
            for bx in range(nb1):
                b = bx + nb1 * by
                for p in range(nm):
                    for q in range(nm):
                        ip = (bs * bx + p % bs, bs * by + p // bs)
                        iq = (bs * bx + q % bs, bs * by + q // bs)
                        present = max(ip + iq) < n
                        want = Lt[ip[0] + n * ip[1], iq[0] + n * iq[1]] if present else 0.0
                        assert T[b, (l * nm + p) * nm + q] == pytest.approx(want, rel=1e-13, abs=1e-15)


def test_forward_rounds_the_weights_to_bf16():
    """The products take BF16 weights: with weights that BF16 represents the
    rounded and exact forward passes agree bitwise; with generic weights
    they differ, by no more than a relative rounding of u = 2^-9 + 2^-23 per
    weight (FP32 master, then BF16) can move each output through the three
    layers (ReLU is 1-Lipschitz): ((1 + u)^3 - 1) times the forward pass on
    |X|, |W|, |b|."""
    rng = np.random.default_rng(3)
    nin, nhid, nout, B = 9, 8, 5, 7
    n = nhid * nin + nhid + nhid * nhid + nhid + nout * nhid + nout
    X = rng.standard_normal((B, nin))
    p = rng.standard_normal(n) * 0.4
    W1, b1, W2, b2, W3, b3 = om.unpack(p, nin, nhid, nout)
    # BF16-representable weights (8 significant bits), biases left as they are
    pr = p.copy()
    o = 0
    for shape in ((nhid, nin), (nhid,), (nhid, nhid), (nhid,), (nout, nhid), (nout,)):
        k = int(np.prod(shape))
        if len(shape) == 2:
            m, e = np.frexp(pr[o:o + k])
            pr[o:o + k] = np.ldexp(np.round(m * 256) / 256, e)
        o += k
    Yr, _ = om.forward(pr, X, nin, nhid, nout, bf16=True)
    Ye, _ = om.forward(pr, X, nin, nhid, nout, bf16=False)
    assert np.array_equal(Yr, Ye)
    Yg, _ = om.forward(p, X, nin, nhid, nout, bf16=True)
    Yx, _ = om.forward(p, X, nin, nhid, nout, bf16=False)
    Ya = np.abs(X)
    for W, bb in ((W1, b1), (W2, b2), (W3, b3)):
        Ya = Ya @ np.abs(W).T + np.abs(bb)
    bound = ((1 + 2.0 ** -9 + 2.0 ** -23) ** 3 - 1) * Ya * (1 + 1e-12)
    diff = np.abs(Yg - Yx)
    assert diff.max() > 0 and np.all(diff <= bound)
