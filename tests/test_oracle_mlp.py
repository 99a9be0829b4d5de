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
