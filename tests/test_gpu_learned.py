"""The learned setup: feature / target extraction and the network's forward
pass and gradients against the FP64 oracle (oracle/mlp.py), training by the
library's own kernels, and the learned cascade inside a solve."""
import numpy as np
import pytest

import oracle
import problems
from oracle import mlp as om
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    return True


def test_features_and_targets_match_oracle(built):
    import paper_2606_12577_gb300 as cmg
    A = problems.q1_jittered(23, 4)
    hg = gu.gpu_hierarchy(A, block=3, max_levels=1)
    cg = cmg.setup_cascade(hg, "additive", nu=3)
    F = _host(cmg.block_features(hg, 0))
    T = _host(cmg.block_targets(cg, 0))
    Fo = om.block_features(A, 3)
    ho = oracle.Hierarchy(A, bs=3, max_levels=1)
    co = oracle.Cascade(ho, "additive", nu=3)
    To = om.block_targets(co.lam(0), A, 3, 3)
    assert np.abs(F - Fo).max() <= 1e-6 * np.abs(Fo).max()
    assert np.abs(T - To).max() <= 1e-6 * np.abs(To).max()


def test_forward_and_gradients_match_oracle(built):
    import torch

    import paper_2606_12577_gb300 as cmg
    nin, nhid, nout, B = 225, 128, 243, 300
    m = cmg.MLP(nin, nhid, nout, max_batch=512, seed=3)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((B, nin)).astype(np.float32) * 0.3
    T = rng.standard_normal((B, nout)).astype(np.float32) * 0.1
    Xd = torch.tensor(X, device="cuda")
    Td = torch.tensor(T, device="cuda")
    p = m.get_params().astype(np.float64)
    Y = _host(m.forward(Xd))
    Yo, _ = om.forward(p, X.astype(np.float64), nin, nhid, nout, bf16=True)
    assert np.abs(Y - Yo).max() <= 1e-4 * np.abs(Yo).max()
    loss, g = m.gradients(Xd, Td)
    lo, go = om.loss_and_grad(p, X, T, nin, nhid, nout, bf16=True)
    assert loss == pytest.approx(lo, rel=1e-5)
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()


def test_training_and_learned_setup(built):
    """Training on labels of the exact setup lowers the loss; the learned
    cascade (accepted or replaced by the exact one through the Frobenius
    check) solves to 1e-10; an accepted prediction's convergence factor is
    reported against the exact one."""
    import torch

    import paper_2606_12577_gb300 as cmg
    from paper_2606_12577_gb300 import learned
    meshes = [problems.q1_jittered(47, 100 + k) for k in range(8)]
    X, T = learned.make_dataset(meshes)
    m = cmg.MLP(X.shape[1], 128, T.shape[1], max_batch=4096, seed=7)
    hist = learned.train(m, X, T, steps=600, batch=1024, lr=2e-3, log_every=1)
    assert np.mean(hist[-20:]) < 0.2 * np.mean(hist[:5])
    A = problems.q1_jittered(95, 9999)
    h, res = learned.setup_pair(A, m)
    b = torch.tensor(problems.rhs(A.N, 5), dtype=torch.float64, device="cuda")
    used, ratio = cmg.learned_status(res["learned"][0])
    assert used in (0, 1) and ratio > 0
    st = cmg.learned_stats(res["learned"][0])
    assert st["blocks"] == 32 * 32 and st["full_blocks"] == 31 * 31  # 95 = 3 * 31 + 2
    if used == 1:
        # every kept block is within 5% of its exact level-1 objective and
        # every other block carries the exact level-1 block
        assert 0 < st["predicted_blocks"] <= st["full_blocks"]
        assert st["ratio_used"] <= 1.05 + 1e-12
    else:
        assert st["predicted_blocks"] == 0
    rhos = {}
    for name in ("exact", "learned"):
        c = res[name][0]
        x = torch.zeros(A.N, dtype=torch.float64, device="cuda")
        info = cmg.solve(h, c, b, x, method="gmres", tol=1e-10, maxit=200)
        assert info.converged
        r = problems.rhs(A.N, 5) - gu.stencil_matvec(A, _host(x))
        assert np.linalg.norm(r) / np.linalg.norm(problems.rhs(A.N, 5)) <= 1e-10
        rhos[name] = oracle.rho_from_history(info.history)
    if used == 1:
        assert rhos["learned"] < 1.0
