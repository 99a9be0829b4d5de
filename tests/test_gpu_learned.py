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


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 243, 232), (4096, 128, 512), (130, 20, 8), (256, 256, 1024),
                                   (1000, 300, 200), (640, 512, 4096), (4096, 2560, 256), (39000, 100, 72)])
def test_tc_gemm_matches_bf16_products(built, M, N, K):
    """The tcgen05 GEMM (TMA-staged 128 x 64 boxes, 128-byte swizzle, FP32
    accumulator in tensor memory; 128 x 128 tiles, or 128 x 256 when N > 128)
    against the exact products of the same BF16 values in FP64: every entry
    within the FP32 accumulation bound K 2^-24 sum_k |a_ik| |b_jk| (ragged M,
    N and K exercise the zero-filled tile edges, N = 300 a second 256-wide
    tile whose upper box starts past the last row; the last two shapes have
    enough tiles for the persistent kernel, with two TMEM accumulators, in
    128 x 256 and ragged 128 x 128 tiles)."""
    import torch

    import paper_2606_12577_gb300 as cmg
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = cmg.tc_gemm_bf16(A.cuda(), B.cuda()).cpu().numpy().astype(np.float64)
    a = A.to(torch.float64).numpy()
    b = B.to(torch.float64).numpy()
    ref = a @ b.T
    bound = K * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T) + 1e-30
    assert np.all(np.abs(C - ref) <= bound), float(np.max(np.abs(C - ref) / bound))


def test_tc_gemm_rejects_memory_off_the_device(built):
    """The C entry checks its operands before any launch: host memory is
    refused with CS_ERR_ARG."""
    from paper_2606_12577_gb300 import _capi
    a = np.zeros((128, 64), dtype=np.uint16)
    c = np.zeros((128, 128), dtype=np.float32)
    st = _capi.lib().cs_tc_gemm_bf16(128, 128, 64, a.ctypes.data, a.ctypes.data, c.ctypes.data, None)
    assert st == _capi.CS_ERR_ARG


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


def test_network_gains_over_the_method_without_it(built):
    """What the trained network gains: on a held-out 255^2 mesh, the learned
    setup (predicted blocks for Lambda_1..3, exact level-1 fallback) against
    the method without the network at the same sweeps per cycle (the exact
    level-1 blocks repeated: a nu = 1 cascade applied mu = 3 times).  Trained
    on 32 meshes of 63^2, the network's cascade contracts faster (stationary
    V-cycle convergence factor at least 0.03 lower) and its GMRES needs fewer
    iterations to 1e-10; it also stays within 0.03 of the exact cascade's
    convergence factor."""
    import torch

    import paper_2606_12577_gb300 as cmg
    from paper_2606_12577_gb300 import learned
    meshes = [problems.q1_jittered(63, 50000 + k) for k in range(32)]
    X, T = learned.make_dataset(meshes)
    m = cmg.MLP(X.shape[1], 128, T.shape[1], max_batch=4096, seed=1)
    learned.train(m, X, T, steps=3000, batch=4096, lr=2e-3)
    A = problems.q1_jittered(255, 10001)
    h, res = learned.setup_pair(A, m)
    used, _ = cmg.learned_status(res["learned"][0])
    assert used == 1
    res["level1_repeated"] = (cmg.setup_cascade(h, "additive", nu=1), 0.0, 0.0)
    b = torch.tensor(problems.rhs(A.N, 6), dtype=torch.float64, device="cuda")
    rho, its = {}, {}
    for name in ("exact", "learned", "level1_repeated"):
        c = res[name][0]
        mu = 3 if name == "level1_repeated" else 1
        x = torch.zeros(A.N, dtype=torch.float64, device="cuda")
        st = cmg.solve(h, c, b, x, method="stationary", tol=1e-10, maxit=40, mu_pre=mu, mu_post=mu,
                       raise_on_error=False)
        rho[name] = oracle.rho_from_history(st.history)
        x = torch.zeros(A.N, dtype=torch.float64, device="cuda")
        info = cmg.solve(h, c, b, x, method="gmres", tol=1e-10, maxit=200, mu_pre=mu, mu_post=mu)
        assert info.converged
        its[name] = info.iterations
    assert rho["learned"] <= rho["level1_repeated"] - 0.03, rho
    assert its["learned"] < its["level1_repeated"], its
    assert abs(rho["learned"] - rho["exact"]) <= 0.03, rho
