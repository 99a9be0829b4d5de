"""Block cascades (blocks of bs^dim nodes, Algorithm 2 with n_b > 1) and the
multi-RHS block product X_b -= Lambda_b R_b, through the C ABI, against the
FP64 oracle: Lambda to 1e-12 relative, smoothing (forward and reverse, i.e.
transposed blocks), V-cycles and solves to 1e-12 / the oracle's iteration
counts.  Sizes leave partial blocks at the upper edges."""
import numpy as np
import pytest

import oracle
import problems
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu
TOL = 1e-12
# FP32 products in the block setup: R and E entries carry a few (nst + 1) u of
# their row sums (u = 2^-24), the n_b x n_b Gram matrices about nR u of their
# entries, and the FP64 block solve multiplies that by cond(G) (up to ~1e2 on
# these variable-coefficient 2x2 blocks), over nu steps: 1e-3.
FP32_BLOCK_TOL = 1e-3
# On the contrast-1e4 correlated field the coarse levels' block Gram matrices
# have eigenvalues between 1e-14 and 1e-5 of their trace: FP64 keeps them,
# FP32 products cannot resolve them and the 1e-5 cutoff drops them, so Lambda
# differs by a few 1e-2 there (2.7e-2 measured on level 3); the smoother, and
# the iteration count, stay as good.
FP32_BLOCK_TOL_CONTRAST = 1e-1


def _dev(a, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _var(dim, n, seed, lo=-1.0, hi=1.0):
    return problems.variable_poisson(problems.random_coefficients(dim, n, seed, lo, hi))


PROBS = {
    "v2d_37": lambda: _var(2, 37, 3),
    "c2d_66": lambda: problems.variable_poisson(problems.log_uniform_field(2, 66, 6.0, 266, -2.0, 2.0)),
    "v3d_17": lambda: _var(3, 17, 5),
    "p2d_33": lambda: problems.poisson(2, 33),
}


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    return True


@pytest.mark.parametrize("name,kind,nu,alpha,tol", [("v2d_37", "additive", 3, 0, FP32_BLOCK_TOL),
                                                  ("v3d_17", "additive", 2, 0, FP32_BLOCK_TOL),
                                                  ("v2d_37", "multiplicative", 3, 0, FP32_BLOCK_TOL),
                                                  ("c2d_66", "multiplicative", 3, 0, FP32_BLOCK_TOL_CONTRAST)])
def test_fp32_block_setup_matches_oracle(built, name, kind, nu, alpha, tol):
    """setup_precision fp32 on block levels: R and E rows in FP32, the block
    Gram and cross products in FP32 over chunks of 8 and FP64 across them,
    the least squares in FP64 with the minimum-norm cutoff at 1e-5 tr(G)
    (FP32 products lift an exactly null eigenvalue to ~1e-7 tr(G); such Gram
    matrices occur from the second step on the 9-point levels).  Lambda
    within FP32_BLOCK_TOL of the oracle, and the FP32-cycle GMRES reaches
    1e-10."""
    import torch

    import paper_2606_12577_gb300 as cmg
    A = PROBS[name]()
    ho = oracle.Hierarchy(A, bs=2)
    co = oracle.Cascade(ho, kind, nu=nu, alpha=alpha)
    hg = gu.gpu_hierarchy(A, block=2)
    cg = cmg.setup_cascade(hg, kind, nu=nu, alpha=alpha, lowp=True, setup_precision="fp32")
    errs = [gu.rel_max(cmg.export_lambda(cg, l), co.lam(l)) for l in range(co.nlev)]
    assert max(errs) <= tol, errs
    assert max(errs) > 0.0
    c64 = cmg.setup_cascade(hg, kind, nu=nu, alpha=alpha, lowp=True)
    b = problems.rhs(A.N, 13)
    its = []
    for c in (cg, c64):
        x = torch.zeros(A.N, dtype=torch.float64, device="cuda")
        info = cmg.solve(hg, c, _dev(b), x, method="gmres_right", precision="fp32", tol=1e-10, maxit=300)
        assert info.converged
        its.append(info.iterations)
    assert its[0] <= its[1] + max(2, its[1] // 5), its
    with pytest.raises(cmg.CascadeError, match="CS_ERR_UNSUPPORTED"):  # FP32 products would flip the ranking
        cmg.setup_cascade(hg, kind, nu=nu, alpha=3, lowp=True, setup_precision="fp32")


@pytest.mark.parametrize("name,bs,kind,alpha,nu", [("v2d_37", 2, "additive", 4, 3), ("v2d_37", 2, "multiplicative", 5, 3),
                                                  ("v2d_37", 3, "multiplicative", 5, 2),
                                                  ("c2d_66", 2, "multiplicative", 6, 3), ("v3d_17", 2, "additive", 7, 3)])
def test_block_truncation_parity(built, name, bs, kind, alpha, nu):
    """Truncation on block levels (Algorithm 2's optional step with n_b > 1):
    after every update a block's rows keep the alpha column blocks of largest
    Frobenius norm over the block (ties to the smaller block index).  Lambda
    on every level equals the oracle's to 1e-12, the truncation changed the
    cascade, and the truncated cascade solves with the oracle's iterations.
    Variable coefficients keep the ranking free of exact ties.  3x3 blocks of
    the 9-point coarse operators have exactly singular Gram matrices from the
    second step on (the centre node's row of A~ E vanishes), so there the
    minimum-norm solves of two correct FP64 setups agree to a few 1e-12
    (2.5e-12 measured) and the case is held to 1e-10."""
    import torch

    import paper_2606_12577_gb300 as cmg
    A = PROBS[name]()
    ho = oracle.Hierarchy(A, bs=bs)
    co = oracle.Cascade(ho, kind, nu=nu, alpha=alpha)
    cu = oracle.Cascade(ho, kind, nu=nu)
    hg = gu.gpu_hierarchy(A, block=bs)
    cg = cmg.setup_cascade(hg, kind, nu=nu, alpha=alpha)
    differs = False
    tol = TOL if bs == 2 else 1e-10
    for l in range(co.nlev):
        assert gu.rel_max(cmg.export_lambda(cg, l), co.lam(l)) <= tol, l
        differs |= gu.rel_max(co.lam(l), cu.lam(l)) > 1e-6
    assert differs
    b = problems.rhs(A.N, 12)
    xo, ito, hist_o, _ = oracle.solve(ho, co, b, method="gmres_right", tol=1e-10)
    x = torch.zeros(A.N, dtype=torch.float64, device="cuda")
    info = cmg.solve(hg, cg, _dev(b), x, method="gmres_right", tol=1e-10)
    assert info.converged and info.iterations == ito


@pytest.mark.parametrize("name,bs,kind,nu", [
    ("v2d_37", 2, "additive", 3), ("v2d_37", 2, "multiplicative", 2), ("v2d_37", 3, "additive", 2),
    ("v2d_37", 3, "multiplicative", 1), ("c2d_66", 2, "additive", 3), ("v3d_17", 2, "additive", 2),
    ("v3d_17", 2, "multiplicative", 1), ("p2d_33", 3, "additive", 3)])
def test_block_lambda_parity(built, name, bs, kind, nu):
    import paper_2606_12577_gb300 as cmg
    A = PROBS[name]()
    ho = oracle.Hierarchy(A, bs=bs)
    co = oracle.Cascade(ho, kind, nu=nu)
    hg = gu.gpu_hierarchy(A, block=bs)
    cg = cmg.setup_cascade(hg, kind, nu=nu)
    assert hg.nlevels == ho.nlev
    for l in range(co.nlev):
        assert cmg.query_level(hg, l)["lamsize"] == co.lamsize(l)
        assert gu.rel_max(cmg.export_lambda(cg, l), co.lam(l)) <= TOL, f"level {l}"


@pytest.mark.parametrize("name,bs,kind", [("v2d_37", 2, "additive"), ("v2d_37", 3, "multiplicative"),
                                          ("v3d_17", 2, "multiplicative"), ("c2d_66", 2, "additive")])
def test_block_smooth_and_vcycle(built, name, bs, kind):
    import paper_2606_12577_gb300 as cmg
    A = PROBS[name]()
    ho = oracle.Hierarchy(A, bs=bs)
    co = oracle.Cascade(ho, kind, nu=2)
    hg = gu.gpu_hierarchy(A, block=bs)
    cg = cmg.setup_cascade(hg, kind, nu=2)
    for l in range(min(2, co.nlev)):
        N = ho.N(l)
        b = problems.uniform(100 + l, N)
        x0 = problems.uniform(200 + l, N)
        for rev in (False, True):
            xg = _dev(x0)
            cmg.smooth(hg, cg, l, _dev(b), xg, reverse=rev)
            assert gu.rel_max(_host(xg), oracle.smooth(ho, co, l, b, x0, reverse=rev)) <= TOL, f"{l} {rev}"
    b = problems.rhs(A.N, 7)
    for order in ("RF", "FF"):
        xo = oracle.vcycle(ho, co, b, mu_pre=1, mu_post=1, rf=order == "RF")
        xg = _dev(np.zeros(A.N))
        cmg.vcycle(hg, cg, _dev(b), xg, mu_pre=1, mu_post=1, order=order)
        assert gu.rel_max(_host(xg), xo) <= TOL


@pytest.mark.parametrize("name,bs,kind,method", [("c2d_66", 2, "additive", "gmres"),
                                                 ("v3d_17", 2, "multiplicative", "stationary")])
def test_block_solve(built, name, bs, kind, method):
    import paper_2606_12577_gb300 as cmg
    A = PROBS[name]()
    ho = oracle.Hierarchy(A, bs=bs)
    co = oracle.Cascade(ho, kind, nu=3)
    b = problems.rhs(A.N, 9)
    xo, ito, _, _ = oracle.solve(ho, co, b, method=method, tol=1e-10)
    assert ito > 0
    hg = gu.gpu_hierarchy(A, block=bs)
    cg = cmg.setup_cascade(hg, kind, nu=3, lowp=True)
    xg = _dev(np.zeros(A.N))
    info = cmg.solve(hg, cg, _dev(b), xg, method=method, tol=1e-10)
    assert info.converged and info.iterations == ito
    assert gu.rel_max(_host(xg), xo) <= 1e-11
    x32 = _dev(np.zeros(A.N))
    info32 = cmg.solve(hg, cg, _dev(b), x32, method="refine" if method == "stationary" else method,
                       precision="fp32", tol=1e-10)
    assert info32.converged
    r = b - gu.stencil_matvec(A, _host(x32))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10


@pytest.mark.parametrize("name,bs,kind,m", [("c2d_66", 2, "additive", 32), ("v2d_37", 3, "additive", 5),
                                            ("v3d_17", 2, "multiplicative", 32), ("v2d_37", 1, "additive", 7),
                                            ("v3d_17", 1, "multiplicative", 3), ("v2d_37", 2, "multiplicative", 16),
                                            ("v2d_37", 2, "additive", 4), ("v3d_17", 2, "additive", 8),
                                            ("v3d_17", 2, "multiplicative", 16)])
def test_multi_rhs_block_steps(built, name, bs, kind, m):
    """A full forward and reverse cascade application built from cs_sweep_rhs
    steps (n_b x m block products) equals the oracle's smoother applied to
    every right-hand side; FP32 steps agree to FP32 accuracy."""
    import torch

    import paper_2606_12577_gb300 as cmg
    A = PROBS[name]()
    nu = 2
    ho = oracle.Hierarchy(A, bs=bs)
    co = oracle.Cascade(ho, kind, nu=nu)
    hg = gu.gpu_hierarchy(A, block=bs)
    cg = cmg.setup_cascade(hg, kind, nu=nu, lowp=True)
    N = A.N
    B = problems.uniform(31, N * m).reshape(N, m)
    X0 = problems.uniform(32, N * m).reshape(N, m)
    ncol = 2 if kind == "multiplicative" else 1
    for rev in (False, True):
        for dt, tol in ((torch.float64, TOL), (torch.float32, 2e-5)):
            bg = _dev(B, dt)
            cur, oth = _dev(X0, dt), _dev(np.zeros((N, m)), dt)
            for st in range(nu):
                lv = nu - 1 - st if rev else st
                for kk in range(ncol):
                    col = (ncol - 1 - kk if rev else kk) if ncol == 2 else -1
                    cmg.sweep_rhs(hg, cg, 0, lv, bg, cur, oth, m, colour=col, transpose=rev)
                    cur, oth = oth, cur
            got = _host(cur).astype(np.float64)
            ref = np.stack([oracle.smooth(ho, co, 0, B[:, r], X0[:, r], reverse=rev) for r in range(m)], axis=1)
            assert gu.rel_max(got, ref) <= tol, f"reverse={rev} {dt}"


@pytest.mark.parametrize("m", [32, 16, 4])
def test_multi_rhs_colour_steps_in_place(built, m):
    """On a 5-point level red-black block steps may overwrite x in place
    (block red-black is a graph colouring of the 5-point stencil): in-place
    FP32 steps give bitwise the result of out-of-place ones."""
    import torch

    import paper_2606_12577_gb300 as cmg
    A = PROBS["v2d_37"]()
    hg = gu.gpu_hierarchy(A, block=2)
    cg = cmg.setup_cascade(hg, "multiplicative", nu=2, lowp=True)
    N = A.N
    B = _dev(problems.uniform(41, N * m).reshape(N, m), torch.float32)
    X0 = problems.uniform(42, N * m).reshape(N, m)
    xin = _dev(X0, torch.float32)
    cur, oth = _dev(X0, torch.float32), _dev(np.zeros((N, m)), torch.float32)
    for st in range(2):
        for col in (0, 1):
            cmg.sweep_rhs(hg, cg, 0, st, B, xin, xin, m, colour=col)
            cmg.sweep_rhs(hg, cg, 0, st, B, cur, oth, m, colour=col)
            cur, oth = oth, cur
    assert np.array_equal(_host(xin), _host(cur))


INTERFACE_LAMBDA_TOL = 1e-9


@pytest.mark.parametrize("n,count,method,maxit", [(63, 8, "gmres", 100), (127, 60, "gmres_right", 100),
                                                  (255, 200, "gmres_right", 60)])
def test_interface_workload_parity(built, n, count, method, maxit):
    """The elliptic interface family (problems.interface2d: ~count circular
    inclusions of contrast up to 1e8, 2x2-node blocks, additive nu = 3) at
    sizes the oracle solves in seconds: Lambda blocks, the FP64 solve's
    iteration count and residual history equal the oracle's; FP32 cycles
    reach the same 1e-10 true residual.  At 255^2 the left-preconditioned
    GMRES stagnates in the oracle too (its test in the oracle pins); the
    right-preconditioned one converges on both sides."""
    import paper_2606_12577_gb300 as cmg
    A = problems.interface2d(n, count)
    ho = oracle.Hierarchy(A, bs=2)
    co = oracle.Cascade(ho, "additive", nu=3)
    hg = gu.gpu_hierarchy(A, block=2)
    cg = cmg.setup_cascade(hg, "additive", nu=3, lowp=True)
    # Lambda: from cascade step 2 on, blocks on inclusion boundaries have Gram
    # matrices with exact null spaces and kept eigenvalues down to 1e-4 of the
    # largest at 63^2 (smaller at larger sizes and contrast), so correct FP64
    # implementations agree only to kappa x u propagated through E: the oracle
    # and a dense LAPACK emulation differ by 6e-12 at 63^2
    # (test_interface_blocks_are_ill_conditioned_from_step_two).  Measured
    # GPU - oracle: 2.8e-12 (63^2), 1.8e-12 (127^2), 2.7e-10 (255^2).
    for l in range(co.nlev):
        assert gu.rel_max(cmg.export_lambda(cg, l), co.lam(l)) <= INTERFACE_LAMBDA_TOL, l
    b = problems.rhs(A.N, 9)
    xo, ito, hist_o, fin_o = oracle.solve(ho, co, b, method=method, tol=1e-10, maxit=maxit)
    assert ito > 0
    xg = _dev(np.zeros(A.N))
    info = cmg.solve(hg, cg, _dev(b), xg, method=method, tol=1e-10, maxit=maxit)
    assert info.converged and info.iterations == ito
    np.testing.assert_allclose(info.history, hist_o, rtol=1e-8, atol=1e-13)
    assert gu.rel_max(_host(xg), xo) <= 1e-9
    x32 = _dev(np.zeros(A.N))
    info32 = cmg.solve(hg, cg, _dev(b), x32, method=method, precision="fp32", tol=1e-10, maxit=2 * maxit)
    assert info32.converged
    r = b - gu.stencil_matvec(A, _host(x32))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
