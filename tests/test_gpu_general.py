"""The general sparse path (CSR operator, user transfers and blocks, greedy
colouring) against the oracle's CSR hierarchy on a jittered Q1 mesh whose
unknowns are renumbered at random (nothing structured survives): Galerkin
operators to 1e-14, colour ids bit-exact, Lambda, cascade steps, V-cycles
and solves to 1e-12 / the oracle's iteration counts."""
import numpy as np
import pytest

import oracle
import problems
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu
TOL = 1e-12
OVERLAP_MULT_TOL = 1e-8


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    return True


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


MESHES = {"q1_31": (31, 3), "q1_63": (63, 4), "q1_40": (40, 6)}


def _pair(name, blocks=False, seed=11):
    import paper_2606_12577_gb300 as cmg
    n, s = MESHES[name]
    u = problems.unstructured_q1(n, s)
    bl = u["blocks"] if blocks else None
    ho = oracle.Hierarchy.from_csr(u["A"], u["Ps"], rscale=0.25, blocks=bl, seed=seed)
    hg = cmg.gsetup_hierarchy(u["A"], u["Ps"], rscale=0.25, blocks=bl, seed=seed)
    return u, ho, hg


@pytest.mark.parametrize("name", list(MESHES))
def test_general_hierarchy_matches_oracle(built, name):
    u, ho, hg = _pair(name)
    assert hg.nlevels == ho.nlev
    for l in range(ho.nlev):
        rp, ci, v = hg.operator(l)
        orp, oci, ov = ho.csr(l)
        assert np.array_equal(rp, orp) and np.array_equal(ci, oci), l
        assert np.abs(v - ov).max() <= 1e-14 * np.abs(ov).max(), l
        assert np.array_equal(hg.colours(l), ho.blocks(l)[2]), l  # bit-exact colour ids
        assert hg.level(l)["ncolours"] == ho.ncolours(l)
    assert ho.ncolours(0) > 2


@pytest.mark.parametrize("name,kind,nu,blocks", [("q1_31", "additive", 3, False), ("q1_31", "multiplicative", 2, False),
                                                 ("q1_63", "multiplicative", 3, False), ("q1_40", "additive", 3, True),
                                                 ("q1_31", "multiplicative", 2, True)])
def test_general_lambda_matches_oracle(built, name, kind, nu, blocks):
    import paper_2606_12577_gb300 as cmg
    u, ho, hg = _pair(name, blocks)
    co = oracle.Cascade(ho, kind, nu=nu)
    cg = cmg.gsetup_cascade(hg, kind, nu=nu)
    for l in range(co.nlev):
        assert gu.rel_max(cmg.gexport_lambda(cg, l), co.lam(l)) <= TOL, l


@pytest.mark.parametrize("name,kind,blocks", [("q1_31", "additive", False), ("q1_63", "multiplicative", False),
                                              ("q1_40", "additive", True), ("q1_31", "multiplicative", True)])
def test_general_steps_and_cycles_match_oracle(built, name, kind, blocks):
    """One cascade application forward and reverse on the first two levels
    (one-thread-per-row kernel on point levels, warp-per-block kernel on the
    3x3-node blocks, colour steps in place), and two V-cycles in RF and FF
    order."""
    import paper_2606_12577_gb300 as cmg
    u, ho, hg = _pair(name, blocks)
    co = oracle.Cascade(ho, kind, nu=2)
    cg = cmg.gsetup_cascade(hg, kind, nu=2)
    for l in range(min(2, co.nlev)):
        N = ho.N(l)
        b = problems.uniform(100 + l, N)
        x0 = problems.uniform(200 + l, N)
        for rev in (False, True):
            xg = _dev(x0)
            cmg.gsmooth(hg, cg, l, _dev(b), xg, reverse=rev)
            assert gu.rel_max(_host(xg), oracle.smooth(ho, co, l, b, x0, reverse=rev)) <= TOL, (l, rev)
    b = problems.rhs(ho.N(0), 7)
    for order in ("RF", "FF"):
        xo = oracle.vcycle(ho, co, b, rf=order == "RF")
        xo = oracle.vcycle(ho, co, b, xo, rf=order == "RF")
        xg = _dev(np.zeros(ho.N(0)))
        for _ in range(2):
            cmg.gvcycle(hg, cg, _dev(b), xg, order=order)
        assert gu.rel_max(_host(xg), xo) <= TOL, order


@pytest.mark.parametrize("name,kind,method,blocks", [("q1_63", "additive", "gmres_right", False),
                                                     ("q1_63", "multiplicative", "stationary", False),
                                                     ("q1_40", "additive", "gmres_right", True),
                                                     ("q1_31", "multiplicative", "gmres_right", True)])
def test_general_solve_matches_oracle(built, name, kind, method, blocks):
    import paper_2606_12577_gb300 as cmg
    u, ho, hg = _pair(name, blocks)
    co = oracle.Cascade(ho, kind, nu=3)
    cg = cmg.gsetup_cascade(hg, kind, nu=3)
    b = problems.rhs(ho.N(0), 9)
    xo, ito, hist_o, _ = oracle.solve(ho, co, b, method=method, tol=1e-10)
    assert ito > 0
    x = _dev(np.zeros(ho.N(0)))
    info = cmg.gsolve(hg, cg, _dev(b), x, method=method, tol=1e-10)
    assert info.converged and info.iterations == ito
    np.testing.assert_allclose(info.history, hist_o, rtol=1e-9, atol=1e-13)
    r = b - u["A"] @ _host(x)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    assert gu.rel_max(_host(x), xo) <= 1e-11


def test_general_path_reduces_to_the_structured_path(built):
    """A structured operator given as CSR with the bilinear transfers: the
    general path's additive Lambda equals the structured path's, and the
    solves take the same iterations."""
    import scipy.sparse as sp
    import torch

    import paper_2606_12577_gb300 as cmg
    A = problems.variable_poisson(problems.random_coefficients(2, 47, 3))
    Ps, n = [], 47
    while n > 4:
        P1 = sp.csr_matrix(problems.interpolation_1d(n))
        Ps.append(sp.kron(P1, P1, format="csr"))
        n //= 2
    hg = cmg.gsetup_hierarchy(problems.stencil_csr(A), Ps, rscale=0.25)
    cg = cmg.gsetup_cascade(hg, "additive", nu=3)
    hs = gu.gpu_hierarchy(A)
    cs = cmg.setup_cascade(hs, "additive", nu=3)
    assert hg.nlevels == hs.nlevels
    for l in range(hs.nlevels - 1):
        assert gu.rel_max(cmg.gexport_lambda(cg, l), cmg.export_lambda(cs, l)) <= TOL, l
    b = problems.rhs(A.N, 5)
    x1 = torch.zeros(A.N, dtype=torch.float64, device="cuda")
    x2 = torch.zeros(A.N, dtype=torch.float64, device="cuda")
    i1 = cmg.gsolve(hg, cg, _dev(b), x1, method="gmres_right")
    i2 = cmg.solve(hs, cs, _dev(b), x2, method="gmres_right")
    assert i1.iterations == i2.iterations
    assert gu.rel_max(_host(x1), _host(x2)) <= 1e-10


def test_general_path_rejects_bad_input(built):
    import scipy.sparse as sp

    import paper_2606_12577_gb300 as cmg
    u = problems.unstructured_q1(15, 2)
    bptr, bidx = u["blocks"]
    bad = bidx.copy()
    bad[0] = bad[1]  # a node twice in block 0 (and the node it replaced in no block)
    with pytest.raises(cmg.CascadeError, match="CS_ERR_ARG"):
        cmg.gsetup_hierarchy(u["A"], u["Ps"], rscale=0.25, blocks=(bptr, bad))
    with pytest.raises(cmg.CascadeError, match="CS_ERR_ARG"):
        cmg.gsetup_hierarchy(u["A"], [sp.csr_matrix(np.ones((3, 2)))], rscale=0.25)  # wrong shape


def _stokes_pair(n, seed=3):
    import paper_2606_12577_gb300 as cmg
    u = problems.mac_stokes_2d(n)
    ho = oracle.Hierarchy.from_csr(u["A"], u["Ps"], rscale=0.25, blocks=u["blocks"], fields=u["fields"], seed=seed)
    hg = cmg.gsetup_hierarchy(u["A"], u["Ps"], rscale=0.25, blocks=u["blocks"], fields=u["fields"], seed=seed)
    return u, ho, hg


@pytest.mark.parametrize("n,kind,mode", [(16, "additive", "stokes1"), (32, "multiplicative", "stokes1"),
                                         (32, "additive", "stokesinf"), (16, "multiplicative", "stokes2")])
def test_stokes_prescaled_cascade_matches_oracle(built, n, kind, mode):
    """The MAC Stokes operator with (d+1)-DOF cell blocks on every level and
    Stokes prescaling (SM "Prescaling Stokes problems"): Galerkin levels,
    colours, Lambda and the right-GMRES solve equal the oracle's."""
    import paper_2606_12577_gb300 as cmg
    u, ho, hg = _stokes_pair(n)
    for l in range(ho.nlev):
        rp, ci, v = hg.operator(l)
        orp, oci, ov = ho.csr(l)
        assert np.array_equal(ci, oci) and np.abs(v - ov).max() <= 1e-14 * np.abs(ov).max(), l
        assert np.array_equal(hg.colours(l), ho.blocks(l)[2]), l
    co = oracle.Cascade(ho, kind, nu=3, prescale=mode)
    cg = cmg.gsetup_cascade(hg, kind, nu=3, prescale=mode)
    for l in range(co.nlev):
        assert gu.rel_max(cmg.gexport_lambda(cg, l), co.lam(l)) <= TOL, l
    b = problems.rhs(u["A"].shape[0], 11)
    xo, ito, hist_o, _ = oracle.solve(ho, co, b, method="gmres_right", tol=1e-10, maxit=200)
    assert ito > 0
    x = _dev(np.zeros(len(b)))
    info = cmg.gsolve(hg, cg, _dev(b), x, method="gmres_right", tol=1e-10, maxit=200)
    assert info.converged and info.iterations == ito
    np.testing.assert_allclose(info.history, hist_o, rtol=1e-8, atol=1e-13)
    r = b - u["A"] @ _host(x)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10


def test_stokes_prescaling_needs_fields_and_rejects_elliptic(built):
    import paper_2606_12577_gb300 as cmg
    u, ho, hg = _stokes_pair(16)
    with pytest.raises(cmg.CascadeError, match="CS_ERR_ARG"):
        cmg.gsetup_cascade(hg, "additive", nu=2, prescale="elliptic")  # the pressure diagonal is negative
    hn = cmg.gsetup_hierarchy(u["A"], u["Ps"], rscale=0.25, blocks=u["blocks"])
    with pytest.raises(cmg.CascadeError, match="fields"):
        cmg.gsetup_cascade(hn, "additive", nu=2, prescale="stokes1")


def _cells_pair(n, seed=3):
    """The jittered Q1 mesh with the nodes of every element as a block on
    level 0: an interior node lies in 4 blocks (Sec. 3.6.2)."""
    import paper_2606_12577_gb300 as cmg
    u = problems.unstructured_q1(n, seed)
    ho = oracle.Hierarchy.from_csr(u["A"], u["Ps"], rscale=0.25, blocks=u["cells"], seed=seed)
    hg = cmg.gsetup_hierarchy(u["A"], u["Ps"], rscale=0.25, blocks=u["cells"], seed=seed)
    return u, ho, hg


@pytest.mark.parametrize("n,kind,nu", [(31, "additive", 2), (31, "multiplicative", 2), (40, "additive", 3)])
def test_overlapping_blocks_match_oracle(built, n, kind, nu):
    """Overlapping element blocks: colours (blocks sharing a node separated)
    bit-exact, Lambda of the averaged additive form and of the overwriting
    multiplicative form, one smoother application forward and reverse (the
    additive one through the block corrections and the theta-averaging
    kernels), two V-cycles and the right-GMRES solve."""
    import paper_2606_12577_gb300 as cmg
    u, ho, hg = _cells_pair(n)
    assert ho.overlapping(0)
    bp, bi = hg.blocks(0)
    obp, obi, ocol = ho.blocks(0)
    assert np.array_equal(bp, obp) and np.array_equal(bi, obi)
    assert np.array_equal(hg.colours(0), ocol) and hg.level(0)["ncolours"] == ho.ncolours(0)
    co = oracle.Cascade(ho, kind, nu=nu)
    cg = cmg.gsetup_cascade(hg, kind, nu=nu)
    # multiplicative: a cell whose nodes earlier colours have overwritten has
    # a nearly singular Gram matrix; the oracle's own Lambda moves by up to
    # 2e-9 under 1e-15 relative perturbations of A there (pinned on the CPU
    # by test_overlapping_multiplicative_blocks_are_ill_conditioned)
    tol = TOL if kind == "additive" else OVERLAP_MULT_TOL
    for l in range(co.nlev):
        assert gu.rel_max(cmg.gexport_lambda(cg, l), co.lam(l)) <= tol, l
    N = ho.N(0)
    b = problems.uniform(31, N)
    x0 = problems.uniform(32, N)
    for rev in (False, True):
        xg = _dev(x0)
        cmg.gsmooth(hg, cg, 0, _dev(b), xg, reverse=rev)
        assert gu.rel_max(_host(xg), oracle.smooth(ho, co, 0, b, x0, reverse=rev)) <= tol, rev
    b = problems.rhs(N, 7)
    for order in ("RF", "FF"):
        xo = oracle.vcycle(ho, co, b, rf=order == "RF")
        xo = oracle.vcycle(ho, co, b, xo, rf=order == "RF")
        xg = _dev(np.zeros(N))
        for _ in range(2):
            cmg.gvcycle(hg, cg, _dev(b), xg, order=order)
        assert gu.rel_max(_host(xg), xo) <= tol, order
    xo, ito, hist_o, _ = oracle.solve(ho, co, b, method="gmres_right", tol=1e-10)
    assert ito > 0
    x = _dev(np.zeros(N))
    info = cmg.gsolve(hg, cg, _dev(b), x, method="gmres_right", tol=1e-10)
    assert info.converged and info.iterations == ito
    np.testing.assert_allclose(info.history, hist_o, rtol=1e-9 if kind == "additive" else 1e-6, atol=1e-13)


@pytest.mark.parametrize("blocks", ["points", "blocks", "cells"])
def test_spd_cascade_and_pcg_match_oracle(built, blocks):
    """The SPD-projected additive cascade (each Lambda~ block moved between
    0 and the block-Jacobi block before the next step uses it) and PCG with
    the RF V-cycle: Lambda to 1e-10 (the projection goes through two
    Jacobi eigendecompositions per block), the PCG iteration count equal,
    its recurrence history to 1e-8 and the true residual below tol."""
    import paper_2606_12577_gb300 as cmg
    u = problems.unstructured_q1(31, 3)
    bl = {"points": None, "blocks": u["blocks"], "cells": u["cells"]}[blocks]
    ho = oracle.Hierarchy.from_csr(u["A"], u["Ps"], rscale=0.25, blocks=bl, seed=3)
    hg = cmg.gsetup_hierarchy(u["A"], u["Ps"], rscale=0.25, blocks=bl, seed=3)
    co = oracle.Cascade(ho, "additive", nu=3, spd=True)
    cg = cmg.gsetup_cascade(hg, "additive", nu=3, spd=True)
    for l in range(co.nlev):
        assert gu.rel_max(cmg.gexport_lambda(cg, l), co.lam(l)) <= 1e-10, l
    b = problems.rhs(ho.N(0), 8)
    xo, ito, hist_o, fin_o = oracle.solve(ho, co, b, method="pcg", tol=1e-10, maxit=100)
    assert ito > 0 and fin_o <= 1e-10
    x = _dev(np.zeros(ho.N(0)))
    info = cmg.gsolve(hg, cg, _dev(b), x, method="pcg", tol=1e-10, maxit=100)
    assert info.converged and info.iterations == ito
    np.testing.assert_allclose(info.history, hist_o, rtol=1e-8, atol=1e-13)
    r = b - u["A"] @ _host(x)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    assert gu.rel_max(_host(x), xo) <= 1e-9
