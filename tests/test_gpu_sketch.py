"""Sketched cascade setup (the reformulation of the paper's concluding
remarks, Sec. 4) on the GPU against the FP64 oracle's sketched setup with the
same Rademacher sketch (each side generates it from the published
SplitMix64 definition): Lambda within 1e-12 in FP64, within a derived bound
with FP32 sketch vectors; the V-cycle with a sketched cascade solves to
1e-10 in the oracle's iteration count."""
import numpy as np
import pytest

import oracle
import problems
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    return True


def _var(dim, n, seed, lo=-1.0, hi=1.0):
    return problems.variable_poisson(problems.random_coefficients(dim, n, seed, lo, hi))


PROBS = {
    "p2d_64": lambda: problems.poisson(2, 64),
    "v2d_37": lambda: _var(2, 37, 3),
    "v3d_17": lambda: _var(3, 17, 5),
    "c3d_33": lambda: problems.variable_poisson(problems.log_uniform_field(3, 33, 4.0, 333, -2.0, 2.0)),
}


@pytest.mark.parametrize("name,kind,s,exact_first", [
    ("p2d_64", "additive", 8, False), ("p2d_64", "multiplicative", 32, False), ("v2d_37", "additive", 64, True),
    ("v2d_37", "multiplicative", 100, True), ("v3d_17", "additive", 32, False), ("v3d_17", "multiplicative", 16, True),
    ("c3d_33", "multiplicative", 32, False), ("c3d_33", "additive", 4, False)])
def test_sketched_lambda_matches_oracle(built, name, kind, s, exact_first):
    """FP64 sketched setup on every smoothing level (7/5-point fine levels,
    27/9-point Galerkin levels; 1..4 sketch entries per lane) equals the
    oracle's to 1e-12.  (A sketch needs more columns than a block has nodes:
    with s = 1 a point's first step leaves Y = 0 in exact arithmetic and
    every later lambda is a ratio of rounding errors.)"""
    import paper_2606_12577_gb300 as cmg
    A = PROBS[name]()
    ho = oracle.Hierarchy(A)
    seed = 0x1234567890ABCDEF
    co = oracle.Cascade(ho, kind, nu=3, sketch=s, seed=seed, exact_first=exact_first)
    hg = gu.gpu_hierarchy(A)
    cg = cmg.setup_cascade(hg, kind, nu=3, sketch=s, sketch_seed=seed, sketch_exact_first=exact_first)
    for l in range(co.nlev):
        assert gu.rel_max(cmg.export_lambda(cg, l), co.lam(l)) <= TOL, l
    if exact_first:  # the first step is the exact one
        ce = oracle.Cascade(ho, kind, nu=1)
        lam1 = co.lam(0)[0]
        ex = ce.lam(0)[0]
        if kind == "multiplicative":  # only the first colour's step is unsketched
            red = ho.colours(0) == 0
            lam1, ex = lam1[red], ex[red]
        assert gu.rel_max(lam1, ex) <= 1e-13


# FP32 sketch vectors: a Z entry sums nst + 1 FP32 products (relative error
# about (nst + 1) u of sum |a| |y|), <Y, Z> and <Z, Z> carry a few u of their
# magnitudes, and Y inherits the rounding of every earlier step, so lambda
# agrees with the FP64 sketch to ~10 (nst + 1) nu u <= 2e-4 on 27-point
# levels; measured well below.
FP32_TOL = 2e-4


@pytest.mark.parametrize("name,kind", [("p2d_64", "additive"), ("v3d_17", "multiplicative"), ("c3d_33", "additive")])
def test_fp32_sketch_matches_oracle(built, name, kind):
    import paper_2606_12577_gb300 as cmg
    A = PROBS[name]()
    ho = oracle.Hierarchy(A)
    co = oracle.Cascade(ho, kind, nu=3, sketch=32, seed=77)
    hg = gu.gpu_hierarchy(A)
    cg = cmg.setup_cascade(hg, kind, nu=3, sketch=32, sketch_seed=77, setup_precision="fp32")
    for l in range(co.nlev):
        err = gu.rel_max(cmg.export_lambda(cg, l), co.lam(l))
        assert err <= FP32_TOL, (l, err)
        assert err > 0.0 or ho.N(l) <= 16


@pytest.mark.parametrize("name,kind,method", [("p2d_64", "additive", "stationary"),
                                              ("c3d_33", "multiplicative", "gmres_right"),
                                              ("v3d_17", "additive", "gmres")])
def test_sketched_cascade_solves_like_the_oracle(built, name, kind, method):
    """Solves with the sketched cascade (s = 32): the FP64 solve takes the
    oracle's iteration count with the oracle's residual history, and FP32
    cycles in FP64 refinement reach the same 1e-10 true residual."""
    import torch

    import paper_2606_12577_gb300 as cmg
    A = PROBS[name]()
    ho = oracle.Hierarchy(A)
    co = oracle.Cascade(ho, kind, nu=3, sketch=32, seed=5)
    b = problems.rhs(A.N, 21)
    xo, ito, hist_o, _ = oracle.solve(ho, co, b, method=method, tol=1e-10)
    assert ito > 0
    hg = gu.gpu_hierarchy(A)
    cg = cmg.setup_cascade(hg, kind, nu=3, sketch=32, sketch_seed=5, lowp=True)
    x = torch.zeros(A.N, dtype=torch.float64, device="cuda")
    info = cmg.solve(hg, cg, torch.tensor(b, device="cuda"), x, method=method, tol=1e-10)
    assert info.converged and info.iterations == ito
    np.testing.assert_allclose(info.history, hist_o, rtol=1e-9, atol=1e-13)
    x32 = torch.zeros(A.N, dtype=torch.float64, device="cuda")
    info32 = cmg.solve(hg, cg, torch.tensor(b, device="cuda"), x32,
                       method="refine" if method == "stationary" else method, precision="fp32", tol=1e-10)
    assert info32.converged
    r = b - gu.stencil_matvec(A, x32.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10


def test_sketch_options_are_validated(built):
    import paper_2606_12577_gb300 as cmg
    A = PROBS["v2d_37"]()
    hg = gu.gpu_hierarchy(A)
    with pytest.raises(cmg.CascadeError, match="CS_ERR_ARG"):
        cmg.setup_cascade(hg, "additive", nu=2, sketch=129)
    with pytest.raises(cmg.CascadeError, match="sketched setup"):
        cmg.setup_cascade(hg, "additive", nu=2, sketch=8, alpha=3)
    hb = gu.gpu_hierarchy(A, block=2)
    with pytest.raises(cmg.CascadeError, match="sketched setup"):
        cmg.setup_cascade(hb, "additive", nu=2, sketch=8)
