"""FP32 kernels against the FP64 oracle, element by element.

The FP32 cycle (the headline form) runs the cascade step, the restricted
residual and the prolongation in FP32 storage and arithmetic.  Each test
rounds its inputs to FP32 once, gives the same values to both sides, forms
the exact result from the oracle's FP64 operator, Lambda and transfers, and
checks every node against a bound derived from the roundings the FP32 path
adds (u = 2^-24, first order in u):

* cascade step  out = x - lam (A x - b), nst stencil entries:
  A and lam are stored in FP32 (u each), the residual is a sum of nst + 1
  terms (gamma_{nst+1}), the product and the update round once each, so
  |out - ref| <= u |ref| + (nst + 5) u |lam| (|A| |x| + |b|).
  On 27-point levels with symmetric FP32 storage a backward coupling is read
  from the neighbour's row; the two differ by at most 1e-12 of the diagonal
  (the symmetry test that enables that storage), far below u.
* restricted residual rc = R (A x - b): each fine residual carries
  (nst + 3) u (|A| |x| + |b|), the gather sums 3^dim weighted terms with
  binary-exact weights, so |rc - ref| <= R [(nst + 3) u (|A||x| + |b|) +
  (3^dim + 1) u |r|].
* prolongation x - P xc: 2^dim products with binary-exact weights and one
  update, |out - ref| <= (2^dim + 2) u (|x| + P |xc|).

The grids include even-width 3D grids, where the additive step reads two
x-adjacent nodes per thread (float2), spanning several CTAs with ragged
tails, and odd-width / 2D grids, where one node per thread is used.
"""
import numpy as np
import pytest

import oracle
import problems
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    return True


def _rect3(nx, ny, nz, seed):
    from tests.test_gpu_parity import _rect
    return _rect(nx, ny, nz, seed=seed)


CASES = {
    # even nx: the paired (float2) additive kernel on the fine level
    "r3d_34x20x12": lambda: _rect3(34, 20, 12, 5),
    "v3d_64": lambda: problems.variable_poisson(problems.random_coefficients(3, 64, 41, -1.0, 1.0)),
    # odd nx and 2D: one node per thread
    "v3d_33": lambda: problems.variable_poisson(problems.random_coefficients(3, 33, 6, -1.0, 1.0)),
    "v2d_130": lambda: problems.variable_poisson(problems.random_coefficients(2, 130, 4)),
    "p2d_64": lambda: problems.poisson(2, 64),
}


def _f32(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _h(t):
    import torch
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def _rounded(seed, n):
    return problems.uniform(seed, n).astype(np.float32).astype(np.float64)


def _check(got, ref, bound, what):
    err = np.abs(got - ref)
    worst = float(np.max(err / np.maximum(bound, 1e-300)))
    assert np.all(err <= bound), f"{what}: worst error / bound = {worst:.3g}"
    return worst


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("kind", ["additive", "multiplicative"])
def test_fp32_steps_match_oracle(built, name, kind):
    """Every FP32 cascade step on the finest and the first Galerkin level
    (STAR fine level: the paired or one-node kernel; 3D BOX level with
    symmetric FP32 storage: k_sweep_sym), additive and multiplicative
    colour steps (in place on the 5/7-point level, snapshot on the 27-point
    level), element-wise within the FP32 bound."""
    import torch

    import paper_2606_12577_gb300 as cmg
    A = CASES[name]()
    ho = oracle.Hierarchy(A)
    nu = 2
    co = oracle.Cascade(ho, kind, nu=nu)
    hg = gu.gpu_hierarchy(A)
    cg = cmg.setup_cascade(hg, kind, nu=nu, lowp=True)
    for l in range(min(2, co.nlev)):
        N = ho.N(l)
        Ao = gu.oracle_csr(ho, l)
        absA = abs(Ao)
        nst = int(np.diff(Ao.indptr).max())
        col = ho.colours(l)
        lam_all = co.lam(l).reshape(nu, -1)
        for step in range(nu):
            b = _rounded(500 + 10 * l + step, N)
            x = _rounded(600 + 10 * l + step, N)
            lam = lam_all[step]
            ref_full = x - lam * (Ao @ x - b)
            bound_full = U32 * np.abs(ref_full) + (nst + 5) * U32 * np.abs(lam) * (absA @ np.abs(x) + np.abs(b))
            colours = [-1] if kind == "additive" else [0, 1]
            for c in colours:
                bg, xg = _f32(b), _f32(x)
                in_place = c >= 0 and cmg.query_level(hg, l)["nst"] in (5, 7)
                out = xg if in_place else torch.zeros_like(xg)
                cmg.sweep(hg, cg, l, step, bg, xg, out, colour=c)
                got = _h(out)
                if c >= 0:
                    keep = col != c
                    ref = np.where(keep, x, ref_full)
                    bound = np.where(keep, 0.0, bound_full)  # the other colour is copied exactly
                else:
                    ref, bound = ref_full, bound_full
                _check(got, ref, bound, f"level {l} step {step} colour {c}")


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_transfers_match_oracle(built, name):
    """The FP32 restricted residual (fine residual + gather, or the symmetric
    27-point residual on Galerkin levels) and the FP32 prolongation on the
    first two levels, element-wise within the FP32 bounds."""
    import paper_2606_12577_gb300 as cmg
    A = CASES[name]()
    ho = oracle.Hierarchy(A)
    hg = gu.gpu_hierarchy(A)
    cg = cmg.setup_cascade(hg, "additive", nu=1, lowp=True)
    d = A.dim
    for l in range(min(2, ho.nlev - 1)):
        N, Nc = ho.N(l), ho.N(l + 1)
        Ao = gu.oracle_csr(ho, l)
        nst = int(np.diff(Ao.indptr).max())
        b = _rounded(700 + l, N)
        x = _rounded(710 + l, N)
        r = ho.residual(l, b, x)  # A x - b
        ref = ho.restrict(l, r)
        fine = (nst + 3) * U32 * (abs(Ao) @ np.abs(x) + np.abs(b)) + (3 ** d + 1) * U32 * np.abs(r)
        bound = ho.restrict(l, fine)
        rc = _f32(np.zeros(Nc))
        cmg.residual_restrict_lowp(hg, cg, l, _f32(b), _f32(x), rc)
        _check(_h(rc), ref, bound, f"restriction level {l}")
        xc = _rounded(720 + l, Nc)
        ref = ho.prolong_correct(l, xc, x)
        pabs = -ho.prolong_correct(l, np.abs(xc), np.zeros(N))  # P |xc| (P >= 0)
        bound = (2 ** d + 2) * U32 * (np.abs(x) + pabs)
        xg = _f32(x)
        cmg.prolong_correct_lowp(hg, cg, l, _f32(xc), xg)
        _check(_h(xg), ref, bound, f"prolongation level {l}")


def test_fp32_bound_is_tight_enough(built):
    """The bounds above are not vacuous: on the paired-kernel case the
    observed error of a step reaches a visible fraction of the bound, and
    at a typical node a relative error of 1e-5 (about 170 u) would exceed
    it."""
    import torch

    import paper_2606_12577_gb300 as cmg
    A = CASES["r3d_34x20x12"]()
    ho = oracle.Hierarchy(A)
    co = oracle.Cascade(ho, "additive", nu=2)
    hg = gu.gpu_hierarchy(A)
    cg = cmg.setup_cascade(hg, "additive", nu=2, lowp=True)
    N = A.N
    Ao = gu.oracle_csr(ho, 0)
    b, x = _rounded(801, N), _rounded(802, N)
    lam = co.lam(0).reshape(2, -1)[1]
    ref = x - lam * (Ao @ x - b)
    bound = U32 * np.abs(ref) + 12 * U32 * np.abs(lam) * (abs(Ao) @ np.abs(x) + np.abs(b))
    out = torch.zeros(N, dtype=torch.float32, device="cuda")
    cmg.sweep(hg, cg, 0, 1, _f32(b), _f32(x), out)
    got = _h(out)
    worst = _check(got, ref, bound, "paired step")
    assert worst > 0.01
    assert np.median(bound / np.maximum(np.abs(ref), 1e-300)) < 1e-5
