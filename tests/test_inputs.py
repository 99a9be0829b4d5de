"""The synthetic inputs against their stated recipe (CPU).

The seeded generators feed both the oracle and the CUDA path; these tests
pin them to their definitions: the SplitMix64 stream to the generator's
reference outputs, the FD Poisson stencils to their closed form, and the
workload generators to the distributions they draw from (sizes, right-hand
side counts, coefficient ranges, symmetry and diagonal dominance of the
operators)."""
from __future__ import annotations

import numpy as np
import pytest

import problems


def test_splitmix64_reference_outputs():
    # SplitMix64 (Steele, Lea and Flood 2014) from state 0: the first outputs
    # of the reference implementation (Vigna's splitmix64.c)
    got = [int(v) for v in problems.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # draws are addressable: a window starting at draw 1 is the tail of the stream
    assert np.array_equal(problems.splitmix64(5, 4, start=1), problems.splitmix64(5, 5)[1:])


def test_uniform_streams():
    u = problems.uniform01(7, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1.0 / 12.0) < 0.002
    v = problems.uniform(7, 1000, -1.0, 1.0)
    assert np.array_equal(v, -1.0 + 2.0 * u[:1000])
    g = problems.normal(3, 200_000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 5)])
def test_poisson_stencil_closed_form(dim, n):
    """Diagonal 2d/h^2 and off-diagonals -1/h^2 with h = 1/(n+1); couplings to
    the Dirichlet boundary are zero, so a row's sum is (number of boundary
    neighbours)/h^2 and the interior rows sum to 0."""
    A = problems.poisson(dim, n)
    h2 = (n + 1.0) ** 2
    assert A.offsets[0] == (0, 0, 0)
    assert np.allclose(A.coeff[0], 2 * dim * h2, rtol=1e-14, atol=0.0)
    off = np.unique(A.coeff[1:])
    assert len(off) == 2 and off[1] == 0.0 and np.isclose(off[0], -h2, rtol=1e-14, atol=0.0)
    rows = A.coeff.sum(axis=0).reshape((n,) * dim)
    inner = (slice(1, -1),) * dim
    assert np.all(np.abs(rows[inner]) <= 1e-12 * h2)
    assert np.isclose(rows.reshape(-1)[0], dim * h2, rtol=1e-14)  # a corner: one boundary neighbour per axis


def _dense(A):
    from tests.gpu_util import stencil_to_csr
    return stencil_to_csr(A.n, A.offsets, A.coeff, A.periodic).toarray()


def test_variable_poisson_is_a_symmetric_m_matrix():
    mu = problems.random_coefficients(2, 9, 11, -2.0, 2.0)
    A = _dense(problems.variable_poisson(mu))
    assert np.allclose(A, A.T, rtol=1e-14, atol=0.0)
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0.0)
    # weakly diagonally dominant rows: equality in the interior (up to rounding)
    assert np.all(np.diag(A) >= -off.sum(axis=1) * (1 - 1e-14))
    assert np.linalg.eigvalsh(A).min() > 0.0


@pytest.mark.parametrize("k", [0, 1, 5])
def test_batch_problem_recipe(k):
    """Side in 33..513 (shrunk here to 20..40 to stay small), 1..8 RHS,
    coefficients with a log-uniform marginal on [1e-3, 1e3], right-hand
    sides in [-1, 1], independent of the other problems and reproducible."""
    A, m, b = problems.batch_problem(k, nmin=20, nmax=40)
    n = A.n[0]
    assert A.n == (n, n, 1) and 20 <= n <= 40 and 1 <= m <= 8
    assert b.shape == (n * n * m,) and b.min() >= -1.0 and b.max() <= 1.0
    A2, m2, b2 = problems.batch_problem(k, nmin=20, nmax=40)
    assert m2 == m and np.array_equal(A2.coeff, A.coeff) and np.array_equal(b2, b)
    mu = problems.log_uniform_field(2, n, 8.0, problems.config_seed(4, k) + 1_000_000)
    assert mu.min() >= 1e-3 * (1 - 1e-12) and mu.max() <= 1e3 * (1 + 1e-12)
    assert mu.max() / mu.min() > 10.0  # the field does vary
    D = _dense(A)
    assert np.allclose(D, D.T, rtol=1e-13, atol=0.0)


def test_batch_sizes_cover_the_range():
    """The first problems of the full batched workload: sides drawn from
    33..513 and 1..8 right-hand sides each."""
    sides, ms = [], []
    for k in range(24):
        A, m, b = problems.batch_problem(k)
        sides.append(A.n[0])
        ms.append(m)
        assert b.shape == (A.N * m,)
    assert min(sides) >= 33 and max(sides) <= 513 and max(sides) - min(sides) > 200
    assert min(ms) >= 1 and max(ms) <= 8 and len(set(ms)) >= 5


def test_inclusion_field_recipe():
    """Background 1 and inclusions with coefficients 10^U[-4, 4]: every cell is
    1 or an inclusion value, at most `count` distinct inclusion values."""
    mu = problems.inclusions_2d(127, 20, 5, rmin=2.0, rmax=16.0)
    vals = np.unique(mu)
    inc = vals[vals != 1.0]
    assert 0 < len(inc) <= 20
    assert inc.min() >= 1e-4 and inc.max() <= 1e4
    assert 0.0 < np.mean(mu != 1.0) < 1.0


def test_rhs_layout():
    b = problems.rhs(10, 3, nrhs=4)
    assert b.shape == (10, 4)
    assert np.array_equal(b.reshape(-1), problems.uniform(3, 40, -1.0, 1.0))  # RHS contiguous per node
