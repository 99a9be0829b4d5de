"""Seeded synthetic problem generators shared by the oracle and the CUDA path.

This module only builds inputs: structured-grid operators ``A`` in stencil
form (the discretisation the method is applied to, Sec. 2 "block-partitioned
Ax = b" and Sec. 3.3.1 "finite difference Poisson") and right-hand sides.  It
holds none of the cascading-smoother arithmetic (no setup, no smoothing, no
transfers): the oracle under ``oracle/`` and the CUDA library each implement
that on their own.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw k of stream ``seed`` is ``mix(seed*G + (k+1)*G)`` with
``G = 0x9E3779B97F4A7C15``; the top 53 bits give a uniform double in [0, 1).

Layout of a structured operator (``Stencil``):
  * unknowns are the interior nodes of a ``nx x ny x nz`` grid (``nz = 1`` in
    2D), numbered ``i = ix + nx*(iy + ny*iz)`` (x fastest);
  * ``offsets[s] = (dx, dy, dz)`` with entries in {-1, 0, 1};
  * ``coeff[s, i]`` couples unknown ``i`` to the node at ``i + offsets[s]``;
    it is zero where that node is a (homogeneous) Dirichlet boundary node,
    so boundary nodes are eliminated and are not unknowns;
  * with ``periodic=True`` neighbours wrap around instead (used only to pin
    the setup against the constant-coefficient values of Table 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Return ``count`` SplitMix64 outputs (uint64) of stream ``seed``,
    beginning at draw ``start``."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed) * _G + k * _G
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0, start: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, count, start)


@dataclass
class Stencil:
    """A structured-grid operator in stencil (SoA) form; see module doc."""

    dim: int
    n: Tuple[int, int, int]
    offsets: List[Tuple[int, int, int]]
    coeff: np.ndarray  # float64 [nst, N]
    periodic: bool = False
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def nst(self) -> int:
        return len(self.offsets)

    def offsets_array(self) -> np.ndarray:
        return np.asarray(self.offsets, dtype=np.int32).reshape(-1, 3)


def _grid_coords(n):
    nx, ny, nz = n
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ix.ravel(), iy.ravel(), iz.ravel()


def _inside(n, ix, iy, iz, off):
    jx, jy, jz = ix + off[0], iy + off[1], iz + off[2]
    return (jx >= 0) & (jx < n[0]) & (jy >= 0) & (jy < n[1]) & (jz >= 0) & (jz < n[2])


def _star_offsets(dim):
    offs = [(0, 0, 0)]
    for d in range(dim):
        for sgn in (-1, 1):
            o = [0, 0, 0]
            o[d] = sgn
            offs.append(tuple(o))
    return offs


def poisson(dim: int, n: int, periodic: bool = False, h: float | None = None) -> Stencil:
    """Second-order FD negative Laplacian on an ``n^dim`` interior-node grid
    (5-point in 2D, 7-point in 3D, diagonal ``2d/h^2``; Sec. 3.3.1).

    Dirichlet: ``h = 1/(n+1)`` and couplings to boundary nodes are zero.
    Periodic: ``h = 1/n`` and every row carries the full stencil."""
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    shape = (n, n, n if dim == 3 else 1)
    if h is None:
        h = 1.0 / n if periodic else 1.0 / (n + 1)
    offs = _star_offsets(dim)
    N = shape[0] * shape[1] * shape[2]
    coeff = np.zeros((len(offs), N), dtype=np.float64)
    ix, iy, iz = _grid_coords(shape)
    inv_h2 = 1.0 / (h * h)
    for s, o in enumerate(offs):
        if o == (0, 0, 0):
            coeff[s] = 2 * dim * inv_h2
        else:
            coeff[s] = -inv_h2 if periodic else np.where(_inside(shape, ix, iy, iz, o), -inv_h2, 0.0)
    return Stencil(dim, shape, offs, coeff, periodic, name=f"poisson{dim}d_{n}")


def variable_poisson(mu_cells: np.ndarray, h: float | None = None) -> Stencil:
    """Cell-coefficient FD/FV operator ``-div(mu grad u)`` on interior nodes
    (5-point in 2D, 7-point in 3D), homogeneous Dirichlet.

    ``mu_cells`` has shape ``(n+1,)*dim`` (cells between nodes, C order
    ``[cz,] cy, cx``).  The coefficient of the edge joining two nodes is the
    arithmetic mean of the ``2^(dim-1)`` cells sharing that edge."""
    dim = mu_cells.ndim
    n1 = mu_cells.shape[-1]
    n = n1 - 1
    if h is None:
        h = 1.0 / n1
    inv_h2 = 1.0 / (h * h)
    shape = (n, n, n if dim == 3 else 1)
    offs = _star_offsets(dim)
    N = shape[0] * shape[1] * shape[2]
    ix, iy, iz = _grid_coords(shape)
    # node (ix,iy[,iz]) in 0-based interior numbering sits at 1-based node
    # index ix+1; cell c lies between nodes c and c+1 (1-based node indices).
    mu = mu_cells if dim == 3 else mu_cells[None, :, :]

    def edge(axis, sgn):
        # coefficient of the edge from node p to node p + sgn*e_axis
        X, Y, Z = ix + 1, iy + 1, iz + 1  # 1-based node coordinates
        lo = [X, Y, Z]
        lo = [a.copy() for a in lo]
        lo[axis] = lo[axis] + (0 if sgn > 0 else -1)  # cell index along axis
        others = [a for a in range(dim) if a != axis]
        tot = np.zeros(N)
        cnt = 0
        for a in (-1, 0):
            for b in ((-1, 0) if dim == 3 else (0,)):
                c = [lo[0].copy(), lo[1].copy(), lo[2].copy()]
                c[others[0]] = c[others[0]] + a
                if dim == 3:
                    c[others[1]] = c[others[1]] + b
                if dim == 2:
                    tot += mu[0, c[1], c[0]]
                else:
                    tot += mu[c[2], c[1], c[0]]
                cnt += 1
        return tot / cnt

    coeff = np.zeros((len(offs), N), dtype=np.float64)
    diag = np.zeros(N)
    for s, o in enumerate(offs):
        if o == (0, 0, 0):
            continue
        axis = int(np.nonzero(o)[0][0])
        sgn = o[axis]
        w = edge(axis, sgn) * inv_h2
        diag += w
        coeff[s] = np.where(_inside(shape, ix, iy, iz, o), -w, 0.0)
    coeff[0] = diag
    return Stencil(dim, shape, offs, coeff, False, name=f"varpoisson{dim}d_{n}")


def random_coefficients(dim: int, n: int, seed: int, lo: float = -2.0, hi: float = 2.0) -> np.ndarray:
    """i.i.d. log-uniform cell coefficients ``10^U[lo,hi]`` on ``(n+1)^dim``
    cells (a small variable-coefficient test case)."""
    shape = (n + 1,) * dim
    u = uniform(seed, int(np.prod(shape)), lo, hi)
    return (10.0 ** u).reshape(shape)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform of two uniform
    streams (draws [0, count) and [count, 2 count) of stream ``seed``)."""
    u1 = 1.0 - uniform01(seed, count, 0)  # (0, 1]
    u2 = uniform01(seed, count, count)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def gaussian_field(shape, corr: float, seed: int) -> np.ndarray:
    """Zero-mean, unit-variance stationary Gaussian random field on a grid of
    ``shape`` cells with Gaussian covariance exp(-r^2 / (2 corr^2)) (corr in
    cells), by spectral synthesis: white noise on a periodic grid padded by
    3 corr per side, filtered with the square root of the spectral density
    exp(-corr^2 |k|^2 / 2), cropped and normalised."""
    pad = int(np.ceil(3 * corr))
    big = tuple(int(n) + 2 * pad for n in shape)
    w = normal(seed, int(np.prod(big))).reshape(big)
    ks = np.meshgrid(*[2.0 * np.pi * np.fft.fftfreq(n) for n in big], indexing="ij")
    k2 = sum(k * k for k in ks)
    f = np.real(np.fft.ifftn(np.fft.fftn(w) * np.exp(-0.25 * corr * corr * k2)))
    f = f[tuple(slice(pad, pad + int(n)) for n in shape)]
    return (f - f.mean()) / f.std()


def log_uniform_field(dim: int, n: int, corr: float, seed: int, lo: float = -3.0, hi: float = 3.0) -> np.ndarray:
    """Cell coefficients with a log-uniform marginal on [10^lo, 10^hi] and
    spatial correlation: a Gaussian field mapped through the normal CDF to
    u in [0, 1], mu = 10^(lo + (hi - lo) u).  Shape ``(n+1,)*dim``."""
    from scipy.special import ndtr
    g = gaussian_field((n + 1,) * dim, corr, seed)
    return 10.0 ** (lo + (hi - lo) * ndtr(g))


def inclusions_2d(n: int, count: int, seed: int, rmin: float = 8.0, rmax: float = 64.0,
                  lo: float = -4.0, hi: float = 4.0) -> np.ndarray:
    """Piecewise-constant cell coefficients on ``(n+1)^2`` cells: background 1
    and ``count`` circular inclusions with centres ~ U(0,1)^2, radii ~
    U[rmin, rmax] cells and mu = 10^U[lo, hi]; a cell belongs to an inclusion
    when its centre does, later inclusions overwrite earlier ones (the
    elliptic interface workload)."""
    n1 = n + 1
    h = 1.0 / n1
    u = uniform01(seed, 4 * count).reshape(count, 4)
    cx, cy = u[:, 0], u[:, 1]
    rad = (rmin + (rmax - rmin) * u[:, 2]) * h
    mu_inc = 10.0 ** (lo + (hi - lo) * u[:, 3])
    xc = (np.arange(n1) + 0.5) * h
    X, Y = np.meshgrid(xc, xc, indexing="xy")  # [cy, cx]
    mu = np.ones((n1, n1))
    for k in range(count):
        mu[(X - cx[k]) ** 2 + (Y - cy[k]) ** 2 <= rad[k] ** 2] = mu_inc[k]
    return mu


def interface2d(n: int = 1024, count: int = 200):
    """2D elliptic interface problem: FV 5-point operator on the inclusion
    field above (seed of workload 3), Dirichlet."""
    return variable_poisson(inclusions_2d(n, count, config_seed(3)))


def q1_jittered(n: int, seed: int, sigma: float = 2.0, corr: float = 16.0, jitter: float = 0.3,
                kappa: np.ndarray | None = None) -> Stencil:
    """Bilinear (Q1) finite elements for -div(kappa grad u) = f on the unit
    square with (n+1)^2 quadrilateral elements, homogeneous Dirichlet.
    Interior nodes are moved by U[-jitter h, jitter h] per coordinate
    (isoparametric elements, 2x2 Gauss quadrature); kappa is constant per
    element, log kappa = sigma g with g a unit-variance Gaussian field of
    correlation length corr elements (workload 5).  Returns the 9-point
    stencil of the interior nodes."""
    n1 = n + 1
    h = 1.0 / n1
    I, J = np.meshgrid(np.arange(n + 2), np.arange(n + 2), indexing="xy")  # [J, I]
    X = I * h
    Y = J * h
    if jitter > 0:
        d = uniform(seed, 2 * n * n, -jitter * h, jitter * h).reshape(2, n, n)
        X = X.copy(); Y = Y.copy()
        X[1:-1, 1:-1] += d[0]
        Y[1:-1, 1:-1] += d[1]
    if kappa is None:
        kappa = np.exp(sigma * gaussian_field((n1, n1), corr, seed + 7919))  # [ey, ex]
    # element corners (ex,ey),(ex+1,ey),(ex+1,ey+1),(ex,ey+1)
    cx = np.stack([X[:-1, :-1], X[:-1, 1:], X[1:, 1:], X[1:, :-1]], axis=-1)  # [ey, ex, 4]
    cy = np.stack([Y[:-1, :-1], Y[:-1, 1:], Y[1:, 1:], Y[1:, :-1]], axis=-1)
    xi_a = np.array([-1.0, 1.0, 1.0, -1.0])
    eta_a = np.array([-1.0, -1.0, 1.0, 1.0])
    g = 1.0 / np.sqrt(3.0)
    K = np.zeros(cx.shape[:2] + (4, 4))
    for xi in (-g, g):
        for eta in (-g, g):
            dNdxi = 0.25 * xi_a * (1 + eta_a * eta)
            dNdeta = 0.25 * eta_a * (1 + xi_a * xi)
            j11 = cx @ dNdxi; j12 = cy @ dNdxi   # d(x,y)/dxi
            j21 = cx @ dNdeta; j22 = cy @ dNdeta  # d(x,y)/deta
            det = j11 * j22 - j12 * j21
            # grad_x N = J^{-T} grad_xi N, with J = [[j11, j12], [j21, j22]] (rows: xi, eta)
            gx = (j22[..., None] * dNdxi - j12[..., None] * dNdeta) / det[..., None]
            gy = (-j21[..., None] * dNdxi + j11[..., None] * dNdeta) / det[..., None]
            K += (kappa * det)[..., None, None] * (gx[..., :, None] * gx[..., None, :] + gy[..., :, None] * gy[..., None, :])
    offs = [(dx, dy, 0) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]  # BOX order
    coeff = np.zeros((9, n, n))  # [s, iy, ix]
    corner = [(0, 0), (1, 0), (1, 1), (0, 1)]  # (di, dj) of corner a
    for a in range(4):
        for b in range(4):
            dx = corner[b][0] - corner[a][0]
            dy = corner[b][1] - corner[a][1]
            s = (dx + 1) + 3 * (dy + 1)
            # node of corner a of element (ex, ey) is (ex + ia, ey + ja); interior when 1..n
            ia, ja = corner[a]
            ib, jb = corner[b]
            ex0, ex1 = max(0, 1 - ia, 1 - ib), min(n1, n + 1 - ia, n + 1 - ib)  # keep a and b interior
            ey0, ey1 = max(0, 1 - ja, 1 - jb), min(n1, n + 1 - ja, n + 1 - jb)
            blk = K[ey0:ey1, ex0:ex1, a, b]
            coeff[s, ey0 + ja - 1:ey1 + ja - 1, ex0 + ia - 1:ex1 + ia - 1] += blk
    return Stencil(2, (n, n, 1), offs, coeff.reshape(9, n * n), False, name=f"q1_{n}",
                   meta={"kappa": kappa})


def rhs(N: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """Right-hand side with i.i.d. entries ~ U[-1, 1] (Sec. 3.1 footnote).
    Shape ``(N,)`` for one RHS, else ``(N, nrhs)`` (RHS-contiguous)."""
    v = uniform(seed, N * nrhs, -1.0, 1.0)
    return v if nrhs == 1 else v.reshape(N, nrhs)


def batch_problem(k: int, nmin: int = 33, nmax: int = 513, mmax: int = 8, corr: float = 8.0,
                  config: int = 4):
    """Problem ``k`` of the batched workload: a 2D variable-coefficient
    Poisson problem (5-point, Dirichlet) with side N ~ U{nmin..nmax} interior
    nodes, nrhs ~ U{1..mmax}, correlated cell coefficients with a log-uniform
    marginal on [1e-3, 1e3] (Gaussian field, correlation ``corr`` cells) and
    right-hand sides ~ U[-1, 1], RHS-contiguous ``[N^2, nrhs]`` flattened.
    Independent streams: sizes from seed s, field from s + 10^6, RHS from
    s + 2*10^6, with s = config_seed(config, k).  Returns (Stencil, nrhs, b)."""
    s = config_seed(config, k)
    u = uniform01(s, 2)
    n = nmin + int(u[0] * (nmax - nmin + 1))
    m = 1 + int(u[1] * mmax)
    A = variable_poisson(log_uniform_field(2, n, corr, s + 1_000_000))
    b = uniform(s + 2_000_000, A.N * m, -1.0, 1.0)
    return A, m, b


def nonsymmetric_3d(n: int, seed: int) -> Stencil:
    """3D 7-point operator with unequal couplings in the two directions of
    every edge, each ~ -U[0.5, 2] from stream ``700 + 10 seed + s`` for
    stencil entry s, and a diagonal 0.1 above the row sum of their
    magnitudes: a nonsymmetric, diagonally dominant M-matrix (a
    convection-diffusion-like test operator whose Galerkin levels are
    nonsymmetric 27-point operators)."""
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    N = n ** 3
    coeff = np.zeros((7, N))
    for s in range(1, 7):
        coeff[s] = -uniform(700 + 10 * seed + s, N, 0.5, 2.0)
    coeff[0] = -coeff[1:].sum(axis=0) + 0.1
    return Stencil(3, (n, n, n), offs, coeff, False, name=f"nonsym3d_{n}")


def stencil_csr(A: Stencil):
    """The operator of a Stencil as a scipy CSR matrix (couplings to nodes
    outside the grid dropped; periodic stencils wrap)."""
    import scipy.sparse as sp
    nx, ny, nz = A.n
    N = A.N
    i = np.arange(N)
    ix, iy, iz = i % nx, (i // nx) % ny, i // (nx * ny)
    rows, cols, vals = [], [], []
    for s_, (dx, dy, dz) in enumerate(A.offsets):
        jx, jy, jz = ix + dx, iy + dy, iz + dz
        if A.periodic:
            jx, jy, jz = jx % nx, jy % ny, jz % nz
            ok = np.ones(N, bool)
        else:
            ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
        rows.append(i[ok])
        cols.append((jx + nx * (jy + ny * jz))[ok])
        vals.append(A.coeff[s_][ok])
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    M.sum_duplicates()
    M.sort_indices()
    return M


def interpolation_1d(n: int):
    """Linear interpolation from the coarse nodes (the fine nodes with even
    1-based index, n // 2 of them) to the n fine nodes of one axis, as a
    dense (n, n // 2) array."""
    nc = n // 2
    P = np.zeros((n, nc))
    for c in range(nc):
        f = 2 * c + 1
        P[f, c] = 1.0
        P[f - 1, c] = 0.5
        if f + 1 < n:
            P[f + 1, c] = 0.5
    return P


def permutation(n: int, seed: int) -> np.ndarray:
    """A seeded random permutation of range(n): perm[new] = old."""
    return np.argsort(uniform01(seed, n), kind="stable")


def unstructured_q1(n: int, seed: int, coarse_side: int = 3, block: int = 3, renumber: bool = True):
    """The jittered Q1 operator of ``q1_jittered(n, seed)`` handed over as a
    general sparse problem: its CSR matrix with the interior nodes renumbered
    by a seeded random permutation, the bilinear interpolations P_l of the
    even-index coarsening (down to sides <= coarse_side) renumbered the same
    way on both of their levels, and a partition of level 0 into
    block x block node blocks (partial at the upper edges) in the new
    numbering.  Nothing of the grid survives in the numbering, so a solver
    that reads it sees an unstructured mesh (renumber=False keeps the grid
    order).  Returns a dict with A (scipy CSR), Ps (list of scipy CSR),
    blocks (bptr, bidx), cells (overlapping blocks: the interior nodes of
    every element) and perms (perm[new] = old per level)."""
    import scipy.sparse as sp
    St = q1_jittered(n, seed)
    sides = [n]
    while sides[-1] > coarse_side and sides[-1] // 2 >= 1:
        sides.append(sides[-1] // 2)
    perms = [permutation(m * m, seed + 7919 * (k + 1)) if renumber else np.arange(m * m)
             for k, m in enumerate(sides)]
    inv = [np.argsort(pm) for pm in perms]  # inv[old] = new
    A = stencil_csr(St)
    A = A[perms[0]][:, perms[0]].tocsr()
    A.sort_indices()
    Ps = []
    for k in range(len(sides) - 1):
        P1 = sp.csr_matrix(interpolation_1d(sides[k]))
        P = sp.kron(P1, P1, format="csr")  # index ix + n iy: kron(P_y, P_x)
        P = P[perms[k]][:, perms[k + 1]].tocsr()
        P.sort_indices()
        Ps.append(P)
    nb1 = (n + block - 1) // block
    old = np.arange(n * n)
    bid = (old % n) // block + nb1 * ((old // n) // block)
    new = inv[0][old]
    order = np.lexsort((new, bid))  # by block, then by new index
    bptr = np.zeros(nb1 * nb1 + 1, dtype=np.int32)
    bptr[1:] = np.cumsum(np.bincount(bid, minlength=nb1 * nb1))
    bidx = new[order].astype(np.int32)
    # overlapping cell blocks: the interior nodes of each of the (n+1)^2
    # elements (an interior node lies in 4 of them)
    ex, ey = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    cptr, cidx = [0], []
    for cx, cy in zip(ex.ravel(), ey.ravel()):
        mem = [inv[0][x + n * y] for y in (cy - 1, cy) for x in (cx - 1, cx) if 0 <= x < n and 0 <= y < n]
        cidx += sorted(int(v) for v in mem)
        cptr.append(len(cidx))
    cells = (np.array(cptr, dtype=np.int32), np.array(cidx, dtype=np.int32))
    return {"A": A, "Ps": Ps, "blocks": (bptr, bidx), "cells": cells, "perms": perms, "sides": sides}


def _mac_index(n: int):
    """Unknown numbering of a MAC grid of n x n cells on the unit square:
    u at the interior vertical faces (i = 1..n-1, j = 0..n-1), then v at the
    interior horizontal faces (i = 0..n-1, j = 1..n-1), then p at the cells."""
    nu = (n - 1) * n
    U = lambda i, j: (i - 1) + (n - 1) * j  # noqa: E731
    V = lambda i, j: nu + i + n * (j - 1)  # noqa: E731
    Pc = lambda i, j: 2 * nu + i + n * j  # noqa: E731
    return nu, U, V, Pc


def mac_stokes_2d(n: int, mu: float = 1.0, delta: float = 1e-3, coarse_cells: int = 4):
    """Steady Stokes, -mu Lap u + grad p = f, -div u = g, on the unit square
    with no-slip walls, discretised by the MAC staggered-grid finite
    difference method on n x n cells (n a power of two times coarse_cells),
    in finite-volume scaling (every equation times h^2): the viscous block
    mu (4 u_c - sum of neighbours, a wall-side tangential neighbour replaced
    by the reflected ghost -u_c), G = h (p_right - p_left), D = G^T, and a
    small pressure stabilisation -delta h^2 I that removes the constant
    pressure mode.  Unknowns as in _mac_index; fields 0 (velocity) / 1
    (pressure).  Transfers per coarsening (n -> n/2): pressure piecewise
    constant over the 2 x 2 subcells; a u face linear along x between the
    coarse faces it lies between (wall faces contribute zero) and constant
    along y over the coarse cell row; v likewise with x and y exchanged.
    Blocks: per cell its pressure and its right and top faces (d + 1 = 3
    unknowns; fewer at the upper walls), on every level.  Returns a dict
    with A (scipy CSR), fields, Ps, blocks (list per level) and sides."""
    import scipy.sparse as sp

    def operator(m):
        h = 1.0 / m
        nu, U, V, Pc = _mac_index(m)
        N = 2 * nu + m * m
        rows, cols, vals = [], [], []

        def add(r, c, v):
            rows.append(r)
            cols.append(c)
            vals.append(v)
        for j in range(m):  # u momentum
            for i in range(1, m):
                r, d = U(i, j), 4.0
                for ii in (i - 1, i + 1):
                    if 1 <= ii <= m - 1:
                        add(r, U(ii, j), -mu)
                for jj in (j - 1, j + 1):
                    if 0 <= jj <= m - 1:
                        add(r, U(i, jj), -mu)
                    else:
                        d += 1.0  # ghost -u across the wall
                add(r, r, mu * d)
                add(r, Pc(i, j), h)
                add(r, Pc(i - 1, j), -h)
        for j in range(1, m):  # v momentum
            for i in range(m):
                r, d = V(i, j), 4.0
                for jj in (j - 1, j + 1):
                    if 1 <= jj <= m - 1:
                        add(r, V(i, jj), -mu)
                for ii in (i - 1, i + 1):
                    if 0 <= ii <= m - 1:
                        add(r, V(ii, j), -mu)
                    else:
                        d += 1.0
                add(r, r, mu * d)
                add(r, Pc(i, j), h)
                add(r, Pc(i, j - 1), -h)
        for j in range(m):  # continuity: -div u (= G^T) and the stabilisation
            for i in range(m):
                r = Pc(i, j)
                if i + 1 <= m - 1:
                    add(r, U(i + 1, j), -h)
                if i >= 1:
                    add(r, U(i, j), h)
                if j + 1 <= m - 1:
                    add(r, V(i, j + 1), -h)
                if j >= 1:
                    add(r, V(i, j), h)
                add(r, r, -delta * h * h)
        A = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
        A.sum_duplicates()
        A.sort_indices()
        return A

    def transfer(m):
        mc = m // 2
        nuf, Uf, Vf, Pf = _mac_index(m)
        nuc, Uc, Vc, Pcc = _mac_index(mc)
        rows, cols, vals = [], [], []
        for j in range(m):
            for i in range(1, m):
                J = j // 2
                for I, wgt in (((i // 2, 1.0),) if i % 2 == 0 else (((i - 1) // 2, 0.5), ((i + 1) // 2, 0.5))):
                    if 1 <= I <= mc - 1:
                        rows.append(Uf(i, j)); cols.append(Uc(I, J)); vals.append(wgt)
        for j in range(1, m):
            for i in range(m):
                I = i // 2
                for J, wgt in (((j // 2, 1.0),) if j % 2 == 0 else (((j - 1) // 2, 0.5), ((j + 1) // 2, 0.5))):
                    if 1 <= J <= mc - 1:
                        rows.append(Vf(i, j)); cols.append(Vc(I, J)); vals.append(wgt)
        for j in range(m):
            for i in range(m):
                rows.append(Pf(i, j)); cols.append(Pcc(i // 2, j // 2)); vals.append(1.0)
        P = sp.csr_matrix((vals, (rows, cols)), shape=(2 * nuf + m * m, 2 * nuc + mc * mc))
        P.sum_duplicates()
        P.sort_indices()
        return P

    def blocks(m):
        nu, U, V, Pc = _mac_index(m)
        bptr, bidx = [0], []
        for j in range(m):
            for i in range(m):
                mem = [Pc(i, j)]
                if i + 1 <= m - 1:
                    mem.append(U(i + 1, j))
                if j + 1 <= m - 1:
                    mem.append(V(i, j + 1))
                bidx += sorted(mem)
                bptr.append(len(bidx))
        return np.array(bptr, dtype=np.int32), np.array(bidx, dtype=np.int32)

    sides = [n]
    while sides[-1] > coarse_cells and sides[-1] % 2 == 0:
        sides.append(sides[-1] // 2)
    nu0 = (n - 1) * n
    fields = np.concatenate([np.zeros(2 * nu0, dtype=np.int32), np.ones(n * n, dtype=np.int32)])
    return {"A": operator(n), "fields": fields, "Ps": [transfer(m) for m in sides[:-1]],
            "blocks": [blocks(m) for m in sides], "sides": sides}


def config_seed(config: int, problem: int = 0) -> int:
    """Seed of problem ``problem`` of workload ``config`` (run seed 0)."""
    return 1000 * config + problem


def poisson2d_64() -> Tuple[Stencil, np.ndarray]:
    """2D Poisson, 5-point FD on a 64x64 interior grid, Dirichlet; RHS ~ U[-1,1]."""
    A = poisson(2, 64)
    return A, rhs(A.N, config_seed(1))


def poisson3d(n: int = 256) -> Tuple[Stencil, np.ndarray]:
    """3D Poisson, 7-point FD on an n^3 interior grid, Dirichlet; RHS ~ U[-1,1]."""
    A = poisson(3, n)
    return A, rhs(A.N, config_seed(2))
