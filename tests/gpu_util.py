"""Helpers shared by the GPU parity tests: feed a ``problems.Stencil`` to the
CUDA library and bring its exported state back as scipy matrices."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def gpu_hierarchy(A, **kw):
    import torch

    import paper_2606_12577_gb300 as cmg
    coeff = torch.tensor(A.coeff, dtype=torch.float64, device="cuda")
    h = cmg.setup_hierarchy(A.dim, A.n, A.offsets, coeff, periodic=A.periodic, **kw)
    torch.cuda.synchronize()
    return h


def stencil_to_csr(n3, offsets, coeff, periodic=False) -> sp.csr_matrix:
    nx, ny, nz = n3
    N = nx * ny * nz
    i = np.arange(N)
    ix, iy, iz = i % nx, (i // nx) % ny, i // (nx * ny)
    rows, cols, vals = [], [], []
    for s, (dx, dy, dz) in enumerate(offsets):
        jx, jy, jz = ix + dx, iy + dy, iz + dz
        if periodic:
            jx, jy, jz = jx % nx, jy % ny, jz % nz
            ok = np.ones(N, bool)
        else:
            ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
        rows.append(i[ok])
        cols.append((jx + nx * (jy + ny * jz))[ok])
        vals.append(coeff[s][ok])
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    M.sum_duplicates()
    return M


def oracle_csr(h, l) -> sp.csr_matrix:
    rp, ci, v = h.csr(l)
    N = len(rp) - 1
    return sp.csr_matrix((v, ci, rp), shape=(N, N))


def rel_max(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def stencil_matvec(A, x) -> np.ndarray:
    """y = A x straight from the stencil arrays (FP64, numpy)."""
    nx, ny, nz = A.n
    X = x.reshape(nz, ny, nx)
    y = np.zeros_like(X)
    for s, (dx, dy, dz) in enumerate(A.offsets):
        sh = np.zeros_like(X)
        sh[max(-dz, 0):nz + min(-dz, 0), max(-dy, 0):ny + min(-dy, 0), max(-dx, 0):nx + min(-dx, 0)] = \
            X[max(dz, 0):nz + min(dz, 0), max(dy, 0):ny + min(dy, 0), max(dx, 0):nx + min(dx, 0)]
        y += A.coeff[s].reshape(nz, ny, nx) * sh
    return y.ravel()
