"""Brute-force dense restatements used only to pin the oracle.

Everything here forms matrices explicitly (numpy, FP64) on tiny grids and
uses library routines (``numpy.linalg.lstsq``, ``solve``, ``kron``) for the
steps, so that a mistake in the oracle's sparse bookkeeping (fill-in
patterns, block rows, colour commits, transposes, index maps) shows up as a
mismatch.  It shares nothing with the oracle's C code.
"""
from __future__ import annotations

import numpy as np


def dense_from_stencil(A) -> np.ndarray:
    """Dense matrix of a ``problems.Stencil`` (Dirichlet: drop outside
    neighbours; periodic: wrap)."""
    nx, ny, nz = A.n
    N = A.N
    M = np.zeros((N, N))
    for s, (dx, dy, dz) in enumerate(A.offsets):
        for iz in range(nz):
            for iy in range(ny):
                for ix in range(nx):
                    jx, jy, jz = ix + dx, iy + dy, iz + dz
                    if A.periodic:
                        jx %= nx; jy %= ny; jz %= nz
                    elif not (0 <= jx < nx and 0 <= jy < ny and 0 <= jz < nz):
                        continue
                    i = ix + nx * (iy + ny * iz)
                    j = jx + nx * (jy + ny * jz)
                    M[i, j] += A.coeff[s, i]
    return M


def block_partition(n3, dim, bs):
    """List of member-index arrays (ascending) of the bs^d-node blocks and
    their red-black parity ((bx+1)+(by+1)[+(bz+1)]) % 2."""
    nx, ny, nz = n3
    nbx, nby = -(-nx // bs), -(-ny // bs)
    nbz = -(-nz // bs) if dim == 3 else 1
    members = [[] for _ in range(nbx * nby * nbz)]
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                bz = iz // bs if dim == 3 else 0
                members[ix // bs + nbx * (iy // bs + nby * bz)].append(ix + nx * (iy + ny * iz))
    par = []
    for bz in range(nbz):
        for by in range(nby):
            for bx in range(nbx):
                par.append(((bx + 1) + (by + 1) + ((bz + 1) if dim == 3 else 0)) % 2)
    return [np.array(sorted(m)) for m in members], np.array(par)


def dense_cascade(Ad, blocks, parity, kind, nu, alpha=0, bs_blocks=None, w=None):
    """Cascade setup by explicit dense matrices and numpy lstsq.

    Returns (lam_tilde, lam, Es): prescaled and unscaled Lambda per step as
    dense block-diagonal matrices (list over l of list over colours), and the
    dense residual E~ after every (l, k) step (prescaled space)."""
    N = Ad.shape[0]
    if w is None:  # elliptic prescaling
        w = 1.0 / np.sqrt(np.diag(Ad))
    At = w[:, None] * Ad * w[None, :]
    E = np.eye(N)
    ncol = (int(np.max(parity)) + 1 if len(parity) else 1) if kind == "multiplicative" else 1
    blk_of = np.zeros(N, dtype=int)
    for b, m in enumerate(blocks):
        blk_of[m] = b
    lam_t, lam_u, Es = [], [], [E.copy()]
    for l in range(nu):
        per_col_t, per_col_u = [], []
        for k in range(ncol):
            L = np.zeros((N, N))
            Enew = E.copy()
            AE = At @ E
            for b, rows in enumerate(blocks):
                if kind == "multiplicative" and parity[b] != k:
                    continue
                Rb = AE[rows, :]
                Eb = E[rows, :]
                # Lam Rb ~= Eb in the least-squares sense  <=>  Rb^T Lam^T ~= Eb^T,
                # minimum norm where Rb is rank deficient: singular values with
                # sigma^2 <= 1e-14 sum(sigma^2) count as zero (the method's rule,
                # eigenvalues of G = Rb Rb^T at or below 1e-14 tr G), as lstsq's rcond
                sv = np.linalg.svd(Rb, compute_uv=False)
                rc = np.sqrt(1e-14 * np.sum(sv ** 2)) / sv[0] if sv.size and sv[0] > 0 else 1.0
                lt = np.linalg.lstsq(Rb.T, Eb.T, rcond=rc)[0].T
                L[np.ix_(rows, rows)] = lt
                new = Eb - lt @ Rb
                if alpha > 0:
                    cols = np.nonzero(np.any(new != 0.0, axis=0) | np.any(Rb != 0.0, axis=0) | np.any(Eb != 0.0, axis=0))[0]
                    cb = sorted(set(blk_of[cols].tolist()))
                    if len(cb) > alpha:
                        norms = {c: float(np.sum(new[:, blk_of == c] ** 2)) for c in cb}
                        keep = sorted(cb, key=lambda c: (-norms[c], c))[:alpha]
                        mask = np.isin(blk_of, keep)
                        new = new * mask[None, :]
                Enew[rows, :] = new
            E = Enew
            Es.append(E.copy())
            per_col_t.append(L)
            per_col_u.append(w[:, None] * L * w[None, :])
        lam_t.append(per_col_t)
        lam_u.append(per_col_u)
    return lam_t, lam_u, Es


def prolongation_1d(nf: int) -> np.ndarray:
    """Interior-node linear interpolation, coarse nodes = even 1-based fine
    indices (built from the geometric definition, not from the oracle)."""
    nc = nf // 2
    P = np.zeros((nf, nc))
    xf = np.arange(1, nf + 1, dtype=float)          # fine node positions (units of h)
    xc = 2.0 * np.arange(1, nc + 1, dtype=float)    # coarse node positions
    for j in range(nc):
        # hat function of coarse node j with support radius 2h
        P[:, j] = np.maximum(0.0, 1.0 - np.abs(xf - xc[j]) / 2.0)
    return P


def prolongation(n3, dim) -> np.ndarray:
    Px = prolongation_1d(n3[0])
    Py = prolongation_1d(n3[1])
    if dim == 2:
        return np.kron(Py, Px)
    return np.kron(prolongation_1d(n3[2]), np.kron(Py, Px))


def dense_overlap_cascade(Ad, blocks, nu, w=None):
    """Overlapping-block additive cascade (Sec. 3.6.2) by explicit dense
    matrices: Theta (M x N) replicates the nodes of the blocks, theta its
    column sums; per step Lambda_l = argmin over block-diagonal Lambda of
    ||(Theta - Lambda Theta A~) E_{l-1}||_F (per block lstsq with the
    method's rank rule) and E_l = diag(theta)^-1 Theta^T (Theta - Lambda_l
    Theta A~) E_{l-1}.  Returns the unscaled per-block Lambda per step (list
    over steps of lists over blocks), the dense Theta, and ||E_l||_F for
    l = 0..nu."""
    N = Ad.shape[0]
    if w is None:
        w = 1.0 / np.sqrt(np.diag(Ad))
    At = w[:, None] * Ad * w[None, :]
    M = sum(len(b) for b in blocks)
    Th = np.zeros((M, N))
    r = 0
    for b in blocks:
        for i in b:
            Th[r, i] = 1.0
            r += 1
    theta = Th.sum(axis=0)
    E = np.eye(N)
    out, norms = [], [np.linalg.norm(E)]
    for _ in range(nu):
        AE = At @ E
        new = np.zeros((M, N))
        lams = []
        r = 0
        for b in blocks:
            Rb, Eb = AE[b, :], E[b, :]
            sv = np.linalg.svd(Rb, compute_uv=False)
            rc = np.sqrt(1e-14 * np.sum(sv ** 2)) / sv[0] if sv.size and sv[0] > 0 else 1.0
            lt = np.linalg.lstsq(Rb.T, Eb.T, rcond=rc)[0].T
            new[r:r + len(b)] = Eb - lt @ Rb
            lams.append(w[b][:, None] * lt * w[b][None, :])
            r += len(b)
        E = (Th.T @ new) / theta[:, None]
        out.append(lams)
        norms.append(np.linalg.norm(E))
    return out, Th, np.array(norms)
