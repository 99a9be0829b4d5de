"""FP64 CPU oracle for cascading-smoother multigrid -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_2606_12577_gb300`` never does, and the two share no code: the only
thing both sides consume is the seeded input module ``problems``.

The arithmetic lives in ``cs_oracle.c`` (plain C loops over CSR matrices,
one function per step of the paper; see its header for the citations).  This
file compiles it with gcc on first use, marshals numpy arrays through ctypes,
and implements the paper's reporting metrics (rho, eta, C_d) in numpy.

Parity pins: see ``tests/test_oracle_pins.py`` (Table 1, Fourier closed
forms, brute-force dense least squares, monotonicity, propagators, V-cycle
symmetry, Galerkin stencils, special cases, convergence).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libcs_oracle.so")
_lock = threading.Lock()
_lib = None

KINDS = {"additive": 0, "multiplicative": 1}
PRESCALE = {"none": 0, "elliptic": 1, "stokes1": 2, "stokes2": 3, "stokesinf": 4, False: 0, True: 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction so that
    x86 and Arm hosts round identically)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P, I, D, L = C.c_void_p, C.c_int, C.c_double, C.c_int64
        sig = {
            "ora_hier_create": (P, [I, P, I, P, P, I, I, I, I, I]),
            "ora_hier_free": (None, [P]),
            "ora_hier_nlev": (I, [P]),
            "ora_hier_dims": (None, [P, I, P]),
            "ora_hier_nnz": (L, [P, I]),
            "ora_hier_csr": (None, [P, I, P, P, P]),
            "ora_hier_nblocks": (I, [P, I]),
            "ora_hier_blocks": (None, [P, I, P, P, P]),
            "ora_casc_create": (P, [P, I, I, I, I]),
            "ora_casc_empty": (P, [P, I, I]),
            "ora_casc_free": (None, [P]),
            "ora_casc_nlev": (I, [P]),
            "ora_casc_lamsize": (L, [P, I]),
            "ora_casc_lambda": (None, [P, I, P]),
            "ora_casc_set_lambda": (None, [P, I, P]),
            "ora_casc_efrob": (None, [P, I, P]),
            "ora_residual": (None, [P, I, P, P, P]),
            "ora_smooth": (None, [P, P, I, I, P, P]),
            "ora_restrict": (None, [P, I, P, P]),
            "ora_prolong_correct": (None, [P, I, P, P]),
            "ora_coarse_solve": (None, [P, P, P]),
            "ora_vcycle": (None, [P, P, I, I, I, P, P]),
            "ora_solve": (I, [P, P, I, I, I, I, D, I, I, P, P, P, P, P]),
            "ora_set_threads": (None, [I]),
            "ora_ghier_new": (P, [I, P, P, P, D]),
            "ora_ghier_add_level": (I, [P, I, P, P, P]),
            "ora_ghier_set_blocks": (I, [P, I, I, P, P]),
            "ora_ghier_set_fields": (None, [P, P]),
            "ora_ghier_finish": (I, [P, C.c_uint64]),
            "ora_prescale_weights": (I, [P, I, I, P]),
            "ora_hier_nbidx": (I, [P, I]),
            "ora_hier_overlap": (I, [P, I]),
            "ora_casc_create_ex": (P, [P, I, I, I, I, I]),
            "ora_hier_ncol": (I, [P, I]),
            "ora_block_prio": (C.c_uint64, [C.c_uint64, I, I]),
            "ora_casc_create_sketch": (P, [P, I, I, I, I, C.c_uint64, I]),
            "ora_rademacher": (D, [C.c_uint64, I, L, I, I]),
            "ora_max_threads": (I, []),
            "ora_plant": (None, [I]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def rademacher(seed: int, level: int, i: int, t: int, s: int) -> float:
    """Entry (i, t) of the level's Rademacher sketch (the counter-based
    SplitMix64 stream described in cs_oracle.c)."""
    return float(_load().ora_rademacher(int(seed) & 0xFFFFFFFFFFFFFFFF, level, i, t, s))


def block_priority(seed: int, level: int, b: int) -> int:
    """Priority of block b of a level in the greedy colouring (SplitMix64
    output at counter level 2^40 + b of the stream seeded with `seed`)."""
    return int(_load().ora_block_prio(int(seed) & 0xFFFFFFFFFFFFFFFF, level, b))


# the planted mistakes of cs_oracle.c, in the order of its enum (ids 1, 2, ...)
PLANTS = ("prescale_off", "update_sign", "lambda_t", "smooth_t", "colour_order", "reverse_order",
          "smooth_sign", "interp_one_sided", "restrict_unscaled", "coarse_chol", "trunc_smallest",
          "minnorm_off", "overlap_sum", "stokes_q2", "spd_no_upper", "pcg_beta", "greedy_ascending",
          "sketch_stale", "prescale_power", "overlap_smooth_sum", "galerkin_rscale", "parity",
          "givens_sign", "right_update_v", "inplace_colour",
          "sketch_first_t", "boundary_wrap", "prolong_sign", "rf_forward", "stokes_vel_l1",
          "sketch_z_once", "spd_unweighted")


@contextlib.contextmanager
def planted(name: str):
    """Inside the block the oracle takes one known-wrong step (tests only,
    to show that the pins reject it); outside it every step is as stated."""
    lib = _load()
    lib.ora_plant(PLANTS.index(name) + 1)
    try:
        yield
    finally:
        lib.ora_plant(0)


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (results do not depend on it)."""
    _load().ora_set_threads(int(n))


def max_threads() -> int:
    return int(_load().ora_max_threads())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Hierarchy:
    """Geometric hierarchy (Sec. 2.4): even-index node coarsening until the
    largest side is <= coarse_max, bilinear/trilinear P, Galerkin
    A_2h = R A_h P with R = 2^{-d} P^T (rscale_mode=1: R = P^T)."""

    def __init__(self, A, bs: int = 1, coarse_max: int = 4, max_levels: int = 0, rscale_mode: int = 0):
        lib = _load()
        self.dim = A.dim
        self.bs = bs
        n3 = np.asarray(A.n, dtype=np.int32)
        off = np.ascontiguousarray(A.offsets_array(), dtype=np.int32)
        coeff = _f64(A.coeff)
        self._h = lib.ora_hier_create(A.dim, _ptr(n3), A.nst, _ptr(off), _ptr(coeff), int(A.periodic),
                                      bs, coarse_max, max_levels, rscale_mode)
        if not self._h:
            raise RuntimeError("oracle hierarchy creation failed")
        self.nlev = lib.ora_hier_nlev(self._h)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ora_hier_free(self._h)
            self._h = None

    @classmethod
    def from_csr(cls, A, Ps, rscale: float = 1.0, blocks=None, seed: int = 0, fields=None):
        """Hierarchy of a general sparse operator (the CSR path): A (scipy
        CSR, N0 x N0), one interpolation P_l per coarser level (scipy CSR,
        N_l x N_{l+1}), Galerkin A_{l+1} = rscale P_l^T A_l P_l; blocks =
        (bptr, bidx) of level 0, or a list of such pairs per level (None:
        point blocks); greedy colouring with the block priorities of `seed`;
        fields: 0 (velocity / scalar) or 1 (pressure) per finest unknown."""
        lib = _load()
        self = cls.__new__(cls)
        self.dim, self.bs = 0, 0
        A = A.tocsr()
        A.sort_indices()
        rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
        ci = np.ascontiguousarray(A.indices, dtype=np.int32)
        v = _f64(A.data)
        self._h = lib.ora_ghier_new(A.shape[0], _ptr(rp), _ptr(ci), _ptr(v), float(rscale))
        for P in Ps:
            P = P.tocsr()
            P.sort_indices()
            prp = np.ascontiguousarray(P.indptr, dtype=np.int64)
            pci = np.ascontiguousarray(P.indices, dtype=np.int32)
            if lib.ora_ghier_add_level(self._h, P.shape[1], _ptr(prp), _ptr(pci), _ptr(_f64(P.data))) != 0:
                raise RuntimeError("too many levels")
        if blocks is not None:
            per_level = blocks if isinstance(blocks, list) else [blocks]
            for l, bl in enumerate(per_level):
                if bl is None:
                    continue
                bptr = np.ascontiguousarray(bl[0], dtype=np.int32)
                bidx = np.ascontiguousarray(bl[1], dtype=np.int32)
                if lib.ora_ghier_set_blocks(self._h, l, len(bptr) - 1, _ptr(bptr), _ptr(bidx)) != 0:
                    raise ValueError(f"level {l}: blocks are not a partition of the unknowns")
        if fields is not None:
            f = np.ascontiguousarray(fields, dtype=np.int32)
            lib.ora_ghier_set_fields(self._h, _ptr(f))
        if lib.ora_ghier_finish(self._h, int(seed) & 0xFFFFFFFFFFFFFFFF) != 0:
            raise ValueError("an interpolation maps one coarse unknown to fine unknowns of two fields")
        self.nlev = lib.ora_hier_nlev(self._h)
        return self

    def prescale_weights(self, l: int, mode) -> np.ndarray:
        """The diagonal of W on level l: mode 'none', 'elliptic' or
        'stokes1' / 'stokes2' / 'stokesinf' (q = 1, 2, infinity)."""
        out = np.zeros(self.N(l))
        if _lib.ora_prescale_weights(self._h, l, PRESCALE[mode], _ptr(out)) != 0:
            raise ValueError("prescaling weight undefined (non-positive diagonal or norm)")
        return out

    def overlapping(self, l: int) -> bool:
        return bool(_lib.ora_hier_overlap(self._h, l))

    def ncolours(self, l: int) -> int:
        return int(_lib.ora_hier_ncol(self._h, l))

    def dims(self, l: int):
        out = np.zeros(3, dtype=np.int32)
        _lib.ora_hier_dims(self._h, l, _ptr(out))
        return tuple(int(v) for v in out)

    def N(self, l: int) -> int:
        d = self.dims(l)
        return d[0] * d[1] * d[2]

    def csr(self, l: int):
        """(rowptr, colind, values) of the level-l operator."""
        N = self.N(l)
        nnz = _lib.ora_hier_nnz(self._h, l)
        rp = np.zeros(N + 1, dtype=np.int64)
        ci = np.zeros(nnz, dtype=np.int32)
        v = np.zeros(nnz, dtype=np.float64)
        _lib.ora_hier_csr(self._h, l, _ptr(rp), _ptr(ci), _ptr(v))
        return rp, ci, v

    def dense(self, l: int) -> np.ndarray:
        rp, ci, v = self.csr(l)
        N = len(rp) - 1
        M = np.zeros((N, N))
        for i in range(N):
            M[i, ci[rp[i]:rp[i + 1]]] += v[rp[i]:rp[i + 1]]
        return M

    def blocks(self, l: int):
        """(bptr, members, parity) of the level-l block partition."""
        nb = _lib.ora_hier_nblocks(self._h, l)
        bptr = np.zeros(nb + 1, dtype=np.int32)
        bidx = np.zeros(_lib.ora_hier_nbidx(self._h, l), dtype=np.int32)
        bpar = np.zeros(nb, dtype=np.int32)
        _lib.ora_hier_blocks(self._h, l, _ptr(bptr), _ptr(bidx), _ptr(bpar))
        return bptr, bidx, bpar

    def colours(self, l: int) -> np.ndarray:
        """Red-black colour id (0 = red) of every unknown on level l."""
        bptr, bidx, bpar = self.blocks(l)
        out = np.zeros(self.N(l), dtype=np.int8)
        for b in range(len(bpar)):
            out[bidx[bptr[b]:bptr[b + 1]]] = bpar[b]
        return out

    # ---- single steps of Algorithm 1
    def residual(self, l, b, x):
        r = np.zeros(self.N(l))
        _lib.ora_residual(self._h, l, _ptr(_f64(b)), _ptr(_f64(x)), _ptr(r))
        return r

    def restrict(self, l, r):
        rc = np.zeros(self.N(l + 1))
        _lib.ora_restrict(self._h, l, _ptr(_f64(r)), _ptr(rc))
        return rc

    def prolong_correct(self, l, xc, x):
        x = _f64(x).copy()
        _lib.ora_prolong_correct(self._h, l, _ptr(_f64(xc)), _ptr(x))
        return x

    def coarse_solve(self, b):
        x = np.zeros(self.N(self.nlev - 1))
        _lib.ora_coarse_solve(self._h, _ptr(_f64(b)), _ptr(x))
        return x


class Cascade:
    """Cascading smoothers on every smoothing level of a hierarchy
    (Algorithm 2; SM Algorithm for kind='multiplicative', red-black)."""

    def __init__(self, hier: Hierarchy, kind: str = "additive", nu: int = 3, prescale: bool = True,
                 alpha: int = 0, _empty: bool = False, sketch: int = 0, seed: int = 0, exact_first: bool = False,
                 spd: bool = False):
        """sketch > 0: the sketched setup of the concluding remarks (Sec. 4)
        with a Rademacher sketch of `sketch` columns from `seed` (see
        ``rademacher``); exact_first: step 1 unsketched."""
        self.hier = hier
        self.kind = kind
        self.nu = nu
        self.ncol = 2 if kind == "multiplicative" else 1
        if _empty:
            self._c = _lib.ora_casc_empty(hier._h, KINDS[kind], nu)
        elif sketch > 0:
            self._c = _lib.ora_casc_create_sketch(hier._h, KINDS[kind], nu, PRESCALE[prescale], int(sketch),
                                                  int(seed) & 0xFFFFFFFFFFFFFFFF, int(exact_first))
        else:
            self._c = _lib.ora_casc_create_ex(hier._h, KINDS[kind], nu, PRESCALE[prescale], alpha, int(spd))
        if not self._c:
            raise RuntimeError("oracle cascade setup failed (non-positive diagonal under prescaling?)")
        self.nlev = _lib.ora_casc_nlev(self._c)

    @classmethod
    def empty(cls, hier, kind="additive", nu=1):
        return cls(hier, kind, nu, _empty=True)

    def __del__(self):
        if getattr(self, "_c", None) and _lib is not None:
            _lib.ora_casc_free(self._c)
            self._c = None

    def lamsize(self, l: int) -> int:
        return int(_lib.ora_casc_lamsize(self._c, l))

    def lam(self, l: int) -> np.ndarray:
        """Lambda_{l'} on hierarchy level l as [nu, lamsize]: block b's
        n_b x n_b matrix row-major at its offset (point blocks: one value per
        unknown).  Multiplicative: Lambda_{l',k} sits on the blocks of colour k."""
        out = np.zeros((self.nu, self.lamsize(l)))
        _lib.ora_casc_lambda(self._c, l, _ptr(out))
        return out

    def set_lam(self, l: int, lam: np.ndarray):
        lam = _f64(lam).reshape(self.nu, self.lamsize(l))
        _lib.ora_casc_set_lambda(self._c, l, _ptr(lam))

    def efrob(self, l: int) -> np.ndarray:
        """||E~||_F after each setup step (prescaled space), starting with E_0 = I."""
        out = np.zeros(self.nu * self.ncol + 1)
        _lib.ora_casc_efrob(self._c, l, _ptr(out))
        return out


def smooth(h: Hierarchy, c: Cascade, l: int, b, x, reverse: bool = False) -> np.ndarray:
    x = _f64(x).copy()
    _lib.ora_smooth(h._h, c._c, l, int(reverse), _ptr(_f64(b)), _ptr(x))
    return x


def vcycle(h: Hierarchy, c: Cascade, b, x=None, mu_pre: int = 1, mu_post: int = 1, rf: bool = True) -> np.ndarray:
    x = np.zeros(h.N(0)) if x is None else _f64(x).copy()
    _lib.ora_vcycle(h._h, c._c, mu_pre, mu_post, int(rf), _ptr(_f64(b)), _ptr(x))
    return x


def solve(h: Hierarchy, c: Cascade, b, x=None, method: str = "stationary", mu_pre: int = 1,
          mu_post: int = 1, rf: bool = True, tol: float = 1e-10, maxit: int = 100, restart: int = 30):
    """Returns (x, iterations or -1, history, final relative true residual).

    method: "stationary" (x <- V(x, b)), "gmres" (left-preconditioned
    restarted GMRES, Sec. 3.1; history = preconditioned residual estimates
    ||M r|| / ||M b||) or "gmres_right" (the cycle applied on the right,
    minimising the true residual; history = ||b - A x|| / ||b|| estimates)."""
    x = np.zeros(h.N(0)) if x is None else _f64(x).copy()
    hist = np.zeros(2 * maxit + 4)
    nh = C.c_int(0)
    fin = C.c_double(0.0)
    code = {"stationary": 0, "gmres": 1, "gmres_right": 2, "pcg": 3}[method]
    it = _lib.ora_solve(h._h, c._c, code, mu_pre, mu_post, int(rf), tol,
                        maxit, restart, _ptr(_f64(b)), _ptr(x), _ptr(hist), C.byref(nh), C.byref(fin))
    return x, int(it), hist[: nh.value].copy(), float(fin.value)


# ---------------------------------------------------------------- metrics
def rho_from_history(r) -> float:
    """Convergence rate by least-squares regression of log r_i on i
    (Sec. 3.1 footnote)."""
    r = np.asarray(r, dtype=np.float64)
    r = r[r > 0]
    i = np.arange(len(r), dtype=np.float64)
    slope = np.polyfit(i, np.log(r), 1)[0]
    return float(np.exp(slope))


def eta(rho: float) -> float:
    """eta = log 0.1 / log rho (eq. eta)."""
    return float(np.log(0.1) / np.log(rho))


def cost_cd(d: int, nu: int, eta_value: float) -> float:
    """C_d(nu, eta) = eta (1 + (2 nu + 1) / (1 - 2^{-d})) (eq. cost)."""
    return float(eta_value * (1.0 + (2 * nu + 1) / (1.0 - 2.0 ** (-d))))
