"""Cascading-smoother geometric multigrid on GB300 (sm_103a).

Python binding of the C ABI declared in ``include/cascade_mg.h``: the same
entry points (``setup_hierarchy``, ``setup_cascade``, ``vcycle``, ``solve``,
``smooth``, ``residual_restrict``, ``prolong_correct``, ``coarse_solve``,
``residual`` and the exports), marshalling torch CUDA tensors (device
memory) and streams into plain pointers.  All arithmetic runs in the CUDA
kernels of ``libcascade_mg.so``; when the library is missing every call
raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _capi
from ._capi import CascadeError

__all__ = ["setup_hierarchy", "setup_cascade", "vcycle", "solve", "smooth", "sweep", "sweep_rhs", "residual_restrict",
           "prolong_correct", "coarse_solve", "residual", "query_level", "export_operator", "export_colours",
           "export_lambda", "kernel_launches", "smooth_noalloc", "MLP", "block_features", "block_targets", "learned_status", "learned_stats", "setup_many", "Batch", "solve_batched", "Hierarchy", "Cascade", "SolveInfo",
           "CascadeError", "GHierarchy", "GCascade", "gsetup_hierarchy", "gsetup_cascade", "gexport_lambda", "tc_gemm_bf16", "gsweep",
           "gsmooth", "gvcycle", "gsolve", "residual_restrict_lowp", "prolong_correct_lowp"]


def _torch():
    import torch
    return torch


def _stream(stream):
    if stream is None:
        torch = _torch()
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dev_ptr(t, n=None, name="tensor"):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return C.c_void_p(t.data_ptr())


class Hierarchy:
    """Handle of a geometric hierarchy (owns its device memory)."""

    def __init__(self, ptr, dim):
        self._p = ptr
        self.dim = dim
        self._infos = {}
        lvl = self.level_info(0)
        self.nlevels = lvl["nlevels"]

    @property
    def ptr(self):
        return self._p

    def level_info(self, level):
        if level not in self._infos:
            info = _capi.cs_level_info()
            _capi.check(_capi.lib().cs_query_level(self._p, level, C.byref(info)), "cs_query_level")
            self._infos[level] = {
                "dim": info.dim, "n": tuple(info.n), "N": int(info.N), "nst": info.nst,
                "offsets": [tuple(info.off[s]) for s in range(info.nst)], "nlevels": info.nlevels,
                "block": info.block, "lamsize": int(info.lamsize), "sym32": bool(info.sym32)}
        return self._infos[level]

    def N(self, level=0):
        return self.level_info(level)["N"]

    def nbytes(self):
        return int(_capi.lib().cs_hierarchy_bytes(self._p))

    def __del__(self):
        if getattr(self, "_p", None) and _capi._lib is not None:
            _capi._lib.cs_destroy_hierarchy(self._p)
            self._p = None


class Cascade:
    """Handle of a cascade built on a hierarchy (keeps the hierarchy alive)."""

    def __init__(self, ptr, hier, kind, nu, lowp):
        self._p = ptr
        self.hier = hier
        self.kind = kind
        self.nu = nu
        self.lowp = lowp

    @property
    def ptr(self):
        return self._p

    def nbytes(self):
        return int(_capi.lib().cs_cascade_bytes(self._p))

    def __del__(self):
        if getattr(self, "_p", None) and _capi._lib is not None:
            _capi._lib.cs_destroy_cascade(self._p)
            self._p = None


@dataclass
class SolveInfo:
    status: int
    iterations: int
    converged: bool
    final_rel_residual: float
    history: np.ndarray


def setup_hierarchy(dim, n, offsets, coeff, periodic=False, coarse_max=4, max_levels=0, block=1, reuse=True,
                    stream=None):
    """Build the hierarchy of the structured operator given by ``offsets``
    (list of (dx,dy,dz)) and ``coeff`` ([nst, N] float64: a CUDA tensor, or a
    host numpy array copied during the call)."""
    st = _capi.cs_stencil()
    st.dim = dim
    nn = list(n) + [1] * (3 - len(n))
    for d in range(3):
        st.n[d] = int(nn[d])
    st.nst = len(offsets)
    for s, o in enumerate(offsets):
        for d in range(3):
            st.off[s][d] = int(o[d])
    keep = coeff
    if isinstance(coeff, np.ndarray):
        keep = np.ascontiguousarray(coeff, dtype=np.float64)
        st.coeff = keep.ctypes.data_as(C.c_void_p)
        st.coeff_on_host = 1
    else:
        st.coeff = _dev_ptr(coeff, name="coeff").value
        st.coeff_on_host = 0
    st.periodic = int(bool(periodic))
    opts = _capi.cs_hierarchy_opts(coarse_max, max_levels, block, int(not reuse))
    out = C.c_void_p()
    _capi.check(_capi.lib().cs_setup_hierarchy(C.byref(st), C.byref(opts), _stream(stream), C.byref(out)),
                "cs_setup_hierarchy")
    del keep
    return Hierarchy(out.value, dim)


def setup_cascade(h: Hierarchy, kind="additive", nu=3, prescale=True, alpha=0, lowp=False, reuse=True, model=None,
                  model_tol=0.05, setup_precision="fp64", sketch=0, sketch_seed=0, sketch_exact_first=False,
                  stream=None):
    """Build the cascade; ``lowp``: False, True (FP32 copies for FP32
    cycles) or 2 (FP32 and BF16 copies); ``model`` (an ``MLP``) predicts the
    finest level's Lambda blocks, kept per block when its level-1 Frobenius
    objective is within ``model_tol`` of the exact one; ``setup_precision``
    "fp32" forms the setup's residual and propagator rows (or the sketch
    vectors) in FP32; ``sketch`` > 0 builds the sketched cascade with that
    many Rademacher columns from ``sketch_seed``."""
    k = _capi.CS_MULTIPLICATIVE if kind == "multiplicative" else _capi.CS_ADDITIVE
    opts = _capi.cs_cascade_opts(k, nu, int(prescale), alpha, int(lowp), int(not reuse),
                                 C.c_void_p(model.ptr if model is not None else None), float(model_tol),
                                 _capi.CS_FP32 if setup_precision == "fp32" else _capi.CS_FP64, int(sketch),
                                 int(bool(sketch_exact_first)), int(sketch_seed) & 0xFFFFFFFFFFFFFFFF)
    out = C.c_void_p()
    _capi.check(_capi.lib().cs_setup_cascade(h.ptr, C.byref(opts), _stream(stream), C.byref(out)),
                "cs_setup_cascade")
    c = Cascade(out.value, h, kind, nu, lowp)
    c.model = model
    return c


def learned_status(c):
    """(used, ratio): 1 predicted blocks in use / 0 exact fallback / -1 no
    model; level-1 Frobenius objective of the prediction over the exact one."""
    used, ratio = C.c_int(0), C.c_double(0.0)
    _capi.check(_capi.lib().cs_learned_status(c.ptr, C.byref(used), C.byref(ratio)), "cs_learned_status")
    return int(used.value), float(ratio.value)


def learned_stats(c):
    """Per-block detail of the learned setup (``cs_learned_stats``)."""
    nb, nf, npred = C.c_int64(), C.c_int64(), C.c_int64()
    rp, ru = C.c_double(), C.c_double()
    _capi.check(_capi.lib().cs_learned_stats(c.ptr, C.byref(nb), C.byref(nf), C.byref(npred), C.byref(rp),
                                             C.byref(ru)), "cs_learned_stats")
    return {"blocks": nb.value, "full_blocks": nf.value, "predicted_blocks": npred.value,
            "ratio_predicted": rp.value, "ratio_used": ru.value}


class MLP:
    """The learned-setup network (in -> hid -> hid -> out, ReLU; BF16 weights
    with FP32 accumulation), trained by the library's own kernels."""

    def __init__(self, nin, nhid, nout, max_batch=32768, seed=0):
        out = C.c_void_p()
        _capi.check(_capi.lib().cs_mlp_create(nin, nhid, nout, max_batch, seed, C.byref(out)), "cs_mlp_create")
        self._p = out.value
        self.nin, self.nhid, self.nout, self.max_batch = nin, nhid, nout, max_batch
        self.nparam = int(_capi.lib().cs_mlp_nparam(self._p))

    @property
    def ptr(self):
        return self._p

    def __del__(self):
        if getattr(self, "_p", None) and _capi._lib is not None:
            _capi._lib.cs_mlp_destroy(self._p)
            self._p = None

    def get_params(self):
        out = np.zeros(self.nparam, dtype=np.float32)
        _capi.check(_capi.lib().cs_mlp_get_params(self._p, out.ctypes.data_as(C.c_void_p)), "cs_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.nparam:
            raise ValueError(f"expected {self.nparam} parameters")
        _capi.check(_capi.lib().cs_mlp_set_params(self._p, p.ctypes.data_as(C.c_void_p)), "cs_mlp_set_params")

    def forward(self, X, Y=None, stream=None):
        torch = _torch()
        B = X.shape[0]
        if Y is None:
            Y = torch.empty((B, self.nout), dtype=torch.float32, device=X.device)
        _f32(X, B * self.nin, "X"), _f32(Y, B * self.nout, "Y")
        _capi.check(_capi.lib().cs_mlp_forward(self._p, B, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                                               _stream(stream)), "cs_mlp_forward")
        return Y

    def gradients(self, X, T, stream=None):
        B = X.shape[0]
        _f32(X, B * self.nin, "X"), _f32(T, B * self.nout, "T")
        g = np.zeros(self.nparam, dtype=np.float32)
        loss = C.c_float(0.0)
        _capi.check(_capi.lib().cs_mlp_gradients(self._p, B, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                                 g.ctypes.data_as(C.c_void_p), C.byref(loss), _stream(stream)),
                    "cs_mlp_gradients")
        return float(loss.value), g

    def train_step(self, X, T, lr, with_loss=True, stream=None):
        """One Adam step; returns the loss before it (the call then
        synchronises), or None with ``with_loss=False`` (no synchronisation)."""
        B = X.shape[0]
        _f32(X, B * self.nin, "X"), _f32(T, B * self.nout, "T")
        loss = C.c_float(0.0)
        _capi.check(_capi.lib().cs_mlp_train_step(self._p, B, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                                  float(lr), C.byref(loss) if with_loss else None, _stream(stream)),
                    "cs_mlp_train_step")
        return float(loss.value) if with_loss else None


def _f32(t, n, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} values, expected {n}")


def block_features(h, level=0, stream=None):
    """Features of every block of a 2D block level: [nblocks, bs^2 (bs+2)^2] (CUDA float32)."""
    torch = _torch()
    info = h.level_info(level)
    bs = info["block"]
    n = info["n"]
    nb = (-(-n[0] // bs)) * (-(-n[1] // bs))
    F = torch.empty((nb, bs * bs * (bs + 2) ** 2), dtype=torch.float32, device="cuda")
    _capi.check(_capi.lib().cs_block_features(h.ptr, level, C.c_void_p(F.data_ptr()), _stream(stream)),
                "cs_block_features")
    return F


def block_targets(c, level=0, stream=None):
    """Prescaled Lambda~ blocks of an exact additive cascade: [nblocks, nu bs^4] (CUDA float32)."""
    torch = _torch()
    info = c.hier.level_info(level)
    bs = info["block"]
    n = info["n"]
    nb = (-(-n[0] // bs)) * (-(-n[1] // bs))
    T = torch.empty((nb, c.nu * bs ** 4), dtype=torch.float32, device="cuda")
    _capi.check(_capi.lib().cs_block_targets(c.ptr, level, C.c_void_p(T.data_ptr()), _stream(stream)),
                "cs_block_targets")
    return T


def _cycle_opts(mu_pre, mu_post, order, precision):
    prec = {"fp64": _capi.CS_FP64, "fp32": _capi.CS_FP32, "bf16": _capi.CS_BF16}[precision]
    return _capi.cs_vcycle_opts(mu_pre, mu_post, _capi.CS_RF if order.upper() == "RF" else _capi.CS_FF, prec)


def vcycle(h, c, b, x, mu_pre=1, mu_post=1, order="RF", precision="fp64", stream=None):
    """x <- V(x, b) in place (Algorithm 1)."""
    N = h.N(0)
    o = _cycle_opts(mu_pre, mu_post, order, precision)
    _capi.check(_capi.lib().cs_vcycle(h.ptr, c.ptr, C.byref(o), _dev_ptr(b, N, "b"), _dev_ptr(x, N, "x"),
                                      _stream(stream)), "cs_vcycle")


def smooth(h, c, level, b, x, reverse=False, stream=None):
    N = h.N(level)
    _capi.check(_capi.lib().cs_smooth(h.ptr, c.ptr, level, int(reverse), _dev_ptr(b, N, "b"), _dev_ptr(x, N, "x"),
                                      _stream(stream)), "cs_smooth")


def sweep(h, c, level, step, b, x, out, colour=-1, stream=None):
    """One cascade step (one kernel): out = x - Lambda_{step+1[,colour]} (A x - b).
    float64 tensors run the FP64 kernel, float32 tensors the FP32 one (lowp),
    bfloat16 tensors the BF16-storage one (lowp=2)."""
    torch = _torch()
    N = h.N(level)
    ts = (b, x, out)
    if any((not isinstance(t, torch.Tensor)) or (not t.is_cuda) or (not t.is_contiguous()) or t.numel() != N
           for t in ts):
        raise ValueError(f"b, x, out must be contiguous CUDA tensors of {N} values")
    if all(t.dtype == torch.float32 for t in ts):
        prec = _capi.CS_FP32
    elif all(t.dtype == torch.float64 for t in ts):
        prec = _capi.CS_FP64
    elif all(t.dtype == torch.bfloat16 for t in ts):
        prec = _capi.CS_BF16
    else:
        raise TypeError("b, x, out must all be float64, all float32 or all bfloat16")
    _capi.check(_capi.lib().cs_sweep(h.ptr, c.ptr, level, step, colour, prec, C.c_void_p(b.data_ptr()),
                                     C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), _stream(stream)),
                "cs_sweep")


NOALLOC_MAX_N = 1 << 21


def smooth_noalloc(dim, n, box, coeff, lam, nu, b, x, kind="additive", reverse=False, stream=None):
    """cs_smooth_noalloc: one cascade application on a caller-given operator
    (canonical stencil layout) and Lambda ([nu, N]) without any device
    allocation; the ping-pong vector comes from a fixed internal 16 MiB
    device array (N <= 2,097,152).  For callers that cannot allocate."""
    nn = list(n) + [1] * (3 - len(n))
    N = int(nn[0] * nn[1] * (nn[2] if dim == 3 else 1))
    nst = (27 if dim == 3 else 9) if box else 2 * dim + 1
    narr = (C.c_int * 3)(*[int(v) for v in nn])
    k = _capi.CS_MULTIPLICATIVE if kind == "multiplicative" else _capi.CS_ADDITIVE
    torch = _torch()
    for name, t in (("coeff", coeff), ("lam", lam), ("b", b), ("x", x)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on {t.device}, not on the current device cuda:{torch.cuda.current_device()}")
    _capi.check(_capi.lib().cs_smooth_noalloc(dim, narr, int(bool(box)), _dev_ptr(coeff, nst * N, "coeff"),
                                              _dev_ptr(lam, nu * N, "lam"), nu, k, int(bool(reverse)),
                                              _dev_ptr(b, N, "b"), _dev_ptr(x, N, "x"), _stream(stream)),
                "cs_smooth_noalloc")


def sweep_rhs(h, c, level, step, b, x, out, nrhs, colour=-1, transpose=False, stream=None):
    """One cascade step with nrhs right-hand sides (RHS-contiguous [N, nrhs]
    tensors, float64 or float32): out = x - Lambda^(T) (A x - b) block by block."""
    torch = _torch()
    N = h.N(level)
    ts = (b, x, out)
    if any((not isinstance(t, torch.Tensor)) or (not t.is_cuda) or (not t.is_contiguous()) or t.numel() != N * nrhs
           for t in ts):
        raise ValueError(f"b, x, out must be contiguous CUDA tensors of {N}x{nrhs} values")
    if all(t.dtype == torch.float32 for t in ts):
        prec = _capi.CS_FP32
    elif all(t.dtype == torch.float64 for t in ts):
        prec = _capi.CS_FP64
    else:
        raise TypeError("b, x, out must all be float64 or all float32")
    _capi.check(_capi.lib().cs_sweep_rhs(h.ptr, c.ptr, level, step, colour, int(bool(transpose)), prec, nrhs,
                                         C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                         C.c_void_p(out.data_ptr()), _stream(stream)), "cs_sweep_rhs")


def kernel_launches() -> int:
    """Kernel launches issued by the library in this process so far."""
    return int(_capi.lib().cs_kernel_launches())


def residual_restrict(h, level, b, x, rc, stream=None):
    N, Nc = h.N(level), h.N(level + 1)
    _capi.check(_capi.lib().cs_residual_restrict(h.ptr, level, _dev_ptr(b, N, "b"), _dev_ptr(x, N, "x"),
                                                 _dev_ptr(rc, Nc, "rc"), _stream(stream)), "cs_residual_restrict")


def prolong_correct(h, level, xc, x, stream=None):
    N, Nc = h.N(level), h.N(level + 1)
    _capi.check(_capi.lib().cs_prolong_correct(h.ptr, level, _dev_ptr(xc, Nc, "xc"), _dev_ptr(x, N, "x"),
                                               _stream(stream)), "cs_prolong_correct")


def _lowp_vectors(ts, sizes, what):
    torch = _torch()
    for t, n in zip(ts, sizes):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{what}: contiguous CUDA tensors of sizes {sizes} expected")
    if all(t.dtype == torch.float32 for t in ts):
        return _capi.CS_FP32
    if all(t.dtype == torch.bfloat16 for t in ts):
        return _capi.CS_BF16
    raise TypeError(f"{what}: all float32 or all bfloat16 tensors expected")


def residual_restrict_lowp(h, c, level, b, x, rc, stream=None):
    """rc = R (A x - b) with the FP32 (float32 tensors) or BF16-storage
    (bfloat16 tensors) kernels of a low-precision V-cycle."""
    N, Nc = h.N(level), h.N(level + 1)
    prec = _lowp_vectors((b, x, rc), (N, N, Nc), "residual_restrict_lowp")
    _capi.check(_capi.lib().cs_residual_restrict_lowp(h.ptr, c.ptr, level, prec, C.c_void_p(b.data_ptr()),
                                                      C.c_void_p(x.data_ptr()), C.c_void_p(rc.data_ptr()),
                                                      _stream(stream)), "cs_residual_restrict_lowp")


def prolong_correct_lowp(h, c, level, xc, x, stream=None):
    """x <- x - P xc with the FP32 / BF16-storage kernels (dtype of the tensors)."""
    N, Nc = h.N(level), h.N(level + 1)
    prec = _lowp_vectors((xc, x), (Nc, N), "prolong_correct_lowp")
    _capi.check(_capi.lib().cs_prolong_correct_lowp(h.ptr, c.ptr, level, prec, C.c_void_p(xc.data_ptr()),
                                                    C.c_void_p(x.data_ptr()), _stream(stream)),
                "cs_prolong_correct_lowp")


def coarse_solve(h, b, x, stream=None):
    N = h.N(h.nlevels - 1)
    _capi.check(_capi.lib().cs_coarse_solve(h.ptr, _dev_ptr(b, N, "b"), _dev_ptr(x, N, "x"), _stream(stream)),
                "cs_coarse_solve")


def residual(h, level, b, x, r, norm=False, stream=None):
    """r = b - A x on ``level``; returns ||r||_2 when norm=True."""
    N = h.N(level)
    nrm = C.c_double(0.0)
    _capi.check(_capi.lib().cs_residual(h.ptr, level, _dev_ptr(b, N, "b"), _dev_ptr(x, N, "x"), _dev_ptr(r, N, "r"),
                                        C.byref(nrm) if norm else None, _stream(stream)), "cs_residual")
    return float(nrm.value) if norm else None


_METHODS = {"stationary": _capi.CS_STATIONARY, "gmres": _capi.CS_GMRES, "refine": _capi.CS_REFINE,
            "gmres_right": _capi.CS_GMRES_RIGHT, "pcg": _capi.CS_PCG}


def solve(h, c, b, x, method="stationary", tol=1e-10, maxit=100, restart=30, mu_pre=1, mu_post=1, order="RF",
          precision="fp64", host_buffers=False, raise_on_error=True, stream=None) -> SolveInfo:
    """Solve A x = b from the initial x (in place).  With host_buffers=True,
    b and x are host float64 arrays (numpy or CPU tensors; pinned memory is
    fastest) and the host<->device copies happen inside the call."""
    N = h.N(0)
    hist = np.zeros(4 * maxit + 8)
    o = _capi.cs_solve_opts(_METHODS[method], restart, maxit, tol, _cycle_opts(mu_pre, mu_post, order, precision),
                            int(host_buffers), hist.ctypes.data_as(C.POINTER(C.c_double)), len(hist))
    if host_buffers:
        bp, xp = _host_ptr(b, N, "b"), _host_ptr(x, N, "x")
    else:
        bp, xp = _dev_ptr(b, N, "b"), _dev_ptr(x, N, "x")
    info = _capi.cs_solve_info()
    st = _capi.lib().cs_solve(h.ptr, c.ptr, C.byref(o), bp, xp, C.byref(info), _stream(stream))
    if raise_on_error and st not in (_capi.CS_OK,):
        _capi.check(st, "cs_solve")
    return SolveInfo(st, info.iterations, bool(info.converged), info.final_rel_residual, hist[: info.nhist].copy())


def _stencil_struct(dim, n, offsets, coeff, periodic=False):
    """cs_stencil for (dim, n, offsets, coeff); returns (struct, keep-alive)."""
    st = _capi.cs_stencil()
    st.dim = dim
    nn = list(n) + [1] * (3 - len(n))
    for d in range(3):
        st.n[d] = int(nn[d])
    st.nst = len(offsets)
    for s_, o in enumerate(offsets):
        for d in range(3):
            st.off[s_][d] = int(o[d])
    keep = coeff
    if isinstance(coeff, np.ndarray):
        keep = np.ascontiguousarray(coeff, dtype=np.float64)
        st.coeff = keep.ctypes.data_as(C.c_void_p)
        st.coeff_on_host = 1
    else:
        st.coeff = _dev_ptr(coeff, name="coeff").value
        st.coeff_on_host = 0
    st.periodic = int(bool(periodic))
    return st, keep


def setup_many(problems, kind="multiplicative", nu=3, lowp=True, coarse_max=4, block=1, reuse=True, nthreads=0,
               stream=None):
    """Hierarchies and cascades of many independent problems, set up
    concurrently (``cs_setup_many``).  ``problems``: objects with ``dim``,
    ``n``, ``offsets``, ``coeff`` (host numpy or CUDA tensors) and optionally
    ``periodic``.  Returns (hierarchies, cascades)."""
    probs = list(problems)
    n = len(probs)
    arr = (_capi.cs_stencil * n)()
    keep = []
    for k, A in enumerate(probs):
        st, kp = _stencil_struct(A.dim, A.n, A.offsets, A.coeff, getattr(A, "periodic", False))
        arr[k] = st
        keep.append(kp)
    ho = _capi.cs_hierarchy_opts(coarse_max, 0, block, int(not reuse))
    k = _capi.CS_MULTIPLICATIVE if kind == "multiplicative" else _capi.CS_ADDITIVE
    co = _capi.cs_cascade_opts(k, nu, 1, 0, int(lowp), int(not reuse), C.c_void_p(None), 0.05, _capi.CS_FP64)
    hp = (C.c_void_p * n)()
    cp = (C.c_void_p * n)()
    _capi.check(_capi.lib().cs_setup_many(n, arr, C.byref(ho), C.byref(co), int(nthreads), _stream(stream), hp, cp),
                "cs_setup_many")
    del keep
    hs = [Hierarchy(hp[i], probs[i].dim) for i in range(n)]
    cs = [Cascade(cp[i], hs[i], kind, nu, lowp) for i in range(n)]
    return hs, cs


_BATCH_METHODS = {"refine": _capi.CS_REFINE, "gmres": _capi.CS_GMRES, "gmres_right": _capi.CS_GMRES_RIGHT}


class Batch:
    """A planned batched solve over existing (hierarchy, cascade) pairs
    (``cs_batch_create``); ``solve`` runs one persistent cooperative launch.
    Vectors of problem p are CUDA float64 tensors of N_p * nrhs[p] values,
    right-hand sides contiguous per node."""

    def __init__(self, hs, cs, nrhs, precision="fp32", order="RF", mu_pre=1, mu_post=1, autotune=False, threads=0,
                 tiles_per_cta=0, method="refine", restart=30, stream=None):
        self.hs, self.cs = list(hs), list(cs)
        self.nprob = len(self.hs)
        self.nrhs = [int(m) for m in nrhs]
        self.N = [h.N(0) for h in self.hs]
        o = _capi.cs_batch_opts(_capi.CS_FP32 if precision == "fp32" else _capi.CS_FP64,
                                _capi.CS_RF if order == "RF" else _capi.CS_FF, mu_pre, mu_post, int(autotune),
                                threads, tiles_per_cta, _BATCH_METHODS[method], restart)
        hp = (C.c_void_p * self.nprob)(*[h.ptr for h in self.hs])
        cp = (C.c_void_p * self.nprob)(*[c.ptr for c in self.cs])
        mp = (C.c_int * self.nprob)(*self.nrhs)
        out = C.c_void_p()
        _capi.check(_capi.lib().cs_batch_create(self.nprob, hp, cp, mp, C.byref(o), _stream(stream), C.byref(out)),
                    "cs_batch_create")
        self._p = out.value

    def config(self):
        t, tn, ct, nt = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        buf = (_capi.cs_batch_tune * 64)()
        _capi.check(_capi.lib().cs_batch_config(self._p, C.byref(t), C.byref(tn), C.byref(ct), buf, 64,
                                                C.byref(nt)), "cs_batch_config")
        return {"threads": t.value, "tiles_per_cta": tn.value, "ctas": ct.value,
                "tuned": [(buf[i].threads, buf[i].tiles_per_cta, buf[i].ms) for i in range(min(nt.value, 64))]}

    def set_config(self, threads, tiles_per_cta, stream=None):
        _capi.check(_capi.lib().cs_batch_set_config(self._p, threads, tiles_per_cta, _stream(stream)),
                    "cs_batch_set_config")

    def nbytes(self):
        return int(_capi.lib().cs_batch_bytes(self._p))

    def solve(self, bs, xs, tol=1e-10, maxit=100, raise_on_error=True, stream=None):
        """Solve every problem in place from its x; returns a list of SolveInfo."""
        if len(bs) != self.nprob or len(xs) != self.nprob:
            raise ValueError("one b and one x per problem")
        bp = (C.c_void_p * self.nprob)(*[_dev_ptr(b, self.N[i] * self.nrhs[i], f"b[{i}]").value
                                         for i, b in enumerate(bs)])
        xp = (C.c_void_p * self.nprob)(*[_dev_ptr(x, self.N[i] * self.nrhs[i], f"x[{i}]").value
                                         for i, x in enumerate(xs)])
        infos = (_capi.cs_solve_info * self.nprob)()
        st = _capi.lib().cs_batch_solve(self._p, bp, xp, float(tol), int(maxit), infos, _stream(stream))
        if raise_on_error and st != _capi.CS_OK:
            _capi.check(st, "cs_batch_solve")
        return [SolveInfo(st, infos[i].iterations, bool(infos[i].converged), infos[i].final_rel_residual,
                          np.zeros(0)) for i in range(self.nprob)]

    def __del__(self):
        if getattr(self, "_p", None) and _capi._lib is not None:
            _capi._lib.cs_batch_destroy(self._p)
            self._p = None


def solve_batched(hs, cs, bs, xs, nrhs, tol=1e-10, maxit=100, mu_pre=1, mu_post=1, order="RF", precision="fp32",
                  method="refine", restart=30, raise_on_error=True, stream=None):
    """One-shot batched solve (``cs_solve_batched``: plan without autotuning,
    solve, release)."""
    n = len(hs)
    o = _capi.cs_solve_opts(_BATCH_METHODS[method], restart, maxit, tol,
                            _cycle_opts(mu_pre, mu_post, order, precision), 0, None, 0)
    hp = (C.c_void_p * n)(*[h.ptr for h in hs])
    cp = (C.c_void_p * n)(*[c.ptr for c in cs])
    mp = (C.c_int * n)(*[int(m) for m in nrhs])
    bp = (C.c_void_p * n)(*[_dev_ptr(b, hs[i].N(0) * int(nrhs[i]), f"b[{i}]").value for i, b in enumerate(bs)])
    xp = (C.c_void_p * n)(*[_dev_ptr(x, hs[i].N(0) * int(nrhs[i]), f"x[{i}]").value for i, x in enumerate(xs)])
    infos = (_capi.cs_solve_info * n)()
    st = _capi.lib().cs_solve_batched(n, hp, cp, C.byref(o), bp, xp, mp, infos, _stream(stream))
    if raise_on_error and st != _capi.CS_OK:
        _capi.check(st, "cs_solve_batched")
    return [SolveInfo(st, infos[i].iterations, bool(infos[i].converged), infos[i].final_rel_residual, np.zeros(0))
            for i in range(n)]


def _host_ptr(a, n, name):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != n:
            raise TypeError(f"{name} must be a contiguous float64 array of {n} values")
        return a.ctypes.data_as(C.c_void_p)
    torch = _torch()
    if isinstance(a, torch.Tensor) and not a.is_cuda:
        if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n:
            raise TypeError(f"{name} must be a contiguous float64 tensor of {n} values")
        return C.c_void_p(a.data_ptr())
    raise TypeError(f"{name} must be a host array")


def query_level(h, level):
    return h.level_info(level)


def export_operator(h, level):
    """(offsets, coeff [nst, N]) of ``level`` as host arrays."""
    info = h.level_info(level)
    out = np.zeros((info["nst"], info["N"]))
    _capi.check(_capi.lib().cs_export_operator(h.ptr, level, out.ctypes.data_as(C.c_void_p)), "cs_export_operator")
    return info["offsets"], out


def export_colours(h, level):
    out = np.zeros(h.N(level), dtype=np.int8)
    _capi.check(_capi.lib().cs_export_colours(h.ptr, level, out.ctypes.data_as(C.c_void_p)), "cs_export_colours")
    return out


def export_lambda(c, level):
    out = np.zeros((c.nu, c.hier.level_info(level)["lamsize"]))
    _capi.check(_capi.lib().cs_export_lambda(c.ptr, level, out.ctypes.data_as(C.c_void_p)), "cs_export_lambda")
    return out


# ------------------------------------------------ general sparse operators
def _csr_struct(M, keep):
    """cs_csr of a scipy CSR matrix (host arrays, kept alive in `keep`)."""
    M = M.tocsr()
    M.sort_indices()
    rp = np.ascontiguousarray(M.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(M.indices, dtype=np.int32)
    v = np.ascontiguousarray(M.data, dtype=np.float64)
    keep += [rp, ci, v]
    return _capi.cs_csr(M.shape[0], M.shape[1], rp.ctypes.data, ci.ctypes.data, v.ctypes.data, 1)


class GHierarchy:
    """Handle of a general sparse hierarchy (``cs_gsetup_hierarchy``)."""

    def __init__(self, ptr):
        self._p = ptr
        self.nlevels = _capi.lib().cs_gnlevels(ptr)

    @property
    def ptr(self):
        return C.c_void_p(self._p)

    def level(self, l):
        n, nb, nc = C.c_int(), C.c_int(), C.c_int()
        nnz = C.c_int64()
        _capi.check(_capi.lib().cs_gquery_level(self._p, l, C.byref(n), C.byref(nnz), C.byref(nb), C.byref(nc)),
                    "cs_gquery_level")
        return {"N": n.value, "nnz": nnz.value, "nblocks": nb.value, "ncolours": nc.value}

    def N(self, l):
        return self.level(l)["N"]

    def operator(self, l):
        """(rowptr, col, val) of the level's operator (host arrays)."""
        q = self.level(l)
        rp = np.zeros(q["N"] + 1, dtype=np.int64)
        ci = np.zeros(max(q["nnz"], 1), dtype=np.int32)
        v = np.zeros(max(q["nnz"], 1))
        _capi.check(_capi.lib().cs_gexport_operator(self._p, l, rp.ctypes.data, ci.ctypes.data, v.ctypes.data),
                    "cs_gexport_operator")
        return rp, ci[: q["nnz"]], v[: q["nnz"]]

    def colours(self, l):
        out = np.zeros(self.level(l)["nblocks"], dtype=np.int32)
        _capi.check(_capi.lib().cs_gexport_colours(self._p, l, out.ctypes.data), "cs_gexport_colours")
        return out

    def blocks(self, l):
        q = self.level(l)
        bptr = np.zeros(q["nblocks"] + 1, dtype=np.int32)
        _capi.check(_capi.lib().cs_gexport_blocks(self._p, l, bptr.ctypes.data, None), "cs_gexport_blocks")
        bidx = np.zeros(max(int(bptr[-1]), 1), dtype=np.int32)
        _capi.check(_capi.lib().cs_gexport_blocks(self._p, l, bptr.ctypes.data, bidx.ctypes.data), "cs_gexport_blocks")
        return bptr, bidx[: bptr[-1]]

    def __del__(self):
        if getattr(self, "_p", None) and _capi._lib is not None:
            _capi._lib.cs_gdestroy_hierarchy(self._p)
            self._p = None


class GCascade:
    def __init__(self, ptr, h, kind, nu):
        self._p, self.h, self.kind, self.nu = ptr, h, kind, nu

    @property
    def ptr(self):
        return C.c_void_p(self._p)

    def __del__(self):
        if getattr(self, "_p", None) and _capi._lib is not None:
            _capi._lib.cs_gdestroy_cascade(self._p)
            self._p = None


def gsetup_hierarchy(A, Ps, rscale=1.0, blocks=None, seed=0, fields=None, stream=None):
    """General sparse hierarchy: A (scipy sparse, N0 x N0), interpolations
    Ps (scipy sparse, N_l x N_{l+1}), Galerkin coarse operators
    rscale P^T A P; blocks: (bptr, bidx) of level 0 or a list of such pairs
    (or None) per level, point blocks elsewhere; the greedy colouring's
    priority seed; fields (0 velocity / scalar, 1 pressure) of the finest
    unknowns for Stokes prescaling."""
    keep = []
    a = _csr_struct(A, keep)
    ps = (_capi.cs_csr * max(len(Ps), 1))(*[_csr_struct(P, keep) for P in Ps])
    nlev = len(Ps) + 1
    per = [None] * nlev
    if blocks is not None:
        lst = blocks if isinstance(blocks, list) else [blocks]
        per[:len(lst)] = lst
    nbl = (C.c_int * nlev)()
    bpp = (C.c_void_p * nlev)()
    bip = (C.c_void_p * nlev)()
    for l, bl in enumerate(per):
        if bl is None:
            continue
        bp = np.ascontiguousarray(bl[0], dtype=np.int32)
        bi = np.ascontiguousarray(bl[1], dtype=np.int32)
        keep += [bp, bi]
        nbl[l], bpp[l], bip[l] = len(bp) - 1, bp.ctypes.data, bi.ctypes.data
    fp = None
    if fields is not None:
        f = np.ascontiguousarray(fields, dtype=np.int32)
        keep.append(f)
        fp = f.ctypes.data
    out = C.c_void_p()
    _capi.check(_capi.lib().cs_gsetup_hierarchy(C.byref(a), len(Ps), ps, float(rscale), C.cast(nbl, C.c_void_p),
                                                C.cast(bpp, C.c_void_p), C.cast(bip, C.c_void_p), fp,
                                                int(seed) & 0xFFFFFFFFFFFFFFFF, _stream(stream), C.byref(out)),
                "cs_gsetup_hierarchy")
    return GHierarchy(out.value)


def gsetup_cascade(h, kind="additive", nu=3, prescale=True, spd=False, stream=None):
    """prescale: True / "elliptic", False / "none", or "stokes1", "stokes2",
    "stokesinf" (Stokes prescaling with q = 1, 2, infinity); spd: project
    every Lambda~ block between 0 and the block-Jacobi block, for PCG."""
    k = _capi.CS_MULTIPLICATIVE if kind == "multiplicative" else _capi.CS_ADDITIVE
    out = C.c_void_p()
    _capi.check(_capi.lib().cs_gsetup_cascade(h.ptr, k, nu, _capi.PRESCALE[prescale], int(bool(spd)),
                                              _stream(stream), C.byref(out)), "cs_gsetup_cascade")
    return GCascade(out.value, h, kind, nu)


def tc_gemm_bf16(A, B, stream=None):
    """C = A B^T (FP32) for CUDA bf16 tensors A [M, K] and B [N, K] (K a
    multiple of 8, contiguous) on the tcgen05 tensor cores."""
    import torch
    if A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16 or not A.is_cuda or not B.is_cuda:
        raise TypeError("tc_gemm_bf16 takes CUDA bfloat16 tensors")
    A, B = A.contiguous(), B.contiguous()
    M, K = A.shape
    N, K2 = B.shape
    if K != K2:
        raise ValueError("A and B need the same K")
    out = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _capi.check(_capi.lib().cs_tc_gemm_bf16(M, N, K, A.data_ptr(), B.data_ptr(), out.data_ptr(), _stream(stream)),
                "cs_tc_gemm_bf16")
    return out


def gexport_lambda(c, level):
    ls = int(_capi.lib().cs_glamsize(c.ptr, level))
    out = np.zeros((c.nu, ls))
    _capi.check(_capi.lib().cs_gexport_lambda(c.ptr, level, out.ctypes.data), "cs_gexport_lambda")
    return out


def gsweep(h, c, level, step, b, x, out, colour=-1, stream=None):
    N = h.N(level)
    _capi.check(_capi.lib().cs_gsweep(h.ptr, c.ptr, level, step, colour, _dev_ptr(b, N, "b"), _dev_ptr(x, N, "x"),
                                      _dev_ptr(out, N, "out"), _stream(stream)), "cs_gsweep")


def gsmooth(h, c, level, b, x, reverse=False, stream=None):
    N = h.N(level)
    _capi.check(_capi.lib().cs_gsmooth(h.ptr, c.ptr, level, int(reverse), _dev_ptr(b, N, "b"), _dev_ptr(x, N, "x"),
                                       _stream(stream)), "cs_gsmooth")


def gvcycle(h, c, b, x, mu_pre=1, mu_post=1, order="RF", stream=None):
    N = h.N(0)
    o = _cycle_opts(mu_pre, mu_post, order, "fp64")
    _capi.check(_capi.lib().cs_gvcycle(h.ptr, c.ptr, C.byref(o), _dev_ptr(b, N, "b"), _dev_ptr(x, N, "x"),
                                       _stream(stream)), "cs_gvcycle")


def gsolve(h, c, b, x, method="gmres_right", tol=1e-10, maxit=100, restart=30, mu_pre=1, mu_post=1, order="RF",
           raise_on_error=True, stream=None) -> SolveInfo:
    N = h.N(0)
    hist = np.zeros(4 * maxit + 8)
    o = _capi.cs_solve_opts(_METHODS[method], restart, maxit, tol, _cycle_opts(mu_pre, mu_post, order, "fp64"), 0,
                            hist.ctypes.data_as(C.POINTER(C.c_double)), len(hist))
    info = _capi.cs_solve_info()
    st = _capi.lib().cs_gsolve(h.ptr, c.ptr, C.byref(o), _dev_ptr(b, N, "b"), _dev_ptr(x, N, "x"), C.byref(info),
                               _stream(stream))
    if raise_on_error and st != _capi.CS_OK:
        _capi.check(st, "cs_gsolve")
    return SolveInfo(st, info.iterations, bool(info.converged), info.final_rel_residual, hist[: info.nhist].copy())
