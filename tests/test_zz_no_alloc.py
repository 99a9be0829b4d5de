"""cs_smooth_noalloc: the allocation-free variant of cs_smooth for callers
that cannot allocate device memory.  Its output must match cs_smooth (the
handle-based entry point, same kernels) to the 1e-12 relative tolerance the
parity tests use, on two calls in a row (the second call starts with the
first call's leftovers in the shared internal array).

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import problems
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = [
    # (problem, kind, level, reverse): level 0 is a 7-point STAR level, level 1 a 27-point BOX level
    ("v3d", "additive", 0, False),
    ("v3d", "additive", 1, True),
    ("v3d", "multiplicative", 0, True),
    ("v3d", "multiplicative", 1, False),
    ("c2d", "additive", 0, True),
    ("c2d", "multiplicative", 1, False),
]


def _problem(name):
    if name == "v3d":
        return problems.variable_poisson(problems.random_coefficients(3, 41, 19, -1.0, 1.0))
    return problems.variable_poisson(problems.log_uniform_field(2, 130, 8.0, 231, -2.0, 2.0))


@pytest.mark.parametrize("name,kind,level,reverse", CASES)
def test_noalloc_matches_cs_smooth(name, kind, level, reverse):
    import __graft_entry__ as g
    g.build()
    import paper_2606_12577_gb300 as cmg
    A = _problem(name)
    h = gu.gpu_hierarchy(A)
    nu = 3
    c = cmg.setup_cascade(h, kind, nu=nu)
    info = cmg.query_level(h, level)
    offs, coeff = cmg.export_operator(h, level)
    box = int(info["nst"] in (9, 27))
    lam = cmg.export_lambda(c, level)
    N = info["N"]
    coeff_d, lam_d = _dev(coeff), _dev(lam)
    b_d = _dev(problems.uniform(500 + level, N))
    for call in range(2):  # two calls in a row share the internal array
        x0 = problems.uniform(600 + 10 * level + call, N)
        x_ref = _dev(x0)
        cmg.smooth(h, c, level, b_d, x_ref, reverse=reverse)
        x_new = _dev(x0)
        cmg.smooth_noalloc(A.dim, info["n"], box, coeff_d, lam_d, nu, b_d, x_new, kind=kind, reverse=reverse)
        ref = _host(x_ref)
        got = _host(x_new)
        assert np.abs(got - ref).max() <= TOL * np.abs(ref).max(), f"call {call}"


def test_noalloc_rejects_oversize():
    import __graft_entry__ as g
    g.build()
    import paper_2606_12577_gb300 as cmg
    n = (130, 130, 130)  # 2,197,000 > 2,097,152
    N = n[0] * n[1] * n[2]
    z = _dev(np.zeros(1))
    import torch
    big = torch.zeros(7 * N, dtype=torch.float64, device="cuda")
    lam = torch.zeros(N, dtype=torch.float64, device="cuda")
    v = torch.zeros(N, dtype=torch.float64, device="cuda")
    with pytest.raises(cmg.CascadeError, match="CS_ERR_ARG"):
        cmg.smooth_noalloc(3, n, 0, big, lam, 1, v, v.clone())
    del z


def test_noalloc_rejects_grids_beyond_the_launch_limits():
    """N within the array's limit but a grid whose node-kernel launch would
    exceed the CTA grid limits (nz > 65535, or ny > 4 x 65535 in 2D) is
    rejected with CS_ERR_ARG before any launch."""
    import __graft_entry__ as g
    g.build()
    import torch

    import paper_2606_12577_gb300 as cmg
    for dim, n in ((3, (1, 1, 1 << 17)), (2, (1, 1 << 19))):
        N = 1 << 17 if dim == 3 else 1 << 19
        nst = 2 * dim + 1
        coeff = torch.zeros(nst * N, dtype=torch.float64, device="cuda")
        lam = torch.zeros(N, dtype=torch.float64, device="cuda")
        v = torch.zeros(N, dtype=torch.float64, device="cuda")
        with pytest.raises(cmg.CascadeError, match="launch limits"):
            cmg.smooth_noalloc(dim, n, 0, coeff, lam, 1, v, v.clone())


def test_noalloc_rejects_memory_of_another_device():
    """A vector that is not device memory of the current device (here host
    memory, passed through the C ABI directly) is rejected with CS_ERR_ARG
    before any launch; the binding rejects CPU tensors itself."""
    import ctypes

    import __graft_entry__ as g
    g.build()
    import torch

    import paper_2606_12577_gb300 as cmg
    from paper_2606_12577_gb300 import _capi
    n = (8, 8, 1)
    N = 64
    coeff = torch.zeros(5 * N, dtype=torch.float64, device="cuda")
    lam = torch.zeros(N, dtype=torch.float64, device="cuda")
    v = torch.zeros(N, dtype=torch.float64, device="cuda")
    host = np.zeros(N)
    narr = (ctypes.c_int * 3)(*n)
    st = _capi.lib().cs_smooth_noalloc(2, narr, 0, ctypes.c_void_p(coeff.data_ptr()),
                                       ctypes.c_void_p(lam.data_ptr()), 1, _capi.CS_ADDITIVE, 0,
                                       ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(v.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _capi.CS_ERR_ARG
    assert b"current device" in _capi.lib().cs_last_error() or b"not a CUDA device pointer" in \
        _capi.lib().cs_last_error()
    with pytest.raises(TypeError):
        cmg.smooth_noalloc(2, n, 0, coeff, lam, 1, torch.zeros(N, dtype=torch.float64), v)
