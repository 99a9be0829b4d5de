"""Batched solve of many uneven problems (one persistent cooperative launch):
parity with the single-problem path and with the oracle, schedule
independence, the autotuner, edge cases."""
import numpy as np
import pytest

import oracle
import problems
from tests.gpu_util import rel_max, stencil_matvec

pytestmark = pytest.mark.gpu

# ragged sides (several tiles per problem and partial ones: a tile holds about
# one CTA of items at this batch size) and every
# class of right-hand-side count
SIDES = [17, 24, 33, 40, 47, 63]
NRHS = [1, 2, 3, 5, 8, 4]


def _batch(kind="multiplicative", nu=3):
    out = []
    for k, (n, m) in enumerate(zip(SIDES, NRHS)):
        A = problems.variable_poisson(problems.log_uniform_field(2, n, 4.0, 7000 + k))
        b = problems.uniform(8000 + k, A.N * m, -1.0, 1.0)
        out.append((A, m, b))
    return out


def _setup(probs, **kw):
    import paper_2606_12577_gb300 as cmg
    return cmg.setup_many([A for A, _, _ in probs], kind=kw.pop("kind", "multiplicative"), nu=kw.pop("nu", 3),
                          lowp=True, **kw)


def _vectors(probs):
    import torch
    bs = [torch.tensor(b, dtype=torch.float64, device="cuda") for _, _, b in probs]
    xs = [torch.zeros(A.N * m, dtype=torch.float64, device="cuda") for A, m, _ in probs]
    return bs, xs


def test_fixed_iterations_match_single_problem_path():
    """FP64 cycles, 3 iterations: every problem and right-hand side equals the
    single-problem refinement (x += V0(b - A x)) after 3 iterations."""
    import torch

    import paper_2606_12577_gb300 as cmg
    probs = _batch()
    hs, cs = _setup(probs)
    bt = cmg.Batch(hs, cs, NRHS, precision="fp64")
    bs, xs = _vectors(probs)
    infos = bt.solve(bs, xs, tol=1e-300, maxit=3, raise_on_error=False)
    assert all(i.iterations == 3 and not i.converged for i in infos)
    for p, (A, m, b) in enumerate(probs):
        X = xs[p].cpu().numpy().reshape(A.N, m)
        B = b.reshape(A.N, m)
        for r in range(m):
            x1 = torch.zeros(A.N, dtype=torch.float64, device="cuda")
            cmg.solve(hs[p], cs[p], torch.tensor(B[:, r].copy(), device="cuda"), x1, method="refine",
                      precision="fp64", tol=1e-300, maxit=3, raise_on_error=False)
            assert rel_max(X[:, r], x1.cpu().numpy()) <= 1e-12, (p, r)


def test_oracle_parity_small_problem():
    """One problem of the batch against the oracle's stationary V(1,1)-RF
    iteration (x <- V(x, b) equals x + V0(b - A x) for this linear cycle)."""
    import paper_2606_12577_gb300 as cmg
    probs = _batch()[:3]
    hs, cs = _setup(probs)
    bt = cmg.Batch(hs, cs, NRHS[:3], precision="fp64")
    bs, xs = _vectors(probs)
    bt.solve(bs, xs, tol=1e-300, maxit=4, raise_on_error=False)
    for p in (0, 2):
        A, m, b = probs[p]
        ho = oracle.Hierarchy(A)
        co = oracle.Cascade(ho, "multiplicative", nu=3)
        X = xs[p].cpu().numpy().reshape(A.N, m)
        for r in range(m):
            xo, _, _, _ = oracle.solve(ho, co, b.reshape(A.N, m)[:, r].copy(), method="stationary", tol=1e-300,
                                       maxit=4)
            assert rel_max(X[:, r], xo) <= 1e-12, (p, r)


def test_fp32_cycles_match_single_problem_path_to_convergence():
    """FP32 cycles inside FP64 refinement, run to 1e-10: each problem takes as
    many iterations as the single-problem path needs for its slowest
    right-hand side (+-1: the norms are summed in another order) and ends in
    the same state; every converged right-hand side meets ||b - A x|| / ||b||
    <= 1e-10 recomputed here from the stencil.  (Stationary V(1,1) cycles on
    these 10^6-contrast fields converge slowly; problems that need more than
    maxit iterations do so on both paths.)"""
    import torch

    import paper_2606_12577_gb300 as cmg
    probs = _batch()
    hs, cs = _setup(probs)
    bt = cmg.Batch(hs, cs, NRHS, precision="fp32")
    bs, xs = _vectors(probs)
    infos = bt.solve(bs, xs, tol=1e-10, maxit=100, raise_on_error=False)
    nconv = 0
    for p, (A, m, b) in enumerate(probs):
        X = xs[p].cpu().numpy().reshape(A.N, m)
        B = b.reshape(A.N, m)
        worst_it, all_conv = 0, True
        for r in range(m):
            x1 = torch.zeros(A.N, dtype=torch.float64, device="cuda")
            inf1 = cmg.solve(hs[p], cs[p], torch.tensor(B[:, r].copy(), device="cuda"), x1, method="refine",
                             precision="fp32", tol=1e-10, maxit=100, raise_on_error=False)
            worst_it = max(worst_it, inf1.iterations)
            all_conv &= inf1.converged
        assert infos[p].converged == all_conv
        assert abs(infos[p].iterations - worst_it) <= 1, (p, infos[p].iterations, worst_it)
        if infos[p].converged:
            nconv += 1
            for r in range(m):
                res = B[:, r] - stencil_matvec(A, X[:, r])
                assert np.linalg.norm(res) / np.linalg.norm(B[:, r]) <= 1.0001e-10
    assert nconv >= 2


def test_gmres_fixed_steps_match_single_problem_gmres():
    """FP64 cycles, GMRES(30) stopped after 5 Arnoldi steps: every problem and
    right-hand side equals the single-problem left-preconditioned GMRES after
    5 steps.  The two sum their dot products in different orders (tiles vs
    grid-stride blocks): relative differences of order sqrt(N) eps per inner
    product, amplified by the small least-squares problem, stay far below the
    1e-10 bound used here."""
    import torch

    import paper_2606_12577_gb300 as cmg
    probs = _batch()
    hs, cs = _setup(probs)
    bt = cmg.Batch(hs, cs, NRHS, precision="fp64", method="gmres", restart=30)
    bs, xs = _vectors(probs)
    infos = bt.solve(bs, xs, tol=1e-300, maxit=5, raise_on_error=False)
    assert all(i.iterations == 5 and not i.converged for i in infos)
    for p, (A, m, b) in enumerate(probs):
        X = xs[p].cpu().numpy().reshape(A.N, m)
        B = b.reshape(A.N, m)
        for r in range(m):
            x1 = torch.zeros(A.N, dtype=torch.float64, device="cuda")
            cmg.solve(hs[p], cs[p], torch.tensor(B[:, r].copy(), device="cuda"), x1, method="gmres",
                      precision="fp64", tol=1e-300, maxit=5, restart=30, raise_on_error=False)
            assert rel_max(X[:, r], x1.cpu().numpy()) <= 1e-10, (p, r)


def test_gmres_converges_on_the_batched_workload():
    """The first problems of the batched workload (correlation 8 cells,
    log-uniform coefficients on [1e-3, 1e3]; sides shrunk to <= 65), GMRES
    with FP64 cycles: every right-hand side reaches 1e-10 in the true
    residual.  A problem takes at least as many Arnoldi steps as the
    single-problem GMRES needs for its slowest right-hand side (-1: the norms
    are summed in another order); it can take more when one right-hand side
    has to restart while another is still extending (restarts happen per
    problem), but never more than twice as many."""
    import torch

    import paper_2606_12577_gb300 as cmg
    probs = [problems.batch_problem(k, nmin=20, nmax=65) for k in range(8)]
    hs, cs = _setup(probs)
    bt = cmg.Batch(hs, cs, [m for _, m, _ in probs], precision="fp64", method="gmres")
    bs = [torch.tensor(b, dtype=torch.float64, device="cuda") for _, _, b in probs]
    xs = [torch.zeros_like(b) for b in bs]
    infos = bt.solve(bs, xs, tol=1e-10, maxit=200)
    for p, (A, m, b) in enumerate(probs):
        assert infos[p].converged
        X = xs[p].cpu().numpy().reshape(A.N, m)
        B = b.reshape(A.N, m)
        worst = 0
        for r in range(m):
            res = B[:, r] - stencil_matvec(A, X[:, r])
            assert np.linalg.norm(res) / np.linalg.norm(B[:, r]) <= 1.0001e-10
            x1 = torch.zeros(A.N, dtype=torch.float64, device="cuda")
            worst = max(worst, cmg.solve(hs[p], cs[p], torch.tensor(B[:, r].copy(), device="cuda"), x1,
                                         method="gmres", precision="fp64", tol=1e-10, maxit=200).iterations)
        assert worst - 1 <= infos[p].iterations <= 2 * worst + 1, (p, infos[p].iterations, worst)


def test_results_do_not_depend_on_the_schedule():
    """Tiles per CTA and CTA size change only how work is dealt out: x after
    a fixed number of iterations is bitwise the same."""
    import paper_2606_12577_gb300 as cmg
    probs = _batch()
    hs, cs = _setup(probs)
    bt = cmg.Batch(hs, cs, NRHS, precision="fp32")
    outs = []
    for threads, tile in ((128, 1), (512, 4), (256, 7), (64, 300)):
        bt.set_config(threads, tile)
        bs, xs = _vectors(probs)
        bt.solve(bs, xs, tol=1e-300, maxit=3, raise_on_error=False)
        outs.append([x.cpu().numpy() for x in xs])
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


def test_autotuner_picks_the_fastest_measured_candidate():
    import paper_2606_12577_gb300 as cmg
    probs = _batch()
    hs, cs = _setup(probs)
    bt = cmg.Batch(hs, cs, NRHS, precision="fp32", autotune=True, method="gmres")
    cfg = bt.config()
    assert len(cfg["tuned"]) >= 3
    best = min(cfg["tuned"], key=lambda t: t[2])
    assert (cfg["threads"], cfg["tiles_per_cta"]) == (best[0], best[1])
    assert cfg["ctas"] > 0
    bs, xs = _vectors(probs)
    assert all(i.converged for i in bt.solve(bs, xs, tol=1e-10))


def test_zero_rhs_and_one_shot_entry_point():
    """A problem with b = 0 returns x = 0 at once; cs_solve_batched (plan,
    solve, release) gives the planned solver's result."""
    import paper_2606_12577_gb300 as cmg
    probs = _batch()[:3]
    probs[1] = (probs[1][0], probs[1][1], np.zeros_like(probs[1][2]))
    hs, cs = _setup(probs)
    bs, xs = _vectors(probs)
    xs[1].fill_(3.0)
    infos = cmg.solve_batched(hs, cs, bs, xs, NRHS[:3], tol=1e-10, method="gmres")
    assert infos[1].converged and infos[1].iterations == 0
    assert float(xs[1].abs().max()) == 0.0
    bt = cmg.Batch(hs, cs, NRHS[:3], method="gmres")
    bs2, xs2 = _vectors(probs)
    bt.solve(bs2, xs2, tol=1e-10)
    for a, b in zip(xs, xs2):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_rejected_batches():
    import paper_2606_12577_gb300 as cmg
    from paper_2606_12577_gb300._capi import CS_ERR_ARG, CS_ERR_UNSUPPORTED
    probs = _batch()[:2]
    hs, cs = _setup(probs)
    with pytest.raises(cmg.CascadeError) as e:
        cmg.Batch(hs, cs, [1, 33])
    assert e.value.status == CS_ERR_ARG
    hs2, cs2 = _setup(probs, kind="additive")
    with pytest.raises(cmg.CascadeError) as e:  # mixed cascade kinds
        cmg.Batch([hs[0], hs2[1]], [cs[0], cs2[1]], [1, 1])
    assert e.value.status == CS_ERR_ARG
    hs3, cs3 = _setup(probs[:1], nu=2)
    with pytest.raises(cmg.CascadeError) as e:
        cmg.Batch([hs[0], hs3[0]], [cs[0], cs3[0]], [1, 1])
    assert e.value.status == CS_ERR_ARG
    h9, c9 = _setup(probs[:1], block=3)
    with pytest.raises(cmg.CascadeError) as e:
        cmg.Batch(h9, c9, [1])
    assert e.value.status == CS_ERR_UNSUPPORTED


def _interface(n, seed):
    """A small elliptic-interface problem (12 inclusions of radius 2..6 cells)."""
    mu = problems.inclusions_2d(n, 12, seed, rmin=2.0, rmax=6.0)
    return problems.variable_poisson(mu)


@pytest.mark.parametrize("kind,bs,m", [("additive", 1, 3), ("additive", 2, 32), ("multiplicative", 2, 8),
                                       ("additive", 2, 5)])
def test_additive_and_block_batches_match_single_problem_path(kind, bs, m):
    """Additive cascades (out-of-place steps, the iterate alternating between
    two buffers) and 2x2-node block cascades (block steps, red-black on
    blocks), with up to 32 right-hand sides: after 3 iterations with FP64
    cycles every problem and RHS equals the single-problem path within 1e-12,
    and with FP32 cycles bitwise."""
    import torch

    import paper_2606_12577_gb300 as cmg
    probs = []
    for k, n in enumerate((23, 36, 41)):
        A = _interface(n, 300 + k)
        probs.append((A, m, problems.uniform(400 + k, A.N * m, -1.0, 1.0)))
    hs, cs = cmg.setup_many([A for A, _, _ in probs], kind=kind, nu=3, lowp=True, block=bs)
    for prec in ("fp64", "fp32"):
        bt = cmg.Batch(hs, cs, [m] * len(probs), precision=prec)
        bs_, xs = _vectors(probs)
        infos = bt.solve(bs_, xs, tol=1e-300, maxit=3, raise_on_error=False)
        assert all(i.iterations == 3 for i in infos)
        for p, (A, _, b) in enumerate(probs):
            X = xs[p].cpu().numpy().reshape(A.N, m)
            B = b.reshape(A.N, m)
            for r in range(0, m, max(1, m // 4)):
                x1 = torch.zeros(A.N, dtype=torch.float64, device="cuda")
                cmg.solve(hs[p], cs[p], torch.tensor(B[:, r].copy(), device="cuda"), x1, method="refine",
                          precision=prec, tol=1e-300, maxit=3, raise_on_error=False)
                if prec == "fp64":
                    assert rel_max(X[:, r], x1.cpu().numpy()) <= 1e-12, (p, r)
                else:
                    assert np.array_equal(X[:, r], x1.cpu().numpy()), (p, r)


def test_block_gmres_with_32_rhs_converges():
    """2x2-node blocks, additive nu = 3, 32 RHS solved together by GMRES with
    FP32 cycles: every RHS reaches 1e-10 in the true residual."""
    import torch

    import paper_2606_12577_gb300 as cmg
    A = _interface(63, 77)
    m = 32
    B = problems.uniform(78, A.N * m, -1.0, 1.0)
    hs, cs = cmg.setup_many([A], kind="additive", nu=3, lowp=True, block=2)
    bt = cmg.Batch(hs, cs, [m], precision="fp32", method="gmres")
    b = torch.tensor(B, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    info = bt.solve([b], [x], tol=1e-10, maxit=300)[0]
    assert info.converged
    X = x.cpu().numpy().reshape(A.N, m)
    Bm = B.reshape(A.N, m)
    for r in range(m):
        res = Bm[:, r] - stencil_matvec(A, X[:, r])
        assert np.linalg.norm(res) / np.linalg.norm(Bm[:, r]) <= 1.0001e-10


def test_right_gmres_fixed_steps_match_single_problem_gmres():
    """FP64 cycles, right-preconditioned GMRES(30) stopped after 5 Arnoldi
    steps: every problem and right-hand side equals the single-problem
    right-preconditioned GMRES after 5 steps (classical Gram-Schmidt with
    reprojection against modified Gram-Schmidt: the same basis in exact
    arithmetic)."""
    import torch

    import paper_2606_12577_gb300 as cmg
    probs = _batch()
    hs, cs = _setup(probs)
    bt = cmg.Batch(hs, cs, NRHS, precision="fp64", method="gmres_right", restart=30)
    bs, xs = _vectors(probs)
    infos = bt.solve(bs, xs, tol=1e-300, maxit=5, raise_on_error=False)
    assert all(i.iterations == 5 and not i.converged for i in infos)
    for p, (A, m, b) in enumerate(probs):
        X = xs[p].cpu().numpy().reshape(A.N, m)
        B = b.reshape(A.N, m)
        for r in range(m):
            x1 = torch.zeros(A.N, dtype=torch.float64, device="cuda")
            cmg.solve(hs[p], cs[p], torch.tensor(B[:, r].copy(), device="cuda"), x1, method="gmres_right",
                      precision="fp64", tol=1e-300, maxit=5, restart=30, raise_on_error=False)
            assert rel_max(X[:, r], x1.cpu().numpy()) <= 1e-10, (p, r)


def test_right_gmres_batch_matches_oracle_iterations():
    """FP64 cycles: the batched right-preconditioned GMRES converges on every
    right-hand side of the batched workload's first problems (sides <= 129)
    in about the oracle's right-preconditioned GMRES step count (the batch
    restarts per problem, so a problem can take more steps than its slowest
    right-hand side alone, never more than twice as many)."""
    import torch

    import paper_2606_12577_gb300 as cmg
    probs = [problems.batch_problem(k, nmin=40, nmax=129) for k in range(6)]
    hs, cs = _setup(probs)
    bt = cmg.Batch(hs, cs, [m for _, m, _ in probs], precision="fp64", method="gmres_right")
    bs = [torch.tensor(b, dtype=torch.float64, device="cuda") for _, _, b in probs]
    xs = [torch.zeros_like(b) for b in bs]
    infos = bt.solve(bs, xs, tol=1e-10, maxit=300)
    for p, (A, m, b) in enumerate(probs):
        assert infos[p].converged
        X = xs[p].cpu().numpy().reshape(A.N, m)
        B = b.reshape(A.N, m)
        ho = oracle.Hierarchy(A)
        co = oracle.Cascade(ho, "multiplicative", nu=3)
        worst = 0
        for r in range(m):
            res = B[:, r] - stencil_matvec(A, X[:, r])
            assert np.linalg.norm(res) / np.linalg.norm(B[:, r]) <= 1.0001e-10
            _, ito, _, _ = oracle.solve(ho, co, B[:, r].copy(), method="gmres_right", tol=1e-10, maxit=300)
            assert ito > 0
            worst = max(worst, ito)
        assert worst - 1 <= infos[p].iterations <= 2 * worst + 1, (p, infos[p].iterations, worst)


@pytest.mark.parametrize("n,count", [(127, 60), (255, 200)])
def test_right_gmres_interface_32_rhs_fp32(n, count):
    """The elliptic interface family with 32 right-hand sides solved together
    (2x2-node blocks, additive nu = 3, FP32 cycles and Krylov vectors,
    right-preconditioned GMRES-IR): every right-hand side reaches 1e-10 in the
    FP64 true residual, at 255^2 where the left-preconditioned form
    stagnates (in the oracle as well)."""
    import torch

    import paper_2606_12577_gb300 as cmg
    A = problems.interface2d(n, count)
    m = 32
    B = problems.uniform(79, A.N * m, -1.0, 1.0)
    hs, cs = cmg.setup_many([A], kind="additive", nu=3, lowp=True, block=2)
    bt = cmg.Batch(hs, cs, [m], precision="fp32", method="gmres_right")
    b = torch.tensor(B, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    info = bt.solve([b], [x], tol=1e-10, maxit=300)[0]
    assert info.converged
    X = x.cpu().numpy().reshape(A.N, m)
    Bm = B.reshape(A.N, m)
    for r in range(m):
        res = Bm[:, r] - stencil_matvec(A, X[:, r])
        assert np.linalg.norm(res) / np.linalg.norm(Bm[:, r]) <= 1.0001e-10


def test_long_restart_stages_coefficients_in_chunks():
    """Restart 100 with 32 right-hand sides (FP64): the projection
    coefficients no longer fit the kernel's shared buffer at once and are
    staged in chunks of slots; after 80 Arnoldi steps (one cycle) every
    right-hand side checked equals the single-problem right-preconditioned
    GMRES(100) after 80 steps."""
    import torch

    import paper_2606_12577_gb300 as cmg
    A, _, _ = problems.batch_problem(0, nmin=120, nmax=129)
    m = 32
    B = problems.uniform(91, A.N * m, -1.0, 1.0)
    hs, cs = _setup([(A, m, B)])
    bt = cmg.Batch(hs, cs, [m], precision="fp64", method="gmres_right", restart=100)
    b = torch.tensor(B, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    info = bt.solve([b], [x], tol=1e-300, maxit=80, raise_on_error=False)[0]
    assert info.iterations == 80 and not info.converged
    X = x.cpu().numpy().reshape(A.N, m)
    Bm = B.reshape(A.N, m)
    for r in (0, 13, 31):
        x1 = torch.zeros(A.N, dtype=torch.float64, device="cuda")
        cmg.solve(hs[0], cs[0], torch.tensor(Bm[:, r].copy(), device="cuda"), x1, method="gmres_right",
                  precision="fp64", tol=1e-300, maxit=80, restart=100, raise_on_error=False)
        assert rel_max(X[:, r], x1.cpu().numpy()) <= 1e-8, r
