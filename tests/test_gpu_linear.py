"""GPU parity of the shared-kernel linear smoother (Sec. 6, eq. full-coarsening-smoother):
V-cycle solve histories, the standalone smoother and the transposed cycle, through the
C ABI against the FP64 oracle (oracle/linear.py).

Tolerance: the per-cycle relative residual within 1e-5 of the oracle's, the bar of every
other solve path here (FP32 cycle, float-float outer iterate and residual).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import linear as OL
from paper_2102_12071_gb300 import inputs
from paper_2102_12071_gb300 import solver as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2102_12071_gb300 import build

    build.build()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def lin_params(nsets, d, seed, scale=0.01):
    """Weighted Jacobi (omega/d) plus a small random chain: a convergent smoother whose
    five chained kernels all act."""
    rng = np.random.default_rng(seed)
    return np.stack([OL.jacobi_params(d) + scale * rng.standard_normal((6, 9)) for _ in range(nsets)]).astype(
        np.float32)


def _solve_both(problems, fields, params, b, cycles):
    """The GPU solve and the oracle's, each from its own operators: the oracle forms every
    coarse level as its FP64 Galerkin product of the level-0 field."""
    mg = S.MultigridSolver(problems, "cnn", torch.from_numpy(params).cuda(), net_arch="linear")
    bb = torch.from_numpy(np.stack(b).astype(np.float32)).cuda().contiguous()
    _, _, gh, cyc, _ = mg.solve(bb, rtol=0.0, max_cycles=cycles)
    out = []
    for p, st in enumerate(fields):
        om = OL.LinearMultigrid(st, [f32(q) for q in params])
        _, oh = om.solve(f32(b[p]), rtol=0.0, max_cycles=cycles)
        assert cyc[p] == cycles
        out.append((gh[p][: cycles + 1], oh))
    mg.close()
    return out


@pytest.mark.parametrize("n,cycles,nsets", [(7, 6, 1), (63, 40, 1), (255, 20, 3), (511, 8, 2), (1023, 4, 4)])
def test_linear_solve_history_matches_oracle(n, cycles, nsets):
    """n <= 63: whole solves in one CTA; above: batched level kernels, then the tail."""
    pe = [(0.05, 0.7), (0.01, 2.2)]
    problems = [S.rotated(n, e, t) for e, t in pe]
    fields = [O.const_field(n, f32(O.q1_rotated_stencil(e, t))) for e, t in pe]
    d = fields[0][4, n // 2, n // 2]
    params = lin_params(nsets, d, seed=n)
    b = [inputs.rhs_uniform(20 + p, n) for p in range(len(pe))]
    for gh, oh in _solve_both(problems, fields, params, b, cycles):
        rel = np.abs(gh - oh) / oh
        assert rel.max() <= 1e-5, rel.max()


@pytest.mark.parametrize("coef", ["sine1", "sine10", "grf"])
def test_linear_solve_per_point_field(coef):
    """Variable coefficients (per-point stencil fields) at 127^2: the paper's own problem of
    Sec. 6.3, -div((sin(kappa pi x y) + 1.1) grad u) = f with kappa = 1 and 10, and the
    unit-variance GRF coefficient of the benchmark, both on the 5-point cell-coefficient
    scheme.  One kernel set serves every point, so its Jacobi part is omega over the largest
    diagonal plus a small random chain.  The oracle builds its own FP64 Galerkin fields."""
    n = 127
    a = {"sine1": lambda: inputs.sine_cells(n, 1.0), "sine10": lambda: inputs.sine_cells(n, 10.0),
         "grf": lambda: inputs.grf_cells(12, n)}[coef]()
    st0 = O.varcoef5_field(n, f32(a))
    dmax = st0[4].max()
    params = lin_params(2, dmax, seed=5, scale=0.02 * (2.0 / 3.0) / dmax)
    problems = [S.varcoef5(n, torch.from_numpy(a).cuda())]
    b = [inputs.rhs_uniform(31, n)]
    for gh, oh in _solve_both(problems, [f32(st0)], params, b, 15):
        rel = np.abs(gh - oh) / oh
        assert rel.max() <= 1e-5, rel.max()


@pytest.mark.parametrize("n", [63, 255])
def test_linear_at_the_jacobi_point_solves_like_jacobi(n):
    eps, theta = 0.02, 1.0
    s = O.q1_rotated_stencil(eps, theta).astype(np.float32).reshape(9)
    params = OL.jacobi_params(float(s[4]))[None].astype(np.float32)
    b = torch.from_numpy(inputs.rhs_uniform(3, n)).cuda()[None].contiguous()
    lin = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(params).cuda(), net_arch="linear")
    jac = S.MultigridSolver([S.rotated(n, eps, theta)], "jacobi")
    _, _, hl, cl, _ = lin.solve(b, rtol=1e-8, max_cycles=3000)
    _, _, hj, cj, _ = jac.solve(b, rtol=1e-8, max_cycles=3000)
    assert abs(int(cl[0]) - int(cj[0])) <= 1
    k = min(cl[0], cj[0]) + 1
    assert np.max(np.abs(hl[0][:k] - hj[0][:k]) / hj[0][:k]) < 1e-5


def test_linear_standalone_smoother_matches_oracle():
    n, level = 255, 1
    eps, theta = 0.1, 0.3
    params = lin_params(2, O.q1_rotated_stencil(eps, theta).reshape(9)[4], seed=9)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(params).cuda(), net_arch="linear")
    nl = mg.sizes[level]
    st = mg.stencil_field(0, level).double().cpu().numpy()
    rng = np.random.default_rng(4)
    f = rng.standard_normal((nl, nl)).astype(np.float32)
    u = rng.standard_normal((nl, nl)).astype(np.float32)
    ug = torch.from_numpy(u).cuda()
    mg.smooth(0, level, torch.from_numpy(f).cuda(), ug, nsteps=2)
    uo = f32(u)
    for _ in range(2):
        uo = uo + OL.apply_H(f32(params[level]), f32(f) - O.apply(st, uo))
    np.testing.assert_allclose(ug.double().cpu().numpy(), uo, rtol=0, atol=2e-5 * np.abs(uo).max())


def test_transposed_linear_cycle_is_the_adjoint():
    """With every level's chain transposed, one V-cycle from zero applies M^T (the adjoint
    coarse solve of Algorithm 2's training objective)."""
    n = 127
    eps, theta = 0.05, 2.5
    params = torch.from_numpy(lin_params(3, O.q1_rotated_stencil(eps, theta).reshape(9)[4], seed=2)).cuda()
    M = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", params, net_arch="linear")
    MT = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", params, net_arch="linear", transpose=True)
    rng = np.random.default_rng(1)
    r, s = (torch.from_numpy(v.astype(np.float32)).cuda()[None].contiguous() for v in rng.standard_normal((2, n, n)))
    xr = torch.zeros_like(r)
    xs = torch.zeros_like(s)
    M.vcycle(r, xr)
    MT.vcycle(s, xs)
    lhs = float((xr.double() * s.double()).sum())
    rhs = float((r.double() * xs.double()).sum())
    assert math.isclose(lhs, rhs, rel_tol=1e-4), (lhs, rhs)


# ------------------------------------------------------------------ training
def _lin_batch(n, pe, nvec, seed, cycles=1, checkpoint=False):
    from paper_2102_12071_gb300 import train as T

    batch = T.TwoGridBatch([S.rotated(n, e, t) for e, t in pe], nvec, cycles=cycles, checkpoint=checkpoint,
                           net_arch="linear")
    z = np.random.default_rng(seed).standard_normal((len(pe), nvec, n, n)).astype(np.float32)
    return batch, z


@pytest.mark.parametrize("n,cycles,ckpt", [(15, 1, False), (31, 1, False), (15, 3, False), (15, 3, True)])
def test_linear_train_step_matches_oracle(n, cycles, ckpt):
    """Loss and gradient of the 54 weights (Sec. 3.2 objective, k cycles) against the oracle's
    analytic adjoint; checkpointing recomputes the cycle products and changes nothing."""
    pe = [(0.05, 0.7), (0.01, 2.0)]
    phi = lin_params(1, O.q1_rotated_stencil(*pe[0]).reshape(9)[4], seed=n, scale=0.05)[0]
    batch, z = _lin_batch(n, pe, 3, seed=1, cycles=cycles, checkpoint=ckpt)
    loss, grad = batch.loss_and_grad(torch.from_numpy(phi.reshape(-1)).cuda(), torch.from_numpy(z).cuda())
    lo, go = 0.0, np.zeros((6, 9))
    for b, (e, t) in enumerate(pe):
        st = O.const_field(n, f32(O.q1_rotated_stencil(e, t)))
        l, g = OL.loss_and_grad(st, f32(phi), f32(z[b]), cycles=cycles)
        lo += l / len(pe)
        go += g / len(pe)
    assert math.isclose(float(loss[0]), lo, rel_tol=2e-5), (float(loss[0]), lo)
    g = grad.double().cpu().numpy().reshape(6, 9)
    assert np.max(np.abs(g - go)) <= 1e-4 * np.max(np.abs(go)), np.max(np.abs(g - go)) / np.max(np.abs(go))


def test_linear_vcycle_coarse_train_step_matches_oracle():
    """Algorithm 2's objective: the coarse solve replaced by one V-cycle of the trained
    linear smoothers below, its adjoint by the cycle with transposed chains."""
    n = 31
    pe = [(0.02, 1.2), (0.3, 0.4)]
    d = O.q1_rotated_stencil(*pe[0]).reshape(9)[4]
    lower = lin_params(2, d, seed=3, scale=0.02)
    phi = lin_params(1, d, seed=4, scale=0.05)[0]
    batch, z = _lin_batch(n, pe, 2, seed=2)
    batch.attach_coarse(torch.from_numpy(lower.reshape(2, -1)).cuda())
    loss, grad = batch.loss_and_grad(torch.from_numpy(phi.reshape(-1)).cuda(), torch.from_numpy(z).cuda())
    coarse_fields = [f.double().cpu().numpy() for f in batch.coarse_fields()]
    lo, go = 0.0, np.zeros((6, 9))
    for b, (e, t) in enumerate(pe):
        st = O.const_field(n, f32(O.q1_rotated_stencil(e, t)))
        M = OL.coarse_vcycle(coarse_fields[b], [f32(q) for q in lower])
        MT = OL.coarse_vcycle(coarse_fields[b], [f32(q) for q in lower], transpose=True)
        l, g = OL.loss_and_grad(st, f32(phi), f32(z[b]), coarse=M, coarse_t=MT)
        lo += l / len(pe)
        go += g / len(pe)
    batch.close()
    assert math.isclose(float(loss[0]), lo, rel_tol=1e-4), (float(loss[0]), lo)
    g = grad.double().cpu().numpy().reshape(6, 9)
    assert np.max(np.abs(g - go)) <= 2e-4 * np.max(np.abs(go)), np.max(np.abs(g - go)) / np.max(np.abs(go))


def test_adaptively_trained_linear_smoother_gains_over_jacobi():
    """Sec. 6's alpha-CNN for one problem: per-level linear smoothers trained coarse to fine
    (Algorithm 2) on a 31^2 hierarchy, then used on every level of a 255^2 solve.  The
    objective falls on every level and the solve needs fewer cycles than weighted Jacobi."""
    from paper_2102_12071_gb300 import train as T

    eps, theta = 0.01, math.pi / 6
    at = T.AdaptiveTrainer(n_fine=31, per_size=1, nvec=64, steps_per_level=150, lr=3e-3, conv_bf16=False,
                           net_arch="linear", problem=(eps, theta))
    at.train()
    for n, h in at.losses.items():
        assert np.mean(h[-10:]) < 0.9 * np.mean(h[:10]), (n, h[:3], h[-3:])
    n = 255
    b = torch.from_numpy(inputs.rhs_uniform(5, n)).cuda()[None].contiguous()
    lin = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", at.hierarchy_params(n), net_arch="linear")
    jac = S.MultigridSolver([S.rotated(n, eps, theta)], "jacobi")
    _, _, _, cl, sl = lin.solve(b, rtol=1e-8, max_cycles=5000)
    _, _, _, cj, sj = jac.solve(b, rtol=1e-8, max_cycles=5000)
    assert sl == 0 and sj == 0
    assert cl[0] < cj[0], (cl, cj)


def test_fgmres_with_the_linear_smoother_matches_oracle():
    """Sec. 6.4's solver with the linear smoother's V-cycle as the preconditioner: iterations
    within two of the FP64 oracle's, first restart cycle's residual estimates within 1e-3,
    true residual of the float-float solution below rtol."""
    from paper_2102_12071_gb300 import binding as B

    n, eps, theta = 255, 0.01, math.pi / 4
    d = O.q1_rotated_stencil(eps, theta).reshape(9)[4]
    params = lin_params(3, d, seed=8, scale=0.01)
    b_np = inputs.rhs_uniform(inputs.SEED_RHS + 1600, n)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(params).cuda(), net_arch="linear")
    xh, xl, gh, its, st = S.fgmres(mg, torch.from_numpy(b_np).cuda()[None].contiguous(), restart=30, rtol=1e-6,
                                   max_iters=300)
    assert st == B.MG_OK
    st0 = O.const_field(n, f32(O.q1_rotated_stencil(eps, theta)))
    om = OL.LinearMultigrid(st0, [f32(q) for q in params])
    xo, oh, oits = O.fgmres(lambda v: O.apply(st0, v), lambda v: om.vcycle(v, np.zeros_like(v)), f32(b_np),
                            restart=30, rtol=1e-6, max_iters=300)
    assert abs(int(its[0]) - oits) <= 2, (int(its[0]), oits)
    k = min(int(its[0]), oits, 30) + 1
    assert np.max(np.abs(gh[0][:k] - oh[:k]) / oh[:k]) <= 1e-3
    x = xh[0].double().cpu().numpy() + xl[0].double().cpu().numpy()
    assert np.linalg.norm(f32(b_np) - O.apply(st0, x)) / np.linalg.norm(f32(b_np)) < 1e-6


def test_per_problem_linear_smoothers_batch_like_separate_contexts():
    """net_per_problem: each problem of one context smooths with its own group of per-level
    sets; the batched solve equals one context per problem (same kernels, same order)."""
    n = 255
    pe = [(0.01, math.pi / 12), (0.01, math.pi / 4), (0.2, 2.0)]
    groups = np.stack([lin_params(3, O.q1_rotated_stencil(e, t).reshape(9)[4], seed=40 + i)
                       for i, (e, t) in enumerate(pe)])
    b = torch.from_numpy(np.stack([inputs.rhs_uniform(60 + i, n) for i in range(len(pe))])).cuda().contiguous()
    mg = S.MultigridSolver([S.rotated(n, e, t) for e, t in pe], "cnn", torch.from_numpy(groups).cuda(),
                           net_arch="linear", per_problem=True)
    _, _, gh, gc, _ = mg.solve(b, rtol=1e-8, max_cycles=3000)
    for i, (e, t) in enumerate(pe):
        one = S.MultigridSolver([S.rotated(n, e, t)], "cnn", torch.from_numpy(groups[i]).cuda(), net_arch="linear")
        _, _, h1, c1, _ = one.solve(b[i:i + 1].contiguous(), rtol=1e-8, max_cycles=3000)
        assert int(gc[i]) == int(c1[0])
        k = int(c1[0]) + 1
        assert np.array_equal(gh[i][:k], h1[0][:k])


# ------------------------------------------------------------------ nu1, nu2 > 1
@pytest.mark.parametrize("n,nu1,nu2,cycles", [(63, 2, 2, 20), (255, 3, 2, 12), (255, 6, 6, 8), (1023, 6, 6, 3)])
def test_multistep_jacobi_matches_oracle(n, nu1, nu2, cycles):
    """Algorithm 1 with nu1 pre- and nu2 post-smoothing Jacobi steps (the paper's cost-equalised
    Jacobi takes six): batched level kernels above 63, the one-CTA tail below."""
    eps, theta = 0.01, math.pi / 3
    b = inputs.rhs_uniform(70, n)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], "jacobi", nu1=nu1, nu2=nu2)
    _, _, gh, cyc, _ = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=0.0, max_cycles=cycles)
    om = O.Multigrid(O.const_field(n, f32(O.q1_rotated_stencil(eps, theta))), nu1=nu1, nu2=nu2)
    _, oh = om.solve(f32(b), rtol=0.0, max_cycles=cycles)
    rel = np.abs(gh[0][: cycles + 1] - oh) / oh
    assert rel.max() <= 1e-5, rel.max()


def test_multistep_linear_smoother_matches_oracle():
    n, cycles = 255, 10
    pe = [(0.05, 0.7), (0.01, 2.2)]
    fields = [O.const_field(n, f32(O.q1_rotated_stencil(e, t))) for e, t in pe]
    params = lin_params(3, fields[0][4, n // 2, n // 2], seed=77)
    mg = S.MultigridSolver([S.rotated(n, e, t) for e, t in pe], "cnn", torch.from_numpy(params).cuda(),
                           net_arch="linear", nu1=2, nu2=3)
    b = [inputs.rhs_uniform(80 + p, n) for p in range(2)]
    _, _, gh, _, _ = mg.solve(torch.from_numpy(np.stack(b).astype(np.float32)).cuda().contiguous(), rtol=0.0,
                              max_cycles=cycles)
    for p in range(2):
        _, oh = OL.LinearMultigrid(fields[p], [f32(q) for q in params], nu1=2, nu2=3).solve(f32(b[p]), rtol=0.0,
                                                                                            max_cycles=cycles)
        rel = np.abs(gh[p][: cycles + 1] - oh) / oh
        assert rel.max() <= 1e-5, rel.max()


def test_multistep_smoothing_needs_jacobi_or_the_linear_smoother():
    from paper_2102_12071_gb300 import binding as B

    p = torch.zeros(1260, device="cuda")
    with pytest.raises(B.MGError) as ei:  # refused while sizing the workspace
        S.MultigridSolver([S.rotated(255, 0.1, 0.3)], "cnn", p, nu1=2)
    assert "need the Jacobi or the linear smoother" in str(ei.value)
