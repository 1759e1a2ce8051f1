"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Tolerances: per-cycle relative residual within 1e-5 relative; asymptotic convergence
factor within 1e-3; element-wise FP32 results within a few ulps of the stencil width.
"""
import math
import time

import numpy as np
import pytest
import torch

import oracle as O
from paper_2102_12071_gb300 import binding as B
from paper_2102_12071_gb300 import inputs
from paper_2102_12071_gb300 import solver as S

pytestmark = pytest.mark.gpu

HIST_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2102_12071_gb300 import build

    build.build()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def oracle_rotated(n, eps, theta):
    return O.const_field(n, f32(O.q1_rotated_stencil(eps, theta)))


def _cmp_hist(gh, oh, tol=HIST_RTOL, upto=None):
    k = min(len(oh), np.count_nonzero(~np.isnan(gh)))
    if upto:
        k = min(k, upto)
    rel = np.abs(gh[:k] - oh[:k]) / oh[:k]
    assert rel.max() <= tol, (rel.max(), int(rel.argmax()), gh[:k][rel.argmax()], oh[:k][rel.argmax()])
    return k


def test_hierarchy_stencils_match_oracle():
    n = 255
    eps, theta = 0.01, math.pi / 6
    mg = S.MultigridSolver([S.rotated(n, eps, theta)])
    om = O.Multigrid(oracle_rotated(n, eps, theta))
    assert mg.sizes == [om.n(l) for l in range(om.levels)] == [255, 127, 63, 31, 15, 7, 3]
    for l in range(mg.levels):
        g = mg.stencil_field(0, l).cpu().double().numpy()
        if l == 0:
            np.testing.assert_array_equal(g, f32(om.field(l)))
        else:
            # the library carries the constant-stencil Galerkin recursion in float-float and
            # rounds each level once for storage: within one ulp of the oracle's FP64 chain
            np.testing.assert_allclose(g, om.field(l), rtol=0, atol=2.0 ** -23 * np.abs(om.field(l)).max())
        if l < mg.levels - 1:
            np.testing.assert_allclose(mg.kernels(0, l).cpu().double().numpy(), O.jacobi_kernels(om.field(l)),
                                       rtol=3 * 2.0 ** -24, atol=0)


@pytest.mark.parametrize("n", [3, 7, 63])
def test_c1_jacobi_solve_matches_oracle(n):
    """63 x 63 (C1): eps = 0.01, theta = pi/6, V(1,1) Jacobi, 5 levels, rhs U[-1,1] seed 0."""
    eps, theta = 0.01, math.pi / 6
    b = inputs.rhs_uniform(0, n)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)])
    x_hi, x_lo, gh, cyc, st = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=1e-8, max_cycles=500)
    assert st == B.MG_OK
    om = O.Multigrid(oracle_rotated(n, eps, theta))
    xo, oh = om.solve(f32(b), rtol=1e-8, max_cycles=500)
    assert abs(int(cyc[0]) - (len(oh) - 1)) <= 1
    if n > 3:  # n = 3 is a single direct solve: its history is FP32 rounding of the exact x
        _cmp_hist(gh[0], oh)
    assert gh[0][cyc[0]] < 1e-8
    # the float-float iterate is the oracle's solution, and its true residual (FP64) is < 1e-8
    x = x_hi[0].double().cpu().numpy() + x_lo[0].double().cpu().numpy()
    st0 = oracle_rotated(n, eps, theta)
    true_rel = np.linalg.norm(f32(b) - O.apply(st0, x)) / np.linalg.norm(f32(b))
    assert true_rel < 1.0001e-8 and abs(true_rel - gh[0][cyc[0]]) <= 1e-3 * gh[0][cyc[0]] + 1e-12
    if n == 63:
        assert 195 <= cyc[0] <= 207
        # asymptotic factor over the last 50 cycles
        fg = (gh[0][cyc[0]] / gh[0][cyc[0] - 50]) ** (1 / 50)
        fo = (oh[-1] / oh[-51]) ** (1 / 50)
        assert abs(fg - fo) <= 1e-3 * fo


@pytest.mark.parametrize("n,cycles,ct", [(127, 40, True), (255, 60, True), (1023, 4, True), (127, 40, False),
                                         (255, 60, False), (1023, 4, False)])
def test_large_grid_jacobi_history_matches_oracle(n, cycles, ct):
    """Tiled kernels (k_residual/k_down/k_up) plus the coarse levels in one CTA cluster per
    problem (ct) or in one CTA (levels <= 63, tiled above); 1023 is the bench size."""
    eps, theta = 0.05, 1.1
    b = inputs.rhs_uniform(1000, n)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], cluster_tail=ct)
    _, _, gh, cyc, st = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=0.0, max_cycles=cycles)
    assert st == B.MG_ERR_NOT_CONVERGED and cyc[0] == cycles
    om = O.Multigrid(oracle_rotated(n, eps, theta))
    _, oh = om.solve(f32(b), rtol=0.0, max_cycles=cycles)
    assert _cmp_hist(gh[0], oh) == cycles + 1


def test_vcycle_elementwise_matches_oracle():
    """One cycle from a random iterate: x_new element-wise vs the oracle (FP32 cycle on the
    error equation, so the difference is bounded by FP32 rounding of the correction)."""
    n = 127
    rng = np.random.default_rng(5)
    eps, theta = 0.2, 2.2
    b = rng.uniform(-1, 1, (n, n)).astype(np.float32)
    x = rng.uniform(-1, 1, (n, n)).astype(np.float32)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)])
    xh = torch.from_numpy(x).cuda()[None].contiguous()
    xl = torch.zeros_like(xh)
    rel = torch.zeros(1, device="cuda")
    mg.vcycle(torch.from_numpy(b).cuda()[None].contiguous(), xh, xl, rel)
    got = (xh.double() + xl.double()).cpu().numpy()[0]
    om = O.Multigrid(oracle_rotated(n, eps, theta))
    want = om.vcycle(f32(b), f32(x))
    corr = want - f32(x)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(corr).max()
    st0 = oracle_rotated(n, eps, theta)
    want_rel = np.linalg.norm(f32(b) - O.apply(st0, want)) / np.linalg.norm(f32(b))
    assert abs(rel.item() - want_rel) <= 1e-5 * want_rel


def test_smoother_apply_matches_oracle():
    n = 63
    rng = np.random.default_rng(6)
    mg = S.MultigridSolver([S.rotated(n, 0.3, 0.4)])
    om = O.Multigrid(oracle_rotated(n, 0.3, 0.4))
    for level in (0, 1):
        nl = mg.sizes[level]
        f = rng.standard_normal((nl, nl)).astype(np.float32)
        u = rng.standard_normal((nl, nl)).astype(np.float32)
        ug = torch.from_numpy(u).cuda().contiguous()
        mg.smooth(0, level, torch.from_numpy(f).cuda().contiguous(), ug, nsteps=3)
        want = O.smooth(om.field(level), om.kernels(level), f32(f), f32(u), 3)
        np.testing.assert_allclose(ug.double().cpu().numpy(), want, rtol=0, atol=2e-5 * np.abs(want).max())


def test_batch_equals_single_problems():
    """16 instances of the bench family (eps log-uniform, theta uniform) at 255^2: each
    problem's history in the batch equals its own single-problem solve bit for bit."""
    n = 255
    params = inputs.rotated_params(inputs.SEED_PARAMS, 16)
    b = torch.from_numpy(np.stack([inputs.rhs_uniform(inputs.SEED_RHS + i, n) for i in range(16)])).cuda()
    mg = S.MultigridSolver([S.rotated(n, e, t) for e, t in params])
    _, _, gh, cyc, _ = mg.solve(b.contiguous(), rtol=1e-8, max_cycles=40)
    for i in (0, 7, 15):
        one = S.MultigridSolver([S.rotated(n, *params[i])])
        _, _, h1, c1, _ = one.solve(b[i:i + 1].contiguous(), rtol=1e-8, max_cycles=40)
        assert c1[0] == cyc[i]
        np.testing.assert_array_equal(h1[0][: c1[0] + 1], gh[i][: cyc[i] + 1])


def test_solve_status_codes():
    n = 63
    mg = S.MultigridSolver([S.rotated(n, 0.01, 0.5)])
    b = torch.from_numpy(inputs.rhs_uniform(3, n)).cuda()[None].contiguous()
    _, _, h, c, st = mg.solve(b, rtol=1e-8, max_cycles=5)
    assert st == B.MG_ERR_NOT_CONVERGED and c[0] == 5 and np.all(np.isnan(h[0][6:]))
    bad = b.clone()
    bad[0, 3, 3] = float("nan")
    with pytest.raises(B.MGError) as ei:
        mg.solve(bad, rtol=1e-8, max_cycles=5)
    assert ei.value.status == B.MG_ERR_NUMERIC
    # the context stays usable after an error
    _, _, _, c, st = mg.solve(b, rtol=1e-8, max_cycles=400)
    assert st == B.MG_OK and c[0] > 10


@pytest.mark.parametrize("ct", [True, False])
def test_timeout_status_and_recovery(ct):
    """Failure detection without a GPU fault: the test setting makes the first bounded wait
    for every tile's copies give up at once (the wait for the copies in flight keeps its
    full bound, so they land before each CTA exits).  The solve reports MG_ERR_TIMEOUT;
    with the setting off, the same context then solves like the oracle."""
    n, cycles = 255, 12
    eps, theta = 0.1, 0.8
    b = torch.from_numpy(inputs.rhs_uniform(15, n)).cuda()[None].contiguous()
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], cluster_tail=ct)
    B.mg_debug_short_wait(mg.ctx, True)
    with pytest.raises(B.MGError) as ei:
        mg.solve(b, rtol=1e-8, max_cycles=cycles)
    assert ei.value.status == B.MG_ERR_TIMEOUT
    B.mg_debug_short_wait(mg.ctx, False)
    _, _, gh, cyc, st = mg.solve(b, rtol=0.0, max_cycles=cycles)
    assert st == B.MG_ERR_NOT_CONVERGED and cyc[0] == cycles
    _, oh = O.Multigrid(oracle_rotated(n, eps, theta)).solve(f32(b[0].cpu().numpy()), rtol=0.0, max_cycles=cycles)
    assert _cmp_hist(gh[0], oh) == cycles + 1
    mg.close()


def test_warm_start_continues_history():
    """x_lo carries the float-float low part between calls: 10 + 10 cycles == 20 cycles."""
    n = 255
    mg = S.MultigridSolver([S.rotated(n, 0.1, 0.3)])
    b = torch.from_numpy(inputs.rhs_uniform(4, n)).cuda()[None].contiguous()
    _, _, h20, _, _ = mg.solve(b, rtol=0, max_cycles=20)
    xh, xl, _, _, _ = mg.solve(b, rtol=0, max_cycles=10)
    _, _, h10, _, _ = mg.solve(b, xh, xl, rtol=0, max_cycles=10)
    np.testing.assert_allclose(h10[0][1:], h20[0][11:], rtol=1e-6)


def test_varcoef_field_path_at_bench_size_matches_oracle():
    """Per-point (variable-coefficient) stencils at 1023 x 1023 with the tiled kernels:
    stencil field of level 0 bit-exact and the first cycles of the history."""
    n, cycles = 1023, 3
    a = inputs.grf_cells(inputs.SEED_GRF, n)
    mg = S.MultigridSolver([S.varcoef5(n, torch.from_numpy(a).cuda())])
    st0 = O.varcoef5_field(n, f32(a))
    np.testing.assert_array_equal(mg.stencil_field(0, 0).double().cpu().numpy(), f32(st0))
    b = inputs.rhs_uniform(9, n)
    _, _, gh, cyc, _ = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=0.0, max_cycles=cycles)
    _, oh = O.Multigrid(f32(st0)).solve(f32(b), rtol=0.0, max_cycles=cycles)
    assert _cmp_hist(gh[0], oh) == cycles + 1


def test_vcycle_without_low_part_on_tiled_path():
    """x_lo = NULL: the iterate is plain FP32 (the low part is taken as zero, not returned)."""
    n = 255
    rng = np.random.default_rng(12)
    b = rng.uniform(-1, 1, (n, n)).astype(np.float32)
    mg = S.MultigridSolver([S.rotated(n, 0.3, 0.9)])
    xh = torch.zeros((1, n, n), device="cuda")
    rel = torch.zeros(1, device="cuda")
    for _ in range(3):
        mg.vcycle(torch.from_numpy(b).cuda()[None].contiguous(), xh, None, rel)
    om = O.Multigrid(oracle_rotated(n, 0.3, 0.9))
    x = np.zeros((n, n))
    for _ in range(3):
        x = om.vcycle(f32(b), x)
    assert np.abs(xh[0].double().cpu().numpy() - x).max() <= 1e-5 * np.abs(x).max()


def test_cluster_and_one_cta_tails_agree_on_a_batch():
    """16 problems of the bench family at 511^2 (CNN-free, Jacobi): the cycle laid out as
    one CTA cluster per problem for levels <= 127 (Jacobi's layout) and as tiled kernels
    plus a one-CTA tail for levels <= 63 computes the same histories."""
    n = 511
    params = inputs.rotated_params(inputs.SEED_PARAMS, 16)
    b = torch.from_numpy(np.stack([inputs.rhs_uniform(inputs.SEED_RHS + i, n) for i in range(16)])).cuda()
    hs = []
    for ct in (True, False):
        mg = S.MultigridSolver([S.rotated(n, e, t) for e, t in params], cluster_tail=ct)
        _, _, gh, cyc, _ = mg.solve(b.contiguous(), rtol=1e-8, max_cycles=30)
        hs.append((gh, cyc))
        mg.close()
    np.testing.assert_array_equal(hs[0][1], hs[1][1])
    for p in range(16):
        k = int(hs[0][1][p]) + 1
        np.testing.assert_allclose(hs[0][0][p][:k], hs[1][0][p][:k], rtol=1e-6)


def test_batch_solve_is_deterministic():
    """Two solves of a 16-problem 511^2 batch (CUDA-graph cycles with programmatic launches,
    CNN-free) give bit-identical histories and iterates."""
    n = 511
    params = inputs.rotated_params(inputs.SEED_PARAMS, 16)
    b = torch.from_numpy(np.stack([inputs.rhs_uniform(inputs.SEED_RHS + i, n) for i in range(16)])).cuda()
    mg = S.MultigridSolver([S.rotated(n, e, t) for e, t in params])
    runs = [mg.solve(b.contiguous(), rtol=1e-8, max_cycles=40) for _ in range(3)]
    for xh, xl, gh, cyc, _ in runs[1:]:
        np.testing.assert_array_equal(cyc, runs[0][3])
        np.testing.assert_array_equal(np.nan_to_num(gh, nan=-1.0), np.nan_to_num(runs[0][2], nan=-1.0))
        assert torch.equal(xh, runs[0][0]) and torch.equal(xl, runs[0][1])


@pytest.mark.parametrize("ct", [True, False])
def test_bench_batch_first_cycles_match_oracle(ct):
    """The 16-problem 1023^2 bench batch: every tiled level runs in several waves of CTAs
    (level 0: 16384 tiles, level 1: 4096), so a kernel that overwrote an array other CTAs
    still read with halos would show here.  Problems 0 and 9 (the slowest Jacobi one)
    against the oracle over the first cycles."""
    n, cycles = 1023, 3
    params = inputs.rotated_params(inputs.SEED_PARAMS, 16)
    b = torch.from_numpy(np.stack([inputs.rhs_uniform(inputs.SEED_RHS + i, n) for i in range(16)])).cuda()
    mg = S.MultigridSolver([S.rotated(n, e, t) for e, t in params], cluster_tail=ct)
    _, _, gh, cyc, _ = mg.solve(b.contiguous(), rtol=0.0, max_cycles=cycles)
    assert np.all(cyc == cycles)
    for p in (0, 9):
        om = O.Multigrid(oracle_rotated(n, *params[p]))
        _, oh = om.solve(f32(b[p].cpu().numpy()), rtol=0.0, max_cycles=cycles)
        assert _cmp_hist(gh[p], oh) == cycles + 1


def _mixed_problems():
    """Five problems in three groups: rotated 63 and 255 (two each, the second pair with
    different eps/theta) and one GRF 5-point problem at 127."""
    params = inputs.rotated_params(inputs.SEED_PARAMS + 31, 4)
    probs = [S.rotated(63, *params[0]), S.rotated(255, *params[1]), S.rotated(63, *params[2]),
             S.rotated(255, *params[3])]
    cells = torch.from_numpy(inputs.grf_cells(inputs.SEED_GRF + 31, 127)).cuda()
    probs.append(S.varcoef5(127, cells))
    b = [torch.from_numpy(inputs.rhs_uniform(inputs.SEED_RHS + 300 + i, p["n"])).cuda() for i, p in enumerate(probs)]
    return probs, b


@pytest.mark.parametrize("autotune,shapes", [(False, ("32x32",)), (False, ("strip8x32",)), (False, ("strip4x32",)),
                                             (True, None)])
def test_solve_multi_matches_single_context_solves(autotune, shapes):
    """mg_solve_multi over several contexts on their own streams gives, per problem, the
    iterate and cycle count of a plain mg_solve of the same group (bit-identical), with the
    tile shapes fixed or chosen by the autotuner; every problem's time to its stopping test
    is reported and lies inside the solve."""
    probs, b = _mixed_problems()
    mb = S.MixedBatchSolver(probs, "jacobi", autotune=autotune, tune_cycles=4, shapes=shapes)
    assert sorted(mb.groups) == [(63, "const"), (127, "field"), (255, "const")]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, cycles, st = mb.solve(b, rtol=1e-8, max_cycles=5000)
    torch.cuda.synchronize()
    wall_ms = 1e3 * (time.perf_counter() - t0)
    assert st == B.MG_OK, cycles
    assert np.all(mb.last_times_ms > 0) and np.all(mb.last_times_ms <= wall_ms), (mb.last_times_ms, wall_ms)
    for key, idx in mb.groups.items():
        ct, shape = mb.layout[key]
        if shapes and key[0] > 63:
            assert shape == shapes[0]
        mg = S.MultigridSolver([probs[i] for i in idx], "jacobi", cluster_tail=ct, tile_shape=shape)
        bb = torch.stack([b[i] for i in idx]).contiguous()
        xh, _, _, cyc, st1 = mg.solve(bb, rtol=1e-8, max_cycles=5000, history=False)
        assert st1 == B.MG_OK
        for j, i in enumerate(idx):
            assert cycles[i] == cyc[j], (key, i)
            assert torch.equal(x[i], xh[j]), (key, i)
        mg.close()
    mb.close()
    # and the 63 x 63 problem against the oracle
    om = O.Multigrid(oracle_rotated(63, *inputs.rotated_params(inputs.SEED_PARAMS + 31, 4)[0]))
    _, oh = om.solve(f32(b[0].cpu().numpy()), rtol=1e-8, max_cycles=5000)
    assert abs(int(cycles[0]) - (len(oh) - 1)) <= 1


def test_solve_multi_rejects_bad_arguments():
    probs, b = _mixed_problems()
    mg = S.MultigridSolver(probs[:1], "jacobi")
    bb = b[0][None].contiguous()
    xh, xl = torch.zeros_like(bb), torch.zeros_like(bb)
    with pytest.raises(B.MGError):
        B.mg_solve_multi([mg.ctx, mg.ctx], [bb, bb], [xh, xh], [xl, xl], 1e-8, 10)
    with pytest.raises(B.MGError):
        B.mg_solve_multi([], [], [], [], 1e-8, 10)
    mg.close()


@pytest.mark.parametrize("ct", [True, False])
def test_small_tiled_batches_repeat_bit_identically(ct):
    """Batches whose problems converge at different cycles at the smallest tiled sizes
    (one tile level above the coarse tail): repeated solves give identical iterates and
    cycle counts, and every problem reaches rtol.  Problems drop out of the launches one by
    one here, so every kernel sees the stopping flags change between cycles."""
    for n, count in ((127, 6), (255, 5)):
        params = inputs.rotated_params(inputs.SEED_PARAMS + 41 + n, count, eps_lo=0.05)
        mg = S.MultigridSolver([S.rotated(n, e, t) for e, t in params], cluster_tail=ct)
        b = torch.from_numpy(np.stack([inputs.rhs_uniform(inputs.SEED_RHS + 700 + i, n) for i in range(count)]))
        b = b.cuda().contiguous()
        runs = []
        for _ in range(3):
            xh, xl, gh, cyc, st = mg.solve(b, rtol=1e-8, max_cycles=3000)
            assert st == B.MG_OK
            assert len(set(cyc.tolist())) > 1  # the problems stop at different cycles
            runs.append((xh.clone(), cyc.copy()))
        for xh, cyc in runs[1:]:
            assert np.array_equal(cyc, runs[0][1])
            assert torch.equal(xh, runs[0][0])
        mg.close()
