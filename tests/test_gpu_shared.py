"""GPU parity of the shared-kernel network (MG_NET_CONV_SHARED, Sec. 6.2's 378 parameters)
through the C ABI against the FP64 oracle: the kernels on every level (class tables and
per-point fields, per-level sets), the solve history, and the two-grid loss with its
gradient.  Tolerances as for the dense network (same FP32 arithmetic after the expansion)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2102_12071_gb300 import binding as B
from paper_2102_12071_gb300 import inputs
from paper_2102_12071_gb300 import solver as S
from paper_2102_12071_gb300 import train as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2102_12071_gb300 import build

    build.build()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def shared_net(seed, scale=0.05):
    """Kaiming-bound convolutions, a small last layer: a convergent smoother."""
    p = T.init_params_shared(seed).numpy()
    p[135:] = np.random.default_rng(seed).standard_normal(243) * scale
    return p.astype(np.float32)


@pytest.mark.parametrize("kind", ["rotated", "varcoef"])
def test_shared_kernels_match_oracle_on_every_level(kind):
    n = 31
    p = shared_net(1)
    if kind == "rotated":
        prob = S.rotated(n, 0.03, 2.0)
        st0 = O.const_field(n, f32(O.q1_rotated_stencil(0.03, 2.0)))
    else:
        cells = inputs.grf_cells(inputs.SEED_GRF + 80, n)
        prob = S.varcoef5(n, torch.from_numpy(cells).cuda())
        st0 = f32(O.varcoef5_field(n, f32(cells)))
    mg = S.MultigridSolver([prob], "cnn", torch.from_numpy(p).cuda(), net_arch="conv_shared")
    om = O.Multigrid(st0)
    for l in range(mg.levels - 1):
        Wg = mg.kernels(0, l).double().cpu().numpy()
        Wo = O.shared_forward(om.field(l), f32(p))
        np.testing.assert_allclose(Wg, Wo, rtol=2e-5, atol=2e-6 * np.abs(Wo).max())


def test_shared_per_level_sets():
    n = 31
    cells = torch.from_numpy(inputs.grf_cells(inputs.SEED_GRF + 81, n)).cuda()
    sets = np.stack([shared_net(10 + j, 0.1) for j in range(2)])
    mg = S.MultigridSolver([S.varcoef5(n, cells)], "cnn", torch.from_numpy(sets).cuda(), net_arch="conv_shared")
    om = O.Multigrid(f32(O.varcoef5_field(n, f32(cells.cpu().numpy()))))
    for l in range(mg.levels - 1):
        Wo = O.shared_forward(om.field(l), f32(sets[min(l, 1)]))
        Wg = mg.kernels(0, l).double().cpu().numpy()
        np.testing.assert_allclose(Wg, Wo, rtol=2e-5, atol=2e-6 * np.abs(Wo).max())


@pytest.mark.parametrize("n,cycles", [(63, 30), (255, 20)])
def test_shared_solve_history_matches_oracle(n, cycles):
    eps, theta = 0.05, 0.7
    p = shared_net(3)
    b = inputs.rhs_uniform(17, n)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(p).cuda(), net_arch="conv_shared")
    _, _, gh, cyc, _ = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=0.0, max_cycles=cycles)
    om = O.Multigrid(O.const_field(n, f32(O.q1_rotated_stencil(eps, theta))))
    om.set_cnn(O.shared_to_dense(f32(p)))
    _, oh = om.solve(f32(b), rtol=0.0, max_cycles=cycles)
    assert cyc[0] == cycles
    rel = np.abs(gh[0][: cycles + 1] - oh) / oh
    assert rel.max() <= 1e-5, rel.max()


@pytest.mark.parametrize("n,cycles", [(15, 1), (31, 1), (15, 2)])
def test_shared_train_step_matches_oracle(n, cycles):
    nprob, nvec = 3, 4
    params = inputs.rotated_params(140 + n + cycles, nprob)
    probs = [{"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": e, "theta": t} for e, t in params]
    z = inputs.gaussian_vectors(141 + n + cycles, nprob * nvec, n).reshape(nprob, nvec, n, n)
    p = shared_net(5, 0.1)
    batch = T.TwoGridBatch(probs, nvec, 2.0 / 3.0, False, cycles=cycles, net_arch="conv_shared")
    loss, grad = batch.loss_and_grad(torch.from_numpy(p).cuda(), torch.from_numpy(z).cuda().contiguous())
    batch.close()
    assert grad.numel() == 378
    lo, go = 0.0, np.zeros(p.size)
    for k, (e, t) in enumerate(params):
        st = O.const_field(n, f32(O.q1_rotated_stencil(e, t)))
        l1, g1 = O.shared_loss_and_grad(st, f32(p), f32(z[k]), cycles=cycles)
        lo += l1 / nprob
        go += g1 / nprob
    assert abs(loss.item() - lo) <= 1e-5 * lo, (loss.item(), lo)
    g = grad.double().cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)


def test_shared_trainer_reduces_the_loss():
    tr = T.Trainer(sizes=(15,), per_size=8, nvec=8, lr=3e-3, net_arch="conv_shared", conv_bf16=False)
    assert tr.params.numel() == 378
    losses = [tr.step() for _ in range(60)]
    assert np.mean(losses[-10:]) < 0.9 * np.mean(losses[:10]), (losses[:5], losses[-5:])


def test_shared_preconditioned_fgmres_matches_oracle():
    n, eps, theta = 255, 0.01, np.pi / 4
    p = shared_net(22)
    b_np = inputs.rhs_uniform(inputs.SEED_RHS + 1601, n)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(p).cuda(), net_arch="conv_shared")
    xh, xl, gh, its, st = S.fgmres(mg, torch.from_numpy(b_np).cuda()[None].contiguous(), restart=30, rtol=1e-6,
                                   max_iters=200)
    assert st == B.MG_OK
    st0 = O.const_field(n, f32(O.q1_rotated_stencil(eps, theta)))
    om = O.Multigrid(st0)
    om.set_cnn(O.shared_to_dense(f32(p)))
    _, oh, oits = O.fgmres(lambda v: O.apply(st0, v), lambda v: om.vcycle(v, np.zeros_like(v)), f32(b_np),
                           restart=30, rtol=1e-6, max_iters=200)
    assert abs(int(its[0]) - oits) <= 2, (int(its[0]), oits)
    k = min(int(its[0]), oits, 30) + 1
    assert np.max(np.abs(gh[0][:k] - oh[:k]) / oh[:k]) <= 1e-3
    x = xh[0].double().cpu().numpy() + xl[0].double().cpu().numpy()
    assert np.linalg.norm(f32(b_np) - O.apply(st0, x)) / np.linalg.norm(f32(b_np)) < 1e-6
