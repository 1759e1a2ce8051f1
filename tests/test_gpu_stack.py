"""GPU parity of the network with three output kernels applied as a stack (Sec. 4, 4.2:
k = 3; MG_NET_CONV3), through the C ABI against the FP64 stack oracle (oracle/stack.py).
Tolerance: the per-cycle relative residual within 1e-5, as for every solve path."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import stack as OS
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


def stack_params(seed, last=0.02, zero_rest=False):
    """Kaiming-like convolutions and a small last layer: a convergent smoother."""
    rng = np.random.default_rng(seed)
    parts = []
    for k, (co, ci) in enumerate(OS.SIZES):
        scale = last if k == 3 else np.sqrt(6.0 / (ci * 9)) / np.sqrt(3.0)
        parts.append(rng.standard_normal(co * ci * 9) * scale)
    p = np.concatenate(parts).astype(np.float32)
    if zero_rest:
        p[-18 * 27:] = 0.0
    return p


@pytest.mark.parametrize("n,cycles", [(63, 25), (255, 12)])
def test_stack_solve_history_matches_oracle(n, cycles):
    """n = 63: whole solves in one CTA; 255: batched level kernels above 63, then the tail."""
    eps, theta = 0.05, 0.7
    p = stack_params(n)
    b = inputs.rhs_uniform(90, n)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(p).cuda(), net_arch="conv3")
    _, _, gh, cyc, _ = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=0.0, max_cycles=cycles)
    _, oh = OS.StackMultigrid(O.const_field(n, f32(O.q1_rotated_stencil(eps, theta))), f32(p)).solve(
        f32(b), rtol=0.0, max_cycles=cycles)
    assert cyc[0] == cycles
    rel = np.abs(gh[0][: cycles + 1] - oh) / oh
    assert rel.max() <= 1e-5, rel.max()


def test_stack_solve_per_point_field():
    n = 127
    a = inputs.grf_cells(13, n)
    p = stack_params(5)
    mg = S.MultigridSolver([S.varcoef5(n, torch.from_numpy(a).cuda())], "cnn", torch.from_numpy(p).cuda(),
                           net_arch="conv3")
    b = inputs.rhs_uniform(91, n)
    _, _, gh, _, _ = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=0.0, max_cycles=12)
    _, oh = OS.StackMultigrid(f32(O.varcoef5_field(n, f32(a))), f32(p)).solve(f32(b), rtol=0.0, max_cycles=12)
    rel = np.abs(gh[0][:13] - oh) / oh
    assert rel.max() <= 1e-5, rel.max()


def test_stack_with_identity_kernels_two_and_three_solves_like_the_k1_network():
    n, eps, theta = 255, 0.02, 2.0
    p = stack_params(7, zero_rest=True)
    b = torch.from_numpy(inputs.rhs_uniform(92, n)).cuda()[None].contiguous()
    st3 = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(p).cuda(), net_arch="conv3")
    st1 = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(OS.k1_params(p).astype(np.float32)).cuda())
    _, _, h3, c3, _ = st3.solve(b, rtol=1e-8, max_cycles=3000)
    _, _, h1, c1, _ = st1.solve(b, rtol=1e-8, max_cycles=3000)
    assert abs(int(c3[0]) - int(c1[0])) <= 1
    k = min(int(c3[0]), int(c1[0])) + 1
    assert np.max(np.abs(h3[0][:k] - h1[0][:k]) / h1[0][:k]) < 1e-5


@pytest.mark.parametrize("n,cycles", [(15, 1), (31, 1), (15, 2)])
def test_stack_train_step_matches_oracle(n, cycles):
    """The two-grid loss (k cycles) and its gradient through the stack and the 27-output
    network against the oracle's reverse mode (FP64 autograd over the same operations)."""
    nprob, nvec = 2, 3
    params = inputs.rotated_params(150 + n + cycles, nprob)
    probs = [{"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": e, "theta": t} for e, t in params]
    z = inputs.gaussian_vectors(151 + n + cycles, nprob * nvec, n).reshape(nprob, nvec, n, n)
    p = stack_params(9, last=0.05)
    batch = T.TwoGridBatch(probs, nvec, 2.0 / 3.0, False, cycles=cycles, net_arch="conv3")
    loss, grad = batch.loss_and_grad(torch.from_numpy(p).cuda(), torch.from_numpy(z).cuda().contiguous())
    batch.close()
    assert grad.numel() == OS.NPARAMS
    lo, go = 0.0, np.zeros(p.size)
    for k, (e, t) in enumerate(params):
        st = O.const_field(n, f32(O.q1_rotated_stencil(e, t)))
        l1, g1 = OS.loss_and_grad(st, O.rap(st), f32(p), f32(z[k]), cycles=cycles)
        lo += l1 / nprob
        go += g1 / nprob
    assert abs(loss.item() - lo) <= 1e-5 * lo, (loss.item(), lo)
    g = grad.double().cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)
    # kernels 2 and 3 (the last 18 x 27 weights) carry gradient of their own
    assert np.linalg.norm(g[-18 * 27:] - go[-18 * 27:]) <= 1e-4 * np.linalg.norm(go[-18 * 27:])


@pytest.mark.parametrize("n,cycles", [(15, 1), (31, 1), (31, 2)])
def test_stack_vcycle_coarse_train_step_matches_oracle(n, cycles):
    """Algorithm 2 with the three-kernel stack: the two-grid objective whose coarse solve is
    one V-cycle of the hierarchy below smoothed by (already trained) stack networks, and
    its adjoint through the cycle with every stack transposed (smoother_transpose: K1^T
    K2^T K3^T) -- loss and gradient against the oracle, whose adjoint is FP64 autograd
    through its own coarse cycle."""
    nprob, nvec = 2, 3
    params = inputs.rotated_params(170 + n + cycles, nprob)
    probs = [{"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": e, "theta": t} for e, t in params]
    z = inputs.gaussian_vectors(171 + n + cycles, nprob * nvec, n).reshape(nprob, nvec, n, n)
    p = stack_params(25, last=0.05)
    sets = np.stack([stack_params(26 + j, last=0.05) for j in range(2)])
    batch = T.TwoGridBatch(probs, nvec, 2.0 / 3.0, False, cycles=cycles, net_arch="conv3")
    batch.attach_coarse(torch.from_numpy(sets).cuda())
    loss, grad = batch.loss_and_grad(torch.from_numpy(p).cuda(), torch.from_numpy(z).cuda().contiguous())
    batch.close()
    lo, go = 0.0, np.zeros(p.size)
    for k, (e, t) in enumerate(params):
        st = O.const_field(n, f32(O.q1_rotated_stencil(e, t)))
        st_c = O.rap(st)
        l1, g1 = OS.loss_and_grad(st, st_c, f32(p), f32(z[k]), cycles=cycles,
                                  coarse=OS.coarse_vcycle(st_c, [f32(q) for q in sets]))
        lo += l1 / nprob
        go += g1 / nprob
    assert abs(loss.item() - lo) <= 1e-5 * lo, (loss.item(), lo)
    g = grad.double().cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)


def test_stack_transposed_context_applies_the_adjoint_cycle():
    """A context built with smoother_transpose applies M^T: <M u, v> = <u, M^T v> for one
    V-cycle from zero of a 63^2 per-point problem with the stack smoother."""
    n = 63
    cells = torch.from_numpy(inputs.grf_cells(inputs.SEED_GRF + 90, n)).cuda()
    p = torch.from_numpy(stack_params(27, last=0.05)).cuda()
    mgs = [S.MultigridSolver([S.varcoef5(n, cells)], "cnn", p, net_arch="conv3", transpose=t) for t in (False, True)]
    rng = np.random.default_rng(28)
    u = torch.from_numpy(rng.standard_normal((1, n, n)).astype(np.float32)).cuda()
    v = torch.from_numpy(rng.standard_normal((1, n, n)).astype(np.float32)).cuda()
    outs = []
    for mg, rhs in zip(mgs, (u, v)):
        xh, xl = torch.zeros_like(rhs), torch.zeros_like(rhs)
        mg.vcycle(rhs.contiguous(), xh, xl)
        outs.append(xh.double() + xl.double())
        mg.close()
    lhs = (outs[0] * v.double()).sum().item()
    rhs_ = (u.double() * outs[1]).sum().item()
    # FP32 cycles: the two inner products agree to a few FP32 roundings of the vectors' size
    scale = (outs[0].norm() * v.double().norm()).item()
    assert abs(lhs - rhs_) <= 1e-5 * scale, (lhs, rhs_, scale)


def test_stack_trainer_reduces_the_loss():
    tr = T.Trainer(sizes=(15,), per_size=8, nvec=8, lr=3e-3, net_arch="conv3", conv_bf16=False)
    assert tr.params.numel() == OS.NPARAMS
    losses = [tr.step() for _ in range(60)]
    assert np.mean(losses[-10:]) < 0.9 * np.mean(losses[:10]), (losses[:5], losses[-5:])


def test_stack_training_is_fp32_only():
    with pytest.raises(B.MGError):
        T.TwoGridBatch([S.rotated(15, 0.1, 0.2)], 2, 2.0 / 3.0, True, net_arch="conv3")


def test_stack_preconditioned_fgmres_matches_oracle():
    """Flexible GMRES (Sec. 6.4) with one V-cycle of the stack-smoothed hierarchy as M."""
    n, eps, theta = 255, 0.01, np.pi / 12
    p = stack_params(21)
    b_np = inputs.rhs_uniform(inputs.SEED_RHS + 1600, n)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(p).cuda(), net_arch="conv3")
    xh, xl, gh, its, st = S.fgmres(mg, torch.from_numpy(b_np).cuda()[None].contiguous(), restart=30, rtol=1e-6,
                                   max_iters=200)
    assert st == B.MG_OK
    st0 = O.const_field(n, f32(O.q1_rotated_stencil(eps, theta)))
    sm = OS.StackMultigrid(st0, f32(p))
    _, oh, oits = O.fgmres(lambda v: O.apply(st0, v), lambda v: sm.vcycle(v, np.zeros_like(v)), f32(b_np),
                           restart=30, rtol=1e-6, max_iters=200)
    assert abs(int(its[0]) - oits) <= 2, (int(its[0]), oits)
    k = min(int(its[0]), oits, 30) + 1
    assert np.max(np.abs(gh[0][:k] - oh[:k]) / oh[:k]) <= 1e-3
    x = xh[0].double().cpu().numpy() + xl[0].double().cpu().numpy()
    assert np.linalg.norm(f32(b_np) - O.apply(st0, x)) / np.linalg.norm(f32(b_np)) < 1e-6
