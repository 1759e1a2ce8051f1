"""GPU parity of the learned part: network inference, the CNN-smoothed V-cycle and the
two-grid training loss with its gradient, all through the C ABI against the FP64 oracle.

Tolerances: FP32 network path element-wise rtol 2e-5 (a few ulps through ~100-term dot
products); gradients 1e-4 relative; bfloat16 mode checked against the oracle's own
bfloat16 emulation where the two roundings agree, and as a whole against the FP32 result.
"""
import math

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


def small_net(seed=0, scale=0.05):
    """Random network whose smoother stays convergent: Kaiming convolutions, small output layer."""
    p = T.init_params(seed).numpy()
    p[-243:] = np.random.default_rng(seed).standard_normal(243) * scale
    return p.astype(np.float32)


def varcoef_field(n, seed):
    a = inputs.grf_cells(seed, n)
    return f32(O.varcoef5_field(n, f32(a)))


@pytest.mark.parametrize("bf16", [False, True])
def test_net_forward_matches_oracle(bf16):
    n = 45  # three 16-point tiles with a ragged last one
    fields = np.stack([varcoef_field(n, 10), f32(O.const_field(n, O.q1_rotated_stencil(0.02, 0.9)))])
    p = small_net(1, 0.3)
    Wg = S.net_forward(torch.from_numpy(fields.astype(np.float32)).cuda(), torch.from_numpy(p).cuda(),
                       2.0 / 3.0, bf16).double().cpu().numpy()
    for k in range(2):
        Wo = O.hypernet_forward(fields[k], f32(p), 2.0 / 3.0, bf16)
        scale = np.abs(Wo).max()
        if not bf16:
            np.testing.assert_allclose(Wg[k], Wo, rtol=2e-5, atol=2e-6 * scale)
        else:
            # the two sides round FP32 (kernel) and FP64 (oracle) pre-activations to bfloat16;
            # they agree except where a value sits within an FP32 ulp of a rounding boundary
            err = np.abs(Wg[k] - Wo)
            assert np.mean(err <= 2e-5 * scale) > 0.99
            assert err.max() <= 2e-2 * scale


@pytest.mark.parametrize("n", [31, 127])
def test_cnn_kernels_match_oracle_on_every_level(n):
    """Constant stencils use kernel class tables on a proxy grid; expanded, they must equal
    the network evaluated on each level's full field (FP32 network)."""
    eps, theta = 0.03, 2.0
    p = small_net(2)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(p).cuda())
    om = O.Multigrid(O.const_field(n, f32(O.q1_rotated_stencil(eps, theta))))
    for l in range(mg.levels - 1):
        Wg = mg.kernels(0, l).double().cpu().numpy()
        Wo = O.hypernet_forward(om.field(l), f32(p))
        np.testing.assert_allclose(Wg, Wo, rtol=2e-5, atol=2e-6 * np.abs(Wo).max())


@pytest.mark.parametrize("n,cycles,ct", [(63, 60, True), (255, 25, True), (255, 25, False), (511, 8, True)])
def test_cnn_solve_history_matches_oracle(n, cycles, ct):
    """ct: coarse levels in one CTA cluster per problem (True) or one CTA (False)."""
    eps, theta = 0.05, 0.7
    p = small_net(3)
    b = inputs.rhs_uniform(7, n)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(p).cuda(), cluster_tail=ct)
    _, _, gh, cyc, _ = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=0.0, max_cycles=cycles)
    om = O.Multigrid(O.const_field(n, f32(O.q1_rotated_stencil(eps, theta))))
    om.set_cnn(f32(p))
    _, oh = om.solve(f32(b), rtol=0.0, max_cycles=cycles)
    assert cyc[0] == cycles
    rel = np.abs(gh[0][: cycles + 1] - oh) / oh
    assert rel.max() <= 1e-5, rel.max()


@pytest.mark.parametrize("ct", [True, False])
def test_cnn_solve_varcoef_field_path(ct):
    """Per-point kernels (variable coefficients): setup, RAP fields and the CNN solve."""
    n = 127
    a = inputs.grf_cells(11, n)
    p = small_net(4)
    mg = S.MultigridSolver([S.varcoef5(n, torch.from_numpy(a).cuda())], "cnn", torch.from_numpy(p).cuda(),
                           cluster_tail=ct)
    st0 = O.varcoef5_field(n, f32(a))
    om = O.Multigrid(f32(st0))
    for l in range(mg.levels):
        g = mg.stencil_field(0, l).double().cpu().numpy()
        # Per-point Galerkin fields are rounded to FP32 on every level.  Bilinear P sums to 4
        # around a coarse point, so P^T A P multiplies a stencil's row sum by 4; the rounding
        # of a level's (near-zero) row sum therefore grows by 4 per level below it.
        np.testing.assert_allclose(g, om.field(l), rtol=0, atol=4 * 4.0 ** l * 2.0 ** -24 * np.abs(om.field(l)).max())
    om.set_cnn(f32(p))
    b = inputs.rhs_uniform(8, n)
    _, _, gh, cyc, _ = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=0.0, max_cycles=20)
    _, oh = om.solve(f32(b), rtol=0.0, max_cycles=20)
    rel = np.abs(gh[0][:21] - oh) / oh
    assert rel.max() <= 1e-5, rel.max()


def _train_batch(n, nprob, nvec, seed, bf16=False):
    params = inputs.rotated_params(seed, nprob)
    probs = [{"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": e, "theta": t} for e, t in params]
    z = inputs.gaussian_vectors(seed + 1, nprob * nvec, n).reshape(nprob, nvec, n, n)
    return params, probs, z, T.TwoGridBatch(probs, nvec, 2.0 / 3.0, bf16)


@pytest.mark.parametrize("n", [15, 31])
def test_train_step_matches_oracle_loss_and_gradient(n):
    """C3 check at 15 x 15 (and 31 x 31): loss and dloss/dparams vs the FP64 oracle."""
    nprob, nvec = 3, 4
    params, probs, z, batch = _train_batch(n, nprob, nvec, 40 + n)
    p = small_net(5, 0.1)
    loss, grad = batch.loss_and_grad(torch.from_numpy(p).cuda(), torch.from_numpy(z).cuda().contiguous())
    lo, go = 0.0, np.zeros(p.size)
    for k, (e, t) in enumerate(params):
        st = O.const_field(n, f32(O.q1_rotated_stencil(e, t)))
        l1, g1 = O.cnn_loss_and_grad(st, f32(p), f32(z[k]))
        lo += l1 / nprob
        go += g1 / nprob
    assert abs(loss.item() - lo) <= 1e-5 * lo
    g = grad.double().cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    big = np.abs(go) > 1e-2 * np.abs(go).max()
    np.testing.assert_allclose(g[big], go[big], rtol=1e-3)


@pytest.mark.parametrize("n,cycles", [(15, 2), (15, 3), (31, 2)])
def test_k_cycle_train_step_matches_oracle(n, cycles):
    """The loss after k two-grid cycles and its adjoint through all k (north star line 3)
    vs the FP64 oracle; with checkpointing the same numbers come out bit for bit."""
    nprob, nvec = 3, 4
    params = inputs.rotated_params(60 + n + cycles, nprob)
    probs = [{"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": e, "theta": t} for e, t in params]
    z = inputs.gaussian_vectors(61 + n, nprob * nvec, n).reshape(nprob, nvec, n, n)
    zt = torch.from_numpy(z).cuda().contiguous()
    p = small_net(7, 0.1)
    pt = torch.from_numpy(p).cuda()
    res = []
    for ckpt in (False, True):
        batch = T.TwoGridBatch(probs, nvec, 2.0 / 3.0, False, cycles=cycles, checkpoint=ckpt)
        loss, grad = batch.loss_and_grad(pt, zt)
        res.append((loss.item(), grad.double().cpu().numpy()))
        batch.close()
    assert res[0][0] == res[1][0]
    np.testing.assert_array_equal(res[0][1], res[1][1])
    lo, go = 0.0, np.zeros(p.size)
    for k, (e, t) in enumerate(params):
        st = O.const_field(n, f32(O.q1_rotated_stencil(e, t)))
        l1, g1 = O.cnn_loss_and_grad(st, f32(p), f32(z[k]), cycles=cycles)
        lo += l1 / nprob
        go += g1 / nprob
    loss, g = res[0]
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)


def test_train_step_cycle_count_is_settable():
    """A batch set up for k = 3 evaluates k = 1 exactly like a one-cycle batch."""
    n, nprob, nvec = 15, 2, 3
    params = inputs.rotated_params(90, nprob)
    probs = [{"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": e, "theta": t} for e, t in params]
    zt = torch.from_numpy(inputs.gaussian_vectors(91, nprob * nvec, n).reshape(nprob, nvec, n, n)).cuda().contiguous()
    pt = torch.from_numpy(small_net(8, 0.1)).cuda()
    one = T.TwoGridBatch(probs, nvec, 2.0 / 3.0, False)
    three = T.TwoGridBatch(probs, nvec, 2.0 / 3.0, False, cycles=3)
    three.set_cycles(1)
    l1, g1 = one.loss_and_grad(pt, zt)
    l3, g3 = three.loss_and_grad(pt, zt)
    assert l1.item() == l3.item()
    assert torch.equal(g1, g3)
    with pytest.raises(B.MGError):
        three.set_cycles(4)


def test_train_step_gradient_matches_finite_differences_on_gpu_loss():
    """The library's adjoint against central differences of the library's own loss (FP32
    loss, so the step is large and the check loose); the FP64 FD check is the oracle's."""
    n = 15
    _, _, z, batch = _train_batch(n, 2, 4, 77)
    p = small_net(6, 0.1).astype(np.float64)
    zt = torch.from_numpy(z).cuda().contiguous()
    _, grad = batch.loss_and_grad(torch.from_numpy(p.astype(np.float32)).cuda(), zt)
    g = grad.double().cpu().numpy()
    d = np.random.default_rng(0).standard_normal(p.size)
    h = 1e-2 / np.linalg.norm(d)
    lp, _ = batch.loss_and_grad(torch.from_numpy((p + h * d).astype(np.float32)).cuda(), zt, False)
    lm, _ = batch.loss_and_grad(torch.from_numpy((p - h * d).astype(np.float32)).cuda(), zt, False)
    fd = (lp.item() - lm.item()) / (2 * h)
    assert abs(fd - g @ d) <= 2e-2 * abs(g @ d)


@pytest.mark.parametrize("n", [15, 31])
def test_bf16_train_step_matches_oracle_bf16(n):
    """The bfloat16 network of C2/C3 (weights and every layer input rounded to bfloat16,
    FP32 accumulation) against the oracle's own bfloat16 emulation of the same network:
    loss within 1e-5 and gradient within 1e-4 relative."""
    nprob, nvec = 3, 4
    params, probs, z, batch = _train_batch(n, nprob, nvec, 140 + n, bf16=True)
    p = small_net(11, 0.1)
    loss, grad = batch.loss_and_grad(torch.from_numpy(p).cuda(), torch.from_numpy(z).cuda().contiguous())
    batch.close()
    lo, go = 0.0, np.zeros(p.size)
    for k, (e, t) in enumerate(params):
        st = O.const_field(n, f32(O.q1_rotated_stencil(e, t)))
        l1, g1 = O.cnn_loss_and_grad(st, f32(p), f32(z[k]), bf16=True)
        lo += l1 / nprob
        go += g1 / nprob
    assert abs(loss.item() - lo) <= 1e-5 * lo, (loss.item(), lo)
    g = grad.double().cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)


def test_bf16_training_loss_close_to_fp32():
    n = 31
    _, probs, z, b32 = _train_batch(n, 4, 4, 90, bf16=False)
    b16 = T.TwoGridBatch(probs, 4, 2.0 / 3.0, True)
    p = torch.from_numpy(small_net(7, 0.1)).cuda()
    zt = torch.from_numpy(z).cuda().contiguous()
    l32, g32 = b32.loss_and_grad(p, zt)
    l16, g16 = b16.loss_and_grad(p, zt)
    # bfloat16 keeps 8 significant bits (relative rounding 2^-9 per operand); through four
    # layers the kernels move by ~1 % and the loss by a few per cent
    assert abs(l16.item() - l32.item()) <= 5e-2 * l32.item()
    cos = torch.dot(g16, g32) / (g16.norm() * g32.norm())
    assert cos.item() > 0.98


def test_autograd_function_and_adam_step_reduce_loss():
    _, _, z, batch = _train_batch(31, 8, 8, 123)
    zt = torch.from_numpy(z).cuda().contiguous()
    tr = T.Trainer(sizes=(31,), per_size=8, nvec=8, conv_bf16=False, lr=1e-3, seed=0)
    # the autograd path returns the library's adjoint
    p = tr.params.detach().clone().requires_grad_(True)
    T.TwoGridLoss.apply(p, zt, batch).backward()
    _, g = batch.loss_and_grad(p.detach(), zt)
    torch.testing.assert_close(p.grad, g)
    l0 = batch.loss_and_grad(tr.params.detach(), zt, False)[0].item()
    for _ in range(40):
        tr.step()
    l1 = batch.loss_and_grad(tr.params.detach(), zt, False)[0].item()
    assert l1 < l0


def test_trained_network_gains_over_jacobi():
    """What training buys: the committed parameters (trained on the GPU by the two-grid loss
    on 31^2 and 63^2 problems) against the same cycle with the network's starting point,
    weighted Jacobi, on held-out problems of the bench family at 255^2: fewer V(1,1) cycles
    to 1e-8 and a smaller asymptotic factor for every problem, and the CNN history of one
    of them equal to the oracle's."""
    import os

    path = os.path.join(os.path.dirname(S.__file__), "weights", "cnn_rotated.npy")
    w = torch.from_numpy(np.load(path).astype(np.float32)).cuda()
    n = 255
    params = inputs.rotated_params(inputs.SEED_PARAMS + 97, 6)  # not drawn by training or the bench
    b = torch.from_numpy(np.stack([inputs.rhs_uniform(inputs.SEED_RHS + 300 + i, n) for i in range(6)])).cuda()
    probs = [S.rotated(n, e, t) for e, t in params]
    res = {}
    for kind in ("jacobi", "cnn"):
        mg = S.MultigridSolver(probs, kind, net_params=w if kind == "cnn" else None)
        _, _, gh, cyc, st = mg.solve(b.contiguous(), rtol=1e-8, max_cycles=20000)
        assert st == B.MG_OK
        res[kind] = (gh, cyc)
        mg.close()
    for p in range(6):
        cj, cc = int(res["jacobi"][1][p]), int(res["cnn"][1][p])
        assert cc < cj, (p, params[p], cc, cj)
        fj = (res["jacobi"][0][p][cj] / res["jacobi"][0][p][cj // 2]) ** (1.0 / (cj - cj // 2))
        fc = (res["cnn"][0][p][cc] / res["cnn"][0][p][cc // 2]) ** (1.0 / (cc - cc // 2))
        assert fc < fj, (p, fc, fj)
    # the trained network's cycle is the oracle's cycle with the same network
    p = 0
    om = O.Multigrid(O.const_field(n, f32(O.q1_rotated_stencil(*params[p]))))
    om.set_cnn(f32(w.cpu().numpy()))
    k = min(30, int(res["cnn"][1][p]))
    _, oh = om.solve(f32(b[p].cpu().numpy()), rtol=0.0, max_cycles=k)
    rel = np.abs(res["cnn"][0][p][: k + 1] - oh) / oh
    assert rel.max() <= 1e-5, rel.max()


@pytest.mark.parametrize("n,smoother,cycles", [(15, "cnn", 1), (31, "cnn", 2), (31, "jacobi", 1)])
def test_vcycle_coarse_train_step_matches_oracle(n, smoother, cycles):
    """Algorithm 2's objective at one level: the two-grid error propagation whose coarse
    solve is one V-cycle of the (already trained) hierarchy below, loss and gradient vs the
    FP64 oracle (vcycle_cnn_loss_and_grad with coarse_vcycle and its transpose)."""
    nprob, nvec = 3, 4
    params = inputs.rotated_params(80 + n, nprob)
    probs = [{"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": e, "theta": t} for e, t in params]
    z = inputs.gaussian_vectors(81 + n, nprob * nvec, n).reshape(nprob, nvec, n, n)
    p = small_net(9, 0.1)
    nc = (n - 1) // 2
    nsets = 0
    m = nc
    while m > 3:
        nsets += 1
        m = (m - 1) // 2
    sets = [small_net(10 + j, 0.1) for j in range(nsets)]
    batch = T.TwoGridBatch(probs, nvec, 2.0 / 3.0, False, cycles=cycles)
    batch.attach_coarse(torch.from_numpy(np.stack(sets)).cuda() if smoother == "cnn" else None)
    loss, grad = batch.loss_and_grad(torch.from_numpy(p).cuda(), torch.from_numpy(z).cuda().contiguous())
    batch.close()
    lo, go = 0.0, np.zeros(p.size)
    for k, (e, t) in enumerate(params):
        st = O.const_field(n, f32(O.q1_rotated_stencil(e, t)))
        st_c = O.rap(st)
        mgc = O.Multigrid(st_c)
        ker = [O.hypernet_forward(mgc.field(j), f32(sets[j])) if smoother == "cnn" else O.jacobi_kernels(mgc.field(j))
               for j in range(mgc.levels - 1)]
        fwd, adj = O.coarse_vcycle(st_c, ker), O.coarse_vcycle(st_c, ker, transpose=True)
        l1, g1 = O.vcycle_cnn_loss_and_grad(st, f32(p), fwd, adj, f32(z[k]), cycles=cycles)
        lo += l1 / nprob
        go += g1 / nprob
    assert abs(loss.item() - lo) <= 1e-5 * lo, (loss.item(), lo)
    g = grad.double().cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)


def test_per_level_networks_and_transposed_smoothers_in_the_solver():
    """net_params [k, nparams] gives level l the kernels of set min(l, k-1); transpose = 1
    stores the kernels of H^T (per-point problems)."""
    n = 31
    cells = torch.from_numpy(inputs.grf_cells(inputs.SEED_GRF + 60, n)).cuda()
    sets = np.stack([small_net(20 + j, 0.1) for j in range(2)])
    mg = S.MultigridSolver([S.varcoef5(n, cells)], "cnn", torch.from_numpy(sets).cuda())
    mgt = S.MultigridSolver([S.varcoef5(n, cells)], "cnn", torch.from_numpy(sets).cuda(), transpose=True)
    om = O.Multigrid(f32(O.varcoef5_field(n, f32(cells.cpu().numpy()))))
    for l in range(mg.levels - 1):
        Wo = O.hypernet_forward(om.field(l), f32(sets[min(l, 1)]))
        Wg = mg.kernels(0, l).double().cpu().numpy()
        np.testing.assert_allclose(Wg, Wo, rtol=2e-5, atol=2e-6 * np.abs(Wo).max())
        np.testing.assert_array_equal(mgt.kernels(0, l).cpu().numpy(), O.transpose_kernels(Wg).astype(np.float32))


@pytest.mark.parametrize("n", [15])
def test_adaptive_trainer_levels_train(n):
    """Algorithm 2 end to end on a small hierarchy: every level's objective falls."""
    tr = T.AdaptiveTrainer(n_fine=n, per_size=4, nvec=4, steps_per_level=40, lr=3e-3)
    tr.train()
    assert sorted(tr.params) == [7, 15]
    for m, h in tr.losses.items():
        assert np.mean(h[-5:]) < np.mean(h[:5]), (m, h[:5], h[-5:])
    assert tr.hierarchy_params(63).shape == (4, T.NPARAMS)


def test_adaptive_per_level_networks_gain_over_shared_network_and_jacobi():
    """The per-level networks of Algorithm 2 (weights/cnn_rotated_adaptive.npy, trained by
    AdaptiveTrainer on 63^2 hierarchies) on held-out rotated problems at 255^2: fewer mean
    cycles to 1e-8 than the shared network, which needs fewer than Jacobi; one problem's
    residual history matches the oracle run with the same per-level kernels."""
    import os

    root = os.path.dirname(T.__file__)
    Wa = np.load(os.path.join(root, "weights", "cnn_rotated_adaptive.npy")).astype(np.float32)
    Ws = np.load(os.path.join(root, "weights", "cnn_rotated.npy")).astype(np.float32)
    n, count = 255, 8
    params = inputs.rotated_params(inputs.SEED_PARAMS + 211, count)
    probs = [S.rotated(n, e, t) for e, t in params]
    b = torch.from_numpy(np.stack([inputs.rhs_uniform(inputs.SEED_RHS + 1200 + i, n) for i in range(count)]))
    b = b.cuda().contiguous()
    pa = T.adaptive_params(Wa, n)
    cyc = {}
    for name, kind, net in (("jacobi", "jacobi", None), ("shared", "cnn", torch.from_numpy(Ws).cuda()),
                            ("adaptive", "cnn", pa.cuda())):
        mg = S.MultigridSolver(probs, kind, net_params=net)
        _, _, gh, c, st = mg.solve(b, rtol=1e-8, max_cycles=5000)
        assert st == B.MG_OK
        cyc[name] = c.astype(np.float64)
        if name == "adaptive":
            hist0 = gh[0]
        mg.close()
    assert cyc["adaptive"].mean() < cyc["shared"].mean() < cyc["jacobi"].mean(), {k: v.mean() for k, v in cyc.items()}
    # oracle with the same per-level kernels (first 40 cycles of problem 0)
    om = O.Multigrid(O.const_field(n, f32(O.q1_rotated_stencil(*params[0]))))
    for l in range(om.levels - 1):
        om.set_kernels(l, O.hypernet_forward(om.field(l), f32(pa[l].numpy())))
    _, oh = om.solve(f32(b[0].cpu().numpy()), rtol=0.0, max_cycles=40)
    k = min(41, int(np.count_nonzero(~np.isnan(hist0))))
    rel = np.abs(hist0[:k] - oh[:k]) / oh[:k]
    assert rel.max() <= 1e-5, rel.max()


# ------------------------------------------------------------ fully connected network
def _fc_params(seed, scale=0.1):
    return (np.random.default_rng(seed).standard_normal(6800) * scale).astype(np.float32)


@pytest.mark.parametrize("kind", ["rotated", "varcoef"])
def test_fc_kernels_match_oracle_on_every_level(kind):
    """The fully connected network's kernels in a solver context (class tables for constant
    stencils, per-point for fields) against the oracle's network on every level's field."""
    n = 31
    p = _fc_params(40)
    if kind == "rotated":
        prob = S.rotated(n, 0.03, 2.0)
        st0 = O.const_field(n, f32(O.q1_rotated_stencil(0.03, 2.0)))
    else:
        cells = inputs.grf_cells(inputs.SEED_GRF + 70, n)
        prob = S.varcoef5(n, torch.from_numpy(cells).cuda())
        st0 = f32(O.varcoef5_field(n, f32(cells)))
    mg = S.MultigridSolver([prob], "cnn", torch.from_numpy(p).cuda(), net_arch="fc")
    om = O.Multigrid(st0)
    for l in range(mg.levels - 1):
        Wg = mg.kernels(0, l).double().cpu().numpy()
        Wo = O.fc_forward(om.field(l), f32(p))
        np.testing.assert_allclose(Wg, Wo, rtol=2e-5, atol=2e-5 * np.abs(Wo).max())


def _bf16_agree(Wg, Wo):
    """Kernels from bfloat16 networks: the two sides round FP32 (tensor-core or FP32-pipe
    sums) and FP64 (oracle) pre-activations to bfloat16 and agree except where a value lies
    within an FP32 rounding of a bfloat16 boundary; there one activation moves by one
    bfloat16 step.  Returns the fraction of outputs within 2e-5 of the scale and the
    largest difference over the scale."""
    scale = np.abs(Wo).max()
    err = np.abs(Wg - Wo)
    return float(np.mean(err <= 2e-5 * scale)), float(err.max() / scale)


@pytest.mark.parametrize("n", [45, 70])
def test_fc_bf16_tensor_core_forward_matches_oracle(n):
    """The fully connected network in bfloat16 mode runs its four GEMMs on the tensor cores
    (tcgen05.mma, M = 128 points per tile, FP32 accumulation in tensor memory): per-point
    kernels of a GRF field and of a constant stencil (tiles of 8 x 16 points with ragged
    edges) against the oracle's bfloat16 emulation of the same network."""
    fields = np.stack([varcoef_field(n, 13), f32(O.const_field(n, O.q1_rotated_stencil(0.02, 0.9)))])
    p = _fc_params(42, 0.1)
    ft = torch.from_numpy(fields.astype(np.float32)).cuda().contiguous()
    W = torch.empty_like(ft)
    B.mg_net_fc_forward(n, 2, ft, torch.from_numpy(p).cuda(), 2.0 / 3.0, 1, W)
    torch.cuda.synchronize()
    Wg = W.double().cpu().numpy()
    for k in range(2):
        frac, mx = _bf16_agree(Wg[k], O.fc_forward(fields[k], f32(p), 2.0 / 3.0, bf16=True))
        print("fc tc agreement", n, k, frac, mx)
        assert frac > 0.95 and mx <= 2e-2, (frac, mx)


@pytest.mark.parametrize("kind", ["rotated", "varcoef"])
def test_fc_bf16_tensor_core_kernels_in_the_solver(kind):
    """mg_setup with the fully connected network in bfloat16 (tensor cores): class tables of
    a constant stencil and per-point kernels of a GRF field on every level, against the
    oracle's bfloat16 network on that level's own FP64 field."""
    n = 63
    p = _fc_params(43, 0.1)
    if kind == "rotated":
        prob = S.rotated(n, 0.03, 2.0)
        st0 = O.const_field(n, f32(O.q1_rotated_stencil(0.03, 2.0)))
    else:
        cells = inputs.grf_cells(inputs.SEED_GRF + 71, n)
        prob = S.varcoef5(n, torch.from_numpy(cells).cuda())
        st0 = f32(O.varcoef5_field(n, f32(cells)))
    mg = S.MultigridSolver([prob], "cnn", torch.from_numpy(p).cuda(), net_arch="fc", conv_bf16=True)
    om = O.Multigrid(st0)
    for l in range(mg.levels - 1):
        frac, mx = _bf16_agree(mg.kernels(0, l).double().cpu().numpy(), O.fc_forward(om.field(l), f32(p), bf16=True))
        print("fc tc solver agreement", kind, l, frac, mx)
        assert frac > 0.95 and mx <= 2e-2, (l, frac, mx)
    mg.close()


@pytest.mark.parametrize("n,bf16", [(15, False), (31, False), (15, True)])
def test_fc_train_step_matches_oracle(n, bf16):
    """Loss and gradient of the two-grid objective through the fully connected network."""
    nprob, nvec = 3, 4
    params = inputs.rotated_params(120 + n, nprob)
    probs = [{"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": e, "theta": t} for e, t in params]
    z = inputs.gaussian_vectors(121 + n, nprob * nvec, n).reshape(nprob, nvec, n, n)
    p = _fc_params(41, 0.05)
    batch = T.TwoGridBatch(probs, nvec, 2.0 / 3.0, bf16, net_arch="fc")
    loss, grad = batch.loss_and_grad(torch.from_numpy(p).cuda(), torch.from_numpy(z).cuda().contiguous())
    batch.close()
    lo, go = 0.0, np.zeros(p.size)
    for k, (e, t) in enumerate(params):
        st = O.const_field(n, f32(O.q1_rotated_stencil(e, t)))
        l1, g1 = O.fc_loss_and_grad(st, f32(p), f32(z[k]), bf16=bf16)
        lo += l1 / nprob
        go += g1 / nprob
    assert abs(loss.item() - lo) <= 1e-5 * lo, (loss.item(), lo)
    g = grad.double().cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)


def test_fc_trainer_reduces_the_loss():
    tr = T.Trainer(sizes=(15,), per_size=8, nvec=8, lr=1e-3, net_arch="fc")
    losses = [tr.step() for _ in range(60)]
    assert np.mean(losses[-10:]) < 0.8 * np.mean(losses[:10]), (losses[:5], losses[-5:])
