"""GPU parity of the configurations the benchmark times, through the C ABI against the FP64
oracle: the headline batch with the per-level networks of Algorithm 2, and the asymptotic
convergence factor of the learned smoothers.

Tolerances: per-cycle relative residual within 1e-5 relative; asymptotic convergence
factor within 1e-3 relative; cycle counts to 1e-8 within one cycle.
"""
import functools
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from oracle import linear as OL
from paper_2102_12071_gb300 import binding as B
from paper_2102_12071_gb300 import inputs
from paper_2102_12071_gb300 import solver as S
from paper_2102_12071_gb300 import train as T

pytestmark = pytest.mark.gpu

HIST_RTOL = 1e-5
FACTOR_RTOL = 1e-3
WEIGHTS = os.path.join(os.path.dirname(S.__file__), "weights")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2102_12071_gb300 import build

    build.build()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _adaptive(n):
    """The committed per-level networks (Algorithm 2 on 63^2 hierarchies) on an n^2 hierarchy."""
    return T.adaptive_params(np.load(os.path.join(WEIGHTS, "cnn_rotated_adaptive.npy")).astype(np.float32), n)


def _oracle_per_level(n, eps, theta, sets):
    om = O.Multigrid(O.const_field(n, f32(O.q1_rotated_stencil(eps, theta))))
    for l in range(om.levels - 1):
        om.set_kernels(l, O.hypernet_forward(om.field(l), f32(sets[min(l, len(sets) - 1)].numpy())))
    return om


N_BENCH, NPROB_BENCH, CYCLES_BENCH = 1023, 16, 4


def _bench_batch():
    """The benchmark's batch: 16 rotated problems at 1023^2, (eps, theta) and rhs seeds of rank 0."""
    params = inputs.rotated_params(inputs.SEED_PARAMS, NPROB_BENCH)
    b = np.stack([inputs.rhs_uniform(inputs.SEED_RHS + i, N_BENCH) for i in range(NPROB_BENCH)])
    return params, b


@functools.lru_cache(maxsize=None)
def _bench_oracle_history(p):
    params, b = _bench_batch()
    om = _oracle_per_level(N_BENCH, *params[p], _adaptive(N_BENCH))
    _, oh = om.solve(f32(b[p]), rtol=0.0, max_cycles=CYCLES_BENCH)
    return oh


@pytest.mark.parametrize("ct", [True, False])
def test_bench_batch_per_level_networks_first_cycles_match_oracle(ct):
    """The headline solve of the benchmark: 16 x 1023^2 with the per-level networks (class
    tables per level, kernels k_down / k_up0 with the CNN smoother), level 0 in 16 384 CTAs,
    i.e. several waves, and the coarse levels in one CTA cluster per problem (ct) or in one
    CTA below tiled kernels.  Problems 0 and 9 (the slowest one) against the oracle run with
    the same per-level networks evaluated on its own FP64 level operators."""
    params, b = _bench_batch()
    mg = S.MultigridSolver([S.rotated(N_BENCH, e, t) for e, t in params], "cnn", _adaptive(N_BENCH).cuda(),
                           cluster_tail=ct)
    _, _, gh, cyc, _ = mg.solve(torch.from_numpy(b).cuda().contiguous(), rtol=0.0, max_cycles=CYCLES_BENCH)
    mg.close()
    assert np.all(cyc == CYCLES_BENCH)
    for p in (0, 9):
        oh = _bench_oracle_history(p)
        rel = np.abs(gh[p][: CYCLES_BENCH + 1] - oh) / oh
        assert rel.max() <= HIST_RTOL, (p, rel.max())


def _factor(h, c, window):
    return (h[c] / h[c - window]) ** (1.0 / window)


N_F, EPS_F, THETA_F = 255, 0.01, math.pi / 6  # C1's operator on a 255^2 grid


@pytest.mark.parametrize("net", ["shared", "per_level"])
def test_cnn_asymptotic_factor_matches_oracle(net):
    """CNN-smoothed V(1,1) to 1e-8 at 255^2 (eps = 0.01, theta = pi/6; ~140 cycles): the
    committed shared network or the per-level networks; cycle count within one of the
    oracle's, the factor over the last 50 cycles within 1e-3 relative, and the first 50
    cycles of the history within 1e-5."""
    b = inputs.rhs_uniform(inputs.SEED_RHS + 4000, N_F)
    if net == "shared":
        w = torch.from_numpy(np.load(os.path.join(WEIGHTS, "cnn_rotated.npy")).astype(np.float32))
        om = O.Multigrid(O.const_field(N_F, f32(O.q1_rotated_stencil(EPS_F, THETA_F))))
        om.set_cnn(f32(w.numpy()))
    else:
        w = _adaptive(N_F)
        om = _oracle_per_level(N_F, EPS_F, THETA_F, w)
    mg = S.MultigridSolver([S.rotated(N_F, EPS_F, THETA_F)], "cnn", w.cuda())
    _, _, gh, cyc, st = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=1e-8, max_cycles=3000)
    mg.close()
    assert st == B.MG_OK
    _, oh = om.solve(f32(b), rtol=1e-8, max_cycles=3000)
    cg, co = int(cyc[0]), len(oh) - 1
    assert co > 100 and abs(cg - co) <= 1, (cg, co)
    fg, fo = _factor(gh[0], cg, 50), _factor(oh, co, 50)
    assert abs(fg - fo) <= FACTOR_RTOL * fo, (fg, fo)
    rel = np.abs(gh[0][:51] - oh[:51]) / oh[:51]
    assert rel.max() <= HIST_RTOL, rel.max()


def test_linear_alpha_cnn_asymptotic_factor_matches_oracle():
    """The paper's alpha-CNN (Sec. 6): the committed per-angle linear shared-kernel smoothers
    of Algorithm 2 (eps = 0.01, theta = pi/6) on a 255^2 hierarchy, to 1e-8 (~35 cycles):
    cycle count within one and the factor over the last 20 cycles within 1e-3 relative."""
    z = np.load(os.path.join(WEIGHTS, "linear_eps0.01.npz"))
    i = int(np.argmin(np.abs(z["thetas"] - THETA_F)))
    assert abs(float(z["thetas"][i]) - THETA_F) < 1e-9 and abs(float(z["eps"]) - EPS_F) < 1e-12
    sets = T.adaptive_params(z["params"][i].astype(np.float32), N_F, int(z["n_fine"]))
    b = inputs.rhs_uniform(inputs.SEED_RHS + 4000, N_F)
    mg = S.MultigridSolver([S.rotated(N_F, EPS_F, THETA_F)], "cnn", sets.cuda(), net_arch="linear")
    _, _, gh, cyc, st = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=1e-8, max_cycles=500)
    mg.close()
    assert st == B.MG_OK
    st0 = O.const_field(N_F, f32(O.q1_rotated_stencil(EPS_F, THETA_F)))
    _, oh = OL.LinearMultigrid(st0, [f32(q) for q in sets.numpy()]).solve(f32(b), rtol=1e-8, max_cycles=500)
    cg, co = int(cyc[0]), len(oh) - 1
    assert co > 25 and abs(cg - co) <= 1, (cg, co)
    fg, fo = _factor(gh[0], cg, 20), _factor(oh, co, 20)
    assert abs(fg - fo) <= FACTOR_RTOL * fo, (fg, fo)
    # The history is the product of the per-cycle reductions, so a per-cycle difference of
    # FP32 size accumulates: the first 20 cycles within 1e-5, and every cycle's reduction
    # h[k] / h[k-1] within 1e-5 to the end.
    rel = np.abs(gh[0][:21] - oh[:21]) / oh[:21]
    assert rel.max() <= HIST_RTOL, rel.max()
    k = min(cg, co) + 1
    qg, qo = gh[0][1:k] / gh[0][: k - 1], oh[1:k] / oh[: k - 1]
    assert np.max(np.abs(qg - qo) / qo) <= HIST_RTOL
