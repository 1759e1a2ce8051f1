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


def test_stack_network_is_not_trained_here():
    from paper_2102_12071_gb300 import train as T

    with pytest.raises(B.MGError):
        T.TwoGridBatch([S.rotated(15, 0.1, 0.2)], 2, net_arch="conv3")
