"""GPU parity of the multigrid-preconditioned flexible GMRES (Sec. 6.4) against the FP64
oracle, through the C ABI."""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
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


def _weights():
    root = os.path.dirname(S.__file__)
    return np.load(os.path.join(root, "weights", "cnn_rotated.npy")).astype(np.float32)


@pytest.mark.parametrize("n,smoother", [(63, "jacobi"), (255, "jacobi"), (255, "cnn")])
def test_fgmres_matches_oracle(n, smoother):
    """eps = 0.01 (the paper's xi = 100), theta = pi/12 and pi/4, rtol 1e-6, restart 30:
    iteration counts within two steps and the residual estimates of the first restart cycle
    within 1e-3 relative of the FP64 oracle's (FP32 Krylov vectors and preconditioner); the
    float-float solution's true residual (FP64) meets rtol."""
    thetas = [math.pi / 12, math.pi / 4]
    probs = [S.rotated(n, 0.01, t) for t in thetas]
    b_np = np.stack([inputs.rhs_uniform(inputs.SEED_RHS + 1500 + i, n) for i in range(len(thetas))])
    b = torch.from_numpy(b_np).cuda().contiguous()
    W = _weights() if smoother == "cnn" else None
    mg = S.MultigridSolver(probs, smoother, net_params=torch.from_numpy(W).cuda() if W is not None else None)
    xh, xl, gh, its, st = S.fgmres(mg, b, restart=30, rtol=1e-6, max_iters=200)
    assert st == B.MG_OK
    for p, t in enumerate(thetas):
        st0 = O.const_field(n, f32(O.q1_rotated_stencil(0.01, t)))
        om = O.Multigrid(st0)
        if W is not None:
            om.set_cnn(f32(W))
        xo, oh, oits = O.fgmres(lambda v: O.apply(st0, v), lambda v: om.vcycle(v, np.zeros_like(v)), f32(b_np[p]),
                                restart=30, rtol=1e-6, max_iters=200)
        # a restart boundary can cost two steps when the FP32 estimate lands just above rtol
        assert abs(int(its[p]) - oits) <= 2, (int(its[p]), oits)
        k = min(int(its[p]), oits, 30) + 1  # the first restart cycle
        rel = np.abs(gh[p][:k] - oh[:k]) / oh[:k]
        print(f"n={n} {smoother} theta={t:.3f}: its {int(its[p])} vs {oits}, history rel max {rel.max():.2e}")
        assert rel.max() <= 1e-3, rel.max()
        x = xh[p].double().cpu().numpy() + xl[p].double().cpu().numpy()
        true = np.linalg.norm(f32(b_np[p]) - O.apply(st0, x)) / np.linalg.norm(f32(b_np[p]))
        assert true < 1e-6, true


def test_fgmres_beats_the_vcycle_alone_and_reports_non_convergence():
    n = 127
    probs = [S.rotated(n, 0.01, math.pi / 6)]
    b = torch.from_numpy(inputs.rhs_uniform(inputs.SEED_RHS + 1600, n)).cuda()[None].contiguous()
    mg = S.MultigridSolver(probs, "jacobi")
    _, _, _, its, st = S.fgmres(mg, b, rtol=1e-6)
    _, _, _, cyc, st2 = mg.solve(b, rtol=1e-6, max_cycles=5000)
    assert st == B.MG_OK and st2 == B.MG_OK and its[0] < cyc[0]
    _, _, gh, its, st = S.fgmres(mg, b, rtol=1e-6, max_iters=3)
    assert st == B.MG_ERR_NOT_CONVERGED and its[0] == 3 and np.isnan(gh[0][4:]).all()
