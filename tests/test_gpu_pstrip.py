"""The paired warp-strip down-sweep (tile_shape "pstrip") against the 32 x 32 tiles and the
FP64 oracle.

Both layouts perform each point's operations of the pre-smoothing, the residual and the
restriction (Algorithm 1, pre-smoothing and restriction) in the same order, so solves with
either give the same iterate and residual history bit for bit.  The sizes below make the
strips' walks span several 60-column bands with a ragged last band, several segments of the
per-launch height with a ragged last segment (one problem: 8-row walks; sixteen: one wave
of walks about 128 rows high), rows within the network's edge margin, and batches whose
problems leave the launches at different cycles.  By default the strips take only launches
whose walks are at least 32 rows high (the tiles take the rest); most tests lower that
bound to 0 (mg_debug_strip_rows) so that every launch of the cycle runs the strips.
"""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2102_12071_gb300 import binding as B
from paper_2102_12071_gb300 import inputs
from paper_2102_12071_gb300 import solver as S
from paper_2102_12071_gb300 import train as T

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(S.__file__), "weights")


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


def _net(kind, n):
    if kind == "jacobi":
        return None
    if kind == "cnn":
        return torch.from_numpy(small_net(3)).cuda()
    path = os.path.join(WEIGHTS, "cnn_rotated_adaptive.npy")
    if not os.path.exists(path):
        pytest.skip("no per-level networks in the package")
    return T.adaptive_params(np.load(path), n).cuda()


def _solve(n, count, kind, shape, cycles, rtol=0.0, ct=True, seed=0, strip_rows=0):
    params = inputs.rotated_params(inputs.SEED_PARAMS + 50 + seed, count, eps_lo=0.05)
    probs = [S.rotated(n, e, t) for e, t in params]
    net = _net(kind, n)
    mg = S.MultigridSolver(probs, "jacobi" if kind == "jacobi" else "cnn", net, cluster_tail=ct, tile_shape=shape)
    B.mg_debug_strip_rows(mg.ctx, strip_rows)
    b = torch.from_numpy(np.stack([inputs.rhs_uniform(inputs.SEED_RHS + 900 + seed + i, n) for i in range(count)]))
    xh, xl, gh, cyc, st = mg.solve(b.cuda().contiguous(), rtol=rtol, max_cycles=cycles)
    out = (xh.clone(), xl.clone(), np.array(gh), np.array(cyc), st)
    mg.close()
    return out, params, b


@pytest.mark.parametrize("n,count,kind,cycles,rows", [(255, 3, "jacobi", 6, 0), (255, 5, "cnn", 6, 0),
                                                      (511, 4, "adaptive", 4, 0), (1023, 1, "adaptive", 3, 0),
                                                      (1023, 16, "adaptive", 2, 0), (1023, 16, "jacobi", 2, 0),
                                                      (1023, 16, "adaptive", 3, 32), (2047, 4, "jacobi", 2, 32)])
def test_pstrip_equals_tiles_bit_for_bit(n, count, kind, cycles, rows):
    a, _, _ = _solve(n, count, kind, "pstrip", cycles, strip_rows=rows)
    t, _, _ = _solve(n, count, kind, "32x32", cycles)
    assert np.array_equal(a[3], t[3])
    assert np.array_equal(a[2], t[2], equal_nan=True)
    assert torch.equal(a[0], t[0]) and torch.equal(a[1], t[1])


@pytest.mark.parametrize("ct", [True, False])
def test_pstrip_batches_that_drop_out_equal_tiles(ct):
    """Problems stop at different cycles, so the launches' active lists change between
    cycles; both layouts stop each problem at the same cycle with the same iterate."""
    a, _, _ = _solve(255, 5, "adaptive", "pstrip", 3000, rtol=1e-8, ct=ct, seed=7)
    t, _, _ = _solve(255, 5, "adaptive", "32x32", 3000, rtol=1e-8, ct=ct, seed=7)
    assert a[4] == B.MG_OK and t[4] == B.MG_OK
    assert len(set(a[3].tolist())) > 1
    assert np.array_equal(a[3], t[3])
    assert torch.equal(a[0], t[0]) and torch.equal(a[1], t[1])


def test_pstrip_cnn_history_matches_oracle():
    n, cycles, eps, theta = 255, 25, 0.05, 0.7
    p = small_net(3)
    b = inputs.rhs_uniform(7, n)
    mg = S.MultigridSolver([S.rotated(n, eps, theta)], "cnn", torch.from_numpy(p).cuda(), tile_shape="pstrip")
    B.mg_debug_strip_rows(mg.ctx, 0)
    _, _, gh, cyc, _ = mg.solve(torch.from_numpy(b).cuda()[None].contiguous(), rtol=0.0, max_cycles=cycles)
    mg.close()
    om = O.Multigrid(O.const_field(n, f32(O.q1_rotated_stencil(eps, theta))))
    om.set_cnn(f32(p))
    _, oh = om.solve(f32(b), rtol=0.0, max_cycles=cycles)
    assert cyc[0] == cycles
    rel = np.abs(gh[0][: cycles + 1] - oh) / oh
    assert rel.max() <= 1e-5, rel.max()


def test_pstrip_timeout_status_and_recovery():
    """The test setting makes every warp's first bounded wait give up at once; each warp
    then waits, with the full bound, for the copies it has in flight before it exits.  The
    solve reports MG_ERR_TIMEOUT, and the same context then solves like the tiles."""
    n, cycles = 255, 8
    params = inputs.rotated_params(inputs.SEED_PARAMS + 77, 2, eps_lo=0.05)
    b = torch.from_numpy(np.stack([inputs.rhs_uniform(15 + i, n) for i in range(2)])).cuda().contiguous()
    mg = S.MultigridSolver([S.rotated(n, e, t) for e, t in params], tile_shape="pstrip")
    B.mg_debug_strip_rows(mg.ctx, 0)
    B.mg_debug_short_wait(mg.ctx, True)
    with pytest.raises(B.MGError) as ei:
        mg.solve(b, rtol=1e-8, max_cycles=cycles)
    assert ei.value.status == B.MG_ERR_TIMEOUT
    B.mg_debug_short_wait(mg.ctx, False)
    xh, _, gh, cyc, st = mg.solve(b, rtol=0.0, max_cycles=cycles)
    mg.close()
    assert st == B.MG_ERR_NOT_CONVERGED and np.all(cyc == cycles)
    ref = S.MultigridSolver([S.rotated(n, e, t) for e, t in params], tile_shape="32x32")
    xr, _, ghr, _, _ = ref.solve(b, rtol=0.0, max_cycles=cycles)
    ref.close()
    assert torch.equal(xh, xr) and np.array_equal(np.array(gh), np.array(ghr), equal_nan=True)


def test_pstrip_on_field_problems_keeps_tiles():
    """Per-point stencils have no paired strip kernel: the shape falls back to the 32 x 32
    tiles and the solve equals theirs."""
    n = 127
    cells = torch.from_numpy(inputs.grf_cells(inputs.SEED_GRF + 5, n)).cuda()
    b = torch.from_numpy(inputs.rhs_uniform(inputs.SEED_RHS + 5, n)).cuda()[None].contiguous()
    out = []
    for shape in ("pstrip", "32x32"):
        mg = S.MultigridSolver([S.varcoef5(n, cells)], tile_shape=shape)
        B.mg_debug_strip_rows(mg.ctx, 0)
        xh, _, gh, cyc, _ = mg.solve(b, rtol=0.0, max_cycles=5)
        out.append((xh.clone(), np.array(gh)))
        mg.close()
    assert torch.equal(out[0][0], out[1][0])
