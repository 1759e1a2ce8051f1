"""The workspace-free solve entry point against the regular one (GPU).

mg_solve_small_static serves callers that cannot allocate device memory (a host
framework's allocator owns the GPU, a fixed memory budget, or no room for cudaMalloc's
synchronisation).  It must give what mg_workspace_size + mg_setup + mg_solve give, call
after call, although every call reuses the same scratch array inside the library.  This
file is collected last so that a run stopping at the first failure has run everything
else first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2102_12071_gb300 import binding as B
from paper_2102_12071_gb300 import inputs
from paper_2102_12071_gb300 import solver as S

pytestmark = pytest.mark.gpu

HIST_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2102_12071_gb300 import build

    build.build()


def _regular(problems, b, rtol, max_cycles, with_lo=True):
    """mg_workspace_size + mg_setup + mg_solve; without x_lo the low part lives in the
    context's workspace and only x_hi comes back."""
    mg = S.MultigridSolver(problems, "jacobi")
    x_hi = torch.zeros_like(b)
    x_lo = torch.zeros_like(b) if with_lo else None
    hist = np.full((len(problems), max_cycles + 1), np.nan)
    cyc = np.zeros(len(problems), dtype=np.int32)
    st = B.mg_solve(mg.ctx, b, x_hi, x_lo, rtol, max_cycles, hist, cyc, mg.stream)
    torch.cuda.synchronize()
    mg.close()
    return x_hi, x_lo, hist, cyc, st


def _static(problems, b, rtol, max_cycles, with_lo=True):
    """without x_lo the low part lives in the library's scratch array, which keeps the
    previous call's contents: the entry point must clear it itself"""
    probs, keep = B.problems_array(problems)
    x_hi = torch.zeros_like(b)
    x_lo = torch.zeros_like(b) if with_lo else None
    hist = np.full((len(problems), max_cycles + 1), np.nan)
    cyc = np.zeros(len(problems), dtype=np.int32)
    st = B.mg_solve_small_static(probs, len(problems), B.options(), b, x_hi, x_lo, rtol, max_cycles, hist, cyc)
    torch.cuda.synchronize()
    del keep
    return x_hi, x_lo, hist, cyc, st


def _same(got, want, count, with_lo=True):
    assert got[4] == want[4]
    np.testing.assert_array_equal(got[3], want[3])
    for p in range(count):
        k = int(want[3][p]) + 1
        rel = np.abs(got[2][p][:k] - want[2][p][:k]) / want[2][p][:k]
        assert rel.max() <= HIST_RTOL
    x_got = got[0].double() + (got[1].double() if with_lo else 0.0)
    x_want = want[0].double() + (want[1].double() if with_lo else 0.0)
    assert (x_got - x_want).abs().max().item() <= 1e-6 * x_want.abs().max().item()


def _batch(n, count, seed):
    params = inputs.rotated_params(seed, count)
    problems = [S.rotated(n, e, t) for e, t in params]
    b = torch.from_numpy(np.stack([inputs.rhs_uniform(seed + 100 + i, n) for i in range(count)])).cuda().contiguous()
    return problems, b


def test_static_solve_matches_regular_solve_twice_in_a_row():
    # two consecutive calls with different sizes and batch counts share the scratch array
    for n, count, seed, rtol, cap in ((63, 3, 500, 1e-8, 3000), (31, 5, 600, 1e-6, 3000)):
        problems, b = _batch(n, count, seed)
        want = _regular(problems, b, rtol, cap)
        got = _static(problems, b, rtol, cap)
        _same(got, want, count)


def test_static_solve_without_low_part_twice_in_a_row():
    # x_lo = NULL: the float-float low part is kept in the scratch array's own region, which
    # the first call leaves non-zero; the second call must start it from zero again
    for n, count, seed, rtol, cap in ((63, 4, 900, 1e-8, 3000), (63, 4, 900, 1e-8, 3000), (15, 2, 950, 1e-8, 500)):
        problems, b = _batch(n, count, seed)
        want = _regular(problems, b, rtol, cap, with_lo=False)
        got = _static(problems, b, rtol, cap, with_lo=False)
        _same(got, want, count, with_lo=False)


def test_static_solve_rejects_requests_beyond_its_scratch():
    problems, b = _batch(127, 1, 700)
    probs, _ = B.problems_array(problems)
    x = torch.zeros_like(b)
    st = B.lib().mg_solve_small_static(probs, 1, B.options(), b.data_ptr(), x.data_ptr(), None, 1e-8, 10, None, None,
                                       None)
    assert st == B.MG_ERR_INVALID_ARG
    assert b"[3, 63]" in B.lib().mg_last_error()
    problems, b = _batch(31, B_MAX + 1, 800)
    probs, _ = B.problems_array(problems)
    x = torch.zeros_like(b)
    st = B.lib().mg_solve_small_static(probs, B_MAX + 1, B.options(), b.data_ptr(), x.data_ptr(), None, 1e-8, 10,
                                       None, None, None)
    assert st == B.MG_ERR_INVALID_ARG


B_MAX = 16
