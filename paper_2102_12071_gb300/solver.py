"""User-facing wrapper: owns the torch-allocated workspace of one multigrid context.

All computation runs in libmgcnn.so through ``binding``; torch supplies device memory
and the stream.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def rotated(n: int, eps: float, theta: float) -> dict:
    return {"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": float(eps), "theta": float(theta)}


def stencil(n: int, s) -> dict:
    return {"n": n, "kind": B.MG_PROBLEM_STENCIL, "data": [float(v) for v in np.asarray(s).reshape(9)]}


def varcoef5(n: int, cells: torch.Tensor) -> dict:
    assert cells.is_cuda and cells.dtype == torch.float32 and cells.shape == (n + 1, n + 1)
    return {"n": n, "kind": B.MG_PROBLEM_VARCOEF5, "data": cells.contiguous()}


def field(n: int, st: torch.Tensor) -> dict:
    assert st.is_cuda and st.dtype == torch.float32 and st.shape == (9, n, n)
    return {"n": n, "kind": B.MG_PROBLEM_FIELD, "data": st.contiguous()}


def net_arch_code(net_arch: str) -> int:
    codes = {"conv": B.MG_NET_CONV, "fc": B.MG_NET_FC, "linear": B.MG_NET_LINEAR, "conv3": B.MG_NET_CONV3,
             "conv_shared": B.MG_NET_CONV_SHARED}
    if net_arch not in codes:
        raise ValueError(f"unknown net_arch {net_arch!r}")
    return codes[net_arch]


class MultigridSolver:
    """Hierarchy + V-cycle solver for a batch of same-size problems on one GPU."""

    def __init__(self, problems: list[dict], smoother: str = "jacobi", net_params: torch.Tensor | None = None,
                 omega: float = 2.0 / 3.0, conv_bf16: bool = False, coarsest_n: int = 3, device="cuda",
                 stream=None, cluster_tail: bool = True, transpose: bool = False, net_arch: str = "conv",
                 per_problem: bool = False, nu1: int = 1, nu2: int = 1, tile_shape: str | int = 0):
        """net_params: one parameter set [nparams] for every level, or per-level sets
        [k, nparams] (level l uses set min(l, k - 1)).  transpose: smooth with H^T (per-point
        problems), so that a V-cycle applies the transpose of the cycle without it.
        net_arch: "conv" (the convolutional network), "conv3" (the same with three output
        kernels applied as a stack, Sec. 4.2), "fc" (the fully connected one) or
        "linear" (the shared-kernel linear smoother of Sec. 6: net_params are its six 3x3
        kernels per level, [54] or [k, 54]; with per_problem, one group of k sets per
        problem, [nprob, k, 54], as Sec. 6 trains one smoother per problem).  nu1, nu2:
        smoothing steps before / after the coarse correction (> 1 for Jacobi and the linear
        smoother; the paper's cost-equalised Jacobi runs six).  tile_shape: layout of the
        kernels of the levels above the coarse tail, a name of binding.TILE_SHAPES or 0 for
        the library's default; it changes speed, not the cycle."""
        self.nprob = len(problems)
        self.n = problems[0]["n"]
        self.device = torch.device(device)
        self.stream = stream
        self._probs, self._keep = B.problems_array(problems)
        kind = B.MG_SMOOTH_CNN if smoother == "cnn" else B.MG_SMOOTH_JACOBI
        if per_problem:
            assert net_arch == "linear" and net_params is not None and net_params.shape[0] == self.nprob
            net_params = net_params.reshape(self.nprob, -1, 54)
            net_levels = int(net_params.shape[1])
            net_params = net_params.reshape(-1, 54)
        elif net_arch == "linear" and net_params is not None:
            # sets of six 3x3 kernels: [54], [6, 9], [k, 54] or [k, 6, 9] all mean k >= 1 sets
            net_params = net_params.reshape(-1, 54)
            net_levels = int(net_params.shape[0]) if net_params.shape[0] > 1 else 0
        else:
            net_levels = int(net_params.shape[0]) if net_params is not None and net_params.dim() == 2 else 0
        arch = net_arch_code(net_arch)
        shape = B.TILE_SHAPES[tile_shape] if isinstance(tile_shape, str) else int(tile_shape)
        self.opts = B.options(kind, omega, coarsest_n, int(conv_bf16), int(cluster_tail), 1, 0, net_levels,
                              int(transpose), arch, int(per_problem), int(nu1), int(nu2), shape)
        size = B.mg_workspace_size(self._probs, self.nprob, self.opts)
        if size == 0:
            raise B.MGError(B.MG_ERR_INVALID_ARG, "mg_workspace_size", B.lib().mg_last_error().decode())
        self.workspace = torch.empty(size, dtype=torch.uint8, device=self.device)
        if net_params is not None:
            net_params = net_params.to(self.device, torch.float32).contiguous()
        self.ctx = B.mg_setup(self._probs, self.nprob, self.opts, net_params, self.workspace, size, stream)
        self.levels = B.mg_num_levels(self.ctx)
        self.sizes = [B.mg_level_n(self.ctx, l) for l in range(self.levels)]

    def close(self):
        if getattr(self, "ctx", None):
            B.mg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    # ------------------------------------------------------------ inspection
    def stencil_field(self, prob: int, level: int) -> torch.Tensor:
        n = self.sizes[level]
        out = torch.empty((9, n, n), dtype=torch.float32, device=self.device)
        B.mg_get_stencil(self.ctx, prob, level, out, self.stream)
        return out

    def kernels(self, prob: int, level: int) -> torch.Tensor:
        n = self.sizes[level]
        out = torch.empty((9, n, n), dtype=torch.float32, device=self.device)
        B.mg_get_kernels(self.ctx, prob, level, out, self.stream)
        return out

    # ------------------------------------------------------------ solving
    def smooth(self, prob: int, level: int, f: torch.Tensor, u: torch.Tensor, nsteps: int = 1) -> None:
        B.mg_smoother_apply(self.ctx, prob, level, f, u, nsteps, self.stream)

    def vcycle(self, b: torch.Tensor, x_hi: torch.Tensor, x_lo: torch.Tensor | None = None,
               rel: torch.Tensor | None = None) -> None:
        B.mg_vcycle(self.ctx, b, x_hi, x_lo, rel, self.stream)

    def solve(self, b: torch.Tensor, x_hi: torch.Tensor | None = None, x_lo: torch.Tensor | None = None,
              rtol: float = 1e-8, max_cycles: int = 1000, history: bool = True):
        """Returns (x_hi, x_lo, hist [nprob, max_cycles+1] float64 (nan past the end), cycles, status)."""
        shape = (self.nprob, self.n, self.n)
        assert b.shape == shape and b.dtype == torch.float32 and b.is_contiguous()
        if x_hi is None:
            x_hi = torch.zeros(shape, dtype=torch.float32, device=self.device)
        if x_lo is None:
            x_lo = torch.zeros(shape, dtype=torch.float32, device=self.device)
        hist = np.full((self.nprob, max_cycles + 1), np.nan) if history else None
        cycles = np.zeros(self.nprob, dtype=np.int32)
        st = B.mg_solve(self.ctx, b, x_hi, x_lo, rtol, max_cycles, hist, cycles, self.stream)
        return x_hi, x_lo, hist, cycles, st


def fgmres(mg: "MultigridSolver", b: torch.Tensor, x_hi: torch.Tensor | None = None, x_lo: torch.Tensor | None = None,
           restart: int = 30, rtol: float = 1e-6, max_iters: int = 500, history: bool = True):
    """Flexible GMRES with one V-cycle of `mg` as the preconditioner (Sec. 6.4).
    Returns (x_hi, x_lo, hist [nprob, max_iters+1] (nan past the end), iterations, status)."""
    shape = (mg.nprob, mg.n, mg.n)
    assert b.shape == shape and b.dtype == torch.float32 and b.is_contiguous()
    x_hi = torch.zeros(shape, dtype=torch.float32, device=mg.device) if x_hi is None else x_hi
    x_lo = torch.zeros(shape, dtype=torch.float32, device=mg.device) if x_lo is None else x_lo
    size = B.mg_fgmres_workspace_size(mg.ctx, restart)
    ws = torch.empty(size, dtype=torch.uint8, device=mg.device)
    hist = np.full((mg.nprob, max_iters + 1), np.nan) if history else None
    iters = np.zeros(mg.nprob, dtype=np.int32)
    st = B.mg_fgmres(mg.ctx, b, x_hi, x_lo, restart, rtol, max_iters, ws, size, hist, iters, mg.stream)
    return x_hi, x_lo, hist, iters, st


def net_forward(fields: torch.Tensor, params: torch.Tensor, omega: float = 2.0 / 3.0,
                conv_bf16: bool = False) -> torch.Tensor:
    """Per-point smoothing kernels for a batch of stencil fields [nprob, 9, n, n]."""
    nprob, nine, n, _ = fields.shape
    assert nine == 9
    W = torch.empty_like(fields)
    B.mg_net_forward(n, nprob, fields.contiguous(), params.contiguous(), omega, int(conv_bf16), W)
    return W


class MixedBatchSolver:
    """Problems of different sizes and stencil storage in one solve.

    A context holds problems of one size and one storage kind (constant stencils or per-point
    fields), so the batch is split into such groups; every group gets its own context and
    CUDA stream, and mg_solve_multi runs all groups' cycles at once.  net_params maps "const"
    and "field" to the network parameters of each kind (CNN smoother): one set, per-level
    sets, or a function of the group's side returning either.  With `autotune`, the
    first solve times a few cycles of every candidate layout per group -- the coarse-level
    layout (the coarse levels in one CTA cluster per problem -- from 63 with the network
    smoothers on grids of side >= 1023, else from 127 -- or from 63 in one CTA, tiled kernels
    above) crossed with the tile shape of the tiled down-sweeps (`shapes`, names of
    binding.TILE_SHAPES) -- and keeps the fastest; without it the first candidate is used.
    After a solve, `last_times_ms[i]` is problem i's time to its stopping test, from the
    start of the earliest group (GPU timer stamps, mg_solve_times).
    """

    SHAPES = ("pstrip", "32x32", "strip4x32", "strip8x32")

    def __init__(self, problems: list[dict], smoother: str = "jacobi", net_params: dict | None = None,
                 autotune: bool = True, tune_cycles: int = 16, shapes=None, layouts=(True, False)):
        self.problems = problems
        self.smoother = smoother
        self.net_params = net_params or {}
        self.autotune = autotune
        self.tune_cycles = tune_cycles
        self.shapes = tuple(shapes) if shapes else self.SHAPES
        self.layouts = tuple(layouts)
        self.last_times_ms = None
        self.groups: dict[tuple, list[int]] = {}
        for i, p in enumerate(problems):
            field = p["kind"] in (B.MG_PROBLEM_VARCOEF5, B.MG_PROBLEM_FIELD)
            self.groups.setdefault((p["n"], "field" if field else "const"), []).append(i)
        self.solvers: dict[tuple, MultigridSolver] = {}
        self.streams: dict[tuple, torch.cuda.Stream] = {key: torch.cuda.Stream() for key in self.groups}
        self.layout: dict[tuple, tuple] = {}  # group -> (cluster_tail, tile shape) in use

    def _make(self, key, cluster_tail: bool, shape: str) -> MultigridSolver:
        params = self.net_params.get(key[1]) if self.smoother == "cnn" else None
        if callable(params):  # per-level sets that depend on the hierarchy's size
            params = params(key[0])
        return MultigridSolver([self.problems[i] for i in self.groups[key]], self.smoother, net_params=params,
                               stream=self.streams[key].cuda_stream, cluster_tail=cluster_tail, tile_shape=shape)

    def _tune(self, key, b: torch.Tensor) -> MultigridSolver:
        cands = [(ct, sh) for ct in self.layouts for sh in self.shapes]
        if not self.autotune or key[0] <= 63:  # <= 63: whole solves in one CTA, nothing to choose
            self.layout[key] = cands[0]
            return self._make(key, *cands[0])
        best = None
        for ct, sh in cands:
            mg = self._make(key, ct, sh)
            with torch.cuda.stream(self.streams[key]):
                for _ in range(2):
                    mg.solve(b, rtol=0.0, max_cycles=self.tune_cycles, history=False)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                mg.solve(b, rtol=0.0, max_cycles=self.tune_cycles, history=False)
                e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            if best is None or ms < best[0]:
                if best is not None:
                    best[1].close()
                best = (ms, mg, (ct, sh))
            else:
                mg.close()
        self.layout[key] = best[2]
        return best[1]

    def group_b(self, b: list[torch.Tensor]) -> dict[tuple, torch.Tensor]:
        return {key: torch.stack([b[i] for i in idx]).contiguous() for key, idx in self.groups.items()}

    def solve(self, b: list[torch.Tensor], rtol: float = 1e-8, max_cycles: int = 20000):
        """b: one [n, n] device tensor per problem.  Returns (x_hi list, cycles int32 array, status)."""
        gb = self.group_b(b)
        for key in self.groups:
            if key not in self.solvers:
                self.solvers[key] = self._tune(key, gb[key])
        keys = list(self.groups)
        torch.cuda.synchronize()
        xh = {k: torch.zeros_like(gb[k]) for k in keys}
        xl = {k: torch.zeros_like(gb[k]) for k in keys}
        cyc = {k: np.zeros(len(self.groups[k]), dtype=np.int32) for k in keys}
        st = B.mg_solve_multi([self.solvers[k].ctx for k in keys], [gb[k] for k in keys], [xh[k] for k in keys],
                              [xl[k] for k in keys], rtol, max_cycles, [cyc[k] for k in keys],
                              [self.streams[k].cuda_stream for k in keys])
        x = [None] * len(self.problems)
        cycles = np.zeros(len(self.problems), dtype=np.int32)
        stamps = {k: B.mg_solve_times(self.solvers[k].ctx, len(self.groups[k])) for k in keys}
        t0 = min(int(stamps[k][0].min()) for k in keys)
        self.last_times_ms = np.full(len(self.problems), np.nan)
        for k in keys:
            for j, i in enumerate(self.groups[k]):
                x[i] = xh[k][j]
                cycles[i] = cyc[k][j]
                if stamps[k][1][j]:
                    self.last_times_ms[i] = (int(stamps[k][1][j]) - t0) / 1e6
        return x, cycles, st

    def close(self):
        for mg in self.solvers.values():
            mg.close()
        self.solvers = {}
