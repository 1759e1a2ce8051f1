"""Training of the stencil-to-smoother network on the two-grid convergence loss.

Sec. 3.2 trains the smoother by minimising the error left by the multigrid cycle on
random initial errors (eq. overalltrain with u_* = 0); Thm. sbound makes the mean of
||E z||^2 over Gaussian z an estimate of ||E||_F^2.  Here E = S C S is the two-grid error
propagation (eq. twogrid, one pre- and one post-smoothing step), evaluated together with
its exact gradient by mg_train_step in the CUDA library.  This module only draws the
problems and vectors, calls the library and applies Adam (Sec. 6: Adam, learning rate
1e-3) to the ~1.3 k network parameters.
"""
from __future__ import annotations

import math
import os

import numpy as np
import torch

from . import binding as B
from . import inputs

NPARAMS = 1260
LAYERS = [(7, 9), (5, 7), (3, 5), (9, 3)]  # (out, in) channels of the 3x3 layers
NPARAMS_FC = 6800
FC_LAYERS = [(40, 81), (40, 40), (40, 40), (9, 40)]  # the fully connected network (out, in)
NPARAMS_LIN = 54  # the shared-kernel linear smoother of one level: six 3x3 kernels
NPARAMS_K3 = 1746  # the convolutional network with three output kernels (FP32)
NPARAMS_SHARED = 378  # one 3x3 kernel per convolution output channel (Sec. 6.2's count)


def nparams(arch: str = "conv") -> int:
    return {"fc": NPARAMS_FC, "linear": NPARAMS_LIN, "conv3": NPARAMS_K3,
            "conv_shared": NPARAMS_SHARED}.get(arch, NPARAMS)


def init_params_shared(seed: int = 0) -> torch.Tensor:
    """The shared-kernel network: output channel o of a convolution is k_o applied to the sum
    of the layer's ci input channels, so its fan-in is 9 ci as for the dense layer (same
    Kaiming bound); the output layer is zero (the network starts at weighted Jacobi)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for k, (co, ci) in enumerate(LAYERS):
        if k == len(LAYERS) - 1:
            parts.append(torch.zeros(co * ci * 9))
        else:
            bound = math.sqrt(6.0 / ((1 + 0.01 ** 2) * ci * 9))
            parts.append((torch.rand(co * 9, generator=g) * 2 - 1) * bound)
    p = torch.cat(parts)
    assert p.numel() == NPARAMS_SHARED
    return p


def init_params_conv3(seed: int = 0) -> torch.Tensor:
    """The three-kernel network: the convolutions of init_params and a zero 27-output layer,
    so K1 = omega/D, K2 = K3 = identity (the stack starts at weighted Jacobi)."""
    p = torch.cat([init_params(seed)[: NPARAMS - 243], torch.zeros(27 * 27)])
    assert p.numel() == NPARAMS_K3
    return p


def init_for(arch: str, seed: int = 0) -> torch.Tensor:
    """Starting parameters of a trainable architecture (all start at weighted Jacobi)."""
    if arch == "fc":
        return init_params_fc(seed)
    if arch == "conv_shared":
        return init_params_shared(seed)
    if arch == "conv3":
        return init_params_conv3(seed)
    return init_params(seed)


def init_params_linear(d: float, omega: float = 2.0 / 3.0) -> torch.Tensor:
    """The linear smoother at weighted Jacobi for diagonal d: f1..f4 the identity kernel,
    f5 zero, f6 = omega/d at the centre.  (Sec. 6 starts f1..f5 at zero, where the chain's
    gradient vanishes identically; this start is Jacobi as well and lets the chain learn.)"""
    p = torch.zeros(6, 9)
    p[0:4, 4] = 1.0
    p[5, 4] = omega / d
    return p.reshape(-1)


def init_params_fc(seed: int = 0) -> torch.Tensor:
    """The fully connected network: LeakyReLU Kaiming-uniform hidden layers, zero output
    layer (the network starts at weighted Jacobi)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for k, (co, ci) in enumerate(FC_LAYERS):
        if k == len(FC_LAYERS) - 1:
            parts.append(torch.zeros(co * ci))
        else:
            bound = math.sqrt(6.0 / ((1 + 0.01 ** 2) * ci))
            parts.append((torch.rand(co * ci, generator=g) * 2 - 1) * bound)
    return torch.cat(parts)


def init_params(seed: int = 0) -> torch.Tensor:
    """Convolutions: uniform with the LeakyReLU Kaiming bound; the output layer is zero, so
    the network starts exactly at weighted Jacobi (W = omega/D) with live gradients."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for k, (co, ci) in enumerate(LAYERS):
        if k == len(LAYERS) - 1:
            parts.append(torch.zeros(co * ci * 9))
        else:
            bound = math.sqrt(6.0 / ((1 + 0.01 ** 2) * ci * 9))
            parts.append((torch.rand(co * ci * 9, generator=g) * 2 - 1) * bound)
    p = torch.cat(parts)
    assert p.numel() == NPARAMS
    return p


class TwoGridBatch:
    """Device workspace + context for one training batch of same-size problems."""

    def __init__(self, problems: list[dict], nvec: int, omega: float = 2.0 / 3.0, conv_bf16: bool = False,
                 workspace: torch.Tensor | None = None, cycles: int = 1, checkpoint: bool = False,
                 net_arch: str = "conv"):
        self.n = problems[0]["n"]
        self.nprob = len(problems)
        self.nvec = nvec
        self.net_arch = net_arch
        self._probs, self._keep = B.problems_array(problems)
        from .solver import net_arch_code

        self.opts = B.options(B.MG_SMOOTH_CNN, omega, 3, int(conv_bf16), 1, int(cycles), int(checkpoint), 0, 0,
                              net_arch_code(net_arch))
        size = B.mg_train_workspace_size(self._probs, self.nprob, nvec, self.opts)
        if size == 0:
            raise B.MGError(B.MG_ERR_INVALID_ARG, "mg_train_workspace_size", B.lib().mg_last_error().decode())
        if workspace is None or workspace.numel() < size:
            workspace = torch.empty(size, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        self.ctx = B.mg_train_setup(self._probs, self.nprob, nvec, self.opts, workspace, size)

    def close(self):
        self.detach_coarse()
        if getattr(self, "ctx", None):
            B.mg_train_destroy(self.ctx)
            self.ctx = None

    # ------------------------------------------------ Algorithm 2: V-cycle coarse solve
    def coarse_fields(self) -> list[torch.Tensor]:
        """The batch's Galerkin coarse operators P^T A P as per-point fields [9, nc, nc]."""
        nc = (self.n - 1) // 2
        out = []
        for p in range(self.nprob):
            f = torch.empty((9, nc, nc), dtype=torch.float32, device="cuda")
            B.mg_train_get_coarse_field(self.ctx, p, f)
            out.append(f)
        return out

    def attach_coarse(self, level_params: torch.Tensor | None, omega: float | None = None) -> None:
        """Replace the exact coarse solve by one V-cycle of the hierarchy below, smoothed by
        level_params ([k, nparams]: set j on level j of the coarse hierarchy, the last set
        below that; None: weighted Jacobi), as Algorithm 2 does once those levels are trained."""
        from . import solver as S

        self.detach_coarse()
        fields = self.coarse_fields()
        nc = fields[0].shape[-1]
        probs = [S.field(nc, f) for f in fields]
        kind = "cnn" if level_params is not None else "jacobi"
        om = self.opts.omega if omega is None else omega
        self._coarse = [S.MultigridSolver(probs, kind, net_params=level_params, omega=om, conv_bf16=bool(self.opts.conv_bf16),
                                          transpose=t, net_arch=self.net_arch) for t in (False, True)]
        self._coarse_fields = fields

    def detach_coarse(self) -> None:
        for mg in getattr(self, "_coarse", []) or []:
            mg.close()
        self._coarse = None

    def __del__(self):
        self.close()

    def set_cycles(self, cycles: int) -> None:
        """Two-grid cycles k of the loss (at most the `cycles` given at construction)."""
        B.mg_train_set_cycles(self.ctx, cycles)

    def loss_and_grad(self, params: torch.Tensor, z: torch.Tensor, want_grad: bool = True):
        assert z.shape == (self.nprob, self.nvec, self.n, self.n) and z.is_contiguous()
        loss = torch.empty(1, device="cuda")
        grad = torch.empty(nparams(self.net_arch), device="cuda") if want_grad else None
        if getattr(self, "_coarse", None):
            B.mg_train_step_coarse(self.ctx, params.contiguous(), z, self._coarse[0].ctx, self._coarse[1].ctx, grad, loss)
        else:
            B.mg_train_step(self.ctx, params.contiguous(), z, grad, loss)
        return loss, grad


class TwoGridLoss(torch.autograd.Function):
    """loss = mean_b mean_j ||S C S z_bj||^2 / n^2 as a differentiable function of the
    network parameters; the backward pass is the library's hand-written adjoint."""

    @staticmethod
    def forward(ctx, params, z, batch):
        loss, grad = batch.loss_and_grad(params.detach(), z, want_grad=params.requires_grad)
        ctx.save_for_backward(grad if grad is not None else torch.zeros(0, device=params.device))
        return loss[0]

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return gout * grad, None, None


class Trainer:
    """Adam on the two-grid loss over freshly drawn rotated anisotropic problems."""

    def __init__(self, sizes=(31, 63), per_size: int = 32, nvec: int = 32, omega: float = 2.0 / 3.0,
                 conv_bf16: bool = True, lr: float = 1e-3, seed: int = 0, eps_range=(1e-3, 1.0),
                 families=("rotated",), max_cycles: int = 1, checkpoint: bool = False, net_arch: str = "conv",
                 device="cuda"):
        """max_cycles = b of Algorithm 2: each step's loss spans k ~ U{1..b} two-grid cycles.
        net_arch: "conv", "conv_shared" (one kernel per convolution output channel, Sec. 6.2's
        378 parameters), "conv3" (three stacked output kernels, FP32) or "fc" (the fully
        connected network of Sec. 4.2).  A training step needs the library and a GPU; device
        only places the parameters, the optimizer state and the generator of the random
        vectors (checkpoints can be written and read without a GPU)."""
        self.device = torch.device(device)
        self.max_cycles = max_cycles
        self.checkpoint = checkpoint
        self.net_arch = net_arch
        self.sizes = sizes
        self.per_size = per_size
        self.nvec = nvec
        self.omega = omega
        self.conv_bf16 = conv_bf16
        self.eps_range = eps_range
        self.families = families
        self.params = init_for(net_arch, seed).to(self.device).requires_grad_(True)
        self.opt = torch.optim.Adam([self.params], lr=lr)
        self.gen = torch.Generator(device=self.device).manual_seed(inputs.SEED_TRAIN + seed)
        self._ws = {}
        self.step_count = 0

    def problems(self, step: int, n: int, family: str = "rotated") -> list[dict]:
        seed = inputs.SEED_TRAIN + 7919 * step + n
        if family == "rotated":
            params = inputs.rotated_params(seed, self.per_size, *self.eps_range)
            return [{"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": e, "theta": t} for e, t in params]
        # variable coefficients a = exp(g), g a unit-variance Gaussian random field (Sec. 6.2)
        return [{"n": n, "kind": B.MG_PROBLEM_VARCOEF5,
                 "data": torch.from_numpy(inputs.grf_cells(seed * 64 + k, n)).to(self.device)}
                for k in range(self.per_size)]

    def cycles(self, step: int) -> int:
        """k of this step, drawn uniformly from 1..max_cycles (seeded by the step)."""
        if self.max_cycles <= 1:
            return 1
        return int(np.random.default_rng(inputs.SEED_TRAIN + 31 * step).integers(1, self.max_cycles + 1))

    def loss(self, step: int) -> torch.Tensor:
        total = 0.0
        count = 0
        k = self.cycles(step)
        for family in self.families:
            for n in self.sizes:
                probs = self.problems(step, n, family)
                key = (family, n)
                batch = TwoGridBatch(probs, self.nvec, self.omega, self.conv_bf16, self._ws.get(key),
                                     cycles=self.max_cycles, checkpoint=self.checkpoint, net_arch=self.net_arch)
                batch.set_cycles(k)
                self._ws[key] = batch.workspace
                z = torch.randn((self.per_size, self.nvec, n, n), generator=self.gen, device=self.device)
                total = total + TwoGridLoss.apply(self.params, z, batch)
                count += 1
        return total / count

    def step(self) -> float:
        self.opt.zero_grad(set_to_none=True)
        loss = self.loss(self.step_count)
        loss.backward()
        self.opt.step()
        self.step_count += 1
        return float(loss.detach())

    def save(self, path: str) -> None:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        np.save(path, self.params.detach().cpu().numpy().astype(np.float32))

    # ---------------------------------------------------------------- checkpoint / resume
    def config(self) -> dict:
        """What fixes the sequence of batches and losses (a resume must match it)."""
        return {"net_arch": self.net_arch, "sizes": list(self.sizes), "per_size": self.per_size, "nvec": self.nvec,
                "omega": self.omega, "conv_bf16": bool(self.conv_bf16), "eps_range": list(self.eps_range),
                "families": list(self.families), "max_cycles": self.max_cycles}

    def state_dict(self) -> dict:
        """Parameters, Adam state, the state of the random-vector generator and the step:
        a run resumed from it draws the same problems and vectors and takes the same steps."""
        return {"config": self.config(), "step": self.step_count, "params": self.params.detach().cpu().clone(),
                "opt": self.opt.state_dict(), "gen": self.gen.get_state()}

    def load_state_dict(self, state: dict) -> None:
        if state["config"] != self.config():
            raise ValueError(f"checkpoint of another training setup: {state['config']} vs {self.config()}")
        with torch.no_grad():
            self.params.copy_(state["params"].to(self.device))
        self.opt.load_state_dict(state["opt"])
        self.gen.set_state(state["gen"])
        self.step_count = int(state["step"])

    def save_checkpoint(self, path: str) -> None:
        d = os.path.dirname(path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        torch.save(self.state_dict(), tmp)
        os.replace(tmp, path)  # a crash mid-write leaves the previous checkpoint intact

    def load_checkpoint(self, path: str) -> None:
        self.load_state_dict(torch.load(path, map_location="cpu", weights_only=True))


class AdaptiveTrainer:
    """Algorithm 2: one network per level of a hierarchy of side n_fine, trained from the
    second-coarsest level up.  Level l's network minimises the two-grid objective of its own
    operators with the coarse solve replaced by one V-cycle of the levels below, smoothed by
    the networks already trained (the exact solve on the level above the coarsest).  The
    operators of level l are rotated anisotropic problems of that level's size (constant
    stencils are invariant under the Galerkin product, Sec. 6.1)."""

    def __init__(self, n_fine: int = 63, per_size: int = 32, nvec: int = 32, steps_per_level: int = 300,
                 lr: float = 1e-3, omega: float = 2.0 / 3.0, conv_bf16: bool = True, seed: int = 0,
                 eps_range=(1e-3, 1.0), max_cycles: int = 1, init=None, net_arch: str = "conv",
                 problem: tuple[float, float] | None = None):
        """net_arch "linear": the shared-kernel linear smoother of Sec. 6, trained for one
        problem (eps, theta) = `problem` -- Sec. 6 trains each such smoother on instances of
        its own problem: here `per_size` copies of it with nvec random vectors each."""
        self.sizes = []
        n = n_fine
        while n > 3:
            self.sizes.append(n)
            n = (n - 1) // 2
        self.per_size, self.nvec, self.steps = per_size, nvec, steps_per_level
        self.lr, self.omega, self.conv_bf16, self.seed = lr, omega, conv_bf16, seed
        self.eps_range, self.max_cycles = eps_range, max_cycles
        self.init = init  # starting parameters of every level (None: the Jacobi-equivalent net)
        self.net_arch = net_arch
        self.problem = problem
        if net_arch == "linear" and problem is None:
            raise ValueError("the linear smoother is trained for one problem (eps, theta)")
        self.params: dict[int, torch.Tensor] = {}
        self.losses: dict[int, list[float]] = {}
        self.gen = torch.Generator(device="cuda").manual_seed(inputs.SEED_TRAIN + 17 + seed)

    def level_params(self, n: int) -> torch.Tensor | None:
        """Stacked trained parameters of the levels below side n (finest first), or None."""
        below = [m for m in self.sizes if m < n and m in self.params]
        return torch.stack([self.params[m] for m in below]) if below else None

    def problems(self, step: int, n: int) -> list[dict]:
        if self.problem is not None:
            e, t = self.problem
            return [{"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": e, "theta": t}] * self.per_size
        params = inputs.rotated_params(inputs.SEED_TRAIN + 104729 * step + 7 * n + 1, self.per_size, *self.eps_range)
        return [{"n": n, "kind": B.MG_PROBLEM_ROTATED, "eps": e, "theta": t} for e, t in params]

    def _init(self) -> torch.Tensor:
        if self.init is not None:
            return self.init.detach().clone()
        if self.net_arch == "linear":
            s = B.mg_rotated_stencil(*self.problem)
            return init_params_linear(float(s[4]), self.omega)
        return init_for(self.net_arch, self.seed)

    def train_level(self, n: int) -> torch.Tensor:
        p = self._init().cuda().requires_grad_(True)
        opt = torch.optim.Adam([p], lr=self.lr)
        below = self.level_params(n)
        ws = None
        hist = []
        for step in range(self.steps):
            batch = TwoGridBatch(self.problems(step, n), self.nvec, self.omega, self.conv_bf16, ws,
                                 cycles=self.max_cycles, net_arch=self.net_arch)
            ws = batch.workspace
            if (n - 1) // 2 > 3:  # the level above the coarsest keeps the exact coarse solve
                batch.attach_coarse(below)
            if self.max_cycles > 1:
                batch.set_cycles(int(np.random.default_rng(inputs.SEED_TRAIN + 31 * step + n).integers(1, self.max_cycles + 1)))
            z = torch.randn((self.per_size, self.nvec, n, n), generator=self.gen, device="cuda")
            opt.zero_grad(set_to_none=True)
            loss = TwoGridLoss.apply(p, z, batch)
            loss.backward()
            opt.step()
            hist.append(float(loss.detach()))
            batch.close()
        self.losses[n] = hist
        self.params[n] = p.detach().clone()
        return self.params[n]

    def train(self) -> None:
        for n in reversed(self.sizes):
            self.train_level(n)

    def hierarchy_params(self, n_solve: int) -> torch.Tensor:
        """Per-level parameter sets for a solver of side n_solve: each level takes the network
        trained at its own side, levels finer than the finest trained side take that one."""
        sets = []
        n = n_solve
        while n > 3:
            m = n if n in self.params else max(self.params)
            sets.append(self.params[m])
            n = (n - 1) // 2
        return torch.stack(sets)


def adaptive_params(W: np.ndarray | torch.Tensor, n_solve: int, n_fine: int = 63) -> torch.Tensor:
    """Per-level parameter sets for a solver of side n_solve from networks trained by
    AdaptiveTrainer for a hierarchy of side n_fine (W: [levels, nparams], finest first):
    each level takes the network of its own side, finer levels the finest one."""
    W = torch.as_tensor(np.asarray(W, dtype=np.float32))
    sizes = []
    n = n_fine
    while n > 3:
        sizes.append(n)
        n = (n - 1) // 2
    assert W.shape[0] == len(sizes)
    sets = []
    n = n_solve
    while n > 3:
        sets.append(W[sizes.index(n)] if n in sizes else W[0])
        n = (n - 1) // 2
    return torch.stack(sets)


def main():
    import argparse
    import time

    ap = argparse.ArgumentParser(description="train the stencil-to-smoother network on the GPU")
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None,
                    help="default: weights/<cnn|fc>_<first family>.npy next to this module")
    ap.add_argument("--fp32-conv", action="store_true")
    ap.add_argument("--families", default="rotated", help="comma list of rotated,varcoef")
    ap.add_argument("--max-cycles", type=int, default=1, help="b: each step's loss spans k ~ U{1..b} cycles")
    ap.add_argument("--checkpoint", action="store_true", help="recompute cycle products in the backward pass")
    ap.add_argument("--fc", action="store_true", help="train the fully connected network (Sec. 4.2)")
    ap.add_argument("--arch", default=None, choices=["conv", "conv_shared", "conv3", "fc"],
                    help="network architecture (default conv; --fc is --arch fc)")
    ap.add_argument("--state", default=None, metavar="PATH",
                    help="checkpoint: resume from PATH if it exists, write it every 100 steps and at the end")
    ap.add_argument("--adaptive", type=int, default=0, metavar="N_FINE",
                    help="Algorithm 2: one network per level of a hierarchy of this side, trained coarse to fine "
                         "(--steps per level); saves [levels, nparams], finest first")
    ap.add_argument("--linear", action="store_true",
                    help="with --adaptive: the shared-kernel linear smoother of Sec. 6, one per problem "
                         "(eps = --eps, theta in --thetas); saves an .npz of params [thetas, levels, 54]")
    ap.add_argument("--eps", type=float, default=0.01)
    ap.add_argument("--thetas", default="1,2,3,4,5", help="angles in units of pi/12")
    ap.add_argument("--batch", type=int, default=0, metavar="NPROB",
                    help="with --linear: one smoother for each problem (eps, theta) of the seeded rotated batch of "
                         "this size (inputs.rotated_params with the batch seed) instead of --eps / --thetas")
    args = ap.parse_args()
    from . import build

    build.build()
    if args.linear:
        if not args.adaptive:
            ap.error("--linear trains per level: give --adaptive N_FINE")
        t0 = time.time()
        if args.batch:
            pairs = [(float(e), float(t)) for e, t in inputs.rotated_params(inputs.SEED_PARAMS, args.batch)]
        else:
            pairs = [(args.eps, float(k) * math.pi / 12) for k in args.thetas.split(",")]
        sets = []
        for e, th in pairs:
            at = AdaptiveTrainer(n_fine=args.adaptive, per_size=1, nvec=64, steps_per_level=args.steps, lr=args.lr,
                                 seed=args.seed, conv_bf16=False, net_arch="linear", problem=(e, th))
            at.train()
            sets.append(torch.stack([at.params[n] for n in at.sizes]).cpu().numpy().astype(np.float32))
            h = at.losses[at.sizes[0]]
            print(f"eps {e:.4g} theta {th:.4f}: finest-level loss {np.mean(h[:10]):.5f} -> {np.mean(h[-10:]):.5f} "
                  f"({time.time() - t0:.1f} s)", flush=True)
        name = f"linear_batch{args.batch}.npz" if args.batch else f"linear_eps{args.eps:g}.npz"
        out = args.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", name)
        os.makedirs(os.path.dirname(out), exist_ok=True)
        eps_out = np.array([e for e, _ in pairs]) if args.batch else args.eps
        np.savez(out, params=np.stack(sets), thetas=np.array([t for _, t in pairs]), eps=eps_out, n_fine=args.adaptive)
        print("saved", out, "levels", at.sizes)
        return
    if args.adaptive:
        t0 = time.time()
        at = AdaptiveTrainer(n_fine=args.adaptive, steps_per_level=args.steps, lr=args.lr, seed=args.seed,
                             conv_bf16=not args.fp32_conv, max_cycles=args.max_cycles)
        for n in reversed(at.sizes):
            at.train_level(n)
            h = at.losses[n]
            print(f"level n={n}: loss {np.mean(h[:10]):.5f} -> {np.mean(h[-10:]):.5f} ({time.time() - t0:.1f} s)",
                  flush=True)
        out = args.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "cnn_rotated_adaptive.npy")
        os.makedirs(os.path.dirname(out), exist_ok=True)
        np.save(out, torch.stack([at.params[n] for n in at.sizes]).cpu().numpy().astype(np.float32))
        print("saved", out, "levels", at.sizes)
        return
    arch = args.arch or ("fc" if args.fc else "conv")
    tr = Trainer(lr=args.lr, seed=args.seed, conv_bf16=not args.fp32_conv and arch != "conv3",
                 families=tuple(f.strip() for f in args.families.split(",")), max_cycles=args.max_cycles,
                 checkpoint=args.checkpoint, net_arch=arch)
    if args.state and os.path.exists(args.state):
        tr.load_checkpoint(args.state)
        print(f"resumed from {args.state} at step {tr.step_count}", flush=True)
    t0 = time.time()
    while tr.step_count < args.steps:
        s = tr.step_count
        l = tr.step()
        if s % 50 == 0 or s == args.steps - 1:
            print(f"step {s:5d} loss {l:.6f} ({time.time() - t0:.1f} s)", flush=True)
        if args.state and (tr.step_count % 100 == 0 or tr.step_count == args.steps):
            tr.save_checkpoint(args.state)
    prefix = {"conv": "cnn", "fc": "fc", "conv_shared": "cnn378", "conv3": "cnn3"}[arch]
    out = args.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                   f"{prefix}_{tr.families[0]}.npy")
    tr.save(out)
    print("saved", out)


if __name__ == "__main__":
    main()
