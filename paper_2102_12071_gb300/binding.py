"""Thin ctypes binding of libmgcnn.so (C ABI in include/mgcnn.h).

Argument marshalling only: every computation runs in the CUDA library.  Device arrays
are torch CUDA tensors (float32, contiguous); streams default to torch's current stream.
Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmgcnn.so")

MG_OK, MG_ERR_INVALID_ARG, MG_ERR_WORKSPACE, MG_ERR_CUDA, MG_ERR_NOT_CONVERGED, MG_ERR_NUMERIC, \
    MG_ERR_TIMEOUT, MG_ERR_UNSUPPORTED = range(8)
MG_PROBLEM_ROTATED, MG_PROBLEM_STENCIL, MG_PROBLEM_VARCOEF5, MG_PROBLEM_FIELD = range(4)
MG_SMOOTH_JACOBI, MG_SMOOTH_CNN = 0, 1
MG_TILE_DEFAULT, MG_TILE_32x32, MG_TILE_STRIP4x32, MG_TILE_STRIP8x64, MG_TILE_STRIP8x32, MG_TILE_PSTRIP = range(6)
TILE_SHAPES = {"32x32": MG_TILE_32x32, "strip4x32": MG_TILE_STRIP4x32, "strip8x64": MG_TILE_STRIP8x64,
               "strip8x32": MG_TILE_STRIP8x32, "pstrip": MG_TILE_PSTRIP}


class mg_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("kind", ctypes.c_int), ("eps", ctypes.c_double),
                ("theta", ctypes.c_double), ("data", ctypes.c_void_p)]


class mg_options(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("omega", ctypes.c_float), ("coarsest_n", ctypes.c_int), ("conv_bf16", ctypes.c_int),
                ("cluster_tail", ctypes.c_int), ("train_cycles", ctypes.c_int), ("train_checkpoint", ctypes.c_int),
                ("net_levels", ctypes.c_int), ("smoother_transpose", ctypes.c_int), ("net_arch", ctypes.c_int),
                ("net_per_problem", ctypes.c_int), ("tile_shape", ctypes.c_int)]


class MGError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


_lib = None
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load libmgcnn.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "mg_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(mg_problem), ctypes.c_int, ctypes.POINTER(mg_options)]),
        "mg_setup": (ctypes.c_int, [ctypes.POINTER(mg_problem), ctypes.c_int, ctypes.POINTER(mg_options), _P, _P,
                                    ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
        "mg_destroy": (None, [_P]),
        "mg_num_levels": (ctypes.c_int, [_P]),
        "mg_level_n": (ctypes.c_int, [_P, ctypes.c_int]),
        "mg_get_stencil": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
        "mg_get_kernels": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
        "mg_smoother_apply": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
        "mg_vcycle": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
        "mg_solve": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_double, ctypes.c_int, _P, _P, _P]),
        "mg_solve_multi": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.c_double, ctypes.c_int, _P, _P]),
        "mg_net_nparams": (ctypes.c_int, []),
        "mg_net_forward": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_float, ctypes.c_int, _P, _P]),
        "mg_train_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(mg_problem), ctypes.c_int, ctypes.c_int,
                                                      ctypes.POINTER(mg_options)]),
        "mg_train_setup": (ctypes.c_int, [ctypes.POINTER(mg_problem), ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(mg_options), _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
        "mg_train_destroy": (None, [_P]),
        "mg_train_step": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
        "mg_train_set_cycles": (ctypes.c_int, [_P, ctypes.c_int]),
        "mg_fgmres_workspace_size": (ctypes.c_size_t, [_P, ctypes.c_int]),
        "mg_net_param_count": (ctypes.c_int, [ctypes.c_int]),
        "mg_net_fc_forward": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_float, ctypes.c_int, _P, _P]),
        "mg_fgmres": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int, _P, ctypes.c_size_t,
                                     _P, _P, _P]),
        "mg_train_step_coarse": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
        "mg_train_get_coarse_field": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
        "mg_solve_small_static": (ctypes.c_int, [ctypes.POINTER(mg_problem), ctypes.c_int, ctypes.POINTER(mg_options),
                                                 _P, _P, _P, ctypes.c_double, ctypes.c_int, _P, _P, _P]),
        "mg_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
        "mg_debug_short_wait": (ctypes.c_int, [_P, ctypes.c_int]),
        "mg_debug_strip_rows": (ctypes.c_int, [_P, ctypes.c_int]),
        "mg_solve_times": (ctypes.c_int, [_P, _P, _P]),
        "mg_profile_read": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong)]),
        "mg_rotated_stencil": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_float)]),
        "mg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "mg_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int, where: str) -> int:
    if status not in (MG_OK,):
        raise MGError(status, where, lib().mg_last_error().decode())
    return status


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    import torch

    return torch.cuda.current_stream().cuda_stream


def problems_array(problems: list[dict]):
    arr = (mg_problem * len(problems))()
    keep = []
    for k, p in enumerate(problems):
        arr[k].n = p["n"]
        arr[k].kind = p["kind"]
        arr[k].eps = p.get("eps", 0.0)
        arr[k].theta = p.get("theta", 0.0)
        data = p.get("data")
        if data is None:
            arr[k].data = None
        elif isinstance(data, int):
            arr[k].data = data
        elif hasattr(data, "data_ptr"):
            arr[k].data = data.data_ptr()
            keep.append(data)
        else:  # host stencil: 9 floats
            buf = (ctypes.c_float * 9)(*[float(v) for v in data])
            keep.append(buf)
            arr[k].data = ctypes.cast(buf, ctypes.c_void_p)
    return arr, keep


def options(smoother: int = MG_SMOOTH_JACOBI, omega: float = 2.0 / 3.0, coarsest_n: int = 3,
            conv_bf16: int = 0, cluster_tail: int = 1, train_cycles: int = 1, train_checkpoint: int = 0,
            net_levels: int = 0, smoother_transpose: int = 0, net_arch: int = 0,
            net_per_problem: int = 0, nu1: int = 1, nu2: int = 1, tile_shape: int = 0) -> mg_options:
    return mg_options(smoother, nu1, nu2, omega, coarsest_n, conv_bf16, cluster_tail, train_cycles, train_checkpoint,
                      net_levels, smoother_transpose, net_arch, net_per_problem, tile_shape)


def mg_workspace_size(probs, nprob: int, opts: mg_options) -> int:
    return lib().mg_workspace_size(probs, nprob, ctypes.byref(opts))


def mg_setup(probs, nprob: int, opts: mg_options, net_params, workspace, ws_bytes: int, stream=None) -> int:
    out = _P()
    check(lib().mg_setup(probs, nprob, ctypes.byref(opts), _ptr(net_params), _ptr(workspace), ws_bytes,
                         _stream(stream), ctypes.byref(out)), "mg_setup")
    return out.value


def mg_destroy(ctx: int) -> None:
    lib().mg_destroy(ctx)


def mg_num_levels(ctx: int) -> int:
    return lib().mg_num_levels(ctx)


def mg_level_n(ctx: int, level: int) -> int:
    return lib().mg_level_n(ctx, level)


def mg_get_stencil(ctx, prob, level, out, stream=None):
    check(lib().mg_get_stencil(ctx, prob, level, _ptr(out), _stream(stream)), "mg_get_stencil")


def mg_get_kernels(ctx, prob, level, out, stream=None):
    check(lib().mg_get_kernels(ctx, prob, level, _ptr(out), _stream(stream)), "mg_get_kernels")


def mg_smoother_apply(ctx, prob, level, f, u, nsteps=1, stream=None):
    check(lib().mg_smoother_apply(ctx, prob, level, _ptr(f), _ptr(u), nsteps, _stream(stream)), "mg_smoother_apply")


def mg_vcycle(ctx, b, x_hi, x_lo=None, rel_res=None, stream=None):
    check(lib().mg_vcycle(ctx, _ptr(b), _ptr(x_hi), _ptr(x_lo), _ptr(rel_res), _stream(stream)), "mg_vcycle")


def mg_solve(ctx, b, x_hi, x_lo, rtol, max_cycles, hist=None, cycles=None, stream=None) -> int:
    """hist: numpy float64 [nprob, max_cycles+1] or None; cycles: numpy int32 [nprob] or None.
    Returns the status (MG_OK or MG_ERR_NOT_CONVERGED); other failures raise."""
    hp = hist.ctypes.data if hist is not None else None
    cp = cycles.ctypes.data if cycles is not None else None
    st = lib().mg_solve(ctx, _ptr(b), _ptr(x_hi), _ptr(x_lo), float(rtol), int(max_cycles), hp, cp,
                        _stream(stream))
    if st not in (MG_OK, MG_ERR_NOT_CONVERGED):
        check(st, "mg_solve")
    return st


def mg_solve_multi(ctxs, b, x_hi, x_lo, rtol, max_cycles, cycles=None, streams=None) -> int:
    """Per-context lists: b, x_hi, x_lo (tensors or None), cycles (numpy int32 or None),
    streams (raw CUDA stream handles or None).  Returns MG_OK or MG_ERR_NOT_CONVERGED."""
    k = len(ctxs)
    arr = lambda vals: (ctypes.c_void_p * k)(*vals)
    cyc = arr([c.ctypes.data if c is not None else None for c in cycles]) if cycles is not None else None
    st = lib().mg_solve_multi(arr(ctxs), k, arr([_ptr(t) for t in b]), arr([_ptr(t) for t in x_hi]),
                              arr([_ptr(t) for t in x_lo]) if x_lo is not None else None, float(rtol),
                              int(max_cycles), cyc, arr(list(streams)) if streams is not None else None)
    if st not in (MG_OK, MG_ERR_NOT_CONVERGED):
        check(st, "mg_solve_multi")
    return st


def mg_solve_small_static(probs, nprob, opts, b, x_hi, x_lo, rtol, max_cycles, hist=None, cycles=None,
                          stream=None) -> int:
    """Workspace-free solve of small constant-stencil batches (see include/mgcnn.h)."""
    hp = hist.ctypes.data if hist is not None else None
    cp = cycles.ctypes.data if cycles is not None else None
    st = lib().mg_solve_small_static(probs, nprob, ctypes.byref(opts), _ptr(b), _ptr(x_hi), _ptr(x_lo), float(rtol),
                                     int(max_cycles), hp, cp, _stream(stream))
    if st not in (MG_OK, MG_ERR_NOT_CONVERGED):
        check(st, "mg_solve_small_static")
    return st


def mg_net_nparams() -> int:
    return lib().mg_net_nparams()


def mg_net_forward(n, nprob, fields, params, omega, conv_bf16, W, stream=None):
    check(lib().mg_net_forward(n, nprob, _ptr(fields), _ptr(params), float(omega), int(conv_bf16), _ptr(W),
                               _stream(stream)), "mg_net_forward")


def mg_train_workspace_size(probs, nprob, nvec, opts) -> int:
    return lib().mg_train_workspace_size(probs, nprob, nvec, ctypes.byref(opts))


def mg_train_setup(probs, nprob, nvec, opts, workspace, ws_bytes, stream=None) -> int:
    out = _P()
    check(lib().mg_train_setup(probs, nprob, nvec, ctypes.byref(opts), _ptr(workspace), ws_bytes, _stream(stream),
                               ctypes.byref(out)), "mg_train_setup")
    return out.value


def mg_train_destroy(ctx) -> None:
    lib().mg_train_destroy(ctx)


def mg_train_step(ctx, params, z, grad_out, loss_out, stream=None):
    check(lib().mg_train_step(ctx, _ptr(params), _ptr(z), _ptr(grad_out), _ptr(loss_out), _stream(stream)),
          "mg_train_step")


def mg_train_step_coarse(ctx, params, z, coarse, coarse_t, grad_out, loss_out, stream=None):
    check(lib().mg_train_step_coarse(ctx, _ptr(params), _ptr(z), coarse, coarse_t, _ptr(grad_out), _ptr(loss_out),
                                     _stream(stream)), "mg_train_step_coarse")


def mg_train_get_coarse_field(ctx, prob: int, out, stream=None) -> None:
    check(lib().mg_train_get_coarse_field(ctx, int(prob), _ptr(out), _stream(stream)), "mg_train_get_coarse_field")


MG_NET_CONV, MG_NET_FC, MG_NET_LINEAR, MG_NET_CONV3, MG_NET_CONV_SHARED = 0, 1, 2, 3, 4


def mg_net_param_count(arch: int) -> int:
    return lib().mg_net_param_count(int(arch))


def mg_net_fc_forward(n, nprob, fields, params, omega, bf16, W, stream=None):
    check(lib().mg_net_fc_forward(n, nprob, _ptr(fields), _ptr(params), float(omega), int(bf16), _ptr(W),
                                  _stream(stream)), "mg_net_fc_forward")


def mg_fgmres_workspace_size(ctx, restart: int) -> int:
    return lib().mg_fgmres_workspace_size(ctx, int(restart))


def mg_fgmres(ctx, b, x_hi, x_lo, restart, rtol, max_iters, workspace, ws_bytes, hist=None, iters=None,
              stream=None) -> int:
    hp = hist.ctypes.data if hist is not None else None
    ip = iters.ctypes.data if iters is not None else None
    st = lib().mg_fgmres(ctx, _ptr(b), _ptr(x_hi), _ptr(x_lo), int(restart), float(rtol), int(max_iters),
                         _ptr(workspace), int(ws_bytes), hp, ip, _stream(stream))
    if st not in (MG_OK, MG_ERR_NOT_CONVERGED):
        check(st, "mg_fgmres")
    return st


def mg_train_set_cycles(ctx, cycles: int) -> None:
    check(lib().mg_train_set_cycles(ctx, int(cycles)), "mg_train_set_cycles")


def mg_solve_times(ctx, nprob: int):
    """(start_ns, done_ns) numpy uint64 arrays of the last solve of ctx (see include/mgcnn.h)."""
    import numpy as np

    start = np.zeros(nprob, dtype=np.uint64)
    done = np.zeros(nprob, dtype=np.uint64)
    check(lib().mg_solve_times(ctx, start.ctypes.data, done.ctypes.data), "mg_solve_times")
    return start, done


def mg_debug_short_wait(ctx, on: bool) -> None:
    check(lib().mg_debug_short_wait(ctx, int(on)), "mg_debug_short_wait")


def mg_debug_strip_rows(ctx, rows: int) -> None:
    check(lib().mg_debug_strip_rows(ctx, int(rows)), "mg_debug_strip_rows")


def mg_profile_enable(ctx, enable: bool) -> None:
    check(lib().mg_profile_enable(ctx, int(enable)), "mg_profile_enable")


def mg_profile_read(ctx, kernel_class: int) -> tuple[float, int]:
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    check(lib().mg_profile_read(ctx, kernel_class, ctypes.byref(ms), ctypes.byref(n)), "mg_profile_read")
    return ms.value, n.value


def mg_rotated_stencil(eps: float, theta: float):
    out = (ctypes.c_float * 9)()
    check(lib().mg_rotated_stencil(float(eps), float(theta), out), "mg_rotated_stencil")
    return list(out)
