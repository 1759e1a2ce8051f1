"""The C-ABI library builds, loads and exports every entry point of include/mgcnn.h (no GPU).

Only host-side entry points are called here (argument validation, the constant
stencil, status strings); nothing touches a device.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2102_12071_gb300 import binding as B
from paper_2102_12071_gb300 import build as BUILD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.lib()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "mg_solve" in names and "mg_train_step" in names and len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name


def test_rotated_stencil_matches_oracle(lib):
    for eps, theta in [(1.0, 0.0), (0.01, math.pi / 6), (1e-3, 2.9), (0.37, 1.3)]:
        mine = np.array(B.mg_rotated_stencil(eps, theta), dtype=np.float32)
        ref = O.q1_rotated_stencil(eps, theta).reshape(9).astype(np.float32)
        # both round the same FP64 value; allow one ulp for libm differences in cos/sin
        assert np.all(np.abs(mine.view(np.int32) - ref.view(np.int32)) <= 1), (mine, ref)


def test_argument_validation_is_host_side(lib):
    opts = B.options()
    probs, _ = B.problems_array([{"n": 64, "kind": B.MG_PROBLEM_ROTATED, "eps": 0.1, "theta": 0.0}])
    assert B.mg_workspace_size(probs, 1, opts) == 0
    assert b"2^m - 1" in lib.mg_last_error()
    probs, _ = B.problems_array([{"n": 63, "kind": B.MG_PROBLEM_ROTATED, "eps": -1.0, "theta": 0.0}])
    assert B.mg_workspace_size(probs, 1, opts) == 0
    probs, _ = B.problems_array([{"n": 63, "kind": B.MG_PROBLEM_ROTATED, "eps": 0.1, "theta": 0.0},
                                 {"n": 127, "kind": B.MG_PROBLEM_ROTATED, "eps": 0.1, "theta": 0.0}])
    assert B.mg_workspace_size(probs, 2, opts) == 0
    bad = B.options(omega=2.5)
    probs, _ = B.problems_array([{"n": 63, "kind": B.MG_PROBLEM_ROTATED, "eps": 0.1, "theta": 0.0}])
    assert B.mg_workspace_size(probs, 1, bad) == 0
    assert B.mg_workspace_size(probs, 1, opts) > 0
    # setup with a missing / small workspace fails before any device work
    out = ctypes.c_void_p()
    st = lib.mg_setup(probs, 1, ctypes.byref(opts), None, None, 0, None, ctypes.byref(out))
    assert st == B.MG_ERR_WORKSPACE and not out.value
    cnn = B.options(smoother=B.MG_SMOOTH_CNN)
    st = lib.mg_setup(probs, 1, ctypes.byref(cnn), None, None, 0, None, ctypes.byref(out))
    assert st == B.MG_ERR_INVALID_ARG
    assert lib.mg_solve(None, None, None, None, 1e-8, 10, None, None, None) == B.MG_ERR_INVALID_ARG
    assert lib.mg_debug_strip_rows(None, 0) == B.MG_ERR_INVALID_ARG
    assert B.mg_workspace_size(probs, 1, B.options(tile_shape=B.MG_TILE_PSTRIP)) > 0
    assert B.mg_workspace_size(probs, 1, B.options(tile_shape=B.MG_TILE_PSTRIP + 1)) == 0
    assert lib.mg_status_string(B.MG_ERR_NOT_CONVERGED) == b"not converged"
    assert lib.mg_net_nparams() == O.hypernet_nparams() == 1260


def test_workspace_grows_with_batch(lib):
    opts = B.options()
    one, _ = B.problems_array([{"n": 255, "kind": B.MG_PROBLEM_ROTATED, "eps": 0.1, "theta": 0.0}])
    four, _ = B.problems_array([{"n": 255, "kind": B.MG_PROBLEM_ROTATED, "eps": 0.1, "theta": 0.0}] * 4)
    s1, s4 = B.mg_workspace_size(one, 1, opts), B.mg_workspace_size(four, 4, opts)
    assert s4 > 3 * s1 > 0
    # per problem: r and e on every level (4/3 n^2 floats each) dominate
    assert s1 >= 2 * 4 * 255 * 255


def test_smoothing_steps_and_linear_smoother_options_are_checked_on_the_host(lib):
    probs, _ = B.problems_array([{"n": 255, "kind": B.MG_PROBLEM_ROTATED, "eps": 0.1, "theta": 0.0}])
    # nu1, nu2 in 1..8, other than 1 only for Jacobi and the linear smoother
    assert B.mg_workspace_size(probs, 1, B.options(nu1=9)) == 0
    assert b"[1, 8]" in lib.mg_last_error()
    assert B.mg_workspace_size(probs, 1, B.options(nu1=0)) == 0
    assert B.mg_workspace_size(probs, 1, B.options(B.MG_SMOOTH_CNN, nu1=2)) == 0
    assert b"Jacobi or the linear smoother" in lib.mg_last_error()
    jac6 = B.mg_workspace_size(probs, 1, B.options(nu1=6, nu2=6))
    lin2 = B.mg_workspace_size(probs, 1, B.options(B.MG_SMOOTH_CNN, net_arch=B.MG_NET_LINEAR, nu1=2, nu2=3))
    assert jac6 > B.mg_workspace_size(probs, 1, B.options()) > 0 and lin2 > 0  # scratch of the batched path
    # per-problem parameter groups only for the linear smoother
    assert B.mg_workspace_size(probs, 1, B.options(B.MG_SMOOTH_CNN, net_per_problem=1)) == 0
    assert b"linear smoother" in lib.mg_last_error()
    assert B.mg_workspace_size(probs, 1, B.options(B.MG_SMOOTH_CNN, net_arch=B.MG_NET_LINEAR,
                                                   net_per_problem=1)) > 0
    assert B.mg_workspace_size(probs, 1, B.options(B.MG_SMOOTH_CNN, net_arch=7)) == 0
    assert lib.mg_net_param_count(B.MG_NET_LINEAR) == 54


def test_network_architectures_are_checked_on_the_host(lib):
    """Parameter counts per architecture (Sec. 6.2's 6 800 and 378 among them) and which
    architecture/option pairs the setup and the training accept, without a GPU."""
    counts = {B.MG_NET_CONV: 1260, B.MG_NET_FC: 6800, B.MG_NET_LINEAR: 54, B.MG_NET_CONV3: 1746,
              B.MG_NET_CONV_SHARED: 378}
    for arch, count in counts.items():
        assert lib.mg_net_param_count(arch) == count
    assert lib.mg_net_param_count(5) == 0
    rot, _ = B.problems_array([{"n": 63, "kind": B.MG_PROBLEM_ROTATED, "eps": 0.1, "theta": 0.4}])
    cnn = lambda **kw: B.options(B.MG_SMOOTH_CNN, **kw)
    dense = B.mg_workspace_size(rot, 1, cnn())
    shared = B.mg_workspace_size(rot, 1, cnn(net_arch=B.MG_NET_CONV_SHARED))
    assert shared > dense > 0  # plus the expanded dense set
    assert B.mg_workspace_size(rot, 1, cnn(net_arch=B.MG_NET_CONV_SHARED, net_levels=3)) > shared
    assert B.mg_workspace_size(rot, 1, cnn(net_arch=B.MG_NET_CONV3)) > 0
    # the three-kernel stack: FP32, no transposed smoother, one smoothing step
    assert B.mg_workspace_size(rot, 1, cnn(net_arch=B.MG_NET_CONV3, conv_bf16=1)) == 0
    assert b"FP32" in lib.mg_last_error()
    assert B.mg_workspace_size(rot, 1, cnn(net_arch=B.MG_NET_CONV3, nu1=2)) == 0
    # training: every architecture but bf16 with the stack
    for arch in counts:
        assert B.mg_train_workspace_size(rot, 1, 4, cnn(net_arch=arch)) > 0, arch
    assert B.mg_train_workspace_size(rot, 1, 4, cnn(net_arch=B.MG_NET_CONV3, conv_bf16=1)) == 0
    assert b"FP32" in lib.mg_last_error()
    t_dense = B.mg_train_workspace_size(rot, 1, 4, cnn())
    assert B.mg_train_workspace_size(rot, 1, 4, cnn(net_arch=B.MG_NET_CONV3)) > t_dense  # 27 outputs, stack scratch
