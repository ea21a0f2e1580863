"""The C-ABI library loads on a machine without a GPU and exports every
symbol include/slbm.h declares; host-only argument checks answer without
touching CUDA (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_2102_12559_gb300 import _build, slbm

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "slbm.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return slbm.load()


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"SLBM_API\s+(?:const\s+char\s*\*|int)\s*(slbm_\w+)\s*\(", txt)))


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(slbm.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_workspace_bytes_host_only(lib):
    n = slbm.slbm_workspace_bytes(64, 64, 1, 1, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, 3, slbm.SLBM_FP32)
    # two buffers of 9 + 25 planes of at least (64 + 4) x (64 + 2*2) floats
    assert n >= 2 * 34 * 68 * 68 * 4
    n64 = slbm.slbm_workspace_bytes(64, 64, 1, 1, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, 3, slbm.SLBM_FP64)
    assert n64 > n


@pytest.mark.parametrize("args", [
    dict(lat_lo=5, lat_hi=3),            # pair order
    dict(lat_lo=3, lat_hi=6),            # unknown lattice
    dict(tau=0.5),                       # tau must exceed 1/2
    dict(interp_order=0),
    dict(interp_order=6),
    dict(precision=7),
    dict(frame=3),                       # unknown frame
    dict(frame=1, periodic_y=0),         # the co-moving frame needs a periodic grid
    dict(frame=2, periodic_x=0),
    dict(nx=0),
])
def test_invalid_arguments_rejected_before_cuda(lib, args):
    a = dict(nx=32, ny=32, lat_lo=3, lat_hi=5, tau=0.6, interp_order=3, frame=0, precision=0,
             periodic_x=1, periodic_y=1)
    a.update(args)
    g = slbm.slbm_grid(a["nx"], 32, a["periodic_x"], a["periodic_y"])
    h = ctypes.c_void_p()
    rc = lib.slbm_create(ctypes.byref(g), a["lat_lo"], a["lat_hi"], a["tau"], a["interp_order"],
                         a["frame"], a["precision"], None, ctypes.byref(h))
    assert rc == slbm.SLBM_EINVAL
    assert not h.value
    assert slbm.slbm_last_error()


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.slbm_step(None, 1) == slbm.SLBM_EINVAL
    assert lib.slbm_sync(None) == slbm.SLBM_EINVAL
    assert lib.slbm_destroy(None) == slbm.SLBM_EINVAL


@pytest.mark.parametrize("lo,hi", [(3, 4), (3, 5), (4, 5)])
@pytest.mark.parametrize("order", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("frame", [0, 1, 2])
def test_every_pair_and_order_passes_argument_checks(lib, lo, hi, order, frame):
    """All argument checks (including the compile-time stencil pattern the
    kernels assume) accept every supported configuration; on a machine
    without a GPU the call then stops at the first CUDA call."""
    g = slbm.slbm_grid(40, 40, 1, 1)
    h = ctypes.c_void_p()
    rc = lib.slbm_create(ctypes.byref(g), lo, hi, 0.6, order, frame, 0, None, ctypes.byref(h))
    assert rc != slbm.SLBM_EINVAL, slbm.slbm_last_error()
    if h.value:
        lib.slbm_destroy(h)
