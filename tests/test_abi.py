"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every entry point include/gpflbm.h declares, sizes workspaces and
rejects invalid arguments before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2608_26908_gb300 import build, gpflbm, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return gpflbm.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gpflbm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("gpflbm_create", "gpflbm_set_state", "gpflbm_step", "gpflbm_get_fields",
                 "gpflbm_invariants", "gpflbm_destroy", "gpflbm_last_error"):
        assert need in names


def test_binding_constants_match_the_header():
    """Status codes, field bits and exchange flags of the binding are the
    header's."""
    src = open(os.path.join(ROOT, "include", "gpflbm.h")).read()
    defines = {k: int(v) for k, v in re.findall(r"#define\s+(GPFLBM_\w+)\s+\(?(-?\d+)", src)}
    assert defines["GPFLBM_ON_DEVICE"] == gpflbm.ON_DEVICE
    assert defines["GPFLBM_ASYNC"] == gpflbm.ASYNC
    assert gpflbm.ON_DEVICE & gpflbm.ASYNC == 0


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


@pytest.mark.parametrize("name", inputs.WORKLOADS)
def test_workspace_bytes_for_every_workload(L, name):
    sc = inputs.scenario(name)
    n = gpflbm.workspace_bytes(sc)
    cells = inputs.cells(sc)
    q = 19 if sc["grid"]["nz"] > 1 else 9
    rs = 8 if sc["precision"] == "fp64" else 4
    assert n >= 2 * q * cells * (rs if sc["precision"] in ("fp64", "fp32") else 2)
    assert n < 8 * q * cells * rs


@pytest.mark.parametrize("prec", list(gpflbm.PRECISION))
def test_every_precision_is_built(L, prec):
    for name in ("dendrite2d", "eutectic3d"):
        sc = inputs.scenario(name, nx=16, ny=16, nz=16 if "3d" in name else None, precision=prec)
        assert gpflbm.workspace_bytes(sc) > 0


def _status(L, sc, np_=None, nc=None, mutate=None):
    g = gpflbm.grid_struct(sc)
    if mutate:
        mutate(g)
    n = ctypes.c_size_t()
    return L.gpflbm_workspace_bytes(ctypes.byref(g), np_ or sc["n_phases"], nc or sc["n_solutes"],
                                    ctypes.byref(n))


def test_invalid_grids_are_rejected(L):
    sc = inputs.scenario("dendrite2d", nx=16, ny=16)
    assert _status(L, sc) == gpflbm.OK
    assert _status(L, sc, np_=5) == gpflbm.ERR_UNSUPPORTED
    assert _status(L, sc, nc=3) == gpflbm.ERR_UNSUPPORTED
    assert _status(L, sc, mutate=lambda g: setattr(g, "nz", 2)) == gpflbm.ERR_ARG
    assert _status(L, sc, mutate=lambda g: setattr(g, "nx", 2)) == gpflbm.ERR_ARG
    assert _status(L, sc, mutate=lambda g: setattr(g, "lattice", 19)) == gpflbm.ERR_UNSUPPORTED
    assert _status(L, sc, mutate=lambda g: setattr(g, "precision", 7)) == gpflbm.ERR_ARG

    def bad_bc(g):
        g.bc[0] = 3
    assert _status(L, sc, mutate=bad_bc) == gpflbm.ERR_ARG

    def bad_rows(g):
        g.wall_rows[1] = 8
    assert _status(L, sc, mutate=bad_rows) == gpflbm.ERR_ARG
    n = ctypes.c_size_t()
    assert L.gpflbm_workspace_bytes(None, 2, 1, ctypes.byref(n)) == gpflbm.ERR_ARG


def test_create_rejects_bad_arguments_without_a_device(L):
    sc = inputs.scenario("dendrite2d", nx=16, ny=16)
    g = gpflbm.grid_struct(sc)
    p = gpflbm.params_struct(sc)
    h = ctypes.c_void_p(123)
    assert L.gpflbm_create(ctypes.byref(g), 2, 1, None, None, 0, ctypes.byref(h)) == gpflbm.ERR_ARG
    assert h.value is None
    p.tau_f = 0.5
    assert L.gpflbm_create(ctypes.byref(g), 2, 1, ctypes.byref(p), None, 0,
                           ctypes.byref(h)) == gpflbm.ERR_ARG
    p = gpflbm.params_struct(sc)
    p.A[1] = 0.0
    assert L.gpflbm_create(ctypes.byref(g), 2, 1, ctypes.byref(p), None, 0,
                           ctypes.byref(h)) == gpflbm.ERR_ARG
    p = gpflbm.params_struct(sc)
    p.tilt[0][1] = 0.3  # tilt must be symmetric
    assert L.gpflbm_create(ctypes.byref(g), 2, 1, ctypes.byref(p), None, 0,
                           ctypes.byref(h)) == gpflbm.ERR_ARG
    p.tilt[1][0] = float("nan")
    assert L.gpflbm_create(ctypes.byref(g), 2, 1, ctypes.byref(p), None, 0,
                           ctypes.byref(h)) == gpflbm.ERR_ARG
    assert L.gpflbm_create(ctypes.byref(g), 2, 1, ctypes.byref(gpflbm.params_struct(sc)), None, 0,
                           None) == gpflbm.ERR_ARG
    # a caller's workspace that is too small or misaligned is refused before
    # the device is touched (the pointer is only checked, never used)
    g = gpflbm.grid_struct(sc)
    p = gpflbm.params_struct(sc)
    need = gpflbm.workspace_bytes(sc)
    assert L.gpflbm_create(ctypes.byref(g), 2, 1, ctypes.byref(p), ctypes.c_void_p(1 << 20), need - 1,
                           ctypes.byref(h)) == gpflbm.ERR_OOM
    assert h.value is None
    assert L.gpflbm_create(ctypes.byref(g), 2, 1, ctypes.byref(p), ctypes.c_void_p((1 << 20) + 8), need,
                           ctypes.byref(h)) == gpflbm.ERR_ARG
    assert h.value is None
    # calls on a null handle fail cleanly
    assert L.gpflbm_step(None, 1, None) == gpflbm.ERR_ARG
    assert L.gpflbm_set_state(None, None, None, None, 0, 0, None) == gpflbm.ERR_ARG
    assert L.gpflbm_invariants(None, None, None, None, None) == gpflbm.ERR_ARG
    L.gpflbm_destroy(None)
