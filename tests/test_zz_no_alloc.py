"""gpflbm_invariants_noalloc: the conservation totals for callers that cannot
allocate device memory when they ask for them (the reduction scratch is a
fixed device array inside the library).  Checked against gpflbm_invariants
on two calls in a row, and its size limit.  This file is collected last."""
import ctypes

import numpy as np
import pytest

from paper_2608_26908_gb300 import gpflbm, inputs

pytestmark = pytest.mark.gpu

# FP64 sums of the same per-cell values in two orders: rounding-level agreement
RTOL = 1e-12


def noalloc(sim):
    L = gpflbm.lib()
    fn = L.gpflbm_invariants_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    m = ctypes.c_double()
    s = (ctypes.c_double * 2)()
    fr = ctypes.c_double()
    import torch
    st = fn(sim.h, ctypes.byref(m), s, ctypes.byref(fr),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, m.value, np.array(s[: sim.NC]), fr.value


@pytest.mark.parametrize("name,size,prec", [("eutectic2d", dict(nx=200, ny=90), "fp32"),
                                            ("dendrite2d", dict(), "fp64"),
                                            ("eutectic3d", dict(nx=36, ny=34, nz=40), "fp32")])
def test_noalloc_totals_match_invariants_twice(name, size, prec):
    sc = inputs.scenario(name, precision=prec, **size)
    if name == "eutectic3d":
        sc["init"]["height"] = 12
    sim = gpflbm.Sim(sc)
    sim.set_state(*inputs.initial_state(sc))
    sim.step(31)
    for _ in range(2):
        m, s, fr, _ = sim.invariants()
        st, m2, s2, fr2 = noalloc(sim)
        assert st == gpflbm.OK
        assert m2 == pytest.approx(m, rel=RTOL)
        np.testing.assert_allclose(s2, s, rtol=RTOL)
        assert fr2 == pytest.approx(fr, rel=RTOL, abs=1e-15)


def test_noalloc_rejects_grids_beyond_its_scratch():
    sc = inputs.scenario("dendrite2d", nx=4096, ny=4097, precision="fp32")
    sim = gpflbm.Sim(sc)
    st, _, _, _ = noalloc(sim)  # checked before any state is needed
    assert st == gpflbm.ERR_ARG
    assert b"static scratch limit" in gpflbm.lib().gpflbm_last_error(sim.h)
