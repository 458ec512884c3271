"""State exchange through pinned host memory (read and written in place by
the kernels) against the staged path for pageable memory and the device
path: the same bits, before and after steps."""
import ctypes

import numpy as np
import pytest

from oracle import oracle
from paper_2608_26908_gb300 import gpflbm, inputs

pytestmark = pytest.mark.gpu


def _pinned(a, torch):
    t = torch.empty(a.size, dtype=torch.float64 if a.dtype == np.float64 else torch.float32, pin_memory=True)
    t.numpy()[:] = a.reshape(-1)
    return t


@pytest.mark.parametrize("name,size,prec", [
    ("eutectic2d", dict(nx=70, ny=45), "fp32"),
    ("dendrite2d", dict(nx=40, ny=36), "fp64"),
    ("eutectic3d", dict(nx=20, ny=18, nz=16), "fp32"),
    ("dendrite3d", dict(nx=20, ny=18, nz=16), "fp32_f16"),
])
def test_pinned_host_exchange_matches_the_staged_path(name, size, prec):
    import torch
    sc = inputs.scenario(name, precision=prec, **size)
    phi0, mu0 = inputs.initial_state(sc)
    f0 = oracle.rest_populations(sc)
    dt = np.float64 if prec == "fp64" else np.float32
    phi0, mu0, f0 = (np.asarray(a, dtype=dt) for a in (phi0, mu0, f0))
    a = gpflbm.Sim(sc)
    a.set_state(phi0, mu0, f0)  # pageable numpy: staged
    b = gpflbm.Sim(sc)
    b.set_state(*(_pinned(x, torch) for x in (phi0, mu0, f0)))  # pinned: in place
    for steps in (0, 7):
        a.step(steps)
        b.step(steps)
        want = a.fields(("phi", "mu", "c", "f", "rho", "u"))
        names = sorted(want, key=lambda n: gpflbm.FIELD[n])
        outs = [torch.empty(want[n].shape, dtype=torch.float64 if dt == np.float64 else torch.float32,
                            pin_memory=True) for n in names]
        mask = 0
        for n in names:
            mask |= gpflbm.FIELD[n]
        ptrs = (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        st = gpflbm.lib().gpflbm_get_fields(b.h, mask, ptrs, 0,
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == gpflbm.OK
        dev = b.fields(names, device=True)
        for n, o in zip(names, outs):
            np.testing.assert_array_equal(o.numpy(), want[n], err_msg=n)
            np.testing.assert_array_equal(dev[n].cpu().numpy(), want[n], err_msg=n)
