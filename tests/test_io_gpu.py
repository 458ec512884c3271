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


@pytest.mark.parametrize("name,size,prec", [
    ("eutectic2d", dict(nx=72, ny=45), "fp32"),       # 4 | nx: 16-byte loads
    ("eutectic2d", dict(nx=70, ny=45), "fp32_bf16"),  # word loads
    ("dendrite2d", dict(nx=40, ny=36), "fp64"),       # 2 | nx: 16-byte loads
    ("dendrite2d", dict(nx=41, ny=36), "fp64"),       # word loads
    ("dendrite3d", dict(nx=20, ny=18, nz=16), "fp32_f16"),
])
def test_asynchronous_pinned_and_device_sources(name, size, prec):
    """The one-launch load (device or pinned sources, with or without f) and
    the asynchronous flag give the staged path's bits, before and after
    steps; an unknown flag bit is refused."""
    import torch
    sc = inputs.scenario(name, precision=prec, **size)
    phi0, mu0 = inputs.initial_state(sc)
    f0 = oracle.rest_populations(sc) * (1.0 + 1e-3 * np.cos(np.arange(oracle.rest_populations(sc).size)))
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if dt == np.float64 else torch.float32
    phi0, mu0, f0 = (np.asarray(a, dtype=dt) for a in (phi0, mu0, f0))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    names = ["phi", "mu", "f"]
    for with_f in (True, False):
        a = gpflbm.Sim(sc)
        a.set_state(phi0, mu0, f0 if with_f else None)  # pageable numpy: staged
        want = a.fields(names)
        # device sources through the binding
        b = gpflbm.Sim(sc)
        b.set_state(*(torch.from_numpy(x).cuda() for x in (phi0, mu0)),
                    torch.from_numpy(f0).cuda() if with_f else None)
        # pinned sources and destinations, asynchronous
        c = gpflbm.Sim(sc)
        src = [_pinned(x, torch) for x in (phi0, mu0, f0)]
        st = gpflbm.lib().gpflbm_set_state(c.h, ctypes.c_void_p(src[0].data_ptr()),
                                           ctypes.c_void_p(src[1].data_ptr()),
                                           ctypes.c_void_p(src[2].data_ptr() if with_f else None),
                                           gpflbm.ASYNC, 0, stream)
        assert st == gpflbm.OK
        bad = gpflbm.lib().gpflbm_set_state(c.h, ctypes.c_void_p(src[0].data_ptr()),
                                            ctypes.c_void_p(src[1].data_ptr()), None, 4, 0, stream)
        assert bad == gpflbm.ERR_ARG
        for steps in (0, 5):
            a.step(steps)
            b.step(steps)
            c.step(steps)
            want = a.fields(names)
            outs = [torch.empty(want[n].shape, dtype=tdt, pin_memory=True) for n in names]
            mask = gpflbm.FIELD["phi"] | gpflbm.FIELD["mu"] | gpflbm.FIELD["f"]
            ptrs = (ctypes.c_void_p * 3)(*[o.data_ptr() for o in outs])
            assert gpflbm.lib().gpflbm_get_fields(c.h, mask, ptrs, gpflbm.ASYNC, stream) == gpflbm.OK
            assert gpflbm.lib().gpflbm_get_fields(c.h, mask, ptrs, 8, stream) == gpflbm.ERR_ARG
            assert gpflbm.lib().gpflbm_get_deviations(c.h, ptrs[2], 4, stream) == gpflbm.ERR_ARG
            torch.cuda.synchronize()
            got_b = b.fields(names)
            for n, o in zip(names, outs):
                np.testing.assert_array_equal(o.numpy(), want[n], err_msg="pinned async " + n)
                np.testing.assert_array_equal(got_b[n], want[n], err_msg="device " + n)
        assert a.time() == b.time() == c.time() == 5


@pytest.mark.parametrize("name,size,prec", [
    ("eutectic2d", dict(nx=72, ny=45), "fp32"),
    ("dendrite2d", dict(nx=40, ny=36), "fp64"),
    ("dendrite3d", dict(nx=20, ny=18, nz=16), "fp32_f16"),
])
def test_asynchronous_loads_overlapping_the_write_back(name, size, prec):
    """An end-to-end loop with nothing but the final synchronise: each state
    is loaded (asynchronously, into the idle buffer, beside the previous
    write-back), stepped and written back; every written-back state equals,
    bit for bit, the same load, steps and fields done one call at a time."""
    import torch
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if dt == np.float64 else torch.float32
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    names = ["phi", "mu", "f"]
    mask = gpflbm.FIELD["phi"] | gpflbm.FIELD["mu"] | gpflbm.FIELD["f"]
    states = []
    for k in range(4):
        sc = inputs.scenario(name, precision=prec, seed=2000 + k, **size)
        phi0, mu0 = inputs.initial_state(sc)
        f0 = oracle.rest_populations(sc)
        f0 = f0 * (1.0 + 1e-3 * np.cos(np.arange(f0.size) + k))
        states.append([np.asarray(a, dtype=dt) for a in (phi0, mu0, f0)])
    ref = gpflbm.Sim(sc)
    want = []
    for phi0, mu0, f0 in states:
        ref.set_state(phi0, mu0, f0, t0=5)
        ref.step(3)
        want.append(ref.fields(names))
    sim = gpflbm.Sim(sc)
    src = [[_pinned(a, torch) for a in st] for st in states]
    outs = [[torch.empty(want[0][n].shape, dtype=tdt, pin_memory=True) for n in names] for _ in states]
    L = gpflbm.lib()
    for k in range(len(states)):
        assert L.gpflbm_set_state(sim.h, *[ctypes.c_void_p(t.data_ptr()) for t in src[k]],
                                  gpflbm.ASYNC, 5, stream) == gpflbm.OK
        assert L.gpflbm_step(sim.h, 3, stream) == gpflbm.OK
        ptrs = (ctypes.c_void_p * 3)(*[o.data_ptr() for o in outs[k]])
        assert L.gpflbm_get_fields(sim.h, mask, ptrs, gpflbm.ASYNC, stream) == gpflbm.OK
    torch.cuda.synchronize()
    for k in range(len(states)):
        for n, o in zip(names, outs[k]):
            np.testing.assert_array_equal(o.numpy(), want[k][n], err_msg="state %d %s" % (k, n))
    assert sim.time() == 8
    # a read-only call, then a synchronous load, then the async path again
    m0, s0, _, _ = sim.invariants()
    sim.set_state(*states[0], t0=5)
    sim.step(3)
    np.testing.assert_array_equal(sim.fields(["phi"])["phi"], want[0]["phi"])
