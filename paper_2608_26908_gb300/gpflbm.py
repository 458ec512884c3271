"""Thin ctypes binding of libgpflbm.so (include/gpflbm.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  PyTorch provides the device workspace and the current stream.  If
the library has not been built, loading it raises -- there is no CPU path.
"""
import copy
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgpflbm.so")

OK = 0
# exchange flags of gpflbm_set_state / gpflbm_get_fields (include/gpflbm.h)
ON_DEVICE, ASYNC = 1, 2
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_STATE, ERR_UNSUPPORTED = (
    -1, -2, -3, -4, -6, -7)
PERIODIC, WALL = 0, 1
D2Q9, D3Q19, D3Q27 = 9, 19, 27
PRECISION = {"fp64": 0, "fp32": 1, "fp32_f16": 2, "fp32_bf16": 3}
FIELD = {"phi": 1, "mu": 2, "c": 4, "f": 8, "rho": 16, "u": 32}


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lattice", ctypes.c_int), ("bc", ctypes.c_int * 3),
                ("wall_rows", ctypes.c_int * 3), ("precision", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [
        ("tau_f", ctypes.c_double), ("tau_phi", ctypes.c_double), ("eps", ctypes.c_double),
        ("gamma", (ctypes.c_double * 4) * 4), ("delta", (ctypes.c_double * 4) * 4),
        ("A", ctypes.c_double * 4), ("ceq", (ctypes.c_double * 2) * 4), ("S", ctypes.c_double * 4),
        ("D_liq", ctypes.c_double), ("a_at", ctypes.c_double),
        ("h_drag", ctypes.c_double), ("W0", ctypes.c_double),
        ("gbeta_c", ctypes.c_double * 2), ("c_ref", ctypes.c_double * 2),
        ("gbeta_T", ctypes.c_double), ("T_ref", ctypes.c_double),
        ("T_E", ctypes.c_double), ("undercool", ctypes.c_double),
        ("G", ctypes.c_double), ("V", ctypes.c_double), ("v0", ctypes.c_double),
        ("q_floor", ctypes.c_double),
        ("eta_rho", ctypes.c_double * 4),
        ("tilt", (ctypes.c_double * 4) * 4),
        ("dceq_dT", (ctypes.c_double * 2) * 4),
    ]


class Objective(ctypes.Structure):
    """gpflbm_objective: J = w_frac mean h_1 + w_tip tip / nx."""
    _fields_ = [("w_frac", ctypes.c_double), ("w_tip", ctypes.c_double), ("kappa", ctypes.c_double),
                ("x0", ctypes.c_int), ("y0", ctypes.c_int), ("z0", ctypes.c_int), ("solid", ctypes.c_int)]


def objective_struct(obj):
    o = Objective()
    o.w_frac, o.w_tip, o.kappa = float(obj["w_frac"]), float(obj["w_tip"]), float(obj["kappa"])
    o.x0, o.y0, o.z0 = int(obj["x0"]), int(obj["y0"]), int(obj.get("z0", 0))
    o.solid = int(obj.get("solid", 1))
    return o


class GpflbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("gpflbm status %d: %s" % (status, msg))
        self.status = status


_lib = None


def lib():
    """Load libgpflbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgpflbm.so is not built (%s); run __graft_entry__.build()"
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i, u, ll, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_longlong, ctypes.c_size_t
        dp = ctypes.POINTER(ctypes.c_double)
        L.gpflbm_workspace_bytes.argtypes = [ctypes.POINTER(Grid), i, i, ctypes.POINTER(sz)]
        L.gpflbm_create.argtypes = [ctypes.POINTER(Grid), i, i, ctypes.POINTER(Params), vp, sz,
                                    ctypes.POINTER(vp)]
        L.gpflbm_set_params.argtypes = [vp, ctypes.POINTER(Params)]
        L.gpflbm_set_state.argtypes = [vp, vp, vp, vp, i, ll, vp]
        L.gpflbm_step.argtypes = [vp, i, vp]
        L.gpflbm_shift_frame.argtypes = [vp, i, vp]
        L.gpflbm_step_timed.argtypes = [vp, ctypes.POINTER(vp), vp]
        L.gpflbm_get_fields.argtypes = [vp, u, ctypes.POINTER(vp), i, vp]
        L.gpflbm_get_deviations.argtypes = [vp, vp, i, vp]
        L.gpflbm_invariants.argtypes = [vp, dp, dp, dp, vp]
        L.gpflbm_time.argtypes = [vp, ctypes.POINTER(ll)]
        L.gpflbm_adjoint_workspace_bytes.argtypes = [vp, i, i, ctypes.POINTER(sz)]
        L.gpflbm_adjoint.argtypes = [vp, ctypes.POINTER(Objective), i, i, vp, sz, dp, dp, vp, i, vp]
        L.gpflbm_vjp.argtypes = [vp, i, i, vp, sz, vp, vp, dp, i, vp]
        L.gpflbm_slab_workspace_bytes.argtypes = [ctypes.POINTER(Grid), i, i, i, i, ctypes.POINTER(sz)]
        L.gpflbm_create_slab.argtypes = [ctypes.POINTER(Grid), i, i, i, i, ctypes.POINTER(Params), vp, sz,
                                         ctypes.POINTER(vp)]
        L.gpflbm_halo_bytes.argtypes = [vp, ctypes.POINTER(sz)]
        L.gpflbm_step_launches.argtypes = [vp, ctypes.POINTER(i)]
        L.gpflbm_halo_pack.argtypes = [vp, i, vp, vp]
        L.gpflbm_halo_unpack.argtypes = [vp, i, vp, vp]
        L.gpflbm_last_error.argtypes = [vp]
        L.gpflbm_last_error.restype = ctypes.c_char_p
        L.gpflbm_destroy.argtypes = [vp]
        L.gpflbm_destroy.restype = None
        for name in ("gpflbm_workspace_bytes", "gpflbm_create", "gpflbm_set_params",
                     "gpflbm_set_state", "gpflbm_step", "gpflbm_step_timed", "gpflbm_get_fields",
                     "gpflbm_get_deviations", "gpflbm_invariants", "gpflbm_time",
                     "gpflbm_adjoint_workspace_bytes", "gpflbm_adjoint", "gpflbm_vjp",
                     "gpflbm_slab_workspace_bytes", "gpflbm_create_slab", "gpflbm_halo_bytes",
                     "gpflbm_halo_pack", "gpflbm_halo_unpack", "gpflbm_step_launches"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def grid_struct(sc):
    g = sc["grid"]
    s = Grid()
    s.nx, s.ny, s.nz = g["nx"], g["ny"], g.get("nz", 1)
    s.lattice = g.get("lattice") or (D3Q19 if s.nz > 1 else D2Q9)
    for a in range(3):
        s.bc[a] = g["bc"][a]
        s.wall_rows[a] = g["wall_rows"][a] if (a < 2 or s.nz > 1) else 0
    s.precision = PRECISION[sc["precision"]]
    return s


def params_struct(sc):
    pr = sc["params"]
    p = Params()
    for name in ("tau_f", "tau_phi", "eps", "D_liq", "a_at", "h_drag", "W0", "gbeta_T", "T_ref",
                 "T_E", "undercool", "G", "V", "v0", "q_floor"):
        setattr(p, name, float(pr[name]))
    for a in range(4):
        p.A[a] = pr["A"][a]
        p.S[a] = pr["S"][a]
        for b in range(4):
            p.gamma[a][b] = pr["gamma"][a][b]
            p.delta[a][b] = pr["delta"][a][b]
        for i in range(2):
            p.ceq[a][i] = pr["ceq"][a][i]
    for i in range(2):
        p.gbeta_c[i] = pr["gbeta_c"][i]
        p.c_ref[i] = pr["c_ref"][i]
    for a in range(4):
        p.eta_rho[a] = pr.get("eta_rho", [0.0] * 4)[a]
        for b in range(4):
            p.tilt[a][b] = pr.get("tilt", [[0.0] * 4] * 4)[a][b]
        for i in range(2):
            p.dceq_dT[a][i] = pr.get("dceq_dT", [[0.0] * 2] * 4)[a][i]
    return p


def workspace_bytes(sc):
    n = ctypes.c_size_t()
    g = grid_struct(sc)
    st = lib().gpflbm_workspace_bytes(ctypes.byref(g), sc["n_phases"], sc["n_solutes"],
                                      ctypes.byref(n))
    if st != OK:
        raise GpflbmError(st, "workspace_bytes")
    return n.value


def _stream(torch):
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Sim:
    """One simulation on the current CUDA device; the workspace is a torch
    tensor, calls run on torch's current stream.  slab=(v_begin, v_count)
    makes it the slab of planes v_begin .. v_begin + v_count - 1 of a 3D
    grid (gpflbm_create_slab): its fields are those planes."""

    def __init__(self, sc, slab=None):
        import torch
        self.torch = torch
        self.sc = sc
        self.slab = slab
        self.nx, self.ny, self.nz = sc["grid"]["nx"], sc["grid"]["ny"], sc["grid"].get("nz", 1)
        if slab is not None:
            self.nz = int(slab[1])
        self.cells = self.nx * self.ny * self.nz
        self.dim = 3 if sc["grid"].get("nz", 1) > 1 else 2
        self.Q = sc["grid"].get("lattice") or (19 if self.dim == 3 else 9)
        self.NP, self.NC = sc["n_phases"], sc["n_solutes"]
        self.dtype = np.float64 if sc["precision"] == "fp64" else np.float32
        self.tdtype = torch.float64 if sc["precision"] == "fp64" else torch.float32
        self._grid = grid_struct(sc)
        self._params = params_struct(sc)
        if slab is None:
            nbytes = workspace_bytes(sc)
        else:
            n = ctypes.c_size_t()
            st = lib().gpflbm_slab_workspace_bytes(ctypes.byref(self._grid), int(slab[0]), int(slab[1]),
                                                   self.NP, self.NC, ctypes.byref(n))
            if st != OK:
                raise GpflbmError(st, "gpflbm_slab_workspace_bytes")
            nbytes = n.value
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        if slab is None:
            st = lib().gpflbm_create(ctypes.byref(self._grid), self.NP, self.NC,
                                     ctypes.byref(self._params), ctypes.c_void_p(self.workspace.data_ptr()),
                                     nbytes, ctypes.byref(h))
        else:
            st = lib().gpflbm_create_slab(ctypes.byref(self._grid), int(slab[0]), int(slab[1]), self.NP,
                                          self.NC, ctypes.byref(self._params),
                                          ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                          ctypes.byref(h))
        if st != OK:
            raise GpflbmError(st, "gpflbm_create" if slab is None else "gpflbm_create_slab")
        self.h = h

    def halo_bytes(self):
        n = ctypes.c_size_t()
        self._check(lib().gpflbm_halo_bytes(self.h, ctypes.byref(n)), "halo_bytes")
        return n.value

    def halo_pack(self, side, msg):
        """Planes the neighbour on `side` (0 below, 1 above) needs, into the
        uint8 device tensor msg (halo_bytes() long)."""
        self._check(lib().gpflbm_halo_pack(self.h, int(side), ctypes.c_void_p(msg.data_ptr()),
                                           _stream(self.torch)), "halo_pack")

    def halo_unpack(self, side, msg):
        """A message packed by the neighbour on `side` into this slab's halo."""
        self._check(lib().gpflbm_halo_unpack(self.h, int(side), ctypes.c_void_p(msg.data_ptr()),
                                             _stream(self.torch)), "halo_unpack")

    def _check(self, st, what):
        if st != OK:
            msg = lib().gpflbm_last_error(self.h).decode()
            raise GpflbmError(st, "%s: %s" % (what, msg))

    def close(self):
        if getattr(self, "h", None):
            lib().gpflbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptr(self, a):
        """(pointer, is_device, keepalive) of a numpy array or torch tensor."""
        torch = self.torch
        if a is None:
            return None, None, None
        if isinstance(a, torch.Tensor):
            a = a.contiguous()
            if a.dtype != self.tdtype:
                a = a.to(self.tdtype)
            return ctypes.c_void_p(a.data_ptr()), a.is_cuda, a
        a = np.ascontiguousarray(a, dtype=self.dtype)
        return ctypes.c_void_p(a.ctypes.data), False, a

    def shift_frame(self, rows):
        """Moving frame: the state moves `rows` cells down the vertical axis
        and v0 drops by `rows` (this object's scenario follows)."""
        self._check(lib().gpflbm_shift_frame(self.h, int(rows), _stream(self.torch)), "shift_frame")
        self.sc = copy.deepcopy(self.sc)
        self.sc["params"]["v0"] = self.sc["params"]["v0"] - rows
        self._params = params_struct(self.sc)

    def set_params(self, sc):
        self.sc = sc
        self._params = params_struct(sc)
        self._check(lib().gpflbm_set_params(self.h, ctypes.byref(self._params)), "set_params")

    def set_state(self, phi, mu, f=None, t0=0):
        pp, dphi, k1 = self._ptr(phi)
        pm, dmu, k2 = self._ptr(mu)
        pf, df, k3 = self._ptr(f)
        dev = bool(dphi)
        if dmu != dev or (f is not None and df != dev):
            raise ValueError("phi, mu and f must all be host arrays or all device tensors")
        self._check(lib().gpflbm_set_state(self.h, pp, pm, pf, int(dev), int(t0),
                                           _stream(self.torch)), "set_state")
        del k1, k2, k3

    def step(self, n=1):
        self._check(lib().gpflbm_step(self.h, int(n), _stream(self.torch)), "step")

    def step_timed(self, events):
        """One step recording two torch.cuda.Event objects (before and after
        the step kernel) on the current stream."""
        raw = (ctypes.c_void_p * 2)(*[e.cuda_event for e in events[:2]])
        self._check(lib().gpflbm_step_timed(self.h, raw, _stream(self.torch)), "step_timed")

    def step_launches(self):
        n = ctypes.c_int()
        self._check(lib().gpflbm_step_launches(self.h, ctypes.byref(n)), "step_launches")
        return n.value

    def time(self):
        t = ctypes.c_longlong()
        self._check(lib().gpflbm_time(self.h, ctypes.byref(t)), "time")
        return t.value

    def _planes(self, name):
        return {"phi": self.NP, "mu": self.NC, "c": self.NC, "f": self.Q, "rho": 1,
                "u": self.dim}[name]

    def fields(self, names=("phi", "mu"), device=False):
        """dict name -> (planes, cells) array (numpy) or tensor (device=True)."""
        torch = self.torch
        names = sorted(set(names), key=lambda n: FIELD[n])
        mask = 0
        outs = []
        for n in names:
            mask |= FIELD[n]
            shape = (self._planes(n), self.cells)
            if device:
                outs.append(torch.empty(shape, dtype=self.tdtype, device="cuda"))
            else:
                outs.append(np.empty(shape, dtype=self.dtype))
        ptrs = (ctypes.c_void_p * len(outs))(
            *[o.data_ptr() if device else o.ctypes.data for o in outs])
        self._check(lib().gpflbm_get_fields(self.h, mask, ptrs, int(device), _stream(torch)),
                    "get_fields")
        return dict(zip(names, outs))

    def deviations(self):
        out = np.empty((self.Q, self.cells), dtype=self.dtype)
        self._check(lib().gpflbm_get_deviations(self.h, ctypes.c_void_p(out.ctypes.data), 0,
                                                _stream(self.torch)), "get_deviations")
        return out

    def invariants(self, allow_nonfinite=False):
        """(mass, solute[K-1], solid_frac) from the fixed-order FP64 reduction."""
        m = ctypes.c_double()
        s = (ctypes.c_double * 2)()
        fr = ctypes.c_double()
        st = lib().gpflbm_invariants(self.h, ctypes.byref(m), s, ctypes.byref(fr),
                                     _stream(self.torch))
        if not (allow_nonfinite and st == ERR_NONFINITE):
            self._check(st, "invariants")
        return m.value, np.array(s[: self.NC]), fr.value, st

    def adjoint_workspace_bytes(self, horizon, ckpt_every):
        n = ctypes.c_size_t()
        self._check(lib().gpflbm_adjoint_workspace_bytes(self.h, int(horizon), int(ckpt_every),
                                                         ctypes.byref(n)), "adjoint_workspace_bytes")
        return n.value

    def adjoint(self, obj, horizon, ckpt_every, device=False, workspace=None):
        """Run `horizon` steps from the current state and the adjoint back.

        Returns (J, dparams, dmu0): dparams = dJ/d(1/tau_phi, delta_01,
        gbeta_c[0]) as a numpy array, dmu0 = dJ/dmu of the starting state (one
        plane; a device tensor if device=True).  The state is left at
        t0 + horizon.  workspace: optional uint8 device tensor of at least
        adjoint_workspace_bytes() bytes (else the library allocates one).
        """
        torch = self.torch
        o = objective_struct(obj)
        J = ctypes.c_double()
        dpar = (ctypes.c_double * 3)()
        if device:
            dmu = torch.empty(self.cells, dtype=self.tdtype, device="cuda")
            dptr = ctypes.c_void_p(dmu.data_ptr())
        else:
            dmu = np.empty(self.cells, dtype=self.dtype)
            dptr = ctypes.c_void_p(dmu.ctypes.data)
        if workspace is not None:
            wptr, wbytes = ctypes.c_void_p(workspace.data_ptr()), workspace.numel()
        else:
            wptr, wbytes = None, 0
        self._check(lib().gpflbm_adjoint(self.h, ctypes.byref(o), int(horizon), int(ckpt_every), wptr,
                                         wbytes, ctypes.byref(J), dpar, dptr, int(device),
                                         _stream(torch)), "adjoint")
        return J.value, np.array(dpar[:]), dmu

    def vjp(self, seed, horizon, ckpt_every):
        """Vector-Jacobian product of `horizon` steps from the current state:
        seed is an (11, cells) array of the exchange type (planes phi_1, mu,
        f_0..f_8 of the final state); returns (grad, dparams) with grad the
        (11, cells) planes of d<seed, S^{t0+H}>/dS^{t0} and dparams its
        derivatives by (1/tau_phi, delta_01, gbeta_c[0]).  Host buffers."""
        seed = np.ascontiguousarray(seed, dtype=self.dtype).reshape(11, self.cells)
        grad = np.empty((11, self.cells), dtype=self.dtype)
        dpar = (ctypes.c_double * 3)()
        self._check(lib().gpflbm_vjp(self.h, int(horizon), int(ckpt_every), None, 0,
                                     ctypes.c_void_p(seed.ctypes.data), ctypes.c_void_p(grad.ctypes.data),
                                     dpar, 0, _stream(self.torch)), "vjp")
        return grad, np.array(dpar[:])


def with_parameters(sc, mobility=None, delta=None, gbeta=None):
    """Copy of a scenario with 1/tau_phi, delta_01 and g beta_c[0] replaced."""
    import copy
    sc = copy.deepcopy(sc)
    pr = sc["params"]
    if mobility is not None:
        pr["tau_phi"] = 1.0 / float(mobility)
    if delta is not None:
        pr["delta"][0][1] = pr["delta"][1][0] = float(delta)
    if gbeta is not None:
        pr["gbeta_c"][0] = float(gbeta)
    return sc


def _make_function():
    import torch

    class GPFLBMFunction(torch.autograd.Function):
        """J(mu0, 1/tau_phi, delta, g beta_c) after `horizon` steps from
        (phi0, mu0), differentiable through the library's adjoint.

        The adjoint runs inside forward (its forward pass produces J, so J
        and all gradients cost two forward passes plus the adjoint steps);
        backward scales the stored gradients by grad_output.
        """

        @staticmethod
        def forward(ctx, mu0, mobility, delta, gbeta, sim, phi0, obj, horizon, ckpt_every):
            sim.set_params(with_parameters(sim.sc, float(mobility), float(delta), float(gbeta)))
            # phi0 and mu0 go in together: both device tensors or both host arrays
            if mu0.is_cuda:
                phi = torch.as_tensor(phi0).to(device=mu0.device, dtype=sim.tdtype)
                sim.set_state(phi, mu0.detach())
            else:
                phi = phi0.numpy() if isinstance(phi0, torch.Tensor) else phi0
                sim.set_state(phi, mu0.detach().numpy())
            J, dpar, dmu = sim.adjoint(obj, horizon, ckpt_every, device=mu0.is_cuda)
            if not mu0.is_cuda:
                dmu = torch.from_numpy(dmu)
            ctx.save_for_backward(dmu.to(mu0.dtype).reshape(mu0.shape),
                                  torch.tensor(dpar, dtype=torch.float64))
            return torch.tensor(J, dtype=torch.float64, device=mu0.device)

        @staticmethod
        def backward(ctx, g):
            dmu, dpar = ctx.saved_tensors
            gd = g.to(torch.float64).cpu()
            return ((g.to(dmu.dtype) * dmu), (gd * dpar[0]), (gd * dpar[1]), (gd * dpar[2]),
                    None, None, None, None, None)

    return GPFLBMFunction


_function = None


def GPFLBMFunction():
    """The torch.autograd.Function class (created on first use)."""
    global _function
    if _function is None:
        _function = _make_function()
    return _function
