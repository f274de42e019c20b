"""Thin ctypes binding of libgks.so (the C ABI of include/gks_api.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of the library. torch provides the device memory (the state and work
buffers are torch uint8 tensors owned by :class:`Grid`) and the stream. The
functions of the C ABI are available under their own names as attributes of
:data:`lib` after :func:`load`. There is no CPU fallback: loading raises if
the library has not been built or no CUDA device is present.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

GKS_OK = 0
ERRORS = {-1: "GKS_ERR_ARG", -2: "GKS_ERR_CUDA", -3: "GKS_ERR_NONFINITE", -4: "GKS_ERR_CFL",
          -5: "GKS_ERR_STATE", -6: "GKS_ERR_RANGE",
          -7: "GKS_ERR_DEBUG_BOUNDS"}
FP64, FP32C = 0, 1
PRECISIONS = {"fp64": FP64, "fp32c": FP32C}
MAX_BLADES = 8

_dp = C.POINTER(C.c_double)


class GridDesc(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("faces", _dp * 3), ("mach", C.c_double), ("u_ref", C.c_double),
                ("mu", C.c_double), ("bc", (C.c_int * 2) * 3), ("precision", C.c_int), ("cfl", C.c_double),
                ("dt_fixed", C.c_double), ("rho_ref", C.c_double), ("stream", C.c_void_p)]


class RotorDesc(C.Structure):
    _fields_ = [("n_blades", C.c_int), ("n_pts", C.c_int), ("hub", C.c_double * 3), ("omega", C.c_double),
                ("azimuth0", C.c_double), ("radius", C.c_double), ("eps", C.c_double),
                ("rho_inf", C.c_double), ("u_inf_ref", C.c_double), ("r", _dp), ("chord", _dp),
                ("twist", _dp), ("width", _dp), ("correction", C.c_int),
                ("tip_correction", C.c_int)]


class ForcesOut(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_blades", C.c_int), ("thrust", C.c_double * MAX_BLADES),
                ("torque", C.c_double * MAX_BLADES), ("power", C.c_double), ("cp", C.c_double),
                ("ct", C.c_double), ("body_force", C.c_double * 3), ("iters", C.c_int),
                ("residual", C.c_double)]


NUM_KERNEL_GROUPS = 9


class ProfileOut(C.Structure):
    _fields_ = [("launches", C.c_long * NUM_KERNEL_GROUPS), ("ms", C.c_double * NUM_KERNEL_GROUPS),
                ("total_launches", C.c_long)]


# name -> (restype, argtypes); every entry point that include/gks_api.h declares
SIGNATURES = {
    "gks_workspace_bytes": (C.c_int, [C.POINTER(GridDesc), C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "gks_create_grid": (C.c_int, [C.POINTER(GridDesc), C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "gks_destroy_grid": (C.c_int, [C.c_void_p]),
    "gks_last_error": (C.c_char_p, [C.c_void_p]),
    "gks_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gks_set_state": (C.c_int, [C.c_void_p, _dp]),
    "gks_get_state": (C.c_int, [C.c_void_p, _dp]),
    "gks_set_inflow": (C.c_int, [C.c_void_p] + [C.c_double] * 4),
    "gks_set_body_force": (C.c_int, [C.c_void_p] + [C.c_double] * 3),
    "gks_add_actuator_lines": (C.c_int, [C.c_void_p, C.POINTER(RotorDesc), C.POINTER(C.c_int)]),
    "gks_set_force_scales": (C.c_int, [C.c_void_p, C.c_int, _dp]),
    "gks_add_ib_points": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, C.c_double, C.c_int, C.c_double,
                                    C.POINTER(C.c_int)]),
    "gks_step": (C.c_int, [C.c_void_p, C.c_int, _dp]),
    "gks_slab_step": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, _dp]),
    "gks_set_slab_lattice": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int]),
    "gks_share_actuator_lines": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int)]),
    "gks_get_time": (C.c_int, [C.c_void_p, _dp, _dp]),
    "gks_set_time": (C.c_int, [C.c_void_p, C.c_double]),
    "gks_forces": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(ForcesOut), _dp]),
    "gks_diagnostics": (C.c_int, [C.c_void_p, _dp]),
    "gks_checkpoint_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "gks_save_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "gks_load_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "gks_state_layout": (C.c_int, [C.c_void_p, C.POINTER(C.c_long)]),
    "gks_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "gks_profile_read": (C.c_int, [C.c_void_p, C.POINTER(ProfileOut)]),
    "gks_kernel_group_name": (C.c_char_p, [C.c_int]),
    "gks_set_state_device": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gks_get_state_device": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gks_adjoint_workspace_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "gks_forces_record_len": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_size_t)]),
    "gks_step_async": (C.c_int, [C.c_void_p, C.c_int]),
    "gks_set_graphs": (C.c_int, [C.c_void_p, C.c_int]),
    "gks_set_fp64_arithmetic": (C.c_int, [C.c_void_p, C.c_int]),
    "gks_sync": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "gks_forces_async": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]),
    "gks_adjoint_tape_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "gks_adjoint_scratch_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "gks_step_record": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "gks_step_reverse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                   _dp, _dp]),
    "gks_set_adjoint_precision": (C.c_int, [C.c_void_p, C.c_int]),
    "gks_step_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_double, _dp, _dp]),
    "gks_diagnostics_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p]),
    "gks_alu_peak_probe": (C.c_int, [C.c_int, C.c_long, C.c_void_p, C.c_void_p, _dp]),
}

lib = None


def library_path() -> str:
    """The plain library, or the debug-bounds one when the environment
    variable GKS_DEBUG_BOUNDS=1 (built by ``build.build(debug=True)``)."""
    return _build.LIB_DEBUG if os.environ.get("GKS_DEBUG_BOUNDS") == "1" else _build.LIB


def load(path: str | None = None):
    """Load libgks.so (built in-tree by ``build.build()``) and declare the
    signatures. Raises when the library is missing."""
    global lib
    if lib is not None:
        return lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError("libgks.so is not built (%s); run paper_2603_11102_gb300.build.build()" % path)
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    lib = L
    return L


class GKSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


def _check(rc, handle=None):
    if rc != GKS_OK:
        msg = lib.gks_last_error(handle)
        raise GKSError(rc, msg.decode() if msg else "")


def _arr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


class Grid:
    """One grid on the current CUDA device; device buffers are torch tensors.

    Parameters mirror ``gks_grid_desc``; ``bc`` is [(lo, hi)] per axis with the
    integer kinds of the C ABI (0 periodic, 1 no-slip, 2 slip, 3 inflow,
    4 outflow, 5 exchange: an x side shared with the next slab of a
    :class:`SlabGroup`)."""

    def __init__(self, n, faces, mach, u_ref, mu, bc, precision="fp64", cfl=0.5, dt_fixed=0.0,
                 rho_ref=1.0, device=None, stream=None):
        import torch
        load()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device")
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.n = tuple(int(x) for x in n)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._faces = [np.ascontiguousarray(f, dtype=np.float64) for f in faces]
        d = GridDesc()
        for a in range(3):
            d.n[a] = self.n[a]
            d.faces[a] = self._faces[a].ctypes.data_as(_dp)
            d.bc[a][0] = int(bc[a][0])
            d.bc[a][1] = int(bc[a][1])
        d.mach, d.u_ref, d.mu = float(mach), float(u_ref), float(mu)
        d.precision = self.precision
        d.cfl, d.dt_fixed, d.rho_ref = float(cfl), float(dt_fixed), float(rho_ref)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        d.stream = C.c_void_p(stream.cuda_stream)
        self._desc = d
        self.dt_fixed = float(dt_fixed)
        sb, wb = C.c_size_t(), C.c_size_t()
        _check(lib.gks_workspace_bytes(C.byref(d), C.byref(sb), C.byref(wb)))
        self.state_bytes, self.work_bytes = sb.value, wb.value
        self.state_buf = torch.empty(self.state_bytes, dtype=torch.uint8, device=self.device)
        self.work_buf = torch.empty(self.work_bytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        _check(lib.gks_create_grid(C.byref(d), C.c_void_p(self.state_buf.data_ptr()),
                                   C.c_void_p(self.work_buf.data_ptr()), C.byref(h)))
        self.h = h
        self.objects = []

    @classmethod
    def from_workload(cls, w, precision="fp64", **kw):
        g = cls(w.n, w.faces, w.mach, w.u_ref, w.mu, w.bc, precision=precision, cfl=w.cfl,
                dt_fixed=w.dt_fixed, rho_ref=w.rho_ref, **kw)
        g.set_inflow(*w.inflow)
        g.set_body_force(*w.body_force)
        for r in w.rotors:
            g.add_rotor(r)
        for b in w.bodies:
            g.add_body(b)
        if w.state0 is not None:
            g.set_state(w.state0)
        return g

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib.gks_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (4, self.n[2], self.n[1], self.n[0])

    def set_state(self, Q):
        Q, p = _arr(np.asarray(Q).reshape(self.shape))
        _check(lib.gks_set_state(self.h, p), self.h)
        self.stream.synchronize()

    def set_state_pinned(self, host_tensor):
        """Asynchronous upload from a page-locked float64 torch tensor."""
        _check(lib.gks_set_state(self.h, C.cast(host_tensor.data_ptr(), _dp)), self.h)

    def get_state(self):
        Q = np.zeros(self.shape)
        _check(lib.gks_get_state(self.h, Q.ctypes.data_as(_dp)), self.h)
        return Q

    def set_inflow(self, rho, u, v=0.0, w=0.0):
        _check(lib.gks_set_inflow(self.h, float(rho), float(u), float(v), float(w)), self.h)

    def set_body_force(self, fx, fy=0.0, fz=0.0):
        _check(lib.gks_set_body_force(self.h, float(fx), float(fy), float(fz)), self.h)

    def add_rotor(self, rot):
        arrs = [_arr(x) for x in (rot.r, rot.chord, rot.twist, rot.width)]
        d = RotorDesc()
        d.n_blades, d.n_pts = int(rot.n_blades), int(arrs[0][0].size)
        for a in range(3):
            d.hub[a] = float(rot.hub[a])
        d.omega, d.azimuth0, d.radius, d.eps = float(rot.omega), float(rot.azimuth0), float(rot.radius), float(rot.eps)
        d.rho_inf, d.u_inf_ref = float(rot.rho_inf), float(rot.u_inf_ref)
        d.r, d.chord, d.twist, d.width = (p for _, p in arrs)
        d.correction = int(bool(rot.correction))
        d.tip_correction = int(bool(getattr(rot, "tip_correction", False)))
        rid = C.c_int()
        _check(lib.gks_add_actuator_lines(self.h, C.byref(d), C.byref(rid)), self.h)
        self.objects.append(("rotor", d.n_blades, d.n_pts))
        return rid.value

    def set_slab_lattice(self, x0, hx, cells_before):
        """The x lattice of a slab group's domain (gks_set_slab_lattice)."""
        _check(lib.gks_set_slab_lattice(self.h, float(x0), float(hx), int(cells_before)), self.h)

    def share_rotor(self, owner, rid):
        """This slab's share of rotor rid of the neighbouring slab owner
        (gks_share_actuator_lines); returns the share's object id."""
        out = C.c_int()
        _check(lib.gks_share_actuator_lines(owner.h, int(rid), self.h, C.byref(out)), self.h)
        self.objects.append(owner.objects[rid])   # its loads are the owner's
        return out.value

    def set_force_scales(self, rid, s):
        s, p = _arr(s)
        _check(lib.gks_set_force_scales(self.h, int(rid), p), self.h)

    def add_body(self, body):
        xyz, px = _arr(body.xyz)
        dS, pd = _arr(body.dS)
        if body.vel is None:
            pv = None
        else:
            vel, pv = _arr(body.vel)
        bid = C.c_int()
        _check(lib.gks_add_ib_points(self.h, int(dS.size), px, pd, pv, float(body.eps), int(body.niter),
                                     float(body.tol), C.byref(bid)), self.h)
        self.objects.append(("body", int(dS.size), int(body.niter)))
        return bid.value

    def step(self, nsteps=1, sync=True):
        """nsteps steps; returns the time after them. sync=False enqueues
        them without waiting (returns None; errors flagged on the device
        surface at the next synchronising step or sync())."""
        if not sync:
            _check(lib.gks_step_async(self.h, int(nsteps)), self.h)
            return None
        t = C.c_double()
        _check(lib.gks_step(self.h, int(nsteps), C.byref(t)), self.h)
        return t.value

    def set_graphs(self, on=True):
        """Replay a CUDA graph of one step in the steady state (see
        gks_set_graphs); the same results as plain steps."""
        _check(lib.gks_set_graphs(self.h, int(bool(on))), self.h)

    def sync(self):
        """Wait for the grid's stream; report device-side errors; the time."""
        t = C.c_double()
        _check(lib.gks_sync(self.h, C.byref(t)), self.h)
        return t.value

    @property
    def time(self):
        t, dt = C.c_double(), C.c_double()
        _check(lib.gks_get_time(self.h, C.byref(t), C.byref(dt)), self.h)
        return t.value

    @property
    def last_dt(self):
        t, dt = C.c_double(), C.c_double()
        _check(lib.gks_get_time(self.h, C.byref(t), C.byref(dt)), self.h)
        return dt.value

    def set_time(self, t):
        _check(lib.gks_set_time(self.h, float(t)), self.h)

    def forces(self, oid):
        kind, a, b = self.objects[oid]
        out = ForcesOut()
        if kind == "rotor":
            pts = np.zeros(4 * a * b)
            _check(lib.gks_forces(self.h, int(oid), C.byref(out), pts.ctypes.data_as(_dp)), self.h)
            nb, npt = a, b
            return {"thrust": np.array(out.thrust[:nb]), "torque": np.array(out.torque[:nb]),
                    "power": out.power, "cp": out.cp, "ct": out.ct,
                    "Fx": pts[:nb * npt].reshape(nb, npt), "Ft": pts[nb * npt:2 * nb * npt].reshape(nb, npt),
                    "alpha": pts[2 * nb * npt:3 * nb * npt].reshape(nb, npt),
                    "phi": pts[3 * nb * npt:].reshape(nb, npt)}
        res = np.zeros(b)
        _check(lib.gks_forces(self.h, int(oid), C.byref(out), res.ctypes.data_as(_dp)), self.h)
        return {"force": np.array(out.body_force[:]), "iters": out.iters, "residual": out.residual,
                "residual_history": res[:out.iters].copy()}

    def forces_record(self, oid):
        """A page-locked float64 tensor for the load record of object oid
        (see forces_async)."""
        import torch
        n = C.c_size_t()
        _check(lib.gks_forces_record_len(self.h, int(oid), C.byref(n)), self.h)
        return torch.empty(n.value, dtype=torch.float64).pin_memory()

    def forces_async(self, oid, record):
        """Enqueue on the grid's stream the copy of object oid's load record
        (rotor: thrust per blade, torque per blade, power, C_P, C_T) into the
        page-locked tensor `record`; read it after the stream (an event
        recorded on it) has reached that point."""
        _check(lib.gks_forces_async(self.h, int(oid), C.c_void_p(record.data_ptr()), record.numel()), self.h)

    def diagnostics(self):
        out = np.zeros(5)
        _check(lib.gks_diagnostics(self.h, out.ctypes.data_as(_dp)), self.h)
        return out

    def save_state(self) -> bytes:
        nb = C.c_size_t()
        _check(lib.gks_checkpoint_bytes(self.h, C.byref(nb)), self.h)
        buf = C.create_string_buffer(nb.value)
        _check(lib.gks_save_state(self.h, buf, nb.value), self.h)
        return buf.raw

    def load_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib.gks_load_state(self.h, buf, len(blob)), self.h)

    def state_tensor(self):
        """The conserved state as a (4, nz, ny, nx) float64 tensor on the device."""
        import torch
        out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        _check(lib.gks_get_state_device(self.h, C.c_void_p(out.data_ptr())), self.h)
        return out

    def set_state_tensor(self, t, sync=True):
        """Enqueue the scatter of a (4, nz, ny, nx) float64 device tensor into
        the state on the grid's stream. sync=False returns at once: the caller
        keeps t alive and unchanged until the grid's stream has passed the
        scatter (t must then already be float64, contiguous, on this device)."""
        import torch
        if not sync:
            if t.dtype != torch.float64 or not t.is_contiguous() or t.device != self.device:
                raise ValueError("sync=False needs a contiguous float64 tensor on the grid's device")
            _check(lib.gks_set_state_device(self.h, C.c_void_p(t.data_ptr())), self.h)
            return
        t = t.to(device=self.device, dtype=torch.float64).contiguous()
        _check(lib.gks_set_state_device(self.h, C.c_void_p(t.data_ptr())), self.h)
        self.stream.synchronize()

    def set_adjoint_precision(self, precision):
        """Arithmetic of the local reverse maps of step_adjoint: "fp64" or
        "fp32" (FP64 recompute, storage and sums either way)."""
        code = {"fp64": PRECISIONS["fp64"], "fp32": PRECISIONS["fp32c"]}[precision]
        _check(lib.gks_set_adjoint_precision(self.h, code), self.h)

    def adjoint_workspace(self):
        import torch
        nb = C.c_size_t()
        _check(lib.gks_adjoint_workspace_bytes(self.h, C.byref(nb)))
        return torch.empty(nb.value, dtype=torch.uint8, device=self.device)

    def adjoint_tape_bytes(self):
        nb = C.c_size_t()
        _check(lib.gks_adjoint_tape_bytes(self.h, C.byref(nb)))
        return nb.value

    def adjoint_tape(self):
        """Device buffer for the tape of one recorded step."""
        import torch
        return torch.empty(self.adjoint_tape_bytes(), dtype=torch.uint8, device=self.device)

    def adjoint_scratch(self):
        """Device scratch of step_reverse."""
        import torch
        nb = C.c_size_t()
        _check(lib.gks_adjoint_scratch_bytes(self.h, C.byref(nb)))
        return torch.empty(nb.value, dtype=torch.uint8, device=self.device)

    def step_record(self, tape):
        """One step of the grid (as step(1)) that also fills tape; returns
        the time after the step."""
        t = C.c_double()
        _check(lib.gks_step_record(self.h, C.c_void_p(tape.data_ptr()), C.byref(t)), self.h)
        return t.value

    def step_reverse(self, tape, scratch, adj_np1, power_seed=0.0, grad_scales=None):
        """Reverse of the recorded step: returns (lambda^n, grad_uinf of the
        step); adds its force-scale gradient into grad_scales (numpy). The
        tape is only read: it can be reversed again (another seed)."""
        import torch
        adj_np1 = adj_np1.to(self.device, torch.float64).contiguous()
        out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        gu = C.c_double(0.0)
        gs = None if grad_scales is None else grad_scales.ctypes.data_as(_dp)
        _check(lib.gks_step_reverse(self.h, C.c_void_p(tape.data_ptr()), C.c_void_p(scratch.data_ptr()),
                                    C.c_void_p(adj_np1.data_ptr()), C.c_void_p(out.data_ptr()), float(power_seed),
                                    gs, C.byref(gu)), self.h)
        return out, gu.value

    def step_adjoint(self, work, t_n, state_n, adj_np1, power_seed=0.0, grad_scales=None):
        """One reverse step: returns (lambda^n, grad_uinf of this step); adds
        the force-scale gradient of this step into grad_scales (numpy)."""
        import torch
        state_n = state_n.to(self.device, torch.float64).contiguous()
        adj_np1 = adj_np1.to(self.device, torch.float64).contiguous()
        out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        gu = C.c_double(0.0)
        gs = None if grad_scales is None else grad_scales.ctypes.data_as(_dp)
        _check(lib.gks_step_adjoint(self.h, C.c_void_p(work.data_ptr()), float(t_n), C.c_void_p(state_n.data_ptr()),
                                    C.c_void_p(adj_np1.data_ptr()), C.c_void_p(out.data_ptr()), float(power_seed),
                                    gs, C.byref(gu)), self.h)
        return out, gu.value

    def set_fp64_arithmetic(self, mode):
        """"fp64" (default) or "ds": double-single reconstruction and flux on
        an FP64 grid (gks_set_fp64_arithmetic)."""
        if mode not in ("fp64", "ds"):
            raise ValueError(mode)
        _check(lib.gks_set_fp64_arithmetic(self.h, int(mode == "ds")), self.h)

    def profile_enable(self, timing=True):
        _check(lib.gks_profile_enable(self.h, int(bool(timing))), self.h)

    def profile_read(self):
        out = ProfileOut()
        _check(lib.gks_profile_read(self.h, C.byref(out)), self.h)
        return {"launches": {lib.gks_kernel_group_name(k).decode(): out.launches[k]
                             for k in range(NUM_KERNEL_GROUPS)},
                "ms": {lib.gks_kernel_group_name(k).decode(): out.ms[k] for k in range(NUM_KERNEL_GROUPS)},
                "total_launches": out.total_launches}

    def layout(self):
        out = (C.c_long * 7)()
        _check(lib.gks_state_layout(self.h, out), self.h)
        return list(out)


def alu_peak_probe(kind, iters: int, sink, stream) -> float:
    """Launch the FMA-loop peak probe of the library on stream (async); sink
    is a device tensor of at least 4 x SMs doubles. kind: False / 0 FP32,
    True / 1 FP64, 2 FP32 packed pairs. Returns the operations of that
    launch; time it with CUDA events on the same stream."""
    load()
    out = C.c_double(0.0)
    rc = lib.gks_alu_peak_probe(int(kind), int(iters), C.c_void_p(sink.data_ptr()),
                                C.c_void_p(stream.cuda_stream), C.byref(out))
    if rc != GKS_OK:
        raise GKSError(rc, lib.gks_last_error(None).decode())
    return out.value


EXCHANGE = 5


def plan_slabs(w, cuts):
    """The slabs of a workload cut along x at the cell indices ``cuts``: per
    slab its cells, faces, boundary kinds (exchange sides between slabs, and
    at both ends of a periodic x axis) and share of the initial state; and
    the slab of every rotor (by its hub) and body (by the mean x of its
    points), in the workload's order. Host-side bookkeeping (no device)."""
    nx = int(w.n[0])
    cuts = [0] + [int(c) for c in cuts] + [nx]
    if any(b - a < 3 for a, b in zip(cuts[:-1], cuts[1:])):
        raise ValueError("every slab needs at least 3 x cells: %s" % (cuts,))
    periodic = w.bc[0][0] == 0
    ns = len(cuts) - 1
    fx = np.asarray(w.faces[0], dtype=np.float64)
    slabs = []
    for s in range(ns):
        a, b = cuts[s], cuts[s + 1]
        lo = EXCHANGE if (s > 0 or periodic) else w.bc[0][0]
        hi = EXCHANGE if (s + 1 < ns or periodic) else w.bc[0][1]
        slabs.append({"n": (b - a, w.n[1], w.n[2]), "faces": [fx[a:b + 1], w.faces[1], w.faces[2]], "cells_before": a,
                      "bc": [(lo, hi), tuple(w.bc[1]), tuple(w.bc[2])],
                      "state0": None if w.state0 is None else np.ascontiguousarray(w.state0[:, :, :, a:b])})

    def slab_of(x):
        for s in range(ns):
            f0, f1 = fx[cuts[s]], fx[cuts[s + 1]]
            if f0 <= x < f1 or (s == ns - 1 and x == f1):
                return s
        raise ValueError("x = %g outside the domain" % x)

    h = fx[1] - fx[0]
    xc = 0.5 * (fx[1:] + fx[:-1])

    def rotor_slabs(r):
        # the owner samples the hub plane: both cell centres around it inside
        # the slab; the slabs that the 3 eps support (with a cell of margin)
        # reaches get shares
        owner = None
        for s in range(ns):
            if xc[cuts[s]] <= r.hub[0] <= xc[cuts[s + 1] - 1]:
                owner = s
        if owner is None:
            raise ValueError("a cut lies within half a cell of the rotor plane at x = %g" % r.hub[0])
        lo, hi = r.hub[0] - 3 * r.eps - 2 * h, r.hub[0] + 3 * r.eps + 2 * h
        shares = [s for s in range(ns) if s != owner and fx[cuts[s]] < hi and fx[cuts[s + 1]] > lo]
        return owner, shares

    objects, shares = [], []
    for r in w.rotors:
        owner, sh = rotor_slabs(r)
        objects.append(("rotor", r, owner))
        shares.append(sh)
    objects += [("body", b, slab_of(float(np.mean(np.asarray(b.xyz).reshape(-1, 3)[:, 0])))) for b in w.bodies]
    return {"cuts": cuts, "slabs": slabs, "objects": objects, "rotor_shares": shares,
            "lattice": (float(fx[0]), float(h))}


class SlabGroup:
    """A workload's domain split along x into slabs at the cell indices
    ``cuts`` (0 < c_1 < c_2 < ... < n_x), one grid per slab on the same device
    and stream, stepped together by ``gks_slab_step`` (the halo exchange of
    every stage, the common time step). Each rotor and body goes to the slab
    that holds its x position (its kernel support must not reach a cut).
    Host-side bookkeeping only: splitting the faces, the boundary kinds and
    the initial state, and joining the slabs' states."""

    def __init__(self, w, cuts, precision="fp64", **kw):
        plan = plan_slabs(w, cuts)
        self.cuts = plan["cuts"]
        self.slabs = []
        for sp in plan["slabs"]:
            g = Grid(sp["n"], sp["faces"], w.mach, w.u_ref, w.mu, sp["bc"], precision=precision, cfl=w.cfl,
                     dt_fixed=w.dt_fixed, rho_ref=w.rho_ref,
                     stream=self.slabs[0].stream if self.slabs else kw.get("stream"), device=kw.get("device"))
            g.set_inflow(*w.inflow)
            g.set_body_force(*w.body_force)
            if sp["state0"] is not None:
                g.set_state(sp["state0"])
            if w.rotors or w.bodies:
                g.set_slab_lattice(plan["lattice"][0], plan["lattice"][1], sp["cells_before"])
            self.slabs.append(g)
        # object id of the whole workload -> (slab, id in that slab)
        self.objects = []
        for k, (kind, obj, s) in enumerate(plan["objects"]):
            sid = self.slabs[s].add_rotor(obj) if kind == "rotor" else self.slabs[s].add_body(obj)
            self.objects.append((s, sid))
            if kind == "rotor":
                for t in plan["rotor_shares"][k]:
                    self.slabs[t].share_rotor(self.slabs[s], sid)
        self._handles = (C.c_void_p * len(self.slabs))(*[g.h for g in self.slabs])

    def step(self, nsteps=1):
        t = C.c_double()
        _check(lib.gks_slab_step(self._handles, len(self.slabs), int(nsteps), C.byref(t)))
        return t.value

    def get_state(self):
        """The (4, nz, ny, nx) FP64 state of the whole domain."""
        return np.concatenate([g.get_state() for g in self.slabs], axis=3)

    def forces(self, oid):
        s, i = self.objects[oid]
        return self.slabs[s].forces(i)

    def close(self):
        for g in self.slabs:
            g.close()

