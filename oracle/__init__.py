"""Plain FP64 CPU oracle of the S2O4 gas-kinetic step with ALM/IBM forcing.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The product path (the
CUDA library and its Python binding) never imports this package.

The C source (``gks_oracle.c``) follows the paper step by step (Sec. 2, Sec. 3
and the Appendix); this module only marshals arguments through ctypes and
builds the shared library with gcc on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gks_oracle.c")
_HDR = os.path.join(_HERE, "gks_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libgks_oracle.so")
_lock = threading.Lock()
_lib = None

BC = {"periodic": 0, "noslip": 1, "slip": 2, "inflow": 3, "outflow": 4}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_lp = C.POINTER(C.c_long)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over k-planes)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        sig = {
            "og_create": (C.c_void_p, [_ip, _dp, _dp, _dp, C.c_double, C.c_double, C.c_double,
                                       _ip, C.c_double, C.c_double]),
            "og_destroy": (None, [C.c_void_p]),
            "og_last_error": (C.c_char_p, [C.c_void_p]),
            "og_num_cells": (C.c_long, [C.c_void_p]),
            "og_set_inflow": (None, [C.c_void_p] + [C.c_double] * 4),
            "og_set_body_force": (None, [C.c_void_p] + [C.c_double] * 3),
            "og_set_state": (None, [C.c_void_p, _dp]),
            "og_get_state": (None, [C.c_void_p, _dp]),
            "og_time": (C.c_double, [C.c_void_p]),
            "og_last_dt": (C.c_double, [C.c_void_p]),
            "og_set_time": (None, [C.c_void_p, C.c_double]),
            "og_cfl_dt": (C.c_double, [C.c_void_p]),
            "og_step": (C.c_int, [C.c_void_p, C.c_int]),
            "og_rhs": (None, [C.c_void_p, _dp, _dp, _dp]),
            "og_ghost_filled": (None, [C.c_void_p, _dp, _dp]),
            "og_diagnostics": (None, [C.c_void_p, _dp]),
            "og_add_rotor": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _dp, C.c_double, C.c_double,
                                       C.c_double, C.c_double, C.c_double, C.c_double, _dp, _dp,
                                       _dp, _dp, C.c_int, C.c_int]),
            "og_set_force_scales": (C.c_int, [C.c_void_p, C.c_int, _dp]),
            "og_add_body": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, C.c_double, C.c_int,
                                      C.c_double]),
            "og_body_fields": (C.c_long, [C.c_void_p, C.c_int, _lp, _dp, _dp]),
            "og_forces": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp]),
            "og_set_threads": (None, [C.c_int]),
            "og_get_threads": (C.c_int, []),
            "og_weno5": (C.c_double, [_dp]),
            "og_weno5_parts": (None, [_dp, _dp, _dp, _dp]),
            "og_normal_derivative": (C.c_double, [C.c_double, _dp]),
            "og_tangential": (None, [_dp, _dp, _dp]),
            "og_linear5_face": (C.c_double, [_dp]),
            "og_stencil_table": (None, [_dp, _dp, _dp, _dp]),
            "og_moments": (None, [C.c_double, C.c_double, C.c_int, _dp]),
            "og_half_moments": (None, [C.c_double, C.c_double, C.c_int, _dp]),
            "og_coeff_solve": (None, [C.c_double, C.c_double, C.c_double, C.c_double, _dp, _dp]),
            "og_flux_local": (None, [C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp, _dp]),
            "og_equilibrium_local": (None, [C.c_double, _dp, _dp, _dp]),
            "og_gauss_kernel": (C.c_double, [C.c_double, C.c_double]),
            "og_s2o4_stage1": (None, [C.c_long, C.c_double, _dp, _dp, _dp, _dp]),
            "og_s2o4_stage2": (None, [C.c_long, C.c_double, _dp, _dp, _dp, _dp, _dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def set_threads(n: int) -> None:
    _load().og_set_threads(int(n))


def get_threads() -> int:
    return int(_load().og_get_threads())


# --- building blocks (pins) -------------------------------------------------

def weno5(q):
    q, p = _d(q)
    return _load().og_weno5(p)


def weno5_parts(q):
    q, p = _d(q)
    a, b, c = np.zeros(3), np.zeros(3), np.zeros(3)
    _load().og_weno5_parts(p, _d(a)[1], _d(b)[1], _d(c)[1])
    return a, b, c


def normal_derivative(q0, cells):
    c, p = _d(cells)
    return _load().og_normal_derivative(float(q0), p)


def tangential(q):
    q, p = _d(q)
    val, der = np.zeros(2), np.zeros(2)
    _load().og_tangential(p, val.ctypes.data_as(_dp), der.ctypes.data_as(_dp))
    return val, der


def linear5_face(q):
    q, p = _d(q)
    return _load().og_linear5_face(p)


def stencil_table():
    dn, tv, td, wd = np.zeros(5), np.zeros(10), np.zeros(10), np.zeros(3)
    _load().og_stencil_table(*(x.ctypes.data_as(_dp) for x in (dn, tv, td, wd)))
    return dn, tv.reshape(2, 5), td.reshape(2, 5), wd


def moments(U, lam, kmax):
    M = np.zeros(kmax + 1)
    _load().og_moments(float(U), float(lam), int(kmax), M.ctypes.data_as(_dp))
    return M


def half_moments(U, lam, sign):
    out = np.zeros(2)
    _load().og_half_moments(float(U), float(lam), int(sign), out.ctypes.data_as(_dp))
    return out


def coeff_solve(U, V, W, lam, d):
    d, p = _d(d)
    a = np.zeros(4)
    _load().og_coeff_solve(float(U), float(V), float(W), float(lam), p, a.ctypes.data_as(_dp))
    return a


def flux_local(lam, mu, Q, Dn, Dt1, Dt2):
    arrs = [_d(x) for x in (Q, Dn, Dt1, Dt2)]
    F0, F1 = np.zeros(4), np.zeros(4)
    _load().og_flux_local(float(lam), float(mu), *(p for _, p in arrs),
                          F0.ctypes.data_as(_dp), F1.ctypes.data_as(_dp))
    return F0, F1


def equilibrium_local(lam, Ql, Qr):
    (_, pl), (_, pr) = _d(Ql), _d(Qr)
    Q0 = np.zeros(4)
    _load().og_equilibrium_local(float(lam), pl, pr, Q0.ctypes.data_as(_dp))
    return Q0


def gauss_kernel(r, eps):
    return _load().og_gauss_kernel(float(r), float(eps))


def s2o4_stage1(dt, W, L, Lt):
    W, pw = _d(W)
    (_, pl), (_, plt) = _d(L), _d(Lt)
    out = np.zeros_like(W)
    _load().og_s2o4_stage1(W.size, float(dt), pw, pl, plt, out.ctypes.data_as(_dp))
    return out


def s2o4_stage2(dt, W, L, Lt, Lts):
    W, pw = _d(W)
    (_, pl), (_, plt), (_, plts) = _d(L), _d(Lt), _d(Lts)
    out = np.zeros_like(W)
    _load().og_s2o4_stage2(W.size, float(dt), pw, pl, plt, plts, out.ctypes.data_as(_dp))
    return out


# --- whole-grid driver --------------------------------------------------------

class OracleGrid:
    """One grid of the oracle. State arrays are (4, nz, ny, nx) float64 with
    components (rho, rho U, rho V, rho W)."""

    def __init__(self, n, faces, mach, u_ref, mu, bc, cfl=0.5, dt_fixed=0.0):
        self.lib = _load()
        self.n = tuple(int(x) for x in n)
        self._faces = [np.ascontiguousarray(f, dtype=np.float64) for f in faces]
        for d in range(3):
            assert self._faces[d].shape == (self.n[d] + 1,)
        nn = (C.c_int * 3)(*self.n)
        bcs = []
        for d in range(3):
            lo, hi = bc[d]
            bcs += [BC[lo] if isinstance(lo, str) else int(lo), BC[hi] if isinstance(hi, str) else int(hi)]
        bb = (C.c_int * 6)(*bcs)
        self.h = self.lib.og_create(nn, *(f.ctypes.data_as(_dp) for f in self._faces), float(mach),
                                    float(u_ref), float(mu), bb, float(cfl), float(dt_fixed))
        if not self.h:
            raise ValueError("oracle rejected the grid description")
        self.nobj_kind = []

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.og_destroy(h)
            self.h = None

    @property
    def shape(self):
        return (4, self.n[2], self.n[1], self.n[0])

    def set_state(self, Q):
        Q, p = _d(np.asarray(Q).reshape(self.shape))
        self.lib.og_set_state(self.h, p)

    def get_state(self):
        Q = np.zeros(self.shape)
        self.lib.og_get_state(self.h, Q.ctypes.data_as(_dp))
        return Q

    def set_inflow(self, rho, u, v=0.0, w=0.0):
        self.lib.og_set_inflow(self.h, float(rho), float(u), float(v), float(w))

    def set_body_force(self, fx, fy=0.0, fz=0.0):
        self.lib.og_set_body_force(self.h, float(fx), float(fy), float(fz))

    @property
    def time(self):
        return self.lib.og_time(self.h)

    @time.setter
    def time(self, t):
        self.lib.og_set_time(self.h, float(t))

    @property
    def last_dt(self):
        return self.lib.og_last_dt(self.h)

    def cfl_dt(self):
        return self.lib.og_cfl_dt(self.h)

    def step(self, nsteps=1):
        if self.lib.og_step(self.h, int(nsteps)) != 0:
            raise RuntimeError(self.lib.og_last_error(self.h).decode())

    def rhs(self, Q):
        Q, p = _d(np.asarray(Q).reshape(self.shape))
        L, Lt = np.zeros(self.shape), np.zeros(self.shape)
        self.lib.og_rhs(self.h, p, L.ctypes.data_as(_dp), Lt.ctypes.data_as(_dp))
        return L, Lt

    def ghost_filled(self, Q):
        Q, p = _d(np.asarray(Q).reshape(self.shape))
        G = 3
        out = np.zeros((4, self.n[2] + 2 * G, self.n[1] + 2 * G, self.n[0] + 2 * G))
        self.lib.og_ghost_filled(self.h, p, out.ctypes.data_as(_dp))
        return out

    def diagnostics(self):
        out = np.zeros(5)
        self.lib.og_diagnostics(self.h, out.ctypes.data_as(_dp))
        return out

    def add_rotor(self, nb, r, chord, twist, width, hub, omega, azimuth0, radius, eps,
                  rho_inf=1.0, u_inf_ref=1.0, correction=False, tip_correction=False):
        arrs = [_d(x) for x in (r, chord, twist, width)]
        npt = arrs[0][0].size
        hub_a, hp = _d(hub)
        rid = self.lib.og_add_rotor(self.h, int(nb), int(npt), hp, float(omega), float(azimuth0),
                                    float(radius), float(eps), float(rho_inf), float(u_inf_ref),
                                    *(p for _, p in arrs), int(bool(correction)), int(bool(tip_correction)))
        if rid < 0:
            raise ValueError(self.lib.og_last_error(self.h).decode())
        self.nobj_kind.append(("rotor", int(nb), int(npt)))
        return rid

    def set_force_scales(self, rid, s):
        s, p = _d(s)
        if self.lib.og_set_force_scales(self.h, int(rid), p) != 0:
            raise ValueError("bad rotor id")

    def add_body(self, xyz, dS, eps, vel=None, niter=5, tol=0.0):
        xyz, px = _d(xyz)
        dS, pd = _d(dS)
        n = dS.size
        if vel is None:
            pv = None
        else:
            vel, pv = _d(vel)
        bid = self.lib.og_add_body(self.h, int(n), px, pd, pv, float(eps), int(niter), float(tol))
        if bid < 0:
            raise ValueError(self.lib.og_last_error(self.h).decode())
        self.nobj_kind.append(("body", int(n), int(niter)))
        return bid

    def body_fields(self, bid):
        bb = (C.c_long * 6)()
        nbx = self.lib.og_body_fields(self.h, int(bid), bb, None, None)
        Vb, ph = np.zeros(nbx), np.zeros(nbx)
        self.lib.og_body_fields(self.h, int(bid), bb, Vb.ctypes.data_as(_dp), ph.ctypes.data_as(_dp))
        box = [(bb[2 * d], bb[2 * d + 1]) for d in range(3)]
        shape = tuple(box[d][1] - box[d][0] + 1 for d in (2, 1, 0))
        return box, Vb.reshape(shape), ph.reshape(shape)

    def forces(self, oid):
        kind, a, b = self.nobj_kind[oid]
        if kind == "rotor":
            nb, npt = a, b
            out = np.zeros(2 * nb + 3)
            pts = np.zeros(4 * nb * npt)
            self.lib.og_forces(self.h, int(oid), out.ctypes.data_as(_dp), pts.ctypes.data_as(_dp))
            return {"thrust": out[:nb].copy(), "torque": out[nb:2 * nb].copy(),
                    "power": out[2 * nb], "cp": out[2 * nb + 1], "ct": out[2 * nb + 2],
                    "Fx": pts[:nb * npt].reshape(nb, npt), "Ft": pts[nb * npt:2 * nb * npt].reshape(nb, npt),
                    "alpha": pts[2 * nb * npt:3 * nb * npt].reshape(nb, npt),
                    "phi": pts[3 * nb * npt:].reshape(nb, npt)}
        out = np.zeros(5)
        res = np.zeros(b)
        self.lib.og_forces(self.h, int(oid), out.ctypes.data_as(_dp), res.ctypes.data_as(_dp))
        return {"force": out[:3].copy(), "iters": int(out[3]), "residual": out[4],
                "residual_history": res[:int(out[3])].copy()}
