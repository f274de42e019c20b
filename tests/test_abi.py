"""The C-ABI library builds, loads and exports every entry point that
include/gks_api.h declares; the ctypes structures of the binding have the
header's layout; host-side validation and workspace sizing work without a
GPU (no compute call is made here)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gks_api.h")


@pytest.fixture(scope="module")
def gks():
    from paper_2603_11102_gb300 import build, gks
    build.build()
    gks.load()
    return gks


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(gks_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for must in ("gks_create_grid", "gks_set_inflow", "gks_add_actuator_lines", "gks_add_ib_points",
                 "gks_step", "gks_forces"):
        assert must in names


def test_library_exports_every_declared_symbol(gks):
    names = declared_functions()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", gks.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(names) == set(gks.SIGNATURES), set(names) ^ set(gks.SIGNATURES)


def test_struct_layouts_match_header(gks):
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "gks_api.h"
#define P(s, f) printf(#s "." #f " %zu\n", offsetof(s, f))
int main(void) {
  printf("gks_grid_desc %zu\n", sizeof(gks_grid_desc));
  P(gks_grid_desc, faces); P(gks_grid_desc, mach); P(gks_grid_desc, bc); P(gks_grid_desc, precision);
  P(gks_grid_desc, cfl); P(gks_grid_desc, rho_ref); P(gks_grid_desc, stream);
  printf("gks_rotor_desc %zu\n", sizeof(gks_rotor_desc));
  P(gks_rotor_desc, hub); P(gks_rotor_desc, omega); P(gks_rotor_desc, r); P(gks_rotor_desc, width);
  P(gks_rotor_desc, correction);
  printf("gks_forces_out %zu\n", sizeof(gks_forces_out));
  P(gks_forces_out, thrust); P(gks_forces_out, power); P(gks_forces_out, body_force);
  P(gks_forces_out, iters); P(gks_forces_out, residual);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "p.c"), os.path.join(d, "p")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, src], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    ref = dict(l.split() for l in lines if l.strip())
    S = {"gks_grid_desc": gks.GridDesc, "gks_rotor_desc": gks.RotorDesc, "gks_forces_out": gks.ForcesOut}
    for key, val in ref.items():
        if "." in key:
            s, f = key.split(".")
            assert getattr(S[s], f).offset == int(val), key
        else:
            assert C.sizeof(S[key]) == int(val), key


def make_desc(gks, n=(8, 6, 5), precision=0, bc=((0, 0), (0, 0), (0, 0)), faces=None, cfl=0.5):
    faces = faces or [np.linspace(0.0, 1.0, k + 1) for k in n]
    keep = [np.ascontiguousarray(f, dtype=np.float64) for f in faces]
    d = gks.GridDesc()
    for a in range(3):
        d.n[a] = n[a]
        d.faces[a] = keep[a].ctypes.data_as(C.POINTER(C.c_double))
        d.bc[a][0], d.bc[a][1] = bc[a]
    d.mach, d.u_ref, d.mu = 0.1, 1.0, 1e-3
    d.precision, d.cfl, d.dt_fixed, d.rho_ref = precision, cfl, 0.0, 1.0
    return d, keep


def test_workspace_sizes_and_validation(gks):
    lib = gks.lib
    sb, wb = C.c_size_t(), C.c_size_t()
    for prec in (0, 1):
        d, keep = make_desc(gks, precision=prec)
        assert lib.gks_workspace_bytes(C.byref(d), C.byref(sb), C.byref(wb)) == 0
        P = (8 + 6) * (6 + 6) * (5 + 6)
        per = 4 * 8 if prec == 0 else 8 * 4
        assert sb.value >= P * per and sb.value % 8 == 0
        assert wb.value > sb.value
    # invalid descriptions are rejected with GKS_ERR_ARG and a message
    bad = [dict(n=(2, 6, 5), bc=((1, 1), (0, 0), (0, 0))),   # too few cells for a wall
           dict(bc=((0, 1), (0, 0), (0, 0))),                # periodic on one end only
           dict(faces=[np.linspace(1, 0, 9), np.linspace(0, 1, 7), np.linspace(0, 1, 6)]),
           dict(precision=7), dict(cfl=0.0),
           dict(bc=((0, 0), (5, 5), (0, 0))),                # exchange sides are x sides only
           dict(bc=((0, 0), (0, 0), (2, 5))),
           dict(bc=((0, 5), (0, 0), (0, 0))),                # periodic on one end only
           dict(bc=((4, 6), (0, 0), (0, 0))),                # no such kind
           dict(n=(0, 6, 5), faces=[np.zeros(1), np.linspace(0, 1, 7), np.linspace(0, 1, 6)]),   # empty axis
           # more cells than the 32-bit face-tile indices of the flux kernels cover
           dict(n=(2000, 1100, 1000), faces=[np.linspace(0, 1, 2001), np.linspace(0, 1, 1101),
                                              np.linspace(0, 1, 1001)])]
    for kw in bad:
        d, keep = make_desc(gks, **kw)
        assert lib.gks_workspace_bytes(C.byref(d), C.byref(sb), C.byref(wb)) == -1, kw
        assert lib.gks_last_error(None)
    # an x-slab of a slab group: exchange sides on x
    d, keep = make_desc(gks, bc=((5, 5), (0, 0), (0, 0)))
    assert lib.gks_workspace_bytes(C.byref(d), C.byref(sb), C.byref(wb)) == 0
    d, keep = make_desc(gks, bc=((3, 5), (2, 2), (1, 1)))
    assert lib.gks_workspace_bytes(C.byref(d), C.byref(sb), C.byref(wb)) == 0
    # null handles
    assert lib.gks_slab_step(None, 1, 1, None) == -1
    assert lib.gks_step(None, 1, None) == -1
    assert lib.gks_step_async(None, 1) == -1
    assert lib.gks_sync(None, None) == -1
    assert lib.gks_step_record(None, None, None) == -1
    assert lib.gks_step_reverse(None, None, None, None, None, 0.0, None, None) == -1
    assert lib.gks_forces_async(None, 0, None, 0) == -1
    assert lib.gks_destroy_grid(None) == -1
