"""Parity at the full size of the benchmark workload (rotor with IBM tower and
nacelle, 384 x 256 x 256, CFL time step), in the launch configuration
bench.py times.

One step of the whole grid on the GPU is compared element by element with
the CPU oracle run on a window of the grid that holds every ALM and IBM
support plus a margin: a cell's update depends on cells at most 6 away (3
per stage), so cells at least 7 cells inside the window's cut faces see the
same inputs in both runs. The ground (slip wall) is a true boundary of both.
The oracle takes the GPU's time step (the CFL reduction over the full grid
is checked separately against numpy). Full-size invariants: a uniform
stream stays bitwise uniform."""
import numpy as np
import pytest

from paper_2603_11102_gb300 import workloads as WL

from _setup import oracle_from_workload

pytestmark = pytest.mark.gpu

FULL = (384, 256, 256)
WIN_LO = (78, 74, 0)          # window origin (cells): x, y, z (z starts at the ground)
WIN_N = (42, 108, 180)
MARGIN = 7
TOL = {"fp64": 1e-12, "fp32c": 1e-5, "fp64ds": 1e-12}


@pytest.fixture(scope="module")
def gks():
    from paper_2603_11102_gb300 import build, gks
    build.build()
    gks.load()
    return gks


@pytest.fixture(scope="module")
def workload():
    w = WL.alm_ibm_rotor(FULL)
    w.state0 = WL.perturbed(w, 0.02, seed=21)
    return w


def window(w, dt):
    lo, n = WIN_LO, WIN_N
    faces = [w.faces[a][lo[a]:lo[a] + n[a] + 1].copy() for a in range(3)]
    Q = w.state0[:, lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]].copy()
    # cut faces: any boundary kind (outflow); the ground keeps its slip wall
    bc = [(4, 4), (4, 4), (2, 4)]
    return WL.Workload("window", n, faces, w.mach, w.u_ref, w.mu, bc, cfl=w.cfl, dt_fixed=dt,
                       inflow=w.inflow, state0=Q, rotors=w.rotors, bodies=w.bodies)


@pytest.mark.parametrize("precision", ["fp32c", "fp64", "fp64ds"])
def test_full_size_step_matches_oracle_window(gks, workload, precision):
    """fp64ds: the FP64 grid with double-single reconstruction and flux."""
    w = workload
    g = gks.Grid.from_workload(w, precision="fp64" if precision == "fp64ds" else precision)
    if precision == "fp64ds":
        g.set_fp64_arithmetic("ds")
    g.step(1)
    dt = g.last_dt
    A = g.get_state()
    frot, ftow, fnac = g.forces(0), g.forces(1), g.forces(2)
    g.close()
    # the CFL step over the whole grid
    Q = w.state0
    umax = np.sqrt(np.max((Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0] ** 2))
    hmin = min(np.min(np.diff(f)) for f in w.faces)
    ref_dt = w.cfl * hmin / (umax + 1.0 / w.mach)
    assert abs(dt - ref_dt) <= (1e-6 if precision == "fp32c" else 1e-13) * ref_dt
    # the oracle on the window with the same time step
    o = oracle_from_workload(window(w, dt))
    o.step(1)
    B = o.get_state()
    lo, n, m = WIN_LO, WIN_N, MARGIN
    Ag = A[:, lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]]
    sl = (slice(None), slice(0, n[2] - m), slice(m, n[1] - m), slice(m, n[0] - m))
    err = np.max(np.abs(Ag[sl] - B[sl])) / np.max(np.abs(B[sl]))
    assert err <= TOL[precision], err
    # the forcing acted inside the compared region
    assert np.max(np.abs(Ag[sl][1] - w.state0[1, lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]][sl[1:]])) > 0
    tol = 2e-4 if precision == "fp32c" else 1e-11
    fo = o.forces(0)
    for k in ("thrust", "torque"):
        assert np.max(np.abs(frot[k] - fo[k])) <= tol * np.max(np.abs(fo[k])), (k, frot[k], fo[k])
    for oid, fg in ((1, ftow), (2, fnac)):
        fb = o.forces(oid)
        assert np.max(np.abs(fg["force"] - fb["force"])) <= tol * np.max(np.abs(fb["force"])), (fg, fb)


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_full_size_free_stream_is_bitwise_uniform(gks, precision):
    w = WL.alm_ibm_rotor(FULL)
    w.rotors, w.bodies = [], []
    g = gks.Grid.from_workload(w, precision=precision)
    Q0 = g.get_state()
    g.step(2)
    assert np.array_equal(g.get_state(), Q0)
    g.close()


# The other two grids the benchmark runs at full size, compared the same way:
# the turbulent channel on 128^3 (tanh-stretched y between no-slip walls,
# periodic x and z, driving body force) through the whole height, and the
# rotor without tower on 512 x 192 x 192 (inflow, outflow, periodic y, slip z;
# anisotropic cells) on a window that holds the actuator-line supports and
# every sampled point at least MARGIN cells inside its cut faces.
OTHER = {
    # name: (window origin x, y, z), window size, boundary kinds of the window
    "channel-128^3": ((40, 0, 50), (30, 128, 30), None),
    "alm-rotor-512x192x192": ((108, 56, 56), (40, 80, 80), [(4, 4), (4, 4), (4, 4)]),
}


def other_workload(name):
    if name == "channel-128^3":
        return WL.channel((128, 128, 128))
    w = WL.alm_rotor((512, 192, 192))
    w.state0 = WL.perturbed(w, 0.02, seed=23)
    return w


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("name", sorted(OTHER))
def test_other_full_size_grids_match_oracle_window(gks, name, precision):
    w = other_workload(name)
    lo, n, bcw = OTHER[name]
    if bcw is None:   # channel: the walls are true boundaries, x and z are cut
        bcw = [(4, 4), tuple(w.bc[1]), (4, 4)]
    g = gks.Grid.from_workload(w, precision=precision)
    g.step(1)
    dt = g.last_dt
    A = g.get_state()
    frot = g.forces(0) if w.rotors else None
    g.close()
    faces = [w.faces[a][lo[a]:lo[a] + n[a] + 1].copy() for a in range(3)]
    Q = w.state0[:, lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]].copy()
    win = WL.Workload("window", n, faces, w.mach, w.u_ref, w.mu, bcw, cfl=w.cfl, dt_fixed=dt, inflow=w.inflow,
                      body_force=w.body_force, state0=Q, rotors=w.rotors, bodies=w.bodies)
    o = oracle_from_workload(win)
    o.step(1)
    B = o.get_state()
    m = MARGIN
    # a window face inside the full grid is cut; compare only MARGIN cells in from it
    cut = [[lo[a] > 0, lo[a] + n[a] < w.n[a]] for a in range(3)]
    rng = [slice(m if cut[a][0] else 0, n[a] - m if cut[a][1] else n[a]) for a in range(3)]
    sl = (slice(None), rng[2], rng[1], rng[0])
    Ag = A[:, lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]]
    err = np.max(np.abs(Ag[sl] - B[sl])) / np.max(np.abs(B[sl]))
    assert err <= TOL[precision], err
    assert np.max(np.abs(Ag[sl][1:] - Q[sl][1:])) > 1e-6   # the state moved in the compared region
    if frot is not None:
        tol = 1e-11 if precision == "fp64" else 2e-4
        fo = o.forces(0)
        for k in ("thrust", "torque"):
            assert np.max(np.abs(frot[k] - fo[k])) <= tol * np.max(np.abs(fo[k])), (k, frot[k], fo[k])
