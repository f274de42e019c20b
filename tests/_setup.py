"""Test helpers: build the oracle twin of a workload, compare states."""
import numpy as np

import oracle
from paper_2603_11102_gb300 import workloads as WL


def oracle_from_workload(w, state=None):
    o = oracle.OracleGrid(w.n, w.faces, w.mach, w.u_ref, w.mu, w.bc, cfl=w.cfl, dt_fixed=w.dt_fixed)
    o.set_inflow(*w.inflow)
    o.set_body_force(*w.body_force)
    for r in w.rotors:
        o.add_rotor(r.n_blades, r.r, r.chord, r.twist, r.width, r.hub, r.omega, r.azimuth0, r.radius,
                    r.eps, r.rho_inf, r.u_inf_ref, r.correction, r.tip_correction)
    for b in w.bodies:
        o.add_body(b.xyz, b.dS, b.eps, vel=b.vel, niter=b.niter, tol=b.tol)
    o.set_state(w.state0 if state is None else state)
    return o


def rel_linf(a, b):
    """max |a - b| / max |b| over the whole conserved state."""
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def rel_linf_components(a, b):
    return [float(np.max(np.abs(a[v] - b[v])) / max(np.max(np.abs(b[v])), 1e-300)) for v in range(4)]


def smooth_workload(n, bc, faces=None, mu=2e-3, seed=0, amp=0.05, cfl=0.5, dt_fixed=0.0):
    """A smooth, non-trivial state on an arbitrary grid (seeded)."""
    rng = np.random.default_rng(seed)
    if faces is None:
        faces = [np.linspace(0.0, 2 * np.pi * (1 + 0.1 * d), n[d] + 1) for d in range(3)]
    xc = [0.5 * (f[1:] + f[:-1]) for f in faces]
    Z, Y, X = np.meshgrid(xc[2], xc[1], xc[0], indexing="ij")
    a = rng.random(8)
    Q = np.zeros((4, n[2], n[1], n[0]))
    Q[0] = 1.0 + 0.01 * np.sin(X + a[0]) * np.cos(Y + a[1]) + 0.005 * np.cos(Z + a[2])
    Q[1] = Q[0] * (0.3 + 0.2 * np.sin(Y + a[3]) * np.cos(Z + a[4]))
    Q[2] = Q[0] * (0.1 * np.cos(X + a[5]) * np.sin(Z))
    Q[3] = Q[0] * (0.05 + 0.1 * np.sin(X) * np.cos(Y + a[6]))
    Q[1:] += amp * 0.1 * (2 * rng.random(Q[1:].shape) - 1)
    return WL.Workload("smooth-%dx%dx%d" % tuple(n), tuple(n), faces, 0.1, 1.0, mu, [tuple(x) for x in bc],
                       cfl=cfl, dt_fixed=dt_fixed, state0=Q)


def paper_values():
    """Values the paper prints (tests/golden/paper_values.txt): name -> list of floats."""
    import os
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].split()
            if line:
                out[line[0]] = [float(v) for v in line[1:]]
    return out



def report(case, precision, steps, a=None, b=None, **extra):
    """Record a parity case's measured errors (one JSON line per call) in the
    file named by GKS_PARITY_REPORT, when that variable is set: the whole-state
    relative L-infinity, the same per component, and any extra figures."""
    import json
    import os
    path = os.environ.get("GKS_PARITY_REPORT")
    if not path:
        return
    rec = {"case": case, "precision": precision, "steps": int(steps)}
    if a is not None:
        rec.update(rel_linf=rel_linf(a, b), components=rel_linf_components(a, b))
    rec.update({k: (float(v) if np.isscalar(v) else [float(x) for x in np.ravel(v)]) for k, v in extra.items()})
    with open(path, "a") as fh:
        fh.write(json.dumps(rec) + "\n")
