"""Run a rotor workload and record its load history.

For the rotor workloads (actuator lines, optionally with immersed tower and
nacelle) the quantities a run reports every few steps are the rotor's
thrust, torque, power and their coefficients, the force on each immersed
body and the conserved totals. This module steps a grid through the public
binding and collects them, so that an FP32-compensated run can be held
against an FP64 run of the same workload:

    python -m paper_2603_11102_gb300.history --workload alm-ibm-rotor \\
        --precision fp32c --steps 2000 --every 10 --out history.csv
"""
from __future__ import annotations

import argparse
import csv
import time

import numpy as np

from . import gks
from . import workloads as WL

FIELDS = ["step", "t", "thrust", "torque", "power", "cp", "ct", "body_fx", "body_fy", "body_fz",
          "mass", "mom_x", "mom_y", "mom_z", "ke"]


def make(name):
    if name == "alm-ibm-rotor":
        return WL.alm_ibm_rotor()
    if name == "alm-rotor":
        return WL.alm_rotor()
    raise ValueError("unknown workload %r" % name)


def record(w, precision, steps, every, device="cuda:0"):
    """Step `w` `steps` times; every `every` steps (and after the last) a row
    of FIELDS. Returns (rows, seconds of stepping)."""
    g = gks.Grid.from_workload(w, precision=precision, device=device)
    rotor = next(i for i, o in enumerate(g.objects) if o[0] == "rotor")
    bodies = [i for i, o in enumerate(g.objects) if o[0] == "body"]
    rows, secs, done = [], 0.0, 0
    while done < steps:
        k = min(every, steps - done)
        t0 = time.perf_counter()
        t = g.step(k)
        secs += time.perf_counter() - t0
        done += k
        f = g.forces(rotor)
        bf = np.zeros(3)
        for b in bodies:
            bf += g.forces(b)["force"]
        d = g.diagnostics()
        rows.append([done, t, float(np.sum(f["thrust"])), float(np.sum(f["torque"])), f["power"], f["cp"],
                     f["ct"], *bf.tolist(), *d.tolist()])
    g.close()
    return rows, secs


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="alm-ibm-rotor", choices=["alm-ibm-rotor", "alm-rotor"])
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--out", default="history.csv")
    args = ap.parse_args(argv)
    from . import build
    build.build()
    gks.load()
    w = make(args.workload)
    rows, secs = record(w, args.precision, args.steps, args.every)
    with open(args.out, "w", newline="") as fh:
        wr = csv.writer(fh)
        wr.writerow(FIELDS)
        wr.writerows(rows)
    print("%s %s: %d steps in %.2f s (%.1f MLUPS incl. the load reads), last cp %.6f ct %.6f"
          % (args.workload, args.precision, args.steps, secs, w.cells * args.steps / secs / 1e6, rows[-1][5],
             rows[-1][6]))


if __name__ == "__main__":
    main()
