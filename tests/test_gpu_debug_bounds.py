"""The debug-bounds build (compiled with GKS_DEBUG_BOUNDS; loaded with the
environment variable GKS_DEBUG_BOUNDS=1): every kernel checks its
data-dependent indices against its buffer and a failed check skips the
access and makes the call return GKS_ERR_DEBUG_BOUNDS. Representative steps
(Taylor-Green, rotor with tower and nacelle, FP64 and FP32C, ragged sizes)
and a recorded step with its reverse run through it without a failed check
and give what the plain build gives. Each build runs in a child process (a
process loads one library)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys
import numpy as np
sys.path.insert(0, {root!r})
sys.path.insert(0, os.path.join({root!r}, "tests"))
import torch
from paper_2603_11102_gb300 import build, gks, workloads as WL
build.build(debug=os.environ.get("GKS_DEBUG_BOUNDS") == "1")
gks.load()
import test_gpu_adjoint as TA
out = {{}}
for prec in ("fp64", "fp32c"):
    w = WL.taylor_green_3d(24)
    g = gks.Grid.from_workload(w, precision=prec)
    g.step(3)
    out["tgv_" + prec] = g.get_state()
    g.close()
    w = WL.alm_ibm_rotor(n=(70, 36, 34), steps=1, n_pts=10)
    w.state0 = WL.perturbed(w, 0.02, seed=6)
    g = gks.Grid.from_workload(w, precision=prec)
    g.step(2)
    out["rotor_" + prec] = g.get_state()
    out["power_" + prec] = np.array([g.forces(0)["power"]])
    g.close()
w = TA.rotor_body_workload()
g = gks.Grid.from_workload(w, precision="fp64")
g.set_adjoint_precision("fp32")
W = torch.tensor(TA.perturbed_state(w, 4), dtype=torch.float64, device="cuda")
lam1 = torch.tensor(np.random.default_rng(2).standard_normal(W.shape), dtype=torch.float64, device="cuda")
g.set_state_tensor(W)
g.set_time(0.3)
tape = g.adjoint_tape()
g.step_record(tape)
gs = np.zeros(18)
lam0, gu = g.step_reverse(tape, g.adjoint_scratch(), lam1, 0.5, gs)
out["lam0"] = lam0.cpu().numpy()
out["gs"] = gs
out["gu"] = np.array([gu])
g.close()
np.savez({path!r}, **out)
"""


def run_child(tmp_path, debug):
    path = str(tmp_path / ("debug.npz" if debug else "plain.npz"))
    env = dict(os.environ)
    env["GKS_DEBUG_BOUNDS"] = "1" if debug else "0"
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, path=path)], env=env, capture_output=True,
                       text=True, timeout=1500)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(path))


def test_debug_bounds_build_runs_clean_and_matches_the_plain_build(tmp_path):
    plain = run_child(tmp_path, False)
    debug = run_child(tmp_path, True)
    assert set(plain) == set(debug)
    for k in plain:
        a, b = plain[k], debug[k]
        scale = max(float(np.max(np.abs(a))), 1e-300)
        assert np.max(np.abs(a - b)) <= 1e-12 * scale, k
