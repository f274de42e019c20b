"""Pin of the oracle's derivative scales on a stretched axis (reading R10).

The channel of Sec. 4.1 stretches the wall-normal axis with a tanh map. The
oracle reconstructs in index space and scales the normal slope at a face by
the distance of the two cell centres beside it, and a tangential slope by the
width of the cell it is taken in. Free-stream and conservation tests are blind
to those scales, so this pin measures them directly:

* The smooth flux of Eq. (flux) is affine in mu (tau = mu/p multiplies the only
  mu-dependent term and the reconstruction does not depend on mu), so
  (L(mu) - L(0)) / mu is the discrete viscous operator exactly.
* Its continuum limit for rho = 1 is div(grad U + grad U^T), i.e.
  lap U_k + d_k(div U) (isothermal BGK: stress mu (dU_i/dx_j + dU_j/dx_i), no
  bulk term), whose cell averages over a separable trigonometric field are
  closed forms.
* With the reading's scales the metric error of a smooth map is second order,
  so the operator converges at order 2 on the tanh axis; a cell width in place
  of the centre distance (or the neighbour's width, or the centre distance, for
  a tangential slope) leaves a first-order error, and no scale at all does not
  converge. ``test_planted_metric_mistakes_fail_the_pin`` compiles copies of
  the oracle with each of these mistakes and checks that the pin rejects them.
"""
import math
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_2603_11102_gb300 import workloads as WL

HERE = os.path.dirname(os.path.abspath(__file__))

# Velocity field: sums of separable terms coef * f_x(x) f_y(y) f_z(z), each
# factor ("s"|"c", alpha, beta) = sin|cos(alpha s + beta), or None for 1.
A, B = 1.3, 0.2      # U = sin x cos(A y + B)
C_, E = 0.9, 0.4     # V = cos x sin(C y + E) + cos z sin(K y)
K = 1.1
M, Qp = 0.7, 0.3     # W = sin z cos(M y + Qp)
S = lambda a=1.0, b=0.0: ("s", a, b)   # noqa: E731
Cc = lambda a=1.0, b=0.0: ("c", a, b)  # noqa: E731

VELOCITY = [
    [(1.0, S(), Cc(A, B), None)],
    [(1.0, Cc(), S(C_, E), None), (1.0, None, S(K), Cc())],
    [(1.0, None, Cc(M, Qp), S())],
]
# lap U_k + d_k(div U), derived by hand from the field above
VISCOUS = [
    [(-(2 + A * A), S(), Cc(A, B), None), (-C_, S(), Cc(C_, E), None)],
    [(-(1 + 2 * C_ * C_), Cc(), S(C_, E), None), (-(1 + 2 * K * K), None, S(K), Cc()),
     (-A, Cc(), S(A, B), None), (-M, None, S(M, Qp), Cc())],
    [(-(2 + M * M), None, Cc(M, Qp), S()), (-K, None, Cc(K), S())],
]


def _avg1(fac, faces):
    """Exact average of one factor over each cell [faces[i], faces[i+1]]."""
    if fac is None:
        return np.ones(len(faces) - 1)
    kind, a, b = fac
    lo, hi = faces[:-1], faces[1:]
    if kind == "s":
        return (np.cos(a * lo + b) - np.cos(a * hi + b)) / (a * (hi - lo))
    return (np.sin(a * hi + b) - np.sin(a * lo + b)) / (a * (hi - lo))


def cell_average(terms, faces):
    out = 0.0
    for coef, fx, fy, fz in terms:
        ax, ay, az = _avg1(fx, faces[0]), _avg1(fy, faces[1]), _avg1(fz, faces[2])
        out = out + coef * az[:, None, None] * ay[None, :, None] * ax[None, None, :]
    return out


def viscous_operator_errors(N, mu=0.05, amp=0.01):
    """Max |discrete - exact| viscous operator per momentum component over the
    cells with |y| <= 0.7 (their stencils stay off the y ghosts) on an
    (N/2, N, N/2) grid, x and z uniform periodic over 2 pi, y on the tanh map
    of Sec. 4.1 (b_g = 2)."""
    faces = [np.linspace(0.0, 2 * math.pi, N // 2 + 1), WL.tanh_faces(N),
             np.linspace(0.0, 2 * math.pi, N // 2 + 1)]
    n = (N // 2, N, N // 2)
    Q = np.zeros((4, n[2], n[1], n[0]))
    Q[0] = 1.0
    for k in range(3):
        Q[1 + k] = amp * cell_average(VELOCITY[k], faces)
    bc = [("periodic", "periodic"), ("outflow", "outflow"), ("periodic", "periodic")]
    L = []
    for m in (0.0, mu):
        g = O.OracleGrid(n, faces, 0.1, 1.0, m, bc)
        L.append(g.rhs(Q)[0])
    D = (L[1] - L[0]) / (mu * amp)
    yc = 0.5 * (faces[1][1:] + faces[1][:-1])
    sel = np.abs(yc) <= 0.7
    return [float(np.max(np.abs(D[1 + k][:, sel, :] - cell_average(VISCOUS[k], faces)[:, sel, :])))
            for k in range(3)]


def observed_orders():
    e32, e64 = viscous_operator_errors(32), viscous_operator_errors(64)
    return e64, [math.log2(a / b) for a, b in zip(e32, e64)]


def test_closed_form_viscous_operator_matches_the_field():
    """The hand-derived operator equals central differences of the field's own
    derivatives (guards the closed forms the pin compares against)."""
    rng = np.random.default_rng(1)
    h = 1e-4

    def val(terms, p):
        s = 0.0
        for coef, *facs in terms:
            t = coef
            for fac, xx in zip(facs, p):
                if fac is not None:
                    kind, a, b = fac
                    t *= math.sin(a * xx + b) if kind == "s" else math.cos(a * xx + b)
            s += t
        return s

    def d(terms, p, i, j=None):
        e = np.eye(3) * h
        if j is None:
            return (val(terms, p + e[i]) - val(terms, p - e[i])) / (2 * h)
        return (val(terms, p + e[i] + e[j]) - val(terms, p + e[i] - e[j]) - val(terms, p - e[i] + e[j])
                + val(terms, p - e[i] - e[j])) / (4 * h * h)

    for _ in range(5):
        p = rng.uniform(-2, 2, 3)
        for k in range(3):
            lap = sum((val(VELOCITY[k], p + np.eye(3)[n] * h) - 2 * val(VELOCITY[k], p)
                       + val(VELOCITY[k], p - np.eye(3)[n] * h)) / (h * h) for n in range(3))
            grad_div = sum(d(VELOCITY[n], p, n, k) if n != k else
                           (val(VELOCITY[k], p + np.eye(3)[k] * h) - 2 * val(VELOCITY[k], p)
                            + val(VELOCITY[k], p - np.eye(3)[k] * h)) / (h * h) for n in range(3))
            assert abs(lap + grad_div - val(VISCOUS[k], p)) < 1e-5


def test_viscous_operator_converges_at_second_order_on_the_tanh_axis():
    """R10 scales: order >= 1.8 per momentum component between 32 and 64 cells
    across the channel (measured 2.0-2.4), error <= 1e-2 at 64."""
    e64, orders = observed_orders()
    assert min(orders) >= 1.8, (e64, orders)
    assert max(e64) <= 1e-2, (e64, orders)


# Each planted mistake: (name, exact text in the oracle, replacement)
_NORMAL = "double hfc = 0.5 * (g->h[d][G + f - 1] + g->h[d][G + f]);"
_TANG = "double ih1 = 1.0 / g->h[t1][G + a], ih2 = 1.0 / g->h[t2][G + b];"
MUTANTS = [
    ("normal slope over the cell width", _NORMAL, "double hfc = g->h[d][G + f];"),
    ("normal slope unscaled", _NORMAL, "double hfc = 1.0;"),
    ("t1 slope over the next cell's width", _TANG,
     "double ih1 = 1.0 / g->h[t1][G + a + 1], ih2 = 1.0 / g->h[t2][G + b];"),
    ("t2 slope over the next cell's width", _TANG,
     "double ih1 = 1.0 / g->h[t1][G + a], ih2 = 1.0 / g->h[t2][G + b + 1];"),
    ("t1 slope over the centre distance", _TANG,
     "double ih1 = 2.0 / (g->h[t1][G + a] + g->h[t1][G + a + 1]), ih2 = 1.0 / g->h[t2][G + b];"),
]


@pytest.mark.slow
def test_planted_metric_mistakes_fail_the_pin():
    src_path = os.path.join(os.path.dirname(O.__file__), "gks_oracle.c")
    hdr_path = os.path.join(os.path.dirname(O.__file__), "gks_oracle.h")
    src = open(src_path).read()
    hdr = open(hdr_path).read()
    with tempfile.TemporaryDirectory() as tmp:
        for i, (name, old, new) in enumerate(MUTANTS):
            assert src.count(old) == 1, "the pin's planted mistake no longer matches the oracle: " + name
            d = os.path.join(tmp, "m%d" % i)
            os.makedirs(d)
            with open(os.path.join(d, "gks_oracle.c"), "w") as fh:
                fh.write(src.replace(old, new))
            with open(os.path.join(d, "gks_oracle.h"), "w") as fh:
                fh.write(hdr)
            code = (
                "import sys, os\n"
                "sys.path[:0] = [%r, %r]\n"
                "import oracle as O\n"
                "O._SRC = os.path.join(%r, 'gks_oracle.c'); O._HDR = os.path.join(%r, 'gks_oracle.h')\n"
                "O._OUT_DIR = %r; O._LIB = os.path.join(%r, 'lib.so')\n"
                "import test_oracle_stretched as T\n"
                "e, o = T.observed_orders()\n"
                "print(min(o) >= 1.8 and max(e) <= 1e-2)\n"
            ) % (os.path.dirname(HERE), HERE, d, d, d, d)
            out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
            assert out.returncode == 0, out.stderr
            assert out.stdout.strip().splitlines()[-1] == "False", "pin passed a planted mistake: " + name
