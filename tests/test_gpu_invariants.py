"""Properties of the CUDA path that hold at any size, independent of the
oracle: axis-permutation symmetry, fourth-order self-convergence, the
viscous decay rate of a 2D Taylor-Green vortex, and FP32C against FP64 load
histories.

Axis permutation: the scheme treats the three axes alike (the same WENO5,
equilibrium, tangential reconstruction and flux in the local frame of each
face), while the GPU runs each direction through a different kernel (x and y
faces: TMA face tiles with the flux stored per face; z faces: the flux fused
with the update). A problem and its cyclically permuted copy (x' = y,
y' = z, z' = x, momentum components permuted alike) must give the permuted
solution: FP64 to round-off, FP32C within the FP32 flux rounding. The sizes
are ragged (no axis a multiple of the 32 x 8 face tile) and every extent and
spacing differs, so a swapped stride, extent or cell width shows."""
import math

import numpy as np
import pytest

from paper_2603_11102_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-13, "fp32c": 2e-6}


@pytest.fixture(scope="module")
def gks():
    from paper_2603_11102_gb300 import build, gks
    build.build()
    gks.load()
    return gks


def smooth_periodic(n, L, seed):
    """rho, rho u, rho v, rho w from a few seeded Fourier modes per
    component (periodic on the box), amplitude 0.3 in velocity."""
    rng = np.random.default_rng(seed)
    xc = [(np.arange(n[a]) + 0.5) * L[a] / n[a] for a in range(3)]
    Z, Y, X = np.meshgrid(xc[2], xc[1], xc[0], indexing="ij")
    Q = np.zeros((4,) + tuple(n[::-1]))
    for c in range(4):
        for _ in range(3):
            k = rng.integers(1, 3, size=3)
            ph = rng.uniform(0, 2 * math.pi, size=3)
            amp = (0.02 if c == 0 else 0.3) * rng.uniform(0.3, 1.0)
            Q[c] += amp * (np.sin(2 * math.pi * k[0] * X / L[0] + ph[0]) * np.cos(2 * math.pi * k[1] * Y / L[1] + ph[1])
                           * np.cos(2 * math.pi * k[2] * Z / L[2] + ph[2]))
    Q[0] += 1.0
    Q[1:] *= Q[0]
    return Q


def permute(Q):
    """(x, y, z) -> (x', y', z') = (y, z, x): A'[x][z][y] = A[z][y][x]
    (arrays are z, y, x), momentum (u', v', w') = (v, w, u)."""
    T = np.transpose(Q, (0, 3, 1, 2))
    return T[[0, 2, 3, 1]].copy()


def unpermute(Qp):
    T = Qp[[0, 3, 1, 2]]
    return np.transpose(T, (0, 2, 3, 1)).copy()


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_cyclic_axis_permutation(gks, precision):
    n = (45, 38, 27)
    L = (2.0, 1.7, 1.3)
    faces = [WL.uniform_faces(0.0, L[a], n[a]) for a in range(3)]
    Q = smooth_periodic(n, L, seed=11)
    dt = 0.4 * min(L[a] / n[a] for a in range(3)) / (1.0 + 10.0)
    periodic = [(0, 0)] * 3
    w = WL.Workload("perm", n, faces, 0.1, 1.0, 2e-3, periodic, dt_fixed=dt, state0=Q)
    np_ = (n[1], n[2], n[0])
    wp = WL.Workload("perm'", np_, [faces[1], faces[2], faces[0]], 0.1, 1.0, 2e-3, periodic, dt_fixed=dt,
                     state0=permute(Q))
    steps = 4
    g = gks.Grid.from_workload(w, precision=precision)
    g.step(steps)
    A = g.get_state()
    g.close()
    gp = gks.Grid.from_workload(wp, precision=precision)
    gp.step(steps)
    B = unpermute(gp.get_state())
    gp.close()
    assert A.shape == B.shape
    # the solution moved: the comparison is not of two unchanged states
    assert np.max(np.abs(A - Q)) > 1e-3
    for c in range(4):
        scale = np.max(np.abs(A[c]))
        err = np.max(np.abs(A[c] - B[c]))
        assert err <= TOL[precision] * scale, (precision, c, err, scale)


def test_load_history_fp32c_against_fp64(gks):
    """The load history of a small rotor + tower + nacelle run (every 5
    steps): FP32C and FP64 give the same thrust, power, coefficients and body
    force to FP32-flux accuracy, and the same conserved totals."""
    from paper_2603_11102_gb300 import history
    w = WL.alm_ibm_rotor(n=(64, 32, 32), n_pts=10)
    w.state0 = WL.perturbed(w, 0.02, seed=5)
    r32, _ = history.record(w, "fp32c", 20, 5)
    r64, _ = history.record(w, "fp64", 20, 5)
    a32, a64 = np.array(r32), np.array(r64)
    assert a32.shape == (4, len(history.FIELDS)) and np.array_equal(a32[:, 0], [5, 10, 15, 20])
    for name in ("thrust", "torque", "power", "cp", "ct", "body_fx", "mass", "ke"):
        i = history.FIELDS.index(name)
        scale = np.max(np.abs(a64[:, i]))
        assert scale > 0 and np.max(np.abs(a32[:, i] - a64[:, i])) <= 1e-5 * scale, name


def _periodic_2d(n, mu, state, dt_fixed=0.0, cfl=0.5):
    L = 2 * math.pi
    h = L / n
    faces = [np.linspace(0, L, n + 1), np.linspace(0, L, n + 1), np.array([0.0, h])]
    return WL.Workload("periodic-2d", (n, n, 1), faces, 0.1, 1.0, mu, [(0, 0)] * 3, cfl=cfl,
                       dt_fixed=dt_fixed, state0=state)


def test_smooth_field_converges_at_fourth_order_on_the_gpu(gks):
    """The CUDA FP64 path on its own: self-convergence (against 256^2,
    restricted by cell averaging) of a smooth periodic small-amplitude
    acoustic and shear wave at fixed CFL in the inviscid limit, observed
    order >= 3.5 (WENO5 in space, the two-stage fourth-order method in
    time; the CPU oracle passes the same test)."""
    T = 0.1

    def run(n):
        h = 2 * math.pi / n
        x0 = np.arange(n) * h
        x1 = x0 + h
        a0, a1 = x0[None, :], x1[None, :]
        b0, b1 = x0[:, None], x1[:, None]
        s = (-np.sin(a1 + b1) + np.sin(a1 + b0) + np.sin(a0 + b1) - np.sin(a0 + b0)) / h ** 2
        Q = np.zeros((4, 1, n, n))
        Q[0, 0] = 1 - 1e-3 * s
        Q[1, 0] = 0.1 + 5e-3 * ((np.cos(x0) - np.cos(x1)) / h)[:, None]
        Q[2, 0] = 5e-3 * ((np.sin(x1) - np.sin(x0)) / h)[None, :]
        g = gks.Grid.from_workload(_periodic_2d(n, 0.0, Q, dt_fixed=T / (n // 4), cfl=0.9), precision="fp64")
        g.step(n // 4)
        out = g.get_state()[:, 0]
        g.close()
        return out

    sol = {n: run(n) for n in (16, 32, 64, 256)}

    def restrict(q, f):
        m = q.shape[-1] // f
        return q.reshape(4, m, f, m, f).mean(axis=(2, 4))

    errs = [np.max(np.abs(sol[n] - restrict(sol[256], 256 // n))) for n in (16, 32, 64)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 3.5, (errs, orders)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_taylor_green_2d_viscous_decay_rate_on_the_gpu(gks, precision):
    """Low-Mach 2D Taylor-Green vortex (Ma 0.1, Re 100, 48^2 periodic, CFL
    0.5) on the CUDA path: kinetic energy decays as exp(-4 nu t); the fitted
    rate over t in [0, 2] is within 1 % of 4 nu."""
    n, nu = 48, 0.01
    xc = (np.arange(n) + 0.5) * 2 * math.pi / n
    y, x = np.meshgrid(xc, xc, indexing="ij")
    Q = np.zeros((4, 1, n, n))
    Q[0, 0] = 1.0
    Q[1, 0] = np.sin(x) * np.cos(y)
    Q[2, 0] = -np.cos(x) * np.sin(y)
    g = gks.Grid.from_workload(_periodic_2d(n, nu, Q), precision=precision)
    ts, ke = [0.0], [g.diagnostics()[4]]
    while ts[-1] < 2.0:
        ts.append(g.step(1))
        ke.append(g.diagnostics()[4])
    g.close()
    rate = -np.polyfit(np.array(ts), np.log(np.array(ke)), 1)[0]
    assert abs(rate / (4 * nu) - 1) < 0.01, rate


def test_alu_peak_probe_counts_its_operations(gks):
    """gks_alu_peak_probe: the operations it reports are 2 per FMA of its
    launch (4 blocks of 256 threads per SM, 128 FMAs per iteration), its
    rate scales with the work (twice the iterations, about twice the time),
    and the FP32 rate lies within the GPU's nominal bounds (FP64 well below
    it on GB300)."""
    import torch
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(4 * sms, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)

    def timed(fp64, iters):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        fl = gks.alu_peak_probe(fp64, iters, sink, st)
        b.record(st)
        b.synchronize()
        return fl, a.elapsed_time(b) / 1e3

    gks.alu_peak_probe(False, 1000, sink, st)   # warm-up
    fl1, t1 = timed(False, 20000)
    fl2, t2 = timed(False, 40000)
    assert fl1 == 2.0 * 4 * sms * 256 * 20000 * 128 and fl2 == 2 * fl1
    assert 1.6 <= t2 / t1 <= 2.4, (t1, t2)
    rate32 = fl2 / t2 / 1e12
    nominal = sms * 128 * 2 * 2.2e9 / 1e12          # FP32 lanes x 2 x a clock above any GB300 boost
    assert 0.3 * nominal <= rate32 <= 1.05 * nominal, (rate32, nominal)
    fl64, t64 = timed(True, 2000)
    assert fl64 / t64 / 1e12 < 0.5 * rate32
    # packed FP32 pairs: the same operations per launch, half the
    # instructions; the FMA pipes stay the bound (no more than the nominal
    # FP32 rate)
    fl2x, t2x = timed(2, 40000)
    assert fl2x == fl2
    assert 0.3 * nominal <= fl2x / t2x / 1e12 <= 1.05 * nominal, (fl2x / t2x / 1e12, nominal)
    assert not torch.any(sink != 0)   # the loop's results stay in registers
