"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper it checks. The expected values come
from independent routes: Gauss-Hermite or adaptive quadrature, polynomial
exactness, a hand derivation of the Chapman-Enskog form of the flux, textbook
reductions (Taylor polynomial of the scalar ODE), and invariants of the
method (free stream, conservation, symmetry).
"""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite as H
from numpy.polynomial import polynomial as P

import oracle as O

from _setup import paper_values

LAM = 0.005          # Ma = 0.1, U_ref = 1
THETA = 1.0 / (2 * LAM)


# ---------------------------------------------------------------- moments ---

def gh_moment(k, U, lam, npts=60):
    """<u^k> of the normalised 1D Maxwellian by Gauss-Hermite quadrature."""
    x, w = H.hermgauss(npts)
    u = U + x / math.sqrt(lam)
    return float(np.sum(w * u ** k) / math.sqrt(math.pi))


@pytest.mark.parametrize("U", [-0.37, 0.0, 1.2, 9.5])
@pytest.mark.parametrize("lam", [0.005, 0.5])
def test_moment_recursion_matches_gauss_hermite(U, lam):
    """Appendix: <u^{n+2}> = (n+1)/(2 lambda) <u^n> + U <u^{n+1}>."""
    M = O.moments(U, lam, 7)
    for k in range(8):
        ref = gh_moment(k, U, lam)
        scale = (abs(U) + 1.0 / math.sqrt(lam)) ** k   # size of the quadrature terms
        assert abs(M[k] - ref) <= 1e-13 * max(1.0, scale), (k, M[k], ref)


@pytest.mark.parametrize("U", [-0.8, -0.05, 0.0, 0.3, 2.0])
def test_half_space_moments_match_quadrature(U):
    """Half-space moments used to form the equilibrium state at a face."""
    from scipy.integrate import quad
    lam = LAM
    g = lambda u: math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
    for sign in (+1, -1):
        h = O.half_moments(U, lam, sign)
        lo, hi = (0.0, np.inf) if sign > 0 else (-np.inf, 0.0)
        for k in range(2):
            ref = quad(lambda u: u ** k * g(u), lo, hi, epsabs=1e-14, epsrel=1e-13)[0]
            assert abs(h[k] - ref) <= 1e-11 * max(1.0, abs(ref)), (sign, k, h[k], ref)
    hp, hn = O.half_moments(U, lam, +1), O.half_moments(U, lam, -1)
    assert abs(hp[0] + hn[0] - 1.0) <= 1e-15
    assert abs(hp[1] + hn[1] - U) <= 1e-14 * max(1, abs(U))


def maxwellian_matrix(U, V, W, lam, npts=20):
    """M = <psi psi^T>, psi = (1, u, v, w), by tensor Gauss-Hermite quadrature."""
    x, w = H.hermgauss(npts)
    s = 1.0 / math.sqrt(lam)
    M = np.zeros((4, 4))
    for i, (xi, wi) in enumerate(zip(x, w)):
        for j, (xj, wj) in enumerate(zip(x, w)):
            for k, (xk, wk) in enumerate(zip(x, w)):
                psi = np.array([1.0, U + s * xi, V + s * xj, W + s * xk])
                M += wi * wj * wk * np.outer(psi, psi)
    return M / math.pi ** 1.5


def test_coefficient_solve_satisfies_moment_system():
    """Appendix: the closed-form solution solves M a = d."""
    rng = np.random.default_rng(1)
    for _ in range(4):
        U, V, W = rng.normal(size=3)
        M = maxwellian_matrix(U, V, W, LAM)
        d = rng.normal(size=4)
        a = O.coeff_solve(U, V, W, LAM, d)
        r = M @ a - d
        assert np.max(np.abs(r)) <= 1e-12 * np.max(np.abs(M)) * max(1, np.max(np.abs(a)))


# ------------------------------------------------------------------- flux ---

def chapman_enskog_flux(lam, mu, Q, Dn, Dt1, Dt2):
    """Hand derivation (independent of the moment algebra): with the Maxwellian
    centred at U and theta = 1/(2 lambda), the solution of the coefficient
    systems gives a.u + A = (1/theta) dU_j/dx_i (c_i c_j - theta delta_ij),
    c = u - U, and A = A0 + A_j c_j with A0 = -U.grad(ln rho) - div U,
    A_k = -d_k ln rho - (1/theta) U_i d_i U_k. Taking moments:
      F0 = (m_n, m_n U_k + p delta_nk - mu (d_n U_k + d_k U_n)),
      F1 = rho (A0 U_n + theta A_n,  A0 (U_n U_k + theta delta_nk) + theta (A_k U_n + A_n U_k))."""
    th = 1.0 / (2 * lam)
    rho = Q[0]
    U = np.array(Q[1:]) / rho
    D = np.array([Dn, Dt1, Dt2], dtype=float)          # D[i] = d/dx_i of (rho, m)
    grho = D[:, 0]
    G = (D[:, 1:] - np.outer(grho, U)) / rho             # G[i, j] = d_i U_j
    glr = grho / rho
    A0 = -U @ glr - np.trace(G)
    Ak = -glr - (U @ G) / th
    F0 = np.zeros(4)
    F1 = np.zeros(4)
    F0[0] = Q[1]
    F1[0] = rho * (A0 * U[0] + th * Ak[0])
    for k in range(3):
        dnk = 1.0 if k == 0 else 0.0
        F0[1 + k] = Q[1] * U[k] + rho * th * dnk - mu * (G[0, k] + G[k, 0])
        F1[1 + k] = rho * (A0 * (U[0] * U[k] + th * dnk) + th * (Ak[k] * U[0] + Ak[0] * U[k]))
    return F0, F1


def test_flux_of_uniform_state_is_isothermal_euler_flux():
    """Sec. 2 Eq. (flux) with zero slopes: F0 = (m_n, m_n U + p, m_n V, m_n W),
    p = rho / (2 lambda); F1 = 0."""
    Q = [1.03, 0.41, -0.2, 0.07]
    F0, F1 = O.flux_local(LAM, 1e-3, Q, [0] * 4, [0] * 4, [0] * 4)
    U = np.array(Q[1:]) / Q[0]
    ref = np.array([Q[1], Q[1] * U[0] + Q[0] * THETA, Q[1] * U[1], Q[1] * U[2]])
    assert np.allclose(F0, ref, rtol=1e-14, atol=1e-13)
    assert np.all(np.abs(F1) <= 1e-12)


def test_flux_shear_gives_newtonian_stress():
    """tau p = mu: a linear shear U_n = gamma x_t1 across an n-face gives the
    tangential momentum flux -mu gamma exactly."""
    mu, gam = 2.3e-3, 0.7
    F0, F1 = O.flux_local(LAM, mu, [1.0, 0.0, 0.0, 0.0], [0] * 4, [0, gam, 0, 0], [0] * 4)
    assert abs(F0[2] - (-mu * gam)) <= 1e-15
    assert abs(F0[1] - THETA) <= 1e-12


def test_flux_compression_has_no_second_viscosity():
    """Isothermal BGK: d_n U_n = kappa gives rho U^2 + p - 2 mu kappa (no -2/3
    divergence term)."""
    mu, kap, rho, U = 1.7e-3, 0.9, 1.1, 0.3
    F0, _ = O.flux_local(LAM, mu, [rho, rho * U, 0, 0], [0, rho * kap, 0, 0], [0] * 4, [0] * 4)
    assert abs(F0[1] - (rho * U * U + rho * THETA - 2 * mu * kap)) <= 1e-12


def test_flux_matches_chapman_enskog_form_random():
    """The moment-based flux (Appendix) equals the hand-derived closed form."""
    rng = np.random.default_rng(7)
    for lam in (LAM, 0.2):
        for _ in range(20):
            rho = 1.0 + 0.2 * rng.random()
            Q = np.r_[rho, rho * rng.normal(size=3)]
            Dn, Dt1, Dt2 = (rng.normal(size=4) for _ in range(3))
            mu = 1e-3 * (1 + rng.random())
            F0, F1 = O.flux_local(lam, mu, Q, Dn, Dt1, Dt2)
            R0, R1 = chapman_enskog_flux(lam, mu, Q, Dn, Dt1, Dt2)
            sc0 = np.max(np.abs(R0)) + 1.0
            sc1 = np.max(np.abs(R1)) + 1.0
            assert np.max(np.abs(F0 - R0)) <= 1e-12 * sc0, (F0, R0)
            assert np.max(np.abs(F1 - R1)) <= 1e-11 * sc1, (F1, R1)


def test_equilibrium_of_equal_states_is_that_state():
    """Sec. 2: equal left and right states give back the same state (the two
    half Maxwellians add up to the full one)."""
    Q = np.array([1.02, 0.3, -0.1, 0.05])
    Q0 = O.equilibrium_local(LAM, Q, Q)
    assert np.allclose(Q0, Q, rtol=2e-15, atol=1e-15)


@pytest.mark.parametrize("lam", [LAM, 0.5])
def test_equilibrium_of_unequal_states_by_quadrature(lam):
    """Sec. 2, Eq. (flux) and the equilibrium state below it: Q0 collects the
    particles of the left Maxwellian moving right (u > 0) and those of the
    right one moving left (u < 0). Integrated here over the normal velocity
    by adaptive quadrature of the 1D Maxwellian; a tangential velocity enters
    as the mean of its Gaussian factor. Unequal densities and velocities in
    every component, including a left state drifting left and a right state
    drifting right."""
    from scipy.integrate import quad

    def half(rho, U, sign, k):
        f = lambda u: u ** k * math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
        lo, hi = (0.0, np.inf) if sign > 0 else (-np.inf, 0.0)
        return rho * quad(f, lo, hi, epsabs=0.0, epsrel=1e-13, limit=200)[0]

    cases = [((1.03, 0.4, 0.2, -0.1), (0.97, -0.3, -0.05, 0.15)),
             ((1.2, -2.5, 0.7, 0.3), (0.8, 3.0, -0.4, -0.9))]
    for (rl, ul, vl, wl), (rr, ur, vr, wr) in cases:
        Ql = np.array([rl, rl * ul, rl * vl, rl * wl])
        Qr = np.array([rr, rr * ur, rr * vr, rr * wr])
        Q0 = O.equilibrium_local(lam, Ql, Qr)
        n0l, n0r = half(rl, ul, +1, 0), half(rr, ur, -1, 0)
        ref = np.array([n0l + n0r, half(rl, ul, +1, 1) + half(rr, ur, -1, 1), vl * n0l + vr * n0r,
                        wl * n0l + wr * n0r])
        assert np.allclose(Q0, ref, rtol=1e-11, atol=1e-12 * max(abs(ul), abs(ur), 1.0)), (Q0, ref)


def test_cfl_time_step_of_the_oracle():
    """Sec. 2 (CFL condition): dt = CFL min(dx, dy, dz) / (max |U| + C) over
    the interior cells, C = sqrt(1 / (2 lambda)) = U_ref / Ma, on a stretched
    grid whose smallest cell is not where the fastest cell is."""
    n = (10, 8, 6)
    faces = [np.linspace(0.0, 1.0, n[0] + 1), np.cumsum(np.r_[0.0, np.linspace(0.05, 0.2, n[1])]),
             np.linspace(0.0, 0.9, n[2] + 1)]
    mach, cfl = 0.2, 0.7
    g = O.OracleGrid(n, faces, mach, 1.0, 1e-3, [("periodic", "periodic")] * 3, cfl=cfl)
    rng = np.random.default_rng(4)
    Q = np.zeros((4,) + tuple(n[::-1]))
    Q[0] = 1.0 + 0.1 * rng.random(Q[0].shape)
    Q[1:] = Q[0] * (rng.random(Q[1:].shape) - 0.5)
    Q[1, 4, 5, 7] = Q[0, 4, 5, 7] * 1.9
    g.set_state(Q)
    umax = np.sqrt(np.max((Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0] ** 2))
    hmin = min(np.min(np.diff(f)) for f in faces)
    assert hmin == pytest.approx(0.05)
    assert g.cfl_dt() == pytest.approx(cfl * hmin / (umax + 1.0 / mach), rel=1e-14)


# -------------------------------------------------------- reconstruction ---

def cell_avgs(c, offsets, half=0.5):
    ci = P.polyint(c)
    return np.array([(P.polyval(o + half, ci) - P.polyval(o - half, ci)) / (2 * half)
                     for o in offsets])


def test_weno5_exact_on_quadratics():
    """Each Jiang-Shu candidate is exact for quadratics, so is any convex
    combination."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        c = rng.normal(size=3)
        q = cell_avgs(c, range(-2, 3))
        assert abs(O.weno5(q) - P.polyval(0.5, c)) <= 1e-13 * (1 + np.abs(c).sum())


def test_weno5_linear_weights_give_fifth_order_linear_scheme():
    """Linear weights (1/10, 6/10, 3/10) combine the three candidates into the
    5-cell quartic reconstruction; that one is exact on quartics."""
    rng = np.random.default_rng(4)
    _, _, _, wd = O.stencil_table()
    for _ in range(20):
        q = rng.normal(size=5)
        p, _, _ = O.weno5_parts(q)
        assert abs(np.dot(wd, p) - O.linear5_face(q)) <= 1e-13
        c = rng.normal(size=5)
        assert abs(O.linear5_face(cell_avgs(c, range(-2, 3))) - P.polyval(0.5, c)) <= 1e-12


def test_weno5_convergence_and_eno_property():
    errs = []
    for n in (20, 40, 80):
        h = 2 * math.pi / n
        e = 0.0
        for i in range(n):
            xs = [(i + o) * h for o in range(-2, 3)]
            q = [(math.cos(x) - math.cos(x + h)) / h for x in xs]   # averages of sin
            e = max(e, abs(O.weno5(q) - math.sin((i + 1) * h)))
        errs.append(e)
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(orders) > 4.5, orders
    # a jump between cell 0 and cell 1: the smooth left stencil takes the weight
    v = O.weno5([0.0, 0.0, 0.0, 1.0, 1.0])
    assert abs(v) < 1e-9
    _, _, w = O.weno5_parts([0.2, -1.0, 3.0, 0.5, 0.1])
    assert abs(w.sum() - 1) < 1e-15 and np.all(w >= 0)


def test_normal_derivative_stencil():
    """Quartic through the face value and the cell averages i-1..i+2 has the
    face derivative [15 (Q_{i+1} - Q_i) - (Q_{i+2} - Q_{i-1})] / 12, with no
    weight on the face value; exact on quartics."""
    dn, _, _, _ = O.stencil_table()
    assert np.allclose(dn, np.array([0.0, 1.0, -15.0, 15.0, -1.0]) / 12, atol=1e-14)
    rng = np.random.default_rng(5)
    for _ in range(20):
        c = rng.normal(size=5)
        ci = P.polyint(c)
        cells = [P.polyval(b, ci) - P.polyval(b - 1, ci) for b in (-1, 0, 1, 2)]
        assert abs(O.normal_derivative(P.polyval(0.0, c), cells) - c[1]) <= 1e-12


def test_tangential_reconstruction_exact_on_quartics():
    """Quartic through 5 face averages, evaluated at the Gauss points
    +-1/(2 sqrt 3) of the centre cell: values and derivatives."""
    g = 1.0 / (2 * math.sqrt(3))
    rng = np.random.default_rng(6)
    for _ in range(20):
        c = rng.normal(size=5)
        val, der = O.tangential(cell_avgs(c, range(-2, 3)))
        dc = P.polyder(c)
        for m, x in enumerate((-g, g)):
            assert abs(val[m] - P.polyval(x, c)) <= 1e-12
            assert abs(der[m] - P.polyval(x, dc)) <= 1e-12
    # the two-point Gauss rule at these nodes integrates cubics exactly
    c = rng.normal(size=4)
    avg = P.polyval(0.5, P.polyint(c)) - P.polyval(-0.5, P.polyint(c))
    assert abs(0.5 * (P.polyval(-g, c) + P.polyval(g, c)) - avg) < 1e-14


# ------------------------------------------------------------ time stepping --

def test_s2o4_reproduces_fourth_order_taylor_polynomial():
    """Two-stage fourth-order method on y' = k y with exact dL/dt = k^2 y."""
    for k, dt in ((-1.3, 0.2), (0.7, 0.05), (-20.0, 0.01)):
        y = np.array([1.7])
        ys = O.s2o4_stage1(dt, y, k * y, k * k * y)
        yn = O.s2o4_stage2(dt, y, k * y, k * k * y, k * k * ys)
        z = k * dt
        ref = 1.7 * (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24)
        assert abs(yn[0] - ref) <= 1e-15 * abs(ref) * 4


# ------------------------------------------------------- projection kernel --

def test_gaussian_kernel_normalisation_and_truncation():
    """Sec. 3.1 Eq. (Gaussian) and Sec. 4.3.1: the kernel integrates to
    erf(3) - (6/sqrt(pi)) e^-9 inside 3 eps, drops to 1 % near 2.15 eps and is
    cut beyond 3 eps."""
    from scipy.integrate import quad
    eps = 0.37
    ref = math.erf(3) - 6 / math.sqrt(math.pi) * math.exp(-9)
    mass = quad(lambda r: 4 * math.pi * r * r * O.gauss_kernel(r, eps), 0, 3 * eps,
                epsabs=1e-14, epsrel=1e-12, limit=200)[0]
    assert abs(mass - ref) < 1e-12
    pv = paper_values()
    r1 = pv["gaussian_one_percent_radius_over_eps"][0]
    ratio = O.gauss_kernel(r1 * eps, eps) / O.gauss_kernel(0.0, eps)
    # the printed radius is rounded to 3 digits: exp(-2.15^2) = 0.0098
    assert abs(ratio - pv["gaussian_one_percent_level"][0]) < 3e-4
    assert O.gauss_kernel(3 * eps * (1 + 1e-12), eps) == 0.0
    assert O.gauss_kernel(3 * eps * (1 - 1e-12), eps) > 0.0
    # on a lattice with eps = 2h the sampled sum is close to the continuum value
    rng = np.random.default_rng(2)
    h = 1.0
    ax = np.arange(-9, 10) + 0.5
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    for _ in range(3):
        X = rng.random(3)
        r = np.sqrt((x - X[0]) ** 2 + (y - X[1]) ** 2 + (z - X[2]) ** 2)
        s = sum(O.gauss_kernel(v, 2 * h) for v in r.ravel()) * h ** 3
        assert abs(s - ref) < 5e-5
