"""The hand-written adjoint (reverse mode) of the FP64 step, through the C ABI.

One step: <lambda^{n+1}, dW^{n+1}> from central differences of the CUDA
forward step equals <lambda^n, dW^n> (+ the force-scale, inflow-speed and
power-seed terms) from gks_step_adjoint. Rollout: the checkpointed
torch.autograd.Function gives the gradient of the wake-deficit plus power
objective that central differences (h = 1e-6, FP64) of the CUDA forward and
of the CPU oracle give. The same with an immersed body (fixed IBM iteration
count) next to the rotor."""
import numpy as np
import pytest

from paper_2603_11102_gb300 import workloads as WL

from _setup import oracle_from_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch

    from paper_2603_11102_gb300 import adjoint, build, gks
    build.build()
    gks.load()
    return gks, adjoint, torch


def rotor_box_workload(n=(24, 16, 16), n_pts=6, uinf=1.0):
    nx, ny, nz = n
    faces = [np.linspace(-1.5, 1.5, nx + 1), np.linspace(-1.0, 1.0, ny + 1), np.linspace(-1.0, 1.0, nz + 1)]
    dx = 3.0 / nx
    hmin = min(3.0 / nx, 2.0 / ny, 2.0 / nz)
    dt = 0.5 * hmin / (uinf + 10.0)
    rot = WL.rotor_3x50(D=1.0, hub=(0.0, 0.0, 0.0), dx=dx, n_pts=n_pts, u_inf=uinf)
    Q = np.zeros((4, nz, ny, nx))
    Q[0], Q[1] = 1.0, uinf
    return WL.Workload("adjoint-rotor", n, faces, 0.1, 1.0, 2e-3, [(3, 4), (0, 0), (2, 2)], cfl=0.9, dt_fixed=dt,
                       inflow=(1.0, uinf, 0.0, 0.0), state0=Q, rotors=[rot])


def rotor_body_workload():
    """The rotor box plus a cylinder (axis z, behind the rotor) forced by IBM
    with a fixed iteration count."""
    w = rotor_box_workload()
    dx = 3.0 / w.n[0]
    xyz, dS = WL.cylinder_points((0.4, 0.1, 0.0), 2, 0.12, -0.8, 0.2, 0.09, caps=False)
    w.bodies = [WL.Body(xyz, dS, 2 * dx, niter=4, tol=0.0)]
    return w


def rotor_corrections_workload():
    """The rotor box with the ALM velocity correction and the tip factors."""
    w = rotor_box_workload()
    w.rotors[0].correction = True
    w.rotors[0].tip_correction = True
    return w


def walls_workload(n=(20, 12, 10)):
    faces = [np.linspace(0, 2.0, n[0] + 1), WL.tanh_faces(n[1]), np.linspace(0, 1.0, n[2] + 1)]
    Q = np.zeros((4, n[2], n[1], n[0]))
    Q[0], Q[1] = 1.0, 0.6
    return WL.Workload("adjoint-walls", n, faces, 0.1, 1.0, 3e-3, [(3, 4), (1, 2), (0, 0)], cfl=0.9, dt_fixed=1.5e-3,
                       inflow=(1.0, 0.6, 0.0, 0.0), state0=Q)


def perturbed_state(w, seed, amp=0.03):
    rng = np.random.default_rng(seed)
    Q = w.state0.copy()
    xc = [0.5 * (f[1:] + f[:-1]) for f in w.faces]
    Z, Y, X = np.meshgrid(xc[2], xc[1], xc[0], indexing="ij")
    Q[0] += 0.01 * np.sin(2 * X + 0.3) * np.cos(3 * Y)
    Q[1] += amp * np.cos(X) * np.sin(2 * Z + 0.1)
    Q[2] += amp * np.sin(Y + Z)
    Q[3] += amp * np.cos(2 * X - Y)
    Q += 1e-3 * rng.standard_normal(Q.shape) * np.array([0.1, 1, 1, 1])[:, None, None, None]
    return Q


def forward_step(g, torch, W, t_n, scales=None, uinf=None):
    if scales is not None:
        g.set_force_scales(0, scales)
    if uinf is not None:
        g.set_inflow(1.0, uinf, 0.0, 0.0)
    g.set_state_tensor(W)
    g.set_time(t_n)
    g.step(1)
    out = g.state_tensor()
    P = g.forces(0)["power"] if g.objects else 0.0
    return out, P


@pytest.mark.parametrize("rev", ["fp64", "fp32", "fp32c"])
@pytest.mark.parametrize("case", ["rotor", "walls", "rotor_body", "rotor_corrections"])
def test_one_step_adjoint_matches_central_differences(mods, case, rev):
    """rev: arithmetic of the local reverse maps of the FP64 step (FP64 within
    1e-5 of the central differences of the FP64 step; FP32 within 1e-4), or
    fp32c: the recorded FP32C step and its reverse (FP32 arithmetic), against
    the central differences of the FP64 step: within 1e-4 for the inflow
    speed and the force scales. In the state direction the inner product
    <lambda^n, dW> of this random direction nearly cancels (|sum| ~ 1 against
    terms of total magnitude ~1e4), so the FP32C adjoint, whose elements sit
    within ~1e-5 of the FP64 step's adjoint (FP32 flux arithmetic: its slopes
    are small differences of O(1) values), is held to 1e-6 of the summed
    magnitude of the terms, element by element to 3e-5 of the FP64 step's
    adjoint, and along a direction that follows the sign of that adjoint
    (no cancellation) to 1e-4 of the central difference."""
    gks, adjoint, torch = mods
    w = {"rotor": rotor_box_workload, "walls": walls_workload, "rotor_body": rotor_body_workload,
         "rotor_corrections": rotor_corrections_workload}[case]()
    g = gks.Grid.from_workload(w, precision="fp64")
    g.set_adjoint_precision("fp32" if rev == "fp32c" else rev)
    tol = 1e-5 if rev == "fp64" else 1e-4
    W = torch.tensor(perturbed_state(w, 3), dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(5)
    lam1 = torch.tensor(rng.standard_normal(W.shape), dtype=torch.float64, device="cuda")
    beta = 0.0 if case == "walls" else 0.7
    t_n = 0.37
    npts = 0 if case == "walls" else 3 * 6
    s0 = np.ones(max(npts, 1))
    u0 = w.inflow[1]

    def J(Wx, s=None, u=None):
        out, P = forward_step(g, torch, Wx, t_n, s if npts else None, u)
        return float((lam1 * out).sum().item()) + beta * P

    gs = np.zeros(max(npts, 1))
    if rev == "fp32c":
        ga = gks.Grid.from_workload(w, precision="fp32c")
        if npts:
            ga.set_force_scales(0, s0)
        ga.set_inflow(1.0, u0, 0.0, 0.0)
        ga.set_state_tensor(W)
        ga.set_time(t_n)
        tape = ga.adjoint_tape()
        ga.step_record(tape)
        lam0, gu = ga.step_reverse(tape, ga.adjoint_scratch(), lam1, beta, gs if npts else None)
        ga.close()
    else:
        work = g.adjoint_workspace()
        if npts:
            g.set_force_scales(0, s0)
        g.set_inflow(1.0, u0, 0.0, 0.0)
        lam0, gu = g.step_adjoint(work, t_n, W, lam1, beta, gs if npts else None)

    # state direction. The WENO weights of this noisy state sit in the
    # beta ~ eps_w regime, where they bend on a 1e-3 scale: the central
    # differences need h ~ 1e-7 for their O(h^2) error to drop below 1e-6.
    dW = torch.tensor(rng.standard_normal(W.shape), dtype=torch.float64, device="cuda")
    dW[0] *= 0.1
    h = 1e-7
    fd = (J(W + h * dW, s0, u0) - J(W - h * dW, s0, u0)) / (2 * h)
    ad = float((lam0 * dW).sum().item())
    if rev == "fp32c":
        mag = float((lam0 * dW).abs().sum().item())
        assert abs(fd - ad) <= 1e-6 * mag, (fd, ad, mag)
        ref, _ = g.step_adjoint(g.adjoint_workspace(), t_n, W, lam1, beta, None)
        assert float((lam0 - ref).abs().max()) <= 3e-5 * float(ref.abs().max())
        # a direction whose inner product cannot cancel: every element along
        # the sign of the FP64 step's adjoint, with a random size
        dWa = torch.sign(ref) * torch.tensor(0.5 + rng.random(W.shape), dtype=torch.float64, device="cuda")
        dWa[0] *= 0.1
        fda = (J(W + h * dWa, s0, u0) - J(W - h * dWa, s0, u0)) / (2 * h)
        ada = float((lam0 * dWa).sum().item())
        assert abs(fda - ada) <= 1e-4 * abs(fda), (fda, ada)
    else:
        assert abs(fd - ad) <= tol * max(abs(ad), 1e-12), (fd, ad)
    # inflow speed
    fdu = (J(W, s0, u0 + h) - J(W, s0, u0 - h)) / (2 * h)
    assert abs(fdu - gu) <= tol * max(abs(fdu), 1e-3), (fdu, gu)
    # force scales
    if npts:
        h = 1e-6
        ds = rng.standard_normal(npts)
        fds = (J(W, s0 + h * ds, u0) - J(W, s0 - h * ds, u0)) / (2 * h)
        assert abs(fds - float(np.dot(gs, ds))) <= tol * max(abs(fds), 1e-12), (fds, np.dot(gs, ds))
    g.close()


@pytest.mark.parametrize("rev", ["fp64", "fp32"])
def test_ibm_tolerance_mode_through_recorded_steps(mods, rev):
    """IBM with a residual tolerance: the iteration count is piecewise
    constant in the state, so the step's derivative is that of the realised
    count, which the recorded step keeps. The tolerance is set between the
    residuals after the second and third iteration of this state, so that
    the count (3 of at most 6) is the same at every finite-difference point."""
    gks, adjoint, torch = mods
    w = rotor_body_workload()
    w.bodies[0].niter = 6
    w.bodies[0].tol = 1e-300   # a tolerance it never meets: the residual after every iteration
    W = torch.tensor(perturbed_state(w, 3), dtype=torch.float64, device="cuda")
    t_n = 0.37
    g0 = gks.Grid.from_workload(w, precision="fp64")
    forward_step(g0, torch, W, t_n)
    r = g0.forces(1)["residual_history"]
    g0.close()
    assert len(r) == 6 and r[2] < r[1]
    w.bodies[0].tol = float(np.sqrt(r[1] * r[2]))
    g = gks.Grid.from_workload(w, precision="fp64")
    g.set_adjoint_precision(rev)
    rng = np.random.default_rng(5)
    lam1 = torch.tensor(rng.standard_normal(W.shape), dtype=torch.float64, device="cuda")
    beta, npts, u0 = 0.7, 18, w.inflow[1]
    s0 = np.ones(npts)

    def J(Wx, s=None, u=None):
        out, P = forward_step(g, torch, Wx, t_n, s, u)
        assert g.forces(1)["iters"] == 3
        return float((lam1 * out).sum().item()) + beta * P

    g.set_force_scales(0, s0)
    g.set_inflow(1.0, u0, 0.0, 0.0)
    g.set_state_tensor(W)
    g.set_time(t_n)
    tape = g.adjoint_tape()
    g.step_record(tape)
    assert g.forces(1)["iters"] == 3
    gs = np.zeros(npts)
    lam0, gu = g.step_reverse(tape, g.adjoint_scratch(), lam1, beta, gs)
    tol = 1e-5 if rev == "fp64" else 1e-4
    dW = torch.tensor(rng.standard_normal(W.shape), dtype=torch.float64, device="cuda")
    dW[0] *= 0.1
    h = 1e-7
    fd = (J(W + h * dW, s0, u0) - J(W - h * dW, s0, u0)) / (2 * h)
    ad = float((lam0 * dW).sum().item())
    assert abs(fd - ad) <= tol * max(abs(ad), 1e-12), (fd, ad)
    fdu = (J(W, s0, u0 + h) - J(W, s0, u0 - h)) / (2 * h)
    assert abs(fdu - gu) <= tol * max(abs(fdu), 1e-3), (fdu, gu)
    ds = rng.standard_normal(npts)
    h = 1e-6
    fds = (J(W, s0 + h * ds, u0) - J(W, s0 - h * ds, u0)) / (2 * h)
    assert abs(fds - float(np.dot(gs, ds))) <= tol * max(abs(fds), 1e-12), (fds, np.dot(gs, ds))
    # the per-step recomputation keeps refusing the tolerance mode
    with pytest.raises(gks.GKSError) as e:
        g.step_adjoint(g.adjoint_workspace(), t_n, W, lam1)
    assert e.value.code == -5
    g.close()


def oracle_objective(w, s, u, nsteps, iplane, beta):
    w = WL.Workload(w.name, w.n, w.faces, w.mach, w.u_ref, w.mu, w.bc, cfl=w.cfl, dt_fixed=w.dt_fixed,
                    inflow=(1.0, u, 0.0, 0.0), state0=None, rotors=w.rotors, bodies=w.bodies)
    Q = np.zeros((4,) + w.n[::-1])
    Q[0], Q[1] = 1.0, u
    o = oracle_from_workload(w, Q)
    o.set_force_scales(0, s)
    o.step(nsteps)
    A = o.get_state()
    return float(np.mean(u - A[1, :, :, iplane] / A[0, :, :, iplane])) + beta * o.forces(0)["power"]


@pytest.mark.parametrize("rev", ["fp64", "fp32", "fp32c"])
@pytest.mark.parametrize("case", ["rotor", "rotor_body", "rotor_corrections"])
def test_rollout_gradient_vs_finite_differences_and_oracle(mods, case, rev):
    """rev as in the one-step test; fp32c: the gradient of the FP32C
    rollout, checked against central differences of the FP64 rollout and of
    the oracle. Recorded steps and per-step recomputation give the same
    gradient (FP32C: to 1e-6, since a checkpoint's FP64 copy of the
    compensated state can drop the lowest bits of its lo part)."""
    gks, adjoint, torch = mods
    w = {"rotor": rotor_box_workload, "rotor_body": rotor_body_workload,
         "rotor_corrections": rotor_corrections_workload}[case]()
    g = gks.Grid.from_workload(w, precision="fp32c" if rev == "fp32c" else "fp64")
    g.set_adjoint_precision("fp32" if rev == "fp32c" else rev)
    gfd = gks.Grid.from_workload(w, precision="fp64") if rev == "fp32c" else g
    N, K, beta = 6, 2, 1.0
    iplane = 20          # x index downstream of the rotor
    npts = 18
    s = torch.ones(npts, dtype=torch.float64, requires_grad=True)
    u = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    J = adjoint.rotor_objective(g, s, u, N, K=K, iplane=iplane, beta=beta, tape="on")
    J.backward()
    gs, gu = s.grad.numpy().copy(), float(u.grad)
    # recorded steps and per-step recomputation give the same gradient
    s2 = torch.ones(npts, dtype=torch.float64, requires_grad=True)
    u2 = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    adjoint.rotor_objective(g, s2, u2, N, K=K, iplane=iplane, beta=beta, tape="off").backward()
    same = 1e-6 if rev == "fp32c" else 1e-12
    assert np.max(np.abs(s2.grad.numpy() - gs)) <= same * np.max(np.abs(gs))
    assert abs(float(u2.grad) - gu) <= same * abs(gu)

    def Jgpu(sv, uv):
        return float(adjoint.rotor_objective(gfd, torch.tensor(sv, dtype=torch.float64),
                                             torch.tensor(uv, dtype=torch.float64), N, K=K, iplane=iplane,
                                             beta=beta))

    h = 1e-6
    s0 = np.ones(npts)
    scale = np.max(np.abs(gs))
    for p in (0, 7, 17):
        e = np.zeros(npts)
        e[p] = h
        fd = (Jgpu(s0 + e, 1.0) - Jgpu(s0 - e, 1.0)) / (2 * h)
        assert abs(fd - gs[p]) <= 1e-4 * scale, (p, fd, gs[p])
    fdu = (Jgpu(s0, 1.0 + h) - Jgpu(s0, 1.0 - h)) / (2 * h)
    assert abs(fdu - gu) <= 1e-4 * abs(gu), (fdu, gu)
    # reference gradient from the CPU oracle (central differences of its J)
    for p in (0, 17):
        e = np.zeros(npts)
        e[p] = h
        fo = (oracle_objective(w, s0 + e, 1.0, N, iplane, beta) -
              oracle_objective(w, s0 - e, 1.0, N, iplane, beta)) / (2 * h)
        assert abs(fo - gs[p]) <= 1e-4 * scale, (p, fo, gs[p])
    fou = (oracle_objective(w, s0, 1.0 + h, N, iplane, beta) -
           oracle_objective(w, s0, 1.0 - h, N, iplane, beta)) / (2 * h)
    assert abs(fou - gu) <= 1e-4 * abs(gu), (fou, gu)
    if w.bodies or w.rotors[0].correction:
        # the body or the corrections act on the objective (the case is not
        # the rotor case again)
        J1 = oracle_objective(w, s0, 1.0, N, iplane, beta)
        w0 = rotor_box_workload()
        J0 = oracle_objective(w0, s0, 1.0, N, iplane, beta)
        assert abs(J1 - J0) > 1e-6 * abs(J0), (J1, J0)
    g.close()


@pytest.mark.parametrize("rev", ["fp64", "fp32", "fp32c"])
def test_recorded_step_and_its_reverse(mods, rev):
    """gks_step_record steps the grid as gks_step does, and gks_step_reverse
    from its tape gives what gks_step_adjoint gives from W^n; the reverse
    only reads the tape, so a second reverse gives the same bits. fp32c: an
    FP32C grid (its own fused FP32 reverse, and gks_step_adjoint recomputing
    the FP32C step in its workspace)."""
    gks, adjoint, torch = mods
    w = rotor_body_workload()
    g = gks.Grid.from_workload(w, precision="fp32c" if rev == "fp32c" else "fp64")
    g.set_adjoint_precision("fp32" if rev == "fp32c" else rev)
    W = torch.tensor(perturbed_state(w, 4), dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(9)
    lam1 = torch.tensor(rng.standard_normal(W.shape), dtype=torch.float64, device="cuda")
    t_n = 0.21
    ref, _ = forward_step(g, torch, W, t_n)
    tape, scratch = g.adjoint_tape(), g.adjoint_scratch()
    g.set_state_tensor(W)
    g.set_time(t_n)
    t1 = g.step_record(tape)
    assert torch.equal(g.state_tensor(), ref)
    assert t1 == g.time
    gs_r = np.zeros(18)
    lam_r, gu_r = g.step_reverse(tape, scratch, lam1, 0.4, gs_r)
    gs_a = np.zeros(18)
    lam_a, gu_a = g.step_adjoint(g.adjoint_workspace(), t_n, W, lam1, 0.4, gs_a)
    assert torch.equal(lam_r, lam_a)
    assert np.array_equal(gs_r, gs_a) and gu_r == gu_a
    # the grid's state and time are those the recorded step left
    assert torch.equal(g.state_tensor(), ref) and g.time == t1
    gs_2 = np.zeros(18)
    lam_2, gu_2 = g.step_reverse(tape, scratch, lam1, 0.4, gs_2)
    assert torch.equal(lam_2, lam_r) and np.array_equal(gs_2, gs_r) and gu_2 == gu_r
    with pytest.raises(gks.GKSError) as e:
        g.step_reverse(torch.zeros_like(tape), scratch, lam1)
    assert e.value.code == -5
    if rev == "fp32c":
        g.close()
        return
    # a tape is reversed in the adjoint precision it was recorded with
    g.set_state_tensor(W)
    g.step_record(tape)
    g.set_adjoint_precision("fp64" if rev == "fp32" else "fp32")
    with pytest.raises(gks.GKSError) as e:
        g.step_reverse(tape, g.adjoint_scratch(), lam1)
    assert e.value.code == -5
    g.close()


def test_adjoint_rejects_unsupported_grids(mods):
    gks, adjoint, torch = mods
    w = rotor_box_workload()
    w.dt_fixed = 0.0
    g = gks.Grid.from_workload(w, precision="fp64")
    work = g.adjoint_workspace()
    W = g.state_tensor()
    with pytest.raises(gks.GKSError) as e:
        g.step_adjoint(work, 0.0, W, W)
    assert e.value.code == -5
    # per-step recomputation needs a fixed IBM iteration count, FP32C too
    w6 = rotor_body_workload()
    w6.bodies[0].tol = 0.05
    g2 = gks.Grid.from_workload(w6, precision="fp32c")
    with pytest.raises(gks.GKSError) as e:
        g2.step_adjoint(g2.adjoint_workspace(), 0.0, W, W)
    assert e.value.code == -5
    w2 = rotor_box_workload()
    w2.dt_fixed = 0.0
    g5 = gks.Grid.from_workload(w2, precision="fp32c")
    with pytest.raises(gks.GKSError) as e:
        g5.step_record(g5.adjoint_tape())
    assert e.value.code == -5
    w4 = rotor_body_workload()
    w4.bodies[0].tol = 0.05
    g4 = gks.Grid.from_workload(w4, precision="fp64")
    with pytest.raises(gks.GKSError) as e:
        g4.step_adjoint(g4.adjoint_workspace(), 0.0, W, W)
    assert e.value.code == -5
    w3 = rotor_box_workload()
    w3.rotors.append(rotor_box_workload().rotors[0])
    g3 = gks.Grid.from_workload(w3, precision="fp64")
    with pytest.raises(gks.GKSError) as e:
        g3.step_adjoint(g3.adjoint_workspace(), 0.0, W, W)
    assert e.value.code == -5
