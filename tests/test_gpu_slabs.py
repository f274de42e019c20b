"""Slab groups (gks_slab_step): a domain split along x into slabs on one
device, stepped with the x halo exchange of every stage and a common time
step, reproduces a single grid of the whole domain (the paper's
decomposition into x-slabs, Sec. 3; run here on one GPU) bit for bit, in FP64
and in FP32C: every kernel rounds a face or a cell the same way wherever the
cut puts it."""
import numpy as np
import pytest

from _setup import rel_linf, smooth_workload
from paper_2603_11102_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gks():
    from paper_2603_11102_gb300 import build, gks
    build.build()
    gks.load()
    return gks


def single_and_slabs(gks, w, cuts, precision, steps):
    g = gks.Grid.from_workload(w, precision=precision)
    t1 = g.step(steps)
    sg = gks.SlabGroup(w, cuts, precision=precision)
    t2 = sg.step(steps)
    return g, sg, t1, t2


def assert_same(g, sg, t1, t2, precision):
    a, b = sg.get_state(), g.get_state()
    assert t1 == t2, (precision, t1, t2)
    assert np.array_equal(a, b), (precision, rel_linf(a, b))


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_periodic_three_slabs_match_the_single_grid_bitwise(gks, precision):
    """Taylor-Green 40^3, periodic in x: three slabs (13, 14, 13 cells), the
    group closing the periodic axis; the CFL step from the group's maximum."""
    w = WL.taylor_green_3d(40, steps=10)
    g, sg, t1, t2 = single_and_slabs(gks, w, [13, 27], precision, 10)
    assert_same(g, sg, t1, t2, precision)
    g.close()
    sg.close()
    # 64^3 cut in the middle, and one slab closing the periodic axis on itself
    w = WL.taylor_green_3d(64, steps=4)
    g, sg, t1, t2 = single_and_slabs(gks, w, [29], precision, 4)
    assert_same(g, sg, t1, t2, precision)
    g.close()
    sg.close()
    g, sg, t1, t2 = single_and_slabs(gks, w, [], precision, 4)
    assert_same(g, sg, t1, t2, precision)
    g.close()
    sg.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_channel_two_slabs_match_the_single_grid_bitwise(gks, precision):
    """The channel on a ragged 70 x 45 x 37 grid: periodic x cut into two
    slabs, tanh-stretched y between no-slip walls, periodic z, driving body
    force."""
    w = WL.channel((70, 45, 37), steps=8)
    g, sg, t1, t2 = single_and_slabs(gks, w, [35], precision, 8)
    assert_same(g, sg, t1, t2, precision)
    g.close()
    sg.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_rotor_and_bodies_in_one_slab_of_two(gks, precision):
    """Rotor, tower and nacelle (inflow x-, outflow x+) with the cut
    downstream of every kernel support: the state, the rotor loads and the
    body forces match the single grid's bit for bit."""
    w = WL.alm_ibm_rotor(n=(96, 64, 64), steps=6, n_pts=20)
    w.state0 = WL.perturbed(w, 0.02, seed=9)
    g, sg, t1, t2 = single_and_slabs(gks, w, [60], precision, 6)
    assert_same(g, sg, t1, t2, precision)
    for oid in range(3):
        a, b = g.forces(oid), sg.forces(oid)
        for k, v in a.items():
            assert np.array_equal(np.asarray(v), np.asarray(b[k])), (oid, k)
    g.close()
    sg.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
@pytest.mark.parametrize("cut", [27, 20])
def test_rotor_support_across_a_cut_is_shared(gks, precision, cut):
    """A rotor whose kernel support crosses the cut: the slab that holds the
    rotor plane samples the flow and computes the loads, the slab behind the
    cut spreads the same point forces into its cells (a share); the rotor
    sits in the first slab (cut 27) or in the second (cut 20, its cells on
    the domain's lattice by their offset)."""
    w = WL.alm_rotor(n=(96, 32, 32), steps=6, n_pts=20)
    w.state0 = WL.perturbed(w, 0.02, seed=3)
    plan = gks.plan_slabs(w, [cut])
    assert plan["rotor_shares"][0] == [1 - plan["objects"][0][2]]
    g, sg, t1, t2 = single_and_slabs(gks, w, [cut], precision, 6)
    assert_same(g, sg, t1, t2, precision)
    a, b = g.forces(0), sg.forces(0)
    for k, v in a.items():
        assert np.array_equal(np.asarray(v), np.asarray(b[k])), k
    g.close()
    sg.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_objects_in_a_later_slab_sit_on_the_domain_lattice(gks, precision):
    """Rotor, tower and nacelle all in the second slab (cut at x cell 10):
    their cells and points on the domain's lattice through the slab's offset,
    so state, loads and body forces have the single grid's bits."""
    w = WL.alm_ibm_rotor(n=(96, 64, 64), steps=4, n_pts=20)
    w.state0 = WL.perturbed(w, 0.02, seed=5)
    g, sg, t1, t2 = single_and_slabs(gks, w, [10], precision, 4)
    assert_same(g, sg, t1, t2, precision)
    for oid in range(3):
        a, b = g.forces(oid), sg.forces(oid)
        for k, v in a.items():
            assert np.array_equal(np.asarray(v), np.asarray(b[k])), (oid, k)
    g.close()
    sg.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_smooth_state_with_walls_and_an_outflow_across_four_slabs(gks, precision):
    """A seeded smooth state with inflow / outflow in x, slip and no-slip
    walls in y and z, four slabs of unequal widths."""
    n = (41, 12, 10)
    faces = [np.linspace(0.0, 2.0, n[0] + 1), np.linspace(0.0, 1.0, n[1] + 1), np.linspace(0.0, 0.8, n[2] + 1)]
    w = smooth_workload(n, [(3, 4), (2, 2), (1, 1)], faces=faces, seed=4)
    w.inflow = (1.0, 0.6, 0.0, 0.05)
    g, sg, t1, t2 = single_and_slabs(gks, w, [9, 20, 31], precision, 6)
    assert_same(g, sg, t1, t2, precision)
    g.close()
    sg.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_stretched_x_axis_cut_three_times(gks, precision):
    """A tanh-stretched x axis (inflow / outflow), periodic y, slip z, cut
    into three slabs of unequal widths: the ghost cells of each cut take the
    neighbour's widths, so the geometry matches the single grid's and the
    state does too."""
    n = (36, 10, 12)
    faces = [WL.tanh_faces(n[0]), np.linspace(0.0, 1.0, n[1] + 1), np.linspace(0.0, 1.2, n[2] + 1)]
    w = smooth_workload(n, [(3, 4), (0, 0), (2, 2)], faces=faces, seed=6)
    w.inflow = (1.0, 0.5, 0.05, 0.0)
    g, sg, t1, t2 = single_and_slabs(gks, w, [10, 23], precision, 6)
    assert_same(g, sg, t1, t2, precision)
    g.close()
    sg.close()


def test_support_across_a_cut_and_mismatched_slabs_are_refused(gks):
    """A rotor whose kernel support reaches a cut without a share behind it is
    refused by the group step (GKS_ERR_RANGE), a body's at registration;
    slabs whose y faces differ are refused by the group step (GKS_ERR_ARG)."""
    import ctypes as C
    w = WL.alm_rotor(n=(96, 32, 32), steps=2, n_pts=10)
    plan = gks.plan_slabs(w, [27])
    grids = []
    for sp in plan["slabs"]:
        gr = gks.Grid(sp["n"], sp["faces"], w.mach, w.u_ref, w.mu, sp["bc"], precision="fp64",
                      stream=grids[0].stream if grids else None)
        gr.set_slab_lattice(plan["lattice"][0], plan["lattice"][1], sp["cells_before"])
        grids.append(gr)
    grids[0].add_rotor(w.rotors[0])   # no share on the second slab
    h = (C.c_void_p * 2)(grids[0].h, grids[1].h)
    assert gks.lib.gks_slab_step(h, 2, 1, None) == -6
    wb = WL.alm_ibm_rotor(n=(96, 64, 64), steps=2, n_pts=10)
    with pytest.raises(gks.GKSError) as e:
        gks.SlabGroup(wb, [27], precision="fp64")   # the nacelle's support crosses x cell 27
    assert e.value.code == -6
    for gr in grids:
        gr.close()
    a = gks.Grid((12, 8, 8), [np.linspace(0, 1, 13), np.linspace(0, 1, 9), np.linspace(0, 1, 9)], 0.1, 1.0, 1e-3,
                 [(4, 5), (0, 0), (0, 0)])
    b = gks.Grid((12, 8, 8), [np.linspace(1, 2, 13), np.linspace(0, 1.5, 9), np.linspace(0, 1, 9)], 0.1, 1.0, 1e-3,
                 [(5, 4), (0, 0), (0, 0)], stream=a.stream)
    h = (C.c_void_p * 2)(a.h, b.h)
    assert gks.lib.gks_slab_step(h, 2, 1, None) == -1
    a.close()
    b.close()
