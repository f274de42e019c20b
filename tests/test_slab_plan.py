"""Host-side planning of slab groups (gks.plan_slabs): the faces, boundary
kinds and state of each x-slab, and the slab of every rotor and body; no
device needed."""
import numpy as np
import pytest

from paper_2603_11102_gb300 import gks, workloads as WL


def test_periodic_axis_is_closed_by_exchange_sides():
    w = WL.taylor_green_3d(40, steps=1)
    p = gks.plan_slabs(w, [13, 27])
    assert p["cuts"] == [0, 13, 27, 40]
    assert [s["n"][0] for s in p["slabs"]] == [13, 14, 13]
    for s in p["slabs"]:
        assert s["bc"][0] == (gks.EXCHANGE, gks.EXCHANGE)
        assert s["bc"][1:] == [tuple(w.bc[1]), tuple(w.bc[2])]
    # the slabs' faces tile the domain's faces, each cut face shared by two slabs
    f = np.concatenate([p["slabs"][0]["faces"][0]] + [s["faces"][0][1:] for s in p["slabs"][1:]])
    assert np.array_equal(f, w.faces[0])
    # and their states tile the domain's state along x
    assert np.array_equal(np.concatenate([s["state0"] for s in p["slabs"]], axis=3), w.state0)
    # one slab of a periodic axis closes on itself
    q = gks.plan_slabs(w, [])
    assert q["slabs"][0]["bc"][0] == (gks.EXCHANGE, gks.EXCHANGE)


def test_physical_ends_stay_and_objects_go_to_their_slab():
    w = WL.alm_ibm_rotor(n=(96, 64, 64), steps=1, n_pts=10)
    p = gks.plan_slabs(w, [40, 70])
    bcs = [s["bc"][0] for s in p["slabs"]]
    assert bcs == [(w.bc[0][0], gks.EXCHANGE), (gks.EXCHANGE, gks.EXCHANGE), (gks.EXCHANGE, w.bc[0][1])]
    fx = np.asarray(w.faces[0])
    for kind, obj, s in p["objects"]:
        x = obj.hub[0] if kind == "rotor" else float(np.mean(np.asarray(obj.xyz).reshape(-1, 3)[:, 0]))
        assert fx[p["cuts"][s]] <= x < fx[p["cuts"][s + 1]]
    assert [k for k, _, _ in p["objects"]] == ["rotor", "body", "body"]


def test_slabs_thinner_than_the_ghost_layers_are_refused():
    w = WL.taylor_green_3d(16, steps=1)
    with pytest.raises(ValueError):
        gks.plan_slabs(w, [2])
    with pytest.raises(ValueError):
        gks.plan_slabs(w, [8, 10])
