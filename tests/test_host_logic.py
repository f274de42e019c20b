"""Host-side logic that needs no GPU: the benchmark's face counts and its
traffic lookup, the load-history rows (against a stand-in grid), and the
tape decision of the checkpointed adjoint."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_face_counts_of_the_benchmark():
    import bench
    fc = bench.face_counts((384, 256, 256))
    # x faces: 385 planes of 256 x 256; the face box adds 2 rows on each
    # tangential side
    assert fc[0]["flux"] == 385 * 256 * 256 and fc[0]["eq"] == 385 * 260 * 260
    assert fc[1]["flux"] == 257 * 384 * 256 and fc[1]["eq"] == 257 * 388 * 260
    assert fc[2]["flux"] == 257 * 384 * 256 and fc[2]["eq"] == 257 * 388 * 260


def test_traffic_figure_only_for_the_current_sources(tmp_path, monkeypatch):
    import bench
    cur = bench.source_hash("face_flux")
    assert len(cur) == 16 and cur != bench.source_hash("face_eq")
    # a figure taken on other sources is not used
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text("face_flux fp32c 1e9 0123456789abcdef\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda group="face_flux": cur)
    assert bench.read_traffic("face_flux", "fp32c") is None
    (prof / "traffic.txt").write_text("face_flux fp32c 1e9 %s\n" % cur)
    assert bench.read_traffic("face_flux", "fp32c") == 1e9
    assert bench.read_traffic("face_flux", "fp64") is None


def test_measured_flops_only_for_the_current_sources(tmp_path, monkeypatch):
    import bench
    hashes = {g: bench.source_hash(g) for g in bench.SECTIONS}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "flops.txt").write_text(
        "# comment\n"
        "face_eq fp32c - 470.0 %s\n"
        "face_flux fp32c 1 1200.0 %s\n"
        "face_flux fp32c 2 1100.0 %s\n"
        "flux_update fp32c 1 1300.0 0123456789abcdef\n" % (hashes["face_eq"], hashes["face_flux"],
                                                            hashes["face_flux"]))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda group="face_flux": hashes[group])
    fl, src = bench.read_flops("fp32c")
    assert fl["face_eq"] == 470.0 and fl["face_flux_stage1"] == 1200.0 and fl["face_flux_stage2"] == 1100.0
    assert src["face_eq"].startswith("measured") and src["face_flux"].startswith("measured")
    # a stale line falls back to the hand estimate
    assert fl["flux_update_stage1"] == bench.FLOPS_ESTIMATE["flux_update_stage1"]
    assert src["flux_update"] == "hand estimate"
    fl64, src64 = bench.read_flops("fp64")
    assert all(v == "hand estimate" for v in src64.values())


class _FakeGrid:
    """Stand-in for gks.Grid with one rotor and one body and fixed loads."""

    def __init__(self):
        self.objects = [("rotor", 3, 4), ("body", 10, 5)]
        self.t = 0.0
        self.closed = False

    @classmethod
    def from_workload(cls, w, precision="fp64", device=None):
        return cls()

    def step(self, k):
        self.t += 0.5 * k
        return self.t

    def forces(self, oid):
        if oid == 0:
            return {"thrust": np.array([1.0, 2.0, 3.0]), "torque": np.array([0.5, 0.5, 0.5]), "power": 7.0,
                    "cp": 0.4, "ct": 0.8}
        return {"force": np.array([0.1, 0.2, 0.3])}

    def diagnostics(self):
        return np.array([10.0, 1.0, 0.0, 0.0, 2.5])

    def close(self):
        self.closed = True


def test_load_history_rows(monkeypatch):
    from paper_2603_11102_gb300 import gks, history
    monkeypatch.setattr(gks, "Grid", _FakeGrid)
    rows, secs = history.record(object(), "fp32c", 25, 10)
    assert [r[0] for r in rows] == [10, 20, 25]          # every 10 steps and after the last
    assert [r[1] for r in rows] == [5.0, 10.0, 12.5]
    r = dict(zip(history.FIELDS, rows[-1]))
    assert r["thrust"] == 6.0 and r["torque"] == 1.5 and r["power"] == 7.0
    assert (r["body_fx"], r["body_fy"], r["body_fz"]) == (0.1, 0.2, 0.3)
    assert r["mass"] == 10.0 and r["ke"] == 2.5 and secs >= 0.0


class _TapeGrid:
    def __init__(self):
        self.made = 0

    def adjoint_tape_bytes(self):
        return 1 << 30

    def adjoint_tape(self):
        self.made += 1
        return object()


def test_tape_decision_of_the_checkpointed_adjoint():
    from paper_2603_11102_gb300 import adjoint
    g = _TapeGrid()
    assert adjoint._tapes(g, 5, "off") is None and g.made == 0
    tapes = adjoint._tapes(g, 5, "on")
    assert len(tapes) == 5 and g.made == 5
    with pytest.raises(ValueError):
        import torch
        adjoint.rotor_objective(None, torch.ones(3, dtype=torch.float64), torch.tensor(1.0, dtype=torch.float64),
                                10, iplane=3, tape="sometimes")
