"""gks_diagnostics_noalloc, the reduction for callers that cannot allocate
device memory (an application that owns all device memory through its own
pool, or whose device-memory budget is already committed): through the C ABI
it gives the same sums as gks_diagnostics, on two calls in a row with
different states, and rejects a size beyond its static scratch.

Collected last on purpose (file name), so that a run that stops at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2603_11102_gb300 import workloads as WL

from _setup import smooth_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gks():
    from paper_2603_11102_gb300 import build, gks
    build.build()
    gks.load()
    return gks


def call_noalloc(gks, torch, Q, faces, stream):
    n = (Q.shape[3], Q.shape[2], Q.shape[1])
    dq = torch.tensor(Q.reshape(-1), dtype=torch.float64, device="cuda")
    dh = [torch.tensor(np.diff(faces[a]), dtype=torch.float64, device="cuda") for a in range(3)]
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    rc = gks.lib.gks_diagnostics_noalloc(C.c_void_p(dq.data_ptr()), n[0], n[1], n[2],
                                         C.c_void_p(dh[0].data_ptr()), C.c_void_p(dh[1].data_ptr()),
                                         C.c_void_p(dh[2].data_ptr()), C.c_void_p(out.data_ptr()),
                                         C.c_void_p(stream.cuda_stream))
    assert rc == 0, gks.lib.gks_last_error(None)
    stream.synchronize()
    return out.cpu().numpy()


def scales(Q, faces):
    """Sum of absolute terms of each of the 5 sums: the size rounding acts on."""
    vol = np.multiply.outer(np.multiply.outer(np.diff(faces[2]), np.diff(faces[1])), np.diff(faces[0]))
    terms = [Q[0], Q[1], Q[2], Q[3], 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0]]
    return np.array([np.sum(np.abs(t) * vol) for t in terms])


def test_noalloc_matches_diagnostics_on_two_calls(gks):
    import torch
    n = (45, 19, 23)       # several blocks of 4096 cells and a ragged last block
    faces = [np.linspace(0, 2.0, n[0] + 1), WL.tanh_faces(n[1]), np.linspace(0, 1.3, n[2] + 1)]
    w = smooth_workload(n, [(0, 0), (1, 1), (0, 0)], faces=faces, seed=12)
    g = gks.Grid.from_workload(w, precision="fp64")
    stream = g.stream
    for call in range(2):
        g.step(2)                               # a different state for each call
        Q = g.get_state()
        ref = g.diagnostics()
        got = call_noalloc(gks, torch, Q, faces, stream)
        tol = 1e-13 * scales(Q, faces)
        assert np.all(np.abs(got - ref) <= tol), (call, got, ref)
    g.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(gks):
    import torch
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(d.data_ptr())
    rc = gks.lib.gks_diagnostics_noalloc(p, 4096, 4096, 3, p, p, p, p, None)
    assert rc == -1
    assert b"33554432" in gks.lib.gks_last_error(None)
    assert gks.lib.gks_diagnostics_noalloc(None, 2, 2, 2, p, p, p, p, None) == -1
