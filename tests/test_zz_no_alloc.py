"""The allocation-free solve entry point, ers_solve_dev_noalloc.

It is meant for callers that may not allocate device memory when they solve: code whose
device memory belongs to a framework's pool allocator, and latency-bound loops that forbid
allocator calls.  Its kernels keep their scratch in a static device array of the library, so
the check here is that, through the C ABI, it returns the same solution as the ordinary
entry point ers_solve on the same factorisation, on two calls in a row (the shared scratch
must be cleared between calls), and that the host-side refusals (no factorisation yet, NULL
or host buffers) return ERS_ERR_INVALID without touching the GPU.  This file runs last: it
also passes on its own in a fresh process, where the first call does the one-time scratch
set-up."""
import ctypes

import numpy as np
import pytest

from synth import circuits as S

pytestmark = pytest.mark.gpu

ERS_ERR_INVALID = 1


def _lib_and_sim():
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers
    circ = S.rc_mesh_3d(14, 13, 12, seed=2, n_loads=50)   # several supernode chunks per pass
    return ers, circ, ers.Simulator.from_circuit(circ)


def test_noalloc_solve_matches_ordinary_solve():
    torch = pytest.importorskip("torch")
    ers, circ, sim = _lib_and_sim()
    sim.set_state(0.0, np.zeros(circ.n))
    sim.refactor()
    dev_before = torch.cuda.current_device()
    rng = np.random.default_rng(7)
    for _ in range(2):
        b = rng.normal(size=circ.n)
        ref = sim.solve(b)                                   # ordinary entry point
        bd = torch.tensor(b, dtype=torch.float64, device="cuda")
        xd = torch.full_like(bd, float("nan"))
        torch.cuda.synchronize()
        sim.solve_dev_noalloc(bd.data_ptr(), xd.data_ptr())
        x = xd.cpu().numpy()
        # same factor, same kernels: agreement to the solve tests' residual bar
        assert np.all(np.isfinite(x))
        assert np.max(np.abs(x - ref)) <= 1e-11 * np.max(np.abs(ref))
    assert torch.cuda.current_device() == dev_before
    sim.close()


def test_noalloc_solve_refuses_bad_calls_on_the_host():
    torch = pytest.importorskip("torch")
    ers, circ, sim = _lib_and_sim()
    L = ers.lib()
    bd = torch.zeros(circ.n, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    torch.cuda.synchronize()
    # no factorisation yet
    launches0 = sim.stats()["kernel_launches"]
    rc = L.ers_solve_dev_noalloc(sim._ctx, ctypes.c_void_p(bd.data_ptr()),
                                 ctypes.c_void_p(xd.data_ptr()))
    assert rc == ERS_ERR_INVALID
    assert "factorisation" in L.ers_last_error(sim._ctx).decode()
    sim.set_state(0.0, np.zeros(circ.n))
    sim.refactor()
    launches1 = sim.stats()["kernel_launches"]
    # NULL buffers
    assert L.ers_solve_dev_noalloc(sim._ctx, None, ctypes.c_void_p(xd.data_ptr())) == ERS_ERR_INVALID
    assert L.ers_solve_dev_noalloc(sim._ctx, ctypes.c_void_p(bd.data_ptr()), None) == ERS_ERR_INVALID
    # host buffers (plain, unregistered memory) are refused before any kernel runs
    hb = np.zeros(circ.n)
    hx = np.zeros(circ.n)
    rc = L.ers_solve_dev_noalloc(sim._ctx, hb.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.c_void_p(xd.data_ptr()))
    assert rc == ERS_ERR_INVALID
    assert "device memory" in L.ers_last_error(sim._ctx).decode()
    rc = L.ers_solve_dev_noalloc(sim._ctx, ctypes.c_void_p(bd.data_ptr()),
                                 hx.ctypes.data_as(ctypes.c_void_p))
    assert rc == ERS_ERR_INVALID
    assert sim.stats()["kernel_launches"] == launches1
    assert launches1 >= launches0
    # the context still works afterwards
    b = np.random.default_rng(3).normal(size=circ.n)
    bd.copy_(torch.from_numpy(b))
    torch.cuda.synchronize()
    sim.solve_dev_noalloc(bd.data_ptr(), xd.data_ptr())
    ref = sim.solve(b)
    assert np.max(np.abs(xd.cpu().numpy() - ref)) <= 1e-11 * np.max(np.abs(ref))
    sim.close()
