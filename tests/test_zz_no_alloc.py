"""The allocation-free solve entry point, ers_solve_dev_noalloc.

It is meant for callers that must not allocate device memory when they solve (code recording
a CUDA stream capture, code whose device memory belongs to a framework's pool allocator,
latency-bound loops).  Its kernels keep their scratch in a static device array of the
library, so the check here is that, through the C ABI, it returns the same solution as the
ordinary entry point ers_solve on the same factorisation, on two calls in a row (the shared
scratch must be cleared between calls).  This file runs last: it also passes on its own in a
fresh process, where the first call does the one-time scratch set-up."""
import numpy as np
import pytest

from synth import circuits as S

pytestmark = pytest.mark.gpu


def test_noalloc_solve_matches_ordinary_solve():
    torch = pytest.importorskip("torch")
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers

    circ = S.rc_mesh_3d(14, 13, 12, seed=2, n_loads=50)   # several supernode chunks per pass
    sim = ers.Simulator.from_circuit(circ)
    sim.set_state(0.0, np.zeros(circ.n))
    sim.refactor()
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
    sim.close()
