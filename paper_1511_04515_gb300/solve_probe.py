"""Repeated supernodal solves on a 3D RC mesh: a small, self-contained workload for timing or
profiling the triangular-solve kernels in isolation.

    python -m paper_1511_04515_gb300.solve_probe [edge]      # default edge 40 (64,000 nodes)
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1511_04515_gb300 import build, ers  # noqa: E402


def main(k: int = 40, repeats: int = 3):
    build.build()
    from synth import circuits as S
    c = S.rc_mesh_3d(k, k, k, seed=1, n_loads=max(1, k ** 3 // 100))
    sim = ers.Simulator.from_circuit(c)
    sim.set_state(0.0, np.zeros(c.n))
    sim.refactor()
    b = np.random.default_rng(0).normal(size=c.n)
    x = None
    for _ in range(repeats):
        x = sim.solve(b)
    print("ok", float(np.abs(x).max()))


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 40)
