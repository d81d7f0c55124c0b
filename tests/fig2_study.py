"""Fig. 2-style accuracy study on the CPU oracle: ER, ER-C and BENR at equal fixed step sizes
through one switching window of a two-stage inverter chain, against a fine ER reference.

Run: python tests/fig2_study.py   (a few seconds)

The paper's Fig. 2 compares ER, ER-C and backward Euler with Newton (BENR) at equal steps on
a nonlinear circuit.  Here the window is 16 ps starting at 0.11 ns (the first output edge of
the chain), the Krylov tolerance 1e-12 (so only the time discretisation shows), ER-C uses
gamma = 0.1 (Sec. V), and the reference is ER at h = 0.03125 ps.  Errors are the largest
node error at the end of the window, in volts."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path[:0] = [os.path.dirname(HERE), HERE]

from oracle import ers_oracle as O  # noqa: E402
from test_oracle_pins import _fixed_er, _shifted, _switching_window  # noqa: E402


def benr(circ, x0, t0, t1, h):
    x = x0.copy()
    for k in range(int(round((t1 - t0) / h))):
        x = O.be_run(_shifted(circ, t0 + k * h), h, t_end=h, x0=x)
    return x


def study(hs=(2e-12, 1e-12, 0.5e-12)):
    circ, x0, t0, t1 = _switching_window()
    ref = _fixed_er(circ, x0, t0, t1, 0.03125e-12)
    rows = []
    for h in hs:
        er = np.max(np.abs(_fixed_er(circ, x0, t0, t1, h) - ref))
        erc = np.max(np.abs(_fixed_er(circ, x0, t0, t1, h, correction=True) - ref))
        be = np.max(np.abs(benr(circ, x0, t0, t1, h) - ref))
        rows.append((h, er, erc, be))
    return rows


def trajectory(step, circ, x0, t0, t1, h, every):
    """States every `every` seconds through the window, by steps of h."""
    x = x0.copy()
    out = []
    k_per = int(round(every / h))
    for k in range(int(round((t1 - t0) / h))):
        x = step(circ, x, t0 + k * h, h)
        if (k + 1) % k_per == 0:
            out.append(x.copy())
    return np.array(out)


def er_step(circ, x, t, h, correction=False):
    opts = O.Options(correction=correction, eps=1e-12, m_max=circ.n)
    return O.er_step(circ, x, t, h, m=0, opts=opts).x


def be_step(circ, x, t, h):
    return O.be_run(_shifted(circ, t), h, t_end=h, x0=x)


def paper_setting():
    """The paper's Fig. 2 setting: BENR and ER at 1e-13 s, ER-C at 2e-13 s, against REF =
    BENR at 1e-14 s (and, beside it, ER at 1e-14 s), on the inverter output (MOSFET drain)
    that swings most in the window; errors are the largest difference over the common 0.2 ps grid."""
    circ, x0, t0, t1 = _switching_window()
    grid = 0.2e-12
    ref_be = trajectory(be_step, circ, x0, t0, t1, 0.01e-12, grid)
    ref_er = trajectory(er_step, circ, x0, t0, t1, 0.01e-12, grid)
    drains = np.unique(circ.dev["d"][circ.dev["d"] >= 0])
    node = int(drains[np.argmax(np.ptp(ref_er[:, drains], axis=0))])
    runs = {"BENR 0.1 ps": trajectory(be_step, circ, x0, t0, t1, 0.1e-12, grid),
            "ER 0.1 ps": trajectory(er_step, circ, x0, t0, t1, 0.1e-12, grid),
            "ER 0.2 ps": trajectory(er_step, circ, x0, t0, t1, 0.2e-12, grid),
            "ER-C 0.2 ps": trajectory(lambda c, x, t, h: er_step(c, x, t, h, True),
                                      circ, x0, t0, t1, 0.2e-12, grid)}
    return node, {k: (float(np.max(np.abs(v[:, node] - ref_be[:, node]))),
                      float(np.max(np.abs(v[:, node] - ref_er[:, node]))))
                  for k, v in runs.items()}


if __name__ == "__main__":
    print("h (ps)   ER        ER-C      BENR      (end of window, all nodes, vs ER at 0.03125 ps)")
    for h, er, erc, be in study():
        print(f"{h * 1e12:6.3f}  {er:.2e}  {erc:.2e}  {be:.2e}")
    node, errs = paper_setting()
    print(f"paper's setting, node {node}: max error vs REF = BENR 0.01 ps | vs ER 0.01 ps")
    for k, (a, b) in errs.items():
        print(f"  {k:12s} {a:.2e} | {b:.2e}")
