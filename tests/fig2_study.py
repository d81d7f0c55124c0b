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


if __name__ == "__main__":
    print("h (ps)   ER        ER-C      BENR")
    for h, er, erc, be in study():
        print(f"{h * 1e12:6.3f}  {er:.2e}  {erc:.2e}  {be:.2e}")
