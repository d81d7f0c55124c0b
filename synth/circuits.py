"""Seeded synthetic circuits for the exponential Rosenbrock-Euler transient.

This module only builds netlist data (sparse matrices of the linear elements, MOSFET
records, piecewise-linear source waveforms).  It contains none of the integrator's
arithmetic and is shared by the CPU oracle, the CUDA library's tests and the bench.

The circuit model is the one of the paper's problem statement (Sec. II, Eq. 1 and the
linearised form of Sec. III):  C x' + G_lin x + i_dev(x) = B u(t), with
  * x  : node voltages (grounded-capacitor RC networks, so every unknown is a node voltage),
  * C  : linear capacitance matrix (diagonal here: ground caps),
  * G_lin : linear conductance matrix (resistors, pads, gmin on every node),
  * i_dev : square-law MOSFET drain currents (nonlinear part),
  * B u(t): piecewise-linear current sources.
The paper's own circuits (BSIM3 netlists ckt1-ckt8, FreeCPU SPEF) are not available;
these seeded generators stand in for them with the sizes of the paper's workloads.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np
import scipy.sparse as sp

GROUND = -1  # device terminal tied to ground (0 V)
VDD = -2     # device terminal tied to the supply rail (vdd volts)
NMOS = 0
PMOS = 1

DEVICE_DTYPE = np.dtype([
    ("type", np.int32), ("d", np.int32), ("g", np.int32), ("s", np.int32),
    ("vt", np.float64), ("k", np.float64), ("lam", np.float64),
])


@dataclass
class Circuit:
    """One circuit instance.  All matrices are CSR with sorted, unique column indices."""
    name: str
    n: int
    G: sp.csr_matrix            # n x n linear conductances (S)
    C: sp.csr_matrix            # n x n capacitances (F)
    B: sp.csr_matrix            # n x p source incidence
    dev: np.ndarray             # structured array, DEVICE_DTYPE
    pwl: List[Tuple[np.ndarray, np.ndarray]]  # per source: (times s, values A)
    vdd: float = 1.0
    t_end: float = 1e-9
    meta: dict = field(default_factory=dict)
    # starting point for the DC operating point when the netlist knows one (a "nodeset": the
    # logic levels of a gate chain); None = start from 0 V
    nodeset: Optional[np.ndarray] = None

    @property
    def p(self) -> int:
        return self.B.shape[1]

    def breakpoints(self) -> np.ndarray:
        """Sorted unique corner times of all PWL waveforms (steps never straddle one)."""
        if not self.pwl:
            return np.zeros(0)
        return np.unique(np.concatenate([t for t, _ in self.pwl]))

    def u(self, t: float) -> np.ndarray:
        """Source values at time t (linear interpolation, constant outside the table)."""
        return np.array([np.interp(t, tt, vv) for tt, vv in self.pwl], dtype=np.float64)


def _csr(rows, cols, vals, n, m) -> sp.csr_matrix:
    a = sp.coo_matrix((np.asarray(vals, np.float64), (np.asarray(rows), np.asarray(cols))),
                      shape=(n, m)).tocsr()
    a.sum_duplicates()
    a.sort_indices()
    return a


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def _resistor_stamps(a, b, g):
    """Triplets of the conductance stamp of resistors between node arrays a and b."""
    rows = np.concatenate([a, b, a, b])
    cols = np.concatenate([a, b, b, a])
    vals = np.concatenate([g, g, -g, -g])
    return rows, cols, vals


def pulse_pwl(delay, rise, width, fall, amp, t_end):
    """Single trapezoidal pulse 0 -> amp -> 0 as a PWL table that covers [0, t_end]."""
    t = [0.0, delay, delay + rise, delay + rise + width, delay + rise + width + fall]
    v = [0.0, 0.0, amp, amp, 0.0]
    tt, vv = [], []
    for ti, vi in zip(t, v):
        if tt and ti <= tt[-1]:
            if ti == tt[-1]:
                vv[-1] = vi  # delay == 0: the first corner coincides with t=0
            continue
        tt.append(ti)
        vv.append(vi)
    if tt[-1] < t_end:
        tt.append(t_end)
        vv.append(vv[-1])
    return np.array(tt), np.array(vv)


def rc_mesh_2d(nx=32, ny=32, seed=0, n_src=16, gmin=1e-12, t_end=1e-9):
    """Linear 2D RC mesh: 4-neighbour conductances log-uniform 1-10 mS, ground caps
    log-uniform 1-100 fF, four corner pads of 1 S, gmin on every node, and n_src pulse
    current sources (0 -> 1 mA, 10 ps rise/fall, 100 ps width, delay on a 1 ps grid
    in [0, 0.89 ns]) injected at distinct random nodes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    a = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    b = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    g = _log_uniform(rng, 1e-3, 1e-2, a.size)
    r, c, v = _resistor_stamps(a, b, g)
    corners = np.array([idx[0, 0], idx[0, -1], idx[-1, 0], idx[-1, -1]])
    r = np.concatenate([r, corners, np.arange(n)])
    c = np.concatenate([c, corners, np.arange(n)])
    v = np.concatenate([v, np.ones(4), np.full(n, gmin)])
    G = _csr(r, c, v, n, n)
    cap = _log_uniform(rng, 1e-15, 1e-13, n)
    C = _csr(np.arange(n), np.arange(n), cap, n, n)
    nodes = rng.choice(n, size=n_src, replace=False)
    delays = rng.integers(0, 891, size=n_src) * 1e-12
    B = _csr(nodes, np.arange(n_src), np.ones(n_src), n, n_src)
    pwl = [pulse_pwl(d, 10e-12, 100e-12, 10e-12, 1e-3, t_end) for d in delays]
    return Circuit(name=f"rc2d_{nx}x{ny}", n=n, G=G, C=C, B=B,
                   dev=np.zeros(0, DEVICE_DTYPE), pwl=pwl, t_end=t_end,
                   meta=dict(kind="rc2d", nx=nx, ny=ny, seed=seed, h=1e-12, m=20))


def coupled_rc_mesh_2d(nx=32, ny=32, seed=0, n_src=16, t_end=1e-9, cc_lo=1e-15, cc_hi=1e-14):
    """rc_mesh_2d plus a coupling capacitor (log-uniform cc_lo..cc_hi) across every diagonal
    neighbour pair (i, j)-(i+1, j+1): C is no longer diagonal (nnz_C close to nnz_G, as in
    circuits with complex coupling capacitance) and stays symmetric positive definite."""
    base = rc_mesh_2d(nx, ny, seed=seed, n_src=n_src, t_end=t_end)
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    a = idx[:-1, :-1].ravel()
    b = idx[1:, 1:].ravel()
    cc = _log_uniform(rng, cc_lo, cc_hi, a.size)
    r, c, v = _resistor_stamps(a, b, cc)       # same stamp pattern as a conductance
    C = (base.C + _csr(r, c, v, n, n)).tocsr()
    C.sort_indices()
    return Circuit(name=f"rc2dcc_{nx}x{ny}", n=n, G=base.G, C=C, B=base.B, dev=base.dev,
                   pwl=base.pwl, t_end=t_end,
                   meta=dict(kind="rc2dcc", nx=nx, ny=ny, seed=seed))


def rc_mesh_3d(nx=100, ny=100, nz=100, seed=1, n_loads=10000, pad_pitch=10,
               gmin=1e-12, t_end=2e-9, delay_grid=10e-12, n_delay=189):
    """Linear 3D RC power-grid mesh: 6-neighbour conductances log-uniform 0.1-10 S,
    ground caps log-uniform 1 fF-1 pF, pads of 10 S on the top layer every
    pad_pitch nodes in x and y, gmin on every node, and n_loads pulse loads
    (0 -> 1 mA drawn, 10 ps rise/fall, 100 ps width, delay on a 10 ps grid)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    a = np.concatenate([idx[:, :, :-1].ravel(), idx[:, :-1, :].ravel(), idx[:-1, :, :].ravel()])
    b = np.concatenate([idx[:, :, 1:].ravel(), idx[:, 1:, :].ravel(), idx[1:, :, :].ravel()])
    g = _log_uniform(rng, 0.1, 10.0, a.size)
    r, c, v = _resistor_stamps(a, b, g)
    pads = idx[nz - 1, ::pad_pitch, ::pad_pitch].ravel()
    r = np.concatenate([r, pads, np.arange(n)])
    c = np.concatenate([c, pads, np.arange(n)])
    v = np.concatenate([v, np.full(pads.size, 10.0), np.full(n, gmin)])
    G = _csr(r, c, v, n, n)
    cap = _log_uniform(rng, 1e-15, 1e-12, n)
    C = _csr(np.arange(n), np.arange(n), cap, n, n)
    n_loads = min(n_loads, n)
    nodes = rng.choice(n, size=n_loads, replace=False)
    delays = rng.integers(0, n_delay, size=n_loads) * delay_grid
    B = _csr(nodes, np.arange(n_loads), -np.ones(n_loads), n, n_loads)
    pwl = [pulse_pwl(d, 10e-12, 100e-12, 10e-12, 1e-3, t_end) for d in delays]
    return Circuit(name=f"rc3d_{nx}x{ny}x{nz}", n=n, G=G, C=C, B=B,
                   dev=np.zeros(0, DEVICE_DTYPE), pwl=pwl, t_end=t_end,
                   meta=dict(kind="rc3d", nx=nx, ny=ny, nz=nz, seed=seed))


def _random_recursive_tree(rng, size):
    """Parent array of a random recursive tree: parent of node i is uniform in 0..i-1."""
    par = np.full(size, -1, np.int64)
    if size > 1:
        par[1:] = np.floor(rng.random(size - 1) * np.arange(1, size)).astype(np.int64)
    return par


def inverter_chain(stages=2000, tree_nodes=100, seed=2, vdd=1.0, gmin=1e-12,
                   t_end=5e-9, period=1e-9, sigma=0.0, lam=0.1):
    """Nonlinear inverter chain with RC parasitic trees.

    Node 0 is the chain input, driven by a Norton source (1 mS to ground in parallel
    with a PWL current 0 -> 1 mA, 10 ps edges, 1 ns period).  Stage i has an NMOS
    (source at ground) and a PMOS (source at vdd) whose drains form the root of a random
    recursive tree of tree_nodes nodes (resistors log-uniform 10-100 ohm, ground caps
    log-uniform 0.01-0.1 fF); stage i+1's gate is a random leaf of that tree and gets
    an extra 0.5 fF gate cap.  Threshold voltages are uniform 0.3-0.4 V and
    transconductance factors uniform 50-200 uA/V^2 per device, with channel-length
    modulation lam (1/V) so that a saturated device keeps a finite output conductance.
    sigma > 0 applies an
    independent log-normal perturbation (Monte Carlo corner) to vt, k, R and C.
    """
    rng = np.random.Generator(np.random.PCG64(seed))

    def mc(x):
        if sigma <= 0:
            return x
        return x * np.exp(rng.normal(0.0, sigma, np.shape(x)))

    n = 1 + stages * tree_nodes
    # nodeset: logic levels with the input low (u(0) = 0): stage outputs alternate vdd, 0, ...
    # and every node of a stage's tree sits at its output level (no DC current in the trees)
    nodeset = np.zeros(n)
    for st in range(stages):
        nodeset[1 + st * tree_nodes:1 + (st + 1) * tree_nodes] = vdd if st % 2 == 0 else 0.0
    rows, cols, vals = [], [], []
    caps = np.zeros(n)
    dev = np.zeros(2 * stages, DEVICE_DTYPE)
    gate = 0
    # input Norton conductance
    rows.append(np.array([0])); cols.append(np.array([0])); vals.append(np.array([1e-3]))
    caps[0] = 0.5e-15
    for st in range(stages):
        base = 1 + st * tree_nodes
        par = _random_recursive_tree(rng, tree_nodes)
        child = np.arange(1, tree_nodes)
        gres = 1.0 / mc(_log_uniform(rng, 10.0, 100.0, tree_nodes - 1))
        r, c, v = _resistor_stamps(base + child, base + par[1:], gres)
        rows.append(r); cols.append(c); vals.append(v)
        caps[base:base + tree_nodes] += mc(_log_uniform(rng, 0.01e-15, 0.1e-15, tree_nodes))
        out = base
        vt = mc(rng.uniform(0.3, 0.4, 2))
        kk = mc(rng.uniform(50e-6, 200e-6, 2))
        dev[2 * st] = (NMOS, out, gate, GROUND, vt[0], kk[0], lam)
        dev[2 * st + 1] = (PMOS, out, gate, VDD, vt[1], kk[1], lam)
        is_leaf = np.ones(tree_nodes, bool)
        is_leaf[par[1:]] = False
        leaves = np.nonzero(is_leaf)[0]
        gate = base + int(leaves[rng.integers(0, leaves.size)])
        caps[gate] += 0.5e-15
    rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(np.full(n, gmin))
    G = _csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n, n)
    C = _csr(np.arange(n), np.arange(n), caps, n, n)
    B = _csr(np.array([0]), np.array([0]), np.array([1.0]), n, 1)
    # periodic pulse train: rise at 0.1 ns + k*period, high for half a period
    tt, vv = [0.0], [0.0]
    k = 0
    while True:
        t0 = 0.1e-9 + k * period
        if t0 >= t_end:
            break
        for ti, vi in ((t0, 0.0), (t0 + 10e-12, 1e-3),
                       (t0 + 0.5 * period, 1e-3), (t0 + 0.5 * period + 10e-12, 0.0)):
            if ti <= t_end and ti > tt[-1]:
                tt.append(ti); vv.append(vi)
        k += 1
    if tt[-1] < t_end:
        tt.append(t_end); vv.append(vv[-1])
    pwl = [(np.array(tt), np.array(vv))]
    return Circuit(name=f"invchain_{stages}x{tree_nodes}", n=n, G=G, C=C, B=B, dev=dev,
                   pwl=pwl, vdd=vdd, t_end=t_end, nodeset=nodeset,
                   meta=dict(kind="invchain", stages=stages, tree_nodes=tree_nodes, seed=seed))


def random_rc(n=16, seed=0, density=0.3, p=2, t_end=50e-12, n_alg=0, alg_source=False):
    """Small dense-ish random RC network (every node has a path to ground), used to pin the
    oracle against a dense matrix exponential.  Every node has a ground cap unless n_alg > 0:
    then n_alg nodes (one of them a source node when alg_source) have no capacitance at all,
    which makes C singular (algebraic nodes of a differential-algebraic system)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rows, cols, vals = [], [], []
    # spanning chain keeps the network connected, extra random edges add coupling
    a = list(range(n - 1)); b = list(range(1, n))
    for i in range(n):
        for j in range(i + 2, n):
            if rng.random() < density:
                a.append(i); b.append(j)
    a = np.array(a); b = np.array(b)
    g = _log_uniform(rng, 1e-3, 1e-2, a.size)
    r, c, v = _resistor_stamps(a, b, g)
    ground = _log_uniform(rng, 1e-4, 1e-3, n)
    r = np.concatenate([r, np.arange(n)]); c = np.concatenate([c, np.arange(n)])
    v = np.concatenate([v, ground])
    G = _csr(r, c, v, n, n)
    C = _csr(np.arange(n), np.arange(n), _log_uniform(rng, 1e-15, 1e-14, n), n, n)
    nodes = rng.choice(n, size=p, replace=False)
    B = _csr(nodes, np.arange(p), np.ones(p), n, p)
    pwl = [pulse_pwl(float(rng.integers(0, 5)) * 1e-12, 5e-12, 10e-12, 5e-12, 1e-3, t_end)
           for _ in range(p)]
    alg = np.zeros(0, np.int64)
    if n_alg:
        arng = np.random.Generator(np.random.PCG64(seed + 104729))
        pool = np.setdiff1d(np.arange(n), nodes)
        alg = arng.choice(pool, size=n_alg - int(alg_source), replace=False)
        if alg_source:
            alg = np.concatenate([alg, nodes[:1]])
        alg = np.sort(alg)
        keep = np.setdiff1d(np.arange(n), alg)
        C = _csr(keep, keep, C.diagonal()[keep], n, n)
    return Circuit(name=f"randrc_{n}", n=n, G=G, C=C, B=B, dev=np.zeros(0, DEVICE_DTYPE),
                   pwl=pwl, t_end=t_end, meta=dict(kind="randrc", seed=seed, algebraic=alg))


def single_rc(g=1e-3, c=1e-15, i_amp=1e-3, ramp=None, t_end=10e-12):
    """One node with conductance g and capacitance c to ground, driven by a current step
    of amplitude i_amp at t=0 (ramp=None) or a linear ramp of slope ramp A/s."""
    G = _csr([0], [0], [g], 1, 1)
    C = _csr([0], [0], [c], 1, 1)
    B = _csr([0], [0], [1.0], 1, 1)
    if ramp is None:
        pwl = [(np.array([0.0, t_end]), np.array([i_amp, i_amp]))]
    else:
        pwl = [(np.array([0.0, t_end]), np.array([0.0, ramp * t_end]))]
    return Circuit(name="single_rc", n=1, G=G, C=C, B=B, dev=np.zeros(0, DEVICE_DTYPE),
                   pwl=pwl, t_end=t_end, meta=dict(kind="single_rc"))


def batch_family(n_inst=256, seed0=1000, stage_lo=20, stage_hi=2000, sigma=0.05, t_end=5e-9,
                 tree_nodes=100):
    """Monte Carlo batch of inverter chains with uneven stage counts."""
    rng = np.random.Generator(np.random.PCG64(seed0))
    stages = rng.integers(stage_lo, stage_hi + 1, size=n_inst)
    return [inverter_chain(int(s), tree_nodes=tree_nodes, seed=seed0 + i, sigma=sigma,
                           t_end=t_end) for i, s in enumerate(stages)]
