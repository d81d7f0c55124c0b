"""CPU FP64 oracle for the exponential Rosenbrock-Euler (ER) circuit transient with the
invert-Krylov matrix-exponential-vector product (MEVP).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously-correct statement of
what the CUDA library computes; it is imported only by tests/, by
__graft_entry__.smoke() and by bench.py's CPU-baseline / reference leg.  It shares no
code with the CUDA path (no kernels, tables or helpers); the only thing both sides use is
the seeded netlist generator in synth/, which holds none of the method's arithmetic.

Paper: Zhuang, Yu, Kang, Wang, Cheng, "An Algorithmic Framework for Efficient Large-Scale
Circuit Simulation Using Exponential Integrators", DAC 2015 (arXiv 1511.04515).

Each function cites the passage it follows.  The oracle's own pieces: the sparse LU of G_k
(oracle/olu.c via oracle/sparse_lu.py: minimum-degree ordering, left-looking LU with
threshold partial pivoting), the dense exponential of h H_m^{-1} (scaling and squaring of the
[13/13] Pade approximant, Higham 2005; the paper's "scaling and squaring" step) and a dense LU
with partial pivoting for H_m^{-1} and the Pade denominator.  The singular-C branch uses scipy's ordered Schur form and
Sylvester solver as single library steps.  The remaining arithmetic is written out in the
paper's order and notation.

Readings of points the paper leaves open:
  * F(x) is the Rosenbrock remainder with the device Jacobian frozen at x_k:
    F(x) = G_dev,k x - i_dev(x), so that -G_k x + F(x) = -G_lin x - i_dev(x).
  * Dq/dt = C x' with a constant linear C (grounded capacitors).
  * The phi_1 and phi_2 terms use two Krylov spaces (Alg. 2 "respectively"); an option
    combines them into one space on v1 + v2 (equal in exact arithmetic).
  * Krylov stopping test (Eq. 16, e^T read as e_m^T): ||r_m(h)||_2 <= eps * ||G v||_2.
  * Happy breakdown: h_{j+1,j} <= 1e-12 * ||w|| (w = J^{-1} v_j before orthogonalisation)
    ends Arnoldi at j; if exp(h H_j^{-1}) e_1 is then not finite, v_j was rounding noise
    and the MEVP uses j - 1.  A residual that is not finite (a spurious Ritz value of J^{-1} in the
    right half-plane makes exp(h H^{-1}) overflow) counts as "not converged".
  * E_rr = tol * max(1 V, ||x_k||_inf); steps never straddle a PWL corner.
  * Singular C (nodes without capacitance, Sec. IV-A and Sec. V): e^{h/mu} and e^{h/mu}/mu
    are taken at their limit 0 for the eigenvalue mu = 0 of H_m and for any |mu| <= h/700
    (exp_hinv_e1); circuits whose C has no zero row keep the plain exponential.  For a linear index-1 circuit this makes the ER step the exact solution
    of the differential-algebraic system.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle.sparse_lu import SparseLU

GROUND = -1
VDD = -2
BREAKDOWN_TOL = 1e-12


# ----------------------------------------------------------------------------------------
# Device model (stand-in for BSIM3, Sec. V): symmetric square-law MOSFET.
# ----------------------------------------------------------------------------------------
def _nmos_forward(vgs, vds, vt, k, lam):
    """Square-law drain current and its partials for vds >= 0.
    Returns (I, dI/dVgs, dI/dVds)."""
    vov = vgs - vt
    if vov <= 0.0:
        return 0.0, 0.0, 0.0
    clm = 1.0 + lam * vds
    if vds < vov:  # triode
        core = vov * vds - 0.5 * vds * vds
        return k * core * clm, k * vds * clm, k * (vov - vds) * clm + k * core * lam
    core = 0.5 * vov * vov  # saturation
    return k * core * clm, k * vov * clm, k * core * lam


def mosfet_eval(dtype, vd, vg, vs, vt, k, lam):
    """Current flowing from the drain terminal to the source terminal through the device,
    and its partial derivatives with respect to (vd, vg, vs).  Source and drain swap
    roles when vds < 0; a PMOS is the NMOS equation on negated terminal voltages."""
    sgn = 1.0
    if dtype == 1:  # PMOS: I_p(vd,vg,vs) = -I_n(-vd,-vg,-vs); partials keep their values
        vd, vg, vs = -vd, -vg, -vs
        sgn = -1.0
    if vd >= vs:
        i, gm, gds = _nmos_forward(vg - vs, vd - vs, vt, k, lam)
        i_ds, d_vd, d_vg, d_vs = i, gds, gm, -gm - gds
    else:  # reversed: the physical source is the d terminal
        i, gm, gds = _nmos_forward(vg - vd, vs - vd, vt, k, lam)
        i_ds, d_vd, d_vg, d_vs = -i, gm + gds, -gm, -gds
    return sgn * i_ds, d_vd, d_vg, d_vs


def _term_voltage(node, x, vdd):
    if node == GROUND:
        return 0.0
    if node == VDD:
        return vdd
    return x[node]


def device_eval(circ, x):
    """i_dev(x) (KCL currents leaving each node into the devices) and the device Jacobian
    G_dev(x) = d i_dev / dx (Alg. 2: 'derive C_k, G_k, F_k from device models at x_k')."""
    n = circ.n
    idev = np.zeros(n)
    rows, cols, vals = [], [], []
    for d in circ.dev:
        dn, gn, sn = int(d["d"]), int(d["g"]), int(d["s"])
        vd = _term_voltage(dn, x, circ.vdd)
        vg = _term_voltage(gn, x, circ.vdd)
        vs = _term_voltage(sn, x, circ.vdd)
        i_ds, d_vd, d_vg, d_vs = mosfet_eval(int(d["type"]), vd, vg, vs,
                                             float(d["vt"]), float(d["k"]), float(d["lam"]))
        for node, sign in ((dn, 1.0), (sn, -1.0)):
            if node < 0:
                continue
            idev[node] += sign * i_ds
            for term, der in ((dn, d_vd), (gn, d_vg), (sn, d_vs)):
                if term >= 0:
                    rows.append(node); cols.append(term); vals.append(sign * der)
    Gdev = sp.csr_matrix((vals, (rows, cols)), shape=(n, n)) if rows else sp.csr_matrix((n, n))
    return idev, Gdev


@dataclass
class Linearization:
    """Quantities fixed for one time step at x_k (Sec. III, Eq. 11-12)."""
    x: np.ndarray
    Gdev: sp.csr_matrix
    Gk: sp.csr_matrix
    F: np.ndarray
    lu: object

    def solve(self, b):
        """G_k^{-1} b by the sparse LU of G_k (Alg. 2, LU_decompose(G_k))."""
        return self.lu.solve(b)

    def remainder(self, circ, y):
        """F(y) with the device Jacobian frozen at x_k: G_dev,k y - i_dev(y)."""
        if circ.dev.size == 0:
            return np.zeros(circ.n)
        idev, _ = device_eval(circ, y)
        return self.Gdev @ y - idev


def linearize(circ, x) -> Linearization:
    """Device evaluation + stamping at x_k, then one LU of G_k only (never of C or C/h+G)."""
    if circ.dev.size:
        idev, Gdev = device_eval(circ, x)
    else:
        idev, Gdev = np.zeros(circ.n), sp.csr_matrix((circ.n, circ.n))
    Gk = (circ.G + Gdev).tocsc()
    F = Gdev @ x - idev
    lu = SparseLU(Gk)
    return Linearization(x=x.copy(), Gdev=Gdev, Gk=Gk.tocsr(), F=F, lu=lu)


# ----------------------------------------------------------------------------------------
# Small dense matrix functions (Sec. IV, Eq. 14 and the residual of Eq. 16).
# ----------------------------------------------------------------------------------------
def dense_lu_solve(A, B):
    """X = A^{-1} B by Gaussian elimination with partial pivoting (row interchanges to the
    largest remaining entry of each column).  A: m x m, B: m x k; real or complex."""
    A = np.array(A, dtype=np.result_type(A, B, np.float64))
    X = np.array(B, dtype=A.dtype).reshape(A.shape[0], -1)
    m = A.shape[0]
    for k in range(m):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if A[p, k] == 0:
            raise ZeroDivisionError("singular matrix")
        if p != k:
            A[[k, p]] = A[[p, k]]
            X[[k, p]] = X[[p, k]]
        f = A[k + 1:, k] / A[k, k]
        A[k + 1:, k:] -= np.outer(f, A[k, k:])
        X[k + 1:] -= np.outer(f, X[k])
    for k in range(m - 1, -1, -1):
        X[k] = (X[k] - A[k, k + 1:] @ X[k + 1:]) / A[k, k]
    return X.reshape(np.shape(B))


def _pade_coefficients(q):
    """c_j = (2q - j)! q! / ((2q)! j! (q - j)!), the numerator of the [q/q] Pade approximant
    of e^z (the denominator is the same polynomial at -z)."""
    return [math.factorial(2 * q - j) * math.factorial(q) /
            (math.factorial(2 * q) * math.factorial(j) * math.factorial(q - j))
            for j in range(q + 1)]


PADE13 = _pade_coefficients(13)
THETA13 = 5.371920351148152   # largest ||A||_1 with [13/13] backward error <= 2^-53 (Higham 2005)


def expm_pade13(A):
    """e^A by scaling and squaring of the diagonal [13/13] Pade approximant (N. J. Higham,
    "The scaling and squaring method for the matrix exponential revisited", SIAM J. Matrix
    Anal. Appl. 26, 2005): s = max(0, ceil(log2(||A||_1 / theta_13))), X = A / 2^s,
    U = X [X6 (c13 X6 + c11 X4 + c9 X2) + c7 X6 + c5 X4 + c3 X2 + c1 I],
    V = X6 (c12 X6 + c10 X4 + c8 X2) + c6 X6 + c4 X4 + c2 X2 + c0 I,
    e^X ~ (V - U)^-1 (V + U), then squared s times."""
    A = np.asarray(A)
    m = A.shape[0]
    dt = np.result_type(A, np.float64)
    if m == 0:
        return np.zeros((0, 0), dtype=dt)
    nrm = float(np.max(np.sum(np.abs(A), axis=0)))
    if not np.isfinite(nrm):
        return np.full(A.shape, np.nan, dtype=dt)
    s = max(0, int(np.ceil(np.log2(nrm / THETA13)))) if nrm > THETA13 else 0
    s = min(s, 1000)
    X = np.ldexp(A.real, -s) + 1j * np.ldexp(A.imag, -s) if np.iscomplexobj(A) \
        else np.ldexp(A, -s)
    c = PADE13
    I = np.eye(m, dtype=dt)
    X2 = X @ X
    X4 = X2 @ X2
    X6 = X4 @ X2
    U = X @ (X6 @ (c[13] * X6 + c[11] * X4 + c[9] * X2) + c[7] * X6 + c[5] * X4
             + c[3] * X2 + c[1] * I)
    V = X6 @ (c[12] * X6 + c[10] * X4 + c[8] * X2) + c[6] * X6 + c[4] * X4 + c[2] * X2 \
        + c[0] * I
    E = dense_lu_solve(V - U, V + U)
    for _ in range(s):
        E = E @ E
    return E


ALGEBRAIC_EXPONENT = 700.0   # e^{-700} ~ 1e-304: below it e^{h/mu} is zero in FP64


def exp_hinv_e1(Hm, h, singular_c=False):
    """exp(h H_m^{-1}) e_1 and e_m^T H_m^{-1} exp(h H_m^{-1}) e_1 (Eq. 14 and Eq. 16).

    Both are functions of H_m: f(mu) = e^{h/mu} and g(mu) = e^{h/mu} / mu; for a C without
    zero rows they are the plain dense exponential of h H_m^{-1}.  The paper keeps C out of
    every factorisation so that a singular C needs no regularisation (Sec. IV-A); with
    singular_c (C has nodes without capacitance) J^{-1} = -G^{-1} C has the eigenvalue 0 on
    ker C, and f, g are taken at their limit 0 from the stable side (such modes relax
    instantly).  The same limit is used for every eigenvalue with |mu| <= h / 700: a real
    stiff mode there has e^{h/mu} below 1e-304 anyway, and a tiny eigenvalue of either sign is
    the rounding image of a zero one.  Those eigenvalues are split off by an ordered Schur
    form H = Z T Z^*, where f(T) = [[f(T11), F12], [0, 0]] and F12 solves
    T11 F12 - F12 T22 = f(T11) T12 (from T f(T) = f(T) T); same for g."""
    m = Hm.shape[0]
    tau = h / ALGEBRAIC_EXPONENT
    if not singular_c or np.all(np.abs(np.linalg.eigvals(Hm)) > tau):
        Hinv = dense_lu_solve(Hm, np.eye(m))
        with np.errstate(over="ignore", invalid="ignore"):
            E = expm_pade13(h * Hinv)
        y = E[:, 0].copy()
        return y, float((Hinv @ y)[m - 1])
    T, Z, s = sla.schur(Hm.astype(complex), output="complex", sort=lambda mu: abs(mu) > tau)
    if s == 0:
        return np.zeros(m), 0.0
    T11, T12, T22 = T[:s, :s], T[:s, s:], T[s:, s:]
    T11inv = dense_lu_solve(T11, np.eye(s, dtype=complex))
    fT = np.zeros((m, m), complex)
    gT = np.zeros((m, m), complex)
    fT[:s, :s] = expm_pade13(h * T11inv)
    gT[:s, :s] = T11inv @ fT[:s, :s]
    fT[:s, s:] = sla.solve_sylvester(T11, -T22, fT[:s, :s] @ T12)
    gT[:s, s:] = sla.solve_sylvester(T11, -T22, gT[:s, :s] @ T12)
    z1 = Z.conj().T[:, 0]                       # Z^* e_1
    y = (Z @ (fT @ z1)).real
    return y, float((Z @ (gT @ z1))[m - 1].real)


def has_capacitor_free_node(C):
    """True when some node has no capacitance at all (a zero row of C), i.e. the circuit is
    differential-algebraic and J^{-1} = -G^{-1} C has the eigenvalue 0."""
    return bool(np.any(abs(sp.csr_matrix(C)).sum(axis=1) == 0))


# ----------------------------------------------------------------------------------------
# MEVP_IKS (Algorithm 1).
# ----------------------------------------------------------------------------------------
@dataclass
class KrylovBasis:
    """Invert-Krylov basis K_m(J^{-1}, v) of Sec. IV-A with its Hessenberg matrix.
    It does not depend on h (time-step scaling invariance), so a rejected step reuses it."""
    beta: float
    V: np.ndarray                  # n x (j+1) orthonormal columns v_1..v_{j+1}
    H: np.ndarray                  # (j+1) x j upper Hessenberg
    m: int                         # dimension used for the MEVP
    built: int                     # number of Arnoldi iterations performed
    breakdown: bool = False
    gv_norm: float = 0.0           # ||G v_1||_2 (scale of the relative residual test)
    gvnext_norm: List[float] = field(default_factory=list)  # ||G v_{j+1}||_2 per j
    singular_c: bool = False       # C has nodes without capacitance (see exp_hinv_e1)

    def residual(self, j, h):
        """||r_j(h)||_2 / (beta ||G v_1||) from Eq. 16 with e^T = e_j^T."""
        if self.breakdown and j == self.built:
            return 0.0
        with np.errstate(all="ignore"):
            _, last = exp_hinv_e1(self.H[:j, :j], h, self.singular_c)
        return self.H[j, j - 1] * self.gvnext_norm[j - 1] * abs(last) / self.gv_norm

    def mevp(self, h, m=None):
        """m_evp = ||v|| V_m exp(h H_m^{-1}) e_1 (last line of Algorithm 1)."""
        m = self.m if m is None else m
        if self.beta == 0.0:
            return np.zeros(self.V.shape[0])
        y, _ = exp_hinv_e1(self.H[:m, :m], h, self.singular_c)
        return self.beta * (self.V[:, :m] @ y)


def arnoldi_iks(C, lin, G, v, h, eps, m_max, m_min=1, fixed_m=0):
    """Algorithm 1 (MEVP_IKS) up to the MEVP: Arnoldi on J^{-1} = -G^{-1} C with modified
    Gram-Schmidt.  With fixed_m > 0 exactly fixed_m iterations run (unless breakdown);
    otherwise iterations stop at the first j >= m_min whose residual (Eq. 16) at h is
    below eps, or at m_max (Algorithm 1's loop bound m_c).  When the test never passes,
    the MEVP uses the dimension with the smallest finite residual: the last directions of a
    long run can be rounding noise whose spurious Ritz values make exp(h H^{-1}) overflow.
    If no tested dimension had a finite residual, it uses the largest dimension whose
    exp(h H^{-1}) e_1 is finite."""
    n = v.shape[0]
    sing = has_capacitor_free_node(C)
    beta = float(np.linalg.norm(v))
    mc = fixed_m if fixed_m > 0 else m_max
    V = np.zeros((n, mc + 1))
    H = np.zeros((mc + 1, mc))
    if beta == 0.0:
        return KrylovBasis(beta=0.0, V=V[:, :1], H=H[:1, :0], m=0, built=0)
    V[:, 0] = v / beta
    basis = KrylovBasis(beta=beta, V=V, H=H, m=mc, built=0,
                        gv_norm=float(np.linalg.norm(G @ V[:, 0])), singular_c=sing)
    best_j, best_res = mc, np.inf
    for j in range(mc):
        w = -lin.solve(C @ V[:, j])                 # solve -G w = C v_j
        w0 = float(np.linalg.norm(w))
        for i in range(j + 1):                      # modified Gram-Schmidt
            H[i, j] = float(w @ V[:, i])
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = float(np.linalg.norm(w))
        basis.built = j + 1
        if H[j + 1, j] <= BREAKDOWN_TOL * w0:      # happy breakdown: K_j is invariant
            basis.breakdown = True
            basis.m = j + 1
            basis.gvnext_norm.append(0.0)
            with np.errstate(all="ignore"):
                y, _ = exp_hinv_e1(H[:j + 1, :j + 1], h, sing)
            if j > 0 and not np.all(np.isfinite(y)):
                # v_{j+1} was rounding noise (its Ritz value sits at ~+0): drop it
                basis.m = j
            break
        V[:, j + 1] = w / H[j + 1, j]
        basis.gvnext_norm.append(float(np.linalg.norm(G @ V[:, j + 1])))
        if fixed_m == 0 and j + 1 >= m_min:
            res = basis.residual(j + 1, h)
            if np.isfinite(res) and res < best_res:
                best_j, best_res = j + 1, res
            if res < eps:
                basis.m = j + 1
                break
    else:
        if fixed_m == 0:
            basis.m = best_j   # never converged: the dimension with the smallest residual
            if not np.isfinite(best_res):
                # no tested dimension had a finite residual: the largest dimension whose
                # exp(h H^{-1}) e_1 is finite
                with np.errstate(all="ignore"):
                    while basis.m > 1 and not np.all(np.isfinite(
                            exp_hinv_e1(H[:basis.m, :basis.m], h, sing)[0])):
                        basis.m -= 1
    basis.V = V[:, :basis.built + 1]
    basis.H = H[:basis.built + 1, :basis.built]
    return basis


# ----------------------------------------------------------------------------------------
# ER / ER-C step (Sec. III, Eq. 13; error Eq. 15/19; correction Eq. 20).
# ----------------------------------------------------------------------------------------
@dataclass
class Options:
    eps: float = 1e-7          # Krylov residual tolerance (Sec. V uses 1e-7)
    m_max: int = 40
    m_min: int = 3
    alpha: float = 0.5         # Alg. 2: h = alpha h on rejection
    beta: float = 2.0          # Alg. 2: h = beta h after a fast acceptance
    i_grow: int = 5            # Alg. 2: grow when the retry count i < i_grow
    gamma: float = 0.1         # ER-C correction weight
    correction: bool = False   # ER-C when True
    combined: bool = False     # one Krylov space on v1 + v2
    h_min: float = 1e-20
    h_max: float = 0.0         # 0: t_end / 100
    h_init: float = 0.0        # 0: h_max


@dataclass
class StepSetup:
    """Vectors of one step that do not depend on h within a PWL segment."""
    lin: Linearization
    uk: np.ndarray
    slope: np.ndarray
    v1: np.ndarray
    w1: np.ndarray
    v2: np.ndarray
    K1: KrylovBasis = None
    K2: KrylovBasis = None


def step_setup(circ, lin, t, slope):
    """v1 = J^{-1} g_k = x_k - G_k^{-1}(F_k + B u(t_k))   (Eq. 12 with the C^{-1} cancelled)
    w1 = G_k^{-1} B s,  v2 = J^{-2} b_k = G_k^{-1} C w1    (Eq. 13's h^2 phi_2 term, Eq. 12)
    where s is the PWL slope of u on the step."""
    uk = circ.u(t)
    v1 = lin.x - lin.solve(lin.F + circ.B @ uk)
    if np.any(slope != 0.0):
        w1 = lin.solve(circ.B @ slope)
        v2 = lin.solve(circ.C @ w1)
    else:
        w1 = np.zeros(circ.n)
        v2 = np.zeros(circ.n)
    return StepSetup(lin=lin, uk=uk, slope=slope, v1=v1, w1=w1, v2=v2)


def er_update(st: StepSetup, h, m1=None, m2=None):
    """x_{k+1}(h) = x_k + h phi_1(hJ) g_k + h^2 phi_2(hJ) b_k   (Eq. 13), in the form
    x_k + (e^{hJ} - I) v1 + (e^{hJ} - I) v2 + h w1."""
    x = st.lin.x + (st.K1.mevp(h, m1) - st.v1) + h * st.w1
    if st.K2 is not None:
        x = x + (st.K2.mevp(h, m2) - st.v2)
    return x


def error_vector(circ, st, x_new, h, C, opts, fixed_m=0):
    """e_rr = h phi_1(hJ) C^{-1} dF = -(e^{hJ} - I) G_k^{-1} dF with dF = F(x_{k+1}) - F_k
    (Eq. 15; computed through one more MEVP as in Eq. 19).  Returns (e_rr, v_e, K_e)."""
    dF = st.lin.remainder(circ, x_new) - st.lin.F
    if not np.any(dF):
        return np.zeros(circ.n), np.zeros(circ.n), None
    ve = st.lin.solve(dF)
    Ke = arnoldi_iks(C, st.lin, st.lin.Gk, ve, h, opts.eps, opts.m_max, opts.m_min, fixed_m)
    return ve - Ke.mevp(h), ve, Ke


def correction_term(circ, st, ve, h, C, opts, fixed_m=0):
    """ER-C: D = gamma h phi_2(hJ) C^{-1} dF = (gamma/h)[(e^{hJ}-I) G^{-1} C v_e + h v_e]
    (Eq. 17 and Eq. 20)."""
    if not np.any(ve):
        return np.zeros(circ.n)
    z = st.lin.solve(C @ ve)
    Kz = arnoldi_iks(C, st.lin, st.lin.Gk, z, h, opts.eps, opts.m_max, opts.m_min, fixed_m)
    return (opts.gamma / h) * ((Kz.mevp(h) - z) + h * ve)


def pwl_slope(circ, t, h):
    return (circ.u(t + h) - circ.u(t)) / h


@dataclass
class StepResult:
    x: np.ndarray
    err_inf: float
    m1: int
    m2: int
    me: int


def er_step(circ, x, t, h, m=20, opts: Options = None, lin: Linearization = None):
    """One ER (or ER-C) step of exactly h from (t, x) with a fixed Krylov dimension m
    (m = 0: adaptive by the Eq.-16 residual at h).  The step must not cross a PWL corner."""
    opts = opts or Options()
    lin = lin or linearize(circ, x)
    st = step_setup(circ, lin, t, pwl_slope(circ, t, h))
    C = circ.C
    if opts.combined:
        st.v1 = st.v1 + st.v2
        st.v2 = np.zeros(circ.n)
    st.K1 = arnoldi_iks(C, lin, lin.Gk, st.v1, h, opts.eps, opts.m_max, opts.m_min, m)
    st.K2 = arnoldi_iks(C, lin, lin.Gk, st.v2, h, opts.eps, opts.m_max, opts.m_min, m) \
        if np.any(st.v2) else None
    x_new = er_update(st, h)
    err = 0.0
    me = 0
    if circ.dev.size:
        e, ve, Ke = error_vector(circ, st, x_new, h, C, opts, m)
        err = float(np.max(np.abs(e)))
        me = Ke.m if Ke is not None else 0
        if opts.correction:
            x_new = x_new - correction_term(circ, st, ve, h, C, opts, m)
    return StepResult(x=x_new, err_inf=err, m1=st.K1.m,
                      m2=st.K2.m if st.K2 is not None else 0, me=me)


# ----------------------------------------------------------------------------------------
# DC operating point and the transient loop (Algorithm 2).
# ----------------------------------------------------------------------------------------
def dc_solution(circ, x0=None, max_iter=50, vstep=0.5, tol=1e-12):
    """x(0) = DC solution: Newton on G_lin x + i_dev(x) = B u(0).  A Newton update is
    x <- G_k^{-1}(F(x) + B u(0)), i.e. the same G_k solve as v1 of the ER step."""
    x = np.zeros(circ.n) if x0 is None else np.array(x0, dtype=np.float64)
    bu = circ.B @ circ.u(0.0)
    for _ in range(max_iter):
        lin = linearize(circ, x)
        idev = lin.Gdev @ x - lin.F
        res = circ.G @ x + idev - bu
        if np.max(np.abs(res), initial=0.0) <= tol:
            return x
        x_new = lin.solve(lin.F + bu)
        dx = np.clip(x_new - x, -vstep, vstep)
        x = x + dx
        if circ.dev.size == 0:
            return x
    return x


@dataclass
class RunStats:
    steps: int = 0
    rejects: int = 0
    lu: int = 0
    krylov: int = 0
    ts: list = field(default_factory=list)
    hs: list = field(default_factory=list)
    ms: list = field(default_factory=list)


def er_run(circ, t_end=None, tol=1e-6, opts: Options = None, x0=None, max_steps=10 ** 7,
           trace=False):
    """Adaptive ER / ER-C transient of Algorithm 2 from the DC solution to t_end.
    One LU per step (a linear circuit keeps its single LU of G); a rejected step shrinks h by alpha and reuses the Krylov bases of
    the solution (no new LU, no new basis for v1/v2, same m; only exp(h H_m^{-1}) is
    re-evaluated); h grows by beta when i < i_grow."""
    opts = opts or Options()
    t_end = circ.t_end if t_end is None else t_end
    h_max = opts.h_max if opts.h_max > 0 else t_end / 100.0
    h_prop = opts.h_init if opts.h_init > 0 else h_max
    bps = circ.breakpoints()
    bps = bps[(bps > 0) & (bps < t_end)]
    x = dc_solution(circ) if x0 is None else np.array(x0, dtype=np.float64)
    t = 0.0
    stats = RunStats()
    C = circ.C
    lin = None
    while t < t_end * (1 - 1e-12) and stats.steps < max_steps:
        nb = bps[bps > t * (1 + 1e-14) + 1e-30]
        t_next = min(nb[0], t_end) if nb.size else t_end
        h = min(h_prop, h_max, t_next - t)
        if lin is None or circ.dev.size:
            # one LU of G_k per step; a linear circuit has G_k = G_lin at every step, so its
            # single factorisation is kept (the same factors a refactor would produce)
            lin = linearize(circ, x)
            stats.lu += 1
        else:
            lin = Linearization(x=x.copy(), Gdev=lin.Gdev, Gk=lin.Gk, F=lin.F, lu=lin.lu)
        st = step_setup(circ, lin, t, pwl_slope(circ, t, h))
        if opts.combined:
            st.v1 = st.v1 + st.v2
            st.v2 = np.zeros(circ.n)
        st.K1 = arnoldi_iks(C, lin, lin.Gk, st.v1, h, opts.eps, opts.m_max, opts.m_min)
        st.K2 = arnoldi_iks(C, lin, lin.Gk, st.v2, h, opts.eps, opts.m_max, opts.m_min) \
            if np.any(st.v2) else None
        stats.krylov += st.K1.built + (st.K2.built if st.K2 is not None else 0)
        E_rr = tol * max(1.0, float(np.max(np.abs(x))))
        i = 0
        while True:
            # the bases and their dimensions m are reused; only exp(h H_m^{-1}) changes
            x_new = er_update(st, h)
            err = 0.0
            if circ.dev.size:
                e, ve, Ke = error_vector(circ, st, x_new, h, C, opts)
                if Ke is not None:
                    stats.krylov += Ke.built
                err = float(np.max(np.abs(e)))
                if opts.correction:
                    x_new = x_new - correction_term(circ, st, ve, h, C, opts)
            if err <= E_rr:
                break
            i += 1
            stats.rejects += 1
            h *= opts.alpha
            if h < opts.h_min:
                raise FloatingPointError("step size underflow")
        landed = h == t_next - t
        t = t_next if landed else t + h
        x = x_new
        stats.steps += 1
        if trace:
            stats.ts.append(t); stats.hs.append(h); stats.ms.append(st.K1.m)
        h_prop = min(opts.beta * h, h_max) if i < opts.i_grow else h
    return x, t, stats


# ----------------------------------------------------------------------------------------
# Backward Euler + Newton-Raphson (Sec. II-A, Eq. 2-3): reference solutions only.
# ----------------------------------------------------------------------------------------
def be_run(circ, h, t_end=None, x0=None, newton_tol=1e-12, max_newton=50, record=None):
    """Fixed-step BENR.  Each Newton iteration factors C/h + G(x) (Eq. 3)."""
    t_end = circ.t_end if t_end is None else t_end
    x = dc_solution(circ) if x0 is None else np.array(x0, dtype=np.float64)
    nsteps = int(round(t_end / h))
    Ch = circ.C / h
    out = []
    for k in range(nsteps):
        t1 = (k + 1) * h
        bu = circ.B @ circ.u(t1)
        xk = x.copy()
        for _ in range(max_newton):
            if circ.dev.size:
                idev, Gdev = device_eval(circ, x)
            else:
                idev, Gdev = np.zeros(circ.n), sp.csr_matrix((circ.n, circ.n))
            T = Ch @ (x - xk) + circ.G @ x + idev - bu
            Jac = (Ch + circ.G + Gdev).tocsc()
            dx = SparseLU(Jac).solve(-T)
            x = x + dx
            if np.max(np.abs(dx)) <= newton_tol * max(1.0, np.max(np.abs(x))):
                break
        if record is not None and (k + 1) % record == 0:
            out.append(x.copy())
    return (x, out) if record is not None else x
