"""Pins of the oracle's own numerical pieces against facts outside them: the sparse LU
(oracle/olu.c) by the factorisation identity P A Q = L U and by SuperLU solutions as a
cross-check, the minimum-degree order by being a permutation that beats the natural order's
fill, and the [13/13] Pade exponential by closed forms (eigendecomposition of a symmetric
matrix, nilpotent and scalar cases, e^A e^-A = I) and scipy's expm as a cross-check."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from synth import circuits as S
from oracle import ers_oracle as O
from oracle import sparse_lu as SL


def _families():
    rng = np.random.default_rng(5)
    A = sp.random(60, 60, density=0.08, random_state=3) + sp.diags(rng.uniform(0.5, 1.0, 60))
    # a matrix that needs row interchanges: zero diagonal in the leading rows
    P = sp.csr_matrix(np.roll(np.eye(30), 1, axis=0)) + sp.random(30, 30, density=0.05,
                                                                   random_state=4)
    chain = S.inverter_chain(stages=6, tree_nodes=12, seed=4)
    lin = O.linearize(chain, O.dc_solution(chain))
    return [("random", A.tocsc()), ("permuted", P.tocsc()),
            ("mesh2d", S.rc_mesh_2d(12, 9, seed=3).G), ("mesh3d", S.rc_mesh_3d(7, 6, 5, seed=2).G),
            ("chain_Gk", lin.Gk), ("coupled", S.coupled_rc_mesh_2d(6, 6, seed=1).G)]


@pytest.mark.parametrize("name,A", _families())
def test_sparse_lu_factorisation_identity(name, A):
    lu = SL.SparseLU(A)
    L, U, prow, q = lu.factors()
    assert sorted(prow.tolist()) == list(range(A.shape[0]))
    assert sorted(q.tolist()) == list(range(A.shape[0]))
    Ad = sp.csc_matrix(A).toarray()
    Ld, Ud = L.toarray(), U.toarray()
    assert np.allclose(np.triu(Ld, 1), 0) and np.allclose(np.diag(Ld), 1)
    assert np.allclose(np.tril(Ud, -1), 0)
    resid = np.max(np.abs(Ad[prow][:, q] - Ld @ Ud))
    assert resid <= 1e-14 * np.max(np.abs(Ad)) * max(1, A.shape[0] ** 0.5)
    # threshold pivoting keeps every multiplier below 1 / tau
    assert np.max(np.abs(np.tril(Ld, -1))) <= 1 / 0.1 + 1e-12


@pytest.mark.parametrize("name,A", _families())
def test_sparse_lu_solves_like_superlu(name, A):
    rng = np.random.default_rng(11)
    B = rng.normal(size=(A.shape[0], 3))
    X = SL.SparseLU(A).solve(B)
    ref = spla.splu(sp.csc_matrix(A)).solve(B)
    cond = np.linalg.cond(sp.csc_matrix(A).toarray())
    assert np.max(np.abs(X - ref)) <= 1e-14 * cond * np.max(np.abs(ref))
    x1 = SL.SparseLU(A).solve(B[:, 0])
    assert x1.shape == (A.shape[0],)
    assert np.array_equal(x1, X[:, 0])


def test_sparse_lu_reports_singular_matrix():
    A = sp.csc_matrix(np.array([[1.0, 2.0, 0.0], [2.0, 4.0, 0.0], [0.0, 0.0, 1.0]]))
    with pytest.raises(SL.SingularMatrixError):
        SL.SparseLU(A)


def test_minimum_degree_order_is_a_permutation_with_less_fill():
    G = S.rc_mesh_3d(9, 9, 9, seed=1).G
    q = SL.min_degree_order(G)
    assert sorted(q.tolist()) == list(range(G.shape[0]))
    natural = SL.SparseLU(G, order=np.arange(G.shape[0], dtype=np.int32)).nnz
    assert SL.SparseLU(G, order=q).nnz < 0.7 * natural
    # a tree orders without fill (leaves first): nnz(L) + nnz(U) = nnz(A) + n
    chain = S.inverter_chain(stages=1, tree_nodes=40, seed=3)
    T = chain.G
    assert SL.SparseLU(T).nnz == T.nnz + T.shape[0]


def test_pade13_symmetric_matrix_matches_eigendecomposition():
    rng = np.random.default_rng(2)
    for scale in (1e-3, 1.0, 30.0, 3e3):
        M = rng.normal(size=(12, 12))
        A = -scale * (M @ M.T) / 12 + 0.1 * (M + M.T)   # symmetric, stable for large scales
        lam, Q = np.linalg.eigh(A)
        ref = (Q * np.exp(lam)) @ Q.T
        E = O.expm_pade13(A)
        assert np.max(np.abs(E - ref)) <= 1e-12 * np.max(np.abs(ref)) * max(1.0, scale / 30)


def test_pade13_closed_forms():
    # nilpotent: e^N = I + N + N^2 / 2 exactly
    N = np.array([[0.0, 3.0, -1.0], [0.0, 0.0, 2.0], [0.0, 0.0, 0.0]])
    assert np.max(np.abs(O.expm_pade13(N) - (np.eye(3) + N + N @ N / 2))) <= 1e-14
    # scalars across the scaling range, and a stiff negative one that underflows to 0
    for z in (-1e-8, 0.3, -7.0, 40.0, -1e4):
        assert abs(O.expm_pade13(np.array([[z]]))[0, 0] - np.exp(z)) <= 1e-13 * np.exp(z) + 1e-300
    # e^A e^-A = I on a non-normal matrix
    rng = np.random.default_rng(8)
    A = np.triu(rng.normal(size=(10, 10))) * 3
    assert np.max(np.abs(O.expm_pade13(A) @ O.expm_pade13(-A) - np.eye(10))) <= 1e-9
    # complex input (the singular-C branch uses it on a Schur block)
    B = rng.normal(size=(6, 6)) + 1j * rng.normal(size=(6, 6))
    assert np.max(np.abs(O.expm_pade13(B) - sla.expm(B))) <= 1e-13 * np.max(np.abs(sla.expm(B)))


def test_pade13_matches_scipy_expm():
    rng = np.random.default_rng(9)
    for scale in (1e-2, 1.0, 50.0):
        A = scale * rng.normal(size=(16, 16)) / 4
        ref = sla.expm(A)
        assert np.max(np.abs(O.expm_pade13(A) - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_dense_lu_solve_with_pivoting():
    A = np.array([[0.0, 1.0, 2.0], [1.0, 0.0, 3.0], [4.0, -3.0, 8.0]])
    B = np.arange(6.0).reshape(3, 2)
    X = O.dense_lu_solve(A, B)
    assert np.max(np.abs(A @ X - B)) <= 1e-13
    rng = np.random.default_rng(1)
    M = rng.normal(size=(40, 40))
    b = rng.normal(size=40)
    assert np.max(np.abs(O.dense_lu_solve(M, b) - np.linalg.solve(M, b))) <= 1e-10
