"""Pins of the oracle's block ILU(0)-preconditioned BiCGStab (the linear step used where the sparse
LU is too large): on a block-tridiagonal system ILU(0) has no fill to drop, so it is the exact
factorization and BiCGStab converges in one iteration to the LU solution; on random block systems
and on Jacobians it reaches the dense solution; whole timesteps with it reach the same fields and
Newton counts as with the LU."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2008_01539_gb300 import casegen as cg

PSI = cg.PSI


def _dense(row_ptr, col, diag, off):
    nb = row_ptr.shape[0] - 1
    A = np.zeros((2 * nb, 2 * nb))
    for i in range(nb):
        A[2 * i:2 * i + 2, 2 * i:2 * i + 2] = diag[i]
        for e in range(row_ptr[i], row_ptr[i + 1]):
            A[2 * i:2 * i + 2, 2 * col[e]:2 * col[e] + 2] = off[e]
    return A


def test_tridiagonal_block_system_is_solved_exactly_in_one_iteration():
    rng = np.random.default_rng(1)
    nb = 60
    rows, cols = [], []
    for i in range(nb):
        for j in (i - 1, i + 1):
            if 0 <= j < nb:
                rows.append(i)
                cols.append(j)
    G = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(nb, nb))
    off = rng.standard_normal((G.nnz, 2, 2))
    diag = rng.standard_normal((nb, 2, 2)) + 6.0 * np.eye(2)
    rhs = rng.standard_normal((nb, 2))
    x, st, its = O.ilu0_bicgstab(G.indptr, G.indices, diag, off, rhs, rtol=1e-12)
    ref, _ = O.lu_solve(G.indptr, G.indices, diag, off, rhs)
    assert st == 0 and its == 1, (st, its)
    assert np.abs(x - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_block_systems_match_dense(seed):
    rng = np.random.default_rng(seed)
    nb = 80
    G = sp.random(nb, nb, density=0.06, random_state=seed)
    G = ((G + G.T) > 0).tolil()
    G.setdiag(0)
    G = sp.csr_matrix(G)
    G.sort_indices()
    off = rng.standard_normal((G.nnz, 2, 2))
    diag = rng.standard_normal((nb, 2, 2)) + np.eye(2) * 8.0
    rhs = rng.standard_normal((nb, 2))
    x, st, its = O.ilu0_bicgstab(G.indptr, G.indices, diag, off, rhs, rtol=1e-12)
    ref = np.linalg.solve(_dense(G.indptr, G.indices, diag, off), rhs.ravel()).reshape(-1, 2)
    assert st == 0 and its > 1
    assert np.abs(x - ref).max() < 1e-9 * np.abs(ref).max()


def test_jacobian_system_matches_lu():
    case = cg.small_dfn()
    m = O.Model(case)
    rng = np.random.default_rng(4)
    p = rng.uniform(3000.0, 5000.0, case.n) * PSI
    sw = rng.uniform(0.3, 0.6, case.n)
    F, Jd, Jo = O.assemble(m, p, sw, p + 10 * PSI, sw, cg.DAY)
    x, st, its = O.ilu0_bicgstab(case.row_ptr, case.nbr, Jd, Jo, -F, rtol=1e-12)
    ref, _ = O.lu_solve(case.row_ptr, case.nbr, Jd, Jo, -F)
    assert st == 0
    rel = np.abs(x - ref).max(axis=0) / np.abs(ref).max(axis=0)
    assert np.all(rel < 1e-8), rel


@pytest.mark.parametrize("mode", [0, 1])
def test_timesteps_with_ilu0_match_lu(mode):
    case = cg.config0()
    tight = dict(tol_dp=1.0, tol_cnv=1e-10)
    a = O.Sim(case, O.Options(mode=mode, **tight))
    b = O.Sim(case, O.Options(mode=mode, linear=1, lin_rtol=1e-12, **tight))
    for dt in case.dt_schedule:
        sa = a.timestep(dt)
        sb = b.timestep(dt)
        assert sa["status"] == 0 and sb["status"] == 0
        assert abs(sa["iterations"] - sb["iterations"]) <= 1
    assert np.max(np.abs(a.p - b.p) / a.p) < 1e-9
    assert np.max(np.abs(a.sw - b.sw)) < 1e-9
