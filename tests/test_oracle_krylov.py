"""Pins of the oracle's solvers (paper Sec. 4: CG and MG-CG) and of the
critical-mass finder, against dense linear algebra on small lattices."""
import numpy as np
import pytest

import workloads as W
from oracle import critical, krylov
from oracle import multigrid as mg
from oracle import wilson as w


def hierarchy(L, m, blocks, Nv, beta=6.0, sweeps=50, seed=3):
    Lx, Lt = L
    U = W.links_from_angles(W.quenched_u1_angles(Lx, Lt, beta, sweeps, seed))
    return U, mg.setup(U, m, list(blocks), list(Nv), W.setup_noise(Lx, Lt, blocks, Nv, 11))


@pytest.mark.parametrize("m", [0.05, -1.8])
def test_cg_and_mgcg_match_dense_inverse_8x8(m):
    U, H = hierarchy((8, 8), m, [(2, 2)], [2])
    A = H.levels[0].op.dense()
    chi = W.gaussian_field((8, 8, 2), 101)
    b = w.apply_D(U, m, chi, dagger=True)
    xs = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    kappa = np.linalg.cond(A)
    tol = 1e-10
    for x, it, info in (krylov.cg(H.levels[0].op.apply, b, tol, 5000), krylov.mgcg(H, b, tol)):
        assert info["true_res"] <= tol
        assert np.linalg.norm(b - (A @ x.ravel()).reshape(b.shape)) <= tol * np.linalg.norm(b)
        assert np.linalg.norm(x - xs) <= 2 * kappa * tol * np.linalg.norm(xs)


def test_mgcg_three_level_16x16_matches_dense():
    U, H = hierarchy((16, 16), -1.5, [(4, 4), (2, 2)], [3, 4])
    A = H.levels[0].op.dense()
    b = W.gaussian_field((16, 16, 2), 7)
    x, it, info = krylov.mgcg(H, b, 1e-12)
    xs = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    assert np.linalg.norm(x - xs) <= 2 * np.linalg.cond(A) * 1e-12 * np.linalg.norm(xs)
    x_cg, it_cg, _ = krylov.cg(H.levels[0].op.apply, b, 1e-12, 5000)
    assert it < it_cg


def test_zero_rhs_gives_zero():
    U, H = hierarchy((8, 8), 0.1, [(2, 2)], [2])
    x, it, info = krylov.mgcg(H, np.zeros((8, 8, 2), np.complex128), 1e-10)
    assert it == 0 and not np.any(x)


def test_coarsest_cg_branch_agrees_with_dense():
    U, H = hierarchy((8, 8), -0.7, [(2, 2)], [2])
    b = W.gaussian_field((4, 4, 4), 5)
    xd = mg.coarsest_solve(H, b)
    H.coarsest_chol = None
    xc = mg.coarsest_solve(H, b)
    assert np.linalg.norm(xd - xc) < 1e-11 * np.linalg.norm(xd)


def test_critical_mass_small_lattice():
    """m_crit makes D singular; at m_nc lambda_min(A) < 1e-5 (dense check)."""
    th = W.quenched_u1_angles(16, 16, 3.0, 100, 2)    # Q = 2: real modes exist
    U = W.links_from_angles(th)
    res = critical.near_critical_mass(U)
    if res is None:
        pytest.skip("no real eigenvalue of D_0 for this configuration")
    D = w.dirac_matrix(U, res["m_crit"]).toarray()
    assert np.linalg.svd(D, compute_uv=False).min() < 1e-9
    Dn = w.dirac_matrix(U, res["m_nc"]).toarray()
    lam = np.linalg.svd(Dn, compute_uv=False).min() ** 2
    assert lam < 1e-5 and lam == pytest.approx(res["lambda_min"], rel=1e-6)
    # no real eigenvalue of D_0 lies below -m_crit
    ev = np.linalg.eigvals(w.dirac_matrix(U, 0.0).toarray())
    real = ev[np.abs(ev.imag) < 1e-7 * np.abs(ev)].real
    assert real.min() == pytest.approx(-res["m_crit"], abs=1e-10)


@pytest.mark.parametrize("L,beta,sweeps,seed", [(16, 3.0, 100, 2), (32, 6.0, 200, 1), (32, 3.0, 100, 3)])
def test_flow_finder_matches_dense_real_eigenvalue(L, beta, sweeps, seed):
    """The spectral-flow finder used on large lattices returns the heaviest
    singular mass, -(smallest real eigenvalue of D_0), found here by a dense
    eigendecomposition; these configurations have two or more real modes."""
    U = W.links_from_angles(W.quenched_u1_angles(L, L, beta, sweeps, seed))
    ev = np.linalg.eigvals(w.dirac_matrix(U, 0.0).toarray())
    real = np.sort(ev[np.abs(ev.imag) < 1e-7 * np.abs(ev)].real)
    assert real.size >= 2
    m = critical.critical_mass_by_flow(U)
    assert m == pytest.approx(-real[0], abs=1e-9)
