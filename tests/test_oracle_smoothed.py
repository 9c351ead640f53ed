"""Pins of the oracle's smoothed aggregation (Sec. 3, the Richardson step on
the vectors before the prolongator is formed, damping chosen to minimise the
condition number of the coarse operator).

Facts checked: omega = 0 gives the tentative prolongator, whose sparse Galerkin
product equals the block-formula Galerkin operator of ``multigrid``, and whose
two-level V-cycle equals ``multigrid.vcycle``; A = D^dagger D couples no
sites two apart along an axis, so smoothing keeps the 9-point coarse stencil
for 4 x 4 blocks and widens it to 25 points for 2 x 2 blocks; the smoothed
coarse operator is Hermitian positive definite; the chosen omega is a minimum
of the condition number (no better on a fine grid around it, better than
omega = 0); and smoothing lowers the MG-CG iteration count near the critical
mass.
"""
import numpy as np
import pytest

import workloads as W
from oracle import critical, krylov
from oracle import multigrid as mg
from oracle import smoothed as sa
from oracle import wilson as w


def make(L, b, nv, m, beta=3.0, sweeps=20, seed=1):
    U = W.quenched_u1(L, L, beta, sweeps, seed)
    H = mg.setup(U, m, [(b, b)], [nv], W.setup_noise(L, L, [(b, b)], [nv], 7))
    lv = H.levels[0]
    return U, H, sa.normal_matrix(U, m), sa.tentative_prolongator(lv.V, b, b)


def test_unsmoothed_equals_the_block_galerkin_and_vcycle():
    U, H, A, P = make(16, 4, 2, -0.5)
    lv = H.levels[0]
    G = mg.galerkin(lv.op, lv.V, 4, 4).dense()
    Ac = sa.coarse_operator(A, sa.smoothed_prolongator(A, P, 0.0)).toarray()
    assert np.max(np.abs(G - Ac)) <= 1e-14 * np.max(np.abs(G))
    T = sa.TwoLevelSA(A, P, lv.c0, lv.c1)
    r = W.gaussian_field((16, 16, 2), 4)
    assert np.linalg.norm(T.vcycle(r) - mg.vcycle(H, r)) <= 1e-12 * np.linalg.norm(mg.vcycle(H, r))


def test_normal_operator_has_no_two_hop_terms():
    U = W.quenched_u1(8, 8, 3.0, 10, 2)
    A = sa.normal_matrix(U, 0.3).tocoo()
    x, t = (A.row // 2) % 8, (A.row // 2) // 8
    x2, t2 = (A.col // 2) % 8, (A.col // 2) // 8
    dx = np.minimum(np.abs(x - x2), 8 - np.abs(x - x2))
    dt = np.minimum(np.abs(t - t2), 8 - np.abs(t - t2))
    nz = np.abs(A.data) > 1e-14
    assert np.max(np.maximum(dx, dt)[nz]) == 1
    # while the single hops of D are there
    assert np.any(nz & (dx == 1) & (dt == 0)) and np.any(nz & (dx == 1) & (dt == 1))


@pytest.mark.parametrize("b,reach", [(4, 1), (2, 2)])
def test_stencil_reach_of_the_smoothed_coarse_operator(b, reach):
    L = 16
    U, H, A, P = make(L, b, 2, -0.5)
    assert sa.block_reach(sa.coarse_operator(A, P), L // b, L // b, 4) == 1
    Ac = sa.coarse_operator(A, sa.smoothed_prolongator(A, P, 0.1))
    assert sa.block_reach(Ac, L // b, L // b, 4) == reach
    D = Ac.toarray()
    assert np.max(np.abs(D - D.conj().T)) <= 1e-13 * np.max(np.abs(D))
    assert np.linalg.eigvalsh(D)[0] > 0


def test_optimal_omega_is_a_minimum_of_the_condition_number():
    L = 16
    U, H, A, P = make(L, 4, 2, -0.5)
    lam = mg.power_lambda_max(H.levels[0].op.apply, W.gaussian_field((L, L, 2), 5), 60)
    om, c = sa.optimal_omega(A, P, lam)
    cond = lambda x: sa.condition_number(sa.coarse_operator(A, sa.smoothed_prolongator(A, P, x)))  # noqa: E731
    assert 0 < om < 2 / lam and abs(cond(om) - c) <= 1e-12 * c
    assert c < cond(0.0)
    for dw in (-1e-3, 1e-3):
        assert cond(om + dw / lam) >= c * (1 - 1e-9)


def test_smoothing_lowers_iterations_near_the_critical_mass():
    """32 x 32, beta = 3, 0.02 above the critical mass, two vectors per
    chirality on 4 x 4 blocks: MG-CG with the smoothed prolongator at the
    chosen omega takes at most 90% of the iterations of the tentative one."""
    L = 32
    U = W.quenched_u1(L, L, 3.0, 100, 1)
    m = critical.critical_mass_by_flow(U) + 0.02
    H = mg.setup(U, m, [(4, 4)], [2], W.setup_noise(L, L, [(4, 4)], [2], 7))
    lv = H.levels[0]
    A, P = sa.normal_matrix(U, m), sa.tentative_prolongator(lv.V, 4, 4)
    lam = mg.power_lambda_max(lv.op.apply, W.gaussian_field((L, L, 2), 5), 50)
    om, _ = sa.optimal_omega(A, P, lam)
    b = w.apply_D(U, m, W.gaussian_field((L, L, 2), 3), dagger=True)
    _, it_tent, _ = krylov.mgcg(H, b, 1e-10, 5000)
    T = sa.TwoLevelSA(A, sa.smoothed_prolongator(A, P, om), lv.c0, lv.c1)
    _, it_sa, info = krylov.pcg(lv.op.apply, b, 1e-10, 5000, precond=T.vcycle)
    assert info["true_res"] <= 1e-10
    assert it_sa <= 0.9 * it_tent, (it_sa, it_tent)
