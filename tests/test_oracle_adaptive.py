"""Pins of the oracle's adaptive refinement by V-cycles (Sec. 3, the adaptive
step after the first vector set).

Facts checked: the error left by V-cycles with no source equals the two-grid
error propagator in product form (I - R A)(I - P A_c^{-1} P^dagger A)(I - R A)
applied to e0, on the finest level and on a coarse level; the A-norm of the
error never grows and rho is the measured per-cycle ratio; the refined vector
set keeps the old vectors and appends, per block and chirality, the unit
component of e'' orthogonal to them (computed here by one projection onto the
old block basis, not by Gram-Schmidt); finer levels are kept and the operators
below are the Galerkin products of the new vectors; and the method's claim:
near the critical mass a refined vector set gives far fewer MG-CG iterations
than a relaxation-only set of the same size.
"""
import numpy as np
import pytest

import workloads as W
from oracle import critical, krylov
from oracle import multigrid as mg
from oracle import wilson as w


def make(L, blocks, Nv, m, beta=3.0, sweeps=20, seed=1, nseed=7):
    U = W.links_from_angles(W.quenched_u1_angles(L, L, beta, sweeps, seed))
    return U, mg.setup(U, m, list(blocks), list(Nv), W.setup_noise(L, L, blocks, Nv, nseed))


def dense_prolongator(lv):
    Ltc, Lxc = lv.Lt // lv.bt, lv.Lx // lv.bx
    nc = Ltc * Lxc * 2 * lv.Nv
    cols = []
    for i in range(nc):
        e = np.zeros(nc, dtype=np.complex128)
        e[i] = 1
        cols.append(mg.prolong(lv.V, lv.bx, lv.bt, e.reshape(Ltc, Lxc, 2 * lv.Nv)).ravel())
    return np.stack(cols, axis=1)


def two_grid_propagator(H, l):
    """(I - R A)(I - P A_c^{-1} P^dagger A)(I - R A) on level l (level l+1 coarsest)."""
    lv = H.levels[l]
    A = lv.op.dense()
    I = np.eye(A.shape[0])
    R = lv.c0 * I + lv.c1 * A
    P = dense_prolongator(lv)
    Ac = H.levels[l + 1].op.dense()
    S = I - R @ A
    return S @ (I - P @ np.linalg.solve(Ac, P.conj().T @ A)) @ S


@pytest.mark.parametrize("ncycles", [1, 3])
def test_error_propagation_is_the_two_grid_product(ncycles):
    U, H = make(8, [(2, 2)], [2], -0.3)
    e0 = W.gaussian_field((8, 8, 2), 5)
    E = two_grid_propagator(H, 0)
    want = np.linalg.matrix_power(E, ncycles) @ e0.ravel()
    got = mg.vcycle_error_propagation(H, e0, ncycles).ravel()
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(e0)
    # the sign matters: e + V A e is not the propagator
    wrong = e0 + mg.vcycle(H, H.levels[0].op.apply(e0))
    assert np.linalg.norm(wrong.ravel() - E @ e0.ravel()) > 1e-2 * np.linalg.norm(e0)


def test_error_propagation_on_a_coarse_level():
    U, H = make(16, [(4, 4), (2, 2)], [2, 2], -0.6)
    lv = H.levels[1]
    e0 = W.gaussian_field((lv.Lt, lv.Lx, lv.n), 6)
    want = two_grid_propagator(H, 1) @ (two_grid_propagator(H, 1) @ e0.ravel())
    got = mg.vcycle_error_propagation(H, e0, 2, level=1).ravel()
    assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(e0)


def test_energy_norm_never_grows_and_rho_is_the_measured_ratio():
    U, H = make(16, [(4, 4)], [2], -0.8)
    e = W.gaussian_field((16, 16, 2), 7)
    norms = [mg.energy_norm(H, e)]
    for _ in range(6):
        e = mg.vcycle_error_propagation(H, e, 1)
        norms.append(mg.energy_norm(H, e))
    assert all(b < a for a, b in zip(norms, norms[1:]))
    noise = W.refine_noise(16, 16, [(4, 4)], [3], 0, 8)
    _, e6, rho = mg.refine(H, W.gaussian_field((16, 16, 2), 7), 6, noise)
    assert abs(rho - (norms[-1] / norms[0]) ** (1 / 6)) <= 1e-12
    assert np.linalg.norm(e6 - e) <= 1e-14 * np.linalg.norm(e) + 1e-300
    # |e|_A^2 = <e, A e> with A = D^dagger D is |D e|^2
    De = w.apply_D(U, H.m, e)
    assert abs(norms[-1] - np.linalg.norm(De)) <= 1e-12 * norms[-1]


def _blocks_of(v, bx, bt, c):
    h = v.shape[-1] // 2
    B = mg.to_blocks(v[..., c * h:(c + 1) * h], bx, bt)         # [..., Ltc, Lxc, b2, h]
    return B.reshape(*B.shape[:-4], -1, B.shape[-2] * B.shape[-1])   # [..., Nc, b2*h]


@pytest.mark.parametrize("level", [0, 1])
def test_refined_vectors_append_the_orthogonal_block_component(level):
    U, H = make(16, [(4, 4), (2, 2)], [2, 3], -0.7)
    lv = H.levels[level]
    Nv = [2, 3]
    Nv[level] += 1
    e0 = W.gaussian_field((lv.Lt, lv.Lx, lv.n), 9)
    H2, e, _ = mg.refine(H, e0, 4, W.refine_noise(16, 16, [(4, 4), (2, 2)], Nv, level, 10), level=level)
    new = H2.levels[level]
    assert new.Nv == lv.Nv + 1 and [x.Nv for x in H2.levels[:-1]] == Nv
    assert np.max(np.abs(new.V[:lv.Nv] - lv.V)) <= 1e-13
    for c in (0, 1):
        Q = _blocks_of(lv.V, lv.bx, lv.bt, c)                  # [Nv, Nc, m], orthonormal per block
        eb = _blocks_of(e, lv.bx, lv.bt, c)                    # [Nc, m]
        coef = np.einsum("kja,ja->kj", np.conj(Q), eb)
        q = eb - np.einsum("kj,kja->ja", coef, Q)
        q /= np.linalg.norm(q, axis=-1, keepdims=True)
        got = _blocks_of(new.V[lv.Nv], lv.bx, lv.bt, c)
        assert np.max(np.abs(got - q)) <= 1e-10
    for x, y in zip(H.levels[:level], H2.levels[:level]):       # finer levels kept
        assert np.array_equal(x.V, y.V)
    # the operator below is P^dagger A P of the new vectors
    P = dense_prolongator(new)
    Ad = new.op.dense()
    assert np.allclose(H2.levels[level + 1].op.dense(), P.conj().T @ Ad @ P, rtol=0, atol=1e-12 * np.abs(Ad).max())


def test_refinement_removes_critical_slowing_down():
    """Sec. 3: the surviving error carries what the first vector set misses.
    32 x 32, beta = 3, 0.002 above the critical mass; two adaptive passes
    on two relaxed vectors beat a relaxation-only set of the same size (4
    vectors) by at least 1.5x in MG-CG iterations."""
    L = 32
    U = W.quenched_u1(L, L, 3.0, 100, 1)
    m = critical.critical_mass_by_flow(U) + 0.002
    b = w.apply_D(U, m, W.gaussian_field((L, L, 2), 3), dagger=True)

    def iters(H):
        _, it, info = krylov.mgcg(H, b, 1e-10, 5000)
        assert info["true_res"] <= 1e-10
        return it

    H = mg.setup(U, m, [(4, 4)], [2], W.setup_noise(L, L, [(4, 4)], [2], 7))
    counts = [iters(H)]
    for p in range(2):
        Nv = [H.levels[0].Nv + 1]
        H, _, rho = mg.refine(H, W.gaussian_field((L, L, 2), 100 + p), 20,
                              W.refine_noise(L, L, [(4, 4)], Nv, 0, 8 + p))
        assert 0 < rho < 1
        counts.append(iters(H))
    relax4 = iters(mg.setup(U, m, [(4, 4)], [4], W.setup_noise(L, L, [(4, 4)], [4], 7)))
    assert counts[2] < counts[1] < counts[0]
    assert 1.5 * counts[2] <= relax4


def test_setup_with_a_refinement_plan_reads_the_extended_noise():
    """setup(refine_levels=...) = the first pass followed by refine() on each
    level of the plan, with every random input taken from one buffer in the
    order of ``workloads.setup_noise``; the buffer is read to its end."""
    L, blocks, Nv, plan = 16, [(4, 4), (2, 2)], [2, 2], [0, 1, 1]
    U = W.links_from_angles(W.quenched_u1_angles(L, L, 3.0, 20, 1))
    noise = W.setup_noise(L, L, blocks, Nv, 4, refine_levels=plan)
    assert noise.size == W.setup_noise_len(L, L, blocks, Nv, plan)
    H = mg.setup(U, -0.7, blocks, Nv, noise, refine_levels=plan, refine_cycles=3)
    pos = W.setup_noise_len(L, L, blocks, Nv)
    G = mg.setup(U, -0.7, blocks, Nv, noise[:pos])
    nv = list(Nv)
    for level in plan:
        nv[level] += 1
        lx, lt, n = W.level_shapes(L, L, blocks, nv)[level]
        e0 = noise[pos:pos + lx * lt * n].reshape(lt, lx, n)
        pos += lx * lt * n
        tail = W.setup_noise_len(L, L, blocks, nv) - W.setup_noise_len(L, L, blocks[:level + 1], nv[:level + 1])
        G, _, _ = mg.refine(G, e0, 3, noise[pos:pos + tail], level)
        pos += tail
    assert pos == noise.size
    assert [lv.Nv for lv in H.levels[:-1]] == [3, 4]
    for a, b in zip(H.levels, G.levels):
        assert np.array_equal(a.op.dense(), b.op.dense())
    assert len(H.stats["refine_rho"]) == 3
    with pytest.raises(ValueError):
        mg.setup(U, -0.7, blocks, Nv, noise[:-1], refine_levels=plan, refine_cycles=3)
