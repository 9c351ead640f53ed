"""Pins of the oracle's multigrid hierarchy (paper Secs. 2-4).

Facts checked: block map by brute force; P^dagger P = I and the chirality
structure of P; the relaxed vectors lie in range(P); P and P^dagger are
adjoint; the Galerkin stencil equals the explicit dense P^dagger A P (also on
a coarse extent of 2 where +1 and -1 neighbours alias); Hermiticity and
positivity of the coarse operator; the full-span case where P is unitary and
the two-level V-cycle is A^{-1}; the V-cycle's closed form with the corrected
sign; Hermiticity and positivity of V; the minimum-residual coefficients; the
application count 2 nu + 2 per level.
"""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as mg
from oracle import wilson as w


def make(L=(8, 8), beta=3.0, sweeps=20, seed=1, m=-0.5, blocks=((2, 2),), Nv=(2,), nseed=7, **kw):
    Lx, Lt = L
    U = W.links_from_angles(W.quenched_u1_angles(Lx, Lt, beta, sweeps, seed))
    noise = W.setup_noise(Lx, Lt, blocks, Nv, nseed)
    return U, mg.setup(U, m, list(blocks), list(Nv), noise, **kw)


def dense_prolongator(lv):
    Ltc, Lxc = lv.Lt // lv.bt, lv.Lx // lv.bx
    nc = Ltc * Lxc * 2 * lv.Nv
    cols = []
    for i in range(nc):
        e = np.zeros(nc, dtype=np.complex128)
        e[i] = 1
        cols.append(mg.prolong(lv.V, lv.bx, lv.bt, e.reshape(Ltc, Lxc, 2 * lv.Nv)).ravel())
    return np.stack(cols, axis=1)


def test_block_map_brute_force():
    Lx, Lt, bx, bt = 12, 8, 4, 2
    coarse, offset = mg.block_map(Lx, Lt, bx, bt)
    seen = {}
    for t in range(Lt):
        for x in range(Lx):
            i = x + Lx * t
            j = coarse[i]
            assert j == (t // bt) * (Lx // bx) + x // bx
            assert offset[i] == (t % bt) * bx + x % bx
            seen.setdefault(int(j), set()).add(int(offset[i]))
    assert len(seen) == (Lx // bx) * (Lt // bt)
    assert all(s == set(range(bx * bt)) for s in seen.values())


def test_blocks_roundtrip():
    v = W.gaussian_field((3, 8, 12, 5), 2)
    b = mg.to_blocks(v, 4, 2)
    assert b.shape == (3, 4, 3, 8, 5)
    assert np.array_equal(mg.from_blocks(b, 4, 2), v)
    # offset (t%bt)*bx + x%bx inside block (jt, jx)
    assert b[1, 2, 1, 1 * 4 + 3, 4] == v[1, 2 * 2 + 1, 1 * 4 + 3, 4]


@pytest.mark.parametrize("blocks,Nv,L", [(((2, 2),), (3,), (8, 8)), (((4, 4),), (4,), (16, 12)),
                                         (((4, 4), (2, 2)), (3, 4), (16, 16))])
def test_prolongator_orthonormal_and_chiral(blocks, Nv, L):
    U, H = make(L=L, blocks=blocks, Nv=Nv)
    for lv in H.levels[:-1]:
        P = dense_prolongator(lv)
        assert np.max(np.abs(P.conj().T @ P - np.eye(P.shape[1]))) < 1e-14
        # gamma_5 P = P gamma_5^(coarse): fine chirality of each column equals its coarse chirality
        n, h = lv.n, lv.n // 2
        g5f = np.tile(np.repeat([1.0, -1.0], h), lv.Lx * lv.Lt)
        g5c = np.tile(np.repeat([1.0, -1.0], lv.Nv), (lv.Lx // lv.bx) * (lv.Lt // lv.bt))
        assert np.max(np.abs(g5f[:, None] * P - P * g5c[None, :])) == 0.0


def test_relaxed_vectors_in_range_of_P():
    U, H = make(L=(16, 16), blocks=((4, 4), (2, 2)), Nv=(3, 4))
    for lv in H.levels[:-1]:
        P = dense_prolongator(lv)
        h = lv.n // 2
        for k in range(lv.Nv):
            for c in (0, 1):
                v = np.zeros_like(lv.E[k])
                v[..., c * h:(c + 1) * h] = lv.E[k][..., c * h:(c + 1) * h]
                v = v.ravel()
                resid = v - P @ (P.conj().T @ v)
                assert np.linalg.norm(resid) <= 1e-12 * np.linalg.norm(v)


def test_restrict_is_adjoint_of_prolong():
    U, H = make(L=(16, 12), blocks=((4, 4),), Nv=(4,))
    lv = H.levels[0]
    r = W.gaussian_field((12, 16, 2), 3)
    ec = W.gaussian_field((3, 4, 8), 4)
    lhs = np.vdot(mg.restrict(lv.V, 4, 4, r), ec)
    rhs = np.vdot(r, mg.prolong(lv.V, 4, 4, ec))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


@pytest.mark.parametrize("blocks,Nv,L", [(((2, 2),), (3,), (8, 8)),      # coarse 4x4
                                         (((4, 4),), (4,), (8, 8)),      # coarse 2x2: aliasing
                                         (((4, 4),), (3,), (12, 16)),    # coarse 3x4
                                         (((2, 2), (2, 2)), (2, 3), (8, 12))])
def test_galerkin_equals_dense_PdagAP(blocks, Nv, L):
    U, H = make(L=L, blocks=blocks, Nv=Nv)
    A = H.levels[0].op.dense()
    for l, lv in enumerate(H.levels[:-1]):
        P = dense_prolongator(lv)
        want = P.conj().T @ A @ P
        got = H.levels[l + 1].op.dense()
        assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))
        A = got


def test_coarse_operator_hermitian_per_displacement_and_pd():
    U, H = make(L=(16, 12), blocks=((4, 4),), Nv=(4,))
    op = H.levels[1].op
    Ltc, Lxc = op.Lt, op.Lx
    for d, (dx, dt) in enumerate(mg.COARSE_DISP):
        dm = mg.COARSE_DISP.index((-dx, -dt))
        for t in range(Ltc):
            for x in range(Lxc):
                nb = op.M[(t + dt) % Ltc, (x + dx) % Lxc, dm]
                assert np.max(np.abs(op.M[t, x, d] - nb.conj().T)) < 1e-14
    ev = np.linalg.eigvalsh(op.dense())
    assert ev.min() > 0


def test_full_span_prolongator_is_unitary_and_vcycle_exact():
    """2x2 blocks at level 0 carry 4 dof per chirality; with Nv = 4 P is unitary,
    spec(A_c) = spec(A), the two-level V-cycle equals A^{-1} and MG-CG converges
    in one iteration."""
    from oracle import krylov
    U, H = make(L=(8, 8), blocks=((2, 2),), Nv=(4,), m=-0.3)
    P = dense_prolongator(H.levels[0])
    assert np.max(np.abs(P @ P.conj().T - np.eye(P.shape[0]))) < 1e-14
    A = H.levels[0].op.dense()
    assert np.max(np.abs(np.linalg.eigvalsh(H.levels[1].op.dense()) - np.linalg.eigvalsh(A))) < 1e-11
    b = W.gaussian_field((8, 8, 2), 5)
    x = mg.vcycle(H, b)
    xs = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    assert np.linalg.norm(x - xs) < 1e-12 * np.linalg.norm(xs)
    _, it, info = krylov.mgcg(H, b, 1e-10)
    assert it == 1


def test_vcycle_closed_form_with_corrected_sign():
    """The five steps give V = 2R - RAR + (1 - RA) P V' P^dagger (1 - AR)
    (R = R^dagger); the printed '+ R A R' form does not match."""
    U, H = make(L=(8, 8), blocks=((2, 2),), Nv=(2,), m=-0.2)
    lv = H.levels[0]
    A = lv.op.dense()
    N = A.shape[0]
    I = np.eye(N)
    R = lv.c0 * I + lv.c1 * A
    P = dense_prolongator(lv)
    Vc = np.linalg.inv(H.levels[1].op.dense())
    V_closed = 2 * R - R @ A @ R + (I - R @ A) @ P @ Vc @ P.conj().T @ (I - A @ R)
    V_printed = 2 * R + R @ A @ R + (I - R @ A) @ P @ Vc @ P.conj().T @ (I - A @ R)
    cols = []
    for i in range(N):
        e = np.zeros(N, dtype=np.complex128)
        e[i] = 1
        cols.append(mg.vcycle(H, e.reshape(8, 8, 2)).ravel())
    V_steps = np.stack(cols, axis=1)
    scale = np.max(np.abs(V_closed))
    assert np.max(np.abs(V_steps - V_closed)) < 1e-12 * scale
    assert np.max(np.abs(V_steps - V_printed)) > 1e-3 * scale


def test_vcycle_hermitian_positive_three_levels():
    U, H = make(L=(16, 16), blocks=((4, 4), (2, 2)), Nv=(3, 4), m=-0.8)
    for s in range(3):
        u = W.gaussian_field((16, 16, 2), 100 + s)
        v = W.gaussian_field((16, 16, 2), 200 + s)
        a = np.vdot(u, mg.vcycle(H, v))
        b = np.vdot(mg.vcycle(H, u), v)
        assert abs(a - b) < 1e-12 * abs(a)
        assert np.vdot(u, mg.vcycle(H, u)).real > 0


def test_mr_coefficients_minimise_residual_and_freeze():
    U, H = make(L=(8, 8), blocks=((2, 2),), Nv=(2,), m=0.1)
    lv = H.levels[0]
    apply = lv.op.apply
    eta = W.gaussian_field((8, 8, 2), 9)
    c0, c1, a0, a1 = mg.mr_smoother_coefficients(apply, eta, 0.8)
    q0 = apply(eta)
    f = lambda a: np.linalg.norm(eta - a * q0)
    assert f(a0) <= min(f(a0 * 1.001), f(a0 * 0.999))
    # the two relaxed MR steps, taken one by one, end at R eta
    x = 0.8 * a0 * eta
    r = eta - 0.8 * a0 * q0
    x = x + 0.8 * a1 * r
    assert np.max(np.abs(x - (c0 * eta + c1 * apply(eta)))) < 1e-13 * np.max(np.abs(x))
    assert a1 == pytest.approx(np.vdot(apply(r), r).real / np.vdot(apply(r), apply(r)).real, rel=1e-13)


def test_applications_per_level_is_2nu_plus_2():
    """Each non-coarsest level applies its operator 2 nu + 2 = 4 times per
    V-cycle (nu = 1: R is one application of A)."""
    U, H = make(L=(16, 16), blocks=((4, 4), (2, 2)), Nv=(2, 3), m=-0.5)
    counts = [0] * H.L
    for l, lv in enumerate(H.levels):
        orig = lv.op.apply

        def counted(v, l=l, orig=orig):
            counts[l] += 1
            return orig(v)
        lv.op.apply = counted
    mg.vcycle(H, W.gaussian_field((16, 16, 2), 1))
    assert counts[:-1] == [4, 4]


def test_block_orthonormalise_detects_rank_deficiency():
    E = W.gaussian_field((3, 4, 4, 2), 2)
    E[2] = 2.0 * E[0] - 1j * E[1]
    with pytest.raises(mg.Breakdown):
        mg.block_orthonormalise(E, 2, 2)


def test_set_mass_matches_fresh_galerkin():
    U, H = make(L=(8, 8), blocks=((2, 2),), Nv=(3,), m=-0.5)
    P = dense_prolongator(H.levels[0])
    mg.set_mass(H, 0.25)
    A = mg.WilsonNormalOp(U, 0.25).dense()
    assert np.max(np.abs(H.levels[1].op.dense() - P.conj().T @ A @ P)) < 1e-13 * np.max(np.abs(A))


def test_coarse_operators_are_quadratic_in_the_mass():
    """A(m) = A0 + m (D0 + D0^dagger) + m^2 and P^dagger P = I on every level,
    so each coarse operator is G0 + m G1 + m^2 I with G0 = A_c(0) and
    G1 = A_c(1) - A_c(0) - I (the identity behind re-massing by combination)."""
    U, H = make(L=(16, 16), blocks=((4, 4), (2, 2)), Nv=(3, 2), m=-0.4)
    ops = {}
    for m in (0.0, 1.0, -0.4, 0.37, -2.1):
        mg.set_mass(H, m)
        ops[m] = [lv.op.dense() for lv in H.levels[1:]]
    for l in range(len(ops[0.0])):
        G0 = ops[0.0][l]
        I = np.eye(G0.shape[0])
        G1 = ops[1.0][l] - G0 - I
        for m in (-0.4, 0.37, -2.1):
            want = ops[m][l]
            assert np.max(np.abs(G0 + m * G1 + m * m * I - want)) <= 1e-12 * np.max(np.abs(want))
        # G1 is Hermitian (P^dagger (D0 + D0^dagger) P)
        assert np.max(np.abs(G1 - G1.conj().T)) <= 1e-12 * np.max(np.abs(G1))
