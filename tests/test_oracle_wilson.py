"""Pins of the oracle's Wilson-Dirac operator (paper Sec. 1, display defining D).

Each test checks a fact fixed by the mathematics, not by re-typing the formula:
plane-wave symbols, adjoint identity, gamma_5-hermiticity, gauge covariance.
A non-square lattice (Lx != Lt) is used so that an exchange of the two
directions or of sigma_1/sigma_2 is caught.
"""
import numpy as np
import pytest

import workloads as W
from oracle import wilson as w

S1, S2, S3 = w.SIGMA1, w.SIGMA2, w.SIGMA3


def plane_wave(Lx, Lt, kx, kt, u):
    """psi(x,t) = exp(i (px x + pt t)) u with px = 2 pi kx / Lx (periodic) and
    pt = pi (2 kt + 1) / Lt (antiperiodic in t)."""
    px = 2 * np.pi * kx / Lx
    pt = np.pi * (2 * kt + 1) / Lt
    t, x = np.meshgrid(np.arange(Lt), np.arange(Lx), indexing="ij")
    phase = np.exp(1j * (px * x + pt * t))
    return phase[..., None] * np.asarray(u)[None, None, :], px, pt


def symbol(m, px, pt, dagger=False):
    """Free-field momentum-space D: (4 + m - cos px - cos pt) + i (s1 sin px + s2 sin pt)."""
    s = 1j * (S1 * np.sin(px) + S2 * np.sin(pt))
    return (4 + m - np.cos(px) - np.cos(pt)) * np.eye(2) + (-s if dagger else s)


@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("kx,kt", [(0, 0), (1, 0), (0, 2), (3, 1), (5, 4), (2, 5)])
def test_free_field_plane_waves(kx, kt, dagger):
    Lx, Lt, m = 8, 6, 0.37
    U = np.ones((2, Lt, Lx), dtype=np.complex128)
    u = np.array([0.3 - 0.7j, 1.1 + 0.2j])
    psi, px, pt = plane_wave(Lx, Lt, kx, kt, u)
    got = w.apply_D(U, m, psi, dagger=dagger)
    want = psi[..., :1] / u[0] * (symbol(m, px, pt, dagger) @ u)[None, None, :]
    assert np.max(np.abs(got - want)) < 5e-14


@pytest.mark.parametrize("kx,kt", [(0, 0), (2, 1), (7, 3)])
def test_constant_background_shifts_momentum(kx, kt):
    """Constant links U^mu = exp(i theta_mu): the forward hop carries U and the
    backward hop U^*, so the symbol is the free one at p + theta."""
    Lx, Lt, m = 8, 6, -0.4
    th = (0.31, -0.77)
    U = np.stack([np.full((Lt, Lx), np.exp(1j * th[0])), np.full((Lt, Lx), np.exp(1j * th[1]))])
    u = np.array([1.0 + 0.5j, -0.25 + 1j])
    psi, px, pt = plane_wave(Lx, Lt, kx, kt, u)
    got = w.apply_D(U, m, psi)
    want = psi[..., :1] / u[0] * (symbol(m, px + th[0], pt + th[1]) @ u)[None, None, :]
    assert np.max(np.abs(got - want)) < 5e-14


def closed_form_spectrum_A(Lx, Lt, m):
    ev = []
    for kx in range(Lx):
        for kt in range(Lt):
            px, pt = 2 * np.pi * kx / Lx, np.pi * (2 * kt + 1) / Lt
            lam = (4 + m - np.cos(px) - np.cos(pt)) ** 2 + np.sin(px) ** 2 + np.sin(pt) ** 2
            ev += [lam, lam]
    return np.sort(np.array(ev))


def matrix_of(apply, shape):
    n = int(np.prod(shape))
    cols = []
    for i in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[i] = 1.0
        cols.append(apply(e.reshape(shape)).ravel())
    return np.stack(cols, axis=1)


def test_free_spectrum_of_A_closed_form():
    Lx, Lt, m = 8, 6, 0.05
    U = np.ones((2, Lt, Lx), dtype=np.complex128)
    Am = matrix_of(lambda v: w.apply_A(U, m, v), (Lt, Lx, 2))
    assert np.allclose(Am, Am.conj().T, atol=1e-13)
    ev = np.linalg.eigvalsh(Am)
    assert np.max(np.abs(ev - closed_form_spectrum_A(Lx, Lt, m))) < 1e-12


def random_links(Lx, Lt, seed):
    return W.links_from_angles(W.quenched_u1_angles(Lx, Lt, 1.0, 3, seed))


def test_adjoint_identity():
    Lx, Lt, m = 10, 8, -0.6
    U = random_links(Lx, Lt, 3)
    psi = W.gaussian_field((Lt, Lx, 2), 4)
    phi = W.gaussian_field((Lt, Lx, 2), 5)
    lhs = np.vdot(phi, w.apply_D(U, m, psi))
    rhs = np.vdot(w.apply_D(U, m, phi, dagger=True), psi)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_dagger_is_conjugate_transpose_of_matrix():
    Lx, Lt, m = 6, 4, 0.2
    U = random_links(Lx, Lt, 8)
    Dm = matrix_of(lambda v: w.apply_D(U, m, v), (Lt, Lx, 2))
    Ddm = matrix_of(lambda v: w.apply_D(U, m, v, dagger=True), (Lt, Lx, 2))
    assert np.max(np.abs(Ddm - Dm.conj().T)) < 1e-15


def test_gamma5_hermiticity():
    Lx, Lt, m = 10, 8, 0.1
    U = random_links(Lx, Lt, 6)
    psi = W.gaussian_field((Lt, Lx, 2), 7)
    s3 = np.array([1.0, -1.0])
    got = s3 * w.apply_D(U, m, s3 * psi)
    assert np.max(np.abs(got - w.apply_D(U, m, psi, dagger=True))) < 1e-14


@pytest.mark.parametrize("dagger", [False, True])
def test_gauge_covariance(dagger):
    """U_x^mu -> g_x U_x^mu g_{x+mu}^*, psi -> g psi  =>  D'(g psi) = g (D psi)."""
    Lx, Lt, m = 10, 8, -1.3
    U = random_links(Lx, Lt, 9)
    g = np.exp(1j * 2 * np.pi * np.random.default_rng(11).random((Lt, Lx)))
    Ug = np.stack([g * U[0] * np.conj(np.roll(g, -1, axis=1)),
                   g * U[1] * np.conj(np.roll(g, -1, axis=0))])
    psi = W.gaussian_field((Lt, Lx, 2), 12)
    lhs = w.apply_D(Ug, m, g[..., None] * psi, dagger=dagger)
    rhs = g[..., None] * w.apply_D(U, m, psi, dagger=dagger)
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_mass_enters_as_identity():
    Lx, Lt = 6, 6
    U = random_links(Lx, Lt, 13)
    psi = W.gaussian_field((Lt, Lx, 2), 14)
    diff = w.apply_D(U, 0.7, psi) - w.apply_D(U, -0.2, psi)
    assert np.max(np.abs(diff - 0.9 * psi)) < 1e-14


def test_sparse_matrix_and_stencils_agree_with_apply():
    """Consistency of the three oracle forms of D and A (not a pin by itself)."""
    Lx, Lt, m = 8, 6, 0.3
    U = random_links(Lx, Lt, 15)
    psi = W.gaussian_field((Lt, Lx, 2), 16)
    Dm = w.dirac_matrix(U, m)
    assert np.max(np.abs(Dm @ psi.ravel() - w.apply_D(U, m, psi).ravel())) < 1e-14
    from oracle.multigrid import StencilOp
    disp, M = w.normal_stencil(U, m)
    assert len(disp) == 13
    assert np.max(np.abs(StencilOp(disp, M).apply(psi) - w.apply_A(U, m, psi))) < 1e-13


def test_normal_operator_positive():
    Lx, Lt, m = 8, 8, -2.0
    U = random_links(Lx, Lt, 17)
    psi = W.gaussian_field((Lt, Lx, 2), 18)
    Dpsi = w.apply_D(U, m, psi)
    assert abs(np.vdot(psi, w.apply_A(U, m, psi)) - np.vdot(Dpsi, Dpsi)) < 1e-12 * np.vdot(Dpsi, Dpsi).real
