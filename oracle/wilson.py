"""Wilson-Dirac operator of the paper, Sec. 1 (the display defining D_{x,y}).

Test infrastructure only (see ``oracle/__init__.py``).

    D_{x,y} = -1/2 sum_mu [ (1 - gamma_mu) U_x^mu delta_{x+mu,y}
                            + (1 + gamma_mu) U_{x-mu}^{mu*} delta_{x-mu,y} ]
              + (2d + m) delta_{x,y}

in d = 2 with the diagonal taken as written, 2d + m = 4 + m.  Readings:
gamma_1 = sigma_1 on the x links (mu = 0 here), gamma_2 = sigma_2 on the t
links (mu = 1), gamma_5 = sigma_3.  The gauge field is periodic; the fermion
field is periodic in x and antiperiodic in t, so a hop across the t boundary
carries a factor -1.  A = D^dagger D (Sec. 1, normal equations).

Layouts: links U[mu][t][x] (complex128, unit modulus), spinors [..., t, x, spin].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

SIGMA1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SIGMA2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SIGMA3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
GAMMA = (SIGMA1, SIGMA2)          # gamma_mu for mu = x, t
ID2 = np.eye(2, dtype=np.complex128)
DIM = 2                            # d in (2d + m)

# Unit displacements (dx, dt) of the two directions.
UNIT = ((1, 0), (0, 1))


def fermion_shift(psi: np.ndarray, dx: int, dt: int) -> np.ndarray:
    """Return phi(x) = psi(x + dx*xhat + dt*that) with |dx|+|dt| <= 1.

    The x direction is periodic; the t direction is antiperiodic, so the
    value fetched across the t boundary is negated.
    """
    out = np.roll(psi, shift=(-dt, -dx), axis=(-3, -2))
    Lt = psi.shape[-3]
    if dt == 1:
        out[..., Lt - 1, :, :] *= -1.0      # psi(Lt) = -psi(0)
    elif dt == -1:
        out[..., 0, :, :] *= -1.0           # psi(-1) = -psi(Lt-1)
    return out


def _proj(matrix: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 2x2 spin matrix to every site of psi [..., t, x, 2]."""
    return np.einsum("ab,...b->...a", matrix, psi)


def apply_D(U: np.ndarray, m: float, psi: np.ndarray, dagger: bool = False) -> np.ndarray:
    """(D psi)_x, or (D^dagger psi)_x when dagger is set.

    D^dagger exchanges the two projectors: its forward hop carries
    (1 + gamma_mu) U_x^mu and its backward hop (1 - gamma_mu) U_{x-mu}^{mu*}
    (the conjugate transpose of the display; gamma_mu is Hermitian).
    """
    out = (2 * DIM + m) * psi
    for mu, (dx, dt) in enumerate(UNIT):
        g = GAMMA[mu]
        p_fwd = ID2 + g if dagger else ID2 - g
        p_bwd = ID2 - g if dagger else ID2 + g
        u_here = U[mu]                                           # U_x^mu
        u_back = np.roll(U[mu], shift=(dt, dx), axis=(0, 1))     # U_{x-mu}^mu (periodic)
        fwd = u_here[..., None] * fermion_shift(psi, dx, dt)
        bwd = np.conj(u_back)[..., None] * fermion_shift(psi, -dx, -dt)
        out = out - 0.5 * (_proj(p_fwd, fwd) + _proj(p_bwd, bwd))
    return out


def apply_A(U: np.ndarray, m: float, psi: np.ndarray) -> np.ndarray:
    """A psi = D^dagger (D psi), the normal operator of Sec. 1."""
    return apply_D(U, m, apply_D(U, m, psi), dagger=True)


def site_index(x: int, t: int, Lx: int) -> int:
    return x + Lx * t


def dirac_matrix(U: np.ndarray, m: float) -> sp.csr_matrix:
    """Explicit sparse matrix of D, entry by entry from the display in Sec. 1.

    Row/column index = 2 * (x + Lx * t) + spin.  Built with plain loops over
    sites, independently of apply_D, for small-lattice checks and for the
    critical-mass finder.
    """
    _, Lt, Lx = U.shape
    rows, cols, vals = [], [], []

    def put(i_site, j_site, block):
        for a in range(2):
            for b in range(2):
                if block[a, b] != 0:
                    rows.append(2 * i_site + a)
                    cols.append(2 * j_site + b)
                    vals.append(block[a, b])

    for t in range(Lt):
        for x in range(Lx):
            i = site_index(x, t, Lx)
            put(i, i, (2 * DIM + m) * ID2)
            for mu, (dx, dt) in enumerate(UNIT):
                g = GAMMA[mu]
                # forward neighbour y = x + mu
                xf, tf = (x + dx) % Lx, t + dt
                sign_f = -1.0 if tf == Lt else 1.0
                tf %= Lt
                put(i, site_index(xf, tf, Lx), -0.5 * sign_f * U[mu, t, x] * (ID2 - g))
                # backward neighbour y = x - mu, link U_{x-mu}^mu
                xb, tb = (x - dx) % Lx, t - dt
                sign_b = -1.0 if tb == -1 else 1.0
                tb %= Lt
                put(i, site_index(xb, tb, Lx),
                    -0.5 * sign_b * np.conj(U[mu, tb, xb]) * (ID2 + g))
    n = 2 * Lx * Lt
    return sp.csr_matrix(sp.coo_matrix((vals, (rows, cols)), shape=(n, n)))


def wilson_stencil(U: np.ndarray, m: float, dagger: bool = False):
    """D (or D^dagger) as a 5-point stencil of 2x2 blocks.

    Returns (disp, M) with disp the list of displacements (dx, dt) and
    M[t, x, e] the 2x2 block coupling site x to x + disp[e] (wrapped); the
    antiperiodic factor of hops across the t boundary is folded into M.
    """
    _, Lt, Lx = U.shape
    disp = [(0, 0)]
    blocks = [np.broadcast_to((2 * DIM + m) * ID2, (Lt, Lx, 2, 2)).copy()]
    tt = np.arange(Lt)[:, None] * np.ones((1, Lx))
    for mu, (dx, dt) in enumerate(UNIT):
        g = GAMMA[mu]
        p_fwd = ID2 + g if dagger else ID2 - g
        p_bwd = ID2 - g if dagger else ID2 + g
        sign_f = np.where((tt == Lt - 1) & (dt == 1), -1.0, 1.0)
        sign_b = np.where((tt == 0) & (dt == 1), -1.0, 1.0)
        u_back = np.roll(U[mu], shift=(dt, dx), axis=(0, 1))
        disp.append((dx, dt))
        blocks.append(-0.5 * (sign_f * U[mu])[..., None, None] * p_fwd)
        disp.append((-dx, -dt))
        blocks.append(-0.5 * (sign_b * np.conj(u_back))[..., None, None] * p_bwd)
    return disp, np.stack(blocks, axis=2)


def normal_stencil(U: np.ndarray, m: float):
    """A = D^dagger D as a stencil of 2x2 blocks over displacements |e|_1 <= 2.

    A[x, e] = sum over e1 + e2 = e of Ddag[x, e1] D[x + e1, e2]
    (matrix product of the two 5-point stencils, written out).
    """
    dd, Md = wilson_stencil(U, m, dagger=True)
    d_, M = wilson_stencil(U, m, dagger=False)
    acc = {}
    for e1, (ax, at) in enumerate(dd):
        M_shift = np.roll(M, shift=(-at, -ax), axis=(0, 1))     # D[x + e1, .]
        for e2, (bx, bt) in enumerate(d_):
            key = (ax + bx, at + bt)
            blk = np.einsum("txab,txbc->txac", Md[:, :, e1], M_shift[:, :, e2])
            acc[key] = acc.get(key, 0) + blk
    disp = sorted(acc.keys(), key=lambda k: (k[1], k[0]))
    return disp, np.stack([acc[k] for k in disp], axis=2)
