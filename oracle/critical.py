"""Critical mass and near-critical masses (Sec. 4: mass gap m_hat = m - m_crit).

Test infrastructure only (see ``oracle/__init__.py``).

Reading: D(m) = D_0 + m, so D(m) is singular exactly at m = -lambda for each
real eigenvalue lambda of D_0 = D(m=0).  m_crit is the first such point met
when m comes down from large positive values: m_crit = -(smallest real
eigenvalue of D_0).  A near-critical mass is m_crit + delta with delta the
largest entry of NEAR_CRITICAL_DELTAS for which lambda_min(A) < 1e-5, where
lambda_min(A(m)) = sigma_min(D(m))^2 = min |eig(sigma_3 D(m))|^2 (sigma_3 D is
Hermitian by gamma_5-hermiticity).

Library primitives: scipy's ARPACK shift-invert eigensolvers on the explicit
sparse matrix of D (``wilson.dirac_matrix``).  Parity unpinned beyond the
small-lattice check against a dense eigendecomposition in the tests.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import wilson

NEAR_CRITICAL_DELTAS = (1e-1, 5e-2, 2e-2, 1e-2, 5e-3, 2e-3, 1e-3, 5e-4, 2e-4, 1e-4, 5e-5, 2e-5, 1e-5)


def _sigma3(n_sites: int) -> sp.dia_matrix:
    return sp.diags(np.tile([1.0, -1.0], n_sites)).astype(np.complex128)


def real_eigenvalues_D0(U: np.ndarray, k: int = 24, shift: float = 1.6, rel_imag: float = 1e-7):
    """Real eigenvalues of D_0 among the k eigenvalues nearest `shift`.

    Dense eigendecomposition for lattices up to 32 x 32, shift-invert ARPACK
    otherwise.  An eigenvalue counts as real when |Im| <= rel_imag * |lambda|.
    """
    D0 = wilson.dirac_matrix(U, 0.0)
    n = D0.shape[0]
    if n <= 2 * 32 * 32:
        lam = np.linalg.eigvals(D0.toarray())
    else:
        lam = spla.eigs(D0.tocsc(), k=k, sigma=shift, which="LM", return_eigenvectors=False,
                        tol=1e-12)
    real = np.sort(lam[np.abs(lam.imag) <= rel_imag * np.abs(lam)].real)
    return real, lam


def lambda_min_A(U: np.ndarray, m: float) -> float:
    """Smallest eigenvalue of A(m) = D(m)^dagger D(m), as min |eig(sigma_3 D(m))|^2."""
    D = wilson.dirac_matrix(U, m)
    n = D.shape[0]
    H = (_sigma3(n // 2) @ D).tocsc()
    if n <= 2 * 16 * 16:
        ev = np.linalg.eigvalsh(H.toarray())
    else:
        ev = spla.eigsh(H, k=2, sigma=0.0, which="LM", return_eigenvectors=False, tol=1e-12)
    return float(np.min(np.abs(ev)) ** 2)


def _min_abs_eig_H(U: np.ndarray, m: float, D0=None) -> float:
    """min |eig(sigma_3 D(m))| by shift-invert Lanczos at 0."""
    D = wilson.dirac_matrix(U, 0.0) if D0 is None else D0
    n = D.shape[0]
    H = (_sigma3(n // 2) @ (D + m * sp.identity(n, dtype=np.complex128, format="csr"))).tocsc()
    ev = spla.eigsh(H, k=1, sigma=0.0, which="LM", return_eigenvectors=False, tol=1e-12)
    return float(np.min(np.abs(ev)))


def critical_mass_by_flow(U: np.ndarray, m_lo: float = -2.4, m_hi: float = -1.9, step: float = 0.01,
                          zero: float = 1e-7):
    """m_crit for large lattices: D(m) is singular where an eigenvalue of the
    Hermitian sigma_3 D(m) crosses zero, i.e. where mu(m) = min |eig(sigma_3 D(m))|
    vanishes.  Scan mu on a grid from heavy to light mass, refine each local
    minimum by golden-section search, and return the heaviest mass where the
    minimum is below `zero` (None if there is none)."""
    D0 = wilson.dirac_matrix(U, 0.0)
    ms = np.arange(m_hi, m_lo - 1e-12, -step)
    mu = [_min_abs_eig_H(U, m, D0) for m in ms]
    g = (np.sqrt(5.0) - 1.0) / 2.0
    for i in range(1, len(ms) - 1):
        if mu[i] <= mu[i - 1] and mu[i] <= mu[i + 1]:
            a, b = ms[i + 1], ms[i - 1]
            c, d = b - g * (b - a), a + g * (b - a)
            fc, fd = _min_abs_eig_H(U, c, D0), _min_abs_eig_H(U, d, D0)
            for _ in range(60):
                if fc < fd:
                    b, d, fd = d, c, fc
                    c = b - g * (b - a)
                    fc = _min_abs_eig_H(U, c, D0)
                else:
                    a, c, fc = c, d, fd
                    d = a + g * (b - a)
                    fd = _min_abs_eig_H(U, d, D0)
                if b - a < 1e-13:
                    break
            m_star = 0.5 * (a + b)
            if _min_abs_eig_H(U, m_star, D0) < zero:
                return float(m_star)
    return None


def near_critical_mass(U: np.ndarray, threshold: float = 1e-5):
    """Returns dict(m_crit, m_nc, delta, lambda_min) or None when D_0 has no real
    eigenvalue near the physical branch (then the caller advances the seed)."""
    if U.shape[1] * U.shape[2] <= 64 * 64:
        real, _ = real_eigenvalues_D0(U)
        if real.size == 0:
            return None
        m_crit = -float(real[0])
    else:
        m_crit = critical_mass_by_flow(U)
        if m_crit is None:
            return None
    for delta in NEAR_CRITICAL_DELTAS:
        lam = lambda_min_A(U, m_crit + delta)
        if lam < threshold:
            return {"m_crit": m_crit, "m_nc": m_crit + delta, "delta": delta, "lambda_min": lam}
    return None
