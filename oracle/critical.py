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
sparse matrix of D (``wilson.dirac_matrix``).  Pinned on small lattices: the
spectral-flow finder used for large lattices against the real eigenvalues of
a dense D_0, and the singularity of D(m_crit) by a dense SVD.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import wilson

NEAR_CRITICAL_DELTAS = (1e-1, 5e-2, 2e-2, 1e-2, 5e-3, 2e-3, 1e-3, 5e-4, 2e-4, 1e-4, 5e-5, 2e-5, 1e-5)


def _sigma3(n_sites: int) -> sp.dia_matrix:
    return sp.diags(np.tile([1.0, -1.0], n_sites)).astype(np.complex128)


def _shift_invert(M: sp.spmatrix) -> spla.LinearOperator:
    """x -> M^-1 x by a sparse LU of M, for ARPACK's shift-invert mode.  The
    lattice matrices have a symmetric sparsity pattern, so the fill-reducing
    ordering is the minimum-degree ordering of M + M^T (far less fill than the
    column ordering scipy's eigensolvers use by default on 2D lattices)."""
    lu = spla.splu(M.tocsc(), permc_spec="MMD_AT_PLUS_A",
                   options=dict(SymmetricMode=True, DiagPivotThresh=0.1))
    return spla.LinearOperator(M.shape, matvec=lu.solve, dtype=np.complex128)


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
        n0 = D0.shape[0]
        lam = spla.eigs(D0.tocsc(), k=k, sigma=shift, which="LM", return_eigenvectors=False,
                        tol=1e-12,
                        OPinv=_shift_invert(D0 - shift * sp.identity(n0, dtype=np.complex128, format="csc")))
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
        ev = spla.eigsh(H, k=2, sigma=0.0, which="LM", return_eigenvectors=False, tol=1e-12,
                        OPinv=_shift_invert(H))
    return float(np.min(np.abs(ev)) ** 2)


def nearest_eig_H(U: np.ndarray, m: float, D0=None):
    """(lambda, dlambda/dm): the eigenvalue of the Hermitian H(m) = sigma_3 D(m)
    nearest zero, by shift-invert Lanczos at 0, and its derivative in m.  Since
    dH/dm = sigma_3, the derivative is <v, sigma_3 v> for the unit eigenvector v
    (first-order perturbation theory, Hellmann-Feynman)."""
    D = wilson.dirac_matrix(U, 0.0) if D0 is None else D0
    n = D.shape[0]
    s3 = _sigma3(n // 2)
    H = (s3 @ (D + m * sp.identity(n, dtype=np.complex128, format="csr"))).tocsc()
    ev, vec = spla.eigsh(H, k=1, sigma=0.0, which="LM", tol=1e-13, OPinv=_shift_invert(H))
    v = vec[:, 0] / np.linalg.norm(vec[:, 0])
    return float(ev[0]), float(np.real(np.vdot(v, s3 @ v)))


def critical_mass_by_flow(U: np.ndarray, m_lo: float = -2.4, m_hi: float = -1.9,
                          zero: float = 1e-11, newton_below: float = 1e-3, safety: float = 0.9,
                          max_evals: int = 2000):
    """m_crit for large lattices: the heaviest mass at which an eigenvalue of
    the Hermitian H(m) = sigma_3 D(m) crosses zero (D(m) is singular exactly
    there).  Changing m by dm moves every eigenvalue of H by at most |dm|
    (dH/dm = sigma_3 has norm 1), so mu(m) = min |eig H(m)| is 1-Lipschitz and
    no crossing lies within mu(m) of m.  Coming down from m_hi in steps of
    safety * mu(m) therefore cannot pass over a crossing.  Once mu < newton_below
    the crossing ahead is located by Newton's method on the nearest eigenvalue
    (derivative from nearest_eig_H); a Newton run that leaves the interval
    (m - 2 mu / |slope| ... m], or stops contracting, is discarded and the
    scan goes on.  Returns None if no crossing lies above m_lo."""
    D0 = wilson.dirac_matrix(U, 0.0)
    m, evals = m_hi, 0
    while m > m_lo and evals < max_evals:
        lam, slope = nearest_eig_H(U, m, D0)
        evals += 1
        mu = abs(lam)
        if mu < zero:
            return float(m)
        if mu < newton_below and abs(slope) > 1e-3:
            mn, ln, ok = m, lam, False
            for _ in range(40):
                step = -ln / slope
                mn_new = mn + step
                if not (m - 4.0 * mu / abs(slope) <= mn_new <= m + 1e-15):
                    break
                ln_new, slope_new = nearest_eig_H(U, mn_new, D0)
                evals += 1
                if abs(ln_new) > 0.5 * abs(ln) and abs(ln_new) > zero:
                    break
                mn, ln, slope = mn_new, ln_new, slope_new
                if abs(ln) < zero:
                    ok = True
                    break
            if ok:
                return float(mn)
        m -= safety * mu
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
