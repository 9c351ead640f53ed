"""Smoothed aggregation (Sec. 3, the refinement applied to the vectors before
the prolongator is formed), plain FP64 numpy/scipy.

Test infrastructure only (see ``oracle/__init__.py``).

The paper smooths the block vectors v_j with one Richardson step before they
define the prolongator, the damping chosen so that the coarse operator has
the smallest condition number.  Readings taken here:
* the step acts on the columns of the tentative prolongator P (the
  chirality-split, block-orthonormal vectors of ``multigrid``):
  P_s(omega) = (1 - omega A) P, with A the operator of the level;
* the coarse operator is the Galerkin product A_c(omega) = P_s^dagger A P_s
  (P_s is no longer orthonormal, so A_c is not P_s^+ A P_s);
* "condition number" is the 2-norm one of the Hermitian positive A_c,
  lambda_max / lambda_min, and omega is searched in [0, 2 / lambda_max(A)],
  where 1 - omega A stays a contraction on every eigenvector of A;
* the V-cycle keeps the five steps of Sec. 2 with P_s in place of P.

Reach of the smoothed operator: A = D^dagger D couples a site only to its
nearest and diagonal neighbours (two hops in one direction carry
(1 + gamma_mu)(1 - gamma_mu) = 0), so a column of P_s spans its block and a
ring of one site around it, and A_c couples blocks whose rings come within one
site: with b x b blocks, b >= 4, still only neighbouring blocks (the 9-point
stencil), with 2 x 2 blocks blocks two apart as well (25 points).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import multigrid, wilson


def tentative_prolongator(V: np.ndarray, bx: int, bt: int) -> sp.csr_matrix:
    """P of Eq. P1 as a sparse matrix (fine dof x coarse dof), coarse dof in the
    order [t][x][s] of ``multigrid.prolong``: column (j, s) holds vector s's
    restriction to block j (chirality c of s only)."""
    Nv, Lt, Lx, n = V.shape
    Pm = multigrid.prolongator_matrix(V)                   # [Lt, Lx, n, 2 Nv]
    Ltc, Lxc, nc = Lt // bt, Lx // bx, 2 * Nv
    rows, cols, vals = [], [], []
    for t in range(Lt):
        for x in range(Lx):
            j = (t // bt) * Lxc + x // bx
            for a in range(n):
                for s in range(nc):
                    v = Pm[t, x, a, s]
                    if v != 0:
                        rows.append((t * Lx + x) * n + a)
                        cols.append(j * nc + s)
                        vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(Lt * Lx * n, Ltc * Lxc * nc))


def normal_matrix(U: np.ndarray, m: float) -> sp.csr_matrix:
    """A = D^dagger D as a sparse matrix (Sec. 1)."""
    D = wilson.dirac_matrix(U, m)
    return (D.conj().T @ D).tocsr()


def smoothed_prolongator(A: sp.spmatrix, P: sp.spmatrix, omega: float) -> sp.csr_matrix:
    """P_s = (1 - omega A) P (one Richardson step on every column)."""
    return (P - omega * (A @ P)).tocsr()


def coarse_operator(A: sp.spmatrix, Ps: sp.spmatrix) -> sp.csr_matrix:
    """A_c = P_s^dagger A P_s (Eq. Galerkin with the smoothed prolongator)."""
    return (Ps.conj().T @ (A @ Ps)).tocsr()


def condition_number(Ac: sp.spmatrix) -> float:
    ev = np.linalg.eigvalsh(Ac.toarray())
    return float(ev[-1] / ev[0])


def optimal_omega(A: sp.spmatrix, P: sp.spmatrix, lam_max: float, samples: int = 41,
                  refine: int = 40):
    """omega in [0, 2 / lam_max] minimising cond(A_c(omega)): the best of an
    even grid, then golden-section search on the bracket around it.  Returns
    (omega, cond)."""
    f = lambda w: condition_number(coarse_operator(A, smoothed_prolongator(A, P, w)))  # noqa: E731
    grid = np.linspace(0.0, 2.0 / lam_max, samples)
    vals = [f(w) for w in grid]
    k = int(np.argmin(vals))
    a, b = grid[max(k - 1, 0)], grid[min(k + 1, samples - 1)]
    g = (np.sqrt(5.0) - 1.0) / 2.0
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(refine):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = f(d)
    best = min([(vals[k], grid[k]), (fc, c), (fd, d)])
    return float(best[1]), float(best[0])


class TwoLevelSA:
    """Two-level V-cycle (the five steps of Sec. 2) with a smoothed prolongator
    and an exact coarse solve; the smoother is the level's frozen MR polynomial
    R = c0 + c1 A taken from a hierarchy of ``multigrid``."""

    def __init__(self, A: sp.spmatrix, Ps: sp.spmatrix, c0: float, c1: float):
        self.A, self.Ps, self.c0, self.c1 = A, Ps, c0, c1
        self.Ac = coarse_operator(A, Ps).toarray()
        self.L = np.linalg.cholesky(self.Ac)

    def smooth(self, b):
        return self.c0 * b + self.c1 * (self.A @ b)

    def vcycle(self, b: np.ndarray) -> np.ndarray:
        shape = b.shape
        b = b.ravel()
        x = self.smooth(b)
        rc = self.Ps.conj().T @ (b - self.A @ x)
        y = np.linalg.solve(self.L, rc)
        ec = np.linalg.solve(self.L.conj().T, y)
        x = x + self.Ps @ ec
        x = x + self.smooth(b - self.A @ x)
        return x.reshape(shape)


def block_reach(Ac: sp.spmatrix, Lxc: int, Ltc: int, nc: int) -> int:
    """Largest block distance (max over both axes, periodic) coupled by a
    nonzero entry of A_c."""
    Ac = Ac.tocoo()
    j, k = Ac.row // nc, Ac.col // nc
    dx = np.abs((j % Lxc) - (k % Lxc))
    dt = np.abs((j // Lxc) - (k // Lxc))
    dx = np.minimum(dx, Lxc - dx)
    dt = np.minimum(dt, Ltc - dt)
    nz = np.abs(Ac.data) > 0
    return int(np.max(np.maximum(dx, dt)[nz]))
