"""Conjugate gradients on A x = b, plain and preconditioned (Sec. 4, MG-CG).

Test infrastructure only (see ``oracle/__init__.py``).

Reading: the V-cycle acts on the residual (standard PCG, z = V r); the paper's
"applied ... to the CG direction vector" would not give a CG method.  The
stopping test is the true residual |b - A x| / |b| <= tol recomputed from x;
when the recursive residual reaches tol first, the true residual replaces it
and the iteration restarts from the steepest-descent direction.
"""
from __future__ import annotations

import numpy as np


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def pcg(apply, b: np.ndarray, tol: float, maxiter: int, precond=None):
    """Returns (x, iterations, info) with info = {"true_res", "history", "applies"}.

    applies counts the operator applications of the Krylov loop itself
    (one per iteration plus the true-residual checks).
    """
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    info = {"history": [], "applies": 0, "true_res": 0.0}
    if bnorm == 0.0:
        return x, 0, info
    M = (lambda v: v) if precond is None else precond
    r = b.copy()
    z = M(r)
    p = z.copy()
    rz = _dot(r, z).real
    it = 0
    while it < maxiter:
        q = apply(p)
        info["applies"] += 1
        pq = _dot(p, q).real
        if not pq > 0.0:
            raise FloatingPointError("CG breakdown: <p, A p> <= 0")
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rel = np.linalg.norm(r) / bnorm
        info["history"].append(rel)
        if rel <= tol:
            r = b - apply(x)
            info["applies"] += 1
            true_rel = np.linalg.norm(r) / bnorm
            if true_rel <= tol:
                info["true_res"] = float(true_rel)
                return x, it, info
            z = M(r)
            p = z.copy()
            rz = _dot(r, z).real
            continue
        z = M(r)
        rz_new = _dot(r, z).real
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    info["true_res"] = float(np.linalg.norm(b - apply(x)) / bnorm)
    return x, it, info


def cg(apply, b: np.ndarray, tol: float, maxiter: int):
    """Plain CG (the unpreconditioned baseline of Sec. 4)."""
    return pcg(apply, b, tol, maxiter, precond=None)


def mgcg(H, b: np.ndarray, tol: float, maxiter: int = 1000):
    """MG-CG: CG on the fine A preconditioned by one V-cycle per iteration (Sec. 4)."""
    from .multigrid import vcycle
    return pcg(H.levels[0].op.apply, b, tol, maxiter, precond=lambda r: vcycle(H, r))
