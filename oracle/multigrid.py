"""Adaptive multigrid hierarchy of the paper, plain FP64 numpy.

Test infrastructure only (see ``oracle/__init__.py``).

Levels are numbered l = 0 (finest, the paper's l = 1) .. L-1 (coarsest).
A level-l vector has shape [..., Lt_l, Lx_l, n_l]; n_0 = 2 spin components,
n_{l+1} = 2 * Nv_l.  Each level's dof split into two chiralities of h_l =
n_l / 2 components each: at level 0 the chirality is the sigma_3 eigenvalue
(spin 0 -> +1, spin 1 -> -1); at coarser levels the coarse dof
s = c * Nv + k carries chirality c (gamma_5 on level l+1 is
diag(+1 x Nv, -1 x Nv)).

Readings of the paper taken here (each listed in the design notes):
* Blocks S_j are fixed bx x bt squares of sites (Sec. 3: "4 x 4 squares").
* Each relaxed vector is split into its two chirality halves before the block
  orthonormalisation, giving 2 * Nv coarse dof per site.
* Orthonormalisation (Sec. 3, "orthogonal ... normalizing them to 1") is
  modified Gram-Schmidt in vector order, two passes, per (block, chirality).
* The relaxation step omega of Eq. relax is 1 / lambda_max(A_l) from a power
  iteration; nu = setup_sweeps sweeps are applied.
* The smoother (Sec. 4) is fixed by two under-relaxed minimum-residual steps
  on a random vector and then frozen: R = c0 + c1 A_l, R = R^dagger.
* V-cycle: the five steps of Sec. 2 with the last step read as the update
  x <- x + R (b - A x) (the printed closed form Eq. vcycle has a garbled sign;
  the steps are implemented, not the printed formula).
* Coarse operator blocks are stored per displacement d in {-1,0,1}^2,
  d = (dx + 1) + 3 (dt + 1); the displacement of a fine coupling i -> i + e is
  floor((o_i + e) / b) per axis, with o_i the in-block offset of i, so blocks
  on coarse extents <= 2 (where +1 and -1 name the same block) stay separate.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np
import scipy.linalg as sla

from . import wilson

COARSE_DISP = [(dx, dt) for dt in (-1, 0, 1) for dx in (-1, 0, 1)]   # index (dx+1) + 3(dt+1)


class Breakdown(RuntimeError):
    """Rank deficiency in the block orthonormalisation."""


# ---------------------------------------------------------------------------
# Level operators
# ---------------------------------------------------------------------------
class StencilOp:
    """y(x) = sum_e M[x, e] v(x + disp[e]) on a periodic lattice of n-dof sites."""

    def __init__(self, disp, M):
        self.disp = list(disp)
        self.M = M                                  # [Lt, Lx, ne, n, n]
        self.Lt, self.Lx = M.shape[:2]
        self.n = M.shape[-1]

    def apply(self, v: np.ndarray) -> np.ndarray:
        out = np.zeros(np.broadcast_shapes(v.shape), dtype=np.complex128)
        for e, (dx, dt) in enumerate(self.disp):
            vs = np.roll(v, shift=(-dt, -dx), axis=(-3, -2))
            out += np.einsum("txab,...txb->...txa", self.M[:, :, e], vs)
        return out

    def stencil(self):
        return self.disp, self.M

    def dense(self) -> np.ndarray:
        """Explicit matrix, index (x + Lx t) * n + a; aliased displacements add."""
        Lt, Lx, n = self.Lt, self.Lx, self.n
        N = Lt * Lx * n
        out = np.zeros((N, N), dtype=np.complex128)
        tt, xx = np.meshgrid(np.arange(Lt), np.arange(Lx), indexing="ij")
        a = np.arange(n)
        for e, (dx, dt) in enumerate(self.disp):
            i = (xx + Lx * tt).ravel()
            j = (((xx + dx) % Lx) + Lx * ((tt + dt) % Lt)).ravel()
            rows = (i[:, None, None] * n + a[None, :, None]) * np.ones((1, 1, n), int)
            cols = (j[:, None, None] * n + a[None, None, :]) * np.ones((1, n, 1), int)
            np.add.at(out, (rows, cols), self.M[:, :, e].reshape(-1, n, n))
        return out


class WilsonNormalOp:
    """Level-0 operator A = D^dagger D (Sec. 1), applied by its definition."""

    def __init__(self, U: np.ndarray, m: float):
        self.U, self.m = U, float(m)
        self.Lt, self.Lx = U.shape[1:]
        self.n = 2

    def apply(self, v):
        return wilson.apply_A(self.U, self.m, v)

    def stencil(self):
        return wilson.normal_stencil(self.U, self.m)

    def dense(self):
        D = wilson.dirac_matrix(self.U, self.m).toarray()
        return D.conj().T @ D


# ---------------------------------------------------------------------------
# Blocking (Sec. 3: S_j are fixed squares of neighbouring sites)
# ---------------------------------------------------------------------------
def block_map(Lx: int, Lt: int, bx: int, bt: int):
    """Coarse site j(i) = (t // bt) * (Lx // bx) + x // bx and in-block offset
    o(i) = (t % bt) * bx + x % bx for every fine site i = x + Lx t."""
    tt, xx = np.meshgrid(np.arange(Lt), np.arange(Lx), indexing="ij")
    coarse = (tt // bt) * (Lx // bx) + xx // bx
    offset = (tt % bt) * bx + xx % bx
    return coarse.ravel().astype(np.int32), offset.ravel().astype(np.int32)


def to_blocks(v: np.ndarray, bx: int, bt: int) -> np.ndarray:
    """[..., Lt, Lx, h] -> [..., Lt/bt, Lx/bx, bt*bx, h], offset (t%bt)*bx + x%bx."""
    *lead, Lt, Lx, h = v.shape
    w = v.reshape(*lead, Lt // bt, bt, Lx // bx, bx, h)
    w = np.moveaxis(w, -4, -3)              # [..., Ltc, Lxc, bt, bx, h]
    return w.reshape(*lead, Lt // bt, Lx // bx, bt * bx, h)


def from_blocks(w: np.ndarray, bx: int, bt: int) -> np.ndarray:
    *lead, Ltc, Lxc, b2, h = w.shape
    v = w.reshape(*lead, Ltc, Lxc, bt, bx, h)
    v = np.moveaxis(v, -3, -4)              # [..., Ltc, bt, Lxc, bx, h]
    return v.reshape(*lead, Ltc * bt, Lxc * bx, h)


def block_orthonormalise(E: np.ndarray, bx: int, bt: int, breakdown_tol: float = 1e-14):
    """Chirality-split block orthonormalisation of Nv vectors E[Nv, Lt, Lx, n].

    For every block S_j and chirality c, the restrictions u_k of Pi_c E_k to
    S_j are made orthonormal by modified Gram-Schmidt in order k = 0..Nv-1,
    two passes, then normalised (Sec. 3: v_1j = e'_j/|e'_j|; later vectors
    orthogonal to earlier ones and of unit norm).  Raises Breakdown when a
    vector loses all but 1e-14 of its norm to the projections.
    """
    Nv, Lt, Lx, n = E.shape
    h = n // 2
    out = np.zeros_like(E)
    for c in (0, 1):
        B = to_blocks(E[..., c * h:(c + 1) * h], bx, bt)       # [Nv, Ltc, Lxc, b2, h]
        shp = B.shape
        B = B.reshape(Nv, -1, shp[-2] * shp[-1])               # [Nv, Nc, b2*h]
        Q = np.zeros_like(B)
        for k in range(Nv):
            u = B[k].copy()
            norm0 = np.linalg.norm(u, axis=-1)
            for _ in range(2):
                for kk in range(k):
                    coef = np.einsum("ja,ja->j", np.conj(Q[kk]), u)
                    u = u - coef[:, None] * Q[kk]
            nrm = np.linalg.norm(u, axis=-1)
            if np.any(nrm <= breakdown_tol * norm0):
                raise Breakdown(f"block Gram-Schmidt breakdown at vector {k}, chirality {c}")
            Q[k] = u / nrm[:, None]
        out[..., c * h:(c + 1) * h] = from_blocks(Q.reshape(shp), bx, bt)
    return out


def prolongator_matrix(V: np.ndarray) -> np.ndarray:
    """Per-site n x 2Nv matrix of P (Eq. P1 with the intrinsic index s = c*Nv + k):
    P[i][c*h + a, c*Nv + k] = V_k(i)[c*h + a]."""
    Nv, Lt, Lx, n = V.shape
    h = n // 2
    P = np.zeros((Lt, Lx, n, 2 * Nv), dtype=np.complex128)
    for c in (0, 1):
        for k in range(Nv):
            P[:, :, c * h:(c + 1) * h, c * Nv + k] = V[k, :, :, c * h:(c + 1) * h]
    return P


def prolong(V: np.ndarray, bx: int, bt: int, ec: np.ndarray) -> np.ndarray:
    """e = P e_c: e(i) = sum_s P[i][:, s] e_c(j(i))[s] (Sec. 2 step 4)."""
    P = prolongator_matrix(V)
    ef = np.repeat(np.repeat(ec, bt, axis=-3), bx, axis=-2)     # e_c(j(i)) at every fine site
    return np.einsum("txas,...txs->...txa", P, ef)


def restrict(V: np.ndarray, bx: int, bt: int, r: np.ndarray) -> np.ndarray:
    """r_c = P^dagger r: r_c(j)[s] = sum_{i in S_j} sum_a conj(P[i][a, s]) r(i)[a] (Sec. 2 step 2)."""
    P = prolongator_matrix(V)
    per_site = np.einsum("txas,...txa->...txs", np.conj(P), r)
    return to_blocks(per_site, bx, bt).sum(axis=-2)


def galerkin(op, V: np.ndarray, bx: int, bt: int) -> StencilOp:
    """Coarse operator A_{l+1} = P^dagger A_l P (Eq. Galerkin) as a 9-point stencil.

    A_{l+1}[j, d] = sum_{i in S_j} sum_e [disp(i, e) = d] P(i)^dagger A_l[i, e] P(i + e),
    with A_l given as a stencil of blocks and disp(i, e) the block displacement
    floor((o_i + e) / b) per axis.
    """
    disp, M = op.stencil()
    Nv, Lt, Lx, n = V.shape
    if bx < 2 or bt < 2:
        raise ValueError("blocks must be at least 2 x 2")
    P = prolongator_matrix(V)
    Ltc, Lxc = Lt // bt, Lx // bx
    A = np.zeros((Ltc, Lxc, 9, 2 * Nv, 2 * Nv), dtype=np.complex128)
    tt, xx = np.meshgrid(np.arange(Lt), np.arange(Lx), indexing="ij")
    jt, jx, ot, ox = tt // bt, xx // bx, tt % bt, xx % bx
    for e, (ex, et) in enumerate(disp):
        P_nb = np.roll(P, shift=(-et, -ex), axis=(0, 1))       # P(i + e)
        T = np.einsum("txab,txbs->txas", M[:, :, e], P_nb)          # A_l[i, e] P(i + e)
        G = np.einsum("txar,txas->txrs", np.conj(P), T)             # P(i)^dagger (...)
        d = (np.floor_divide(ox + ex, bx) + 1) + 3 * (np.floor_divide(ot + et, bt) + 1)
        np.add.at(A, (jt, jx, d), G)
    return StencilOp(COARSE_DISP, A)


# ---------------------------------------------------------------------------
# Smoother (Sec. 4: two under-relaxed MR iterations, then held fixed)
# ---------------------------------------------------------------------------
def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def mr_smoother_coefficients(apply, eta: np.ndarray, omega: float = 0.8):
    """Two steps of MR with under-relaxation omega from x0 = 0, residual r0 = eta:
    alpha_k = <A r_k, r_k> / <A r_k, A r_k>, x_{k+1} = x_k + omega alpha_k r_k,
    r_{k+1} = r_k - omega alpha_k A r_k.  Then x_2 = R eta with the frozen
    polynomial R = c0 + c1 A, c0 = omega (alpha0 + alpha1),
    c1 = -omega^2 alpha0 alpha1.  Returns (c0, c1, alpha0, alpha1)."""
    r0 = eta
    q0 = apply(r0)
    a0 = vdot(q0, r0).real / vdot(q0, q0).real
    r1 = r0 - omega * a0 * q0
    q1 = apply(r1)
    a1 = vdot(q1, r1).real / vdot(q1, q1).real
    return omega * (a0 + a1), -omega * omega * a0 * a1, a0, a1


def power_lambda_max(apply, start: np.ndarray, iters: int) -> float:
    """Rayleigh quotient after `iters` power iterations from `start`."""
    v = start / np.linalg.norm(start)
    lam = 0.0
    for _ in range(iters):
        w = apply(v)
        lam = vdot(v, w).real
        v = w / np.linalg.norm(w)
    return float(lam)


# ---------------------------------------------------------------------------
# Hierarchy, setup and V-cycle
# ---------------------------------------------------------------------------
@dataclass
class Level:
    op: object                    # WilsonNormalOp or StencilOp
    Lx: int
    Lt: int
    n: int
    bx: int = 0                   # blocking to the next level (0 on the coarsest)
    bt: int = 0
    Nv: int = 0
    V: np.ndarray | None = None   # orthonormalised vectors [Nv, Lt, Lx, n]
    E: np.ndarray | None = None   # relaxed vectors before orthonormalisation
    c0: float = 0.0               # frozen smoother R = c0 + c1 A
    c1: float = 0.0
    omega_relax: float = 0.0
    eta: np.ndarray | None = None  # MR start kept for re-massing


@dataclass
class Hierarchy:
    levels: list
    m: float
    U: np.ndarray
    omega_mr: float = 0.8
    coarsest_chol: object = None
    coarsest_dense_max: int = 4096
    coarsest_tol: float = 1e-14
    stats: dict = field(default_factory=dict)

    @property
    def L(self):
        return len(self.levels)


def setup(U: np.ndarray, m: float, blocks, Nv, noise: np.ndarray, sweeps: int = 8,
          power_iters: int = 30, omega_mr: float = 0.8,
          coarsest_dense_max: int = 4096, refine_levels=(), refine_cycles: int = 30) -> Hierarchy:
    """Adaptive setup (Sec. 3, Eq. relax, Eq. P1, Eq. Galerkin), recursively.

    First pass, for each level l < L-1: omega = 1/lambda_max(A_l); Nv random
    vectors are relaxed with e <- (1 - omega A_l) e, `sweeps` times; split by
    chirality and block-orthonormalised; A_{l+1} = P^dagger A_l P.  The
    smoother is then fixed on each level, and the coarsest operator factored.
    Then one adaptive pass (``refine``, `refine_cycles` V-cycles) for each
    entry of `refine_levels` (0 = finest), in order.  `noise` is the flat
    buffer of random starts (layout in ``workloads.setup_noise``): the first
    pass's, then for each adaptive pass its random error and the starts of
    the levels below it.
    """
    _, Lt, Lx = U.shape
    levels = [Level(WilsonNormalOp(U, m), Lx, Lt, 2)]
    shapes = _level_shapes(Lx, Lt, blocks, Nv)
    first = sum((nv + 2) * lx * lt * n for (lx, lt, n), nv in zip(shapes[:-1], Nv))
    _build_levels(levels, blocks, Nv, noise[:first], sweeps, power_iters)
    H = Hierarchy(levels, float(m), U, omega_mr=omega_mr, coarsest_dense_max=coarsest_dense_max)
    _finish_levels(H)
    pos, Nv = first, list(Nv)
    for level in refine_levels:
        Nv[level] += 1
        lx, lt, n = _level_shapes(Lx, Lt, blocks, Nv)[level]
        e0 = noise[pos:pos + lx * lt * n].reshape(lt, lx, n)
        pos += lx * lt * n
        shapes = _level_shapes(Lx, Lt, blocks, Nv)
        tail = sum((nv + 2) * a * b * c for (a, b, c), nv in zip(shapes[level + 1:-1], Nv[level + 1:]))
        H, _, rho = refine(H, e0, refine_cycles, noise[pos:pos + tail], level, sweeps, power_iters)
        H.stats.setdefault("refine_rho", []).append(rho)
        pos += tail
    if pos != noise.size:
        raise ValueError(f"noise has {noise.size} entries, the set-up reads {pos}")
    return H


def _level_shapes(Lx, Lt, blocks, Nv):
    """(Lx_l, Lt_l, n_l) of every level."""
    out = [(Lx, Lt, 2)]
    for (bx, bt), nv in zip(blocks, Nv):
        lx, lt, _ = out[-1]
        out.append((lx // bx, lt // bt, 2 * nv))
    return out


def _build_levels(levels, blocks, Nv, noise, sweeps, power_iters, given=None):
    """Level-by-level body of the setup, from level len(levels) - 1 down.
    With `given` = (E, omega_relax, eta) the first level built takes the
    vectors E instead of relaxing random starts and keeps the given relaxation
    step and smoother start.  `noise` holds the random starts of the relaxed
    levels only, each in the per-level layout of ``workloads.setup_noise``."""
    first = len(levels) - 1
    pos = 0
    for l, ((bx, bt), nv) in enumerate(zip(blocks, Nv)):
        if l < first:
            continue
        lv = levels[l]
        size = lv.Lt * lv.Lx * lv.n
        if l == first and given is not None:
            E, lv.omega_relax, eta = given
            lv.eta = eta.copy()
        else:
            starts = noise[pos:pos + nv * size].reshape(nv, lv.Lt, lv.Lx, lv.n)
            pos += nv * size
            pw = noise[pos:pos + size].reshape(lv.Lt, lv.Lx, lv.n)
            pos += size
            lv.eta = noise[pos:pos + size].reshape(lv.Lt, lv.Lx, lv.n).copy()
            pos += size
            lam = power_lambda_max(lv.op.apply, pw, power_iters)
            lv.omega_relax = 1.0 / lam
            E = starts.copy()
            for _ in range(sweeps):
                E = E - lv.omega_relax * lv.op.apply(E)
        lv.E = E
        lv.V = block_orthonormalise(E, bx, bt)
        lv.bx, lv.bt, lv.Nv = bx, bt, nv
        coarse = galerkin(lv.op, lv.V, bx, bt)
        levels.append(Level(coarse, lv.Lx // bx, lv.Lt // bt, 2 * nv))


def _finish_levels(H: Hierarchy):
    for lv in H.levels[:-1]:
        lv.c0, lv.c1, _, _ = mr_smoother_coefficients(lv.op.apply, lv.eta, H.omega_mr)
    last = H.levels[-1]
    N = last.Lt * last.Lx * last.n
    if N <= H.coarsest_dense_max:
        L = np.linalg.cholesky(last.op.dense())                     # A = L L^dagger
        H.coarsest_chol = np.asfortranarray(L)
    else:
        H.coarsest_chol = None


def set_mass(H: Hierarchy, m: float) -> Hierarchy:
    """Reuse the vectors of the setup for another mass (Sec. 4): rebuild every
    Galerkin operator, the smoothers and the coarsest factor."""
    H.m = float(m)
    H.levels[0].op = WilsonNormalOp(H.U, m)
    for l in range(H.L - 1):
        lv = H.levels[l]
        H.levels[l + 1].op = galerkin(lv.op, lv.V, lv.bx, lv.bt)
    _finish_levels(H)
    return H


def smooth(lv: Level, b: np.ndarray) -> np.ndarray:
    """x = R b = c0 b + c1 A b."""
    return lv.c0 * b + lv.c1 * lv.op.apply(b)


def coarsest_solve(H: Hierarchy, b: np.ndarray) -> np.ndarray:
    """Exact solve on the coarsest level (Sec. 2, Sec. 4): dense Cholesky when the
    level has at most coarsest_dense_max unknowns, else CG to 1e-14 relative."""
    last = H.levels[-1]
    if H.coarsest_chol is not None:
        L = H.coarsest_chol
        y = sla.solve_triangular(L, b.reshape(-1), lower=True, check_finite=False)
        x = sla.solve_triangular(L, y, lower=True, trans="C", check_finite=False)
        return x.reshape(b.shape)
    from .krylov import cg
    x, _, _ = cg(last.op.apply, b, H.coarsest_tol, 100000)
    return x


def vcycle(H: Hierarchy, b: np.ndarray, l: int = 0) -> np.ndarray:
    """The five steps of the V-cycle (Sec. 2) on level l, recursively:
    1. x = R b;  2. r_c = P^dagger (b - A x);  3. e_c = V_{l+1} r_c;
    4. x = x + P e_c;  5. x = x + R (b - A x)."""
    if l == H.L - 1:
        return coarsest_solve(H, b)
    lv = H.levels[l]
    x = smooth(lv, b)
    rc = restrict(lv.V, lv.bx, lv.bt, b - lv.op.apply(x))
    ec = vcycle(H, rc, l + 1)
    x = x + prolong(lv.V, lv.bx, lv.bt, ec)
    x = x + smooth(lv, b - lv.op.apply(x))
    return x


# ---------------------------------------------------------------------------
# Adaptive refinement by V-cycles (Sec. 3, the adaptive step after the first
# vector set)
# ---------------------------------------------------------------------------
def vcycle_error_propagation(H: Hierarchy, e0: np.ndarray, ncycles: int, level: int = 0) -> np.ndarray:
    """The V-cycle of level `level` applied to an error with no source,
    `ncycles` times (Sec. 3): one cycle on A_l x = 0 from x = -e leaves the
    error e <- e - V_l(A_l e), with V_l the V-cycle of Sec. 2 from level l down
    as a linear map of its right-hand side."""
    A = H.levels[level].op.apply
    e = e0.copy()
    for _ in range(ncycles):
        e = e - vcycle(H, A(e), level)
    return e


def energy_norm(H: Hierarchy, e: np.ndarray, level: int = 0) -> float:
    """|e|_A = sqrt(<e, A_l e>)."""
    return float(np.sqrt(vdot(e, H.levels[level].op.apply(e)).real))


def refine(H: Hierarchy, e0: np.ndarray, ncycles: int, noise: np.ndarray, level: int = 0,
           sweeps: int = 8, power_iters: int = 30):
    """One adaptive pass on level `level` (Sec. 3; recursive for coarser
    levels): run `ncycles` V-cycles of that level on the random error e0; the
    error e'' that survives is restricted to every block S_j, made orthogonal
    there (per chirality) to the block's current vectors, normalised, and
    appended as vector Nv_l + 1 of the level.  Finer levels are kept; the level
    keeps its relaxation step and smoother start; the Galerkin operators below
    it, the coarser levels' vectors (first-pass setup on the new coarse
    operators, from `noise`: the random starts of the levels below `level`
    for the refined Nv, as laid out by ``workloads.refine_noise``), the
    smoothers and the coarsest factor are rebuilt.

    Returns (H', e'', rho) with rho = (|e''|_A / |e0|_A)^(1/ncycles), the
    measured error reduction per cycle of the level's V-cycle in H.
    """
    if not 0 <= level < H.L - 1:
        raise ValueError("level must have a coarser level below it")
    e = vcycle_error_propagation(H, e0, ncycles, level)
    rho = (energy_norm(H, e, level) / energy_norm(H, e0, level)) ** (1.0 / ncycles)
    blocks = [(lv.bx, lv.bt) for lv in H.levels[:-1]]
    Nv = [lv.Nv for lv in H.levels[:-1]]
    Nv[level] += 1
    lv = H.levels[level]
    E = np.concatenate([lv.V, e[None]], axis=0)
    levels = [replace(x) for x in H.levels[:level]]
    levels.append(Level(lv.op if level > 0 else WilsonNormalOp(H.U, H.m), lv.Lx, lv.Lt, lv.n))
    _build_levels(levels, blocks, Nv, noise, sweeps, power_iters,
                  given=(E, lv.omega_relax, lv.eta))
    H2 = Hierarchy(levels, H.m, H.U, omega_mr=H.omega_mr,
                   coarsest_dense_max=H.coarsest_dense_max, coarsest_tol=H.coarsest_tol,
                   stats={k: list(v) if isinstance(v, list) else v for k, v in H.stats.items()})
    _finish_levels(H2)
    return H2, e, float(rho)
