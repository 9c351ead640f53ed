"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no arithmetic of the multigrid method.  It produces:

* quenched U(1) gauge fields from the Wilson plaquette action of the
  paper's Results section (S = -beta * sum_p Re U_p; the printed sign is
  garbled, the weight used here is exp(-S) with that S, so that beta > 0
  orders the links), by Metropolis sweeps from a cold start;
* complex Gaussian source vectors chi (E|z|^2 = 1);
* the random starting vectors the adaptive setup draws (Eq. "relax" starts,
  the power-iteration start and the minimum-residual start of the smoother),
  passed to both sides as an input so that no side re-implements a generator;
* gauge diagnostics: the mean plaquette and the topological charge Q.

Array conventions (both sides): a lattice field is indexed [t][x] with the
site index x + Lx * t.  Links are ``U[mu][t][x]`` with mu = 0 the x
direction and mu = 1 the t direction; a spinor is ``psi[t][x][spin]``.
All random numbers come from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "quenched_u1_angles",
    "links_from_angles",
    "quenched_u1",
    "plaquette_angles",
    "mean_plaquette",
    "topological_charge",
    "gaussian_field",
    "level_shapes",
    "setup_noise",
    "setup_noise_len",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def plaquette_angles(theta: np.ndarray) -> np.ndarray:
    """Angle of U_p(x) = U_x^0 U_{x+0}^1 U_{x+1}^{0*} U_x^{1*}, shape [Lt, Lx].

    theta[0] holds the x-links and theta[1] the t-links, both [Lt, Lx].
    """
    th0, th1 = theta[0], theta[1]
    return (th0 + np.roll(th1, -1, axis=1) - np.roll(th0, -1, axis=0) - th1)


def mean_plaquette(theta: np.ndarray) -> float:
    """Volume average of Re U_p."""
    return float(np.mean(np.cos(plaquette_angles(theta))))


def topological_charge(theta: np.ndarray) -> float:
    """Q = (1/2pi) sum_x arg U_p(x) with arg in (-pi, pi]; an integer on a torus."""
    ph = plaquette_angles(theta)
    arg = np.angle(np.exp(1j * ph))
    arg = np.where(arg <= -math.pi, arg + 2 * math.pi, arg)
    return float(np.sum(arg) / (2 * math.pi))


def _metropolis_half(theta, mu, parity, beta, eps, rng):
    """Update every link of direction mu whose other coordinate has the given
    parity.  Such links share no plaquette, so they are updated at once."""
    Lt, Lx = theta.shape[1:]
    u_prop = rng.random((Lt, Lx))
    u_acc = rng.random((Lt, Lx))
    return _metropolis_half_u(theta, mu, parity, beta, eps, u_prop, u_acc)


def _metropolis_half_u(theta, mu, parity, beta, eps, u_prop, u_acc):
    """The half-sweep of _metropolis_half with its uniforms given: u_prop
    proposes theta' = theta + eps (2 u_prop - 1), u_acc accepts (per site)."""
    Lt, Lx = theta.shape[1:]
    th0, th1 = theta[0], theta[1]
    if mu == 0:
        # link theta0(x,t) enters p(x,t) with + and p(x,t-1) with -.
        a = np.roll(th1, -1, axis=1) - np.roll(th0, -1, axis=0) - th1           # p(x,t) = th0 + a
        b = (np.roll(th0, 1, axis=0) + np.roll(np.roll(th1, -1, axis=1), 1, axis=0)
             - np.roll(th1, 1, axis=0))                                           # p(x,t-1) = b - th0
        mask = (np.arange(Lt)[:, None] % 2 == parity) & np.ones((1, Lx), bool)
        cur = th0
    else:
        # link theta1(x,t) enters p(x,t) with - and p(x-1,t) with +.
        a = th0 - np.roll(th0, -1, axis=0) + np.roll(th1, -1, axis=1)           # p(x,t) = a - th1
        b = (np.roll(th0, 1, axis=1) - np.roll(np.roll(th0, -1, axis=0), 1, axis=1)
             - np.roll(th1, 1, axis=1))                                           # p(x-1,t) = b + th1
        mask = (np.arange(Lx)[None, :] % 2 == parity) & np.ones((Lt, 1), bool)
        cur = th1
    new = cur + eps * (2.0 * u_prop - 1.0)
    if mu == 0:
        s_old = np.cos(cur + a) + np.cos(b - cur)
        s_new = np.cos(new + a) + np.cos(b - new)
    else:
        s_old = np.cos(a - cur) + np.cos(b + cur)
        s_new = np.cos(a - new) + np.cos(b + new)
    d_s = -beta * (s_new - s_old)                      # S = -beta sum Re U_p
    accept = mask & (u_acc < np.exp(np.minimum(-d_s, 0.0)))
    cur[accept] = np.mod(new[accept] + math.pi, 2 * math.pi) - math.pi
    return int(np.count_nonzero(accept))


def quenched_u1_angles(Lx: int, Lt: int, beta: float, sweeps: int, seed: int,
                       eps: float = 1.0) -> np.ndarray:
    """Link angles theta[2][Lt][Lx] after `sweeps` Metropolis sweeps from theta = 0.

    One sweep visits every link once, direction by direction, each direction
    in two halves by the parity of the other coordinate.  Proposal
    theta' = theta + eps * (2u - 1); accept if u2 < exp(-dS).  Lx and Lt must
    be even so that the two halves share no plaquette across the boundary.
    """
    if Lx % 2 or Lt % 2:
        raise ValueError("Lx and Lt must be even")
    rng = _rng(seed)
    theta = np.zeros((2, Lt, Lx), dtype=np.float64)
    for _ in range(int(sweeps)):
        for mu in (0, 1):
            for parity in (0, 1):
                _metropolis_half(theta, mu, parity, float(beta), float(eps), rng)
    return theta


# ---------------------------------------------------------------------------
# Counter-based uniforms (Philox4x32-10, Salmon, Moraes, Dror, Shaw, SC'11) for
# the Metropolis generator that has a GPU twin: every uniform is a function of
# (seed, sweep, direction, parity, site), so both sides draw the same numbers
# without sharing a stream.
# ---------------------------------------------------------------------------
PHILOX_M = (0xD2511F53, 0xCD9E8D57)      # round multipliers
PHILOX_W = (0x9E3779B9, 0xBB67AE85)      # key increments (golden ratio, sqrt(3) - 1)
_M32 = np.uint64(0xFFFFFFFF)


def philox4x32(ctr, key, rounds: int = 10):
    """Philox4x32 block function on uint32 counters ctr[..., 4] with key (k0, k1):
    each round multiplies counter words 0 and 2 by M0 and M1 into 64-bit
    products (hi, lo) and forms (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the
    key is advanced by (W0, W1) before every round but the first."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0, k1 = np.uint64(key[0]), np.uint64(key[1])
    for r in range(rounds):
        if r:
            k0 = (k0 + np.uint64(PHILOX_W[0])) & _M32
            k1 = (k1 + np.uint64(PHILOX_W[1])) & _M32
        p0 = np.uint64(PHILOX_M[0]) * c[0]
        p1 = np.uint64(PHILOX_M[1]) * c[2]
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ k0) & _M32, p1 & _M32,
             ((p0 >> np.uint64(32)) ^ c[3] ^ k1) & _M32, p0 & _M32]
    return np.stack(c, axis=-1).astype(np.uint32)


def uniform53(hi, lo):
    """A double in [0, 1) from two uint32 words: 27 + 26 bits, exact."""
    return ((np.asarray(hi, np.uint64) >> np.uint64(5)).astype(np.float64) * 67108864.0
            + (np.asarray(lo, np.uint64) >> np.uint64(6)).astype(np.float64)) * 2.0 ** -53


def metropolis_uniforms(Lx: int, Lt: int, seed: int, sweep: int, mu: int, parity: int):
    """(u_prop, u_acc)[Lt][Lx] of one half-sweep: Philox4x32-10 at counter
    (t Lx + x, 4 sweep + 2 mu + parity (low, high 32 bits), 0), key (seed low,
    seed high); u_prop from words 0, 1 and u_acc from words 2, 3."""
    half = 4 * int(sweep) + 2 * int(mu) + int(parity)
    ctr = np.zeros((Lt * Lx, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(Lt * Lx, dtype=np.uint64)
    ctr[:, 1] = half & 0xFFFFFFFF
    ctr[:, 2] = half >> 32
    out = philox4x32(ctr, (int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF))
    u_prop = uniform53(out[:, 0], out[:, 1]).reshape(Lt, Lx)
    u_acc = uniform53(out[:, 2], out[:, 3]).reshape(Lt, Lx)
    return u_prop, u_acc


def quenched_u1_angles_counter(Lx: int, Lt: int, beta: float, sweeps: int, seed: int,
                               eps: float = 1.0, theta=None, first_sweep: int = 0) -> np.ndarray:
    """The checkerboard Metropolis of quenched_u1_angles with counter-based
    uniforms (metropolis_uniforms): sweeps first_sweep .. first_sweep + sweeps - 1
    from theta (cold start theta = 0 when None).  Returns the angles."""
    if Lx % 2 or Lt % 2:
        raise ValueError("Lx and Lt must be even")
    theta = np.zeros((2, Lt, Lx), dtype=np.float64) if theta is None else np.array(theta, np.float64)
    for sw in range(int(first_sweep), int(first_sweep) + int(sweeps)):
        for mu in (0, 1):
            for parity in (0, 1):
                u_prop, u_acc = metropolis_uniforms(Lx, Lt, seed, sw, mu, parity)
                _metropolis_half_u(theta, mu, parity, float(beta), float(eps), u_prop, u_acc)
    return theta


def links_from_angles(theta: np.ndarray) -> np.ndarray:
    """U = exp(i theta) as complex128 [2][Lt][Lx] (gauge links, no fermion sign)."""
    return np.exp(1j * theta).astype(np.complex128)


def quenched_u1(Lx: int, Lt: int, beta: float, sweeps: int, seed: int) -> np.ndarray:
    return links_from_angles(quenched_u1_angles(Lx, Lt, beta, sweeps, seed))


def gaussian_field(shape, seed: int) -> np.ndarray:
    """i.i.d. complex Gaussian entries with Re, Im ~ N(0, 1/2)."""
    rng = _rng(seed)
    z = rng.standard_normal(tuple(shape) + (2,))
    return ((z[..., 0] + 1j * z[..., 1]) * math.sqrt(0.5)).astype(np.complex128)


def level_shapes(Lx: int, Lt: int, blocks, Nv):
    """(Lx_l, Lt_l, ndof_l) for every level l = 1..L of a blocking schedule.

    Level 1 has 2 spin components per site; level l+1 has 2*Nv_l (Nv_l
    vectors per chirality).  Pure shape bookkeeping.
    """
    shapes = [(Lx, Lt, 2)]
    for (bx, bt), nv in zip(blocks, Nv):
        lx, lt, _ = shapes[-1]
        if lx % bx or lt % bt:
            raise ValueError("lattice extent not divisible by block")
        shapes.append((lx // bx, lt // bt, 2 * nv))
    return shapes


def _noise_len_from(Lx: int, Lt: int, blocks, Nv, first: int) -> int:
    """Entries of the per-level random starts of levels first .. L-2."""
    shapes = level_shapes(Lx, Lt, blocks, Nv)
    return sum((nv + 2) * lx * lt * n
               for (lx, lt, n), nv in list(zip(shapes[:-1], Nv))[first:])


def setup_noise_len(Lx: int, Lt: int, blocks, Nv, refine_levels=()) -> int:
    """Number of complex entries of the setup noise buffer (see setup_noise)."""
    tot = _noise_len_from(Lx, Lt, blocks, Nv, 0)
    Nv = list(Nv)
    for level in refine_levels:
        Nv[level] += 1
        lx, lt, n = level_shapes(Lx, Lt, blocks, Nv)[level]
        tot += lx * lt * n + _noise_len_from(Lx, Lt, blocks, Nv, level + 1)
    return tot


def setup_noise(Lx: int, Lt: int, blocks, Nv, seed: int, refine_levels=()) -> np.ndarray:
    """Random vectors drawn by the adaptive setup, flattened complex128.

    For each non-coarsest level l (finest first) the buffer holds, in order,
    Nv_l starting vectors for the null-space relaxation, one start for the
    power iteration that sets the relaxation step, and one start for the two
    minimum-residual steps that fix the smoother; each is a level-l vector in
    [t][x][dof] order.  Then, for each adaptive pass on level refine_levels[p]
    (0 = finest), the random error it starts from (a level vector) and the
    starts of every level below it for the Nv after the pass, laid out as
    above (see refine_noise).
    """
    return gaussian_field((setup_noise_len(Lx, Lt, blocks, Nv, refine_levels),), seed)


def refine_noise(Lx: int, Lt: int, blocks, Nv, level: int, seed: int) -> np.ndarray:
    """Random starts of the levels below `level` (0 = finest) for the vector
    counts Nv (after the pass), as an adaptive pass on `level` reads them."""
    return gaussian_field((_noise_len_from(Lx, Lt, blocks, Nv, level + 1),), seed)


# ---------------------------------------------------------------------------
# Benchmark workload definitions (sizes and seeds only).
# ---------------------------------------------------------------------------
# 128 x 128, beta = 6 (200 sweeps from cold start), 3 levels (4x4 then 2x2
# blocks), Nv = 8 per chirality, 8 setup sweeps; setup at the near-critical
# mass, reused for the heavier masses of the sweep; one Gaussian source chi,
# b = D^dagger chi, tol 1e-10.
BENCH_WORKLOADS = {
    "L128_b6_massweep": dict(Lx=128, Lt=128, beta=6.0, sweeps=200, seed=1, blocks=[(4, 4), (2, 2)],
                             Nv=[8, 8], setup_sweeps=8, heavy_masses=[-0.05, 0.0, 0.1],
                             critical_key="L128_b6_s1", noise_seed=7, chi_seed=101, tol=1e-10),
}

# Batched workloads at the near-critical mass: nrhs Gaussian sources (seeds
# chi_seed + k), b_k = D^dagger chi_k, all solved in one Krylov loop.
#   256 x 256, beta = 10 (500 sweeps), 3 levels (4x4, 2x2), Nv = 8, 64 RHS;
#   1024 x 1024, beta = 10 (500 sweeps), 4 levels (4x4, 2x2, 2x2), Nv = 12, 16 RHS.
BATCHED_WORKLOADS = {
    "L256_b10_nc64": dict(Lx=256, Lt=256, beta=10.0, sweeps=500, seed=1, blocks=[(4, 4), (2, 2)],
                          Nv=[8, 8], setup_sweeps=8, nrhs=64, critical_key="L256_b10_s1",
                          noise_seed=7, chi_seed=101, tol=1e-10),
    "L1024_b10_nc16": dict(Lx=1024, Lt=1024, beta=10.0, sweeps=500, seed=1,
                           blocks=[(4, 4), (2, 2), (2, 2)], Nv=[12, 12, 12], setup_sweeps=8,
                           nrhs=16, critical_key="L1024_b10_s1", noise_seed=7, chi_seed=101,
                           tol=1e-10),
    # the same with a fifth level (2x2 blocks): 24,576 coarsest unknowns instead
    # of 98,304, inverted densely (FP32 inverse, FP64 refinement)
    "L1024_b10_nc16_l5": dict(Lx=1024, Lt=1024, beta=10.0, sweeps=500, seed=1,
                              blocks=[(4, 4), (2, 2), (2, 2), (2, 2)], Nv=[12, 12, 12, 12],
                              setup_sweeps=8, nrhs=16, critical_key="L1024_b10_s1", noise_seed=7,
                              chi_seed=101, tol=1e-10, params={"coarsest_dense_max": 24576},
                              reps=1),
}
