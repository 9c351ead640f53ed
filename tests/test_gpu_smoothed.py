"""Smoothed aggregation on the GPU (Sec. 3: one Richardson step on the block
vectors before they define the prolongator, the damping chosen to minimise
the condition number of the coarse operator) against oracle/smoothed.py.

The kernels are compared on the GPU's own block vectors V (the tentative
prolongator P of the oracle is built from them), at 1e-12 per element (the
bound |gpu - oracle| <= 1e-12 (|oracle| + M), M the same products of absolute
values): P_s = (1 - omega A) P and P_s^dagger through mg_prolong /
mg_restrict, the level-2 operator P_s^dagger A P_s (probed on the GPU as
P^dagger A P - 2 omega P^dagger A^2 P + omega^2 P^dagger A^3 P, so M sums the
magnitudes of those terms) against the oracle's sparse product on the
couplings of the 9-point stencil, the two-level V-cycle against TwoLevelSA,
and whole MG-CG solves.  The omega search is checked against the oracle's
criterion: the oracle's condition number at the GPU's omega is within 1e-3
of its minimum.
"""
import numpy as np
import pytest

import workloads as W
from oracle import critical, krylov
from oracle import multigrid as omg
from oracle import smoothed as sa
from oracle import wilson as ow

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL64 = 1e-12


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0710_3612_gb300 import mg as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def check(got, want, mag, tol, what):
    err = np.abs(got - want)
    worst = np.max(err / np.maximum(tol * (np.abs(want) + mag), 1e-300))
    assert worst <= 1.0, f"{what}: worst error / bound = {worst:.3g} (max err {err.max():.3e})"


class Case:
    """16 x 16 (coarse 4 x 4) or 24 x 24 (coarse 6 x 6), beta = 3, 4 x 4 blocks."""

    def __init__(self, mg, L, Nv, m, omega, levels=2, **kw):
        self.L, self.m = L, m
        self.blocks = [(4, 4)] + [(2, 2)] * (levels - 2)
        self.Nv = [Nv] * (levels - 1)
        self.U = W.links_from_angles(W.quenched_u1_angles(L, L, 3.0, 30, 3))
        self.noise = W.setup_noise(L, L, self.blocks, self.Nv, 17)
        self.s = mg.Multigrid(dev(self.U), m, self.blocks, self.Nv, dev(self.noise),
                              smooth_omega=omega, max_rhs=4, **kw)
        self.h = self.s.h
        Lx, Lt, n, nv = mg.mg_get_level(self.h, 1)
        out = torch.empty((nv, Lt, Lx, n), dtype=torch.complex128, device=DEV)
        mg.mg_get_null_vectors(self.h, 1, out)
        self.V = host(out)
        self.A = sa.normal_matrix(self.U, m)
        self.P = sa.tentative_prolongator(self.V, 4, 4)
        self.omega, self.cond = mg.mg_get_smoothing(self.h)
        self.Ps = sa.smoothed_prolongator(self.A, self.P, self.omega)
        absA = abs(self.A)
        absP = abs(self.P)
        self.absPs = absP + abs(self.omega) * (absA @ absP)
        self.absA = absA
        self.mag_c = coarse_magnitudes(absA, absP, self.omega)


def check_coarse(got, want, mag, Lc, nc, what):
    """got against want on the couplings of the 9-point stencil at 1e-12 per
    element; outside it the oracle holds only round-off (its sparse
    A = D^dagger D keeps two-hop entries of order 1e-17 that vanish exactly,
    (1 + gamma_mu)(1 - gamma_mu) = 0), which the stencil does not store."""
    j = np.arange(Lc * Lc)
    x, t = j % Lc, j // Lc
    dx = np.abs(x[:, None] - x[None, :])
    dt = np.abs(t[:, None] - t[None, :])
    near = (np.minimum(dx, Lc - dx) <= 1) & (np.minimum(dt, Lc - dt) <= 1)
    near = np.kron(near, np.ones((nc, nc), bool))
    check(got[near], want[near], mag[near], TOL64, what)
    assert np.max(np.abs(got[~near]), initial=0.0) == 0.0
    assert np.max(np.abs(want[~near]), initial=0.0) <= 1e-25 * np.max(np.abs(want)), what


def coarse_magnitudes(absA, absP, omega):
    """Sum of the magnitudes of the terms of P_s^dagger A P_s = P^dagger A P
    - 2 omega P^dagger A^2 P + omega^2 P^dagger A^3 P (dense)."""
    AP = absA @ absP
    A2P = absA @ AP
    A3P = absA @ A2P
    return (absP.T @ AP + 2 * abs(omega) * (absP.T @ A2P) + omega ** 2 * (absP.T @ A3P)).toarray()


@pytest.fixture(scope="module")
def case(mg):
    c = Case(mg, 16, 2, -0.5, 0.1)
    yield c
    c.s.close()


def test_smoothed_transfers(mg, case):
    c = case
    assert c.omega == 0.1
    Lc, nc = c.L // 4, 2 * c.Nv[0]
    for nrhs in (1, 3):
        ec = W.gaussian_field((nrhs, Lc, Lc, nc), 5 + nrhs)
        out = torch.empty((nrhs, c.L, c.L, 2), dtype=torch.complex128, device=DEV)
        mg.mg_prolong(c.h, 1, dev(ec), out, nrhs, mg.PREC_F64)
        want = np.stack([(c.Ps @ e.ravel()).reshape(c.L, c.L, 2) for e in ec])
        mag = np.stack([(c.absPs @ np.abs(e).ravel()).reshape(c.L, c.L, 2) for e in ec])
        check(host(out), want, mag, TOL64, "P_s e")
        r = W.gaussian_field((nrhs, c.L, c.L, 2), 9 + nrhs)
        outc = torch.empty((nrhs, Lc, Lc, nc), dtype=torch.complex128, device=DEV)
        mg.mg_restrict(c.h, 1, dev(r), outc, nrhs, mg.PREC_F64)
        want = np.stack([(c.Ps.conj().T @ x.ravel()).reshape(Lc, Lc, nc) for x in r])
        mag = np.stack([(c.absPs.T @ np.abs(x).ravel()).reshape(Lc, Lc, nc) for x in r])
        check(host(outc), want, mag, TOL64, "P_s^dagger r")
        # FP32 path at the FP32 bound
        out32 = torch.empty((nrhs, c.L, c.L, 2), dtype=torch.complex64, device=DEV)
        mg.mg_prolong(c.h, 1, dev(ec.astype(np.complex64)), out32, nrhs, mg.PREC_F32)
        want = np.stack([(c.Ps @ e.astype(np.complex64).astype(np.complex128).ravel()).reshape(c.L, c.L, 2)
                         for e in ec])
        mag = np.stack([(c.absPs @ np.abs(e).ravel()).reshape(c.L, c.L, 2) for e in ec])
        check(host(out32), want, mag, 1e-6, "P_s e (FP32)")


def test_smoothed_coarse_operator(mg, case):
    """The probed level-2 operator equals the oracle's P_s^dagger A P_s; the
    smoothed operator of 4 x 4 blocks keeps the 9-point stencil."""
    c = case
    Lc, nc = c.L // 4, 2 * c.Nv[0]
    out = torch.empty((Lc, Lc, 9, nc, nc), dtype=torch.complex128, device=DEV)
    mg.mg_get_coarse_op(c.h, 2, out)
    got = omg.StencilOp(omg.COARSE_DISP, host(out)).dense()
    want = sa.coarse_operator(c.A, c.Ps).toarray()
    check_coarse(got, want, c.mag_c, Lc, nc, "P_s^dagger A P_s")
    Ac = sa.coarse_operator(c.A, c.Ps)
    Ac.data[np.abs(Ac.data) < 1e-25 * np.max(np.abs(Ac.data))] = 0
    Ac.eliminate_zeros()
    assert sa.block_reach(Ac, Lc, Lc, nc) == 1


def test_smoothed_vcycle_and_solve(mg, case):
    c = case
    c0, c1, lam, om = mg.mg_get_smoother(c.h, 1)
    T = sa.TwoLevelSA(c.A, c.Ps, c0, c1)
    r = W.gaussian_field((c.L, c.L, 2), 51)
    out = torch.empty_like(dev(r))
    mg.mg_vcycle(c.h, dev(r), out, mg.PREC_F64)
    want = T.vcycle(r)
    assert np.linalg.norm(host(out) - want) <= 1e-10 * np.linalg.norm(want)
    b = ow.apply_D(c.U, c.m, W.gaussian_field((c.L, c.L, 2), 61), dagger=True)
    _, it_ora, info_ora = krylov.pcg(lambda v: ow.apply_A(c.U, c.m, v), b, 1e-10, 5000,
                                     precond=T.vcycle)
    for solver in (mg.SOLVER_MGCG_FP64, mg.SOLVER_MGCG_MIXED):
        x, infos = c.s.solve(dev(b), tol=1e-10, maxiter=5000, solver=solver)
        xs = host(x).reshape(b.shape)
        res = np.linalg.norm(b - ow.apply_A(c.U, c.m, xs)) / np.linalg.norm(b)
        assert res <= 1e-10 and infos[0].true_residual <= 1e-10
        if solver == mg.SOLVER_MGCG_FP64:
            assert abs(infos[0].iterations - it_ora) <= 1


def test_three_levels_with_a_smoothed_first_coarsening(mg):
    c = Case(mg, 24, 3, -0.7, 0.08, levels=3)
    try:
        Lc, nc = 6, 6
        out = torch.empty((Lc, Lc, 9, nc, nc), dtype=torch.complex128, device=DEV)
        mg.mg_get_coarse_op(c.h, 2, out)
        got = omg.StencilOp(omg.COARSE_DISP, host(out)).dense()
        want = sa.coarse_operator(c.A, c.Ps).toarray()
        check_coarse(got, want, c.mag_c, Lc, nc, "P_s^dagger A P_s (three levels)")
        b = ow.apply_D(c.U, c.m, W.gaussian_field((24, 24, 2), 71), dagger=True)
        for solver in (mg.SOLVER_MGCG_FP64, mg.SOLVER_MGCG_MIXED):
            x, infos = c.s.solve(dev(b), tol=1e-10, maxiter=5000, solver=solver)
            res = np.linalg.norm(b - ow.apply_A(c.U, c.m, host(x).reshape(b.shape))) / np.linalg.norm(b)
            assert res <= 1e-10 and infos[0].true_residual <= 1e-10
        # a new mass probes the smoothed operator anew with the same omega
        c.s.set_mass(-0.6)
        assert mg.mg_get_smoothing(c.h)[0] == 0.08
        A2 = sa.normal_matrix(c.U, -0.6)
        Ps2 = sa.smoothed_prolongator(A2, c.P, 0.08)
        mg.mg_get_coarse_op(c.h, 2, out)
        got = omg.StencilOp(omg.COARSE_DISP, host(out)).dense()
        check_coarse(got, sa.coarse_operator(A2, Ps2).toarray(), coarse_magnitudes(abs(A2), abs(c.P), 0.08),
                     Lc, nc, "P_s^dagger A P_s after set_mass")
    finally:
        c.s.close()


def test_omega_search_meets_the_oracle_criterion(mg):
    """Near the critical mass (0.02 above it): the GPU's omega is a minimiser
    of the oracle's condition number to 1e-3, its own condition estimate
    agrees with the oracle's to 1e-3, and MG-CG with it takes no more
    iterations than with the tentative prolongator."""
    L = 16
    U = W.links_from_angles(W.quenched_u1_angles(L, L, 3.0, 30, 3))
    real, _ = critical.real_eigenvalues_D0(U)
    m = -float(real[0]) + 0.02
    noise = W.setup_noise(L, L, [(4, 4)], [2], 17)
    with mg.Multigrid(dev(U), m, [(4, 4)], [2], noise=dev(noise), smooth_omega=-1.0) as s:
        om, cond = mg.mg_get_smoothing(s.h)
        c0, c1, lam, _ = mg.mg_get_smoother(s.h, 1)
        Lx, Lt, n, nv = mg.mg_get_level(s.h, 1)
        out = torch.empty((nv, Lt, Lx, n), dtype=torch.complex128, device=DEV)
        mg.mg_get_null_vectors(s.h, 1, out)
        V = host(out)
        A, P = sa.normal_matrix(U, m), sa.tentative_prolongator(V, 4, 4)
        om_ora, cond_ora = sa.optimal_omega(A, P, lam)
        cond_at = sa.condition_number(sa.coarse_operator(A, sa.smoothed_prolongator(A, P, om)))
        assert 0 < om < 2 / lam
        assert cond_at <= cond_ora * (1 + 1e-3), (om, om_ora, cond_at, cond_ora)
        assert abs(cond - cond_at) <= 1e-3 * cond_at
        b = ow.apply_D(U, m, W.gaussian_field((L, L, 2), 81), dagger=True)
        x, infos = s.solve(dev(b), tol=1e-10, maxiter=5000, solver=mg.SOLVER_MGCG_FP64)
        it_sa = infos[0].iterations
        assert infos[0].true_residual <= 1e-10
    with mg.Multigrid(dev(U), m, [(4, 4)], [2], noise=dev(noise)) as s:
        x, infos = s.solve(dev(b), tol=1e-10, maxiter=5000, solver=mg.SOLVER_MGCG_FP64)
        assert it_sa <= infos[0].iterations


def test_smoothing_argument_checks(mg):
    L = 16
    U = dev(W.quenched_u1(L, L, 3.0, 10, 1))
    for blocks, Nv, kw in [([(2, 2)], [2], dict(smooth_omega=0.1)),                 # reach 2 blocks
                           ([(4, 4), (2, 2)], [2, 2], dict(smooth_omega=-1.0)),     # search: 2 levels
                           ([(4, 4)], [2], dict(smooth_omega=0.1, refine_levels=[1]))]:
        noise = dev(W.setup_noise(L, L, blocks, Nv, 3, refine_levels=[l - 1 for l in kw.get("refine_levels", [])]))
        with pytest.raises(mg.MgError) as e:
            mg.Multigrid(U, -0.5, blocks, Nv, noise, **kw)
        assert e.value.status == 1
