"""Parity at the sizes of the workload configurations (Sec. 4 workloads).

* 32 x 32, beta = 6, m = 0.05: plain FP64 two-level MG-CG (4 x 4 blocks,
  Nv = 4, 8 setup sweeps) against the oracle's own solve of the same system:
  true residual, iteration count within one, and the solution within the
  kappa * tol bound of the oracle's tight solve.
* 256 x 256, beta = 10 (500 sweeps), at the oracle's near-critical mass:
  64 right-hand sides in one batched mixed-precision solve (tensor-core coarse
  contraction).  The oracle cannot run 64 near-critical solves at this size,
  so it checks what holds at any size: D^dagger on sampled right-hand sides
  element by element, and every solution's true FP64 residual, recomputed
  with the oracle's own operator.
* 1024 x 1024, beta = 10, at the oracle's near-critical mass: 16 right-hand
  sides in one batched mixed solve on the five-level hierarchy of the
  benchmark (D^dagger sampled, every true residual recomputed), and at
  m = -1.9 on the configured four levels.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import critical
from oracle import krylov as okr
from oracle import multigrid as omg
from oracle import wilson as ow

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEV = "cuda:0"
TOL = 1e-10


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


def test_cfg_32x32_two_level_plain_fp64(mg):
    L, m, blocks, Nv = 32, 0.05, [(4, 4)], [4]
    U = W.quenched_u1(L, L, 6.0, 200, 1)
    noise = W.setup_noise(L, L, blocks, Nv, 7)
    chi = W.gaussian_field((L, L, 2), 101)
    b = ow.apply_D(U, m, chi, dagger=True)
    H = omg.setup(U, m, blocks, Nv, noise, sweeps=8)
    _, it10, _ = okr.mgcg(H, b, TOL)
    x_ora, _, _ = okr.mgcg(H, b, 1e-13)
    with mg.Multigrid(dev(U), m, blocks, Nv, dev(noise), setup_sweeps=8) as s:
        x, infos = s.solve(dev(b), tol=TOL, maxiter=1000, solver=mg.SOLVER_MGCG_FP64)
        got = host(x).reshape(b.shape)
    A = H.levels[0].op
    res = np.linalg.norm(b - A.apply(got)) / np.linalg.norm(b)
    assert res <= TOL and infos[0].true_residual <= TOL
    assert abs(infos[0].iterations - it10) <= 1
    lam = np.linalg.eigvalsh(A.dense())
    kappa = lam[-1] / lam[0]
    assert np.linalg.norm(got - x_ora) <= (kappa * TOL + 1e-12) * np.linalg.norm(x_ora)


def test_cfg_256x256_batched_64_rhs_near_critical(mg):
    crit = json.load(open(os.path.join(ROOT, "workloads", "critical_masses.json")))["L256_b10_s1"]
    L, blocks, Nv, nrhs = 256, [(4, 4), (2, 2)], [8, 8], 64
    th = W.quenched_u1_angles(L, L, crit["beta"], crit["sweeps"], crit["seed"])
    assert W.mean_plaquette(th) == pytest.approx(crit["plaquette"], abs=1e-12)
    U = W.links_from_angles(th)
    m = crit["m_nc"]
    noise = W.setup_noise(L, L, blocks, Nv, 7)
    chis = np.stack([W.gaussian_field((L, L, 2), 1101 + k) for k in range(nrhs)])
    with mg.Multigrid(dev(U), m, blocks, Nv, dev(noise), setup_sweeps=8, max_rhs=nrhs) as s:
        b_d = torch.empty((nrhs, L, L, 2), dtype=torch.complex128, device=DEV)
        mg.mg_apply_D(s.h, dev(chis), b_d, nrhs, 1, mg.PREC_F64)
        b = host(b_d)
        for k in (0, nrhs - 1):                  # D^dagger at full size, per element
            want = ow.apply_D(U, m, chis[k], dagger=True)
            assert np.max(np.abs(b[k] - want)) <= 1e-12 * np.max(np.abs(want))
        x, infos = s.solve(b_d, tol=TOL, maxiter=20000, solver=mg.SOLVER_MGCG_MIXED)
        got = host(x).reshape(b.shape)
    for k in range(nrhs):
        res = np.linalg.norm(b[k] - ow.apply_A(U, m, got[k])) / np.linalg.norm(b[k])
        assert res <= TOL, f"rhs {k}: true residual {res:.3e}"
        assert infos[k].true_residual <= TOL
        assert abs(infos[k].true_residual - res) <= 1e-3 * TOL


def test_cfg_128x128_mass_sweep(mg):
    """The benchmark workload: set-up at the near-critical mass, re-mass to
    m = 0.1.  At 0.1 both solvers are compared with the oracle's solve of the
    same hierarchy; at m_nc (814 oracle iterations, too slow to repeat here)
    the FP64 iteration count is compared with the oracle's stored count and
    every solution's true residual is recomputed by the oracle."""
    wl = W.BENCH_WORKLOADS["L128_b6_massweep"]
    crit = json.load(open(os.path.join(ROOT, "workloads", "critical_masses.json")))[wl["critical_key"]]
    stored = json.load(open(os.path.join(ROOT, "workloads", "oracle_iterations.json")))
    stored = stored["L128_b6_massweep"]["masses"]
    L, blocks, Nv = wl["Lx"], wl["blocks"], wl["Nv"]
    th = W.quenched_u1_angles(L, L, wl["beta"], wl["sweeps"], wl["seed"])
    assert W.mean_plaquette(th) == pytest.approx(crit["plaquette"], abs=1e-12)
    U = W.links_from_angles(th)
    noise = W.setup_noise(L, L, blocks, Nv, wl["noise_seed"])
    chi = W.gaussian_field((L, L, 2), wl["chi_seed"])
    m_nc = crit["m_nc"]
    with mg.Multigrid(dev(U), m_nc, blocks, Nv, dev(noise), setup_sweeps=wl["setup_sweeps"]) as s:
        b = ow.apply_D(U, m_nc, chi, dagger=True)
        for solver in (mg.SOLVER_MGCG_FP64, mg.SOLVER_MGCG_MIXED):
            x, infos = s.solve(dev(b), tol=TOL, maxiter=20000, solver=solver)
            got = host(x).reshape(b.shape)
            res = np.linalg.norm(b - ow.apply_A(U, m_nc, got)) / np.linalg.norm(b)
            assert res <= TOL and infos[0].true_residual <= TOL
            if solver == mg.SOLVER_MGCG_FP64:
                assert abs(infos[0].iterations - stored[repr(m_nc)]["iterations"]) <= 1
        m = 0.1
        s.set_mass(m)
        H = omg.setup(U, m_nc, blocks, Nv, noise, sweeps=wl["setup_sweeps"])
        H = omg.set_mass(H, m)
        b = ow.apply_D(U, m, chi, dagger=True)
        _, it10, _ = okr.mgcg(H, b, TOL)
        assert it10 == stored[repr(m)]["iterations"]
        x_ora, _, _ = okr.mgcg(H, b, 1e-13)
        # kappa(A) bound: lambda_max(A) = |D|^2 <= (|4 + m| + 4)^2 (each of the four
        # hop terms has norm <= 1); lambda_min(A) = sigma_min(D)^2 = (eigenvalue of
        # the Hermitian sigma_3 D nearest zero)^2
        lam_h, _ = critical.nearest_eig_H(U, m)
        kappa = (abs(4.0 + m) + 4.0) ** 2 / lam_h ** 2
        for solver in (mg.SOLVER_MGCG_FP64, mg.SOLVER_MGCG_MIXED):
            x, infos = s.solve(dev(b), tol=TOL, maxiter=1000, solver=solver)
            got = host(x).reshape(b.shape)
            res = np.linalg.norm(b - ow.apply_A(U, m, got)) / np.linalg.norm(b)
            assert res <= TOL and infos[0].true_residual <= TOL
            assert np.linalg.norm(got - x_ora) <= (kappa * TOL + 1e-12) * np.linalg.norm(x_ora)
            if solver == mg.SOLVER_MGCG_FP64:
                assert abs(infos[0].iterations - it10) <= 1


@pytest.fixture(scope="module")
def field_1024():
    """The 1024 x 1024 beta = 10 field of the oracle's finder (seed 1, 500 sweeps)."""
    crit = json.load(open(os.path.join(ROOT, "workloads", "critical_masses.json")))["L1024_b10_s1"]
    th = W.quenched_u1_angles(1024, 1024, crit["beta"], crit["sweeps"], crit["seed"])
    assert W.mean_plaquette(th) == pytest.approx(crit["plaquette"], abs=1e-12)
    return W.links_from_angles(th), crit


def test_cfg_1024x1024_near_critical_16_rhs(mg, field_1024):
    """1024 x 1024 at the oracle's near-critical mass (m_crit + 0.002,
    lambda_min(A) = 3.4e-6): 16 Gaussian right-hand sides b = D^dagger chi in
    one batched mixed solve, on the five-level hierarchy the benchmark runs
    (4x4, 2x2, 2x2, 2x2 blocks, Nv = 12; 32 x 32 x 24 = 24576 coarsest
    unknowns, FP32 inverse with FP64 refinement).  The oracle checks D^dagger
    per element on two right-hand sides and recomputes every solution's true
    residual with its own operator."""
    U, crit = field_1024
    wl = W.BATCHED_WORKLOADS["L1024_b10_nc16_l5"]
    L, m, nrhs = 1024, crit["m_nc"], wl["nrhs"]
    noise = W.setup_noise(L, L, wl["blocks"], wl["Nv"], wl["noise_seed"])
    chis = np.stack([W.gaussian_field((L, L, 2), 1201 + k) for k in range(nrhs)])
    with mg.Multigrid(dev(U), m, wl["blocks"], wl["Nv"], dev(noise), setup_sweeps=wl["setup_sweeps"],
                      max_rhs=nrhs, **wl["params"]) as s:
        dense, _, res0 = mg.mg_get_coarsest_info(s.h)
        assert dense and 0 < res0 <= s.params.coarsest_tol
        b_d = torch.empty((nrhs, L, L, 2), dtype=torch.complex128, device=DEV)
        mg.mg_apply_D(s.h, dev(chis), b_d, nrhs, 1, mg.PREC_F64)
        b = host(b_d)
        for k in (0, nrhs - 1):
            want = ow.apply_D(U, m, chis[k], dagger=True)
            assert np.max(np.abs(b[k] - want)) <= 1e-12 * np.max(np.abs(want))
        x, infos = s.solve(b_d, tol=TOL, maxiter=20000, solver=mg.SOLVER_MGCG_MIXED)
        got = host(x).reshape(b.shape)
    for k in range(nrhs):
        res = np.linalg.norm(b[k] - ow.apply_A(U, m, got[k])) / np.linalg.norm(b[k])
        assert res <= TOL and infos[k].true_residual <= TOL
        assert abs(infos[k].true_residual - res) <= 1e-3 * TOL


def test_cfg_1024x1024_four_level_16_rhs(mg, field_1024):
    """1024 x 1024, beta = 10 (500 checkerboard sweeps), four levels (4x4, 2x2,
    2x2), Nv = 12, 16 right-hand sides in one batched mixed solve; the
    coarsest level (64 x 64 x 24 = 98304 unknowns) is solved by FP64 CG.  At
    m = -1.9 (between the heavy masses and the critical region; the
    near-critical mass needs about 200 ms per outer iteration here, too slow
    for a test).  The oracle checks D^dagger per element on two right-hand
    sides and every solution's true residual."""
    L, blocks, Nv, nrhs, m = 1024, [(4, 4), (2, 2), (2, 2)], [12, 12, 12], 16, -1.9
    U = field_1024[0]
    noise = W.setup_noise(L, L, blocks, Nv, 7)
    chis = np.stack([W.gaussian_field((L, L, 2), 1101 + k) for k in range(nrhs)])
    with mg.Multigrid(dev(U), m, blocks, Nv, dev(noise), setup_sweeps=8, max_rhs=nrhs) as s:
        assert s.level(4)[0] * s.level(4)[1] * s.level(4)[2] == 98304
        b_d = torch.empty((nrhs, L, L, 2), dtype=torch.complex128, device=DEV)
        mg.mg_apply_D(s.h, dev(chis), b_d, nrhs, 1, mg.PREC_F64)
        b = host(b_d)
        for k in (0, nrhs - 1):
            want = ow.apply_D(U, m, chis[k], dagger=True)
            assert np.max(np.abs(b[k] - want)) <= 1e-12 * np.max(np.abs(want))
        x, infos = s.solve(b_d, tol=TOL, maxiter=5000, solver=mg.SOLVER_MGCG_MIXED)
        got = host(x).reshape(b.shape)
    for k in range(nrhs):
        res = np.linalg.norm(b[k] - ow.apply_A(U, m, got[k])) / np.linalg.norm(b[k])
        assert res <= TOL and infos[k].true_residual <= TOL
        assert abs(infos[k].true_residual - res) <= 1e-3 * TOL
