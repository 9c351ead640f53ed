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
"""
import json
import os

import numpy as np
import pytest

import workloads as W
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
