"""Keeping the coarsest FP32 inverse across re-masses (mg_params.coarsest_reuse).

The coarsest level is solved exactly (Sec. 2): an FP32 inverse refined in FP64
until the set-up's test vectors reach coarsest_tol.  With coarsest_reuse = k,
mg_set_mass first tries the previous mass's inverse inside that refinement and
keeps it when the test vectors reach coarsest_tol within min(k, 11) steps.

Case: 64 x 64, beta = 3 (200 sweeps, seed 1), three levels (4 x 4 then 2 x 2
blocks, Nv = 8, 8; 1024 coarsest unknowns), set up at the oracle's near-critical
mass, then re-massed along -0.05, 0.0, 0.1 like the benchmark step.  Checked
against a hierarchy with the same set-up vectors that inverts anew at every
mass: the jump from the near-critical mass inverts anew; the step to 0.0 keeps
the inverse; at every mass the FP64 V-cycles agree to 1e-11 (both coarsest
solves are exact to coarsest_tol), every mixed solve's true residual,
recomputed with the oracle's operator, is <= 1e-10, and the iteration counts
agree within 2.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import wilson as ow

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEV = "cuda:0"
L, BLOCKS, NV = 64, [(4, 4), (2, 2)], [8, 8]


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0710_3612_gb300 import mg as m
    return m


def test_reuse_keeps_exact_coarsest_solve(mg):
    crit = json.load(open(os.path.join(ROOT, "workloads", "critical_masses_serving.json")))["L64_b3_s1"]
    th = W.quenched_u1_angles(L, L, crit["beta"], crit["sweeps"], crit["seed"])
    assert W.mean_plaquette(th) == pytest.approx(crit["plaquette"], abs=1e-12)
    U = W.links_from_angles(th)
    noise = torch.from_numpy(W.setup_noise(L, L, BLOCKS, NV, 7)).to(DEV)
    Ud = torch.from_numpy(U).to(DEV)
    r = W.gaussian_field((L, L, 2), 5)
    with mg.Multigrid(Ud, crit["m_nc"], BLOCKS, NV, noise, coarsest_reuse=12) as a, \
            mg.Multigrid(Ud, crit["m_nc"], BLOCKS, NV, noise) as fresh:
        for k, m in enumerate((-0.05, 0.0, 0.1)):
            a.set_mass(m)
            fresh.set_mass(m)
            _, reuses = mg.mg_get_coarsest_reuse(a.h)
            if k == 0:
                assert reuses == 0              # the jump from m_nc: a new inverse
            if k == 1:
                assert reuses == 1              # 0.05 apart: the previous inverse kept
            _, _, res = mg.mg_get_coarsest_info(a.h)
            assert 0 < res <= a.params.coarsest_tol
            rd = torch.from_numpy(r).to(DEV)
            ya, yf = torch.empty_like(rd), torch.empty_like(rd)
            mg.mg_vcycle(a.h, rd, ya, mg.PREC_F64)
            mg.mg_vcycle(fresh.h, rd, yf, mg.PREC_F64)
            torch.cuda.synchronize()
            ya, yf = ya.cpu().numpy(), yf.cpu().numpy()
            assert np.linalg.norm(ya - yf) <= 1e-11 * np.linalg.norm(yf)
            b = ow.apply_D(U, m, W.gaussian_field((L, L, 2), 40 + k), dagger=True)
            bd = torch.from_numpy(b).to(DEV)
            for solver in (mg.SOLVER_MGCG_MIXED, mg.SOLVER_MGCG_FP64):
                xa, ia = a.solve(bd, tol=1e-10, solver=solver)
                xf, i_f = fresh.solve(bd, tol=1e-10, solver=solver)
                torch.cuda.synchronize()
                got = xa.cpu().numpy().reshape(b.shape)
                true = np.linalg.norm(b - ow.apply_A(U, m, got)) / np.linalg.norm(b)
                assert true <= 1e-10 and ia[0].true_residual <= 1e-10
                assert abs(ia[0].iterations - i_f[0].iterations) <= 2


def test_reuse_argument_checked(mg):
    U = torch.ones((2, 16, 16), dtype=torch.complex128, device=DEV)
    noise = torch.from_numpy(W.setup_noise(16, 16, [(4, 4)], [2], 7)).to(DEV)
    with pytest.raises(mg.MgError) as e:
        mg.Multigrid(U, 0.1, [(4, 4)], [2], noise, coarsest_reuse=-1)
    assert e.value.status == 1 and "coarsest_reuse" in str(e.value)
