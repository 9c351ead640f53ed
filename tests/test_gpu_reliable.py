"""Reliable-update flexible CG (MG_SOLVER_MGCG_RELIABLE).

The Krylov iteration runs in FP32 (A p by the FP32 stencil; residual, search
direction and solution increment stored in FP32) inside the same FP32
V-cycle preconditioner as MG_SOLVER_MGCG_MIXED; when the iterated residual
norm falls below reliable_delta times its largest value since the last
update, the increment joins the FP64 solution and r = b - A x is recomputed
with the FP64 stencil.  What must hold is what holds for every solver: the
true FP64 residual of every solution, recomputed here with the oracle's own
operator, is at most the tolerance.

Case: 64 x 64, beta = 3 (200 sweeps, seed 1), three levels (4 x 4 then 2 x 2
blocks, Nv = 8, 8), at the near-critical mass of the oracle's finder (0.002
above m_crit) and at m = 0.0; single right-hand sides and a batch of six
(max_rhs 8); reliable_delta 0.1 (default), 0.5 and 0.01.  Reliable updates
take place (each is one FP64 fine application beyond the five per iteration
and the set-up and residual applications).  Near the critical mass the FP32
recursion needs more iterations than the FP64 one (measured on one GB300:
442 against 320 here at delta 0.1, 1420-1686 against 824 on the 128 x 128
workload): A p in FP32 loses about eps32 * kappa of its low modes to
cancellation.  The bound below, three times the FP64-recursion count plus
20, only catches a loop that no longer converges by itself.
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
TOL = 1e-10
L, BLOCKS, NV = 64, [(4, 4), (2, 2)], [8, 8]


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0710_3612_gb300 import mg as m
    return m


@pytest.fixture(scope="module")
def field():
    crit = json.load(open(os.path.join(ROOT, "workloads", "critical_masses_serving.json")))["L64_b3_s1"]
    th = W.quenched_u1_angles(L, L, crit["beta"], crit["sweeps"], crit["seed"])
    assert W.mean_plaquette(th) == pytest.approx(crit["plaquette"], abs=1e-12)
    return W.links_from_angles(th), crit["m_nc"]


def true_residuals(U, m, b, x):
    return [np.linalg.norm(b[k] - ow.apply_A(U, m, x[k])) / np.linalg.norm(b[k])
            for k in range(b.shape[0])]


@pytest.mark.parametrize("where", ["m_nc", "0.0"])
@pytest.mark.parametrize("delta", [0.1, 0.5, 0.01])
def test_reliable_reaches_fp64_residual(mg, field, where, delta):
    U, m_nc = field
    m = m_nc if where == "m_nc" else 0.0
    chis = W.gaussian_field((6, L, L, 2), 17)
    b = np.stack([ow.apply_D(U, m, c, dagger=True) for c in chis])
    noise = W.setup_noise(L, L, BLOCKS, NV, 7)
    Ud = torch.from_numpy(U).to(DEV)
    with mg.Multigrid(Ud, m, BLOCKS, NV, torch.from_numpy(noise).to(DEV), max_rhs=8,
                      reliable_delta=delta) as s:
        for batch in (b[:1], b):
            bd = torch.from_numpy(np.ascontiguousarray(batch)).to(DEV)
            xr, ir = s.solve(bd, tol=TOL, maxiter=20000, solver=mg.SOLVER_MGCG_RELIABLE)
            xm, im = s.solve(bd, tol=TOL, maxiter=20000, solver=mg.SOLVER_MGCG_MIXED)
            torch.cuda.synchronize()
            xr = xr.cpu().numpy().reshape(batch.shape)
            res = true_residuals(U, m, batch, xr)
            assert max(res) <= TOL, res
            assert all(i.true_residual <= TOL for i in ir)
            for a, c in zip(ir, im):
                assert a.iterations <= 3 * c.iterations + 20, (a.iterations, c.iterations)
            # 4 set-up applies, 5 per iteration, 2 true residuals, then the updates
            loop = max(i.iterations for i in ir)
            assert ir[0].fine_applies >= 5 * loop + 7, (ir[0].fine_applies, loop)


@pytest.mark.parametrize("delta", [0.0, 1.0, -0.1, float("nan")])
def test_reliable_delta_checked(mg, field, delta):
    U, m_nc = field
    noise = W.setup_noise(L, L, BLOCKS, NV, 7)
    with pytest.raises(mg.MgError) as e:
        mg.Multigrid(torch.from_numpy(U).to(DEV), 0.1, BLOCKS, NV, torch.from_numpy(noise).to(DEV),
                     reliable_delta=delta)
    assert e.value.status == 1 and "reliable_delta" in str(e.value)
