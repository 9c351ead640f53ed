"""The coarsest solve reports when it cannot be made exact (Sec. 2: the
coarsest level is solved exactly).

The dense path inverts the coarsest operator in FP32 and refines the result
in FP64; that converges only while the operator's condition number stays well
below 1/eps of FP32.  Case: 16 x 16, beta = 3, 2 x 2 blocks with Nv = 4, the
block-chirality dimension, so P is unitary and the coarsest operator has the
spectrum of A itself (its condition number, from the oracle's dense
eigenvalues: 7.6e3 at 0.1 above the critical mass, 4.2e5 at 0.02, 2.3e10 at
1e-4).  Checked: at 0.1 the dense path sets up with a test residual <=
coarsest_tol and solves to 1e-10; at 0.02 the FP64 CG path
(coarsest_dense_max = 0) does the same (the FP32 inverse's refinement does
not converge there on this 512-unknown operator); at 1e-4 the dense path
fails with MG_ERR_NOCONV (or MG_ERR_BREAKDOWN if the FP32 inverse is not
finite) and says so, instead of setting up an inexact coarsest solve.
"""
import numpy as np
import pytest

import workloads as W
from oracle import critical
from oracle import wilson as ow

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
L = 16
BLOCKS, NV = [(2, 2)], [4]


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
    U = W.links_from_angles(W.quenched_u1_angles(L, L, 3.0, 30, 3))
    real, _ = critical.real_eigenvalues_D0(U)
    return U, -float(real[0])


@pytest.mark.parametrize("delta,dense_max", [(0.1, 16384), (0.02, 0)])
def test_conditioned_coarsest_reaches_tolerance(mg, field, delta, dense_max):
    U, m_crit = field
    m = m_crit + delta
    noise = W.setup_noise(L, L, BLOCKS, NV, 103)
    with mg.Multigrid(torch.from_numpy(U).to(DEV), m, BLOCKS, NV,
                      torch.from_numpy(noise).to(DEV), coarsest_dense_max=dense_max) as s:
        dense, steps, res = mg.mg_get_coarsest_info(s.h)
        assert dense == (dense_max > 0)
        assert 1 <= steps <= (s.params.coarsest_refine_max if dense else 5000)
        assert 0 < res <= s.params.coarsest_tol
        b = ow.apply_D(U, m, W.gaussian_field((L, L, 2), 9), dagger=True)
        for solver in (mg.SOLVER_MGCG_FP64, mg.SOLVER_MGCG_MIXED):
            x, infos = s.solve(torch.from_numpy(b).to(DEV), tol=1e-10, maxiter=5000, solver=solver)
            torch.cuda.synchronize()
            xs = x.cpu().numpy().reshape(b.shape)
            true = np.linalg.norm(b - ow.apply_A(U, m, xs)) / np.linalg.norm(b)
            assert true <= 1e-10 and infos[0].true_residual <= 1e-10


def test_ill_conditioned_coarsest_fails_loudly(mg, field):
    U, m_crit = field
    m = m_crit + 1e-4
    noise = W.setup_noise(L, L, BLOCKS, NV, 103)
    with pytest.raises(mg.MgError) as e:
        mg.Multigrid(torch.from_numpy(U).to(DEV), m, BLOCKS, NV, torch.from_numpy(noise).to(DEV))
    assert e.value.status in (4, 5)                  # MG_ERR_NOCONV, MG_ERR_BREAKDOWN
    assert "coarsest" in str(e.value)
    # a handle made at a good mass reports the same failure when re-massed there
    with mg.Multigrid(torch.from_numpy(U).to(DEV), m_crit + 0.1, BLOCKS, NV,
                      torch.from_numpy(noise).to(DEV)) as s:
        with pytest.raises(mg.MgError) as e2:
            s.set_mass(m)
        assert e2.value.status in (4, 5) and "coarsest" in str(e2.value)
