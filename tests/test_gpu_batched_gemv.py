"""Coarsest-level GEMV for 16 to 64 right-hand sides on tensor cores (3xTF32
mma.sync): a batched solve applies the same V-cycle to every right-hand side
as a solve of it alone, so each right-hand side needs the same number of
iterations (within one) and reaches the same true residual; a wrong dense
product would change the preconditioner and the counts.  Checked on a small
3-level case (72 coarsest unknowns) and on the 4096-unknown coarsest level of
the 128 x 128 workload."""
import numpy as np
import pytest

import workloads as W
from oracle import wilson as ow

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("case", [(24, 24, 6.0, 40, 2, -1.2, [(4, 4), (2, 2)], [3, 4], 16),
                                  (128, 128, 6.0, 200, 1, -2.0, [(4, 4), (2, 2)], [8, 8], 24)],
                         ids=["coarsest_72_16rhs", "coarsest_4096_24rhs"])
@pytest.mark.parametrize("solver", ["mixed", "fp64"])
def test_batched_iterations_equal_single(mg, case, solver):
    Lx, Lt, beta, sweeps, seed, m, blocks, Nv, nrhs = case
    code = mg.SOLVER_MGCG_MIXED if solver == "mixed" else mg.SOLVER_MGCG_FP64
    U = W.quenched_u1(Lx, Lt, beta, sweeps, seed)
    noise = dev(W.setup_noise(Lx, Lt, blocks, Nv, 5))
    b = np.stack([ow.apply_D(U, m, W.gaussian_field((Lt, Lx, 2), 300 + k), dagger=True)
                  for k in range(nrhs)])
    with mg.Multigrid(dev(U), m, blocks, Nv, noise, max_rhs=nrhs) as s:
        x, infos = s.solve(dev(b), tol=TOL, maxiter=5000, solver=code)
        xb = host(x).reshape(b.shape)
    with mg.Multigrid(dev(U), m, blocks, Nv, noise) as s:
        single = [s.solve(dev(b[k]), tol=TOL, maxiter=5000, solver=code)[1][0] for k in range(nrhs)]
    for k in range(nrhs):
        res = np.linalg.norm(b[k] - ow.apply_A(U, m, xb[k])) / np.linalg.norm(b[k])
        assert res <= TOL and infos[k].true_residual <= TOL
        assert abs(infos[k].iterations - single[k].iterations) <= 1, \
            f"rhs {k}: batched {infos[k].iterations} vs alone {single[k].iterations}"
