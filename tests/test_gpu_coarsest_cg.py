"""Coarsest levels above coarsest_dense_max unknowns: FP64 CG on the coarsest
stencil instead of the dense inverse (Sec. 2, the coarsest-level solve; CG
for large coarsest levels).  Checked against the oracle's Cholesky solve of
the same coarsest operator, and through whole MG-CG solves.
"""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as okr
from oracle import multigrid as omg
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


# (Lx, Lt, beta, sweeps, seed, mass, blocks, Nv): coarsest 3 x 3 x 8 = 72 and
# 16 x 16 x 8 = 2048 unknowns
CASES = [(24, 24, 6.0, 40, 2, -1.2, [(4, 4), (2, 2)], [3, 4]),
         (32, 32, 6.0, 60, 3, -0.9, [(2, 2)], [4])]


@pytest.mark.parametrize("case", CASES, ids=["3lvl_24", "2lvl_32"])
def test_coarsest_cg_matches_oracle(mg, case):
    Lx, Lt, beta, sweeps, seed, m, blocks, Nv = case
    U = W.quenched_u1(Lx, Lt, beta, sweeps, seed)
    noise = W.setup_noise(Lx, Lt, blocks, Nv, 5)
    H = omg.setup(U, m, blocks, Nv, noise)
    last = H.levels[-1]
    assert H.coarsest_chol is not None                     # the oracle solves it densely
    with mg.Multigrid(dev(U), m, blocks, Nv, dev(noise), coarsest_dense_max=0) as s:
        b = W.gaussian_field((last.Lt, last.Lx, last.n), 41)
        out = torch.empty_like(dev(b))
        mg.mg_coarsest_solve(s.h, dev(b), out)
        want = omg.coarsest_solve(H, b)
        got = host(out)
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
        chi = W.gaussian_field((Lt, Lx, 2), 61)
        bf = ow.apply_D(U, m, chi, dagger=True)
        _, it_ora, _ = okr.mgcg(H, bf, TOL)
        for solver in (mg.SOLVER_MGCG_FP64, mg.SOLVER_MGCG_MIXED):
            x, infos = s.solve(dev(bf), tol=TOL, maxiter=5000, solver=solver)
            xs = host(x).reshape(bf.shape)
            res = np.linalg.norm(bf - ow.apply_A(U, m, xs)) / np.linalg.norm(bf)
            assert res <= TOL and infos[0].true_residual <= TOL
            if solver == mg.SOLVER_MGCG_FP64:
                assert abs(infos[0].iterations - it_ora) <= 1
