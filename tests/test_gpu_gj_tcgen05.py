"""The dense coarsest inverse with its rank-64 updates on tcgen05 tensor cores
(coarsest_gj_tcgen05 = 1: TMEM accumulator, M = 128 x N = 128 kind::tf32 MMAs,
three TF32 products per FP32-accurate product) against the oracle's Cholesky
solve (Sec. 2, the coarsest-level solve), and against the mma.sync path on
the 4096-unknown coarsest level of the 128 x 128 workload."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import multigrid as omg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEV = "cuda:0"


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


@pytest.mark.parametrize("case", [(24, 24, 6.0, 40, 2, -1.2, [(4, 4), (2, 2)], [3, 4]),
                                  (16, 34, 6.0, 40, 4, -0.8, [(2, 2)], [4]),
                                  (40, 40, 6.0, 40, 3, -0.8, [(2, 2)], [4])],
                         ids=["coarsest_72", "coarsest_1088_odd_tiles", "coarsest_3200"])
def test_tcgen05_inverse_matches_oracle(mg, case):
    Lx, Lt, beta, sweeps, seed, m, blocks, Nv = case
    U = W.quenched_u1(Lx, Lt, beta, sweeps, seed)
    noise = W.setup_noise(Lx, Lt, blocks, Nv, 5)
    H = omg.setup(U, m, blocks, Nv, noise)
    last = H.levels[-1]
    b = W.gaussian_field((last.Lt, last.Lx, last.n), 41)
    want = omg.coarsest_solve(H, b)
    with mg.Multigrid(dev(U), m, blocks, Nv, dev(noise), coarsest_gj_tcgen05=1) as s:
        out = torch.empty_like(dev(b))
        mg.mg_coarsest_solve(s.h, dev(b), out)
        got = host(out)
    assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)


def test_tcgen05_and_mma_sync_agree_at_4096_unknowns(mg):
    wl = W.BENCH_WORKLOADS["L128_b6_massweep"]
    crit = json.load(open(os.path.join(ROOT, "workloads", "critical_masses.json")))[wl["critical_key"]]
    L = wl["Lx"]
    U = dev(W.quenched_u1(L, L, wl["beta"], wl["sweeps"], wl["seed"]))
    noise = dev(W.setup_noise(L, L, wl["blocks"], wl["Nv"], wl["noise_seed"]))
    outs = []
    for tc in (0, 1):
        with mg.Multigrid(U, crit["m_nc"], wl["blocks"], wl["Nv"], noise, coarsest_gj_tcgen05=tc) as s:
            Lx, Lt, n, _ = mg.mg_get_level(s.h, 3)
            assert Lx * Lt * n == 4096
            b = dev(W.gaussian_field((Lt, Lx, n), 43))
            out = torch.empty_like(b)
            mg.mg_coarsest_solve(s.h, b, out)
            outs.append(host(out))
    assert np.linalg.norm(outs[1] - outs[0]) <= 1e-11 * np.linalg.norm(outs[0])
