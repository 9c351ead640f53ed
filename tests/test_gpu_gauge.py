"""Gauge generation on the GPU (mg_gauge_metropolis, mg_gauge_links) against
the host generator with the same counter-based uniforms
(workloads.quenched_u1_angles_counter): the same accept decisions and the
same angles bit for bit (both round every angle operation the same way), the
same accepted count, chunked runs equal to one run, links within rounding of
exp(i theta), and a multigrid set-up on the generated field."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0710_3612_gb300 import mg as m
    return m


def host_run(Lx, Lt, beta, sweeps, seed, eps=1.0, theta=None, first=0):
    theta = np.zeros((2, Lt, Lx)) if theta is None else theta.copy()
    acc = 0
    for sw in range(first, first + sweeps):
        for mu in (0, 1):
            for parity in (0, 1):
                u, a = W.metropolis_uniforms(Lx, Lt, seed, sw, mu, parity)
                acc += W._metropolis_half_u(theta, mu, parity, beta, eps, u, a)
    return theta, acc


@pytest.mark.parametrize("Lx,Lt,beta,sweeps,seed,eps", [(64, 64, 3.0, 20, 1, 1.0),
                                                        (48, 32, 10.0, 30, 2**40 + 7, 0.7),
                                                        (2, 6, 1.0, 5, 3, 1.0)],
                         ids=["64x64_b3", "48x32_b10_eps07_seed_above_32bit", "2x6_smallest"])
def test_gpu_metropolis_equals_host(mg, Lx, Lt, beta, sweeps, seed, eps):
    want, acc_want = host_run(Lx, Lt, beta, sweeps, seed, eps)
    th = torch.zeros((2, Lt, Lx), dtype=torch.float64, device=DEV)
    acc = mg.gauge_metropolis(th, beta, sweeps, seed, eps=eps)
    got = th.cpu().numpy()
    assert acc == acc_want
    assert np.array_equal(got, want), f"{np.count_nonzero(got != want)} angles differ"


def test_gpu_metropolis_chunks(mg):
    Lx, Lt = 32, 16
    th = torch.zeros((2, Lt, Lx), dtype=torch.float64, device=DEV)
    mg.gauge_metropolis(th, 4.0, 7, 11)
    th2 = torch.zeros_like(th)
    mg.gauge_metropolis(th2, 4.0, 3, 11)
    mg.gauge_metropolis(th2, 4.0, 4, 11, first_sweep=3)
    assert torch.equal(th, th2)
    assert mg.gauge_metropolis(th2, 4.0, 0, 11, first_sweep=7) == 0   # no sweeps, no change
    assert torch.equal(th, th2)


def test_gpu_links_and_setup(mg):
    Lx = Lt = 64
    th = torch.zeros((2, Lt, Lx), dtype=torch.float64, device=DEV)
    mg.gauge_metropolis(th, 6.0, 50, 5)
    U = mg.gauge_links(th)
    want = W.links_from_angles(th.cpu().numpy())
    assert np.max(np.abs(U.cpu().numpy() - want)) <= 4e-16
    noise = torch.from_numpy(W.setup_noise(Lx, Lt, [(4, 4)], [4], 1)).to(DEV)
    with mg.Multigrid(U, 0.05, [(4, 4)], [4], noise) as s:
        b = torch.from_numpy(W.gaussian_field((Lt, Lx, 2), 2)).to(DEV)
        _, infos = s.solve(b, tol=1e-10)
        assert infos[0].true_residual <= 1e-10


def test_gpu_metropolis_argument_checks(mg):
    th = torch.zeros((2, 5, 8), dtype=torch.float64, device=DEV)     # odd Lt
    with pytest.raises(mg.MgError):
        mg.gauge_metropolis(th, 1.0, 1, 1)
    th = torch.zeros((2, 4, 8), dtype=torch.float64, device=DEV)
    with pytest.raises(mg.MgError):
        mg.gauge_metropolis(th, 1.0, 1, 1, eps=0.0)
