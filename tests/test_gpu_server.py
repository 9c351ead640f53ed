"""Serving engine (include/mg_server.h) on the GPU: exact memory accounting of
a set-up, every result in a mixed request stream the same as the same
request solved alone (within the solver's tolerance, each true residual
recomputed by the oracle), and admission under a budget that holds one
hierarchy at a time."""
import numpy as np
import pytest

import workloads as W
from oracle import critical
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


# (L, beta, sweeps, seed, setup mass, blocks, Nv, masses served)
CONFIGS = [(32, 6.0, 100, 1, -1.5, [(4, 4), (2, 2)], [4, 4], [-1.5, -0.5]),
           (48, 3.0, 60, 2, -1.2, [(4, 4)], [4], [-1.2, 0.05])]


@pytest.mark.parametrize("kw", [dict(), dict(max_rhs=4), dict(coarsest_dense_max=0)],
                         ids=["default", "max_rhs4", "coarsest_cg"])
def test_setup_bytes_equal_the_allocations(mg, kw):
    L, beta, sweeps, seed, m0, blocks, Nv, _ = CONFIGS[0]
    U = dev(W.quenched_u1(L, L, beta, sweeps, seed))
    noise = dev(W.setup_noise(L, L, blocks, Nv, 5))
    with mg.Multigrid(U, m0, blocks, Nv, noise, **kw) as s:
        res, peak = mg.mg_setup_bytes(s.params)
        assert mg.mg_device_bytes(s.h) == res
        assert peak > res


def test_clone_equals_set_mass(mg):
    """mg_clone(h, m) builds the same hierarchy as mg_set_mass(h, m) (bit for
    bit: same vectors, same deterministic kernels) and leaves h unchanged."""
    L, beta, sweeps, seed, m0, blocks, Nv, ms = CONFIGS[0]
    U = dev(W.quenched_u1(L, L, beta, sweeps, seed))
    noise = dev(W.setup_noise(L, L, blocks, Nv, 5))
    m1 = ms[1]
    with mg.Multigrid(U, m0, blocks, Nv, noise) as a, mg.Multigrid(U, m0, blocks, Nv, noise) as b:
        c = mg.mg_clone(a.h, m1)
        try:
            b.set_mass(m1)
            for lvl in range(2, len(blocks) + 2):
                Lx, Lt, n, _ = mg.mg_get_level(a.h, lvl)
                shape = (Lt * Lx * 9 * n * n,)
                oa, ob, oc = (torch.empty(shape, dtype=torch.complex128, device=DEV) for _ in range(3))
                mg.mg_get_coarse_op(a.h, lvl, oa)
                mg.mg_get_coarse_op(b.h, lvl, ob)
                mg.mg_get_coarse_op(c, lvl, oc)
                assert torch.equal(ob, oc)                     # clone == re-massed copy
                assert not torch.equal(oa, oc)                 # the source kept its mass
            assert mg.mg_device_bytes(c) == mg.mg_device_bytes(a.h)
        finally:
            mg.mg_destroy(c)


def _requests():
    """Mixed stream: (config, mass, nrhs, source seeds), interleaved."""
    rng = np.random.default_rng(11)
    reqs = []
    for k in range(12):
        c = k % 2
        m = CONFIGS[c][7][(k // 2) % 2]
        nrhs = int(rng.integers(1, 5))
        reqs.append((c, m, nrhs, [500 + 10 * k + j for j in range(nrhs)]))
    return reqs


def _inputs():
    out = []
    for L, beta, sweeps, seed, m0, blocks, Nv, _ in CONFIGS:
        U = W.quenched_u1(L, L, beta, sweeps, seed)
        out.append((U, W.setup_noise(L, L, blocks, Nv, 5)))
    return out


def _kappa_bound(U, m):
    # lambda_max(A) <= (|4 + m| + 4)^2; lambda_min(A) = (eigenvalue of sigma_3 D nearest 0)^2
    lam, _ = critical.nearest_eig_H(U, m)
    return (abs(4.0 + m) + 4.0) ** 2 / lam ** 2


@pytest.mark.parametrize("solver", ["mixed", "fp64"])
def test_results_same_alone_and_in_the_mix(mg, solver):
    code = mg.SOLVER_MGCG_MIXED if solver == "mixed" else mg.SOLVER_MGCG_FP64
    inputs = _inputs()
    reqs = _requests()
    bs = []
    for c, m, nrhs, seeds in reqs:
        L = CONFIGS[c][0]
        U = inputs[c][0]
        chi = np.stack([W.gaussian_field((L, L, 2), sd) for sd in seeds])
        bs.append(np.stack([ow.apply_D(U, m, chi[j], dagger=True) for j in range(nrhs)]))
    # alone: each request in its own solve on a dedicated handle
    alone = []
    for (c, m, nrhs, _), b in zip(reqs, bs):
        L, beta, sweeps, seed, m0, blocks, Nv, _ = CONFIGS[c]
        with mg.Multigrid(dev(inputs[c][0]), m0, blocks, Nv, dev(inputs[c][1]), max_rhs=nrhs) as s:
            if m != m0:
                s.set_mass(m)
            x, infos = s.solve(dev(b), tol=TOL, maxiter=5000, solver=code)
            alone.append(host(x).reshape(b.shape))
    # in the mix: every request queued at once, two workers, batches up to 8 RHS
    with mg.Server(budget_bytes=8 << 30, max_rhs=8, workers=2) as srv:
        ids = []
        for c, (L, beta, sweeps, seed, m0, blocks, Nv, _) in enumerate(CONFIGS):
            p = mg.make_params(L, L, blocks, Nv)
            ids.append(srv.add_config(dev(inputs[c][0]), p, m0, noise=dev(inputs[c][1])))
        xs, rids = [], []
        for (c, m, nrhs, _), b in zip(reqs, bs):
            bd = dev(b)
            xd = torch.full_like(bd, float("nan"))
            torch.cuda.synchronize()
            rids.append(srv.submit(ids[c], m, bd, xd, nrhs, TOL, code))
            xs.append(xd)
        results = [srv.wait(r, reqs[k][2]) for k, r in enumerate(rids)]
        st = srv.stats()
        assert st.completed == len(reqs) and st.failed == 0
        assert st.batches < len(reqs)              # some requests shared a batch
        assert st.builds == 2 and st.clones == 2      # one set-up per config, one clone per other mass
        assert st.remasses == 0 and st.p99_ms >= st.p50_ms > 0
    for k, ((c, m, nrhs, _), b) in enumerate(zip(reqs, bs)):
        status, infos, lat = results[k]
        assert status == 0 and lat > 0
        got = host(xs[k]).reshape(b.shape)
        U = inputs[c][0]
        kappa = _kappa_bound(U, m)
        for j in range(nrhs):
            res = np.linalg.norm(b[j] - ow.apply_A(U, m, got[j])) / np.linalg.norm(b[j])
            assert res <= TOL and infos[j].true_residual <= TOL
            # both solutions within kappa * tol of the exact one
            assert np.linalg.norm(got[j] - alone[k][j]) <= 2.5 * kappa * TOL * np.linalg.norm(alone[k][j])


def test_admission_one_hierarchy_at_a_time(mg):
    inputs = _inputs()
    need = []
    for c, (L, beta, sweeps, seed, m0, blocks, Nv, _) in enumerate(CONFIGS):
        p = mg.make_params(L, L, blocks, Nv, max_rhs=4)
        p.setup_noise = 1                          # sizes only; never dereferenced
        need.append(mg.mg_setup_bytes(p)[1] + 2 * 4 * L * L * 2 * 16)
    budget = max(need) + min(need) // 2           # never both resident
    with mg.Server(budget_bytes=budget, max_rhs=4, workers=2) as srv:
        ids = []
        for c, (L, beta, sweeps, seed, m0, blocks, Nv, _) in enumerate(CONFIGS):
            ids.append(srv.add_config(dev(inputs[c][0]), mg.make_params(L, L, blocks, Nv), m0,
                                      noise=dev(inputs[c][1])))
        rids, bufs = [], []
        for k in range(6):
            c = k % 2
            L, m = CONFIGS[c][0], CONFIGS[c][7][1]
            b = dev(ow.apply_D(inputs[c][0], m, W.gaussian_field((L, L, 2), 900 + k), dagger=True))
            x = torch.empty_like(b)
            torch.cuda.synchronize()
            rids.append(srv.submit(ids[c], m, b, x, 1, TOL, mg.SOLVER_MGCG_MIXED))
            bufs.append((c, m, b, x))
        for r in rids:
            st, infos, _ = srv.wait(r, 1)
            assert st == 0 and infos[0].true_residual <= TOL
        stats = srv.stats()
        assert stats.evictions >= 1 and stats.builds >= 2
        assert stats.peak_resident_bytes <= budget
    for c, m, b, x in bufs:
        got, bb = host(x), host(b)
        res = np.linalg.norm(bb - ow.apply_A(inputs[c][0], m, got)) / np.linalg.norm(bb)
        assert res <= TOL


def test_configuration_above_the_budget_fails_cleanly(mg):
    L, beta, sweeps, seed, m0, blocks, Nv, _ = CONFIGS[0]
    U = dev(W.quenched_u1(L, L, beta, sweeps, seed))
    noise = dev(W.setup_noise(L, L, blocks, Nv, 5))
    with mg.Server(budget_bytes=1 << 20, max_rhs=2, workers=1) as srv:
        cid = srv.add_config(U, mg.make_params(L, L, blocks, Nv), m0, noise=noise)
        b = torch.ones((L, L, 2), dtype=torch.complex128, device=DEV)
        x = torch.empty_like(b)
        st, _, _ = srv.wait(srv.submit(cid, m0, b, x, 1), 1)
        assert st == 2                                 # MG_ERR_NOMEM
        assert srv.stats().failed == 1


def test_failed_clone_fails_its_own_group_only(mg):
    """Two clones of one configuration built at once, one of them failing (a
    host-side injected MG_ERR_CUDA in place of mg_clone): the requests at the
    failed clone's mass fail with that status, the requests at the other mass
    are solved (true residual recomputed by the oracle), and the server goes on
    serving the failed mass afterwards with a new clone."""
    L, beta, sweeps, seed, m0, blocks, Nv, ms = CONFIGS[0]
    Uh = W.quenched_u1(L, L, beta, sweeps, seed)
    m1, m2 = ms[1], -1.0
    with mg.Server(budget_bytes=8 << 30, max_rhs=4, workers=3) as srv:
        cid = srv.add_config(dev(Uh), mg.make_params(L, L, blocks, Nv), m0,
                             noise=dev(W.setup_noise(L, L, blocks, Nv, 5)))

        def submit(m, sd):
            b = dev(ow.apply_D(Uh, m, W.gaussian_field((L, L, 2), sd), dagger=True))
            x = torch.full_like(b, float("nan"))
            torch.cuda.synchronize()
            return srv.submit(cid, m, b, x, 1, TOL, mg.SOLVER_MGCG_MIXED), b, x

        r0, _, _ = submit(m0, 700)
        assert srv.wait(r0, 1)[0] == 0                 # the set-up is resident
        srv.inject_build_failures(1)
        first = [submit(m1, 710), submit(m1, 711)]     # oldest group: its clone takes the failure
        second = [submit(m2, 720), submit(m2, 721)]
        for rid, _, _ in first:
            assert srv.wait(rid, 1)[0] == 3            # MG_ERR_CUDA
        for rid, b, x in second:
            st, infos, _ = srv.wait(rid, 1)
            assert st == 0 and infos[0].true_residual <= TOL
            res = np.linalg.norm(host(b) - ow.apply_A(Uh, m2, host(x))) / np.linalg.norm(host(b))
            assert res <= TOL
        rid, b, x = submit(m1, 730)                    # served again: a new clone
        st, infos, _ = srv.wait(rid, 1)
        assert st == 0 and infos[0].true_residual <= TOL
        stats = srv.stats()
        assert stats.failed == 2 and stats.completed == 4 and stats.clones == 2
