"""Adaptive refinement by V-cycles on the GPU (mg_refine) against the oracle's
refine (Sec. 3): the error that survives the cycles, the measured reduction
per cycle, every level's vectors, coarse operators and smoother of the refined
hierarchy, and solves with it; then the method's claim on a near-critical
64 x 64 three-level hierarchy, where refining the first and then the second
level removes most of the MG-CG iterations; and the argument checks."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import critical, krylov
from oracle import multigrid as omg
from oracle import wilson as ow

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = 1e-10
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def near_critical_32():
    L = 32
    U = W.quenched_u1(L, L, 3.0, 100, 1)
    m = critical.critical_mass_by_flow(U) + 0.002
    return L, U, m


BLOCKS = [(4, 4), (2, 2)]


@pytest.mark.parametrize("level", [1, 2])
def test_refine_matches_oracle(mg, near_critical_32, level):
    L, U, m = near_critical_32
    Nv = [3, 3]
    H = omg.setup(U, m, BLOCKS, Nv, W.setup_noise(L, L, BLOCKS, Nv, 7))
    lv = H.levels[level - 1]
    e0 = W.gaussian_field((lv.Lt, lv.Lx, lv.n), 20 + level)
    Nv2 = list(Nv)
    Nv2[level - 1] += 1
    noise2 = W.refine_noise(L, L, BLOCKS, Nv2, level - 1, 8)
    H2, e_want, rho_want = omg.refine(H, e0, 6, noise2, level=level - 1)
    with mg.Multigrid(dev(U), m, BLOCKS, Nv, dev(W.setup_noise(L, L, BLOCKS, Nv, 7))) as s:
        e_out = torch.empty(e0.shape, dtype=torch.complex128, device=DEV)
        nz = dev(noise2)
        rho = s.refine(level, dev(e0), 6, nz, e_out=e_out)
        assert rho == pytest.approx(rho_want, rel=1e-9)
        assert rel(host(e_out), e_want) <= 1e-8
        for l in range(H2.L - 1):
            ref = H2.levels[l]
            Lx, Lt, n, nv = mg.mg_get_level(s.h, l + 1)
            assert (Lx, Lt, n, nv) == (ref.Lx, ref.Lt, ref.n, ref.Nv)
            out = torch.empty((nv, Lt, Lx, n), dtype=torch.complex128, device=DEV)
            mg.mg_get_null_vectors(s.h, l + 1, out)
            assert np.max(np.abs(host(out) - ref.V)) <= 1e-8, f"vectors of level {l + 1}"
            c0, c1, _, _ = mg.mg_get_smoother(s.h, l + 1)
            assert c0 == pytest.approx(ref.c0, rel=1e-8) and c1 == pytest.approx(ref.c1, rel=1e-8)
        for l in range(1, H2.L):
            op = H2.levels[l].op
            out = torch.empty(op.M.shape, dtype=torch.complex128, device=DEV)
            mg.mg_get_coarse_op(s.h, l + 1, out)
            got = host(out)
            assert np.max(np.abs(got - op.M)) <= 1e-8 * np.max(np.abs(op.M)), f"A_c level {l + 1}"
        # solves with the refined hierarchy
        b = ow.apply_D(U, m, W.gaussian_field((L, L, 2), 3), dagger=True)
        _, it_want, _ = krylov.mgcg(H2, b, TOL, 5000)
        for solver in (mg.SOLVER_MGCG_FP64, mg.SOLVER_MGCG_MIXED):
            x, infos = s.solve(dev(b), tol=TOL, maxiter=5000, solver=solver)
            assert rel(ow.apply_A(U, m, host(x)), b) <= TOL and infos[0].true_residual <= TOL
            if solver == mg.SOLVER_MGCG_FP64:
                assert abs(infos[0].iterations - it_want) <= 1


def test_refinement_on_the_near_critical_64_hierarchy(mg):
    """64 x 64, beta = 3, seed 1 at its near-critical mass, blocks 4x4 then
    2x2, 8 relaxed vectors per level: two passes on the finest level and three
    on the second take the mixed MG-CG from hundreds of iterations to under
    half of them, every true residual <= 1e-10."""
    crit = json.load(open(os.path.join(ROOT, "workloads", "critical_masses_serving.json")))["L64_b3_s1"]
    L = 64
    th = W.quenched_u1_angles(L, L, 3.0, crit["sweeps"], 1)
    assert abs(W.mean_plaquette(th) - crit["plaquette"]) <= 1e-12
    U = W.links_from_angles(th)
    m = crit["m_nc"]
    Nv = [8, 8]
    b = ow.apply_D(U, m, W.gaussian_field((L, L, 2), 3), dagger=True)
    with mg.Multigrid(dev(U), m, BLOCKS, Nv, dev(W.setup_noise(L, L, BLOCKS, Nv, 7))) as s:
        counts = []
        for p, level in enumerate([None, 1, 1, 2, 2, 2]):
            if level is not None:
                Nv[level - 1] += 1
                Lx, Lt, n, _ = mg.mg_get_level(s.h, level)
                e0 = dev(W.gaussian_field((Lt, Lx, n), 100 + p))
                rho = s.refine(level, e0, 30, dev(W.refine_noise(L, L, BLOCKS, Nv, level - 1, 8 + p)))
                assert 0 < rho < 1
            x, infos = s.solve(dev(b), tol=TOL, maxiter=5000, solver=mg.SOLVER_MGCG_MIXED)
            assert rel(ow.apply_A(U, m, host(x)), b) <= TOL
            counts.append(infos[0].iterations)
        assert mg.mg_get_level(s.h, 1)[3] == 10 and mg.mg_get_level(s.h, 2)[3] == 11
        assert 2 * counts[-1] <= counts[0], counts


def test_refine_argument_checks(mg, near_critical_32):
    L, U, m = near_critical_32
    blocks, Nv = [(2, 2), (2, 2)], [4, 3]
    noise = dev(W.setup_noise(L, L, blocks, Nv, 7))
    with mg.Multigrid(dev(U), m, blocks, Nv, noise) as s:
        e0 = dev(W.gaussian_field((L, L, 2), 1))
        for level, ncyc in [(0, 1), (3, 1), (1, 0)]:
            with pytest.raises(mg.MgError) as ei:
                mg.mg_refine(s.h, level, e0, ncyc, noise)
            assert ei.value.status == 1                      # MG_ERR_ARG
        # 2x2 blocks of 2 spin components hold at most 4 vectors per chirality
        with pytest.raises(mg.MgError) as ei:
            mg.mg_refine(s.h, 1, e0, 1, noise)
        assert ei.value.status == 1
        # a zero error has no energy to measure
        with pytest.raises(mg.MgError) as ei:
            mg.mg_refine(s.h, 2, torch.zeros((L // 2, L // 2, 8), dtype=torch.complex128, device=DEV), 1)
        assert ei.value.status == 5                          # MG_ERR_BREAKDOWN
        # the last level above the coarsest needs no noise; the source is unchanged
        lv2 = mg.mg_get_level(s.h, 2)
        before = torch.empty((lv2[3], lv2[1], lv2[0], lv2[2]), dtype=torch.complex128, device=DEV)
        mg.mg_get_null_vectors(s.h, 2, before)
        h2, rho = mg.mg_refine(s.h, 2, dev(W.gaussian_field((L // 2, L // 2, 8), 2)), 3)
        try:
            assert 0 < rho < 1 and mg.mg_get_level(h2, 2)[3] == 4
            after = torch.empty_like(before)
            mg.mg_get_null_vectors(s.h, 2, after)
            assert torch.equal(before, after)
        finally:
            mg.mg_destroy(h2)


def test_setup_with_a_refinement_plan_matches_oracle(mg, near_critical_32):
    """mg_setup with refine_levels = 1, 2, 2 (the passes made in place, every
    random input from the one setup_noise buffer) against the oracle's setup
    with the same plan: the rho of each pass, every level's vectors and
    coarse operators, the exact memory accounting, solves, and a clone of the
    refined hierarchy at another mass."""
    L, U, m = near_critical_32
    Nv, plan = [3, 3], [1, 2, 2]
    noise = W.setup_noise(L, L, BLOCKS, Nv, 9, refine_levels=[lv - 1 for lv in plan])
    H = omg.setup(U, m, BLOCKS, Nv, noise, refine_levels=[lv - 1 for lv in plan], refine_cycles=5)
    with mg.Multigrid(dev(U), m, BLOCKS, Nv, dev(noise), refine_levels=plan, refine_cycles=5) as s:
        assert mg.mg_get_refine_rho(s.h) == pytest.approx(H.stats["refine_rho"], rel=1e-9)
        res, peak = mg.mg_setup_bytes(s.params)
        assert res == mg.mg_device_bytes(s.h) and peak > res
        for l in range(H.L - 1):
            ref = H.levels[l]
            Lx, Lt, n, nv = mg.mg_get_level(s.h, l + 1)
            assert (Lx, Lt, n, nv) == (ref.Lx, ref.Lt, ref.n, ref.Nv)
            out = torch.empty((nv, Lt, Lx, n), dtype=torch.complex128, device=DEV)
            mg.mg_get_null_vectors(s.h, l + 1, out)
            assert np.max(np.abs(host(out) - ref.V)) <= 1e-8, f"vectors of level {l + 1}"
        for l in range(1, H.L):
            op = H.levels[l].op
            out = torch.empty(op.M.shape, dtype=torch.complex128, device=DEV)
            mg.mg_get_coarse_op(s.h, l + 1, out)
            assert np.max(np.abs(host(out) - op.M)) <= 1e-8 * np.max(np.abs(op.M)), f"A_c level {l + 1}"
        b = ow.apply_D(U, m, W.gaussian_field((L, L, 2), 3), dagger=True)
        _, it_want, _ = krylov.mgcg(H, b, TOL, 5000)
        x, infos = s.solve(dev(b), tol=TOL, maxiter=5000, solver=mg.SOLVER_MGCG_FP64)
        assert rel(ow.apply_A(U, m, host(x)), b) <= TOL and abs(infos[0].iterations - it_want) <= 1
        # a clone at another mass keeps the refined vectors
        m2 = m + 0.5
        c = mg.mg_clone(s.h, m2)
        try:
            assert mg.mg_get_level(c, 2)[3] == 5 and mg.mg_device_bytes(c) == res
            H2 = omg.set_mass(H, m2)
            op = H2.levels[1].op
            out = torch.empty(op.M.shape, dtype=torch.complex128, device=DEV)
            mg.mg_get_coarse_op(c, 2, out)
            assert np.max(np.abs(host(out) - op.M)) <= 1e-8 * np.max(np.abs(op.M))
        finally:
            mg.mg_destroy(c)


def test_server_with_a_refined_configuration(mg, near_critical_32):
    """The serving engine builds a configuration whose parameters ask for
    adaptive passes (its set-up makes them; the other masses are clones of the
    refined hierarchy); every request reaches its tolerance."""
    L, U, m = near_critical_32
    Nv, plan = [3, 3], [1, 2]
    noise = dev(W.setup_noise(L, L, BLOCKS, Nv, 9, refine_levels=[lv - 1 for lv in plan]))
    masses = [m, m + 0.3]
    with mg.Server(budget_bytes=4 << 30, max_rhs=4, workers=2) as srv:
        p = mg.make_params(L, L, BLOCKS, Nv, refine_levels=plan, refine_cycles=10)
        cid = srv.add_config(dev(U), p, m, noise=noise)
        rids, bufs = [], []
        for k in range(6):
            mk = masses[k % 2]
            b = dev(ow.apply_D(U, mk, W.gaussian_field((L, L, 2), 700 + k), dagger=True))
            x = torch.empty_like(b)
            torch.cuda.synchronize()
            rids.append(srv.submit(cid, mk, b, x, 1, TOL, mg.SOLVER_MGCG_MIXED))
            bufs.append((mk, b, x))
        for r in rids:
            st, infos, _ = srv.wait(r, 1)
            assert st == 0 and infos[0].true_residual <= TOL
        stats = srv.stats()
        assert stats.builds == 1 and stats.clones == 1 and stats.failed == 0
    for mk, b, x in bufs:
        assert rel(ow.apply_A(U, mk, host(x)), host(b)) <= TOL
