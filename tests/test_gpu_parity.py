"""GPU parity: every step of the hot path, called through the C ABI, against the
CPU oracle on the same seeded inputs.

Tolerances (per element): |gpu - oracle| <= tol * (|oracle| + M) where M is the
sum of magnitudes of the terms that make up the element (computed by applying
the absolute value of the operator to the absolute value of the input);
tol = 1e-12 for FP64, 1e-6 for FP32, 8e-3 for BF16 coarse blocks (2^-8
relative rounding of each block entry).  Integer maps are compared bit for bit.
"""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as okr
from oracle import multigrid as omg
from oracle import wilson as ow

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32, TOL16 = 1e-12, 1e-6, 8e-3


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0710_3612_gb300 import mg as m
    return m


DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def check(got, want, mag, tol, what=""):
    err = np.abs(got - want)
    bound = tol * (np.abs(want) + mag)
    worst = np.max(err / np.maximum(bound, 1e-300))
    assert worst <= 1.0, f"{what}: worst error / bound = {worst:.3g} (max err {err.max():.3e})"


def bf16_round(a):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def bf16_blocks(M):
    """The GPU's BF16 copy of FP64 coarse blocks: FP64 -> FP32 -> BF16, each rounded to nearest."""
    re = bf16_round(M.real.astype(np.float32)).astype(np.float64)
    im = bf16_round(M.imag.astype(np.float32)).astype(np.float64)
    return re + 1j * im


def gpu_vectors(mg, c, l):
    """The GPU set-up's own block vectors of level l (0 = finest), [Nv, Lt, Lx, n]."""
    Lx, Lt, n, Nv = mg.mg_get_level(c.h, l + 1)
    out = torch.empty((Nv, Lt, Lx, n), dtype=torch.complex128, device=DEV)
    mg.mg_get_null_vectors(c.h, l + 1, out)
    return host(out)


def gpu_coarse_op(mg, c, l):
    """The GPU set-up's own FP64 coarse operator of level l >= 1 as an oracle stencil."""
    op = c.H.levels[l].op
    out = torch.empty(op.M.shape, dtype=torch.complex128, device=DEV)
    mg.mg_get_coarse_op(c.h, l + 1, out)
    return omg.StencilOp(omg.COARSE_DISP, host(out))


def abs_normal_stencil(U, m):
    """|D|^T |D| as a stencil: the sum of magnitudes of the terms of A = D^dagger D."""
    dd, Md = ow.wilson_stencil(U, m, dagger=True)
    d_, M = ow.wilson_stencil(U, m, dagger=False)
    Md, M = np.abs(Md), np.abs(M)
    acc = {}
    for e1, (ax, at) in enumerate(dd):
        Ms = np.roll(M, shift=(-at, -ax), axis=(0, 1))
        for e2, (bx, bt) in enumerate(d_):
            key = (ax + bx, at + bt)
            acc[key] = acc.get(key, 0) + np.einsum("txab,txbc->txac", Md[:, :, e1], Ms[:, :, e2])
    disp = sorted(acc)
    return omg.StencilOp(disp, np.stack([acc[k] for k in disp], axis=2))


# ---------------------------------------------------------------------------
# configurations: (Lx, Lt, beta, sweeps, seed, mass, blocks, Nv)
# ---------------------------------------------------------------------------
CASES = {
    # two levels, coarse 6 x 4
    "2lvl_24x16": (24, 16, 6.0, 40, 1, -0.7, [(4, 4)], [4]),
    # three levels, coarse extents 6x6 -> 3x3 (odd coarse extent)
    "3lvl_24x24": (24, 24, 6.0, 40, 2, -1.2, [(4, 4), (2, 2)], [3, 4]),
    # three levels with a coarsest extent of 2 (+1 and -1 neighbours alias)
    "3lvl_16x16_alias": (16, 16, 3.0, 30, 3, -0.4, [(4, 4), (2, 2)], [2, 3]),
    # the benchmark's coarse shapes: 16 dof (Nv = 8) on 8 x 8, 24 dof (Nv = 12) on 4 x 4
    "3lvl_32x32_nv8_12": (32, 32, 6.0, 40, 4, -0.9, [(4, 4), (2, 2)], [8, 12]),
}


class Case:
    def __init__(self, mg, name):
        Lx, Lt, beta, sweeps, seed, m, blocks, Nv = CASES[name]
        self.Lx, self.Lt, self.m, self.blocks, self.Nv = Lx, Lt, m, blocks, Nv
        self.U = W.links_from_angles(W.quenched_u1_angles(Lx, Lt, beta, sweeps, seed))
        self.noise = W.setup_noise(Lx, Lt, blocks, Nv, seed + 100)
        self.H = omg.setup(self.U, m, blocks, Nv, self.noise)
        self.Ug, self.noise_g = dev(self.U), dev(self.noise)
        self.solver = mg.Multigrid(self.Ug, m, blocks, Nv, self.noise_g)
        self.h = self.solver.h


@pytest.fixture(scope="module", params=list(CASES))
def case(request, mg):
    c = Case(mg, request.param)
    yield c
    c.solver.close()


def abs_dirac(U, m):
    return abs(ow.dirac_matrix(U, m))


# ---------------------------------------------------------------------------
def test_block_map_bit_exact(mg):
    for Lx, Lt, bx, bt in [(16, 8, 4, 4), (12, 18, 2, 3), (128, 128, 4, 4), (6, 4, 2, 2)]:
        c = torch.empty(Lx * Lt, dtype=torch.int32, device=DEV)
        o = torch.empty(Lx * Lt, dtype=torch.int32, device=DEV)
        mg.mg_block_map(Lx, Lt, bx, bt, c, o)
        cw, ow_ = omg.block_map(Lx, Lt, bx, bt)
        assert np.array_equal(host(c), cw) and np.array_equal(host(o), ow_)


@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_apply_D(case, mg, dagger, prec):
    nrhs = 3
    psi = W.gaussian_field((nrhs, case.Lt, case.Lx, 2), 5)
    want = ow.apply_D(case.U, case.m, psi, dagger=bool(dagger))
    Dabs = abs_dirac(case.U, case.m)
    mag = (Dabs @ np.abs(psi).reshape(nrhs, -1).T).T.reshape(psi.shape)
    if prec == "f64":
        out = torch.empty_like(dev(psi))
        mg.mg_apply_D(case.h, dev(psi), out, nrhs, dagger, mg.PREC_F64)
        check(host(out), want, mag, TOL64, "D f64")
    else:
        inp = dev(psi.astype(np.complex64))
        out = torch.empty_like(inp)
        mg.mg_apply_D(case.h, inp, out, nrhs, dagger, mg.PREC_F32)
        check(host(out), want, mag, TOL32, "D f32")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_apply_A(case, mg, prec):
    nrhs = 2
    psi = W.gaussian_field((nrhs, case.Lt, case.Lx, 2), 6)
    want = ow.apply_A(case.U, case.m, psi)
    Dabs = abs_dirac(case.U, case.m)
    mag = (Dabs.T @ (Dabs @ np.abs(psi).reshape(nrhs, -1).T)).T.reshape(psi.shape)
    if prec == "f64":
        out = torch.empty_like(dev(psi))
        mg.mg_apply_A(case.h, dev(psi), out, nrhs, mg.PREC_F64)
        check(host(out), want, mag, TOL64, "A f64")
    else:
        inp = dev(psi.astype(np.complex64))
        out = torch.empty_like(inp)
        mg.mg_apply_A(case.h, inp, out, nrhs, mg.PREC_F32)
        check(host(out), want, mag, TOL32, "A f32")


def test_null_vectors_and_smoother(case, mg):
    H = case.H
    for l in range(H.L - 1):
        lv = H.levels[l]
        Lx, Lt, n, Nv = mg.mg_get_level(case.h, l + 1)
        assert (Lx, Lt, n, Nv) == (lv.Lx, lv.Lt, lv.n, lv.Nv)
        out = torch.empty((Nv, Lt, Lx, n), dtype=torch.complex128, device=DEV)
        mg.mg_get_null_vectors(case.h, l + 1, out)
        got = host(out)
        # unit-norm block vectors: entries O(1/sqrt(block dim)); relaxation and
        # Gram-Schmidt amplify rounding mildly
        check(got, lv.V, np.ones_like(np.abs(lv.V)), 1e-10, f"V level {l + 1}")
        c0, c1, lam, om = mg.mg_get_smoother(case.h, l + 1)
        assert c0 == pytest.approx(lv.c0, rel=1e-10) and c1 == pytest.approx(lv.c1, rel=1e-10)
        assert om == pytest.approx(lv.omega_relax, rel=1e-11)


def test_coarse_operators(case, mg):
    """Two comparisons.  The Galerkin kernels at 1e-12 per element: the GPU's
    A_{l+1} against the oracle's P^dagger A_l P formed from the GPU's own
    vectors V_l and its own A_l (level 0: the oracle's A = D^dagger D), the
    magnitude bound from the same product of absolute values.  The whole
    set-up at 1e-11 of the row maximum: the GPU's A_{l+1} against the oracle's
    own set-up (relaxation and Gram-Schmidt on both sides)."""
    H = case.H
    for l in range(1, H.L):
        op = H.levels[l].op
        got = gpu_coarse_op(mg, case, l).M
        rowmax = np.max(np.abs(op.M), axis=(2, 4), keepdims=True)
        check(got, op.M, rowmax, 1e-11, f"A_c level {l + 1} (set-up)")
        lv = H.levels[l - 1]
        V = gpu_vectors(mg, case, l - 1)
        if l == 1:
            fine = omg.WilsonNormalOp(case.U, case.m)
            fine_abs = abs_normal_stencil(case.U, case.m)
        else:
            fine = gpu_coarse_op(mg, case, l - 1)
            fine_abs = omg.StencilOp(fine.disp, np.abs(fine.M))
        want = omg.galerkin(fine, V, lv.bx, lv.bt).M
        mag = omg.galerkin(fine_abs, np.abs(V), lv.bx, lv.bt).M.real
        check(got, want, mag, TOL64, f"A_c level {l + 1} (Galerkin kernels)")


@pytest.mark.parametrize("prec,nrhs,kernel", [("f64", 2, 0), ("f32", 2, 0), ("bf16", 2, 0),
                                              ("bf16", 16, 0), ("bf16", 13, 0), ("bf16", 64, 0),
                                              ("bf16", 16, 1), ("bf16", 13, 1), ("bf16", 64, 1)])
def test_apply_coarse(case, mg, prec, nrhs, kernel):
    """nrhs >= 8 with BF16 blocks runs on the tensor cores (BF16 operands,
    FP32 accumulation): kernel 0 = tcgen05 (levels with 16 or 24 dof; others
    fall back to mma.sync), 1 = mma.sync; 13 checks the right-hand-side
    padding, 64 the full M tile."""
    mg.mg_set_coarse_tensor_kernel(kernel)
    try:
        _apply_coarse(case, mg, prec, nrhs)
    finally:
        mg.mg_set_coarse_tensor_kernel(0)


def _apply_coarse(case, mg, prec, nrhs):
    H = case.H
    for l in range(1, H.L):
        ora = H.levels[l].op
        op = gpu_coarse_op(mg, case, l)      # the GPU's own blocks: the kernel alone is compared
        v = W.gaussian_field((nrhs, op.Lt, op.Lx, op.n), 11 + l)
        want = op.apply(v)
        mag = omg.StencilOp(op.disp, np.abs(op.M)).apply(np.abs(v))
        # the same input through the oracle's own blocks differs only by the set-up's rounding
        mag_o = omg.StencilOp(ora.disp, np.abs(ora.M)).apply(np.abs(v))
        check(want, ora.apply(v), mag_o, 1e-11, "coarse blocks (set-up)")
        if prec == "f64":
            out = torch.empty_like(dev(v))
            mg.mg_apply_coarse(case.h, l + 1, dev(v), out, nrhs, mg.PREC_F64)
            check(host(out), want, mag, TOL64, "coarse f64")
        else:
            inp = dev(v.astype(np.complex64))
            out = torch.empty_like(inp)
            code = mg.PREC_F32 if prec == "f32" else mg.PREC_BF16
            mg.mg_apply_coarse(case.h, l + 1, inp, out, nrhs, code)
            got = host(out)
            check(got, want, mag, TOL32 if prec == "f32" else TOL16, f"coarse {prec}")
            if prec == "bf16":
                # with the stored BF16 blocks themselves only the split of X into
                # two BF16 parts (2^-18 relative) and FP32 accumulation remain
                want16 = omg.StencilOp(op.disp, bf16_blocks(op.M)).apply(v.astype(np.complex64))
                check(got, want16, mag, 3e-5, "coarse bf16 (stored blocks)")


@pytest.mark.parametrize("prec,nrhs", [("f64", 2), ("f32", 2), ("f64", 9), ("f32", 9)])
def test_restrict_prolong(case, mg, prec, nrhs):
    """Several right-hand sides per call (one CTA per coarse site)."""
    H = case.H
    tol = TOL64 if prec == "f64" else TOL32
    for l in range(H.L - 1):
        lv = H.levels[l]
        V = gpu_vectors(mg, case, l)         # the GPU's own vectors: the kernels alone are compared
        check(V, lv.V, np.ones_like(np.abs(lv.V)), 1e-10, "V (set-up)")
        r = W.gaussian_field((nrhs, lv.Lt, lv.Lx, lv.n), 21 + l)
        ec = W.gaussian_field((nrhs, lv.Lt // lv.bt, lv.Lx // lv.bx, 2 * lv.Nv), 31 + l)
        want_c = omg.restrict(V, lv.bx, lv.bt, r)
        mag_c = np.stack([omg.restrict(np.abs(V), lv.bx, lv.bt, np.abs(x)) for x in r])
        want_f = omg.prolong(V, lv.bx, lv.bt, ec)
        mag_f = np.stack([omg.prolong(np.abs(V), lv.bx, lv.bt, np.abs(x)) for x in ec])
        dt = np.complex128 if prec == "f64" else np.complex64
        code = mg.PREC_F64 if prec == "f64" else mg.PREC_F32
        out_c = torch.empty(want_c.shape, dtype=torch.complex128 if prec == "f64" else torch.complex64, device=DEV)
        mg.mg_restrict(case.h, l + 1, dev(r.astype(dt)), out_c, nrhs, code)
        check(host(out_c), want_c, mag_c, tol, "restrict")
        out_f = torch.empty(want_f.shape, dtype=out_c.dtype, device=DEV)
        mg.mg_prolong(case.h, l + 1, dev(ec.astype(dt)), out_f, nrhs, code)
        check(host(out_f), want_f, mag_f, tol, "prolong")


def test_coarsest_solve(case, mg):
    H = case.H
    last = H.levels[-1]
    b = W.gaussian_field((last.Lt, last.Lx, last.n), 41)
    want = omg.coarsest_solve(H, b)
    out = torch.empty_like(dev(b))
    mg.mg_coarsest_solve(case.h, dev(b), out)
    got = host(out)
    assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)


def test_vcycle_f64(case, mg):
    r = W.gaussian_field((case.Lt, case.Lx, 2), 51)
    want = omg.vcycle(case.H, r)
    out = torch.empty_like(dev(r))
    mg.mg_vcycle(case.h, dev(r), out, mg.PREC_F64)
    got = host(out)
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_vcycle_f32_is_close(case, mg):
    """The FP32 V-cycle (BF16 coarse blocks) is a perturbed preconditioner: close
    to the FP64 one at the BF16 level, and still Hermitian positive in effect."""
    r = W.gaussian_field((case.Lt, case.Lx, 2), 52)
    want = omg.vcycle(case.H, r)
    inp = dev(r.astype(np.complex64))
    out = torch.empty_like(inp)
    mg.mg_vcycle(case.h, inp, out, mg.PREC_F32)
    got = host(out)
    assert np.linalg.norm(got - want) <= 5e-2 * np.linalg.norm(want)
    assert np.vdot(r, got).real > 0


@pytest.mark.parametrize("solver", ["mgcg_fp64", "mixed", "reliable", "cg_fp64"])
def test_solve_matches_oracle(case, mg, solver):
    chi = W.gaussian_field((case.Lt, case.Lx, 2), 61)
    b = ow.apply_D(case.U, case.m, chi, dagger=True)
    tol = 1e-10
    x_ora, it_ora, info_ora = okr.mgcg(case.H, b, 1e-12)
    code = {"mgcg_fp64": mg.SOLVER_MGCG_FP64, "mixed": mg.SOLVER_MGCG_MIXED,
            "reliable": mg.SOLVER_MGCG_RELIABLE, "cg_fp64": mg.SOLVER_CG_FP64}[solver]
    x, infos = case.solver.solve(dev(b), tol=tol, maxiter=20000, solver=code)
    got = host(x).reshape(b.shape)
    A = case.H.levels[0].op
    res = np.linalg.norm(b - A.apply(got)) / np.linalg.norm(b)
    assert res <= tol and infos[0].true_residual <= tol
    assert abs(infos[0].true_residual - res) <= 1e-3 * tol + 1e-15
    # |x - x*| <= kappa * |r| / |b| * |x*|  (kappa from the oracle's dense operator)
    lam = np.linalg.eigvalsh(A.dense()) if case.Lx * case.Lt <= 600 else None
    kappa = lam[-1] / lam[0] if lam is not None else 1e6
    assert np.linalg.norm(got - x_ora) <= (kappa * tol + 1e-10) * np.linalg.norm(x_ora)
    if solver == "mgcg_fp64":
        x10, it10, _ = okr.mgcg(case.H, b, tol)
        assert abs(infos[0].iterations - it10) <= 1


def test_zero_rhs_and_repeatability(case, mg):
    b = torch.zeros((case.Lt, case.Lx, 2), dtype=torch.complex128, device=DEV)
    x, infos = case.solver.solve(b, solver=mg.SOLVER_MGCG_FP64)
    assert infos[0].iterations == 0 and not torch.any(x != 0)
    chi = W.gaussian_field((case.Lt, case.Lx, 2), 71)
    bb = dev(ow.apply_D(case.U, case.m, chi, dagger=True))
    x1, _ = case.solver.solve(bb, solver=mg.SOLVER_MGCG_MIXED)
    x1 = host(x1)
    x2, _ = case.solver.solve(bb, solver=mg.SOLVER_MGCG_MIXED)
    assert np.array_equal(x1, host(x2))     # fixed reduction order: identical bits


@pytest.mark.parametrize("solver", ["mgcg_fp64", "mixed", "reliable", "cg_fp64"])
def test_graph_loop_matches_eager_loop(case, mg, solver):
    """The Krylov loop runs as one CUDA graph with a device-side WHILE condition
    (and, for the reliable-update solver, an IF node for the update); with
    per-kernel profiling on it runs eagerly.  Both give identical bits."""
    code = {"mgcg_fp64": mg.SOLVER_MGCG_FP64, "mixed": mg.SOLVER_MGCG_MIXED,
            "reliable": mg.SOLVER_MGCG_RELIABLE, "cg_fp64": mg.SOLVER_CG_FP64}[solver]
    chi = W.gaussian_field((case.Lt, case.Lx, 2), 81)
    b = dev(ow.apply_D(case.U, case.m, chi, dagger=True))
    xg, ig = case.solver.solve(b, tol=1e-10, maxiter=20000, solver=code)
    xg = host(xg)
    mg.mg_profile_enable(case.h, True)
    try:
        xe, ie = case.solver.solve(b, tol=1e-10, maxiter=20000, solver=code)
        xe = host(xe)
    finally:
        mg.mg_profile_enable(case.h, False)
    assert ig[0].iterations == ie[0].iterations
    assert np.array_equal(xg, xe)


@pytest.mark.parametrize("solver", ["mgcg_fp64", "mixed"])
def test_batched_solve_matches_single(mg, solver):
    """Five right-hand sides with max_rhs = 4 (one batch of 4, one of 1): every
    solution meets the true-residual target and agrees with the one-at-a-time
    solve within kappa * tol; iteration counts within one of each other."""
    c = Case(mg, "3lvl_24x24")
    code = mg.SOLVER_MGCG_FP64 if solver == "mgcg_fp64" else mg.SOLVER_MGCG_MIXED
    try:
        chis = W.gaussian_field((5, c.Lt, c.Lx, 2), 123)
        b = np.stack([ow.apply_D(c.U, c.m, x, dagger=True) for x in chis])
        A = c.H.levels[0].op
        with mg.Multigrid(c.Ug, c.m, c.blocks, c.Nv, c.noise_g, max_rhs=4) as sb:
            xb, ib = sb.solve(dev(b), tol=1e-10, maxiter=20000, solver=code)
            xb = host(xb)
        lam = np.linalg.eigvalsh(A.dense())
        for k in range(5):
            xs, i1 = c.solver.solve(dev(b[k]), tol=1e-10, maxiter=20000, solver=code)
            xs = host(xs).reshape(b[k].shape)
            res = np.linalg.norm(b[k] - A.apply(xb[k])) / np.linalg.norm(b[k])
            assert res <= 1e-10 and ib[k].true_residual <= 1e-10
            assert np.linalg.norm(xb[k] - xs) <= 2 * lam[-1] / lam[0] * 1e-10 * np.linalg.norm(xs)
            assert abs(ib[k].iterations - i1[0].iterations) <= 1
    finally:
        c.solver.close()


def test_batched_tensor_core_vcycle_solve(mg):
    """Eight right-hand sides together: the coarse applies of the FP32 V-cycle
    run on the tensor cores; every solve meets the true-residual target and
    matches the oracle's solution within kappa * tol."""
    c = Case(mg, "3lvl_24x24")
    try:
        chis = W.gaussian_field((8, c.Lt, c.Lx, 2), 321)
        b = np.stack([ow.apply_D(c.U, c.m, x, dagger=True) for x in chis])
        A = c.H.levels[0].op
        lam = np.linalg.eigvalsh(A.dense())
        with mg.Multigrid(c.Ug, c.m, c.blocks, c.Nv, c.noise_g, max_rhs=8) as sb:
            xb, ib = sb.solve(dev(b), tol=1e-10, maxiter=20000, solver=mg.SOLVER_MGCG_MIXED)
            xb = host(xb)
        for k in range(8):
            xo, _, _ = okr.mgcg(c.H, b[k], 1e-12)
            res = np.linalg.norm(b[k] - A.apply(xb[k])) / np.linalg.norm(b[k])
            assert res <= 1e-10 and ib[k].true_residual <= 1e-10
            assert np.linalg.norm(xb[k] - xo) <= 2 * lam[-1] / lam[0] * 1e-10 * np.linalg.norm(xo)
    finally:
        c.solver.close()


@pytest.mark.parametrize("solver", ["mixed", "reliable"])
def test_batched_graph_matches_eager(mg, solver):
    c = Case(mg, "2lvl_24x16")
    code = mg.SOLVER_MGCG_MIXED if solver == "mixed" else mg.SOLVER_MGCG_RELIABLE
    try:
        chis = W.gaussian_field((3, c.Lt, c.Lx, 2), 7)
        b = dev(np.stack([ow.apply_D(c.U, c.m, x, dagger=True) for x in chis]))
        with mg.Multigrid(c.Ug, c.m, c.blocks, c.Nv, c.noise_g, max_rhs=3) as sb:
            xg, ig = sb.solve(b, tol=1e-10, maxiter=20000, solver=code)
            xg = host(xg)
            mg.mg_profile_enable(sb.h, True)
            xe, ie = sb.solve(b, tol=1e-10, maxiter=20000, solver=code)
            xe = host(xe)
        assert [i.iterations for i in ig] == [i.iterations for i in ie]
        assert np.array_equal(xg, xe)
    finally:
        c.solver.close()


def test_iteration_limit_reports_noconv(case, mg):
    chi = W.gaussian_field((case.Lt, case.Lx, 2), 91)
    b = dev(ow.apply_D(case.U, case.m, chi, dagger=True))
    x = torch.empty_like(b)
    st, infos = mg.mg_solve(case.h, b, x, 1, 1e-14, 3, mg.SOLVER_MGCG_FP64)
    assert st == 4 and infos[0].iterations == 3


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_apply_A_streamed_large_ragged(mg, prec):
    """1000 x 998 lattice: the register-streaming stencil (not a multiple of its
    28-site strips or 32-row blocks)."""
    Lx, Lt, m = 1000, 998, -0.9
    U = W.links_from_angles(W.quenched_u1_angles(Lx, Lt, 3.0, 2, 5))
    psi = W.gaussian_field((Lt, Lx, 2), 7)
    want = ow.apply_A(U, m, psi)
    # uniform bound of the term magnitudes: |A_ij| summed over a row <= (4+|m|+2)^2
    mag = np.full(psi.shape, (4 + abs(m) + 2) ** 2 * np.max(np.abs(psi)))
    with mg.Multigrid(dev(U), m, [], []) as s:
        if prec == "f64":
            out = torch.empty_like(dev(psi))
            mg.mg_apply_A(s.h, dev(psi), out, 1, mg.PREC_F64)
            check(host(out), want, mag, TOL64, "A f64 streamed")
        else:
            inp = dev(psi.astype(np.complex64))
            out = torch.empty_like(inp)
            mg.mg_apply_A(s.h, inp, out, 1, mg.PREC_F32)
            check(host(out), want, mag, TOL32, "A f32 streamed")


def test_vcycle_streamed_stencil_768(mg):
    """A V-cycle whose fine level uses the streaming stencil with the fused
    smoother / residual epilogues (768 x 768, 4 levels)."""
    Lx = Lt = 768
    blocks, Nv, m = [(4, 4), (4, 4), (2, 2)], [4, 4, 4], -0.8
    U = W.links_from_angles(W.quenched_u1_angles(Lx, Lt, 6.0, 4, 9))
    noise = W.setup_noise(Lx, Lt, blocks, Nv, 10)
    H = omg.setup(U, m, blocks, Nv, noise, sweeps=2, power_iters=5)
    r = W.gaussian_field((Lt, Lx, 2), 11)
    want = omg.vcycle(H, r)
    with mg.Multigrid(dev(U), m, blocks, Nv, dev(noise), setup_sweeps=2, power_iters=5) as s:
        out = torch.empty_like(dev(r))
        mg.mg_vcycle(s.h, dev(r), out, mg.PREC_F64)
        got = host(out)
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_set_mass_rebuilds_galerkin(mg):
    c = Case(mg, "2lvl_24x16")
    try:
        m2 = 0.3
        omg.set_mass(c.H, m2)
        c.solver.set_mass(m2)
        op = c.H.levels[1].op
        out = torch.empty(op.M.shape, dtype=torch.complex128, device=DEV)
        mg.mg_get_coarse_op(c.h, 2, out)
        rowmax = np.max(np.abs(op.M), axis=(2, 4), keepdims=True)
        check(host(out), op.M, rowmax, 1e-11, "A_c after set_mass")
        c0, c1, _, _ = mg.mg_get_smoother(c.h, 1)
        assert c0 == pytest.approx(c.H.levels[0].c0, rel=1e-10)
    finally:
        c.solver.close()


def test_argument_errors(mg):
    U = W.links_from_angles(W.quenched_u1_angles(16, 16, 6.0, 5, 1))
    noise = dev(W.setup_noise(16, 16, [(4, 4)], [4], 1))
    with pytest.raises(mg.MgError) as e:           # 16 not divisible by 3
        mg.Multigrid(dev(U), 0.1, [(3, 3)], [4], noise)
    assert e.value.status == 1
    with pytest.raises(mg.MgError) as e:           # Nv above block-chirality dimension
        mg.Multigrid(dev(U), 0.1, [(2, 2)], [5], noise)
    assert e.value.status == 1
    bad = U.copy()
    bad[0, 3, 4] *= 1.01
    with pytest.raises(mg.MgError) as e:           # non-unit link
        mg.Multigrid(dev(bad), 0.1, [(4, 4)], [4], noise)
    assert e.value.status == 1
    with mg.Multigrid(dev(U), 0.1, [(4, 4)], [4], noise) as s:
        b = torch.full((16, 16, 2), float("nan"), dtype=torch.complex128, device=DEV)
        with pytest.raises(mg.MgError) as e:
            s.solve(b, solver=mg.SOLVER_MGCG_FP64)
        assert e.value.status == 5


def test_quadratic_remass_equals_galerkin_products(mg):
    """With remass_quadratic (default) every coarse operator after mg_set_mass
    is G0 + m G1 + m^2 I; it matches the Galerkin products of the same vectors
    at that mass (remass_quadratic = 0) to rounding, and the oracle's."""
    Lx, Lt, beta, sweeps, seed, m, blocks, Nv = CASES[list(CASES)[-1]]
    U = W.links_from_angles(W.quenched_u1_angles(Lx, Lt, beta, sweeps, seed))
    noise = W.setup_noise(Lx, Lt, blocks, Nv, seed + 100)
    H = omg.setup(U, m, blocks, Nv, noise)
    with mg.Multigrid(dev(U), m, blocks, Nv, dev(noise)) as q, \
            mg.Multigrid(dev(U), m, blocks, Nv, dev(noise), remass_quadratic=0) as g:
        assert mg.mg_device_bytes(q.h) > mg.mg_device_bytes(g.h)
        for m2 in (m + 0.3, -0.05, m):
            q.set_mass(m2)
            g.set_mass(m2)
            omg.set_mass(H, m2)
            for l in range(1, H.L):
                op = H.levels[l].op
                oq, og = (torch.empty(op.M.shape, dtype=torch.complex128, device=DEV) for _ in range(2))
                mg.mg_get_coarse_op(q.h, l + 1, oq)
                mg.mg_get_coarse_op(g.h, l + 1, og)
                a, b = host(oq), host(og)
                scale = np.max(np.abs(op.M))
                assert np.max(np.abs(a - b)) <= 1e-13 * scale, f"level {l + 1} at m = {m2}"
                rowmax = np.max(np.abs(op.M), axis=(2, 4), keepdims=True)
                check(a, op.M, rowmax, 1e-11, f"A_c level {l + 1} at m = {m2}")
