"""mg_apply_A_dot_noalloc: the allocation-free entry point.

Some callers of this library cannot call cudaMalloc: code that records its
work into a CUDA graph under stream capture, where the allocator may not be
entered, and code that runs inside a fixed device-memory budget owned by
another framework.  For them the library keeps the reduction scratch of the
fused A = D^dagger D with <x, A x> in an array of its own.

Checked here, through the C ABI, on two calls in a row (the library-held
scratch keeps the last call's contents):
* out against the oracle's A x per element (|gpu - oracle| <= 1e-12 (|oracle|
  + M), M the sum of the magnitudes of the terms) and against mg_apply_A;
* <x, A x> against the oracle's inner product of the same vectors;
* the size limit at its exact boundary: 608 thread blocks pass, one more row
  of blocks is rejected with MG_ERR_ARG.

Collected last on purpose: it must pass alone in a fresh process and after
every other test.
"""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as omg
from oracle import wilson as ow

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0710_3612_gb300 import mg as m
    return m


def abs_normal_op(U, m):
    """|D|^T |D| as a stencil: applied to |x| it bounds the terms of (A x)_i."""
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


def blocks_f64(Lx, Lt):
    """Thread blocks of the FP64 fused A with <x, A x>: 32 x 8 tiles once they
    fill two waves of 152 SMs, else 16 x 8 tiles."""
    big = -(-Lx // 32) * -(-Lt // 8)
    return big if big >= 2 * 152 else -(-Lx // 16) * -(-Lt // 8)


# (24, 16): small tiles; (384, 384): 576 blocks; (608, 256): exactly 608 blocks
@pytest.mark.parametrize("L", [(24, 16), (384, 384), (608, 256)])
def test_noalloc_matches_oracle_and_apply_A(mg, L):
    Lx, Lt = L
    assert blocks_f64(Lx, Lt) <= 608
    m = -0.3
    Uh = W.links_from_angles(W.quenched_u1_angles(Lx, Lt, 6.0, 4, 3))
    U = torch.from_numpy(Uh).cuda()
    mag_op = abs_normal_op(Uh, m)
    with mg.Multigrid(U, m, [], []) as s:          # fine operator only
        for call in range(2):
            xh = W.gaussian_field((Lt, Lx, 2), 10 + call)
            x = torch.from_numpy(xh).cuda()
            ref = torch.empty_like(x)
            mg.mg_apply_A(s.h, x, ref, 1, mg.PREC_F64)
            out = torch.full_like(x, float("nan"))
            xax = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
            mg.mg_apply_A_dot_noalloc(s.h, x, out, xax)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            want = ow.apply_A(Uh, m, xh)
            mag = mag_op.apply(np.abs(xh)).real
            worst = np.max(np.abs(got - want) / (TOL64 * (np.abs(want) + mag)))
            assert worst <= 1.0, f"call {call}: worst error / bound {worst:.3g}"
            # the same kernel as mg_apply_A's
            assert np.max(np.abs(got - ref.cpu().numpy())) <= TOL64 * np.max(np.abs(want))
            d = np.vdot(xh, want)
            dmag = np.vdot(np.abs(xh), mag).real
            v = xax.cpu().numpy()
            assert abs(v[0] - d.real) <= TOL64 * dmag and abs(v[1] - d.imag) <= TOL64 * dmag


@pytest.mark.parametrize("L", [(608, 264), (512, 512)])
def test_noalloc_rejects_oversized_lattice(mg, L):
    Lx, Lt = L                                     # 627 and 1024 thread blocks
    assert blocks_f64(Lx, Lt) > 608
    U = torch.ones((2, Lt, Lx), dtype=torch.complex128, device="cuda")
    with mg.Multigrid(U, 0.1, [], []) as s:
        x = torch.zeros((Lt, Lx, 2), dtype=torch.complex128, device="cuda")
        out = torch.empty_like(x)
        xax = torch.empty(2, dtype=torch.float64, device="cuda")
        with pytest.raises(mg.MgError) as e:
            mg.mg_apply_A_dot_noalloc(s.h, x, out, xax)
        assert e.value.status == 1 and "608" in str(e.value)
