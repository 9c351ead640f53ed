"""mg_apply_A_dot_noalloc: the allocation-free entry point for callers that
cannot call cudaMalloc (code recording into a CUDA graph under stream capture,
or running under a fixed device-memory budget).  Its output must match
mg_apply_A, and its <x, A x> the inner product of the same vectors, on two
calls in a row (the library-held scratch keeps the last call's contents).

Collected last on purpose: it must pass alone in a fresh process and after
every other test.
"""
import numpy as np
import pytest

import workloads as W

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


@pytest.mark.parametrize("L", [(24, 16), (128, 128)])
def test_noalloc_matches_apply_A(mg, L):
    Lx, Lt = L
    U = torch.from_numpy(W.quenched_u1(Lx, Lt, 6.0, 20, 3)).cuda()
    with mg.Multigrid(U, -0.3, [], []) as s:          # fine operator only
        for call in range(2):
            x = torch.from_numpy(W.gaussian_field((Lt, Lx, 2), 10 + call)).cuda()
            ref = torch.empty_like(x)
            mg.mg_apply_A(s.h, x, ref, 1, mg.PREC_F64)
            out = torch.full_like(x, float("nan"))
            xax = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
            mg.mg_apply_A_dot_noalloc(s.h, x, out, xax)
            torch.cuda.synchronize()
            want = ref.cpu().numpy()
            got = out.cpu().numpy()
            assert np.max(np.abs(got - want)) <= TOL64 * np.max(np.abs(want))
            d = np.vdot(x.cpu().numpy(), want)
            v = xax.cpu().numpy()
            assert abs(v[0] - d.real) <= TOL64 * abs(d) and abs(v[1] - d.imag) <= TOL64 * abs(d)


def test_noalloc_rejects_oversized_lattice(mg):
    Lx = Lt = 512                                        # needs 1024 thread blocks
    U = torch.ones((2, Lt, Lx), dtype=torch.complex128, device="cuda")
    with mg.Multigrid(U, 0.1, [], []) as s:
        x = torch.zeros((Lt, Lx, 2), dtype=torch.complex128, device="cuda")
        out = torch.empty_like(x)
        xax = torch.empty(2, dtype=torch.float64, device="cuda")
        with pytest.raises(mg.MgError) as e:
            mg.mg_apply_A_dot_noalloc(s.h, x, out, xax)
        assert e.value.status == 1 and "608" in str(e.value)
