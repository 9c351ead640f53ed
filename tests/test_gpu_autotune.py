"""Autotuner of the fused fine A (mg_params.autotune): the launch shapes it
picks give the same bits as the default shape, for FP64 and FP32 and for 1
and several right-hand sides (a lattice first applied with tuning off, then
tuned), the chosen shape is never slower than the default in the tuner's own
timing, and the streaming kernel's lattices are tuned too."""
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


def _tuned(mg, Lx, Lt):
    return [t for t in mg.stencil_tunings() if t["lattice"] == [Lx, Lt]]


@pytest.mark.parametrize("Lx,Lt,nrhs", [(96, 64, 4), (1008, 896, 1)], ids=["96x64_4rhs", "1008x896_stream"])
def test_tuned_shapes_give_the_default_bits(mg, Lx, Lt, nrhs):
    U = torch.from_numpy(W.links_from_angles(W.quenched_u1_angles(Lx, Lt, 3.0, 2, 5))).to(DEV)
    x64 = torch.from_numpy(W.gaussian_field((nrhs, Lt, Lx, 2), 8)).to(DEV)
    x32 = x64.to(torch.complex64)
    assert not _tuned(mg, Lx, Lt)
    outs = {}
    for tune in (0, 1):
        p = mg.make_params(Lx, Lt, [], [], max_rhs=nrhs, autotune=tune)
        h = mg.mg_setup(U, -0.3, p)
        try:
            for prec, x in ((mg.PREC_F64, x64), (mg.PREC_F32, x32)):
                for n in sorted({1, nrhs}):
                    y = torch.empty_like(x[:n])
                    mg.mg_apply_A(h, x[:n].contiguous(), y, n, prec)
                    outs[(tune, prec, n)] = y
            torch.cuda.synchronize()
        finally:
            mg.mg_destroy(h)
        if tune == 0:
            assert not _tuned(mg, Lx, Lt)          # tuning off: nothing timed
    for key, y in outs.items():
        if key[0] == 1:
            assert torch.equal(y, outs[(0,) + key[1:]]), f"bits differ for {key}"
    rec = _tuned(mg, Lx, Lt)
    assert {(t["precision"], t["nrhs"]) for t in rec} == {(p, n) for p in ("f64", "f32") for n in {1, nrhs}}
    for t in rec:
        assert 1 <= t["admitted"] <= t["tried"] and t["us_chosen"] <= t["us_default"]
    if Lx == 1008:
        assert all(t["tried"] >= 2 for t in rec)   # the streaming kernel and the tiles compete
