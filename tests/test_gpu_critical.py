"""Critical mass on the GPU (mg_critical_mass) against the oracle's
spectral-flow finder: 32 x 32, beta = 3 (the oracle runs here) and the
64 x 64, beta = 3 serving configuration (the oracle's stored value), to 1e-11;
and the argument checks."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import critical

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0710_3612_gb300 import mg as m
    return m


def _cases():
    U32 = W.quenched_u1(32, 32, 3.0, 100, 1)
    yield "L32_b3_s1", U32, critical.critical_mass_by_flow(U32), [(4, 4)], [4]
    crit = json.load(open(os.path.join(ROOT, "workloads", "critical_masses_serving.json")))["L64_b3_s1"]
    th = W.quenched_u1_angles(64, 64, 3.0, crit["sweeps"], crit["seed"])
    assert abs(W.mean_plaquette(th) - crit["plaquette"]) <= 1e-12
    yield "L64_b3_s1", W.links_from_angles(th), crit["m_crit"], [(4, 4), (2, 2)], [8, 8]


@pytest.mark.parametrize("case", list(range(2)), ids=["32x32_b3", "64x64_b3"])
def test_critical_mass_equals_oracle(mg, case):
    key, U, m_ref, blocks, Nv = list(_cases())[case]
    L = U.shape[1]
    noise = torch.from_numpy(W.setup_noise(L, L, blocks, Nv, 7)).to(DEV)
    with mg.Multigrid(torch.from_numpy(U).to(DEV), -1.9, blocks, Nv, noise) as s:
        v0 = torch.from_numpy(W.gaussian_field((L, L, 2), 3)).to(DEV)
        m, slope, evals = mg.critical_mass(s.h, v0)
        assert abs(m - m_ref) <= 1e-11, f"{key}: {m!r} against {m_ref!r}"
        assert 0 < abs(slope) <= 1 and 1 <= evals <= 50


def test_critical_mass_argument_checks(mg):
    L = 16
    U = torch.from_numpy(W.quenched_u1(L, L, 3.0, 20, 1)).to(DEV)
    noise = torch.from_numpy(W.setup_noise(L, L, [(4, 4)], [2], 7)).to(DEV)
    with mg.Multigrid(U, -1.0, [(4, 4)], [2], noise) as s:
        v0 = torch.from_numpy(W.gaussian_field((L, L, 2), 3)).to(DEV)
        for kw in (dict(m_hi=-2.4, m_lo=-1.9), dict(safety=1.5), dict(newton_floor=0.1)):
            with pytest.raises(mg.MgError) as ei:
                mg.critical_mass(s.h, v0, **kw)
            assert ei.value.status == 1
        # no crossing between m_hi and m_lo far above the critical region
        with pytest.raises(mg.MgError) as ei:
            mg.critical_mass(s.h, v0, m_hi=1.0, m_lo=0.5, max_evals=20)
        assert ei.value.status == 4                          # MG_ERR_NOCONV
