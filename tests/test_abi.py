"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/*.h declare; the Python binding declares the same set.
No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    inc = os.path.join(ROOT, "include")
    src = "\n".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                    if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mg_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    __graft_entry__.build()
    return __graft_entry__.LIB


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mg_setup", "mg_solve", "mg_apply_D", "mg_apply_coarse", "mg_destroy",
                     "mg_set_mass", "mg_restrict", "mg_prolong", "mg_vcycle", "mg_block_map"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_the_header(lib_path):
    from paper_0710_3612_gb300 import mg
    assert set(declared_functions()) == set(mg._SIGS)
    assert mg.lib() is not None


def test_param_struct_layout_matches(lib_path):
    """mg_params_default and mg_setup_noise_len run on the host only."""
    from paper_0710_3612_gb300 import mg
    import workloads as W
    p = mg.make_params(32, 16, [(4, 4), (2, 2)], [3, 5])
    assert (p.Lx, p.Lt, p.nlevels, p.setup_sweeps, p.power_iters) == (32, 16, 3, 8, 30)
    assert p.omega_mr == 0.8
    assert mg.mg_setup_noise_len(p) == W.setup_noise_len(32, 16, [(4, 4), (2, 2)], [3, 5])
    bad = mg.make_params(30, 16, [(4, 4)], [3])
    assert mg.mg_setup_noise_len(bad) == 0
    # with adaptive passes (1-based levels in the library, 0-based in workloads)
    r = mg.make_params(32, 16, [(4, 4), (2, 2)], [3, 5], refine_levels=[1, 2, 2])
    assert r.refine_cycles == 30 and list(r.refine_levels[:4]) == [1, 2, 2, 0]
    assert p.autotune == 1 and p.remass_quadratic == 1
    assert mg.lib().mg_stencil_tunings(None, 0) == 0        # nothing tuned without a device
    assert mg.mg_setup_noise_len(r) == W.setup_noise_len(32, 16, [(4, 4), (2, 2)], [3, 5], [0, 1, 1])


def test_setup_bytes_is_host_only(lib_path):
    """mg_setup_bytes sizes a hierarchy without touching a device."""
    from paper_0710_3612_gb300 import mg
    p = mg.make_params(128, 128, [(4, 4), (2, 2)], [8, 8])
    p.setup_noise = 1                    # never dereferenced by the size-only pass
    res, peak = mg.mg_setup_bytes(p)
    assert 0 < res < peak
    p8 = mg.make_params(128, 128, [(4, 4), (2, 2)], [8, 8], max_rhs=8)
    p8.setup_noise = 1
    assert mg.mg_setup_bytes(p8)[0] > res
    # adaptive passes: resident = the refined hierarchy's, the peak holds two
    pr = mg.make_params(128, 128, [(4, 4), (2, 2)], [8, 8], refine_levels=[1, 2])
    pr.setup_noise = 1
    ref = mg.make_params(128, 128, [(4, 4), (2, 2)], [9, 9])
    ref.setup_noise = 1
    res_r, peak_r = mg.mg_setup_bytes(pr)
    assert res_r == mg.mg_setup_bytes(ref)[0] and peak_r > res_r + res
    for bad in ([2, 1], [3], [0, 1]):
        q = mg.make_params(128, 128, [(4, 4), (2, 2)], [8, 8], refine_levels=bad)
        q.setup_noise = 1
        if bad == [0, 1]:                  # a leading 0 ends the plan: no passes
            assert mg.mg_setup_bytes(q)[0] == res
            continue
        with pytest.raises(mg.MgError):
            mg.mg_setup_bytes(q)
    # the quadratic re-mass keeps two more FP64 copies of each coarse operator
    p0 = mg.make_params(128, 128, [(4, 4), (2, 2)], [8, 8], remass_quadratic=0)
    p0.setup_noise = 1
    coarse = (32 * 32 * 9 * 16 * 16 + 16 * 16 * 9 * 16 * 16) * 16
    assert res - mg.mg_setup_bytes(p0)[0] == 2 * coarse
    q = mg.make_params(128, 128, [(4, 4), (2, 2)], [16, 8], refine_levels=[1])
    q.setup_noise = 1
    with pytest.raises(mg.MgError):      # 4x4 blocks of 2 components hold 16 vectors at most
        mg.mg_setup_bytes(q)


def test_new_entry_points_reject_arguments_on_the_host(lib_path):
    """mg_refine, mg_critical_mass, mg_gauge_metropolis and mg_gauge_links
    validate their arguments before any device work (no GPU needed)."""
    import ctypes
    from paper_0710_3612_gb300 import mg
    L = mg.lib()
    out, rho = ctypes.c_void_p(), ctypes.c_double()
    assert L.mg_refine(None, 1, None, 1, None, None, ctypes.byref(out), ctypes.byref(rho), None) == 1
    assert L.mg_refine(None, 1, None, 1, None, None, None, None, None) == 1
    m = ctypes.c_double()
    assert L.mg_critical_mass(None, -1.9, -2.4, None, 0.9, 1e-2, 1e-3, 10, ctypes.byref(m), None, None) == 1
    acc = ctypes.c_longlong()
    assert L.mg_gauge_metropolis(None, 8, 8, 1.0, 1.0, 1, 0, 1, None, ctypes.byref(acc)) == 1
    assert L.mg_gauge_links(None, None, 8, 8, None) == 1
    rr = (ctypes.c_double * 4)()
    n = ctypes.c_int()
    assert L.mg_get_refine_rho(None, rr, 4, ctypes.byref(n)) == 1


def test_solver_parameters_on_the_host(lib_path):
    """reliable_delta and coarsest_reuse: their defaults, their checks in the
    size-only pass (no GPU needed), and the sizes they leave unchanged."""
    from paper_0710_3612_gb300 import mg
    p = mg.make_params(64, 64, [(4, 4), (2, 2)], [8, 8])
    assert p.reliable_delta == 0.1 and p.coarsest_reuse == 0
    p.setup_noise = 1
    res = mg.mg_setup_bytes(p)[0]
    ok = mg.make_params(64, 64, [(4, 4), (2, 2)], [8, 8], reliable_delta=0.5, coarsest_reuse=12)
    ok.setup_noise = 1
    assert mg.mg_setup_bytes(ok)[0] == res
    for kw in (dict(reliable_delta=0.0), dict(reliable_delta=1.0), dict(reliable_delta=float("nan")),
               dict(coarsest_reuse=-1)):
        q = mg.make_params(64, 64, [(4, 4), (2, 2)], [8, 8], **kw)
        q.setup_noise = 1
        with pytest.raises(mg.MgError) as e:
            mg.mg_setup_bytes(q)
        assert e.value.status == 1 and next(iter(kw)) in str(e.value)
    assert mg.SOLVER_MGCG_RELIABLE == 3
