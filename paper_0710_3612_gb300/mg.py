"""Thin Python binding of the C ABI in include/mg.h (argument marshalling only).

Every function takes torch tensors that already live on the GPU, passes their
device pointers to libmg.so and returns status-checked results.  No arithmetic
of the method happens here; if libmg.so is missing the import of any entry
point raises (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmg.so")

MG_MAX_LEVELS = 5
MG_MAX_REFINE = 16
PREC_F64, PREC_F32, PREC_BF16 = 0, 1, 2
SOLVER_MGCG_FP64, SOLVER_MGCG_MIXED, SOLVER_CG_FP64, SOLVER_MGCG_RELIABLE = 0, 1, 2, 3
STATUS = {0: "MG_OK", 1: "MG_ERR_ARG", 2: "MG_ERR_NOMEM", 3: "MG_ERR_CUDA", 4: "MG_ERR_NOCONV",
          5: "MG_ERR_BREAKDOWN", 6: "MG_ERR_TIMEOUT"}


class MgError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class MgParams(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Lt", ctypes.c_int), ("nlevels", ctypes.c_int),
                ("block", (ctypes.c_int * 2) * (MG_MAX_LEVELS - 1)),
                ("Nv", ctypes.c_int * (MG_MAX_LEVELS - 1)),
                ("setup_sweeps", ctypes.c_int), ("power_iters", ctypes.c_int),
                ("omega_mr", ctypes.c_double), ("setup_noise", ctypes.c_void_p),
                ("coarsest_tol", ctypes.c_double), ("coarsest_refine_max", ctypes.c_int),
                ("inner_coarsest_refine", ctypes.c_int), ("vcycle_coarse_bf16", ctypes.c_int),
                ("max_rhs", ctypes.c_int), ("profile", ctypes.c_int),
                ("coarsest_dense_max", ctypes.c_int), ("coarsest_gj_tcgen05", ctypes.c_int),
                ("refine_levels", ctypes.c_int * MG_MAX_REFINE), ("refine_cycles", ctypes.c_int),
                ("autotune", ctypes.c_int), ("remass_quadratic", ctypes.c_int),
                ("smooth_omega", ctypes.c_double), ("reliable_delta", ctypes.c_double),
                ("coarsest_reuse", ctypes.c_int)]


class MgStencilTuning(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("Lx", ctypes.c_int), ("Lt", ctypes.c_int),
                ("nrhs", ctypes.c_int), ("tx", ctypes.c_int), ("ty", ctypes.c_int),
                ("rows_per_thread", ctypes.c_int), ("tried", ctypes.c_int),
                ("admitted", ctypes.c_int), ("us_chosen", ctypes.c_double),
                ("us_default", ctypes.c_double)]


class MgSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("fine_applies", ctypes.c_longlong),
                ("vcycles", ctypes.c_longlong), ("milliseconds", ctypes.c_double)]


class MgServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("batches", ctypes.c_longlong),
                ("batched_rhs", ctypes.c_longlong), ("builds", ctypes.c_longlong),
                ("clones", ctypes.c_longlong), ("evictions", ctypes.c_longlong), ("remasses", ctypes.c_longlong),
                ("resident_bytes", ctypes.c_longlong), ("peak_resident_bytes", ctypes.c_longlong),
                ("budget_bytes", ctypes.c_longlong), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double)]


_lib = None
_vp, _i, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_ll = ctypes.c_longlong
_SIGS = {
    "mg_params_default": (_i, [ctypes.POINTER(MgParams), _i, _i]),
    "mg_setup_noise_len": (ctypes.c_size_t, [ctypes.POINTER(MgParams)]),
    "mg_setup": (_i, [_vp, _d, ctypes.POINTER(MgParams), _vp, ctypes.POINTER(_vp)]),
    "mg_set_mass": (_i, [_vp, _d]),
    "mg_solve": (_i, [_vp, _vp, _vp, _i, _d, _i, _i, ctypes.POINTER(MgSolveInfo)]),
    "mg_apply_D": (_i, [_vp, _vp, _vp, _i, _i, _i]),
    "mg_apply_A": (_i, [_vp, _vp, _vp, _i, _i]),
    "mg_apply_coarse": (_i, [_vp, _i, _vp, _vp, _i, _i]),
    "mg_restrict": (_i, [_vp, _i, _vp, _vp, _i, _i]),
    "mg_prolong": (_i, [_vp, _i, _vp, _vp, _i, _i]),
    "mg_vcycle": (_i, [_vp, _vp, _vp, _i]),
    "mg_coarsest_solve": (_i, [_vp, _vp, _vp]),
    "mg_get_level": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                          ctypes.POINTER(_i)]),
    "mg_get_null_vectors": (_i, [_vp, _i, _vp]),
    "mg_get_coarse_op": (_i, [_vp, _i, _vp]),
    "mg_get_smoother": (_i, [_vp, _i, ctypes.POINTER(_d)]),
    "mg_get_coarsest_info": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "mg_get_coarsest_reuse": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "mg_get_smoothing": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "mg_block_map": (_i, [_i, _i, _i, _i, _vp, _vp, _vp]),
    "mg_apply_A_dot_noalloc": (_i, [_vp, _vp, _vp, _vp]),
    "mg_set_coarse_tensor_kernel": (_i, [_i]),
    "mg_setup_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "mg_server_create": (_i, [_ll, _i, _i, ctypes.POINTER(_vp)]),
    "mg_server_add_config": (_i, [_vp, _vp, ctypes.POINTER(MgParams), _d, ctypes.POINTER(_i)]),
    "mg_server_submit": (_i, [_vp, _i, _d, _vp, _vp, _i, _d, _i, ctypes.POINTER(_ll)]),
    "mg_server_wait": (_i, [_vp, _ll, _vp, ctypes.POINTER(_d)]),
    "mg_server_get_stats": (_i, [_vp, ctypes.POINTER(MgServerStats)]),
    "mg_server_inject_build_failures": (_i, [_vp, _i]),
    "mg_server_destroy": (None, [_vp]),
    "mg_device_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "mg_clone": (_i, [_vp, _d, _vp, ctypes.POINTER(_vp)]),
    "mg_refine": (_i, [_vp, _i, _vp, _i, _vp, _vp, ctypes.POINTER(_vp), ctypes.POINTER(_d), _vp]),
    "mg_get_refine_rho": (_i, [_vp, ctypes.POINTER(_d), _i, ctypes.POINTER(_i)]),
    "mg_stencil_tunings": (_i, [_vp, _i]),
    "mg_gauge_metropolis": (_i, [_vp, _i, _i, _d, _d, _i, _ll, ctypes.c_ulonglong, _vp,
                                 ctypes.POINTER(_ll)]),
    "mg_gauge_links": (_i, [_vp, _vp, _i, _i, _vp]),
    "mg_critical_mass": (_i, [_vp, _d, _d, _vp, _d, _d, _d, _i, ctypes.POINTER(_d),
                              ctypes.POINTER(_d), ctypes.POINTER(_i)]),
    "mg_kernel_launches": (ctypes.c_ulonglong, []),
    "mg_profile_enable": (_i, [_vp, _i]),
    "mg_profile_read": (_i, [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_longlong)]),
    "mg_last_error": (ctypes.c_char_p, [_vp]),
    "mg_destroy": (None, [_vp]),
}


def lib():
    """Load libmg.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} missing "
                               "(run `python __graft_entry__.py`)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status, handle=None):
    if status != 0:
        msg = lib().mg_last_error(handle)
        raise MgError(status, msg.decode() if msg else "")


def _ptr(t, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_params(Lx, Lt, blocks, Nv, noise=None, **kw) -> MgParams:
    p = MgParams()
    _check(lib().mg_params_default(ctypes.byref(p), Lx, Lt))
    p.nlevels = len(blocks) + 1
    for l, ((bx, bt), nv) in enumerate(zip(blocks, Nv)):
        p.block[l][0], p.block[l][1] = bx, bt
        p.Nv[l] = nv
    for k, v in kw.items():
        if k == "refine_levels":            # 1-based levels of the adaptive passes
            for j, lv in enumerate(v):
                p.refine_levels[j] = lv
        else:
            setattr(p, k, v)
    if noise is not None:
        p.setup_noise = _ptr(noise).value
    return p


def mg_setup_noise_len(params: MgParams) -> int:
    return int(lib().mg_setup_noise_len(ctypes.byref(params)))


def mg_setup(gauge, mass, params: MgParams, stream=None):
    import torch
    h = ctypes.c_void_p()
    _check(lib().mg_setup(_ptr(gauge, torch.complex128), float(mass), ctypes.byref(params),
                          _stream_ptr(stream), ctypes.byref(h)))
    return h


def mg_setup_bytes(params: MgParams):
    res, peak = ctypes.c_longlong(), ctypes.c_longlong()
    _check(lib().mg_setup_bytes(ctypes.byref(params), ctypes.byref(res), ctypes.byref(peak)))
    return res.value, peak.value


def mg_device_bytes(h) -> int:
    v = ctypes.c_longlong()
    _check(lib().mg_device_bytes(h, ctypes.byref(v)), h)
    return v.value


def mg_clone(h, mass, stream=None):
    out = ctypes.c_void_p()
    _check(lib().mg_clone(h, float(mass), _stream_ptr(stream), ctypes.byref(out)), h)
    return out


def mg_refine(h, level, e0, ncycles, noise=None, stream=None, e_out=None):
    """One adaptive pass on `level` (1 = finest); returns (new handle, rho)."""
    import torch
    out, rho = ctypes.c_void_p(), ctypes.c_double()
    _check(lib().mg_refine(h, int(level), _ptr(e0, torch.complex128), int(ncycles),
                           None if noise is None else _ptr(noise, torch.complex128),
                           _stream_ptr(stream), ctypes.byref(out), ctypes.byref(rho),
                           None if e_out is None else _ptr(e_out, torch.complex128)), h)
    return out, rho.value


def critical_mass(h, v0, m_hi=-1.9, m_lo=-2.4, safety=0.9, newton_below=1e-2,
                  newton_floor=1e-3, max_evals=200):
    """m_crit by the spectral-flow scan on the GPU; returns (m_crit, slope, evals)."""
    import torch
    m, sl, ev = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(lib().mg_critical_mass(h, float(m_hi), float(m_lo), _ptr(v0, torch.complex128),
                                  float(safety), float(newton_below), float(newton_floor),
                                  int(max_evals), ctypes.byref(m), ctypes.byref(sl),
                                  ctypes.byref(ev)), h)
    return m.value, sl.value, ev.value


def gauge_metropolis(theta, beta, sweeps, seed, first_sweep=0, eps=1.0, stream=None):
    """Checkerboard Metropolis on device angles theta[2][Lt][Lx] (float64), in
    place; returns the number of accepted proposals."""
    import torch
    _, Lt, Lx = theta.shape
    acc = ctypes.c_longlong()
    _check(lib().mg_gauge_metropolis(_ptr(theta, torch.float64), Lx, Lt, float(beta), float(eps),
                                     int(sweeps), int(first_sweep), int(seed),
                                     _stream_ptr(stream), ctypes.byref(acc)))
    return acc.value


def gauge_links(theta, stream=None):
    """U = exp(i theta) as a device complex128 [2][Lt][Lx] tensor."""
    import torch
    _, Lt, Lx = theta.shape
    U = torch.empty(theta.shape, dtype=torch.complex128, device=theta.device)
    _check(lib().mg_gauge_links(_ptr(theta, torch.float64), _ptr(U, torch.complex128), Lx, Lt,
                                _stream_ptr(stream)))
    return U


def stencil_tunings():
    """Launch shapes of the fused fine A picked by the autotuner in this process."""
    n = lib().mg_stencil_tunings(None, 0)
    buf = (MgStencilTuning * max(1, n))()
    n = lib().mg_stencil_tunings(buf, n)
    out = []
    for t in buf[:n]:
        out.append({"precision": "f64" if t.precision == PREC_F64 else "f32",
                    "lattice": [t.Lx, t.Lt], "nrhs": t.nrhs,
                    "tile": "stream" if t.tx == 0 else f"{t.tx}x{t.ty}x{t.rows_per_thread}",
                    "tried": t.tried, "admitted": t.admitted,
                    "us_chosen": round(t.us_chosen, 3), "us_default": round(t.us_default, 3)})
    return out


def mg_get_refine_rho(h):
    """rho of each adaptive pass mg_setup made."""
    buf = (ctypes.c_double * 16)()
    n = ctypes.c_int()
    _check(lib().mg_get_refine_rho(h, buf, 16, ctypes.byref(n)), h)
    return list(buf[:n.value])


def mg_set_mass(h, mass):
    _check(lib().mg_set_mass(h, float(mass)), h)


def mg_solve(h, b, x, nrhs, tol, maxiter, solver):
    import torch
    infos = (MgSolveInfo * nrhs)()
    st = lib().mg_solve(h, _ptr(b, torch.complex128), _ptr(x, torch.complex128), nrhs,
                        float(tol), int(maxiter), int(solver), infos)
    return st, list(infos)


def _vec_dtype(precision):
    import torch
    return torch.complex128 if precision == PREC_F64 else torch.complex64


def mg_apply_D(h, inp, out, nrhs, dagger, precision):
    dt = _vec_dtype(precision)
    _check(lib().mg_apply_D(h, _ptr(inp, dt), _ptr(out, dt), nrhs, int(dagger), precision), h)


def mg_apply_A(h, inp, out, nrhs, precision):
    dt = _vec_dtype(precision)
    _check(lib().mg_apply_A(h, _ptr(inp, dt), _ptr(out, dt), nrhs, precision), h)


def mg_apply_coarse(h, level, inp, out, nrhs, precision):
    dt = _vec_dtype(precision)
    _check(lib().mg_apply_coarse(h, level, _ptr(inp, dt), _ptr(out, dt), nrhs, precision), h)


def mg_restrict(h, level, inp, out, nrhs, precision):
    dt = _vec_dtype(precision)
    _check(lib().mg_restrict(h, level, _ptr(inp, dt), _ptr(out, dt), nrhs, precision), h)


def mg_prolong(h, level, inp, out, nrhs, precision):
    dt = _vec_dtype(precision)
    _check(lib().mg_prolong(h, level, _ptr(inp, dt), _ptr(out, dt), nrhs, precision), h)


def mg_vcycle(h, inp, out, precision):
    dt = _vec_dtype(precision)
    _check(lib().mg_vcycle(h, _ptr(inp, dt), _ptr(out, dt), precision), h)


def mg_coarsest_solve(h, inp, out):
    import torch
    _check(lib().mg_coarsest_solve(h, _ptr(inp, torch.complex128), _ptr(out, torch.complex128)), h)


def mg_get_level(h, level):
    a, b, c, d = _i(), _i(), _i(), _i()
    _check(lib().mg_get_level(h, level, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                              ctypes.byref(d)), h)
    return a.value, b.value, c.value, d.value


def mg_get_null_vectors(h, level, out):
    import torch
    _check(lib().mg_get_null_vectors(h, level, _ptr(out, torch.complex128)), h)


def mg_get_coarse_op(h, level, out):
    import torch
    _check(lib().mg_get_coarse_op(h, level, _ptr(out, torch.complex128)), h)


def mg_get_smoother(h, level):
    buf = (ctypes.c_double * 4)()
    _check(lib().mg_get_smoother(h, level, buf), h)
    return tuple(buf)


def mg_get_smoothing(h):
    """(omega, cond) of the smoothed first coarsening (0, 0 when off)."""
    om, cond = ctypes.c_double(), ctypes.c_double()
    _check(lib().mg_get_smoothing(h, ctypes.byref(om), ctypes.byref(cond)), h)
    return om.value, cond.value


COARSE_TC_TCGEN05, COARSE_TC_MMA_SYNC = 0, 1


def mg_set_coarse_tensor_kernel(kind):
    """Process-wide choice of the multi-RHS BF16 coarse-apply kernel (tcgen05 or mma.sync)."""
    _check(lib().mg_set_coarse_tensor_kernel(int(kind)))


def mg_get_coarsest_info(h):
    """(dense, steps, test_residual) of the coarsest solve fixed at set-up."""
    dense, steps, res = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().mg_get_coarsest_info(h, ctypes.byref(dense), ctypes.byref(steps), ctypes.byref(res)), h)
    return bool(dense.value), steps.value, res.value


def mg_get_coarsest_reuse(h):
    """(FP32 V-cycle refinement steps, re-masses that kept the previous inverse)."""
    inner, reuses = ctypes.c_int(), ctypes.c_int()
    _check(lib().mg_get_coarsest_reuse(h, ctypes.byref(inner), ctypes.byref(reuses)), h)
    return inner.value, reuses.value


def mg_block_map(Lx, Lt, bx, bt, coarse, offset, stream=None):
    import torch
    _check(lib().mg_block_map(Lx, Lt, bx, bt, _ptr(coarse, torch.int32), _ptr(offset, torch.int32),
                              _stream_ptr(stream)))


KF_FINE_A, KF_COARSE, KF_TRANSFER, KF_COARSEST, KF_INVERSE, KF_GALERKIN, KF_FINE_A64, KF_DENSE, \
    KF_GJ_UPDATE, KF_COARSE64 = range(10)
KF_COUNT = 10


def mg_apply_A_dot_noalloc(h, inp, out, xAx):
    import torch
    _check(lib().mg_apply_A_dot_noalloc(h, _ptr(inp, torch.complex128), _ptr(out, torch.complex128),
                                        _ptr(xAx, torch.float64)), h)


def mg_kernel_launches() -> int:
    return int(lib().mg_kernel_launches())


def mg_profile_enable(h, on=True):
    _check(lib().mg_profile_enable(h, int(on)), h)


def mg_profile_read(h, family):
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    _check(lib().mg_profile_read(h, family, ctypes.byref(ms), ctypes.byref(n)), h)
    return ms.value, n.value


def mg_last_error(h=None) -> str:
    msg = lib().mg_last_error(h)
    return msg.decode() if msg else ""


def mg_destroy(h):
    if h:
        lib().mg_destroy(h)


class Multigrid:
    """Owns one mg_handle: setup at construction, solve/apply methods, destroy on close."""

    def __init__(self, gauge, mass, blocks, Nv, noise=None, stream=None, **params):
        _, Lt, Lx = gauge.shape
        self.Lx, self.Lt = Lx, Lt
        self.params = make_params(Lx, Lt, list(blocks), list(Nv), noise, **params)
        self._noise = noise
        self.h = mg_setup(gauge.contiguous(), mass, self.params, stream)

    def set_mass(self, mass):
        mg_set_mass(self.h, mass)

    def level(self, level):
        return mg_get_level(self.h, level)

    def refine(self, level, e0, ncycles, noise=None, e_out=None):
        """Replace the hierarchy by its adaptive refinement on `level` (mg_refine);
        returns rho, the error reduction per cycle measured before refining."""
        h, rho = mg_refine(self.h, level, e0, ncycles, noise, e_out=e_out)
        mg_destroy(self.h)
        self.h = h
        self.params.Nv[level - 1] += 1
        return rho

    def solve(self, b, tol=1e-10, maxiter=10000, solver=SOLVER_MGCG_MIXED, x=None):
        import torch
        nrhs = b.numel() // (self.Lx * self.Lt * 2)
        if x is None:
            x = torch.empty_like(b)
        st, infos = mg_solve(self.h, b, x, nrhs, tol, maxiter, solver)
        if st not in (0, 4):
            _check(st, self.h)
        return x, infos

    def close(self):
        if self.h:
            mg_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving engine (include/mg_server.h): configurations registered once,
    solve requests queued and batched by the library's worker threads."""

    def __init__(self, budget_bytes, max_rhs=16, workers=2):
        self.s = ctypes.c_void_p()
        _check(lib().mg_server_create(int(budget_bytes), int(max_rhs), int(workers),
                                      ctypes.byref(self.s)))
        self._keep = {}

    def add_config(self, gauge, params: MgParams, setup_mass, noise=None) -> int:
        """gauge (and noise, which sets params.setup_noise) are copied by the call."""
        import torch
        if noise is not None:
            params.setup_noise = _ptr(noise, torch.complex128).value
        cid = ctypes.c_int()
        _check(lib().mg_server_add_config(self.s, _ptr(gauge, torch.complex128),
                                          ctypes.byref(params), float(setup_mass),
                                          ctypes.byref(cid)))
        return cid.value

    def submit(self, config_id, mass, b, x, nrhs, tol=1e-10, solver=0) -> int:
        import torch
        rid = ctypes.c_longlong()
        _check(lib().mg_server_submit(self.s, int(config_id), float(mass), _ptr(b, torch.complex128),
                                      _ptr(x, torch.complex128), int(nrhs), float(tol), int(solver),
                                      ctypes.byref(rid)))
        self._keep[rid.value] = (b, x)
        return rid.value

    def wait(self, request_id, nrhs):
        infos = (MgSolveInfo * nrhs)()
        lat = ctypes.c_double()
        st = lib().mg_server_wait(self.s, int(request_id), infos, ctypes.byref(lat))
        self._keep.pop(request_id, None)
        return st, list(infos), lat.value

    def inject_build_failures(self, count):
        """The next `count` builds or clones fail on the host (test support)."""
        _check(lib().mg_server_inject_build_failures(self.s, int(count)))

    def stats(self) -> MgServerStats:
        out = MgServerStats()
        _check(lib().mg_server_get_stats(self.s, ctypes.byref(out)))
        return out

    def close(self):
        if self.s:
            lib().mg_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
