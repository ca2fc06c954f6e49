"""Python binding of libselm_mg.so (include/selm_mg.h): argument marshalling only.

Every function below has the name of the C entry point it calls and takes
torch CUDA tensors where the C call takes device pointers.  Streams default to
torch's current stream.  All arithmetic runs in the CUDA library; if the
library cannot be loaded this module raises instead of falling back.
"""

import ctypes
import os

import torch

from . import _build

SELM_OK, SELM_EINVAL, SELM_ENOMEM, SELM_ECUDA, SELM_ENOCONV, SELM_ETIMEOUT, SELM_EBUSY = range(7)
SELM_FP64, SELM_FP32_REFINE64 = 0, 1
SELM_PROJ_NONE, SELM_PROJ_MAC = 0, 1
SELM_COARSE_CHOLESKY, SELM_COARSE_SMOOTH = 0, 1
SELM_SYS_VELOCITY, SELM_SYS_PRESSURE = 0, 1
SELM_OPT_COARSE_ENGINE = 1
SELM_OPT_ENGINE_CLUSTER = 2
SELM_OPT_ENGINE_LEVEL = 3
SELM_OPT_LEVEL_COOP = 4
SELM_OPT_GRAPHS = 5
SELM_OPT_SPECULATE = 6
SELM_OPT_PRESSURE_SPECTRAL = 8
SELM_BATCH_SOLVE, SELM_BATCH_SAMPLE = 0, 1

_STATUS = {0: "SELM_OK", 1: "SELM_EINVAL", 2: "SELM_ENOMEM", 3: "SELM_ECUDA", 4: "SELM_ENOCONV",
           5: "SELM_ETIMEOUT", 6: "SELM_EBUSY"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class SelmDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int), ("mu", ctypes.c_double), ("kT", ctypes.c_double),
        ("levels", ctypes.c_int), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
        ("precision", ctypes.c_int), ("projection", ctypes.c_int), ("coarse_mode", ctypes.c_int),
        ("tol", ctypes.c_double), ("max_cycles", ctypes.c_int), ("proj_tol", ctypes.c_double),
        ("max_particles", ctypes.c_int), ("seed", ctypes.c_uint64), ("instance", ctypes.c_uint64),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
    ]


class SelmRequest(ctypes.Structure):
    _fields_ = [("desc", SelmDesc), ("np", ctypes.c_int), ("X", ctypes.c_void_p), ("F", ctypes.c_void_p),
                ("dt", ctypes.c_double), ("nsteps", ctypes.c_int), ("ncycles_per_step", ctypes.c_int),
                ("user", ctypes.c_void_p)]


class SelmResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("user", ctypes.c_void_p), ("status", ctypes.c_int),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("vcycles", ctypes.c_int)]


class SelmCompDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int), ("K", ctypes.c_int), ("ncomp", ctypes.c_int),
        ("levels", ctypes.c_int), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("nu_patch", ctypes.c_int),
        ("precision", ctypes.c_int), ("coarse_mode", ctypes.c_int), ("mu", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("instance", ctypes.c_uint64),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
    ]


class SelmMacDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int), ("K", ctypes.c_int), ("levels", ctypes.c_int),
        ("mu", ctypes.c_double), ("kT", ctypes.c_double),
        ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("nu_patch", ctypes.c_int),
        ("precision", ctypes.c_int), ("projection", ctypes.c_int),
        ("tol", ctypes.c_double), ("max_cycles", ctypes.c_int), ("proj_tol", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("instance", ctypes.c_uint64),
    ]


class SelmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_U64 = ctypes.c_uint64
_LL = ctypes.c_longlong
_SIGS = {
    "selm_mg_footprint": (ctypes.c_size_t, [ctypes.POINTER(SelmDesc)]),
    "selm_mg_create": (_I, [ctypes.POINTER(SelmDesc), _P, ctypes.POINTER(_P)]),
    "selm_mg_destroy": (_I, [_P]),
    "selm_mg_last_error": (ctypes.c_char_p, [_P]),
    "selm_mg_solve": (_I, [_P, _I, _P, _P, _P, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "selm_mg_sample": (_I, [_P, _I, _P, _I, _P, _P, _P]),
    "selm_mg_step": (_I, [_P, _I, _P, _P, _D, _I, _I, _P]),
    "selm_mg_step_host": (_I, [_P, _I, _P, _P, _D, _I, _I, _P]),
    "selm_mg_levels": (_I, [_P, _I]),
    "selm_mg_ncomp": (_I, [_P, _I]),
    "selm_mg_layout": (_I, [_P, _I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_LL), ctypes.POINTER(_LL)]),
    "selm_mg_inner_bytes": (_I, [_P]),
    "selm_mg_chain": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_U64)]),
    "selm_mg_velocity": (_I, [_P, ctypes.POINTER(_P)]),
    "selm_mg_set_cycle": (_I, [_P, _U64]),
    "selm_mg_fail_waits": (_I, [_P, _I, _P]),
    "selm_mg_stats": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_LL)]),
    "selm_mg_set_option": (_I, [_P, _I, _I]),
    "selm_mg_pressure_spectral": (_I, [_P]),
    "selm_mg_engine_info": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_size_t)]),
    "selm_mg_smooth": (_I, [_P, _I, _I, _P, _P, _I, _U64, _I, _P]),
    "selm_mg_residual_restrict": (_I, [_P, _I, _I, _P, _P, _P, _P]),
    "selm_mg_prolong_correct": (_I, [_P, _I, _I, _P, _P, _P]),
    "selm_mg_coarsest": (_I, [_P, _I, _P, _P, _U64, _I, _P]),
    "selm_mg_vcycle": (_I, [_P, _I, _P, _P, _U64, _I, _P]),
    "selm_mg_vcycle_static": (_I, [ctypes.POINTER(SelmDesc), _P, _P, _U64, _I, _P]),
    "selm_mg_outer_residual": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "selm_mg_outer_update": (_I, [_P, _I, _P, _P, _P]),
    "selm_mg_fac_cycle": (_I, [_P, _I, _P, _P, _U64, _I, _P]),
    "selm_mg_fac_solve": (_I, [_P, _I, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "selm_mg_spread": (_I, [_P, _I, _P, _P, _P, _P]),
    "selm_mg_interp": (_I, [_P, _I, _P, _P, _P, _P]),
    "selm_mg_project": (_I, [_P, _P, ctypes.POINTER(_I), _P]),
    "selm_mg_em_update": (_I, [_P, _I, _P, _P, _P]),
    "selm_philox4x32_10": (_I, [_P, ctypes.c_uint32, ctypes.c_uint32, _P, _I, _P]),
    "selm_batch_create": (_I, [_I, ctypes.POINTER(SelmDesc), _P, ctypes.POINTER(_P)]),
    "selm_batch_destroy": (_I, [_P]),
    "selm_batch_system": (_P, [_P, _I]),
    "selm_batch_last_error": (ctypes.c_char_p, [_P]),
    "selm_batch_step": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I, _I,
                             ctypes.POINTER(_I), _P]),
    "selm_batch_autotune": (_I, [_P, ctypes.POINTER(_I), _P]),
    "selm_batch_cycle": (_I, [_P, _I, _P]),
    "selm_batch_set_persistent": (_I, [_P, _I]),
    "selm_batch_phase_times": (_I, [_P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D),
                                    ctypes.POINTER(_I), _P]),
    "selm_batch_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "selm_server_create": (_I, [ctypes.c_size_t, _I, ctypes.POINTER(_P)]),
    "selm_server_create_batched": (_I, [ctypes.c_size_t, _I, _I, ctypes.POINTER(_P)]),
    "selm_server_batch_stats": (_I, [_P, ctypes.POINTER(_LL), ctypes.POINTER(_LL)]),
    "selm_server_submit": (_I, [_P, ctypes.POINTER(SelmRequest), ctypes.POINTER(_U64)]),
    "selm_server_poll": (_I, [_P, ctypes.POINTER(SelmResult), _I]),
    "selm_server_drain": (_I, [_P]),
    "selm_server_stats": (_I, [_P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_I),
                               ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_I)]),
    "selm_server_clock": (_D, [_P]),
    "selm_server_destroy": (_I, [_P]),
    "selm_comp_footprint": (ctypes.c_size_t, [ctypes.POINTER(SelmCompDesc)]),
    "selm_comp_create": (_I, [ctypes.POINTER(SelmCompDesc), _P, ctypes.POINTER(_P)]),
    "selm_comp_destroy": (_I, [_P]),
    "selm_comp_last_error": (ctypes.c_char_p, [_P]),
    "selm_comp_size": (_LL, [_P]),
    "selm_comp_layout": (_I, [_P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_LL), ctypes.POINTER(_LL)]),
    "selm_comp_inner_bytes": (_I, [_P]),
    "selm_comp_residual": (_I, [_P, _P, _P, _P, ctypes.POINTER(_D), _P]),
    "selm_comp_patch_sweeps": (_I, [_P, _P, _P, _P, _I, _U64, _I, _P]),
    "selm_comp_fac_cycle": (_I, [_P, _P, _P, _U64, _I, _P]),
    "selm_comp_solve": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "selm_comp_sample": (_I, [_P, _I, _P, _P]),
    "selm_comp_chain": (_I, [_P, ctypes.POINTER(_U64)]),
    "selm_comp_set_cycle": (_I, [_P, _U64]),
    "selm_comp_stats": (_I, [_P, ctypes.POINTER(_LL)]),
    "selm_mac_create": (_I, [ctypes.POINTER(SelmMacDesc), _P, ctypes.POINTER(_P)]),
    "selm_mac_destroy": (_I, [_P]),
    "selm_mac_last_error": (ctypes.c_char_p, [_P]),
    "selm_mac_faces": (_LL, [_P]),
    "selm_mac_cells": (_LL, [_P]),
    "selm_mac_levels": (_I, [_P]),
    "selm_mac_colours": (_I, [_P, _I]),
    "selm_mac_inner_bytes": (_I, [_P]),
    "selm_mac_apply": (_I, [_P, _P, _P, _P]),
    "selm_mac_divergence": (_I, [_P, _P, _P, _P]),
    "selm_mac_gradient": (_I, [_P, _P, _P, _P]),
    "selm_mac_project": (_I, [_P, _P, _P, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "selm_mac_fac_cycle": (_I, [_P, _P, _P, _D, _U64, _P]),
    "selm_mac_solve": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "selm_mac_sample": (_I, [_P, _I, _P, _P]),
    "selm_mac_chain": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_U64)]),
    "selm_mac_set_chain": (_I, [_P, _U64, _P]),
    "selm_mac_interp": (_I, [_P, _I, _P, _P, _P, _P]),
    "selm_mac_spread": (_I, [_P, _I, _P, _P, _P, _P]),
    "selm_mac_mobility": (_I, [_P, _I, _P, _P, _P, ctypes.POINTER(_I), _P]),
    "selm_mac_thermal": (_I, [_P, _I, _P, _I, _P, _P]),
    "selm_mac_step": (_I, [_P, _I, _P, _P, _D, _I, _I, _P]),
    "selm_mac_total_cycles": (_LL, [_P]),
    "selm_mac_host_matrix": (_I, [ctypes.POINTER(SelmMacDesc), _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                  ctypes.POINTER(_LL), ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "selm_mac_host_colours": (_I, [ctypes.POINTER(SelmMacDesc), _I, ctypes.POINTER(_I), ctypes.POINTER(_P)]),
    "selm_mac_host_free": (None, [_P]),
    "selm_mg_stokes_solve": (_I, [_P, _P, _P, _D, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "selm_mg_stokes_mobility": (_I, [_P, _I, _P, _P, _P, _P]),
    "selm_mg_rfd_directions": (_I, [_P, _I, _U64, _P, _P]),
    "selm_mg_rfd_drift": (_I, [_P, _I, _P, _P, _D, _P, _P]),
    "selm_mg_stokes_step": (_I, [_P, _I, _P, _P, _D, _I, _I, _D, _P]),
    "selm_kernel_launches": (ctypes.c_longlong, []),
    "selm_profile_enable": (_I, [_I]),
    "selm_profile_reset": (_I, []),
    "selm_profile_read": (_I, [_I, ctypes.POINTER(_D), ctypes.POINTER(_LL)]),
}

KERNEL_CLASSES = ["fine_sweep", "coarse_sweep", "residual", "restrict", "prolong", "coarsest",
                  "outer_residual", "outer_update", "spread", "interp", "projection", "other", "batch_cycle"]


def library_path():
    return _build.LIB


def lib():
    """Load libselm_mg.so (built in-tree by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(h, status):
    if status != SELM_OK:
        msg = lib().selm_mg_last_error(h).decode() if h else ""
        raise SelmError(status, msg)


# -- torch caching allocator as the library's device allocator ----------------
def _alloc(nbytes, ctx):
    return torch.cuda.caching_allocator_alloc(int(nbytes))


def _free(ptr, ctx):
    torch.cuda.caching_allocator_delete(ptr)


_ALLOC_CB = ALLOC_FN(_alloc)
_FREE_CB = FREE_FN(_free)


def make_desc(dim, n, mu=1.0, kT=1.0, levels=0, nu_pre=2, nu_post=2, precision=SELM_FP64,
              projection=SELM_PROJ_NONE, coarse_mode=SELM_COARSE_CHOLESKY, tol=1e-10, max_cycles=100,
              proj_tol=1e-10, max_particles=4096, seed=0, instance=0, torch_allocator=True):
    d = SelmDesc()
    d.dim, d.n, d.mu, d.kT, d.levels = dim, n, mu, kT, levels
    d.nu_pre, d.nu_post, d.precision, d.projection, d.coarse_mode = nu_pre, nu_post, precision, projection, coarse_mode
    d.tol, d.max_cycles, d.proj_tol, d.max_particles = tol, max_cycles, proj_tol, max_particles
    d.seed, d.instance = seed, instance
    if torch_allocator:
        d.alloc, d.free = _ALLOC_CB, _FREE_CB
    return d


def selm_mg_footprint(desc):
    return lib().selm_mg_footprint(ctypes.byref(desc))


def selm_mg_create(desc, stream=None):
    h = _P()
    st = lib().selm_mg_create(ctypes.byref(desc), _stream(stream), ctypes.byref(h))
    if st != SELM_OK:
        raise SelmError(st, "selm_mg_create failed (see stderr)")
    return h.value


def selm_mg_destroy(h):
    _check(None, lib().selm_mg_destroy(h))


def selm_mg_solve(h, X, F, U, stream=None, want_stats=True):
    npart = X.shape[0]
    cyc, res = _I(0), _D(0.0)
    _check(h, lib().selm_mg_solve(h, npart, _ptr(X), _ptr(F), _ptr(U),
                                  ctypes.byref(cyc) if want_stats else None,
                                  ctypes.byref(res) if want_stats else None, _stream(stream)))
    return cyc.value, res.value


def selm_mg_sample(h, X, ncycles, g, xi_out=None, stream=None):
    _check(h, lib().selm_mg_sample(h, X.shape[0], _ptr(X), ncycles, _ptr(g), _ptr(xi_out), _stream(stream)))


def selm_mg_step(h, X, F, dt, nsteps, ncycles_per_step, stream=None):
    _check(h, lib().selm_mg_step(h, X.shape[0], _ptr(X), _ptr(F), dt, nsteps, ncycles_per_step, _stream(stream)))


def selm_mg_step_host(h, X_host, F_host, dt, nsteps, ncycles_per_step, stream=None):
    """X_host, F_host: CPU float64 tensors [np][dim] (pinned for async copies)."""
    assert not X_host.is_cuda and not F_host.is_cuda and X_host.is_contiguous() and F_host.is_contiguous()
    _check(h, lib().selm_mg_step_host(h, X_host.shape[0], X_host.data_ptr(), F_host.data_ptr(), dt, nsteps,
                                      ncycles_per_step, _stream(stream)))


def selm_kernel_launches():
    return lib().selm_kernel_launches()


def selm_profile_enable(on):
    _check(None, lib().selm_profile_enable(int(on)))


def selm_profile_reset():
    _check(None, lib().selm_profile_reset())


def selm_profile_read(kernel_class):
    ms, cnt = _D(0.0), _LL(0)
    _check(None, lib().selm_profile_read(kernel_class, ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def selm_mg_levels(h, system=SELM_SYS_VELOCITY):
    return lib().selm_mg_levels(h, system)


def selm_mg_ncomp(h, system=SELM_SYS_VELOCITY):
    return lib().selm_mg_ncomp(h, system)


def selm_mg_layout(h, system, level, comp):
    dims = (_I * 3)()
    off, size = _LL(0), _LL(0)
    _check(h, lib().selm_mg_layout(h, system, level, comp, dims, ctypes.byref(off), ctypes.byref(size)))
    return (dims[0], dims[1], dims[2]), off.value, size.value


def selm_mg_inner_bytes(h):
    return lib().selm_mg_inner_bytes(h)


def selm_mg_chain(h):
    p, c = _P(), _U64(0)
    _check(h, lib().selm_mg_chain(h, ctypes.byref(p), ctypes.byref(c)))
    return p.value, c.value


def selm_mg_velocity(h):
    """Device address of the handle's velocity solve iterate u (FP64, velocity layout)."""
    p = _P()
    _check(h, lib().selm_mg_velocity(h, ctypes.byref(p)))
    return p.value


def selm_mg_set_cycle(h, cycle):
    _check(h, lib().selm_mg_set_cycle(h, cycle))


def selm_mg_fail_waits(h, system, stream=None):
    _check(h, lib().selm_mg_fail_waits(h, system, _stream(stream)))


def selm_mg_stats(h):
    a, b, c = _I(0), _I(0), _LL(0)
    _check(h, lib().selm_mg_stats(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def selm_mg_set_option(h, option, value):
    _check(h, lib().selm_mg_set_option(h, option, int(value)))


def selm_mg_pressure_spectral(h):
    return int(lib().selm_mg_pressure_spectral(h))


def selm_mg_engine_info(h, system=SELM_SYS_VELOCITY):
    l0, c, sm = _I(0), _I(0), ctypes.c_size_t(0)
    _check(h, lib().selm_mg_engine_info(h, system, ctypes.byref(l0), ctypes.byref(c), ctypes.byref(sm)))
    return l0.value, c.value, sm.value


def selm_mg_smooth(h, system, level, v, b, sweep, cycle, noise, stream=None):
    _check(h, lib().selm_mg_smooth(h, system, level, _ptr(v), _ptr(b), sweep, cycle, int(noise), _stream(stream)))


def selm_mg_residual_restrict(h, system, level, v, b, b_coarse, stream=None):
    _check(h, lib().selm_mg_residual_restrict(h, system, level, _ptr(v), _ptr(b), _ptr(b_coarse), _stream(stream)))


def selm_mg_prolong_correct(h, system, level, v, v_coarse, stream=None):
    _check(h, lib().selm_mg_prolong_correct(h, system, level, _ptr(v), _ptr(v_coarse), _stream(stream)))


def selm_mg_coarsest(h, system, v, b, cycle, noise, stream=None):
    _check(h, lib().selm_mg_coarsest(h, system, _ptr(v), _ptr(b), cycle, int(noise), _stream(stream)))


def selm_mg_vcycle(h, system, v, b, cycle, noise, stream=None):
    _check(h, lib().selm_mg_vcycle(h, system, _ptr(v), _ptr(b), cycle, int(noise), _stream(stream)))


def selm_mg_vcycle_static(desc, v, b, cycle, noise, stream=None):
    """One V-cycle with no device allocation (static scratch inside the library)."""
    _check(None, lib().selm_mg_vcycle_static(ctypes.byref(desc), _ptr(v), _ptr(b), cycle, int(noise),
                                             _stream(stream)))


def selm_mg_outer_residual(h, system, z, b64, r, norm2=None, stream=None):
    _check(h, lib().selm_mg_outer_residual(h, system, _ptr(z), _ptr(b64), _ptr(r), _ptr(norm2), _stream(stream)))


def selm_mg_outer_update(h, system, z, d, stream=None):
    _check(h, lib().selm_mg_outer_update(h, system, _ptr(z), _ptr(d), _stream(stream)))


def selm_mg_fac_cycle(h, system, z, b64, cycle, noise, stream=None):
    _check(h, lib().selm_mg_fac_cycle(h, system, _ptr(z), _ptr(b64), cycle, int(noise), _stream(stream)))


def selm_mg_fac_solve(h, system, z, b64, tol, max_cycles, stream=None):
    cyc, res = _I(0), _D(0.0)
    _check(h, lib().selm_mg_fac_solve(h, system, _ptr(z), _ptr(b64), tol, max_cycles, ctypes.byref(cyc),
                                      ctypes.byref(res), _stream(stream)))
    return cyc.value, res.value


def selm_mg_spread(h, X, F, b, stream=None):
    _check(h, lib().selm_mg_spread(h, X.shape[0], _ptr(X), _ptr(F), _ptr(b), _stream(stream)))


def selm_mg_interp(h, X, u, U, stream=None):
    _check(h, lib().selm_mg_interp(h, X.shape[0], _ptr(X), _ptr(u), _ptr(U), _stream(stream)))


def selm_mg_project(h, w, stream=None):
    c = _I(0)
    _check(h, lib().selm_mg_project(h, _ptr(w), ctypes.byref(c), _stream(stream)))
    return c.value


def selm_mg_em_update(h, X, V, stream=None):
    _check(h, lib().selm_mg_em_update(h, X.shape[0], _ptr(X), _ptr(V), _stream(stream)))


def selm_philox4x32_10(ctr, key0, key1, out, stream=None):
    n = ctr.numel() // 4
    _check(None, lib().selm_philox4x32_10(_ptr(ctr), key0, key1, _ptr(out), n, _stream(stream)))


def _check_batch(b, status):
    if status != SELM_OK:
        msg = lib().selm_batch_last_error(b).decode() if b else ""
        raise SelmError(status, msg)


def selm_batch_create(descs, stream=None):
    arr = (SelmDesc * len(descs))(*descs)
    b = _P()
    st = lib().selm_batch_create(len(descs), arr, _stream(stream), ctypes.byref(b))
    if st != SELM_OK:
        raise SelmError(st, "selm_batch_create failed (see stderr)")
    return b.value


def selm_batch_destroy(b):
    _check_batch(None, lib().selm_batch_destroy(b))


def selm_batch_system(b, i):
    return lib().selm_batch_system(b, i)


def selm_batch_step(b, X, F, dt, nsteps, ncycles_per_step, stream=None):
    """X, F: lists of CUDA float64 tensors [np_i][dim]; returns the solve cycles per system."""
    n = len(X)
    nps = (_I * n)(*[x.shape[0] for x in X])
    xs = (_P * n)(*[_ptr(x) for x in X])
    fs = (_P * n)(*[_ptr(f) for f in F])
    cyc = (_I * n)()
    _check_batch(b, lib().selm_batch_step(b, nps, xs, fs, dt, nsteps, ncycles_per_step, cyc, _stream(stream)))
    return list(cyc)


def selm_batch_autotune(b, stream=None):
    c = _I(0)
    _check_batch(b, lib().selm_batch_autotune(b, ctypes.byref(c), _stream(stream)))
    return c.value


def selm_batch_cycle(b, mode, stream=None):
    _check_batch(b, lib().selm_batch_cycle(b, mode, _stream(stream)))


def selm_batch_set_persistent(b, on):
    _check_batch(b, lib().selm_batch_set_persistent(b, int(on)))


BATCH_PHASE_NAMES = ["outer_residual", "colour_pass", "coarsest_L", "coarsest_LT", "residual", "restrict",
                     "prolong", "outer_update"]


def selm_batch_phase_times(b, mode, stream=None):
    """[(phase name, level, microseconds)] of one persistent batched FAC cycle."""
    n = _I(0)
    _check_batch(b, lib().selm_batch_phase_times(b, mode, 0, None, None, None, ctypes.byref(n), _stream(stream)))
    k = n.value
    t, lv, us = (_I * k)(), (_I * k)(), (_D * k)()
    _check_batch(b, lib().selm_batch_phase_times(b, mode, k, t, lv, us, ctypes.byref(n), _stream(stream)))
    return [(BATCH_PHASE_NAMES[t[p]], lv[p], us[p]) for p in range(k)]


def selm_batch_info(b):
    """{'persistent', 'kc', 'blocks_per_sm', 'cluster'} of a batch."""
    v = [_I(0) for _ in range(4)]
    _check_batch(b, lib().selm_batch_info(b, *[ctypes.byref(x) for x in v]))
    return dict(zip(("persistent", "kc", "blocks_per_sm", "cluster"), (x.value for x in v)))


def selm_server_create(budget_bytes, max_slots):
    s = _P()
    _check(None, lib().selm_server_create(int(budget_bytes), int(max_slots), ctypes.byref(s)))
    return s.value


def selm_server_create_batched(budget_bytes, max_slots, persistent=True):
    s = _P()
    _check(None, lib().selm_server_create_batched(int(budget_bytes), int(max_slots), int(bool(persistent)),
                                                  ctypes.byref(s)))
    return s.value


def selm_server_batch_stats(s):
    steps, rebuilds = _LL(0), _LL(0)
    _check(None, lib().selm_server_batch_stats(s, ctypes.byref(steps), ctypes.byref(rebuilds)))
    return {"steps": steps.value, "rebuilds": rebuilds.value}


def selm_server_submit(s, desc, X, F, dt, nsteps, ncycles_per_step, user=0):
    """X, F: C-contiguous float64 numpy arrays [np][dim] (host); X is overwritten on completion.
    The caller keeps X and F alive until the result is polled."""
    assert X.dtype.kind == "f" and X.itemsize == 8 and X.flags.c_contiguous and F.flags.c_contiguous
    r = SelmRequest()
    r.desc = desc
    r.np = X.shape[0]
    r.X = X.ctypes.data
    r.F = F.ctypes.data
    r.dt, r.nsteps, r.ncycles_per_step, r.user = dt, nsteps, ncycles_per_step, user
    rid = _U64(0)
    _check(None, lib().selm_server_submit(s, ctypes.byref(r), ctypes.byref(rid)))
    return rid.value


def selm_server_poll(s, max_results=256):
    buf = (SelmResult * max_results)()
    n = lib().selm_server_poll(s, buf, max_results)
    return [dict(id=r.id, user=r.user or 0, status=r.status, t_submit=r.t_submit, t_admit=r.t_admit,
                 t_done=r.t_done, vcycles=r.vcycles) for r in buf[:n]]


def selm_server_drain(s):
    _check(None, lib().selm_server_drain(s))


def selm_server_stats(s):
    pb, ps, bu, q = ctypes.c_size_t(0), _I(0), ctypes.c_size_t(0), _I(0)
    _check(None, lib().selm_server_stats(s, ctypes.byref(pb), ctypes.byref(ps), ctypes.byref(bu), ctypes.byref(q)))
    return dict(peak_bytes=pb.value, peak_slots=ps.value, bytes_in_use=bu.value, queued=q.value)


def selm_server_clock(s):
    return lib().selm_server_clock(s)


def selm_server_destroy(s):
    _check(None, lib().selm_server_destroy(s))


# -- composite grid (refined patch, Algorithms 1-2) ----------------------------
def _check_comp(c, status):
    if status != SELM_OK:
        msg = lib().selm_comp_last_error(c).decode() if c else ""
        raise SelmError(status, msg)


def make_comp_desc(dim, n, K, ncomp=1, mu=1.0, levels=0, nu_pre=2, nu_post=2, nu_patch=2, precision=SELM_FP64,
                   coarse_mode=SELM_COARSE_CHOLESKY, seed=0, instance=0, torch_allocator=True):
    d = SelmCompDesc()
    d.dim, d.n, d.K, d.ncomp, d.levels = dim, n, K, ncomp, levels
    d.nu_pre, d.nu_post, d.nu_patch, d.precision, d.coarse_mode = nu_pre, nu_post, nu_patch, precision, coarse_mode
    d.mu, d.seed, d.instance = mu, seed, instance
    if torch_allocator:
        d.alloc, d.free = _ALLOC_CB, _FREE_CB
    return d


def selm_comp_footprint(desc):
    return lib().selm_comp_footprint(ctypes.byref(desc))


def selm_comp_create(desc, stream=None):
    c = _P()
    st = lib().selm_comp_create(ctypes.byref(desc), _stream(stream), ctypes.byref(c))
    if st != SELM_OK:
        raise SelmError(st, "selm_comp_create failed (see stderr)")
    return c.value


def selm_comp_destroy(c):
    _check_comp(None, lib().selm_comp_destroy(c))


def selm_comp_size(c):
    return int(lib().selm_comp_size(c))


def selm_comp_layout(c, part, comp):
    dims = (_I * 3)()
    off, size = _LL(0), _LL(0)
    _check_comp(c, lib().selm_comp_layout(c, part, comp, dims, ctypes.byref(off), ctypes.byref(size)))
    return (dims[0], dims[1], dims[2]), off.value, size.value


def selm_comp_inner_bytes(c):
    return lib().selm_comp_inner_bytes(c)


def selm_comp_residual(c, z, b, r, want_norm=True, stream=None):
    n2 = _D(0.0)
    _check_comp(c, lib().selm_comp_residual(c, _ptr(z), _ptr(b), _ptr(r), ctypes.byref(n2) if want_norm else None,
                                            _stream(stream)))
    return n2.value


def selm_comp_patch_sweeps(c, q_patch, q_base, r_patch, count, cycle, noise, stream=None):
    _check_comp(c, lib().selm_comp_patch_sweeps(c, _ptr(q_patch), _ptr(q_base), _ptr(r_patch), count, cycle,
                                                int(noise), _stream(stream)))


def selm_comp_fac_cycle(c, z, b, cycle, noise, stream=None):
    _check_comp(c, lib().selm_comp_fac_cycle(c, _ptr(z), _ptr(b), cycle, int(noise), _stream(stream)))


def selm_comp_solve(c, z, b, tol, max_cycles, stream=None):
    cyc, rel = _I(0), _D(0.0)
    _check_comp(c, lib().selm_comp_solve(c, _ptr(z), _ptr(b), tol, max_cycles, ctypes.byref(cyc), ctypes.byref(rel),
                                         _stream(stream)))
    return cyc.value, rel.value


def selm_comp_sample(c, ncycles, xi_out=None, stream=None):
    _check_comp(c, lib().selm_comp_sample(c, ncycles, _ptr(xi_out), _stream(stream)))


def selm_comp_chain(c):
    cy = _U64(0)
    _check_comp(c, lib().selm_comp_chain(c, ctypes.byref(cy)))
    return cy.value


def selm_comp_set_cycle(c, cycle):
    _check_comp(c, lib().selm_comp_set_cycle(c, cycle))


def selm_comp_stats(c):
    t = _LL(0)
    _check_comp(c, lib().selm_comp_stats(c, ctypes.byref(t)))
    return t.value


class SelmMG:
    """Owner of one handle; methods forward to the functions above."""

    def __init__(self, **kw):
        self.desc = make_desc(**kw)
        self.h = selm_mg_create(self.desc)

    def close(self):
        if self.h:
            torch.cuda.synchronize()
            selm_mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self, system=SELM_SYS_VELOCITY, level=0):
        n = selm_mg_ncomp(self.h, system)
        comps = [selm_mg_layout(self.h, system, level, c) for c in range(n)]
        return [(dims, off) for dims, off, _ in comps], comps[0][2]

    def inner_dtype(self):
        return torch.float32 if selm_mg_inner_bytes(self.h) == 4 else torch.float64


# -- staggered composite grid (selm_mac.h) --------------------------------------
SELM_MAC_MAT_A, SELM_MAC_MAT_D, SELM_MAC_MAT_G, SELM_MAC_MAT_S = 0, 1, 2, 3
SELM_MAC_MAT_P, SELM_MAC_MAT_E, SELM_MAC_MAT_OPS, SELM_MAC_MAT_PL = 4, 5, 6, 7


def _check_mac(h, status):
    if status != SELM_OK:
        msg = lib().selm_mac_last_error(h).decode() if h else ""
        raise SelmError(status, msg)


def make_mac_desc(dim, n, K, mu=1.0, kT=0.0, levels=0, nu_pre=2, nu_post=2, nu_patch=2, precision=SELM_FP64,
                  projection=SELM_PROJ_NONE, tol=0.0, max_cycles=0, proj_tol=0.0, seed=0, instance=0):
    d = SelmMacDesc()
    d.dim, d.n, d.K, d.levels, d.mu, d.kT = dim, n, K, levels, mu, kT
    d.nu_pre, d.nu_post, d.nu_patch, d.precision, d.projection = nu_pre, nu_post, nu_patch, precision, projection
    d.tol, d.max_cycles, d.proj_tol, d.seed, d.instance = tol, max_cycles, proj_tol, seed, instance
    return d


def selm_mac_create(desc, stream=None):
    h = _P()
    st = lib().selm_mac_create(ctypes.byref(desc), _stream(stream), ctypes.byref(h))
    if st != SELM_OK:
        raise SelmError(st, "selm_mac_create failed (see stderr)")
    return h.value


def selm_mac_destroy(h):
    _check_mac(None, lib().selm_mac_destroy(h))


def selm_mac_faces(h):
    return int(lib().selm_mac_faces(h))


def selm_mac_cells(h):
    return int(lib().selm_mac_cells(h))


def selm_mac_levels(h):
    return int(lib().selm_mac_levels(h))


def selm_mac_colours(h, level):
    return int(lib().selm_mac_colours(h, level))


def selm_mac_inner_bytes(h):
    return int(lib().selm_mac_inner_bytes(h))


def selm_mac_apply(h, u, Au, stream=None):
    _check_mac(h, lib().selm_mac_apply(h, _ptr(u), _ptr(Au), _stream(stream)))


def selm_mac_divergence(h, u, div, stream=None):
    _check_mac(h, lib().selm_mac_divergence(h, _ptr(u), _ptr(div), _stream(stream)))


def selm_mac_gradient(h, p, grad, stream=None):
    _check_mac(h, lib().selm_mac_gradient(h, _ptr(p), _ptr(grad), _stream(stream)))


def selm_mac_project(h, u, out, adjoint=False, stream=None):
    it, res = _I(0), _D(0.0)
    _check_mac(h, lib().selm_mac_project(h, _ptr(u), _ptr(out), int(adjoint), ctypes.byref(it), ctypes.byref(res),
                                         _stream(stream)))
    return it.value, res.value


def selm_mac_fac_cycle(h, z, b, sigma, cycle, stream=None):
    _check_mac(h, lib().selm_mac_fac_cycle(h, _ptr(z), _ptr(b), float(sigma), cycle, _stream(stream)))


def selm_mac_solve(h, z, b, tol=0.0, max_cycles=0, stream=None):
    cyc, rel = _I(0), _D(0.0)
    _check_mac(h, lib().selm_mac_solve(h, _ptr(z), _ptr(b), tol, max_cycles, ctypes.byref(cyc), ctypes.byref(rel),
                                       _stream(stream)))
    return cyc.value, rel.value


def selm_mac_sample(h, ncycles, xi_out=None, stream=None):
    _check_mac(h, lib().selm_mac_sample(h, ncycles, _ptr(xi_out), _stream(stream)))


def selm_mac_chain(h):
    p, cy = _P(), _U64(0)
    _check_mac(h, lib().selm_mac_chain(h, ctypes.byref(p), ctypes.byref(cy)))
    return p.value, cy.value


def selm_mac_set_chain(h, cycle, stream=None):
    _check_mac(h, lib().selm_mac_set_chain(h, cycle, _stream(stream)))


def selm_mac_interp(h, X, u, U, stream=None):
    _check_mac(h, lib().selm_mac_interp(h, X.shape[0], _ptr(X), _ptr(u), _ptr(U), _stream(stream)))


def selm_mac_spread(h, X, F, f, stream=None):
    _check_mac(h, lib().selm_mac_spread(h, X.shape[0], _ptr(X), _ptr(F), _ptr(f), _stream(stream)))


def selm_mac_mobility(h, X, F, U, stream=None):
    cyc = _I(0)
    _check_mac(h, lib().selm_mac_mobility(h, X.shape[0], _ptr(X), _ptr(F), _ptr(U), ctypes.byref(cyc),
                                          _stream(stream)))
    return cyc.value


def selm_mac_thermal(h, X, ncycles, g, stream=None):
    _check_mac(h, lib().selm_mac_thermal(h, X.shape[0], _ptr(X), ncycles, _ptr(g), _stream(stream)))


def selm_mac_step(h, X, F, dt, nsteps, ncycles, stream=None):
    _check_mac(h, lib().selm_mac_step(h, X.shape[0], _ptr(X), _ptr(F), dt, nsteps, ncycles, _stream(stream)))


def selm_mac_total_cycles(h):
    return int(lib().selm_mac_total_cycles(h))


def selm_mac_host_matrix(desc, which, level=0):
    """(nr, nc, indptr, indices, data) of one sparse matrix of the host plan."""
    import numpy as np
    nr, nc, nnz = _I(0), _I(0), _LL(0)
    ptr, col, val = _P(), _P(), _P()
    st = lib().selm_mac_host_matrix(ctypes.byref(desc), which, level, ctypes.byref(nr), ctypes.byref(nc),
                                    ctypes.byref(nnz), ctypes.byref(ptr), ctypes.byref(col), ctypes.byref(val))
    if st != SELM_OK:
        raise SelmError(st, "selm_mac_host_matrix failed")
    try:
        indptr = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(_LL)), (nr.value + 1,)).copy()
        indices = np.ctypeslib.as_array(ctypes.cast(col, ctypes.POINTER(_I)), (max(1, nnz.value),))[:nnz.value].copy()
        data = np.ctypeslib.as_array(ctypes.cast(val, ctypes.POINTER(_D)), (max(1, nnz.value),))[:nnz.value].copy()
    finally:
        for q in (ptr, col, val):
            lib().selm_mac_host_free(q)
    return nr.value, nc.value, indptr, indices, data


def selm_mac_host_colours(desc, level):
    import numpy as np
    n, col = _I(0), _P()
    st = lib().selm_mac_host_colours(ctypes.byref(desc), level, ctypes.byref(n), ctypes.byref(col))
    if st != SELM_OK:
        raise SelmError(st, "selm_mac_host_colours failed")
    try:
        out = np.ctypeslib.as_array(ctypes.cast(col, ctypes.POINTER(_I)), (max(1, n.value),))[:n.value].copy()
    finally:
        lib().selm_mac_host_free(col)
    return out


# -- exact Stokes mobility and the Ito drift --------------------------------------
def selm_mg_stokes_solve(h, f, u, tol=0.0, stream=None):
    it, res = _I(0), _D(0.0)
    _check(h, lib().selm_mg_stokes_solve(h, _ptr(f), _ptr(u), tol, ctypes.byref(it), ctypes.byref(res),
                                         _stream(stream)))
    return it.value, res.value


def selm_mg_stokes_mobility(h, X, F, U, stream=None):
    _check(h, lib().selm_mg_stokes_mobility(h, X.shape[0], _ptr(X), _ptr(F), _ptr(U), _stream(stream)))


def selm_mg_rfd_directions(h, np_, step, W, stream=None):
    _check(h, lib().selm_mg_rfd_directions(h, np_, step, _ptr(W), _stream(stream)))


def selm_mg_rfd_drift(h, X, W, delta, d, stream=None):
    _check(h, lib().selm_mg_rfd_drift(h, X.shape[0], _ptr(X), _ptr(W), delta, _ptr(d), _stream(stream)))


def selm_mg_stokes_step(h, X, F, dt, nsteps, ncycles, delta, stream=None):
    _check(h, lib().selm_mg_stokes_step(h, X.shape[0], _ptr(X), _ptr(F), dt, nsteps, ncycles, delta,
                                        _stream(stream)))
