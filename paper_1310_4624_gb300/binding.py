"""ctypes binding of libpfarna (include/pfarna.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the filter.  Loading fails loudly if the CUDA library has not
been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

PF_OK, PF_ERR_ARG, PF_ERR_STATE, PF_ERR_CUDA, PF_ERR_WORKSPACE, PF_ERR_DEGENERATE, PF_ERR_TIMEOUT, \
    PF_ERR_DEVICE = range(8)
PF_RNA, PF_ARNA = 0, 1
PF_INIT_POINT, PF_INIT_UNIFORM, PF_INIT_SHARING, PF_INIT_USER = range(4)
PF_RESAMPLE_ALWAYS, PF_RESAMPLE_ESS = 0, 1
PF_SEND_SYSTEMATIC, PF_SEND_KEYED = 0, 1
PF_TOPO_RING, PF_TOPO_NODE_RING, PF_TOPO_HYPERCUBE = 0, 1, 2

STATUS_NAMES = {0: "PF_OK", 1: "PF_ERR_ARG", 2: "PF_ERR_STATE", 3: "PF_ERR_CUDA", 4: "PF_ERR_WORKSPACE",
                5: "PF_ERR_DEGENERATE", 6: "PF_ERR_TIMEOUT", 7: "PF_ERR_DEVICE"}

# Every symbol include/pfarna.h declares.
EXPORTS = ("pf_abi_version", "pf_query_workspace", "pf_init", "pf_step", "pf_host_staging_bytes", "pf_step_host",
           "pf_estimate", "pf_estimate_async",
           "pf_exchange_stats",
           "pf_history", "pf_particles", "pf_resample_workspace", "pf_resample", "pf_resample_noalloc", "pf_resample_check",
           "pf_profile_enable", "pf_profile_read", "pf_set_theta", "pf_reset", "pf_backward", "pf_set_replay", "pf_step_table",
           "pf_graph_step", "pf_autotune", "pf_checkpoint_bytes", "pf_save", "pf_load", "pf_destroy",
           "pf_last_error")
THETA_NAMES = ("sigma_psf", "amplitude", "background", "sigma_pos", "sigma_v")
KERNEL_NAMES = ("frame_prep", "propagate_weight", "resample", "global", "fused_step")


class pf_track_config(C.Structure):
    _fields_ = [
        ("G", C.c_int32), ("Np", C.c_int32), ("H", C.c_int32), ("W", C.c_int32),
        ("patch_radius", C.c_int32), ("mode", C.c_int32),
        ("sigma_psf", C.c_float), ("background", C.c_float), ("sigma_obs", C.c_float),
        ("sigma_pos", C.c_float), ("sigma_v", C.c_float), ("sigma_I", C.c_float),
        ("ex_ratio", C.c_float), ("pe_eff_cutoff", C.c_float),
        ("init_kind", C.c_int32),
        ("init_state", C.c_float * 5), ("init_lo", C.c_float * 5), ("init_hi", C.c_float * 5),
        ("init_radius", C.c_float), ("obs_model", C.c_int32),
        ("seed", C.c_uint64), ("track_id", C.c_uint32), ("record_ancestors", C.c_int32),
        ("resample_rule", C.c_int32), ("ess_fraction", C.c_float), ("send_rule", C.c_int32),
        ("topology", C.c_int32), ("node_groups", C.c_int32),
    ]


class pf_step_stats(C.Structure):
    _fields_ = [
        ("step", C.c_int32), ("n_ex", C.c_int32),
        ("pe_eff", C.c_double), ("log_c", C.c_double), ("log_Z", C.c_double),
        ("xhat", C.c_float * 5), ("degenerate_groups", C.c_int32), ("resampled_groups", C.c_int32),
    ]


class PFError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        super().__init__("%s -> %s: %s" % (func, STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None
_P = C.c_void_p


def lib_path() -> str:
    """The library to load: the PF_DEBUG build when PFARNA_DEBUG=1."""
    return _build.LIB_DEBUG if os.environ.get("PFARNA_DEBUG") == "1" else _build.LIB


def load():
    """Open libpfarna.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("libpfarna.so is not built (%s); run `python -c \"import __graft_entry__ as g; "
                           "g.build()\"` first" % path)
    L = C.CDLL(path)
    L.pf_abi_version.restype = C.c_int32
    L.pf_query_workspace.argtypes = [C.POINTER(pf_track_config), C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]
    L.pf_init.argtypes = [C.POINTER(pf_track_config), C.c_int32, C.c_int32, _P, C.c_size_t, _P, _P,
                          C.POINTER(_P)]
    L.pf_step.argtypes = [_P, C.POINTER(_P), _P]
    L.pf_host_staging_bytes.argtypes = [_P, C.POINTER(C.c_size_t)]
    L.pf_step_host.argtypes = [_P, C.POINTER(_P), _P, C.c_size_t, _P]
    L.pf_estimate.argtypes = [_P, _P, _P]
    L.pf_estimate_async.argtypes = [_P, _P, _P, _P]
    L.pf_exchange_stats.argtypes = [_P, C.c_int32, C.c_int32, C.POINTER(pf_step_stats), _P, _P, _P, _P]
    L.pf_history.argtypes = [_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(pf_step_stats)]
    L.pf_particles.argtypes = [_P, C.c_int32, _P, _P, _P, _P, _P]
    L.pf_resample_workspace.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]
    L.pf_resample.argtypes = [_P, _P, C.c_int32, C.c_int32, _P, _P, _P, C.c_size_t, _P]
    L.pf_resample_noalloc.argtypes = [_P, _P, C.c_int32, C.c_int32, _P, _P, _P]
    L.pf_resample_check.argtypes = [_P, _P]
    L.pf_set_replay.argtypes = [_P, _P, C.c_int32, _P]
    L.pf_profile_enable.argtypes = [_P, C.c_int32]
    L.pf_profile_read.argtypes = [_P, C.c_int32, _P, _P]
    L.pf_set_theta.argtypes = [_P, C.c_int32, _P]
    L.pf_step_table.argtypes = [_P, _P, C.c_int32, _P]
    L.pf_graph_step.argtypes = [_P, _P, C.c_int32, _P]
    L.pf_autotune.argtypes = [_P, C.POINTER(_P), _P, _P, _P]
    L.pf_reset.argtypes = [_P, _P]
    L.pf_checkpoint_bytes.argtypes = [_P, C.POINTER(C.c_size_t)]
    L.pf_save.argtypes = [_P, _P, C.c_size_t, _P]
    L.pf_load.argtypes = [_P, _P, C.c_size_t, _P]
    L.pf_backward.argtypes = [_P, C.POINTER(_P), C.c_int32, _P, _P, _P, _P]
    L.pf_destroy.argtypes = [_P]
    L.pf_destroy.restype = None
    L.pf_last_error.argtypes = [_P]
    L.pf_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("pf_abi_version", "pf_destroy", "pf_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(st: int, func: str, handle=None):
    if st != PF_OK:
        raise PFError(st, func, load().pf_last_error(handle).decode(errors="replace"))


def pf_abi_version() -> int:
    return load().pf_abi_version()


def pf_query_workspace(cfgs, history: int) -> int:
    arr = (pf_track_config * len(cfgs))(*cfgs)
    n = C.c_size_t(0)
    _check(load().pf_query_workspace(arr, len(cfgs), history, C.byref(n)), "pf_query_workspace")
    return n.value


def pf_init(cfgs, history: int, workspace_ptr: int, nbytes: int, user_state_ptr, stream_ptr) -> int:
    arr = (pf_track_config * len(cfgs))(*cfgs)
    h = _P()
    _check(load().pf_init(arr, len(cfgs), history, workspace_ptr, nbytes, user_state_ptr, stream_ptr,
                          C.byref(h)), "pf_init")
    return h.value


def pf_step(handle: int, frame_ptrs, stream_ptr) -> None:
    arr = (_P * len(frame_ptrs))(*frame_ptrs)
    _check(load().pf_step(handle, arr, stream_ptr), "pf_step", handle)


def pf_host_staging_bytes(handle: int) -> int:
    n = C.c_size_t(0)
    _check(load().pf_host_staging_bytes(handle, C.byref(n)), "pf_host_staging_bytes", handle)
    return n.value


def pf_step_host(handle: int, frame_ptrs, staging_ptr, staging_bytes: int, stream_ptr) -> None:
    arr = (_P * len(frame_ptrs))(*frame_ptrs)
    _check(load().pf_step_host(handle, arr, staging_ptr, staging_bytes, stream_ptr), "pf_step_host", handle)


def pf_estimate(handle: int, xhat_host_ptr, logZ_host_ptr) -> int:
    """Returns the status (PF_OK or PF_ERR_DEGENERATE); raises on other errors."""
    st = load().pf_estimate(handle, xhat_host_ptr, logZ_host_ptr)
    if st not in (PF_OK, PF_ERR_DEGENERATE):
        _check(st, "pf_estimate", handle)
    return st


def pf_estimate_async(handle: int, xhat_host_ptr, logZ_host_ptr, stream) -> None:
    _check(load().pf_estimate_async(handle, xhat_host_ptr, logZ_host_ptr, stream), "pf_estimate_async", handle)


def pf_exchange_stats(handle: int, track: int, step: int, ring_ptr=None, logW_ptr=None, xhat_ptr=None,
                      ess_ptr=None) -> pf_step_stats:
    out = pf_step_stats()
    _check(load().pf_exchange_stats(handle, track, step, C.byref(out), ring_ptr, logW_ptr, xhat_ptr, ess_ptr),
           "pf_exchange_stats", handle)
    return out


def pf_history(handle: int, track: int, first: int, count: int):
    out = (pf_step_stats * count)()
    _check(load().pf_history(handle, track, first, count, out), "pf_history", handle)
    return list(out)


def pf_particles(handle: int, track: int, states_ptr, anc_ptr, logw_ptr, parent_ptr, stream_ptr) -> None:
    _check(load().pf_particles(handle, track, states_ptr, anc_ptr, logw_ptr, parent_ptr, stream_ptr),
           "pf_particles", handle)


def pf_resample_workspace(G: int, Np: int) -> int:
    n = C.c_size_t(0)
    _check(load().pf_resample_workspace(G, Np, C.byref(n)), "pf_resample_workspace")
    return n.value


def pf_resample(logw_ptr, u_ptr, G: int, Np: int, anc_ptr, q_ptr, ws_ptr, nbytes: int, stream_ptr) -> None:
    _check(load().pf_resample(logw_ptr, u_ptr, G, Np, anc_ptr, q_ptr, ws_ptr, nbytes, stream_ptr), "pf_resample")


def pf_resample_noalloc(logw_ptr, u_ptr, G: int, Np: int, anc_ptr, q_ptr, stream_ptr) -> None:
    _check(load().pf_resample_noalloc(logw_ptr, u_ptr, G, Np, anc_ptr, q_ptr, stream_ptr), "pf_resample_noalloc")


def pf_resample_check(ws_ptr, stream_ptr) -> None:
    _check(load().pf_resample_check(ws_ptr, stream_ptr), "pf_resample_check")


def pf_set_replay(handle: int, parents_ptr, T: int, stream_ptr) -> None:
    _check(load().pf_set_replay(handle, parents_ptr, T, stream_ptr), "pf_set_replay", handle)


def pf_profile_enable(handle: int, enable: bool) -> None:
    _check(load().pf_profile_enable(handle, 1 if enable else 0), "pf_profile_enable", handle)


def pf_profile_read(handle: int):
    """{kernel name: (launches, total ms)} of the recorded steps."""
    import numpy as np
    n = len(KERNEL_NAMES)
    cnt = np.zeros(n, np.int64)
    ms = np.zeros(n, np.float64)
    _check(load().pf_profile_read(handle, n, cnt.ctypes.data_as(_P), ms.ctypes.data_as(_P)), "pf_profile_read",
           handle)
    return {KERNEL_NAMES[i]: (int(cnt[i]), float(ms[i])) for i in range(n)}


def pf_step_table(handle: int, table_ptr, T_table: int, stream_ptr) -> None:
    _check(load().pf_step_table(handle, table_ptr, T_table, stream_ptr), "pf_step_table", handle)


def pf_graph_step(handle: int, table_ptr, T_table: int, stream_ptr) -> None:
    _check(load().pf_graph_step(handle, table_ptr, T_table, stream_ptr), "pf_graph_step", handle)


def pf_autotune(handle: int, frame_ptrs, stream_ptr):
    arr = (_P * len(frame_ptrs))(*frame_ptrs)
    g = C.c_int32(0)
    c = C.c_int32(0)
    _check(load().pf_autotune(handle, arr, C.byref(g), C.byref(c), stream_ptr), "pf_autotune", handle)
    return g.value, c.value


def pf_set_theta(handle: int, track: int, theta) -> None:
    arr = (C.c_float * 5)(*[float(v) for v in theta])
    _check(load().pf_set_theta(handle, track, arr), "pf_set_theta", handle)


def pf_reset(handle: int, stream_ptr) -> None:
    _check(load().pf_reset(handle, stream_ptr), "pf_reset", handle)


def pf_backward(handle: int, frame_ptrs, T: int, dlogZ, grad_ptr, logZ_ptr, stream_ptr) -> None:
    arr = (_P * len(frame_ptrs))(*frame_ptrs)
    seeds = (C.c_float * len(dlogZ))(*[float(v) for v in dlogZ])
    _check(load().pf_backward(handle, arr, T, seeds, grad_ptr, logZ_ptr, stream_ptr), "pf_backward", handle)


def pf_checkpoint_bytes(handle: int) -> int:
    n = C.c_size_t(0)
    _check(load().pf_checkpoint_bytes(handle, C.byref(n)), "pf_checkpoint_bytes", handle)
    return n.value


def pf_save(handle: int, buf, stream_ptr) -> None:
    """buf: a writable buffer (bytearray / numpy uint8) of pf_checkpoint_bytes."""
    mv = (C.c_char * len(buf)).from_buffer(buf)
    _check(load().pf_save(handle, C.addressof(mv), len(buf), stream_ptr), "pf_save", handle)


def pf_load(handle: int, buf, stream_ptr) -> None:
    mv = (C.c_char * len(buf)).from_buffer(buf)
    _check(load().pf_load(handle, C.addressof(mv), len(buf), stream_ptr), "pf_load", handle)


def pf_destroy(handle: int) -> None:
    load().pf_destroy(handle)


def pf_last_error(handle=None) -> str:
    return load().pf_last_error(handle).decode(errors="replace")
