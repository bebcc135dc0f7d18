"""FP64 CPU oracle for the RNA / ARNA particle-filter step (ctypes wrapper).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
CUDA library and its Python binding never import it.

Everything here is argument marshalling around ``pf_oracle.c``; the
arithmetic, and the paper citations for it, live in that file.

Arrays follow the oracle's own conventions: populations and states are
float64 ``(5, N)`` arrays (x, y, vx, vy, I) with slot ``g * Np + j``; group
arrays have length ``G``.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional

import numpy as np

from . import build as _build

RNA, ARNA = 0, 1
OBS_IMAGE, OBS_POINT, OBS_FRAME = 0, 1, 2
RESAMPLE_ALWAYS, RESAMPLE_ESS = 0, 1
SEND_SYSTEMATIC, SEND_KEYED = 0, 1
TOPO_RING, TOPO_NODE_RING, TOPO_HYPERCUBE = 0, 1, 2
INIT_POINT, INIT_UNIFORM, INIT_SHARING = 0, 1, 2


class Cfg(C.Structure):
    _fields_ = [
        ("G", C.c_int32), ("Np", C.c_int32), ("H", C.c_int32), ("W", C.c_int32),
        ("R", C.c_int32), ("mode", C.c_int32), ("obs_kind", C.c_int32), ("resample_rule", C.c_int32),
        ("sigma_psf", C.c_double), ("background", C.c_double), ("sigma_obs", C.c_double),
        ("sigma_pos", C.c_double), ("sigma_v", C.c_double), ("sigma_I", C.c_double),
        ("ex_ratio", C.c_double), ("cutoff", C.c_double),
        ("seed", C.c_uint64), ("track", C.c_uint32), ("send_rule", C.c_int32),
        ("ess_fraction", C.c_double), ("topology", C.c_int32), ("node_groups", C.c_int32),
    ]


_P = C.c_void_p


class _StepOut(C.Structure):
    _fields_ = [(n, _P) for n in (
        "sigma", "n_ex", "pe_eff", "src", "origin", "X", "loglik", "lw", "q", "anc",
        "Lambda_out", "gxhat", "gess", "logc", "xhat", "pop_out", "degenerate", "omega", "resampled")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.ora_philox.argtypes = [C.c_uint64, _P, _P]
        L.ora_uniform.argtypes = [C.c_uint32]
        L.ora_uniform.restype = C.c_double
        L.ora_bounded_batch.argtypes = [_P, C.c_int64, C.c_uint32, _P]
        L.ora_draw_bounded.argtypes = [C.POINTER(Cfg), C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
        L.ora_draw_bounded.restype = C.c_uint32
        L.ora_normals.argtypes = [C.POINTER(Cfg), C.c_uint32, C.c_uint32, C.c_uint32, _P]
        L.ora_fisher_yates.argtypes = [C.c_int32, _P, _P]
        L.ora_ring.argtypes = [C.POINTER(Cfg), C.c_uint32, _P]
        L.ora_pred.argtypes = [C.c_int32, _P, _P]
        L.ora_pred_topo.argtypes = [C.POINTER(Cfg), _P, _P]
        L.ora_hyper_dims.argtypes = [C.c_int32]
        L.ora_hyper_dims.restype = C.c_int32
        L.ora_pe_eff.argtypes = [C.c_int32, _P]
        L.ora_pe_eff.restype = C.c_double
        L.ora_n_ex.argtypes = [C.POINTER(Cfg), C.c_uint32, _P, _P]
        L.ora_n_ex.restype = C.c_int32
        L.ora_exchange_offset.argtypes = [C.POINTER(Cfg), C.c_uint32, C.c_uint32]
        L.ora_exchange_offset.restype = C.c_uint32
        L.ora_exchange.argtypes = [C.POINTER(Cfg), C.c_uint32, _P, C.c_int32, _P, _P, _P, _P]
        L.ora_propagate.argtypes = [C.POINTER(Cfg), C.c_uint32, _P, _P]
        L.ora_loglik_image.argtypes = [C.POINTER(Cfg), _P, C.c_double, C.c_double, C.c_double]
        L.ora_loglik_image.restype = C.c_double
        L.ora_loglik_frame.argtypes = [C.POINTER(Cfg), _P, C.c_double, C.c_double, C.c_double]
        L.ora_loglik_frame.restype = C.c_double
        L.ora_loglik_image_batch.argtypes = [C.POINTER(Cfg), _P, _P, C.c_int64, _P]
        L.ora_exp2_coeffs.argtypes = [_P]
        L.ora_quantize.argtypes = [_P, C.c_int32, _P]
        L.ora_resample.argtypes = [_P, C.c_int32, C.c_uint32, _P]
        L.ora_resample_uniform.argtypes = [C.POINTER(Cfg), C.c_uint32, C.c_uint32]
        L.ora_resample_uniform.restype = C.c_uint32
        L.ora_init.argtypes = [C.POINTER(Cfg), C.c_int32, _P, _P, _P, C.c_double, _P]
        L.ora_perm_bits.argtypes = [C.c_uint32]
        L.ora_perm_bits.restype = C.c_int
        L.ora_send_keys.argtypes = [C.POINTER(Cfg), C.c_uint32, C.c_uint32, _P]
        L.ora_send_perm.argtypes = [C.c_uint32, C.c_uint32, _P]
        L.ora_send_perm.restype = C.c_uint32
        L.ora_send_perm_inv.argtypes = [C.c_uint32, C.c_uint32, _P]
        L.ora_send_perm_inv.restype = C.c_uint32
        L.ora_ess_code.argtypes = [C.c_double]
        L.ora_ess_code.restype = C.c_uint32
        L.ora_ess_test.argtypes = [_P, C.c_int32, C.c_double]
        L.ora_ess_test.restype = C.c_int
        L.ora_step.argtypes = [C.POINTER(Cfg), C.c_uint32, _P, _P, _P, _P, _P, C.POINTER(_StepOut)]
        L.ora_step.restype = C.c_int
        L.ora_run.argtypes = [C.POINTER(Cfg), _P, _P, C.c_int32] + [_P] * 9
        L.ora_loglik_image_grad.argtypes = [C.POINTER(Cfg), _P, C.c_double, C.c_double, C.c_double, _P]
        L.ora_loglik_image_grad.restype = C.c_double
        L.ora_replay_grad.argtypes = [C.POINTER(Cfg), C.c_int32, _P, _P, _P, C.c_double, _P, C.c_int32, _P, _P, _P]
        L.ora_replay_grad.restype = C.c_int
        L.ora_replay_grad_ex.argtypes = [C.POINTER(Cfg), C.c_int32, _P, _P, _P, C.c_double, _P, C.c_int32, _P,
                                         C.c_int32, _P, _P, _P]
        L.ora_replay_grad_ex.restype = C.c_int
        L.ora_run.restype = C.c_int
        L.ora_set_threads.argtypes = [C.c_int]
        L.ora_set_threads.restype = C.c_int
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Host threads of the oracle step's per-particle and per-group loops
    (1 by default); returns the count in effect (1 without OpenMP).  The
    results do not depend on it."""
    return int(lib().ora_set_threads(int(n)))


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def make_cfg(G, Np, H=64, W=64, R=5, mode=RNA, obs_kind=OBS_IMAGE, sigma_psf=1.5, background=1.0,
             sigma_obs=1.0, sigma_pos=0.5, sigma_v=0.1, sigma_I=0.5, ex_ratio=0.1, cutoff=0.99,
             seed=0, track=0, resample_rule=RESAMPLE_ALWAYS, ess_fraction=0.5, send_rule=SEND_SYSTEMATIC,
             topology=TOPO_RING, node_groups=1) -> Cfg:
    return Cfg(G=G, Np=Np, H=H, W=W, R=R, mode=mode, obs_kind=obs_kind, sigma_psf=sigma_psf,
               background=background, sigma_obs=sigma_obs, sigma_pos=sigma_pos, sigma_v=sigma_v,
               sigma_I=sigma_I, ex_ratio=ex_ratio, cutoff=cutoff, seed=seed, track=track,
               resample_rule=resample_rule, ess_fraction=ess_fraction, send_rule=send_rule, topology=topology,
               node_groups=node_groups)


def cfg_from_workload(wl, track: int = 0) -> Cfg:
    """Oracle configuration from a ``synth.Workload`` (plain parameters).

    Real parameters are rounded to FP32 first: the GPU library receives them
    as FP32, and both sides must work from the same numbers."""
    f = lambda v: float(np.float32(v))  # noqa: E731
    obs = OBS_FRAME if getattr(wl, "obs_model", 0) == 1 else OBS_IMAGE
    return make_cfg(G=wl.G, Np=wl.Np, H=wl.H, W=wl.W, R=wl.patch_radius, mode=wl.mode, obs_kind=obs,
                    sigma_psf=f(wl.sigma_psf), background=f(wl.background), sigma_obs=f(wl.sigma_obs),
                    sigma_pos=f(wl.sigma_pos), sigma_v=f(wl.sigma_v), sigma_I=f(wl.sigma_I),
                    ex_ratio=f(wl.ex_ratio), cutoff=f(wl.pe_eff_cutoff), seed=wl.seed, track=track,
                    resample_rule=getattr(wl, "resample_rule", 0), ess_fraction=f(getattr(wl, "ess_fraction", 0.5)),
                    send_rule=getattr(wl, "send_rule", 0), topology=getattr(wl, "topology", 0),
                    node_groups=getattr(wl, "node_groups", 1))


# ---------------------------------------------------------------- primitives
def philox(seed: int, ctr) -> np.ndarray:
    c = _c(ctr, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().ora_philox(seed, _ptr(c), _ptr(out))
    return out


def uniform(w: int) -> float:
    return lib().ora_uniform(w)


def bounded_batch(words: np.ndarray, s: int) -> np.ndarray:
    w = _c(words, np.uint32)
    out = np.empty(w.size, np.int32)
    lib().ora_bounded_batch(_ptr(w), w.size, s, _ptr(out))
    return out


def draw_bounded(cfg: Cfg, stream: int, c0: int, k: int, s: int) -> int:
    return lib().ora_draw_bounded(C.byref(cfg), stream, c0, k, s)


def normals(cfg: Cfg, g: int, j: int, k: int) -> np.ndarray:
    out = np.zeros(5)
    lib().ora_normals(C.byref(cfg), g, j, k, _ptr(out))
    return out


def fisher_yates(r) -> np.ndarray:
    r = _c(r, np.uint32)
    out = np.zeros(r.size, np.int32)
    lib().ora_fisher_yates(r.size, _ptr(r), _ptr(out))
    return out


def ring(cfg: Cfg, k: int) -> np.ndarray:
    out = np.zeros(cfg.G, np.int32)
    lib().ora_ring(C.byref(cfg), k, _ptr(out))
    return out


def pred(sigma) -> np.ndarray:
    s = _c(sigma, np.int32)
    out = np.zeros(s.size, np.int32)
    lib().ora_pred(s.size, _ptr(s), _ptr(out))
    return out


def pred_topo(cfg: Cfg, sigma) -> np.ndarray:
    """The sender of every group under the track's topology."""
    s = _c(sigma, np.int32)
    out = np.zeros(s.size, np.int32)
    lib().ora_pred_topo(C.byref(cfg), _ptr(s), _ptr(out))
    return out


def hyper_dims(G: int) -> int:
    return int(lib().ora_hyper_dims(G))


def pe_eff(Lam) -> float:
    L = _c(Lam, np.float64)
    return lib().ora_pe_eff(L.size, _ptr(L))


def n_ex(cfg: Cfg, k: int, Lam):
    L = _c(Lam, np.float64)
    pe = np.zeros(1)
    n = lib().ora_n_ex(C.byref(cfg), k, _ptr(L), _ptr(pe))
    return n, float(pe[0])


def exchange_offset(cfg: Cfg, g: int, k: int) -> int:
    return lib().ora_exchange_offset(C.byref(cfg), g, k)


def exchange(cfg: Cfg, k: int, sigma, nex: int, pop):
    N = cfg.G * cfg.Np
    s = _c(sigma, np.int32)
    p = _c(pop, np.float64)
    out = np.zeros((5, N))
    src = np.zeros(N, np.int32)
    org = np.zeros(N, np.int32)
    lib().ora_exchange(C.byref(cfg), k, _ptr(s), nex, _ptr(p), _ptr(out), _ptr(src), _ptr(org))
    return out, src, org


def propagate(cfg: Cfg, k: int, pop) -> np.ndarray:
    p = _c(pop, np.float64)
    out = np.zeros_like(p)
    lib().ora_propagate(C.byref(cfg), k, _ptr(p), _ptr(out))
    return out


def loglik_image(cfg: Cfg, frame, x: float, y: float, I: float) -> float:
    f = _c(frame, np.float32)
    return lib().ora_loglik_image(C.byref(cfg), _ptr(f), x, y, I)


def loglik_frame(cfg: Cfg, frame, x: float, y: float, I: float) -> float:
    """The frame likelihood ratio (ora_loglik_frame) of one state."""
    f = _c(frame, np.float32)
    return lib().ora_loglik_frame(C.byref(cfg), _ptr(f), x, y, I)


def loglik_image_many(cfg: Cfg, frame, states) -> np.ndarray:
    """l for each column of a (5, n) state array."""
    f = _c(frame, np.float32)
    st = _c(states, np.float64)
    n = st.shape[1]
    out = np.zeros(n)
    lib().ora_loglik_image_batch(C.byref(cfg), _ptr(f), _ptr(st), n, _ptr(out))
    return out


def exp2_coeffs() -> np.ndarray:
    out = np.zeros(8, np.float32)
    lib().ora_exp2_coeffs(_ptr(out))
    return out


def quantize(lw) -> np.ndarray:
    a = _c(lw, np.float32)
    q = np.zeros(a.size, np.uint64)
    lib().ora_quantize(_ptr(a), a.size, _ptr(q))
    return q


def resample(q, u: int) -> np.ndarray:
    a = _c(q, np.uint64)
    anc = np.zeros(a.size, np.int32)
    lib().ora_resample(_ptr(a), a.size, u, _ptr(anc))
    return anc


def resample_uniform(cfg: Cfg, g: int, k: int) -> int:
    return lib().ora_resample_uniform(C.byref(cfg), g, k)


def init_population(cfg: Cfg, kind: int, x0, lo=None, hi=None, radius: float = 0.0) -> np.ndarray:
    N = cfg.G * cfg.Np
    x0 = _c(x0, np.float64)
    lo = _c(lo if lo is not None else np.zeros(5), np.float64)
    hi = _c(hi if hi is not None else np.zeros(5), np.float64)
    pop = np.zeros((5, N))
    lib().ora_init(C.byref(cfg), kind, _ptr(x0), _ptr(lo), _ptr(hi), radius, _ptr(pop))
    return pop


@dataclasses.dataclass
class StepResult:
    sigma: np.ndarray
    n_ex: int
    pe_eff: float
    src: np.ndarray
    origin: np.ndarray
    X: np.ndarray
    loglik: np.ndarray
    lw: np.ndarray
    q: np.ndarray
    anc: np.ndarray
    Lambda: np.ndarray
    gxhat: np.ndarray
    gess: np.ndarray
    logc: float
    xhat: np.ndarray
    pop_out: np.ndarray
    degenerate: int
    all_degenerate: bool
    omega: np.ndarray      # (N,) log weight of each output slot within its group
    resampled: np.ndarray  # (G,) 1 where the group resampled


def perm_bits(n: int) -> int:
    return int(lib().ora_perm_bits(n))


def send_keys(cfg: Cfg, g: int, k: int) -> np.ndarray:
    """The four Feistel round keys of group g's send permutation at step k."""
    key = np.zeros(4, np.uint32)
    lib().ora_send_keys(C.byref(cfg), g, k, _ptr(key))
    return key


def send_perm(t: int, n: int, key) -> int:
    key = _c(key, np.uint32)
    return int(lib().ora_send_perm(t, n, _ptr(key)))


def send_perm_inv(j: int, n: int, key) -> int:
    key = _c(key, np.uint32)
    return int(lib().ora_send_perm_inv(j, n, _ptr(key)))


def ess_code(ess_fraction: float) -> int:
    return int(lib().ora_ess_code(float(ess_fraction)))


def ess_test(q, ess_fraction: float) -> bool:
    """Alg. 1's N_eff < N_thresh test on one group's weight codes."""
    q = _c(q, np.uint64)
    return bool(lib().ora_ess_test(_ptr(q), len(q), float(ess_fraction)))


def step(cfg: Cfg, k: int, obs, pop_in, Lambda_in=None, lw_override=None, omega_in=None) -> StepResult:
    G, Np = cfg.G, cfg.Np
    N = G * Np
    obs = _c(obs, np.float32)
    pop = _c(pop_in, np.float64)
    Lam = _c(Lambda_in if Lambda_in is not None else np.zeros(G), np.float64)
    lwo = None if lw_override is None else _c(lw_override, np.float32)
    om = None if omega_in is None else _c(omega_in, np.float64)
    a = dict(sigma=np.zeros(G, np.int32), n_ex=np.zeros(1, np.int32), pe_eff=np.zeros(1),
             src=np.zeros(N, np.int32), origin=np.zeros(N, np.int32), X=np.zeros((5, N)),
             loglik=np.zeros(N), lw=np.zeros(N), q=np.zeros(N, np.uint64), anc=np.zeros(N, np.int32),
             Lambda_out=np.zeros(G), gxhat=np.zeros((5, G)), gess=np.zeros(G), logc=np.zeros(1),
             xhat=np.zeros(5), pop_out=np.zeros((5, N)), degenerate=np.zeros(1, np.int32),
             omega=np.zeros(N), resampled=np.zeros(G, np.int32))
    so = _StepOut(**{n: _ptr(v) for n, v in a.items()})
    rc = lib().ora_step(C.byref(cfg), k, _ptr(obs), _ptr(pop), _ptr(Lam), _ptr(om), _ptr(lwo), C.byref(so))
    return StepResult(sigma=a["sigma"], n_ex=int(a["n_ex"][0]), pe_eff=float(a["pe_eff"][0]),
                      src=a["src"], origin=a["origin"], X=a["X"], loglik=a["loglik"], lw=a["lw"],
                      q=a["q"], anc=a["anc"], Lambda=a["Lambda_out"], gxhat=a["gxhat"], gess=a["gess"],
                      logc=float(a["logc"][0]), xhat=a["xhat"], pop_out=a["pop_out"],
                      degenerate=int(a["degenerate"][0]), all_degenerate=bool(rc), omega=a["omega"],
                      resampled=a["resampled"])


@dataclasses.dataclass
class RunResult:
    xhat: np.ndarray      # (T, 5)
    logc: np.ndarray      # (T,)
    n_ex: np.ndarray      # (T,)
    pe_eff: np.ndarray    # (T,)
    sigma: np.ndarray     # (T, G)
    Lambda: np.ndarray    # (T, G)
    gxhat: np.ndarray     # (T, 5, G)
    n_resampled: np.ndarray  # (T,) groups that resampled
    pop_final: np.ndarray  # (5, N)
    failed_step: int


def run(cfg: Cfg, pop0, obs, T: int) -> RunResult:
    G, N = cfg.G, cfg.G * cfg.Np
    pop0 = _c(pop0, np.float64)
    obs = _c(obs, np.float32)
    r = RunResult(xhat=np.zeros((T, 5)), logc=np.zeros(T), n_ex=np.zeros(T, np.int32),
                  pe_eff=np.zeros(T), sigma=np.zeros((T, G), np.int32), Lambda=np.zeros((T, G)),
                  gxhat=np.zeros((T, 5, G)), n_resampled=np.zeros(T, np.int32), pop_final=np.zeros((5, N)),
                  failed_step=-1)
    r.failed_step = lib().ora_run(C.byref(cfg), _ptr(pop0), _ptr(obs), T, _ptr(r.xhat), _ptr(r.logc),
                                  _ptr(r.n_ex), _ptr(r.pe_eff), _ptr(r.sigma), _ptr(r.Lambda),
                                  _ptr(r.gxhat), _ptr(r.n_resampled), _ptr(r.pop_final))
    return r


# ------------------------------------------------------------- gradients
THETA = ("sigma_psf", "A", "b", "sigma_pos", "sigma_v")


def loglik_image_grad(cfg: Cfg, frame, x: float, y: float, I: float):
    """(l, [dl/dx, dl/dy, dl/dI, dl/dsigma_psf, dl/db])."""
    f = _c(frame, np.float32)
    d = np.zeros(5)
    l = lib().ora_loglik_image_grad(C.byref(cfg), _ptr(f), x, y, I, _ptr(d))
    return l, d


def replay_grad(cfg: Cfg, kind: int, x0, frames, T: int, parents, lo=None, hi=None, radius: float = 0.0,
                fp32_states: bool = False, states=None):
    """(log Z, d log Z / d theta) of a replay with frozen ancestry; theta =
    (sigma_psf, A = x0[4], background, sigma_pos, sigma_v).  fp32_states:
    the same replay with every state rounded to FP32 after each propagation
    (the rest in FP64), to measure the estimator's sensitivity to FP32 state
    storage.  states: optional (T, 5, N) states to evaluate the likelihood
    at instead of the replay's own (its tangents still follow the ancestry
    and the noise)."""
    N = cfg.G * cfg.Np
    x0 = _c(x0, np.float64)
    lo = _c(lo if lo is not None else np.zeros(5), np.float64)
    hi = _c(hi if hi is not None else np.zeros(5), np.float64)
    fr = _c(frames, np.float32)
    par = _c(parents, np.int32)
    assert par.shape == (T, N)
    lz = np.zeros(1)
    g = np.zeros(5)
    st = None if states is None else _c(states, np.float64)
    assert st is None or st.shape == (T, 5, N)
    rc = lib().ora_replay_grad_ex(C.byref(cfg), kind, _ptr(x0), _ptr(lo), _ptr(hi), radius, _ptr(fr), T, _ptr(par),
                                  1 if fp32_states else 0, _ptr(st), _ptr(lz), _ptr(g))
    if rc != 0:
        raise ValueError("replay_grad needs resample_rule = RESAMPLE_ALWAYS")
    return float(lz[0]), g


def run_with_parents(cfg: Cfg, pop0, obs, T: int):
    """An oracle run that also returns each step's parents (T, N) -- the
    exchange composed with the previous resampling, track-local slots."""
    G, Np = cfg.G, cfg.Np
    N = G * Np
    par = np.zeros((T, N), np.int32)
    par[0] = np.arange(N)
    pop, lam, logc, prev = pop0, None, [], None
    base = np.repeat(np.arange(G, dtype=np.int64) * Np, Np)
    for k in range(T):
        r = step(cfg, k, obs[k], pop, lam)
        if k > 0:
            par[k] = prev[r.src]
        prev = r.anc.astype(np.int64) + base
        pop, lam = r.pop_out, r.Lambda
        logc.append(r.logc)
    return par, np.array(logc)
