"""ParticleFilter: a PyTorch-facing handle on libpfarna.

PyTorch supplies device memory (the workspace, frames, outputs) and the CUDA
stream; every step of the filter runs in the library's kernels.

Typical use (one track; a list of configurations makes a batch)::

    from paper_1310_4624_gb300 import synth
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wl = synth.tracking()                       # G = 64 x 16384, ARNA, 512 x 512
    frames, truth = synth.make_sequence(wl)
    fr = torch.from_numpy(frames).cuda()
    pf = ParticleFilter([config_from_workload(wl, truth[0])])
    for k in range(wl.T):
        pf.step(fr[k])                          # Alg. 3 for every track
    xhat, log_z, status = pf.estimate()         # x^ and log Z of the last step
    stats = pf.stats(wl.T - 1)                  # N_ex, PE_eff, ring, group weights
    pf.close()

Frames streamed from host memory, with the estimate read back every step and
nothing waiting on the device (the library uploads frame k+1 while step k
runs; page-locked buffers make both directions asynchronous)::

    host = torch.from_numpy(frames).pin_memory()
    outs = [(torch.zeros(1, 5).pin_memory(), torch.zeros(1, dtype=torch.float64).pin_memory())
            for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    for k in range(wl.T):
        pf.step_host(host[k])
        pf.estimate_async(*outs[k & 1])
        done[k & 1].record(pf.stream)
        if k > 0:
            done[(k - 1) & 1].synchronize()     # step k-1's estimate is on the host
            use(outs[(k - 1) & 1][0])

Method variants are fields of the configuration: ``resample_rule`` /
``ess_fraction`` (Alg. 1's N_eff test per group), ``send_rule`` (keyed random
send sets), ``topology`` / ``node_groups`` (Sec. VI's node-aware ring and
hypercube), ``obs_model`` (the frame likelihood ratio).
"""
from __future__ import annotations

import ctypes as C
import struct
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import binding as B
from .synth import INIT_POINT, INIT_SHARING, INIT_UNIFORM, Workload


def config_from_workload(wl: Workload, truth0=None, track_id: int = 0, record_ancestors: bool = False,
                         init_kind: Optional[int] = None) -> B.pf_track_config:
    """The C config of a workload; the initial population is centred on truth0."""
    c = B.pf_track_config()
    c.G, c.Np, c.H, c.W = wl.G, wl.Np, wl.H, wl.W
    c.patch_radius = wl.patch_radius
    c.mode = wl.mode
    c.sigma_psf, c.background, c.sigma_obs = wl.sigma_psf, wl.background, wl.sigma_obs
    c.sigma_pos, c.sigma_v, c.sigma_I = wl.sigma_pos, wl.sigma_v, wl.sigma_I
    c.ex_ratio, c.pe_eff_cutoff = wl.ex_ratio, wl.pe_eff_cutoff
    c.init_kind = wl.init if init_kind is None else init_kind
    x0 = np.zeros(5) if truth0 is None else np.asarray(truth0, np.float64)
    lo = [0.0, 0.0, -wl.share_vmax, -wl.share_vmax, wl.share_I[0]]
    hi = [wl.W - 1.0, wl.H - 1.0, wl.share_vmax, wl.share_vmax, wl.share_I[1]]
    for d in range(5):
        c.init_state[d] = float(x0[d])
        c.init_lo[d] = lo[d]
        c.init_hi[d] = hi[d]
    c.init_radius = wl.share_radius
    c.obs_model = getattr(wl, "obs_model", 0)
    c.seed = wl.seed
    c.track_id = track_id
    c.record_ancestors = 1 if record_ancestors else 0
    c.resample_rule = getattr(wl, "resample_rule", 0)
    c.ess_fraction = getattr(wl, "ess_fraction", 0.5)
    c.send_rule = getattr(wl, "send_rule", 0)
    c.topology = getattr(wl, "topology", 0)
    c.node_groups = max(1, getattr(wl, "node_groups", 1))
    return c


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


class ParticleFilter:
    """One handle over one or more tracks, in a workspace PyTorch allocates."""

    def __init__(self, configs: Sequence[B.pf_track_config], history: int = 128,
                 user_state: Optional[torch.Tensor] = None, device="cuda:0", stream: Optional[torch.cuda.Stream] = None):
        if not torch.cuda.is_available():
            raise RuntimeError("ParticleFilter needs a CUDA device; there is no CPU path")
        self.device = torch.device(device)
        self.configs = list(configs)
        self.n_tracks = len(self.configs)
        self.history = history
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.N = [c.G * c.Np for c in self.configs]
        nbytes = B.pf_query_workspace(self.configs, history)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self._ws_bytes = nbytes
        self._user = user_state
        self.handle = B.pf_init(self.configs, history, self._ws_ptr, nbytes, _ptr(user_state),
                                C.c_void_p(self.stream.cuda_stream))
        self.steps = 0
        self._staging = None  # device staging of step_host (allocated on first use)

    def close(self):
        if getattr(self, "handle", None):
            B.pf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, frames) -> None:
        """Advance every track by one step; frames: one (H, W) float32 CUDA tensor per track."""
        if isinstance(frames, torch.Tensor) and frames.dim() == 2:
            frames = [frames]
        ptrs = []
        for f in frames:
            if f.dtype != torch.float32 or not f.is_cuda or not f.is_contiguous():
                raise ValueError("frames must be contiguous float32 CUDA tensors")
            ptrs.append(f.data_ptr())
        B.pf_step(self.handle, ptrs, C.c_void_p(self.stream.cuda_stream))
        self.steps += 1

    def step_host(self, frames) -> None:
        """Advance every track by one step with frames in host memory: one
        (H, W) float32 CPU tensor per track, page-locked for the upload to
        overlap the previous step (pf_step_host; the device staging buffer
        is allocated on the first call and kept)."""
        if isinstance(frames, torch.Tensor) and frames.dim() == 2:
            frames = [frames]
        ptrs = []
        for f in frames:
            if f.dtype != torch.float32 or f.is_cuda or not f.is_contiguous():
                raise ValueError("frames must be contiguous float32 host tensors")
            ptrs.append(f.data_ptr())
        if self._staging is None:
            n = B.pf_host_staging_bytes(self.handle)
            self._staging = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
            self._staging_ptr = C.c_void_p((self._staging.data_ptr() + 255) // 256 * 256)
            self._staging_bytes = n
        B.pf_step_host(self.handle, ptrs, self._staging_ptr, self._staging_bytes, C.c_void_p(self.stream.cuda_stream))
        self.steps += 1

    def frame_table(self, frames_per_track) -> torch.Tensor:
        """Device table (T x n_tracks int64 pointers) of per-track frame
        tensors (each (T, H, W) float32 CUDA, contiguous)."""
        T = frames_per_track[0].shape[0]
        ptrs = [[f[k].data_ptr() for f in frames_per_track] for k in range(T)]
        return torch.tensor(ptrs, dtype=torch.int64, device=self.device).reshape(T, self.n_tracks)

    def step_table(self, table: torch.Tensor, graph: bool = False) -> None:
        """One step with frames from a device table (see frame_table)."""
        fn = B.pf_graph_step if graph else B.pf_step_table
        fn(self.handle, C.c_void_p(table.data_ptr()), table.shape[0], C.c_void_p(self.stream.cuda_stream))
        self.steps += 1

    def autotune(self, frames):
        """One step that also picks the launch shapes; returns (grid, cluster)."""
        if isinstance(frames, torch.Tensor) and frames.dim() == 2:
            frames = [frames]
        r = B.pf_autotune(self.handle, [f.data_ptr() for f in frames], C.c_void_p(self.stream.cuda_stream))
        self.steps += 1
        return r

    def profile(self, enable: bool = True) -> None:
        """Record CUDA events around each kernel of the following steps."""
        B.pf_profile_enable(self.handle, enable)

    def profile_read(self) -> dict:
        """{kernel: (launches, total ms)} since profiling was enabled / last read."""
        return B.pf_profile_read(self.handle)

    def estimate(self):
        """(xhat (n_tracks, 5) float32, log_Z (n_tracks,) float64, status)."""
        x = np.zeros((self.n_tracks, 5), np.float32)
        z = np.zeros(self.n_tracks, np.float64)
        st = B.pf_estimate(self.handle, x.ctypes.data_as(C.c_void_p), z.ctypes.data_as(C.c_void_p))
        return x, z, st

    def estimate_async(self, xhat: torch.Tensor, log_z: torch.Tensor) -> None:
        """Enqueue the read-back of x^ ((n_tracks, 5) float32) and log Z
        ((n_tracks,) float64) into host tensors on the filter's stream; they
        hold the values once the stream has passed this point.  Page-locked
        tensors are written by the finishing kernel itself (no copy on the
        stream), pageable ones by copies."""
        assert xhat.dtype == torch.float32 and xhat.numel() == 5 * self.n_tracks and not xhat.is_cuda
        assert log_z.dtype == torch.float64 and log_z.numel() == self.n_tracks and not log_z.is_cuda
        B.pf_estimate_async(self.handle, C.c_void_p(xhat.data_ptr()), C.c_void_p(log_z.data_ptr()),
                            C.c_void_p(self.stream.cuda_stream))

    def stats(self, step: int, track: int = 0) -> dict:
        G = self.configs[track].G
        ring = np.zeros(G, np.int32)
        logW = np.zeros(G, np.float64)
        gx = np.zeros((5, G), np.float32)
        ess = np.zeros(G, np.float32)
        s = B.pf_exchange_stats(self.handle, track, step, ring.ctypes.data_as(C.c_void_p),
                                logW.ctypes.data_as(C.c_void_p), gx.ctypes.data_as(C.c_void_p),
                                ess.ctypes.data_as(C.c_void_p))
        return dict(step=s.step, n_ex=s.n_ex, pe_eff=s.pe_eff, log_c=s.log_c, log_Z=s.log_Z,
                    xhat=np.array(s.xhat[:]), degenerate=s.degenerate_groups, resampled=s.resampled_groups,
                    ring=ring, logW=logW, group_xhat=gx, group_ess=ess)

    def history_stats(self, first: int, count: int, track: int = 0) -> List[dict]:
        out = B.pf_history(self.handle, track, first, count)
        return [dict(step=s.step, n_ex=s.n_ex, pe_eff=s.pe_eff, log_c=s.log_c, log_Z=s.log_Z,
                     xhat=np.array(s.xhat[:]), degenerate=s.degenerate_groups, resampled=s.resampled_groups)
                for s in out]

    def save(self) -> bytearray:
        """A checkpoint of the whole filter state (host memory)."""
        buf = bytearray(B.pf_checkpoint_bytes(self.handle))
        B.pf_save(self.handle, buf, C.c_void_p(self.stream.cuda_stream))
        return buf

    def load(self, buf: bytearray) -> None:
        """Restore a checkpoint taken from a filter of the same configurations."""
        B.pf_load(self.handle, buf, C.c_void_p(self.stream.cuda_stream))
        # the checkpoint header: magic, signature, workspace bytes (u64 each),
        # then the ABI version and the step count (int32)
        self.steps = struct.unpack_from("<i", bytes(buf[28:32]))[0]

    def set_theta(self, theta, track: int = 0) -> None:
        """theta = (sigma_psf, A, background, sigma_pos, sigma_v) of one track."""
        B.pf_set_theta(self.handle, track, [float(v) for v in theta])

    def reset(self) -> None:
        """Fresh initial population with the current parameters (step 0 next)."""
        B.pf_reset(self.handle, C.c_void_p(self.stream.cuda_stream))
        self.steps = 0

    def backward(self, frames, dlogZ=None):
        """d log Z / d theta over the steps run so far, ancestry fixed.

        frames: per step a frame tensor (one track) or a list of n_tracks
        frame tensors, the frames of the forward run.  Returns (grad
        (n_tracks, 5) float32 tensor, log Z of the replay (n_tracks,) float64
        tensor)."""
        T = len(frames)
        ptrs = []
        for f in frames:
            fs = [f] if isinstance(f, torch.Tensor) else list(f)
            assert len(fs) == self.n_tracks
            ptrs.extend(x.data_ptr() for x in fs)
        seeds = [1.0] * self.n_tracks if dlogZ is None else [float(v) for v in dlogZ]
        grad = torch.empty((self.n_tracks, 5), dtype=torch.float32, device=self.device)
        logz = torch.empty(self.n_tracks, dtype=torch.float64, device=self.device)
        B.pf_backward(self.handle, ptrs, T, seeds, C.c_void_p(grad.data_ptr()), C.c_void_p(logz.data_ptr()),
                      C.c_void_p(self.stream.cuda_stream))
        self.stream.synchronize()
        return grad, logz

    def set_replay(self, parents: torch.Tensor) -> None:
        """Replace the recorded ancestry of the steps run by `parents`
        ((T, N_total) int32 or uint32 CUDA tensor, row k the step-k parents
        of every track; row 0 ignored), for the next backward()."""
        assert parents.is_cuda and parents.dim() == 2 and parents.is_contiguous()
        assert parents.dtype in (torch.int32, torch.uint32) and parents.shape[1] == sum(self.N)
        B.pf_set_replay(self.handle, _ptr(parents), parents.shape[0], C.c_void_p(self.stream.cuda_stream))

    def particles(self, track: int = 0, parents: bool = False) -> dict:
        """Latest step's X_k (5, N), ancestors, log-weights (and parents)."""
        n = self.N[track]
        st = torch.empty((5, n), dtype=torch.float32, device=self.device)
        anc = torch.empty(n, dtype=torch.int32, device=self.device)
        lw = torch.empty(n, dtype=torch.float32, device=self.device)
        par = torch.empty(n, dtype=torch.int32, device=self.device) if parents else None
        B.pf_particles(self.handle, track, _ptr(st), _ptr(anc), _ptr(lw), _ptr(par),
                       C.c_void_p(self.stream.cuda_stream))
        self.stream.synchronize()
        out = dict(states=st, anc=anc, logw=lw)
        if parents:
            out["parent"] = par
        return out


def resample(logw: torch.Tensor, u: torch.Tensor, G: int, Np: int, want_q: bool = False):
    """GPU per-group systematic resampling (pf_resample) of G*Np log-weights."""
    assert logw.dtype == torch.float32 and logw.is_cuda and logw.numel() == G * Np
    assert u.dtype == torch.int32 and u.numel() == G
    dev = logw.device
    anc = torch.empty(G * Np, dtype=torch.int32, device=dev)
    q = torch.empty(G * Np, dtype=torch.int64, device=dev) if want_q else None
    nb = B.pf_resample_workspace(G, Np)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
    wp = (ws.data_ptr() + 255) // 256 * 256
    s = torch.cuda.current_stream(dev)
    B.pf_resample(_ptr(logw), _ptr(u), G, Np, _ptr(anc), _ptr(q), C.c_void_p(wp), nb, C.c_void_p(s.cuda_stream))
    B.pf_resample_check(C.c_void_p(wp), C.c_void_p(s.cuda_stream))  # waits; raises on a device-side error
    return (anc, q) if want_q else anc


class LogLikelihood(torch.autograd.Function):
    """log Z(theta) of a single-track filter run over `frames`, differentiable
    in theta = (sigma_psf, A, background, sigma_pos, sigma_v) with the
    resampling ancestry of the forward run held fixed (pf_backward).

    forward(theta (5,) tensor, pf, frames (T, H, W) CUDA tensor) sets theta,
    restarts the filter, runs the T steps and returns log Z (a 0-d float64
    tensor on the filter's device)."""

    @staticmethod
    def forward(ctx, theta, pf, frames):
        pf.set_theta(theta.detach().cpu().tolist())
        pf.reset()
        for k in range(frames.shape[0]):
            pf.step(frames[k])
        _, logz, _ = pf.estimate()
        ctx.pf = pf
        ctx.frames = frames
        ctx.theta_dtype = theta.dtype
        ctx.theta_device = theta.device
        return torch.tensor(float(logz[0]), dtype=torch.float64, device=frames.device)

    @staticmethod
    def backward(ctx, g):
        grad, _ = ctx.pf.backward([ctx.frames[k] for k in range(ctx.frames.shape[0])])
        return (g * grad[0].to(torch.float64).to(g.device)).to(ctx.theta_dtype).to(ctx.theta_device), None, None
