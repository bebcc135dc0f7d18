"""Seeded synthetic inputs: workload presets and spot-tracking image sequences.

This module is the one piece shared by the CUDA path's tests/benchmark and the
CPU oracle.  It holds no filter arithmetic: it renders frames and ground truth
and names the parameter sets.  The paper's own ten 512x512 sequences are not
available; these stand in for them with the appearance model the paper
describes (Sec. V, Fig. 1): a small isotropic Gaussian spot of amplitude A on
background b, Poisson noise, moving under constant velocity.

Recipe (all draws from ``numpy.random.default_rng(data_seed)``):
  * start position uniform in the central region [H/4, 3H/4) x [W/4, 3W/4)
    (64x64 frames: [16, 48)^2, the central 32x32);
  * velocity uniform in [-vmax, vmax]^2, redrawn until the whole track stays at
    least ``margin`` px inside the frame;
  * with ``truth_noise`` (the differentiable workload, whose data come from
    the model at the true parameters): the truth follows the nearly-constant-
    velocity dynamics itself, x_{k+1} = x_k + v_k + sigma_pos eps,
    v_{k+1} = v_k + sigma_v eps, intensity constant at the amplitude; the
    whole trajectory is redrawn until it keeps the margin;
  * frame k: z(u, v) ~ Poisson(b + A exp(-((u - x_k)^2 + (v - y_k)^2) / (2 s^2)))
    as float32, pixel (u, v) = (column, row) centred at integer coordinates.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

RNA, ARNA = 0, 1
INIT_POINT, INIT_UNIFORM, INIT_SHARING = 0, 1, 2


@dataclasses.dataclass
class Workload:
    """Parameters of one tracking workload (one track)."""
    name: str
    G: int
    Np: int
    H: int
    W: int
    T: int
    mode: int = RNA
    sigma_psf: float = 1.5
    amplitude: float = 10.0
    background: float = 1.0
    sigma_obs: float = 1.0
    sigma_pos: float = 0.5
    sigma_v: float = 0.1
    sigma_I: float = 0.5
    ex_ratio: float = 0.10
    pe_eff_cutoff: float = 0.99
    patch_radius: int = 5
    seed: int = 0          # Philox key of the filter
    data_seed: int = 0     # numpy seed of the sequence
    init: int = INIT_POINT
    vmax: float = 1.0
    margin: float = 6.0
    share_radius: float = 2.0     # information-sharing init: disc radius of group 0
    share_vmax: float = 2.0       # other groups: velocity range
    share_I: Tuple[float, float] = (1.0, 20.0)
    truth_noise: bool = False     # truth drawn from the NCV dynamics (sigma_pos, sigma_v)
    obs_model: int = 0            # 0: patch residual, 1: frame likelihood ratio
    resample_rule: int = 0        # 0: every step (Alg. 2/3), 1: when N_eff < ess_fraction Np (Alg. 1)
    ess_fraction: float = 0.5
    send_rule: int = 0            # 0: systematic slot subsample, 1: keyed random permutation (Sec. III-C)
    topology: int = 0             # 0: ring (Sec. IV-B), 1: node-aware ring, 2: hypercube (Sec. VI)
    node_groups: int = 1          # topology 1: groups per node
    cell: float = 0.0             # multi-object sequences: the spot's grid cell (size, origin)
    cell_x: float = 0.0
    cell_y: float = 0.0

    @property
    def N(self) -> int:
        return self.G * self.Np

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def small_rna(**kw) -> Workload:
    """One 20-frame 64x64 track, G=4 x 1024, RNA 10% on the fixed ring."""
    return Workload(name="small_rna_64x64_G4x1024", G=4, Np=1024, H=64, W=64, T=20, mode=RNA).replace(**kw)


def tracking(mode: int = ARNA, **kw) -> Workload:
    """100 frames 512x512, G=64 x 16384 (1,048,576 particles), init at the truth."""
    name = "tracking_512x512_G64x16384_" + ("arna" if mode == ARNA else "rna10")
    return Workload(name=name, G=64, Np=16384, H=512, W=512, T=100, mode=mode).replace(**kw)


def sharing(mode: int = ARNA, **kw) -> Workload:
    """100 frames 512x512, G=256 x 4096; group 0 near the truth, the rest uniform."""
    name = "sharing_512x512_G256x4096_" + ("arna" if mode == ARNA else "rna10")
    return Workload(name=name, G=256, Np=4096, H=512, W=512, T=100, mode=mode,
                    init=INIT_SHARING).replace(**kw)


def differentiable(**kw) -> Workload:
    """50 frames 512x512, G=16 x 65536, ARNA."""
    return Workload(name="grad_512x512_G16x65536", G=16, Np=65536, H=512, W=512, T=50,
                    mode=ARNA, truth_noise=True).replace(**kw)


def batched_tracks(n_tracks: int = 512, seed: int = 0, H: int = 256, W: int = 256, T: int = 50,
                   n_range=(4096, 262144), g_range=(4, 128)) -> List[Workload]:
    """Independent tracks with log-uniform particle and group counts; N_t is
    rounded down to a multiple of G_t."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(n_tracks):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        g = int(round(math.exp(rng.uniform(math.log(g_range[0]), math.log(g_range[1])))))
        amp = float(rng.uniform(5.0, 20.0))
        spsf = float(rng.uniform(1.2, 2.0))
        out.append(Workload(name="batched_%d" % t, G=g, Np=max(1, n // g), H=H, W=W, T=T, mode=ARNA,
                            sigma_psf=spsf, amplitude=amp, seed=seed, data_seed=1000 + t))
    return out


def truth_track(wl: Workload) -> np.ndarray:
    """Ground truth (T, 5): x, y, vx, vy, I with constant velocity."""
    rng = np.random.default_rng(wl.data_seed)
    H, W, T = wl.H, wl.W, wl.T
    x0 = rng.uniform(W / 4, 3 * W / 4)
    y0 = rng.uniform(H / 4, 3 * H / 4)
    if wl.truth_noise:
        for _ in range(10000):
            v = rng.uniform(-wl.vmax, wl.vmax, size=2)
            p = np.array([x0, y0])
            tr = np.zeros((T, 5))
            for k in range(T):
                tr[k, :2], tr[k, 2:4], tr[k, 4] = p, v, wl.amplitude
                p = p + v + wl.sigma_pos * rng.standard_normal(2)
                v = v + wl.sigma_v * rng.standard_normal(2)
            if (tr[:, 0].min() >= wl.margin and tr[:, 0].max() <= W - 1 - wl.margin and
                    tr[:, 1].min() >= wl.margin and tr[:, 1].max() <= H - 1 - wl.margin):
                return tr
        raise RuntimeError("no NCV trajectory kept the margin")  # pragma: no cover
    for _ in range(10000):
        vx, vy = rng.uniform(-wl.vmax, wl.vmax, size=2)
        xs = x0 + vx * np.arange(T)
        ys = y0 + vy * np.arange(T)
        if (xs.min() >= wl.margin and xs.max() <= W - 1 - wl.margin and
                ys.min() >= wl.margin and ys.max() <= H - 1 - wl.margin):
            break
    else:  # pragma: no cover - the central start always admits small velocities
        vx = vy = 0.0
        xs = np.full(T, x0)
        ys = np.full(T, y0)
    tr = np.zeros((T, 5))
    tr[:, 0], tr[:, 1], tr[:, 2], tr[:, 3], tr[:, 4] = xs, ys, vx, vy, wl.amplitude
    return tr


def render(wl: Workload, truth: np.ndarray, rng: np.random.Generator, noise: bool = True) -> np.ndarray:
    """Frames (T, H, W) float32 of the spot along ``truth``."""
    T = truth.shape[0]
    u = np.arange(wl.W, dtype=np.float64)
    v = np.arange(wl.H, dtype=np.float64)
    frames = np.empty((T, wl.H, wl.W), np.float32)
    s2 = 2.0 * wl.sigma_psf ** 2
    for k in range(T):
        gx = np.exp(-(u - truth[k, 0]) ** 2 / s2)
        gy = np.exp(-(v - truth[k, 1]) ** 2 / s2)
        lam = wl.background + truth[k, 4] * np.outer(gy, gx)
        frames[k] = rng.poisson(lam).astype(np.float32) if noise else lam.astype(np.float32)
    return frames


def multi_object(n_obj: int = 16, G: int = 16, Np: int = 4096, H: int = 256, W: int = 256, T: int = 30,
                 mode: int = ARNA, seed: int = 0, data_seed: int = 0, cell: int = 64, vmax: float = 0.25,
                 **kw) -> List[Workload]:
    """Several spots in one sequence, one filter (track) per spot: spot i
    starts at a seeded point of cell i of a grid of cell x cell pixel cells
    (at least 14 px from the cell's edges) and drifts at constant velocity
    of at most vmax px per frame, so patches of different spots stay apart
    over T frames.  Every workload shares the frames (make_multi_sequence)."""
    cols = W // cell
    assert n_obj <= cols * (H // cell), "the frame holds fewer cells than spots"
    return [Workload(name="multi_object_%dx%d_%dspots_G%dx%d" % (H, W, n_obj, G, Np), G=G, Np=Np, H=H, W=W, T=T,
                     mode=mode, seed=seed, data_seed=data_seed * 1000 + i, vmax=vmax, cell=float(cell),
                     cell_x=float(cell * (i % cols)), cell_y=float(cell * (i // cols))).replace(**kw)
            for i in range(n_obj)]


def make_multi_sequence(wls: List[Workload], noise: bool = True):
    """(frames (T, H, W) float32 holding every spot, truths (n, T, 5)) for
    multi_object workloads: each spot starts uniformly in its cell, at least
    (14 + vmax T) px from the cell's edges."""
    wl0 = wls[0]
    truths = []
    for wl in wls:
        rng = np.random.default_rng(wl.data_seed)
        m = 14.0 + wl.vmax * wl.T
        assert wl.cell > 2 * m, "cells too small for the drift"
        x0 = wl.cell_x + rng.uniform(m, wl.cell - m)
        y0 = wl.cell_y + rng.uniform(m, wl.cell - m)
        vx, vy = rng.uniform(-wl.vmax, wl.vmax, size=2)
        tr = np.zeros((wl.T, 5))
        tr[:, 0] = x0 + vx * np.arange(wl.T)
        tr[:, 1] = y0 + vy * np.arange(wl.T)
        tr[:, 2], tr[:, 3], tr[:, 4] = vx, vy, wl.amplitude
        truths.append(tr)
    truths = np.array(truths)
    u = np.arange(wl0.W, dtype=np.float64)
    v = np.arange(wl0.H, dtype=np.float64)
    s2 = 2.0 * wl0.sigma_psf ** 2
    rng = np.random.default_rng([wl0.data_seed, 7])
    frames = np.empty((wl0.T, wl0.H, wl0.W), np.float32)
    for k in range(wl0.T):
        lam = np.full((wl0.H, wl0.W), wl0.background)
        for tr in truths:
            lam += tr[k, 4] * np.outer(np.exp(-(v - tr[k, 1]) ** 2 / s2), np.exp(-(u - tr[k, 0]) ** 2 / s2))
        frames[k] = rng.poisson(lam).astype(np.float32) if noise else lam.astype(np.float32)
    return frames, truths


def make_sequence(wl: Workload, noise: bool = True, T: Optional[int] = None):
    """(frames (T, H, W) float32, truth (T, 5) float64) for a workload."""
    if T is not None:
        wl = wl.replace(T=T)
    truth = truth_track(wl)
    rng = np.random.default_rng([wl.data_seed, 1])
    return render(wl, truth, rng, noise=noise), truth


def init_arrays(wl: Workload, truth0: np.ndarray):
    """(kind, x0[5], lo[5], hi[5], radius) of the initial population.

    POINT: every particle at the truth (tracking mode, Sec. V).  SHARING:
    group 0 in a disc of ``share_radius`` around the truth with the true
    velocity and intensity; the other groups uniform over the image, with
    velocity in [-share_vmax, share_vmax]^2 and intensity in ``share_I``
    (information-sharing mode, Sec. V).
    """
    x0 = np.array(truth0, np.float64)
    lo = np.array([0.0, 0.0, -wl.share_vmax, -wl.share_vmax, wl.share_I[0]])
    hi = np.array([wl.W - 1.0, wl.H - 1.0, wl.share_vmax, wl.share_vmax, wl.share_I[1]])
    return wl.init, x0, lo, hi, wl.share_radius


def render_batched_torch(wls: List[Workload], device, seed: int = 0):
    """Frames (n_tracks, T, H, W) float32 on `device` and truths (n_tracks, T,
    5) for equally sized tracks, drawn with torch's seeded generator on the
    device (large batched workloads; the same spot model as ``render``)."""
    import torch
    n, T, H, W = len(wls), wls[0].T, wls[0].H, wls[0].W
    truths = np.stack([truth_track(wl) for wl in wls])
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    u = torch.arange(W, dtype=torch.float32, device=device)
    v = torch.arange(H, dtype=torch.float32, device=device)
    frames = torch.empty((n, T, H, W), dtype=torch.float32, device=device)
    tr = torch.from_numpy(truths).to(device=device, dtype=torch.float32)
    s2 = torch.tensor([2.0 * wl.sigma_psf ** 2 for wl in wls], dtype=torch.float32, device=device)
    bg = torch.tensor([wl.background for wl in wls], dtype=torch.float32, device=device)
    for k in range(T):
        gx = torch.exp(-(u[None, :] - tr[:, k, 0:1]) ** 2 / s2[:, None])
        gy = torch.exp(-(v[None, :] - tr[:, k, 1:2]) ** 2 / s2[:, None])
        lam = bg[:, None, None] + tr[:, k, 4][:, None, None] * gy[:, :, None] * gx[:, None, :]
        frames[:, k] = torch.poisson(lam, generator=gen)
    return frames, truths
