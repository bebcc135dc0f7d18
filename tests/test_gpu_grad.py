"""pf_backward (the adjoint of the filter step, ancestry fixed) against the
FP64 oracle's forward-mode gradient on the same ancestry, and against
central finite differences of the GPU's own replayed log Z (common random
numbers: the recorded parents and Philox streams)."""
import numpy as np
import pytest

import oracle as ora
from paper_1310_4624_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__ as ge
    ge.build()
    return torch.device("cuda:0")


def _forward(dev, wl):
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    T = wl.T
    frames, truth = synth.make_sequence(wl)
    cfg = config_from_workload(wl, truth[0], record_ancestors=True)
    pf = ParticleFilter([cfg], history=T, device=dev)
    fr = torch.from_numpy(frames).to(dev)
    parents = np.zeros((T, wl.N), np.int32)
    parents[0] = np.arange(wl.N)
    for k in range(T):
        pf.step(fr[k])
        if k > 0:
            parents[k] = pf.particles(parents=True)["parent"].cpu().numpy()
    return pf, frames, fr, truth, parents


def _oracle(wl, frames, truth, parents):
    from parity_util import _init
    kind, x0, lo, hi, rad = _init(wl, truth[0])
    return ora.replay_grad(ora.cfg_from_workload(wl), kind, x0, frames, wl.T, parents, lo, hi, rad)


CASES = [("arna", synth.small_rna(G=3, Np=256, H=48, W=48, mode=synth.ARNA, T=6)),
         ("rna", synth.small_rna(G=4, Np=200, H=40, W=56, mode=synth.RNA, T=5, seed=3, data_seed=2)),
         ("sharing", synth.sharing(G=4, Np=256, H=64, W=64, mode=synth.ARNA, T=5)),
         ("frame_model", synth.small_rna(G=3, Np=256, H=48, W=48, mode=synth.ARNA, T=5, obs_model=1))]


@pytest.mark.parametrize("name,wl", CASES, ids=[c[0] for c in CASES])
def test_gradient_matches_fp64_oracle(dev, name, wl):
    pf, frames, fr, truth, parents = _forward(dev, wl)
    grad, lz = pf.backward([fr[k] for k in range(wl.T)])
    lz_o, g_o = _oracle(wl, frames, truth, parents)
    g = grad[0].double().cpu().numpy()
    assert abs(float(lz[0]) - lz_o) <= 1e-5 * abs(lz_o), (float(lz[0]), lz_o)
    scale = np.abs(g_o).max()
    for q in range(5):
        assert abs(g[q] - g_o[q]) <= 1e-3 * abs(g_o[q]) + 1e-5 * scale, (ora.THETA[q], g[q], g_o[q])
    # the forward estimate's log Z and the replay's agree to FP32 accumulation
    _, logz_fwd, _ = pf.estimate()
    assert abs(float(logz_fwd[0]) - lz_o) <= 1e-4 * abs(lz_o)
    pf.close()


def _fd_check(dev, wl, frames, truth, params):
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    pf = ParticleFilter([config_from_workload(wl, truth[0], record_ancestors=True)], history=wl.T, device=dev)
    fr = torch.from_numpy(frames).to(dev)
    for k in range(wl.T):
        pf.step(fr[k])
    flist = [fr[k] for k in range(wl.T)]
    grad, _ = pf.backward(flist)
    g = grad[0].double().cpu().numpy()
    theta = np.array([wl.sigma_psf, float(np.float32(truth[0][4])), wl.background, wl.sigma_pos, wl.sigma_v])
    for q in params:
        h = 1e-3 * max(1.0, abs(theta[q]))
        lz = []
        for sgn in (1, -1):
            t = theta.copy()
            t[q] += sgn * h
            pf.set_theta(t)
            lz.append(float(pf.backward(flist)[1][0]))
        pf.set_theta(theta)
        fd = (lz[0] - lz[1]) / (2 * h)
        assert abs(fd - g[q]) <= 2e-2 * max(abs(g[q]), 1.0), (ora.THETA[q], fd, g[q])
    pf.close()


def test_gradient_matches_central_differences(dev):
    """sigma_psf, A and b change no particle position, so log Z is smooth in
    them with the ancestry fixed: central differences (h = 1e-3) of the
    GPU's own replay under common random numbers.  sigma_pos and sigma_v move
    particles, and a particle crossing a half-pixel boundary switches its
    likelihood patch, so log Z is only piecewise smooth in them: any step
    large enough to rise above FP32 rounding crosses boundaries.  Their GPU
    gradients are checked against the FP64 oracle's analytic gradient, which
    FP64 central differences (h = 1e-5) pin on the CPU."""
    wl = synth.small_rna(G=3, Np=256, H=48, W=48, mode=synth.ARNA, T=5)
    frames, truth = synth.make_sequence(wl)
    _fd_check(dev, wl, frames, truth, (0, 1, 2))


def test_autograd_function(dev):
    from paper_1310_4624_gb300.filter import LogLikelihood, ParticleFilter, config_from_workload
    wl = synth.small_rna(G=2, Np=256, H=48, W=48, mode=synth.ARNA, T=4)
    frames, truth = synth.make_sequence(wl)
    pf = ParticleFilter([config_from_workload(wl, truth[0], record_ancestors=True)], history=wl.T, device=dev)
    fr = torch.from_numpy(frames).to(dev)
    theta = torch.tensor([wl.sigma_psf, truth[0][4], wl.background, wl.sigma_pos, wl.sigma_v], dtype=torch.float64,
                         requires_grad=True)
    lz = LogLikelihood.apply(theta, pf, fr)
    lz.backward()
    g_direct, _ = pf.backward([fr[k] for k in range(wl.T)])
    assert torch.allclose(theta.grad, g_direct[0].double().cpu(), rtol=1e-6, atol=1e-6)
    pf.close()


def test_differentiable_workload_shape(dev):
    """The differentiable workload's shape (G=16 x 65536, 512x512) over its
    first 10 frames: FP32 accumulation in the adjoint and the atomics of
    the reverse sweep over a longer horizon.

    Against the oracle evaluated at the GPU's own FP32 states (its tangents
    in FP64 along the same ancestry and noise): every component within 1e-3
    relative.  Against the oracle's own FP64 run the states differ by FP32
    storage, and over this horizon that alone moves the gradient by ~2e-3
    (a particle within a rounding of a half-pixel boundary changes its patch
    centre, where log Z is discontinuous; the oracle with its states rounded
    to FP32 moves as much): every component within 5e-3 relative there,
    log Z within 1e-5."""
    import os
    wl = synth.differentiable(T=10)
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    frames, truth = synth.make_sequence(wl)
    pf = ParticleFilter([config_from_workload(wl, truth[0], record_ancestors=True)], history=wl.T, device=dev)
    fr = torch.from_numpy(frames).to(dev)
    parents = np.zeros((wl.T, wl.N), np.int32)
    parents[0] = np.arange(wl.N)
    states = np.zeros((wl.T, 5, wl.N), np.float64)
    for k in range(wl.T):
        pf.step(fr[k])
        p = pf.particles(parents=True)
        states[k] = p["states"].double().cpu().numpy()
        if k > 0:
            parents[k] = p["parent"].cpu().numpy()
    grad, lz = pf.backward([fr[k] for k in range(wl.T)])
    g = grad[0].double().cpu().numpy()
    from parity_util import _init
    kind, x0, lo, hi, rad = _init(wl, truth[0])
    cfg = ora.cfg_from_workload(wl)
    ora.set_threads(os.cpu_count() or 1)
    try:
        lz_o, g_o = ora.replay_grad(cfg, kind, x0, frames, wl.T, parents, lo, hi, rad)
        lz_s, g_s = ora.replay_grad(cfg, kind, x0, frames, wl.T, parents, lo, hi, rad, states=states)
    finally:
        ora.set_threads(1)
    assert abs(float(lz[0]) - lz_s) <= 1e-5 * abs(lz_s)
    assert abs(float(lz[0]) - lz_o) <= 1e-5 * abs(lz_o)
    for q in range(5):
        assert abs(g[q] - g_s[q]) <= 1e-3 * abs(g_s[q]) + 1e-5 * np.abs(g_s).max(), (ora.THETA[q], g[q], g_s[q])
        assert abs(g[q] - g_o[q]) <= 5e-3 * abs(g_o[q]) + 1e-5 * np.abs(g_o).max(), (ora.THETA[q], g[q], g_o[q])
    pf.close()
