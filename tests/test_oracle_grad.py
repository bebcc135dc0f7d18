"""Pins for the oracle's gradient of log Z with frozen ancestry: replay
consistency with the oracle's own run, central finite differences of the
replayed log Z, structural zeros, and the likelihood's partial derivatives
against finite differences.  CPU only."""
import numpy as np
import pytest

from paper_1310_4624_gb300 import synth


def _setup(ora, mode=1, G=3, Np=128, T=5, init=None, seed=0):
    wl = synth.small_rna(G=G, Np=Np, mode=mode, seed=seed, data_seed=seed, T=T)
    if init is not None:
        wl = wl.replace(init=init)
    frames, truth = synth.make_sequence(wl)
    cfg = ora.cfg_from_workload(wl)
    kind, x0, lo, hi, rad = synth.init_arrays(wl, truth[0])
    pop0 = ora.init_population(cfg, kind, x0, lo, hi, rad)
    par, logc = ora.run_with_parents(cfg, pop0, frames, T)
    return wl, cfg, frames, (kind, x0, lo, hi, rad), par, logc


def test_replay_reproduces_the_run(ora):
    wl, cfg, frames, (kind, x0, lo, hi, rad), par, logc = _setup(ora)
    lz, _ = ora.replay_grad(cfg, kind, x0, frames, wl.T, par, lo, hi, rad)
    assert abs(lz - logc.sum()) <= 1e-9 * abs(lz)


def _with(cfg, ora, q, v):
    c = ora.make_cfg(G=cfg.G, Np=cfg.Np, H=cfg.H, W=cfg.W, R=cfg.R, mode=cfg.mode, sigma_psf=cfg.sigma_psf,
                     background=cfg.background, sigma_obs=cfg.sigma_obs, sigma_pos=cfg.sigma_pos,
                     sigma_v=cfg.sigma_v, sigma_I=cfg.sigma_I, ex_ratio=cfg.ex_ratio, cutoff=cfg.cutoff,
                     seed=cfg.seed, track=cfg.track)
    name = {0: "sigma_psf", 2: "background", 3: "sigma_pos", 4: "sigma_v"}[q]
    setattr(c, name, v)
    return c


@pytest.mark.parametrize("mode", [0, 1])
def test_gradient_matches_central_differences(ora, mode):
    wl, cfg, frames, (kind, x0, lo, hi, rad), par, _ = _setup(ora, mode=mode)
    lz, g = ora.replay_grad(cfg, kind, x0, frames, wl.T, par, lo, hi, rad)
    base = [cfg.sigma_psf, x0[4], cfg.background, cfg.sigma_pos, cfg.sigma_v]
    for q in range(5):
        h = 1e-5 * max(1.0, abs(base[q]))
        vals = []
        for sgn in (1, -1):
            if q == 1:
                xq = x0.copy()
                xq[4] += sgn * h
                vals.append(ora.replay_grad(cfg, kind, xq, frames, wl.T, par, lo, hi, rad)[0])
            else:
                cq = _with(cfg, ora, q, base[q] + sgn * h)
                vals.append(ora.replay_grad(cq, kind, x0, frames, wl.T, par, lo, hi, rad)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-5 * max(1.0, abs(g[q])), (ora.THETA[q], fd, g[q])


def test_structural_zeros(ora):
    wl, cfg, frames, (kind, x0, lo, hi, rad), par, _ = _setup(ora, T=1)
    _, g = ora.replay_grad(cfg, kind, x0, frames, 1, par[:1], lo, hi, rad)
    assert g[3] == 0.0 and g[4] == 0.0          # no propagation in a one-frame run
    wl, cfg, frames, (kind, x0, lo, hi, rad), par, _ = _setup(ora, init=synth.INIT_UNIFORM)
    _, g = ora.replay_grad(cfg, kind, x0, frames, wl.T, par, lo, hi, rad)
    assert g[1] == 0.0                          # A does not enter a uniform initial population


def test_likelihood_partials_match_differences(ora):
    wl = synth.small_rna()
    frames, truth = synth.make_sequence(wl, T=1)
    cfg = ora.make_cfg(G=1, Np=1, sigma_psf=1.4, sigma_obs=1.2, background=1.1)
    rng = np.random.default_rng(4)
    for (x, y, I) in [(truth[0, 0] + 0.3, truth[0, 1] - 0.2, 9.0), (1.2, 2.4, 5.0), (62.6, 30.2, 3.0)] + \
            [tuple(rng.uniform([4, 4, 1], [60, 60, 15])) for _ in range(10)]:
        l, d = ora.loglik_image_grad(cfg, frames[0], x, y, I)
        assert abs(l - ora.loglik_image(cfg, frames[0], x, y, I)) < 1e-12 * max(1, abs(l))
        h = 1e-6
        fx = (ora.loglik_image(cfg, frames[0], x + h, y, I) - ora.loglik_image(cfg, frames[0], x - h, y, I)) / (2 * h)
        fy = (ora.loglik_image(cfg, frames[0], x, y + h, I) - ora.loglik_image(cfg, frames[0], x, y - h, I)) / (2 * h)
        fI = (ora.loglik_image(cfg, frames[0], x, y, I + h) - ora.loglik_image(cfg, frames[0], x, y, I - h)) / (2 * h)
        cp, cm = _with(cfg, ora, 0, cfg.sigma_psf + h), _with(cfg, ora, 0, cfg.sigma_psf - h)
        fs = (ora.loglik_image(cp, frames[0], x, y, I) - ora.loglik_image(cm, frames[0], x, y, I)) / (2 * h)
        bp, bm = _with(cfg, ora, 2, cfg.background + h), _with(cfg, ora, 2, cfg.background - h)
        fb = (ora.loglik_image(bp, frames[0], x, y, I) - ora.loglik_image(bm, frames[0], x, y, I)) / (2 * h)
        for got, want in zip(d, (fx, fy, fI, fs, fb)):
            assert abs(got - want) <= 1e-5 * max(1.0, abs(want))


def test_fp32_state_replay(ora):
    """The FP32-state form of the replay: a one-frame run from a point whose
    components are floats already changes nothing (exactly); over a run it
    stays within a small distance of the FP64 replay, and its own finite
    differences in sigma_psf (which moves no particle) match its gradient."""
    wl, cfg, frames, (kind, x0, lo, hi, rad), par, _ = _setup(ora, T=1)
    x0f = np.float32(x0).astype(np.float64)
    a = ora.replay_grad(cfg, kind, x0f, frames, 1, par[:1], lo, hi, rad)
    b = ora.replay_grad(cfg, kind, x0f, frames, 1, par[:1], lo, hi, rad, fp32_states=True)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    wl, cfg, frames, (kind, x0, lo, hi, rad), par, _ = _setup(ora, T=6)
    lz, g = ora.replay_grad(cfg, kind, x0, frames, wl.T, par, lo, hi, rad)
    lz32, g32 = ora.replay_grad(cfg, kind, x0, frames, wl.T, par, lo, hi, rad, fp32_states=True)
    assert lz32 != lz                       # the rounding is applied
    assert abs(lz32 - lz) <= 1e-5 * abs(lz)
    assert np.all(np.abs(g32 - g) <= 1e-2 * np.abs(g) + 1e-3 * np.abs(g).max())
    h = 1e-5 * cfg.sigma_psf
    vals = [ora.replay_grad(_with(cfg, ora, 0, cfg.sigma_psf + s * h), kind, x0, frames, wl.T, par, lo, hi, rad,
                            fp32_states=True)[0] for s in (1, -1)]
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - g32[0]) <= 1e-5 * max(1.0, abs(g32[0]))


def test_replay_at_given_states(ora):
    """Given the replay's own states (rebuilt from the ancestry by the
    oracle's propagation), the replay is unchanged bit for bit; given other
    states it evaluates the likelihood there (log Z moves)."""
    wl, cfg, frames, (kind, x0, lo, hi, rad), par, _ = _setup(ora, T=5)
    N = wl.G * wl.Np
    X = [ora.init_population(cfg, kind, x0, lo, hi, rad)]
    for k in range(1, wl.T):
        X.append(ora.propagate(cfg, k, X[-1][:, par[k]]))
    states = np.stack(X)
    assert states.shape == (wl.T, 5, N)
    a = ora.replay_grad(cfg, kind, x0, frames, wl.T, par, lo, hi, rad)
    b = ora.replay_grad(cfg, kind, x0, frames, wl.T, par, lo, hi, rad, states=states)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    moved = states.copy()
    moved[2, 0] += 0.25
    c = ora.replay_grad(cfg, kind, x0, frames, wl.T, par, lo, hi, rad, states=moved)
    assert c[0] != a[0]
