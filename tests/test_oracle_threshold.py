"""Pins for the N_eff-threshold resampling variant (Alg. 1: resample when
N_eff falls below N_thresh), taken per group: the integer test against FP64
effective sample sizes, never resampling reduces to sequential importance
sampling over the particles' own trajectories (the exchange only moves
weighted particles between groups), the always-resample special case, and
the Kalman-filter limit of a linear-Gaussian variant.  CPU only."""
import math

import numpy as np
import pytest

from paper_1310_4624_gb300 import synth


def _fp64_ess(q):
    w = q.astype(np.float64)
    return w.sum() ** 2 / (w ** 2).sum()


def test_ess_test_agrees_with_fp64_effective_sample_size(ora):
    rng = np.random.default_rng(5)
    checked = 0
    for trial in range(400):
        n = int(rng.integers(1, 3000))
        spread = rng.uniform(0.0, 12.0)
        lw = (rng.normal(size=n) * spread).astype(np.float32)
        q = ora.quantize(lw)
        tau = float(rng.uniform(0.0, 1.0))
        ess = _fp64_ess(q)
        thr = ora.ess_code(tau) * n / 65536.0
        if abs(ess - thr) <= 1e-4 * thr + 1e-6:
            continue  # the codes' 2^-20 resolution may decide a near-tie either way
        assert ora.ess_test(q, tau) == (ess < thr), (n, spread, tau, ess, thr)
        checked += 1
    assert checked > 350


def test_ess_test_special_cases(ora):
    n = 1000
    flat = np.full(n, 1 << 40, np.uint64)
    assert not ora.ess_test(flat, 1.0)          # N_eff = Np is not below Np
    assert not ora.ess_test(flat, 0.5)
    one = np.zeros(n, np.uint64)
    one[17] = 1 << 40
    assert ora.ess_test(one, 0.5)               # N_eff = 1
    assert not ora.ess_test(one, 0.0)           # N_thresh = 0: never
    assert ora.ess_test(np.zeros(n, np.uint64), 0.0)  # no weight at all: the identity "resample"
    half = np.zeros(n, np.uint64)
    half[: n // 2] = 1 << 40                    # N_eff = Np / 2 exactly
    assert not ora.ess_test(half, 0.5)
    assert ora.ess_test(half, 0.5 + 2.0 ** -15)
    assert ora.ess_code(0.5) == 32768 and ora.ess_code(1.0) == 65536 and ora.ess_code(2.0) == 65536


@pytest.mark.parametrize("G, mode", [(1, synth.RNA), (4, synth.RNA), (4, synth.ARNA)])
def test_never_resampling_is_importance_sampling_over_trajectories(ora, G, mode):
    """N_thresh = 0: no group ever resamples.  The ring exchange then only
    moves weighted particles, so the filter is sequential importance
    sampling over the N trajectories: w_k(i) is proportional to the product
    of the likelihoods along slot i's trajectory, x^_k is the w-weighted
    mean and sum_k log c_k = log of the mean trajectory likelihood."""
    wl = synth.small_rna(G=G, Np=400, mode=mode, resample_rule=1, ess_fraction=0.0, ex_ratio=0.2, T=6)
    frames, truth = synth.make_sequence(wl)
    cfg = ora.cfg_from_workload(wl)
    N = wl.G * wl.Np
    pop = ora.init_population(cfg, ora.INIT_POINT, truth[0])
    pop[:2] += np.random.default_rng(3).normal(size=(2, N)) * 0.7   # distinct weights from step 0
    lam, om = None, None
    cum = np.zeros(N)
    logz = 0.0
    for k in range(wl.T):
        r = ora.step(cfg, k, frames[k], pop, lam, omega_in=om)
        if k > 0:
            cum = cum[r.src]
        cum = cum + r.loglik
        assert np.array_equal(r.anc, np.tile(np.arange(wl.Np), wl.G))
        assert not r.resampled.any()
        w = np.exp(cum - cum.max())
        w /= w.sum()
        assert np.allclose(r.xhat, r.X @ w, rtol=1e-10, atol=1e-10)
        lw_rel = r.lw - r.lw.max()
        assert np.allclose(lw_rel, cum - cum.max(), atol=1e-9)
        logz += r.logc
        want = cum.max() + math.log(np.mean(np.exp(cum - cum.max())))
        assert abs(logz - want) < 1e-9 * max(1.0, abs(want))
        pop, lam, om = r.pop_out, r.Lambda, r.omega
    if G > 1 and wl.ex_ratio > 0:
        assert r.n_ex > 0 or mode == synth.ARNA


def test_full_threshold_equals_always_resampling(ora):
    """N_thresh = Np resamples every group whose weights are not all equal:
    every group after step 0 here.  At step 0 (every particle at the truth,
    equal weights) no group resamples, and systematic resampling of equal
    weights would have been the identity: the run equals the every-step
    filter up to FP64 rounding of the carried -log Np."""
    wl = synth.small_rna(G=4, Np=512, T=5)
    frames, truth = synth.make_sequence(wl)
    a = ora.cfg_from_workload(wl)
    b = ora.cfg_from_workload(wl.replace(resample_rule=1, ess_fraction=1.0))
    pop0 = ora.init_population(a, ora.INIT_POINT, truth[0])
    ra = ora.run(a, pop0, frames, wl.T)
    rb = ora.run(b, pop0, frames, wl.T)
    assert rb.n_resampled[0] == 0 and np.all(rb.n_resampled[1:] == wl.G)
    assert np.allclose(ra.xhat, rb.xhat, rtol=1e-12, atol=1e-12)
    assert np.allclose(ra.logc, rb.logc, rtol=1e-12, atol=1e-12)
    assert np.array_equal(ra.pop_final, rb.pop_final)


def test_threshold_mixes_resampled_and_carried_groups(ora):
    """At N_thresh = Np / 2 some groups resample and others carry their
    weights; every carried group's within-group weights sum to 1."""
    wl = synth.sharing(G=8, Np=300, H=64, W=64, T=6, resample_rule=1, ess_fraction=0.5, seed=2)
    frames, truth = synth.make_sequence(wl)
    cfg = ora.cfg_from_workload(wl)
    kind, x0, lo, hi, rad = synth.init_arrays(wl, truth[0])
    pop = ora.init_population(cfg, kind, x0, lo, hi, rad)
    lam, om = None, None
    seen = set()
    for k in range(wl.T):
        r = ora.step(cfg, k, frames[k], pop, lam, omega_in=om)
        for m in range(wl.G):
            sl = slice(m * wl.Np, (m + 1) * wl.Np)
            if np.isfinite(r.Lambda[m]):
                assert abs(np.exp(r.omega[sl]).sum() - 1.0) < 1e-9
            seen.add(int(r.resampled[m]))
            if not r.resampled[m]:
                assert np.array_equal(r.anc[sl], np.arange(wl.Np))
        pop, lam, om = r.pop_out, r.Lambda, r.omega
    assert seen == {0, 1}


def test_threshold_variant_converges_to_kalman_filter(ora):
    """Point observations z = (x, y) + N(0, so^2) with N_thresh = Np / 2:
    mean -> KF mean and log Z -> KF log-likelihood, as for the every-step
    filter."""
    from test_oracle_model import _kalman
    sp, sv, so, T = 0.5, 0.1, 0.7, 12
    G, Np = 4, 8192
    cfg = ora.make_cfg(G=G, Np=Np, mode=ora.ARNA, obs_kind=ora.OBS_POINT, sigma_pos=sp, sigma_v=sv,
                       sigma_obs=so, seed=32, resample_rule=ora.RESAMPLE_ESS, ess_fraction=0.5)
    rng = np.random.default_rng(18)
    x = np.array([10.0, -4.0, 0.6, -0.3, 5.0])
    xs = [x.copy()]
    for _ in range(1, T):
        x = x.copy()
        x[0] += x[2] + sp * rng.normal()
        x[1] += x[3] + sp * rng.normal()
        x[2] += sv * rng.normal()
        x[3] += sv * rng.normal()
        xs.append(x)
    xs = np.array(xs)
    z = (xs[:, :2] + so * rng.normal(size=(T, 2))).astype(np.float32)
    pop0 = ora.init_population(cfg, ora.INIT_POINT, xs[0])
    run = ora.run(cfg, pop0, z, T)
    assert 0 < run.n_resampled[1:].sum() < G * (T - 1)   # the test decided both ways
    km, kc, kll = _kalman(z.astype(float), xs[0], sp, sv, so)
    N = G * Np
    for k in range(1, T):
        # effective sample size at most N, at least ~N/10 between resamplings
        se = math.sqrt(max(kc[k][0, 0], kc[k][1, 1]) / (N / 10))
        assert np.all(np.abs(run.xhat[k, :2] - km[k]) < 6 * se + 1e-9)
    # over seeds the error of sum log c spreads ~0.1 here; dropping the carried
    # within-group weights (omega) shifts it by ~ -1 and x^ by ~15 se
    assert abs(run.logc.sum() - kll.sum()) < 0.1 * T ** 0.5
