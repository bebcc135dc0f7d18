"""Step-by-step comparison of the GPU filter with the CPU oracle.

For every step k the oracle is given exactly what the GPU had: the
resampled population of step k-1 (X_{k-1}[anc_{k-1}]), the carried group
log-weights Lambda_{k-1}, the particles' carried within-group log-weights
(under the N_eff-threshold rule; from the GPU's FP32 log-weights), the frame,
and, for the resampler and the group reductions, the GPU's FP32
log-weights.  Integer results (ring order, N_ex,
ancestry, ancestors) must match bit for bit; real results within the
tolerance below.
"""
import numpy as np

import oracle as ora

RTOL, ATOL = 1e-5, 1e-4


def close(a, b, rtol=RTOL, atol=ATOL, scale=None):
    """|a - b| <= atol + rtol * scale elementwise (scale defaults to |b|: for a
    sum, the magnitude its FP32 rounding is relative to is that of the terms,
    which the caller passes as `scale` when it exceeds |b|)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    sc = np.abs(b) if scale is None else np.asarray(scale, np.float64)
    both_inf = np.isinf(a) & np.isinf(b) & (np.sign(a) == np.sign(b))
    return bool(np.all(both_inf | (np.abs(a - b) <= atol + rtol * sc)))


def worst(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.abs(a - b) - RTOL * np.abs(b)
    i = int(np.nanargmax(d))
    return "worst at %d: %r vs %r" % (i, a.flat[i], b.flat[i])


def run_and_compare(pf, wl, frames, truth0, steps, frames_dev, track=0, stepper=None):
    """Run `steps` GPU steps, comparing track `track` with the oracle after
    each.  stepper(k) advances the GPU filter (default: pf.step on the
    frame of step k)."""
    ocfg = ora.cfg_from_workload(wl, track=track)
    G, Np = wl.G, wl.Np
    kind, x0, lo, hi, rad = _init(wl, truth0)
    pop = ora.init_population(ocfg, kind, x0, lo, hi, rad)
    lam = None
    om = None
    prev_anc = None
    report = []
    for k in range(steps):
        if stepper is None:
            pf.step(frames_dev[k])
        else:
            stepper(k)
        p = pf.particles(track=track, parents=True)
        st = pf.stats(k, track=track)
        X = p["states"].double().cpu().numpy()
        lw = p["logw"].cpu().numpy()
        anc = p["anc"].cpu().numpy().astype(np.int64)
        par = p["parent"].cpu().numpy().astype(np.int64)
        r = ora.step(ocfg, k, frames[k], pop, lam, lw_override=lw, omega_in=om)
        assert np.array_equal(r.sigma, st["ring"]), "step %d ring %s vs %s" % (k, r.sigma, st["ring"])
        assert r.n_ex == st["n_ex"], "step %d N_ex %d vs %d" % (k, r.n_ex, st["n_ex"])
        assert abs(r.pe_eff - st["pe_eff"]) <= 1e-9 * max(1.0, abs(r.pe_eff)), "step %d PE_eff" % k
        if k > 0:
            assert np.array_equal(par, prev_anc[r.src]), "step %d ancestry" % k
        assert close(X, r.X), "step %d states: %s" % (k, worst(X, r.X))
        ll = ora.loglik_image_many(ocfg, frames[k], X)
        off = r.lw - r.loglik
        own = ll + off
        # lw = offset + l: with the frame likelihood ratio, l (up to ~10^3 at
        # the spot) and a small carried weight can nearly cancel, so the
        # rounding is relative to |l| + |offset|
        assert close(lw, own, scale=np.abs(ll) + np.abs(off)), "step %d log-weights: %s" % (k, worst(lw, own))
        want_anc = r.anc.astype(np.int64) + np.repeat(np.arange(G, dtype=np.int64) * Np, Np)
        assert np.array_equal(anc, want_anc), "step %d ancestors differ at %d slots" % (
            k, int((anc != want_anc).sum()))
        assert st["resampled"] == int(r.resampled.sum()), "step %d resampled groups %d vs %d" % (
            k, st["resampled"], int(r.resampled.sum()))
        assert close(st["logW"], r.Lambda), "step %d group log-weights: %s" % (k, worst(st["logW"], r.Lambda))
        assert close(st["group_xhat"], r.gxhat), "step %d group estimates" % k
        assert close(st["group_ess"], r.gess, rtol=1e-4, atol=1e-3), "step %d group ESS" % k
        assert close([st["log_c"]], [r.logc]), "step %d log c" % k
        assert close(st["xhat"], r.xhat), "step %d estimate" % k
        report.append(dict(k=k, n_ex=r.n_ex, pe_eff=r.pe_eff, logc=r.logc, resampled=int(r.resampled.sum())))
        pop = X[:, anc]
        lam = st["logW"]
        om = r.omega
        prev_anc = anc
    return report


def _init(wl, truth0):
    from paper_1310_4624_gb300 import synth
    kind, x0, lo, hi, rad = synth.init_arrays(wl, np.float32(truth0).astype(np.float64))
    f = lambda a: np.float32(a).astype(np.float64)  # noqa: E731
    return kind, f(x0), f(lo), f(hi), float(np.float32(rad))
