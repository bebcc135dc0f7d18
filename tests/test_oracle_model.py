"""Pins for the oracle's model steps: Eq. 3/4 exchange count, the ring
exchange (Sec. III-A/C), NCV propagation and the Gaussian-PSF likelihood
(Sec. V), and whole-step properties (G = 1 is SIR, zero exchange decouples
groups, Kalman-filter limit on a linear-Gaussian variant).  CPU only."""
import math

import numpy as np
import pytest

from paper_1310_4624_gb300 import synth


# ------------------------------------------------------------- Eq. 3 / Eq. 4
def test_eq3_end_points_and_hand_values(ora):
    cfg = ora.make_cfg(G=4, Np=1000, mode=ora.ARNA)
    ninf = -np.inf
    assert ora.n_ex(cfg, 1, [0, 0, 0, 0]) == (0, 4.0)              # PE_eff = M -> 0
    assert ora.n_ex(cfg, 1, [0, ninf, ninf, ninf]) == (500, 1.0)   # PE_eff = 1 -> Np/2
    n, pe = ora.n_ex(cfg, 1, [0, 0, ninf, ninf])                  # PE_eff = 2
    assert pe == 2.0 and n == 333                                  # floor(1000 / 3)
    n, pe = ora.n_ex(cfg, 1, [0, math.log(0.5)] + [math.log(0.5)] * 2)
    assert abs(pe - 6.25 / 1.75) < 1e-12 and n == 71             # 0.5 - 0.5 (2.5714 / 3)
    # 99% cut-off (Sec. V-A) and its boundary
    lam = np.log([1.0, 1.0, 1.0, 0.86])
    n, pe = ora.n_ex(cfg, 1, lam)
    assert pe >= 0.99 * 4 and n == 0
    lam = np.log([1.0, 1.0, 1.0, 0.70])
    n, pe = ora.n_ex(cfg, 1, lam)
    assert pe < 0.99 * 4 and n == math.floor((0.5 - 0.5 * (pe - 1) / 3) * 1000)
    # scale invariance of PE_eff
    assert abs(ora.pe_eff([3.0, 2.0, 1.0]) - ora.pe_eff([-7.0, -8.0, -9.0])) < 1e-12
    # no exchange at k = 0 or with a single group
    assert ora.n_ex(cfg, 0, [0, ninf, ninf, ninf])[0] == 0
    assert ora.n_ex(ora.make_cfg(G=1, Np=1000, mode=ora.ARNA), 5, [0.0])[0] == 0


def test_rna_fixed_ratio(ora):
    assert ora.n_ex(ora.make_cfg(G=4, Np=1024, ex_ratio=0.1), 1, np.zeros(4))[0] == 102
    assert ora.n_ex(ora.make_cfg(G=64, Np=16384, ex_ratio=0.1), 1, np.zeros(64))[0] == 1638
    assert ora.n_ex(ora.make_cfg(G=4, Np=100, ex_ratio=0.5), 1, np.zeros(4))[0] == 50
    assert ora.n_ex(ora.make_cfg(G=4, Np=100, ex_ratio=0.0), 1, np.zeros(4))[0] == 0


# ------------------------------------------------------------------ exchange
@pytest.mark.parametrize("send_rule,topology", [(0, 0), (1, 0), (0, 1), (0, 2), (1, 2)])
@pytest.mark.parametrize("mode,G,Np,nex", [(0, 4, 50, 5), (1, 7, 33, 16), (1, 2, 10, 5), (0, 3, 8, 8)])
def test_exchange_is_a_size_and_weight_conserving_bijection(ora, mode, G, Np, nex, send_rule, topology):
    cfg = ora.make_cfg(G=G, Np=Np, mode=mode, seed=4, send_rule=send_rule, topology=topology, node_groups=3)
    N = G * Np
    pop = np.arange(5 * N, dtype=np.float64).reshape(5, N)
    for k in (1, 2, 9):
        sig = ora.ring(cfg, k)
        pr = ora.pred_topo(cfg, sig)
        out, src, org = ora.exchange(cfg, k, sig, nex, pop)
        assert np.array_equal(np.sort(src), np.arange(N))            # bijection
        assert np.array_equal(out, pop[:, src])
        for r in range(G):
            sl = slice(r * Np, (r + 1) * Np)
            recv = org[sl] != r
            assert recv.sum() == (nex if pr[r] != r else 0)           # fixed counts
            assert np.all(org[sl][recv] == pr[r])                    # from pred only
            assert np.all(src[sl][recv] // Np == pr[r])
            assert np.all(src[sl][~recv] == np.arange(r * Np, (r + 1) * Np)[~recv])
        W = np.exp(np.random.default_rng(k).normal(size=G))
        assert abs(W[org].sum() - W.sum() * Np) < 1e-9 * W.sum() * Np   # weight conserved


def test_exchange_zero_is_identity(ora):
    cfg = ora.make_cfg(G=3, Np=10)
    pop = np.random.default_rng(0).normal(size=(5, 30))
    out, src, org = ora.exchange(cfg, 4, ora.ring(cfg, 4), 0, pop)
    assert np.array_equal(out, pop) and np.array_equal(src, np.arange(30))


@pytest.mark.parametrize("send_rule", [0, 1])
def test_exchange_inclusion_probability(ora, send_rule):
    """Every slot is sent (and refilled) with probability N_ex / Np."""
    cfg = ora.make_cfg(G=2, Np=10, seed=8, send_rule=send_rule)
    nex, K = 3, 4000
    hits = np.zeros(10)
    pop = np.zeros((5, 20))
    for k in range(1, K + 1):
        _, _, org = ora.exchange(cfg, k, [0, 1], nex, pop)
        hits += org[:10] != 0
    p = nex / 10
    assert np.all(np.abs(hits / K - p) < 5 * math.sqrt(p * (1 - p) / K))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 16, 17, 100, 1000, 1024, 4097])
def test_keyed_send_permutation_is_a_bijection_with_its_inverse(ora, n):
    cfg = ora.make_cfg(G=3, Np=max(n, 1), seed=12)
    for g, k in ((0, 1), (2, 7)):
        key = ora.send_keys(cfg, g, k)
        fwd = np.array([ora.send_perm(t, n, key) for t in range(n)])
        assert np.array_equal(np.sort(fwd), np.arange(n))
        assert all(ora.send_perm_inv(int(fwd[t]), n, key) == t for t in range(n))
    assert [ora.perm_bits(v) for v in (1, 2, 3, 4, 5, 1 << 20)] == [0, 1, 2, 2, 3, 20]


def test_keyed_send_sets_are_uniform_random_subsets(ora):
    """Sec. III-C: each group randomly selects the particles it sends.  Over
    steps, the keyed send set of N_ex = 10 of 40 slots behaves as a uniform
    random subset: every slot with probability 1/4, two neighbouring slots
    together with probability 10*9/(40*39) (the systematic subsample, one slot
    in every four, never sends neighbours), and the count in the first half
    hypergeometric (mean 5, variance 10*(1/2)(1/2)(30/39))."""
    cfg = ora.make_cfg(G=1, Np=40, seed=21)
    n, m, K = 40, 10, 6000
    single = np.zeros(n)
    pairs = 0
    half = []
    for k in range(1, K + 1):
        key = ora.send_keys(cfg, 0, k)
        sent = np.zeros(n, bool)
        sent[[ora.send_perm(t, n, key) for t in range(m)]] = True
        single += sent
        pairs += int(np.sum(sent[:-1] & sent[1:]))
        half.append(int(sent[:20].sum()))
    p = m / n
    assert np.all(np.abs(single / K - p) < 5 * math.sqrt(p * (1 - p) / K))
    pp = m * (m - 1) / (n * (n - 1))
    assert abs(pairs / (K * (n - 1)) - pp) < 5 * math.sqrt(pp / (K * (n - 1))) * 2
    half = np.array(half, float)
    assert abs(half.mean() - 5.0) < 5 * math.sqrt(1.923 / K)
    assert abs(half.var() - 10 * 0.25 * 30 / 39) < 0.15


# ---------------------------------------------------------------- propagate
def test_ncv_propagation_closed_form_without_noise(ora):
    cfg = ora.make_cfg(G=2, Np=5, sigma_pos=0.0, sigma_v=0.0, sigma_I=0.0)
    pop = np.random.default_rng(1).normal(size=(5, 10)) * 3
    X = ora.propagate(cfg, 3, pop)
    want = pop.copy()
    want[0] += pop[2]      # x += vx (old velocity)
    want[1] += pop[3]
    assert np.array_equal(X, want)


def test_ncv_propagation_noise_moments(ora):
    cfg = ora.make_cfg(G=4, Np=5000, sigma_pos=0.5, sigma_v=0.1, sigma_I=0.7, seed=21)
    N = 20000
    pop = np.zeros((5, N))
    pop[2], pop[3] = 0.25, -0.5
    X = ora.propagate(cfg, 2, pop)
    inc = X - pop
    inc[0] -= 0.25
    inc[1] += 0.5
    for d, s in enumerate([0.5, 0.5, 0.1, 0.1, 0.7]):
        z = inc[d] / s
        assert abs(z.mean()) < 5 / math.sqrt(N)
        assert abs(z.var() - 1) < 5 * math.sqrt(2 / N)


# --------------------------------------------------------------- likelihood
def _separable_loglik(frame, b, spsf, sobs, R, x, y, I):
    """Expanded form: sum r^2 = sum y^2 - 2 I sum_v gy sum_u y gx + I^2 (sum gx^2)(sum gy^2),
    y = zbar - b (zero outside the image)."""
    H, W = frame.shape
    cx, cy = math.floor(x + 0.5), math.floor(y + 0.5)
    us = np.arange(cx - R, cx + R + 1)
    vs = np.arange(cy - R, cy + R + 1)
    Y = np.zeros((2 * R + 1, 2 * R + 1))
    for a, v in enumerate(vs):
        for c, u in enumerate(us):
            if 0 <= u < W and 0 <= v < H:
                Y[a, c] = float(frame[v, u]) - b
    gx = np.exp(-(us - x) ** 2 / (2 * spsf ** 2))
    gy = np.exp(-(vs - y) ** 2 / (2 * spsf ** 2))
    ss = (Y ** 2).sum() - 2 * I * gy @ Y @ gx + I ** 2 * (gx ** 2).sum() * (gy ** 2).sum()
    return -ss / (2 * sobs ** 2)


def test_likelihood_equals_separable_expansion(ora):
    wl = synth.small_rna()
    frames, truth = synth.make_sequence(wl, T=2)
    cfg = ora.make_cfg(G=1, Np=1, H=64, W=64, sigma_psf=1.5, sigma_obs=1.3, background=1.0)
    rng = np.random.default_rng(2)
    pts = [(truth[0, 0], truth[0, 1], 10.0), (0.2, 0.4, 7.0), (63.4, 62.6, 3.0), (-3.0, 30.0, 9.0),
           (30.49, 30.5, 10.0), (70.0, -8.2, 4.0)]
    pts += [tuple(rng.uniform([-5, -5, 0], [68, 68, 20])) for _ in range(50)]
    for (x, y, I) in pts:
        got = ora.loglik_image(cfg, frames[0], x, y, I)
        want = _separable_loglik(frames[0], 1.0, 1.5, 1.3, 5, x, y, I)
        assert abs(got - want) <= 1e-9 * max(1.0, abs(want))


def test_likelihood_noise_free_spot_at_truth_is_zero(ora):
    wl = synth.small_rna()
    frames, truth = synth.make_sequence(wl, noise=False, T=1)
    cfg = ora.make_cfg(G=1, Np=1)
    l = ora.loglik_image(cfg, frames[0], truth[0, 0], truth[0, 1], wl.amplitude)
    assert abs(l) < 1e-9
    assert ora.loglik_image(cfg, frames[0], truth[0, 0] + 1.0, truth[0, 1], wl.amplitude) < -1.0


def test_likelihood_off_image_closed_form(ora):
    cfg = ora.make_cfg(G=1, Np=1, sigma_psf=1.2, sigma_obs=0.8)
    frame = np.full((64, 64), 1.0, np.float32)
    x, y, I = -100.3, 20.2, 6.0
    s2 = 2 * 1.2 ** 2
    gx = np.exp(-(np.arange(-100 - 5, -100 + 6) - x) ** 2 / s2)
    gy = np.exp(-(np.arange(20 - 5, 20 + 6) - y) ** 2 / s2)
    want = -(I ** 2) * (gx ** 2).sum() * (gy ** 2).sum() / (2 * 0.8 ** 2)
    assert abs(ora.loglik_image(cfg, frame, x, y, I) - want) < 1e-9 * abs(want)
    assert math.isnan(ora.loglik_image(cfg, frame, float("nan"), 3.0, 1.0))


def _whole_frame_loglik(frame, b, spsf, sobs, R, x, y, I):
    """Gaussian log-likelihood of the whole frame under the spot model (zero
    outside the (2R+1)^2 patch) minus that of the background alone, each
    summed over every pixel of the frame (brute force; the patch must lie in
    the frame)."""
    H, W = frame.shape
    cx, cy = math.floor(x + 0.5), math.floor(y + 0.5)
    m = np.zeros((H, W))
    for v in range(cy - R, cy + R + 1):
        for u in range(cx - R, cx + R + 1):
            m[v, u] = I * math.exp(-((u - x) ** 2 + (v - y) ** 2) / (2 * spsf ** 2))
    yv = frame.astype(np.float64) - b
    return (-((yv - m) ** 2).sum() + (yv ** 2).sum()) / (2 * sobs ** 2)


def test_frame_likelihood_is_the_whole_frame_ratio(ora):
    """The frame model (Sec. II's p(z_k | x_k) of the whole image, divided by
    the background-only likelihood) restricted to the patch equals the
    brute-force sums over every pixel of the frame."""
    wl = synth.small_rna()
    frames, truth = synth.make_sequence(wl, T=1)
    cfg = ora.make_cfg(G=1, Np=1, H=64, W=64, sigma_psf=1.5, sigma_obs=1.3, background=1.0, obs_kind=ora.OBS_FRAME)
    rng = np.random.default_rng(5)
    pts = [(truth[0, 0], truth[0, 1], 10.0), (30.49, 30.5, 4.0)]
    pts += [tuple(rng.uniform([6, 6, 0], [57, 57, 20])) for _ in range(30)]
    for (x, y, I) in pts:
        got = ora.loglik_frame(cfg, frames[0], x, y, I)
        want = _whole_frame_loglik(frames[0], 1.0, 1.5, 1.3, 5, x, y, I)
        assert abs(got - want) <= 1e-9 * max(1.0, abs(want))
    # the spot outscores plain background, unlike the patch residual with
    # Poisson noise above sigma_obs at the spot
    far = ora.loglik_frame(cfg, frames[0], 5.5, 58.5, 2.0)
    assert ora.loglik_frame(cfg, frames[0], truth[0, 0], truth[0, 1], 10.0) > far + 50.0


def test_frame_likelihood_over_background_closed_form(ora):
    """On a frame that is exactly the background, y = 0 and the frame model
    reduces to -I^2 sum gx^2 sum gy^2 / (2 sigma_obs^2), on or off the frame."""
    cfg = ora.make_cfg(G=1, Np=1, sigma_psf=1.2, sigma_obs=0.8, obs_kind=ora.OBS_FRAME)
    frame = np.full((64, 64), 1.0, np.float32)
    for (x, y, I) in [(30.3, 20.2, 6.0), (-100.3, 20.2, 6.0), (2.1, 62.7, 3.0)]:
        cx, cy = math.floor(x + 0.5), math.floor(y + 0.5)
        s2 = 2 * 1.2 ** 2
        gx = np.exp(-(np.arange(cx - 5, cx + 6) - x) ** 2 / s2)
        gy = np.exp(-(np.arange(cy - 5, cy + 6) - y) ** 2 / s2)
        want = -(I ** 2) * (gx ** 2).sum() * (gy ** 2).sum() / (2 * 0.8 ** 2)
        assert abs(ora.loglik_frame(cfg, frame, x, y, I) - want) < 1e-9 * abs(want)


def test_frame_likelihood_gradient_by_differences(ora):
    """dl/d(x, y, I, sigma_psf, b) of the frame model against FP64 central
    differences of the oracle's own frame likelihood."""
    wl = synth.small_rna()
    frames, truth = synth.make_sequence(wl, T=1)
    base = dict(G=1, Np=1, H=64, W=64, sigma_psf=1.5, sigma_obs=1.1, background=1.0, obs_kind=ora.OBS_FRAME)
    cfg = ora.make_cfg(**base)
    x, y, I = truth[0, 0] + 0.3, truth[0, 1] - 0.2, 9.0
    l, d = ora.loglik_image_grad(cfg, frames[0], x, y, I)
    assert abs(l - ora.loglik_frame(cfg, frames[0], x, y, I)) < 1e-9 * abs(l)
    h = 1e-5
    fd = [(ora.loglik_frame(cfg, frames[0], x + h, y, I) - ora.loglik_frame(cfg, frames[0], x - h, y, I)) / (2 * h),
          (ora.loglik_frame(cfg, frames[0], x, y + h, I) - ora.loglik_frame(cfg, frames[0], x, y - h, I)) / (2 * h),
          (ora.loglik_frame(cfg, frames[0], x, y, I + h) - ora.loglik_frame(cfg, frames[0], x, y, I - h)) / (2 * h)]
    for key, q in (("sigma_psf", 3), ("background", 4)):
        up = ora.make_cfg(**{**base, key: base[key] + h})
        dn = ora.make_cfg(**{**base, key: base[key] - h})
        fd.append((ora.loglik_frame(up, frames[0], x, y, I) - ora.loglik_frame(dn, frames[0], x, y, I)) / (2 * h))
    for q in range(5):
        assert abs(d[q] - fd[q]) <= 1e-5 * max(1.0, abs(fd[q])), (q, d[q], fd[q])


# ------------------------------------------------------------- whole steps
def test_single_group_step_is_plain_sir(ora):
    """G = 1: the estimate and log c are those of one SIR step (Alg. 1)."""
    wl = synth.small_rna(G=1, Np=3000)
    frames, truth = synth.make_sequence(wl, T=2)
    cfg = ora.cfg_from_workload(wl)
    pop = ora.init_population(cfg, ora.INIT_POINT, truth[0])
    r0 = ora.step(cfg, 0, frames[0], pop)
    r1 = ora.step(cfg, 1, frames[1], r0.pop_out, r0.Lambda)
    assert r1.n_ex == 0
    w = np.exp(r1.loglik - r1.loglik.max())
    w /= w.sum()
    assert np.allclose(r1.xhat, r1.X @ w, rtol=1e-12, atol=1e-12)
    want_logc = np.log(np.mean(np.exp(r1.loglik - r1.loglik.max()))) + r1.loglik.max()
    assert abs(r1.logc - want_logc) < 1e-10
    assert abs(r1.gess[0] - 1.0 / (w ** 2).sum()) < 1e-6 * r1.gess[0]


def test_zero_exchange_decouples_groups(ora):
    wl = synth.small_rna(G=3, Np=500, ex_ratio=0.0)
    frames, truth = synth.make_sequence(wl, T=2)
    cfg = ora.cfg_from_workload(wl)
    pop = ora.init_population(cfg, ora.INIT_POINT, truth[0])
    pop[:, 500:1000] += 3.0           # disturb group 1 only
    a = ora.step(cfg, 1, frames[1], ora.init_population(cfg, ora.INIT_POINT, truth[0]), np.zeros(3))
    b = ora.step(cfg, 1, frames[1], pop, np.zeros(3))
    for g in (0, 2):
        sl = slice(g * 500, (g + 1) * 500)
        assert np.array_equal(a.X[:, sl], b.X[:, sl])
        assert np.array_equal(a.anc[sl], b.anc[sl])
        assert a.Lambda[g] == b.Lambda[g]
    assert not np.array_equal(a.X[:, 500:1000], b.X[:, 500:1000])


def _kalman(z, x0, sp, sv, so):
    F = np.array([[1, 0, 1, 0], [0, 1, 0, 1], [0, 0, 1, 0], [0, 0, 0, 1]], float)
    Qm = np.diag([sp ** 2, sp ** 2, sv ** 2, sv ** 2])
    Hm = np.array([[1, 0, 0, 0], [0, 1, 0, 0]], float)
    Rm = np.eye(2) * so ** 2
    m, P = np.array(x0[:4], float), np.zeros((4, 4))
    means, covs, ll = [m[:2].copy()], [P.copy()], [-float(((z[0] - m[:2]) ** 2).sum()) / (2 * so ** 2)]
    for k in range(1, len(z)):
        m, P = F @ m, F @ P @ F.T + Qm
        Sm = Hm @ P @ Hm.T + Rm
        e = z[k] - Hm @ m
        ll.append(-0.5 * e @ np.linalg.solve(Sm, e) - 0.5 * math.log(np.linalg.det(Sm)) + math.log(so ** 2))
        K = P @ Hm.T @ np.linalg.inv(Sm)
        m, P = m + K @ e, (np.eye(4) - K @ Hm) @ P
        means.append(m[:2].copy())
        covs.append(P.copy())
    return np.array(means), covs, np.array(ll)


@pytest.mark.parametrize("mode", [0, 1])
def test_linear_gaussian_variant_converges_to_kalman_filter(ora, mode):
    """Point observations z = (x, y) + N(0, so^2): mean -> KF mean, log Z -> KF
    log-likelihood (up to the constant the point likelihood leaves out)."""
    sp, sv, so, T = 0.5, 0.1, 0.7, 12
    G, Np = 4, 8192
    cfg = ora.make_cfg(G=G, Np=Np, mode=mode, obs_kind=ora.OBS_POINT, sigma_pos=sp, sigma_v=sv,
                       sigma_obs=so, seed=31)
    rng = np.random.default_rng(17)
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
    km, kc, kll = _kalman(z.astype(float), xs[0], sp, sv, so)
    N = G * Np
    for k in range(1, T):
        se = math.sqrt(max(kc[k][0, 0], kc[k][1, 1]) / (N / 3))
        assert np.all(np.abs(run.xhat[k, :2] - km[k]) < 6 * se + 1e-9)
    assert abs(run.logc.sum() - kll.sum()) < 0.05 * T ** 0.5


def test_small_workload_tracks_the_spot(ora):
    wl = synth.small_rna()
    frames, truth = synth.make_sequence(wl)
    cfg = ora.cfg_from_workload(wl)
    pop0 = ora.init_population(cfg, ora.INIT_POINT, truth[0])
    run = ora.run(cfg, pop0, frames, wl.T)
    assert run.failed_step == -1
    err = np.sqrt(((run.xhat[:, :2] - truth[:, :2]) ** 2).sum(1).mean())
    assert err < 0.5
    assert np.all(run.n_ex[1:] == 102) and run.n_ex[0] == 0


def test_multi_object_track_follows_its_own_spot(ora):
    """Several spots in one frame, one filter per spot: the oracle filter
    started at a spot follows it (the other spots lie outside its patches)."""
    wls = synth.multi_object(n_obj=4, G=2, Np=400, H=128, W=128, T=8, cell=64)
    frames, truths = synth.make_multi_sequence(wls)
    for t in (0, 3):
        cfg = ora.cfg_from_workload(wls[t])
        pop0 = ora.init_population(cfg, ora.INIT_POINT, truths[t][0])
        run = ora.run(cfg, pop0, frames, wls[t].T)
        err = np.sqrt(((run.xhat[:, :2] - truths[t][:, :2]) ** 2).sum(1).mean())
        assert err < 0.6, (t, err)
    d = min(np.hypot(*(truths[i, k, :2] - truths[j, k, :2])) for i in range(4) for j in range(i) for k in range(8))
    assert d > 2 * (2 * 5 + 1)


def test_init_samplers_ranges(ora):
    wl = synth.sharing(G=4, Np=2000, H=64, W=64)
    cfg = ora.cfg_from_workload(wl)
    x0 = np.array([30.0, 20.0, 0.5, -0.5, 10.0])
    kind, _, lo, hi, rad = synth.init_arrays(wl, x0)
    pop = ora.init_population(cfg, kind, x0, lo, hi, rad)
    g0 = pop[:, :2000]
    r = np.hypot(g0[0] - 30, g0[1] - 20)
    assert r.max() <= 2.0 and abs((r ** 2).mean() - 2.0) < 0.1      # uniform in the disc: E r^2 = R^2/2
    assert np.all(g0[2] == 0.5) and np.all(g0[4] == 10.0)
    rest = pop[:, 2000:]
    for d in range(5):
        assert lo[d] <= rest[d].min() and rest[d].max() <= hi[d]
        assert abs(rest[d].mean() - (lo[d] + hi[d]) / 2) < 0.05 * (hi[d] - lo[d])


def test_init_samplers_follow_their_distributions(ora):
    """Kolmogorov-Smirnov against the exact laws: uniform components in the
    box (INIT_UNIFORM, and the groups >= 1 of INIT_SHARING); in group 0's
    disc, (r / R)^2 and the angle uniform on [0, 1) and [0, 2 pi), r and the
    angle independent; POINT puts every particle at x0."""
    stats = pytest.importorskip("scipy.stats")
    wl = synth.sharing(G=3, Np=20000, H=64, W=64, seed=17)
    cfg = ora.cfg_from_workload(wl)
    x0 = np.array([30.0, 20.0, 0.5, -0.5, 10.0])
    kind, _, lo, hi, rad = synth.init_arrays(wl, x0)
    pop = ora.init_population(cfg, kind, x0, lo, hi, rad)
    g0 = pop[:, :20000]
    r2 = ((g0[0] - 30) ** 2 + (g0[1] - 20) ** 2) / rad ** 2
    th = np.mod(np.arctan2(g0[1] - 20, g0[0] - 30), 2 * np.pi) / (2 * np.pi)
    assert stats.kstest(r2, "uniform").pvalue > 1e-3
    assert stats.kstest(th, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(r2, th)[0, 1]) < 0.03
    rest = pop[:, 20000:]
    for d in range(5):
        assert stats.kstest((rest[d] - lo[d]) / (hi[d] - lo[d]), "uniform").pvalue > 1e-3, d
    c = np.corrcoef(rest)
    assert np.all(np.abs(c - np.eye(5)) < 0.03)
    pt = ora.init_population(cfg, ora.INIT_POINT, x0)
    assert np.array_equal(pt, np.repeat(x0[:, None], pt.shape[1], axis=1))


@pytest.mark.parametrize("mode", [0, 1])
def test_exchange_preserves_the_weighted_population(ora, mode):
    """Exchanged particles carry their origin group's weight (Alg. 2/3 steps
    3-4), so with a flat likelihood and no motion the weighted estimate after
    the exchange is the pre-exchange mixture sum_g W_g mean(pop_g) / sum W."""
    G, Np = 5, 200
    cfg = ora.make_cfg(G=G, Np=Np, mode=mode, obs_kind=ora.OBS_POINT, sigma_obs=1e7, sigma_pos=0.0,
                       sigma_v=0.0, sigma_I=0.0, ex_ratio=0.3, seed=2)
    rng = np.random.default_rng(9)
    pop = rng.normal(size=(5, G * Np)) * 10
    pop[2:4] = 0.0
    Lam = np.log(rng.uniform(0.05, 1.0, size=G))
    r = ora.step(cfg, 1, np.zeros(2, np.float32), pop, Lam)
    assert r.n_ex > 0
    W = np.exp(Lam - Lam.max())
    want = sum(W[g] * pop[:, g * Np:(g + 1) * Np].mean(1) for g in range(G)) / W.sum()
    assert np.allclose(r.xhat, want, rtol=1e-9, atol=1e-9)
