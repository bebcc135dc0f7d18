"""The identity the lean resampler builds on (Alg. 3 step 7): with S_i the
sum of the weight codes before item i and T_j the integer thresholds of
systematic resampling, item i takes the outputs O_i .. O_{i+1} - 1 where
O_i = #{j : T_j < S_i}.  Writing i + 1 at position O_i of every item with
outputs (and at the first position of every chunk its range covers), then
taking a running maximum over each chunk's positions, gives every output
its item.  Checked on the CPU against the oracle's resampling, with the
kernel's threshold constants (T_j = j A + F1 + floor((j B + F0) / Np) for
Q = A Np + B, F = floor(u Q / 2^32) = F1 Np + F0), on the cluster chunking
the kernel uses and on degenerate, tied and ragged inputs."""
import numpy as np
import pytest

import oracle as ora


def _thresholds(Q, Np, u):
    A, B = divmod(Q, Np)
    F = (u * Q) >> 32
    F1, F0 = divmod(F, Np)
    j = np.arange(Np, dtype=object)
    return np.array([jj * A + F1 + (jj * B + F0) // Np for jj in j], dtype=object)


def _marking(q, u, C):
    Np = len(q)
    Q = int(sum(int(x) for x in q))
    T = _thresholds(Q, Np, u)
    S = np.concatenate([[0], np.cumsum(np.array([int(x) for x in q], dtype=object))])
    # O_i = #{j : T_j < S_i}: T is nondecreasing
    O = np.array([int(np.searchsorted(T.astype(float), float(s), side="left")) for s in S])
    # exact correction of the float search (T and S are integers beyond 2^53)
    for i, s in enumerate(S):
        c = O[i]
        while c < Np and T[c] < s:
            c += 1
        while c > 0 and T[c - 1] >= s:
            c -= 1
        O[i] = c
    chunk = ((Np + C - 1) // C + 7) & ~7
    marks = np.zeros(C * chunk, np.int64)
    for i in range(Np):
        if O[i + 1] > O[i]:
            assert marks[O[i]] == 0
            marks[O[i]] = i + 1
            b = O[i] // chunk + 1
            while b * chunk < O[i + 1]:
                assert marks[b * chunk] == 0
                marks[b * chunk] = i + 1
                b += 1
    anc = np.zeros(Np, np.int64)
    for r in range(C):
        lo, hi = r * chunk, min((r + 1) * chunk, Np)
        if lo >= hi:
            continue
        run = np.maximum.accumulate(marks[lo:hi])
        assert run[0] > 0  # every chunk's first position is marked
        anc[lo:hi] = run - 1
    return anc


CASES = [(1, 1, "normal"), (7, 1, "normal"), (300, 2, "wide"), (1000, 4, "special"), (4097, 2, "ties"),
         (5000, 8, "dominant"), (2049, 3, "normal"), (64, 4, "wide")]


@pytest.mark.parametrize("Np,C,kind", CASES)
def test_marking_reproduces_oracle_resampling(Np, C, kind):
    rng = np.random.default_rng(Np * 31 + C)
    lw = (rng.normal(size=Np) * 4.0 - 300.0).astype(np.float32)
    if kind == "wide":
        lw = rng.uniform(-60.0, 0.0, size=Np).astype(np.float32)
    elif kind == "special":
        lw[rng.integers(0, Np, size=max(1, Np // 7))] = np.nan
        lw[: Np // 3] = -np.inf
    elif kind == "ties":
        lw = np.round(rng.normal(size=Np)).astype(np.float32)
    elif kind == "dominant":
        lw[:] = -50.0
        lw[Np // 2] = 0.0
    q = ora.quantize(lw)
    if int(q.sum()) == 0:
        pytest.skip("no finite weight")
    for u in (0, 1, int(rng.integers(0, 2 ** 32)), 2 ** 32 - 1):
        want = ora.resample(q, u)
        got = _marking(q, u, C)
        assert np.array_equal(got, want), (Np, C, kind, u, int((got != want).sum()))
