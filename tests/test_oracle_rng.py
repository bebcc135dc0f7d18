"""Pins for the oracle's random streams: Philox4x32-10, the uniform map,
Box-Muller normals, Lemire bounded integers and the Fisher-Yates ring
(Sec. IV-B, Alg. 3 step 1).  CPU only."""
import math
import os
import subprocess

import numpy as np
import pytest
from scipy import stats

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def torch_philox(tmp_path_factory):
    """PyTorch's header-only at::philox_engine compiled into a tiny probe."""
    import torch.utils.cpp_extension as ce
    exe = str(tmp_path_factory.mktemp("philox") / "probe")
    inc = sum((["-I", p] for p in ce.include_paths()), [])
    subprocess.run(["g++", "-std=c++17", "-O1", *inc, "-o", exe,
                    os.path.join(HERE, "philox_torch_probe.cpp")], check=True)
    return exe


def test_philox_matches_torch_engine(ora, torch_philox):
    rng = np.random.default_rng(7)
    quads = rng.integers(0, 2 ** 32, size=(300, 6), dtype=np.uint64)
    quads[0] = 0
    quads[1] = 2 ** 32 - 1
    quads[2, 2:] = [0, 0, 5, (3 << 8) | (1 << 4) | 1]   # a typical stream counter
    text = "\n".join(" ".join(str(int(v)) for v in row) for row in quads) + "\n"
    out = subprocess.run([torch_philox], input=text, capture_output=True, text=True, check=True).stdout
    lines = out.strip().splitlines()
    assert len(lines) == len(quads)
    for row, line in zip(quads, lines):
        seed = int(row[0]) | (int(row[1]) << 32)
        ours = ora.philox(seed, row[2:6].astype(np.uint32))
        assert [int(v) for v in ours] == [int(v) for v in line.split()]


def test_philox_known_answer_vectors(ora):
    """The generator's published known-answer vectors (tests/golden, cited
    there): counter, key and the 10-round output."""
    rows = [line.split() for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        ctr, (k0, k1), want = v[0:4], v[4:6], v[6:10]
        ours = ora.philox(k0 | (k1 << 32), np.array(ctr, dtype=np.uint32))
        assert [int(x) for x in ours] == want


def test_uniform_map_open_interval_and_fp32_exact(ora):
    for w in [0, 1, 255, 256, 2 ** 31, 2 ** 32 - 257, 2 ** 32 - 1]:
        u = ora.uniform(w)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u  # exactly representable in FP32
    assert ora.uniform(0) == 0.5 / 2 ** 23
    assert ora.uniform(2 ** 32 - 1) == 1.0 - 0.5 / 2 ** 23
    # monotone in the top 23 bits, constant in the low 9
    assert ora.uniform(0x12345600) == ora.uniform(0x123457FF) < ora.uniform(0x12345800)
    # mean of the 2^23 cell centres is exactly 1/2
    assert sum(ora.uniform(m << 9) for m in (0, 2 ** 23 - 1)) == 1.0


def test_box_muller_normals_moments_and_ks(ora):
    cfg = ora.make_cfg(G=1, Np=1, seed=12345)
    n = 40000
    e = np.array([ora.normals(cfg, 3, j, 9) for j in range(n)])  # (n, 5)
    for d in range(5):
        x = e[:, d]
        assert abs(x.mean()) < 5 / math.sqrt(n)
        assert abs(x.var() - 1.0) < 5 * math.sqrt(2.0 / n)
        assert stats.kstest(x, "norm").pvalue > 1e-4
    c = np.corrcoef(e.T)
    assert np.all(np.abs(c[np.triu_indices(5, 1)]) < 5 / math.sqrt(n))
    # distinct (group, step, seed) give distinct draws
    assert not np.allclose(ora.normals(cfg, 3, 0, 9), ora.normals(cfg, 4, 0, 9))
    assert not np.allclose(ora.normals(cfg, 3, 0, 9), ora.normals(cfg, 3, 0, 10))


@pytest.mark.parametrize("s", [3, 1000003])
def test_lemire_bounded_exactly_uniform_over_all_words(ora, s, tmp_path):
    """Over all 2^32 words every value in [0, s) is hit equally often and
    exactly 2^32 mod s words are rejected (enumerated in C)."""
    from oracle import build as obuild
    exe = str(tmp_path / "lemire_enum")
    subprocess.run(["gcc", "-O2", "-o", exe, os.path.join(HERE, "lemire_enum.c"), obuild.LIB,
                    "-Wl,-rpath," + os.path.dirname(obuild.LIB)], check=True)
    mn, mx, rej = map(int, subprocess.run([exe, str(s)], capture_output=True, text=True,
                                          check=True).stdout.split())
    assert mn == mx == ((1 << 32) - rej) // s
    assert rej == (1 << 32) % s


def test_fisher_yates_is_a_bijection_onto_all_permutations(ora):
    import itertools
    for G in (1, 2, 3, 4, 5):
        perms = set()
        for r in itertools.product(*[range(j + 1) for j in range(1, G)]):
            sig = ora.fisher_yates([0, *r])
            assert sorted(sig) == list(range(G))
            perms.add(tuple(sig))
        assert len(perms) == math.factorial(G)


def test_arna_ring_uniform_over_permutations(ora):
    cfg = ora.make_cfg(G=3, Np=4, mode=ora.ARNA, seed=99)
    K = 6000
    seen = {}
    for k in range(1, K + 1):
        s = tuple(ora.ring(cfg, k))
        seen[s] = seen.get(s, 0) + 1
    assert len(seen) == 6
    chi2 = stats.chisquare(list(seen.values()))
    assert chi2.pvalue > 1e-4


def test_rna_ring_is_the_fixed_ring(ora):
    cfg = ora.make_cfg(G=5, Np=4, mode=ora.RNA)
    for k in (0, 1, 7):
        assert list(ora.ring(cfg, k)) == [0, 1, 2, 3, 4]
    # P_m receives from P_{m-1}
    assert list(ora.pred(ora.ring(cfg, 3))) == [4, 0, 1, 2, 3]
    arna = ora.make_cfg(G=5, Np=4, mode=ora.ARNA)
    assert list(ora.ring(arna, 0)) == [0, 1, 2, 3, 4]   # no exchange at k = 0


def test_pred_inverts_the_ring(ora):
    cfg = ora.make_cfg(G=9, Np=4, mode=ora.ARNA, seed=3)
    for k in range(1, 20):
        s = ora.ring(cfg, k)
        p = ora.pred(s)
        succ = {int(s[i]): int(s[(i + 1) % 9]) for i in range(9)}
        for g in range(9):
            assert succ[int(p[g])] == g
