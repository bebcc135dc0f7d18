"""GPU resampler (pf_resample, the kernel pf_step uses) against the oracle:
weight codes and ancestors bit-exact, on ragged, multi-CTA-cluster and
degenerate inputs."""
import numpy as np
import pytest

import oracle as ora

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def _weights(kind, G, Np, rng):
    lw = (rng.normal(size=(G, Np)) * 4.0 - 300.0).astype(np.float32)
    if kind == "wide":
        lw = rng.uniform(-60.0, 0.0, size=(G, Np)).astype(np.float32)
    elif kind == "special":
        lw[0, :] = -np.inf                                    # a degenerate group
        if G > 1:
            lw[1, rng.integers(0, Np, size=max(1, Np // 7))] = np.nan
        if G > 2:
            lw[2, :] = -50.0
            lw[2, Np // 2] = 0.0                              # one dominant particle
        if G > 3:
            lw[3, :] = 1.25                                   # all equal
    elif kind == "ties":
        lw = np.round(rng.normal(size=(G, Np))).astype(np.float32)
    return lw


CASES = [(1, 1, "normal"), (3, 2, "normal"), (4, 1000, "special"), (2, 4095, "wide"), (2, 4096, "normal"),
         (2, 4097, "ties"), (5, 16384, "normal"), (4, 16384, "special"), (2, 65536, "wide"),
         (1, 131072, "normal"), (1, 200003, "wide"), (64, 16384, "normal"), (256, 4096, "special"),
         (1, 1 << 20, "wide"), (4, 1 << 20, "special")]


@pytest.mark.parametrize("G,Np,kind", CASES)
def test_resample_matches_oracle_bit_exact(dev, G, Np, kind):
    from paper_1310_4624_gb300.filter import resample
    rng = np.random.default_rng(G * 7919 + Np)
    lw = _weights(kind, G, Np, rng)
    u = rng.integers(0, 2 ** 32, size=G, dtype=np.uint64).astype(np.uint32)
    anc, q = resample(torch.from_numpy(lw.ravel()).to(dev), torch.from_numpy(u.view(np.int32)).to(dev), G, Np,
                      want_q=True)
    anc = anc.cpu().numpy().reshape(G, Np)
    q = q.cpu().numpy().view(np.uint64).reshape(G, Np)
    for g in range(G):
        qo = ora.quantize(lw[g])
        assert np.array_equal(q[g], qo), "group %d: %d codes differ" % (g, int((q[g] != qo).sum()))
        ao = ora.resample(qo, int(u[g]))
        assert np.array_equal(anc[g], ao), "group %d: %d ancestors differ" % (g, int((anc[g] != ao).sum()))


def test_resample_repeated_calls_are_deterministic(dev):
    from paper_1310_4624_gb300.filter import resample
    rng = np.random.default_rng(3)
    lw = torch.from_numpy(_weights("wide", 8, 20000, rng).ravel()).to(dev)
    u = torch.from_numpy(rng.integers(0, 2 ** 31, size=8).astype(np.int32)).to(dev)
    a = resample(lw, u, 8, 20000)
    b = resample(lw, u, 8, 20000)
    assert torch.equal(a, b)


@pytest.mark.parametrize("G,Np,kind", CASES)
def test_resample_without_codes_matches_oracle_bit_exact(dev, G, Np, kind):
    """Without codes to return, groups whose chunks fit a CTA's registers run
    the lean instance (ancestors by marking each item's first output and a
    running maximum); larger groups keep the merge path.  Either way the
    ancestors equal the oracle's, on the same degenerate, tied and NaN inputs
    (a single dominant particle's outputs span every CTA of its cluster)."""
    from paper_1310_4624_gb300.filter import resample
    rng = np.random.default_rng(G * 7919 + Np)
    lw = _weights(kind, G, Np, rng)
    u = rng.integers(0, 2 ** 32, size=G, dtype=np.uint64).astype(np.uint32)
    anc = resample(torch.from_numpy(lw.ravel()).to(dev), torch.from_numpy(u.view(np.int32)).to(dev), G, Np)
    anc = anc.cpu().numpy().reshape(G, Np)
    for g in range(G):
        ao = ora.resample(ora.quantize(lw[g]), int(u[g]))
        assert np.array_equal(anc[g], ao), "group %d: %d ancestors differ" % (g, int((anc[g] != ao).sum()))
