"""Pins for the exchange topologies of Sec. VI (the paper's future work):
a ring that keeps each node's groups together, and the hypercube's
dimension exchange.  CPU only."""
import collections
import itertools

import numpy as np
import pytest


def _cfg(ora, **kw):
    base = dict(G=7, Np=16, mode=ora.ARNA, seed=3, topology=ora.TOPO_NODE_RING, node_groups=3)
    base.update(kw)
    return ora.make_cfg(**base)


def test_node_ring_keeps_each_node_together(ora):
    cfg = _cfg(ora)
    nodes = [set(range(n * 3, min(n * 3 + 3, 7))) for n in range(3)]
    for k in range(1, 60):
        sig = list(ora.ring(cfg, k))
        assert sorted(sig) == list(range(7))
        # the ring is a concatenation of whole nodes
        pos = 0
        while pos < 7:
            node = next(s for s in nodes if sig[pos] in s)
            assert set(sig[pos:pos + len(node)]) == node
            pos += len(node)
        # exactly one ring edge leaves each node
        cross = sum(1 for p in range(7) if not any({sig[p], sig[(p + 1) % 7]} <= s for s in nodes))
        assert cross == 3


def test_node_ring_is_uniform_over_node_and_member_orders(ora):
    """G = 4 in two nodes of two: 2 node orders x 2 x 2 member orders = 8
    rings, equally likely."""
    cfg = _cfg(ora, G=4, node_groups=2, seed=9)
    K = 8000
    counts = collections.Counter(tuple(ora.ring(cfg, k)) for k in range(1, K + 1))
    want = {tuple(a + b) for a, b in itertools.product(
        [list(p) for p in itertools.permutations([0, 1])], [list(p) for p in itertools.permutations([2, 3])])}
    want |= {tuple(b + a) for a, b in itertools.product(
        [list(p) for p in itertools.permutations([0, 1])], [list(p) for p in itertools.permutations([2, 3])])}
    assert set(counts) == want
    e = K / 8
    chi2 = sum((c - e) ** 2 / e for c in counts.values())
    assert chi2 < 24.3  # 7 dof, p = 0.001


def test_node_ring_with_one_node_is_the_plain_shuffle_family(ora):
    """node_groups >= G: one node, so the ring is a uniform shuffle of all
    groups (every one of the 4! orders appears)."""
    cfg = _cfg(ora, G=4, node_groups=4)
    seen = {tuple(ora.ring(cfg, k)) for k in range(1, 3000)}
    assert len(seen) == 24


def test_node_ring_under_rna_is_the_fixed_ring(ora):
    cfg = _cfg(ora, mode=ora.RNA)
    for k in (1, 5):
        assert list(ora.ring(cfg, k)) == list(range(7))


@pytest.mark.parametrize("G", [2, 5, 8, 13])
def test_hypercube_partners(ora, G):
    D = ora.hyper_dims(G)
    assert (1 << D) >= G and (D == 0 or (1 << (D - 1)) < G)
    for mode in (ora.RNA, ora.ARNA):
        cfg = ora.make_cfg(G=G, Np=8, mode=mode, topology=ora.TOPO_HYPERCUBE, seed=5)
        dims = []
        for k in range(1, 40):
            sig = ora.ring(cfg, k)
            pr = ora.pred_topo(cfg, sig)
            assert np.array_equal(pr[pr], np.arange(G))          # mutual exchange
            diff = pr ^ np.arange(G)
            bits = {int(x) for x in diff if x}
            assert len(bits) == 1                                   # one dimension per step
            d = bits.pop().bit_length() - 1
            assert all(pr[g] == (g ^ (1 << d) if (g ^ (1 << d)) < G else g) for g in range(G))
            dims.append(d)
        if mode == ora.RNA:
            assert dims == [(k - 1) % D for k in range(1, 40)]
        else:
            assert set(dims) == set(range(D))


def test_hypercube_arna_dimensions_uniform(ora):
    cfg = ora.make_cfg(G=8, Np=8, mode=ora.ARNA, topology=ora.TOPO_HYPERCUBE, seed=11)
    K = 6000
    c = collections.Counter()
    for k in range(1, K + 1):
        pr = ora.pred_topo(cfg, ora.ring(cfg, k))
        c[int(pr[0]).bit_length() - 1] += 1
    e = K / 3
    assert sum((v - e) ** 2 / e for v in c.values()) < 13.8  # 2 dof, p = 0.001


def test_hypercube_spreads_information_in_log2_steps(ora):
    """RNA dimension exchange on G = 2^D groups: the groups that have
    received (directly or through others) from group 0 after s steps number
    2^s, so all G after D steps (the cube's diameter); on the fixed ring
    they number s + 1."""
    def reach(topo, steps):
        cfg = ora.make_cfg(G=16, Np=32, mode=ora.RNA, topology=topo, seed=1)
        got = {0}
        sizes = []
        for k in range(1, steps + 1):
            pr = ora.pred_topo(cfg, ora.ring(cfg, k))
            got |= {r for r in range(16) if pr[r] in got}
            sizes.append(len(got))
        return sizes
    assert reach(ora.TOPO_HYPERCUBE, 4) == [2, 4, 8, 16]
    assert reach(ora.TOPO_RING, 4) == [2, 3, 4, 5]
