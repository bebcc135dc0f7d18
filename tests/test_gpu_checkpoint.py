"""Checkpoint and resume (pf_save / pf_load): a filter restored from a
checkpoint, into the same handle or into a new one, continues bit for bit
as the saved filter did (every random draw is a counter-based Philox word)."""
import numpy as np
import pytest

from paper_1310_4624_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__ as ge
    ge.build()
    return torch.device("cuda:0")


def _snap(pf):
    p = pf.particles()
    st = pf.stats(pf.steps - 1)
    x, lz, _ = pf.estimate()
    return [p["states"].cpu().numpy(), p["anc"].cpu().numpy(), p["logw"].cpu().numpy(), st["ring"],
            np.array([st["n_ex"]]), st["logW"], x, lz]


@pytest.mark.parametrize("mode", [synth.ARNA, synth.RNA])
def test_resume_continues_bit_for_bit(dev, mode):
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wl = synth.sharing(G=6, Np=700, H=64, W=64, mode=mode, T=9, seed=4)
    frames, truth = synth.make_sequence(wl)
    fr = torch.from_numpy(frames).to(dev)
    cfg = config_from_workload(wl, truth[0], record_ancestors=True)
    a = ParticleFilter([cfg], history=16, device=dev)
    for k in range(4):
        a.step(fr[k])
    ck = a.save()
    ref = []
    for k in range(4, wl.T):
        a.step(fr[k])
        ref.append(_snap(a))
    # into a new handle
    b = ParticleFilter([cfg], history=16, device=dev)
    b.load(ck)
    assert b.steps == 4
    for i, k in enumerate(range(4, wl.T)):
        b.step(fr[k])
        for x, y in zip(_snap(b), ref[i]):
            assert np.array_equal(x, y, equal_nan=True)
    # into the saved handle itself, after it ran on
    a.load(ck)
    for i, k in enumerate(range(4, wl.T)):
        a.step(fr[k])
        for x, y in zip(_snap(a), ref[i]):
            assert np.array_equal(x, y, equal_nan=True)
    a.close()
    b.close()


def test_load_rejects_another_configuration(dev):
    from paper_1310_4624_gb300 import binding as B
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wl = synth.small_rna(T=2)
    frames, truth = synth.make_sequence(wl)
    a = ParticleFilter([config_from_workload(wl, truth[0])], history=4, device=dev)
    a.step(torch.from_numpy(frames[0]).to(dev))
    ck = a.save()
    other = wl.replace(Np=wl.Np + 8)
    b = ParticleFilter([config_from_workload(other, truth[0])], history=4, device=dev)
    with pytest.raises(B.PFError):
        b.load(ck)
    a.close()
    b.close()
