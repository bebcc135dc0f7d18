"""The one-launch (fused) step, PFARNA_FUSED=1: the same cases as the
two-launch step against the oracle step by step, a batch bit-equal to its
tracks run alone, the graph step, and the bounded wait of the failure test
(no fault: the staging copy is withheld)."""
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


@pytest.fixture(autouse=True)
def fused(monkeypatch):
    monkeypatch.setenv("PFARNA_FUSED", "1")


CASES = [("cfg1_rna", synth.small_rna()),
         ("arna_ragged", synth.small_rna(G=5, Np=300, H=40, W=40, mode=synth.ARNA)),
         ("single_group", synth.small_rna(G=1, Np=500, mode=synth.ARNA)),
         ("multi_chunk_group", synth.small_rna(G=2, Np=5000, mode=synth.ARNA, seed=9)),
         ("ess_arna_sharing", synth.sharing(G=8, Np=512, H=64, W=64, mode=synth.ARNA, resample_rule=1,
                                            ess_fraction=0.5)),
         ("keyed_arna_ragged", synth.small_rna(G=5, Np=300, H=40, W=40, mode=synth.ARNA, ex_ratio=0.3, send_rule=1)),
         ("frame_model", synth.small_rna(G=4, Np=512, mode=synth.ARNA, obs_model=1)),
         ("max_groups", synth.small_rna(G=1024, Np=16, H=64, W=64, mode=synth.ARNA, ex_ratio=0.5)),
         ("one_particle_groups", synth.small_rna(G=5, Np=1, mode=synth.ARNA))]


@pytest.mark.parametrize("name,wl", CASES, ids=[c[0] for c in CASES])
def test_fused_step_matches_oracle(dev, name, wl):
    from parity_util import run_and_compare
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    frames, truth = synth.make_sequence(wl, T=6)
    pf = ParticleFilter([config_from_workload(wl, truth[0], record_ancestors=True)], history=8, device=dev)
    assert pf.profile_read is not None
    rep = run_and_compare(pf, wl, frames, truth[0], 6, torch.from_numpy(frames).to(dev))
    assert len(rep) == 6
    pf.close()


def test_fused_tracking_scale_matches_oracle(dev):
    import os
    import oracle as ora
    from parity_util import run_and_compare
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wl = synth.tracking(mode=synth.ARNA)
    frames, truth = synth.make_sequence(wl, T=4)
    pf = ParticleFilter([config_from_workload(wl, truth[0], record_ancestors=True)], history=8, device=dev)
    ora.set_threads(os.cpu_count() or 1)
    try:
        run_and_compare(pf, wl, frames, truth[0], 4, torch.from_numpy(frames).to(dev))
    finally:
        ora.set_threads(1)
    pf.profile(True)
    pf.step(torch.from_numpy(frames[0]).to(dev))
    prof = pf.profile_read()
    assert prof["fused_step"][0] == 1 and prof["propagate_weight"][0] == 0
    pf.close()


def test_fused_batch_and_graph_equal_tracks_run_alone(dev, monkeypatch):
    from test_gpu_batched import _configs, _equal, _snapshot, _tracks
    from paper_1310_4624_gb300.filter import ParticleFilter
    wls = _tracks()
    seqs = [synth.make_sequence(wl) for wl in wls]
    frs = [torch.from_numpy(f).to(dev).contiguous() for f, _ in seqs]
    cfgs = _configs(wls, seqs, record=False)
    batch = ParticleFilter(cfgs, history=8, device=dev)
    table = batch.frame_table(frs)
    monkeypatch.setenv("PFARNA_FUSED", "0")
    alone = [ParticleFilter([c], history=8, device=dev) for c in cfgs]  # the two-launch step
    for k in range(wls[0].T):
        batch.step_table(table, graph=True)
        for t, pf in enumerate(alone):
            pf.step(frs[t][k])
    for t, pf in enumerate(alone):
        _equal(_snapshot(batch, t), _snapshot(pf, 0))


def test_fused_bounded_wait_reports_timeout(dev, monkeypatch):
    from paper_1310_4624_gb300 import binding as B
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wl = synth.small_rna(G=3, Np=700, H=64, W=64, mode=synth.ARNA)
    frames, truth = synth.make_sequence(wl, T=2)
    monkeypatch.setenv("PFARNA_TEST_WITHHOLD_COPY", "1")
    pf = ParticleFilter([config_from_workload(wl, truth[0])], history=4, device=dev)
    pf.step(torch.from_numpy(frames[0]).to(dev))
    with pytest.raises(B.PFError) as e:
        pf.estimate()
    assert e.value.status == B.PF_ERR_TIMEOUT
    pf.close()
    monkeypatch.delenv("PFARNA_TEST_WITHHOLD_COPY")
    pf = ParticleFilter([config_from_workload(wl, truth[0])], history=4, device=dev)  # the context still works
    pf.step(torch.from_numpy(frames[0]).to(dev))
    x, _, st = pf.estimate()
    assert st == B.PF_OK and np.all(np.isfinite(x))
    pf.close()
