"""Multi-object tracking as one filter per object in one batched handle:
every track reads the same frames (one pointer per track, all equal) and
starts at its own spot.  Each track matches the oracle step by step and
follows its spot."""
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


def test_tracks_share_frames_and_follow_their_spots(dev):
    from parity_util import run_and_compare
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wls = synth.multi_object(n_obj=8, G=4, Np=1024, H=128, W=256, T=12, cell=64)
    frames, truths = synth.make_multi_sequence(wls)
    fr = torch.from_numpy(frames).to(dev)
    cfgs = [config_from_workload(wl, truths[t][0], track_id=t, record_ancestors=True) for t, wl in enumerate(wls)]
    for t in (0, 5):
        pf = ParticleFilter(cfgs, history=16, device=dev)
        run_and_compare(pf, wls[t], frames, truths[t][0], wls[t].T, None, track=t,
                        stepper=lambda k: pf.step([fr[k]] * len(wls)))
        pf.close()
    pf = ParticleFilter(cfgs, history=16, device=dev)
    for k in range(wls[0].T):
        pf.step([fr[k]] * len(wls))
    for t in range(len(wls)):
        hs = pf.history_stats(0, wls[0].T, track=t)
        err = np.array([np.hypot(*(h["xhat"][:2] - truths[t][h["step"], :2])) for h in hs])
        assert np.sqrt((err ** 2).mean()) < 0.5, (t, err)
    pf.close()


def test_shared_frame_equals_separate_copies(dev):
    """Tracks given the same frame pointer share one prepared copy; the
    results are bit-identical to giving each track its own copy."""
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wls = synth.multi_object(n_obj=6, G=3, Np=700, H=128, W=192, T=6, cell=64, mode=synth.RNA)
    wls[2] = wls[2].replace(background=1.5)  # another background: never shares
    frames, truths = synth.make_multi_sequence(wls)
    fr = torch.from_numpy(frames).to(dev)
    copies = [fr.clone() for _ in wls]
    cfgs = [config_from_workload(wl, truths[t][0], track_id=t) for t, wl in enumerate(wls)]
    a = ParticleFilter(cfgs, history=8, device=dev)
    b = ParticleFilter(cfgs, history=8, device=dev)
    for k in range(wls[0].T):
        a.step([fr[k]] * len(wls))
        b.step([c[k] for c in copies])
    for t in range(len(wls)):
        pa, pb = a.particles(track=t), b.particles(track=t)
        for key in ("states", "anc", "logw"):
            assert torch.equal(pa[key], pb[key]), (t, key)
        sa, sb = a.stats(wls[0].T - 1, track=t), b.stats(wls[0].T - 1, track=t)
        assert sa["log_Z"] == sb["log_Z"] and np.array_equal(sa["xhat"], sb["xhat"])
    a.close()
    b.close()
