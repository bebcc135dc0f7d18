"""Failure detection without a GPU fault: the propagate kernel's wait for a
staging copy is bounded in time.  With the copy withheld (a test knob at
pf_init), the wait runs out, the kernel records a timeout and returns, the
host reads PF_ERR_TIMEOUT at the next synchronising call, and the context
stays usable for a new filter."""
import os

import pytest

from paper_1310_4624_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__ as ge
    ge.build()
    return torch.device("cuda:0")


def test_withheld_copy_times_out_and_context_survives(dev):
    from paper_1310_4624_gb300 import binding as B
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wl = synth.small_rna(G=2, Np=512, T=3)
    frames, truth = synth.make_sequence(wl)
    fr = torch.from_numpy(frames).to(dev)
    os.environ["PFARNA_TEST_WITHHOLD_COPY"] = "1"
    try:
        bad = ParticleFilter([config_from_workload(wl, truth[0])], history=4, device=dev)
    finally:
        del os.environ["PFARNA_TEST_WITHHOLD_COPY"]
    bad.step(fr[0])
    with pytest.raises(B.PFError) as err:
        bad.estimate()
    assert err.value.status == B.PF_ERR_TIMEOUT
    assert "0x2 " in str(err.value)  # the timeout bit alone: no resampling ran on the stale weights
    with pytest.raises(B.PFError) as err:
        bad.step(fr[1])  # a failed handle takes no more steps
    assert err.value.status == B.PF_ERR_STATE
    bad.close()
    torch.cuda.synchronize()  # the context is intact
    good = ParticleFilter([config_from_workload(wl, truth[0])], history=4, device=dev)
    for k in range(wl.T):
        good.step(fr[k])
    x, lz, st = good.estimate()
    assert st == B.PF_OK and abs(x[0, 0] - truth[-1, 0]) < 3.0
    good.close()


def test_backward_refuses_threshold_resampling(dev):
    """pf_backward replays every-step resampling only: a track under Alg. 1's
    N_eff test is refused with PF_ERR_ARG (no launch)."""
    from paper_1310_4624_gb300 import binding as B
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wl = synth.small_rna(G=2, Np=256, T=2, resample_rule=1)
    frames, truth = synth.make_sequence(wl)
    fr = torch.from_numpy(frames).to(dev)
    pf = ParticleFilter([config_from_workload(wl, truth[0], record_ancestors=True)], history=4, device=dev)
    for k in range(wl.T):
        pf.step(fr[k])
    with pytest.raises(B.PFError) as err:
        pf.backward([fr[k] for k in range(wl.T)])
    assert err.value.status == B.PF_ERR_ARG
    pf.close()
