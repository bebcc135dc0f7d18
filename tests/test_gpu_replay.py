"""pf_set_replay: pf_backward along an ancestry supplied by the caller, here
the FP64 oracle's own free-running ancestry (Alg. 3 with its exchange and
resampling choices, steps 3 and 7, held fixed), against the oracle's FP64
forward-mode gradient on that same ancestry: all of theta = (sigma_psf, A,
b, sigma_pos, sigma_v) within 1e-3 relative, log Z within 1e-5."""
import numpy as np
import pytest

import oracle as ora
from paper_1310_4624_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__ as ge
    ge.build()
    return torch.device("cuda:0")


def _gpu_forward(dev, wl, frames, truth):
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    pf = ParticleFilter([config_from_workload(wl, truth[0], record_ancestors=True)], history=wl.T, device=dev)
    fr = torch.from_numpy(frames).to(dev)
    for k in range(wl.T):
        pf.step(fr[k])
    return pf, fr


def _oracle_parents(wl, frames, truth):
    from parity_util import _init
    cfg = ora.cfg_from_workload(wl)
    kind, x0, lo, hi, rad = _init(wl, truth[0])
    pop = ora.init_population(cfg, kind, x0, lo, hi, rad)
    parents, logc = ora.run_with_parents(cfg, pop, frames, wl.T)
    lz, g = ora.replay_grad(cfg, kind, x0, frames, wl.T, parents, lo, hi, rad)
    return parents, logc, lz, g


CASES = [("arna", synth.small_rna(G=3, Np=256, H=48, W=48, mode=synth.ARNA, T=6)),
         ("rna", synth.small_rna(G=4, Np=200, H=40, W=56, mode=synth.RNA, T=5, seed=3, data_seed=2)),
         ("sharing", synth.sharing(G=4, Np=256, H=64, W=64, mode=synth.ARNA, T=5)),
         ("frame_model", synth.small_rna(G=3, Np=256, H=48, W=48, mode=synth.ARNA, T=5, obs_model=1))]


@pytest.mark.parametrize("name,wl", CASES, ids=[c[0] for c in CASES])
def test_backward_on_the_oracles_ancestry(dev, name, wl):
    frames, truth = synth.make_sequence(wl)
    parents, logc, lz_o, g_o = _oracle_parents(wl, frames, truth)
    # the replay of the oracle's own ancestry reproduces its forward log Z
    assert abs(lz_o - float(np.sum(logc))) <= 1e-9 * abs(lz_o)
    pf, fr = _gpu_forward(dev, wl, frames, truth)
    pf.set_replay(torch.from_numpy(parents).to(dev))
    grad, lz = pf.backward([fr[k] for k in range(wl.T)])
    g = grad[0].double().cpu().numpy()
    assert abs(float(lz[0]) - lz_o) <= 1e-5 * abs(lz_o), (float(lz[0]), lz_o)
    scale = np.abs(g_o).max()
    for q in range(5):
        assert abs(g[q] - g_o[q]) <= 1e-3 * abs(g_o[q]) + 1e-5 * scale, (ora.THETA[q], g[q], g_o[q])
    pf.close()


def test_replay_rejects_indices_outside_the_track(dev):
    from paper_1310_4624_gb300 import binding as B
    wl = synth.small_rna(G=2, Np=128, H=40, W=40, mode=synth.ARNA, T=3)
    frames, truth = synth.make_sequence(wl)
    pf, fr = _gpu_forward(dev, wl, frames, truth)
    par = torch.arange(wl.N, dtype=torch.int32, device=dev).repeat(wl.T, 1).contiguous()
    bad = par.clone()
    bad[2, 7] = wl.N  # one past the track
    with pytest.raises(B.PFError) as e:
        pf.set_replay(bad)
    assert e.value.status == B.PF_ERR_ARG
    with pytest.raises(B.PFError) as e:
        pf.backward([fr[k] for k in range(wl.T)])
    assert e.value.status == B.PF_ERR_STATE
    pf.set_replay(par)  # a valid ancestry restores pf_backward
    grad, lz = pf.backward([fr[k] for k in range(wl.T)])
    assert torch.isfinite(grad).all() and np.isfinite(float(lz[0]))
    pf.close()
