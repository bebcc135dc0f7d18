"""Public-API details on the GPU: pf_estimate_async returns what
pf_estimate returns, through page-locked host buffers, without waiting."""
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


def test_estimate_async_equals_estimate(dev):
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wls = [synth.small_rna(G=3, Np=300, mode=synth.ARNA, T=5, data_seed=s) for s in range(3)]
    seqs = [synth.make_sequence(wl) for wl in wls]
    frs = [torch.from_numpy(f).to(dev) for f, _ in seqs]
    pf = ParticleFilter([config_from_workload(wl, seqs[t][1][0], track_id=t) for t, wl in enumerate(wls)],
                        history=8, device=dev)
    x = torch.zeros((3, 5), dtype=torch.float32).pin_memory()
    z = torch.zeros(3, dtype=torch.float64).pin_memory()
    for k in range(wls[0].T):
        pf.step([fr[k] for fr in frs])
        pf.estimate_async(x, z)
        pf.stream.synchronize()
        xs, zs, st = pf.estimate()
        assert np.array_equal(x.numpy(), xs) and np.array_equal(z.numpy(), zs)
    pf.close()
