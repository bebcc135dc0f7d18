"""Public-API details on the GPU: pf_estimate_async returns what
pf_estimate returns, without waiting, into page-locked host buffers (stored
by the finishing kernel), pageable ones (copies) or a mix of the two."""
import ctypes as C

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


def test_estimate_async_host_buffer_kinds(dev):
    from paper_1310_4624_gb300 import binding as B
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wls = [synth.small_rna(G=4, Np=256, mode=synth.ARNA, T=4, data_seed=10 + s) for s in range(2)]
    seqs = [synth.make_sequence(wl) for wl in wls]
    frs = [torch.from_numpy(f).to(dev) for f, _ in seqs]
    pf = ParticleFilter([config_from_workload(wl, seqs[t][1][0], track_id=t) for t, wl in enumerate(wls)],
                        history=8, device=dev)
    pinned = (torch.zeros((2, 5), dtype=torch.float32).pin_memory(), torch.zeros(2, dtype=torch.float64).pin_memory())
    pageable = (np.zeros((2, 5), np.float32), np.zeros(2, np.float64))

    def ptr(a):
        return C.c_void_p(a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data)

    def arr(a):
        return a.numpy() if isinstance(a, torch.Tensor) else a

    stream = C.c_void_p(pf.stream.cuda_stream)
    for k in range(wls[0].T):
        pf.step([fr[k] for fr in frs])
        for xb, zb in [(pinned[0], pinned[1]), (pageable[0], pageable[1]), (pinned[0], pageable[1]),
                       (pageable[0], pinned[1])]:
            arr(xb)[:] = np.nan
            arr(zb)[:] = np.nan
            B.pf_estimate_async(pf.handle, ptr(xb), ptr(zb), stream)  # the first call finishes the step
            pf.stream.synchronize()
            xs, zs, _ = pf.estimate()
            assert np.array_equal(arr(xb), xs) and np.array_equal(arr(zb), zs)
        # one buffer only
        arr(pinned[0])[:] = np.nan
        arr(pinned[1])[:] = -1.0
        B.pf_estimate_async(pf.handle, ptr(pinned[0]), None, stream)
        pf.stream.synchronize()
        assert np.array_equal(arr(pinned[0]), xs) and (arr(pinned[1]) == -1.0).all()
        B.pf_estimate_async(pf.handle, None, ptr(pinned[1]), stream)
        pf.stream.synchronize()
        assert np.array_equal(arr(pinned[1]), zs)
    with pytest.raises(B.PFError):
        B.pf_estimate_async(pf.handle, None, None, stream)
    pf.close()
