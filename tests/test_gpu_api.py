"""Public-API details on the GPU: pf_estimate_async returns what
pf_estimate returns, without waiting, into page-locked host buffers (stored
by the finishing kernel), pageable ones (copies) or a mix of the two; and
pf_step_host (frames in host memory, uploaded by the library) steps exactly
as pf_step on device frames."""
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


def _pair(dev, wls, truths, shared=False):
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    cfgs = [config_from_workload(wl, truths[t][0], track_id=t) for t, wl in enumerate(wls)]
    return (ParticleFilter(cfgs, history=8, device=dev), ParticleFilter(cfgs, history=8, device=dev))


@pytest.mark.parametrize("n_tracks,pinned,shared", [(1, True, False), (3, True, False), (3, False, False),
                                                    (3, True, True)])
def test_step_host_equals_step(dev, n_tracks, pinned, shared):
    """A single track takes the TMA path on the staged frame, several tracks the
    frame-preparation path; `shared` gives every track the same host frame
    (uploaded once) and the device side the same device frame."""
    T = 5
    wls = [synth.small_rna(G=4, Np=512, mode=synth.ARNA, T=T, data_seed=20 + s) for s in range(n_tracks)]
    seqs = [synth.make_sequence(wl) for wl in wls]
    if shared:
        seqs = [seqs[0]] * n_tracks
    a, b = _pair(dev, wls, [tr for _, tr in seqs])
    host = [torch.from_numpy(f) for f, _ in seqs]
    if pinned:
        host = [h.pin_memory() for h in host]
    devf = [h.to(dev) for h in host]
    for k in range(T):
        if shared:
            a.step([devf[0][k]] * n_tracks)
            b.step_host([host[0][k]] * n_tracks)
        else:
            a.step([f[k] for f in devf])
            b.step_host([h[k] for h in host])
        xa, za, _ = a.estimate()
        xb, zb, _ = b.estimate()
        assert np.array_equal(xa, xb) and np.array_equal(za, zb), k
        for t in range(n_tracks):
            sa, sb = a.stats(k, t), b.stats(k, t)
            assert sa["n_ex"] == sb["n_ex"] and np.array_equal(sa["logW"], sb["logW"])
    a.close()
    b.close()


def test_step_host_pipelined_without_waiting(dev):
    """Steps enqueued back to back with the host frames of later steps
    uploaded while earlier steps run (two staging slots): the estimates,
    read asynchronously each step, equal pf_step's."""
    T = 8
    wl = synth.small_rna(G=8, Np=1024, mode=synth.ARNA, T=T, data_seed=31)
    frames, truth = synth.make_sequence(wl)
    a, b = _pair(dev, [wl], [truth])
    host = torch.from_numpy(frames).pin_memory()
    devf = host.to(dev)
    xs_a, xs_b = [], []
    outs = [(torch.zeros((1, 5), dtype=torch.float32).pin_memory(), torch.zeros(1, dtype=torch.float64).pin_memory())
            for _ in range(T)]
    for k in range(T):
        b.step_host(host[k])
        b.estimate_async(*outs[k])
    b.stream.synchronize()
    for k in range(T):
        a.step(devf[k])
        x, z, _ = a.estimate()
        assert np.array_equal(outs[k][0].numpy(), x) and np.array_equal(outs[k][1].numpy(), z), k
    a.close()
    b.close()


def test_step_host_rejects_bad_staging(dev):
    from paper_1310_4624_gb300 import binding as B
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wl = synth.small_rna(G=2, Np=128, T=2)
    frames, truth = synth.make_sequence(wl)
    pf = ParticleFilter([config_from_workload(wl, truth[0])], history=4, device=dev)
    n = B.pf_host_staging_bytes(pf.handle)
    assert n >= 2 * wl.H * wl.W * 4
    buf = torch.empty(n + 512, dtype=torch.uint8, device=dev)
    p = (buf.data_ptr() + 255) // 256 * 256
    host = torch.from_numpy(frames).pin_memory()
    s = C.c_void_p(pf.stream.cuda_stream)
    for ptr, size, msg in [(p, n - 1, "smaller"), (p + 16, n, "aligned"), (0, n, "NULL")]:
        with pytest.raises(B.PFError) as e:
            B.pf_step_host(pf.handle, [host[0].data_ptr()], C.c_void_p(ptr), size, s)
        assert e.value.status == B.PF_ERR_ARG and msg in str(e.value)
    with pytest.raises(B.PFError):
        B.pf_step_host(pf.handle, [None], C.c_void_p(p), n, s)
    B.pf_step_host(pf.handle, [host[0].data_ptr()], C.c_void_p(p), n, s)  # the handle is still usable
    pf.estimate()
    pf.close()
