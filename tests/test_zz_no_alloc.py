"""pf_resample_noalloc against pf_resample, through the C ABI.

pf_resample_noalloc serves callers that cannot allocate device memory where
they resample (a memory budget fixed up front, a caching allocator that must
not be bypassed, a loop that cannot afford cudaMalloc's implicit device
synchronisation); its scratch is a fixed array inside the library.  Its
results must be those of pf_resample, call after call, although every call
reuses the same scratch.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def _inputs(G, Np, seed):
    rng = np.random.default_rng(seed)
    lw = (rng.normal(size=(G, Np)) * 5.0 - 200.0).astype(np.float32)
    lw[0, :] = -np.inf                      # a group without weight
    if G > 1:
        lw[1, : Np // 3] = np.nan
    if G > 2:
        lw[2, :] = -40.0
        lw[2, Np // 2] = 0.0                # one dominant particle
    u = rng.integers(0, 2 ** 32, size=G, dtype=np.uint64).astype(np.uint32)
    return lw, u


def _noalloc(lw_t, u_t, G, Np, dev, want_q=True):
    from paper_1310_4624_gb300 import binding as B
    anc = torch.full((G * Np,), -1, dtype=torch.int32, device=dev)
    q = torch.full((G * Np,), -1, dtype=torch.int64, device=dev) if want_q else None
    s = torch.cuda.current_stream(dev)
    B.pf_resample_noalloc(C.c_void_p(lw_t.data_ptr()), C.c_void_p(u_t.data_ptr()), G, Np,
                          C.c_void_p(anc.data_ptr()), C.c_void_p(q.data_ptr()) if want_q else None,
                          C.c_void_p(s.cuda_stream))
    # the kernel's device-side error word, read back after the stream
    B.pf_resample_check(None, C.c_void_p(s.cuda_stream))
    return anc, q


@pytest.mark.parametrize("G,Np", [(4, 1000), (64, 16384), (3, 70001), (1024, 64)])
def test_noalloc_equals_pf_resample_on_consecutive_calls(dev, G, Np):
    """(1024, 64) fills the scratch: as many groups as it holds."""
    from paper_1310_4624_gb300.filter import resample
    first = _inputs(G, Np, 1)
    second = _inputs(G, Np, 2)
    for lw, u in (first, first, second):   # two identical calls in a row, then new inputs
        lw_t = torch.from_numpy(lw.ravel()).to(dev)
        u_t = torch.from_numpy(u.view(np.int32)).to(dev)
        ref_anc, ref_q = resample(lw_t, u_t, G, Np, want_q=True)
        anc, q = _noalloc(lw_t, u_t, G, Np, dev)
        assert torch.equal(anc, ref_anc)
        assert torch.equal(q, ref_q)


def test_noalloc_without_weight_codes(dev):
    """q_dev may be NULL: the same ancestors, twice in a row."""
    from paper_1310_4624_gb300.filter import resample
    G, Np = 5, 3001
    lw, u = _inputs(G, Np, 3)
    lw_t = torch.from_numpy(lw.ravel()).to(dev)
    u_t = torch.from_numpy(u.view(np.int32)).to(dev)
    ref = resample(lw_t, u_t, G, Np)
    for _ in range(2):
        anc, _ = _noalloc(lw_t, u_t, G, Np, dev, want_q=False)
        assert torch.equal(anc, ref)


def test_noalloc_rejects_more_groups_than_its_scratch(dev):
    from paper_1310_4624_gb300 import binding as B
    G, Np = 1025, 4
    lw = torch.zeros(G * Np, dtype=torch.float32, device=dev)
    u = torch.zeros(G, dtype=torch.int32, device=dev)
    anc = torch.zeros(G * Np, dtype=torch.int32, device=dev)
    with pytest.raises(B.PFError) as e:
        B.pf_resample_noalloc(C.c_void_p(lw.data_ptr()), C.c_void_p(u.data_ptr()), G, Np,
                              C.c_void_p(anc.data_ptr()), None, None)
    assert e.value.status == B.PF_ERR_ARG
    assert "1024" in str(e.value)
