"""The PF_DEBUG build: the same kernels with explicit index checks that report
into the device error word (ERR_DEBUG, with the site, index and bound) in
place of a memory checker, which this pool does not provide.  It runs small
cases of every step path in a child process that loads the debug library:
single-track ARNA and RNA (a ragged group), a batch of tracks with different
group sizes stepped by frame table and CUDA graph, the one-launch step, the
standalone resampler and the adjoint.  Every call that reads the error word
back fails on a set bit, so a clean run means that no check fired."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys
sys.path.insert(0, os.getcwd())
import numpy as np, torch
from paper_1310_4624_gb300 import binding, build, synth
from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload, resample
assert binding.lib_path() == build.LIB_DEBUG, binding.lib_path()
dev = torch.device("cuda:0")

def run(wls, T, record=False, table=False):
    seqs = [synth.make_sequence(wl) for wl in wls]
    cfgs = [config_from_workload(wl, seqs[t][1][0], track_id=t, record_ancestors=record) for t, wl in enumerate(wls)]
    pf = ParticleFilter(cfgs, history=T + 1, device=dev)
    frs = [torch.from_numpy(f).to(dev) for f, _ in seqs]
    if table:
        tab = pf.frame_table([fr[:T].contiguous() for fr in frs])
        for k in range(T):
            pf.step_table(tab, graph=(k % 2 == 1))
    else:
        for k in range(T):
            pf.step([fr[k] for fr in frs])
    pf.estimate()
    for t in range(len(wls)):
        pf.particles(track=t, parents=record)
    if record:
        pf.backward([frs[0][k] for k in range(T)])
    pf.close()

run([synth.small_rna(G=3, Np=300, H=48, W=48, T=5, mode=synth.ARNA)], 5)
run([synth.small_rna(G=4, Np=257, H=40, W=56, T=4, mode=synth.RNA, seed=3, data_seed=2)], 4)
run([synth.small_rna(G=3, Np=256, H=48, W=48, T=4, mode=synth.ARNA)], 4, record=True)
run([synth.small_rna(G=2, Np=700, H=64, W=64, T=4, mode=synth.ARNA, data_seed=5),
     synth.small_rna(G=5, Np=130, H=64, W=64, T=4, mode=synth.RNA, data_seed=6)], 4, table=True)
run([synth.tracking(mode=synth.ARNA, G=8, Np=5000, T=3)], 3)
os.environ["PFARNA_FUSED"] = "1"
run([synth.small_rna(G=3, Np=600, H=48, W=48, T=4, mode=synth.ARNA)], 4)
del os.environ["PFARNA_FUSED"]
g = torch.Generator().manual_seed(7)
lw = (torch.randn(6 * 3000, generator=g, dtype=torch.float64) * 3).float().to(dev)
u = torch.randint(0, 2 ** 32, (6,), generator=g, dtype=torch.int64).to(torch.int32).to(dev)
resample(lw, u, 6, 3000)
torch.cuda.synchronize()
print("debug-clean")
'''


def test_debug_build_runs_clean():
    from paper_1310_4624_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, PFARNA_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0 and "debug-clean" in r.stdout, (r.stdout[-3000:], r.stderr[-3000:])
