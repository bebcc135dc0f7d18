"""The oracle's OpenMP loops (used only to time it on all host cores) give
the same bits as the single-threaded oracle: each loop writes only its own
particle's or group's outputs."""
import os

import numpy as np

from paper_1310_4624_gb300 import synth


def _run(ora, wl, T):
    frames, truth = synth.make_sequence(wl, T=T)
    cfg = ora.cfg_from_workload(wl)
    pop = ora.init_population(cfg, ora.INIT_POINT, np.float32(truth[0]).astype(np.float64))
    return ora.run(cfg, pop, frames, T)


def test_threads_do_not_change_results(ora):
    wl = synth.small_rna(G=6, Np=700, H=48, W=48, mode=synth.ARNA, ex_ratio=0.3)
    n = max(2, min(8, os.cpu_count() or 2))
    try:
        ora.set_threads(1)
        a = _run(ora, wl, 5)
        used = ora.set_threads(n)
        b = _run(ora, wl, 5)
    finally:
        ora.set_threads(1)
    assert used in (1, n)
    for f in ("xhat", "logc", "n_ex", "pe_eff", "sigma", "Lambda", "gxhat", "n_resampled", "pop_final"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
