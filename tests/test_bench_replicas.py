"""The multi-GPU path of bench.py runs independent replicas (the filter does
not shard across GPUs): ranks synchronise with a barrier and report the
maximum time over ranks.  Those host-side pieces, run here as two gloo ranks
on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, lr = bench.dist_setup()
    dist.init_process_group("gloo", rank=r, world_size=w)
    bench.barrier(w)
    out[rank] = (w, r, lr, bench.reduce_max(1.5 + rank, w, "cpu"))
    bench.barrier(w)
    dist.destroy_process_group()


def test_replicas_barrier_and_max_over_ranks():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        got = dict(out)
    assert got[0] == (2, 0, 0, 2.5)
    assert got[1] == (2, 1, 1, 2.5)


def test_reference_arm_prints_one_oracle_line():
    """bench.py --impl reference (the oracle on the host cores) prints one
    JSON line with the headline metric, unit and config, and the fields the
    reference arm carries."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, check=True, cwd=root, timeout=600)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "particle-steps/s" and d["metric"].startswith("particle-steps/s")
    assert d["config"]["workload"] == "tracking_512x512_G64x16384_arna"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
