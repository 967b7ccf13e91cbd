"""The benchmark's multi-process rules on CPU (gloo, two ranks): timing is the
maximum over ranks, whole-job throughput counts every rank's units, and the
reference arm prints one line from rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench

        res = {"max": bench.reduce_max(10.0 + rank, ws), "sum": bench.reduce_sum(100.0 * (rank + 1), ws)}
        res["rate"] = bench.job_rate(1000.0, ws, res["max"])
        bench.barrier(ws)
        # the reference arm under two ranks: a tiny sample of the workload
        bench.REFERENCE_SAMPLE["text+dna"] = 1 << 12
        args = bench.argparse.Namespace(workload="text+dna", steps=1, warmup=0)
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.run_reference(args, ws, rank)
        res["ref"] = buf.getvalue()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch")
    ws = 2
    mp.spawn(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(ws)]
    for k in range(ws):
        assert r[k]["max"] == 11.0
        assert r[k]["sum"] == 300.0
        assert r[k]["rate"] == pytest.approx(2000.0 / 11e-3)
    assert r[1]["ref"] == ""
    line = json.loads(r[0]["ref"].strip())
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1


@pytest.mark.parametrize("workload", ["batch", "serve", "locality", "merge", "matrix"])
def test_reference_arm_of_multi_sequence_workloads_is_unavailable(workload):
    """The oracle is timed on the single-sequence workloads; the others print
    one `unavailable` line and exit 0."""
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          workload], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line
