"""bench.py's multi-rank path on CPU: world size 2 over gloo (one replica per rank,
no data-path collective; timing is the slowest rank's, value = units of all
ranks over it; the reference arm prints one line from rank 0)."""
import json
import socket
import subprocess
import sys
import textwrap
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def _port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, cwd, timeout=300):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_port()), *args]
    return subprocess.run(cmd, cwd=cwd, capture_output=True, text=True, timeout=timeout)


def test_timing_is_the_slowest_rank_and_value_counts_all_ranks(tmp_path):
    script = tmp_path / "agg.py"
    script.write_text(textwrap.dedent(f"""
        import json, os, sys
        sys.path.insert(0, {str(ROOT)!r})
        import torch.distributed as dist
        import bench
        rank, world, _ = bench.dist_env()
        dist.init_process_group("gloo")
        total, value = bench.aggregate_timing(100.0 * (rank + 1), 50, world)
        with open(os.path.join({str(tmp_path)!r}, f"rank{{rank}}.json"), "w") as f:
            json.dump({{"rank": rank, "total": total, "value": value}}, f)
        dist.barrier()
        dist.destroy_process_group()
    """))
    out = _torchrun([str(script)], cwd=tmp_path)
    assert out.returncode == 0, out.stderr[-2000:]
    rows = [json.loads((tmp_path / f"rank{r}.json").read_text()) for r in range(2)]
    assert sorted(r["rank"] for r in rows) == [0, 1]
    for r in rows:
        assert r["total"] == 200.0                  # the slower rank's 200 ms
        assert r["value"] == 2 * 50 / 0.2           # both ranks' 50 steps over it


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    out = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1"],
                    cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "plans/s"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    # the same counts and configuration object as the GPU arm's line
    assert d["steps"] == 2 and d["warmup"] == 1 and d["cycles"] == 2
    import bench
    assert d["config"] == bench.run_config(2, 2)
    assert d["cpu_baseline"]["cores"] == min(bench.host_cores(), 2)
