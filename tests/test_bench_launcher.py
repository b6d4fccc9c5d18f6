"""`bench.py --gpus N` starts N ranks by itself (torch.distributed.run on
127.0.0.1) when no process group is given in the environment.  The dry run
exercises that launcher and the whole-job reduction on the CPU (gloo): rank r
stands in with (r + 1) * 1e6 site updates in 10 + r ms, so the line must
report N ranks, the summed units and the slowest rank's time."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpus_two_starts_two_ranks_on_the_cpu():
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR",
                                                             "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--dry-run"], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = lines[0]
    assert line["dry_run"] is True and line["value"] is None
    assert line["n_gpus"] == 2
    assert line["units"] == 3e6
    assert line["ms"] == 11.0
