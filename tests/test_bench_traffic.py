"""bench.py's recorded DRAM traffic (profiles/traffic_sphere655362_k128.txt): the file
parses, and the stamp that ties each line to its kernel's code is the same wherever the
tree sits (the GPU machine runs a copy of the tree from another directory)."""
import json
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_traffic_file_lines():
    import bench
    path = os.path.join(ROOT, "profiles", "traffic_sphere655362_k128.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert sorted(r[0] for r in rows) == sorted(bench.TRAFFIC_SOURCE)
    for name, nbytes, stamp in rows:
        assert int(nbytes) > 0 and len(stamp) == 16


def test_traffic_stamp_does_not_depend_on_the_tree_location(tmp_path):
    import bench
    here = {k: bench.traffic_stamp(k) for k in bench.TRAFFIC_SOURCE}
    dst = tmp_path / "elsewhere"
    shutil.copytree(os.path.join(ROOT, "paper_1511_07042_gb300"), dst / "paper_1511_07042_gb300",
                    ignore=shutil.ignore_patterns("*.so", "*.o", "__pycache__", "_build"))
    shutil.copytree(os.path.join(ROOT, "include"), dst / "include")
    shutil.copy(os.path.join(ROOT, "bench.py"), dst / "bench.py")
    code = "import json, bench; print(json.dumps({k: bench.traffic_stamp(k) for k in bench.TRAFFIC_SOURCE}))"
    out = subprocess.run([sys.executable, "-c", code], cwd=dst, capture_output=True, text=True, timeout=600,
                         env={**os.environ, "PYTHONPATH": str(dst)})
    assert out.returncode == 0, out.stderr[-2000:]
    assert json.loads(out.stdout.strip().splitlines()[-1]) == here
