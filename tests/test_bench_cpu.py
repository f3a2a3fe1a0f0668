"""bench.py's CPU-side pieces: the reference arm (the FP64 oracle timed on the host cores,
one process per core on independent lattice slabs) prints one JSON line with the
contract's keys; the kernel-source hash is stable."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "4^4_Ls8", "--steps", "1", "--warmup", "0", "--ref-budget", "0.5"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    d = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GB/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and 1 <= d["cpu_baseline"]["cores"] <= os.cpu_count()
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_kernel_source_hash_stable():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.kernel_sources_hash() == bench.kernel_sources_hash()
    assert len(bench.kernel_sources_hash()) == 64
