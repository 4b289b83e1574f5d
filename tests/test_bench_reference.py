"""The reference arm of bench.py (the oracle timed on the host cores) prints
one JSON line with the contract's keys.  CPU only, on the small box."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--small",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    import bench
    assert cb["kind"] == "oracle" and cb["cores"] == bench.host_threads()
    assert cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_under_two_ranks_prints_from_rank_zero_only():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), "bench.py", "--impl", "reference", "--small",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    assert json.loads(lines[0])["n_gpus"] == 2


def test_threaded_oracle_baseline_steps_like_the_single_thread_oracle():
    # grain ranges on separate host threads, deposits summed in range order
    # and the feedback applied after the sum: the same state as the oracle
    # stepping every grain on one thread, up to the order of the deposit sum
    import numpy as np

    import bench
    from paper_1908_10793_gb300 import inputs as I
    for w in (I.sbox3d("small"), I.cyldisk("small")):
        one = bench.cpu_baseline(w, steps=2, threads=1, return_state=True)["state"]
        four = bench.cpu_baseline(w, steps=2, threads=4, return_state=True)["state"]
        q1, p1, g1, a1 = one
        q4, p4, g4, a4 = four
        assert np.array_equal(a1, a4)
        for d in range(3):
            assert np.allclose(q1[d], q4[d], rtol=0, atol=1e-13)
            assert np.allclose(p1[d], p4[d], rtol=1e-12, atol=1e-15)
            assert np.allclose(g1[d], g4[d], rtol=1e-12, atol=1e-15)
