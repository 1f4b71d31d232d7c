"""The benchmark's JSON line contract, checked on the CPU through the reference arm (the oracle timed
on host cores), and its plan-configuration parser."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_plan_config_parser():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.parse_cfg("chunked:2,2") == dict(schedule="chunked", Bu=2, Bv=2)
    assert bench.parse_cfg("chunked:4,2:128") == dict(schedule="chunked", Bu=4, Bv=2, vis_per_chunk=128)
    assert bench.parse_cfg("patch:2,2:64:384") == dict(schedule="patch", Bu=2, Bv=2, vis_per_chunk=64, threads=384)


def test_efficiency_convention_reproduces_the_papers_numbers():
    """Sec. 5 pins the flop count: 365 GGPA/s at 8 flop per grid-point addition on a 5.288 TFLOP/s
    GPU is the 55% the paper reports, and the rate without coarsening (90% lower gain) falls in its
    27-29% range. The bench's fraction helper, given the paper's count, must reproduce both; the
    bench's own count for real taps is half of it."""
    sys.path.insert(0, ROOT)
    import bench
    g = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "sec5_gtx980_rates.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            g[k] = float(v)
    assert bench.PAPER_FLOPS_PER_GPA == g["flops_per_gpa"]
    assert bench.FLOPS_PER_GPA * 2 == bench.PAPER_FLOPS_PER_GPA
    best = bench.fma_fraction(g["best_ggpa"] * 1e9, g["peak_tflops"], g["flops_per_gpa"])
    assert abs(best * 100 - g["best_efficiency_pct"]) < 0.5
    plain = bench.fma_fraction(g["best_ggpa"] * 1e9 / (1 + g["coarsening_gain_pct"] / 100), g["peak_tflops"],
                               g["flops_per_gpa"])
    assert g["uncoarsened_lo_pct"] - 0.5 <= plain * 100 <= g["uncoarsened_hi_pct"] + 0.5
    # the bench's GB300 peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz
    assert abs(bench.fma_peak_tflops(152, 2070.0) - 80.54784) < 1e-6


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the driver launches N>1 (torchrun, two ranks): rank 0 alone times the oracle and
    prints one line; the other rank exits 0 without work."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_threaded_oracle_matches_the_single_thread_oracle():
    """The all-core CPU baseline runs the unchanged oracle from several threads (bands of grid rows,
    slices of visibilities); its grid and degridded values must be the single-thread oracle's up to
    the order of additions, including footprints that straddle a band edge."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import oracle
    from paper_1605_07023_gb300 import synth
    w = synth.plain_single_pol()
    t = oracle.kb_table(w.S, w.oversample, w.beta)
    g1, sk1 = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, t)
    d1, _ = oracle.degrid(w.G, w.S, w.oversample, w.uv, g1, t)
    for n in (1, 3, 8):
        g, d, sk, _ = bench.oracle_threads(w, t, n)
        assert sk == sk1
        assert np.linalg.norm(g - g1) <= 1e-12 * np.linalg.norm(g1)
        assert np.linalg.norm(d - d1) <= 1e-12 * np.linalg.norm(d1)
