"""Host logic of the benchmark's arithmetic roofline: the direct-form MUFU
counts per chain-iteration add up to the totals derived from the models'
expression trees, and the mix's MUFU rate is the harmonic combination of the
per-operation rates the pipe-rate probe measures."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_direct_form_totals(bench):
    # 3-pool: 24 echoes x 3 pools x (exp, sin, cos) + 3 rcp + 5 Box-Muller pairs x 4 + 1
    assert sum(bench.OPS["mwi3_1m"]["mufu"].values()) == 24 * 3 * 3 + 3 + 5 * 4 + 1 == 240
    # SMT: 6 b x (exp + 2 g x (sqrt, erf, rcp)) + 2 pairs x 4 + 1
    assert sum(bench.OPS["smt_1p5m"]["mufu"].values()) == 6 * 7 + 2 * 4 + 1 == 51
    assert sum(bench.OPS["monoexp_4k"]["mufu"].values()) == 12 + 4 + 1 == 17
    # AxCaliberSMT: 2 timings x 18 terms x 3 exp + 16 x (2 exp + 2 g) + 2 pairs + 1
    assert sum(bench.OPS["axcal_250k"]["mufu"].values()) == 2 * 18 * 3 + 16 * (2 + 6) + 2 * 4 + 1 == 245
    # ensemble: no Box-Muller, one acceptance log and one stretch log
    for k, w in (("mwi3_1m", 240 - 20 - 1), ("smt_1p5m", 51 - 8 - 1), ("monoexp_4k", 17 - 4 - 1),
                 ("axcal_250k", 245 - 8 - 1)):
        assert sum(bench.OPS_ENSEMBLE[k]["mufu"].values()) == w + 2


def test_mix_rate_is_harmonic(bench):
    flat = dict.fromkeys(("ex2", "sin", "lg2", "sqrt", "rcp", "rsqrt"), 16.0)
    flat["ffma"] = 128.0
    mufu, fp32, basis = bench._alu_peaks({"ex2": 10, "sin": 30}, flat)
    assert mufu == pytest.approx(16.0) and fp32 == 128.0 and "measured" in basis
    fast = dict(flat, ex2=32.0)
    mufu, _, _ = bench._alu_peaks({"ex2": 10, "sin": 30}, fast)
    assert mufu == pytest.approx(40.0 / (10 / 32.0 + 30 / 16.0))
    assert bench._alu_peaks({"ex2": 1}, None)[:2] == (bench.MUFU_PER_CLK_SM, bench.FP32_PER_CLK_SM)


def test_source_hash_ignores_comments_and_layout(bench):
    a = 'int f(int x) { // doubles x\n  return 2 * x; /* no\n overflow check */ }\nconst char *s = "a//b";\n'
    b = 'int f(int x) {\n    return 2 * x;\n}\nconst char *s = "a//b";'
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(b.replace("2 * x", "3 * x"))
    assert '"a//b"' in bench._code_only(a)  # string literals are kept whole
    for w in bench.MEASURED:  # every measured workload has a hashable source set
        assert len(bench._sources_hash(w)) == 16


def _json_lines(text):
    import json
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def test_reference_arm_line(bench):
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the benchmark contract's keys; under torchrun only rank 0
    prints and every rank exits 0."""
    import subprocess
    import sys
    args = ["--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "monoexp_4k",
            "--n-vox", "256", "--iterations", "200"]
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"] == "monoexp_4k"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["e2e"]["d2h_bytes_per_step"] == 0

    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", "29541", os.path.join(ROOT, "bench.py"),
                        "--gpus", "2", *args], capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert len(_json_lines(r.stdout)) == 1
