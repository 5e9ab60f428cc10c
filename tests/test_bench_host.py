"""Host logic of bench.py on CPU (no GPU): the roofline's DRAM traffic is the
committed ncu count only while the fused pass's sources are the ones it was
taken on; the roofline denominators come from the measured-peaks file, else
the stated fallback; both arms name the workload the same way."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join("paper_1910_14166_gb300", "csrc")
_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


@pytest.fixture(scope="module")
def bench():
    """bench.py as a module, imported only when these tests run (it sets the
    BLAS/OpenMP thread variables for its own process on import; they are
    put back so that the rest of the session keeps its threads)."""
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    sys.path.insert(0, ROOT)
    import bench as b
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    return b


def _copy_sources(dst):
    os.makedirs(os.path.join(dst, CSRC))
    for f in ("fused.cu", "common.cuh"):
        shutil.copy(os.path.join(ROOT, CSRC, f), os.path.join(dst, CSRC, f))


def test_source_hash_changes_with_either_fused_pass_source(bench, monkeypatch, tmp_path):
    real = bench.kernel_source_hash()
    _copy_sources(str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_source_hash() == real
    for f in ("fused.cu", "common.cuh"):
        p = tmp_path / CSRC / f
        text = p.read_text()
        p.write_text(text + "\n// edited\n")
        assert bench.kernel_source_hash() != real
        p.write_text(text)
        assert bench.kernel_source_hash() == real


def test_traffic_is_reported_only_for_the_sources_it_was_taken_on(bench, monkeypatch, tmp_path):
    (tmp_path / "profiles").mkdir()
    rec = {"source_hash": "0123456789abcdef", "kernels": {"k_sketch_grad_fused": 2223404032}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0123456789abcdef")
    assert bench.traffic_for("k_sketch_grad_fused") == 2223404032
    assert bench.traffic_for("k_sketch_dense") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "fedcba9876543210")
    assert bench.traffic_for("k_sketch_grad_fused") is None
    (tmp_path / "profiles" / "traffic.json").unlink()
    assert bench.traffic_for("k_sketch_grad_fused") is None


def test_peaks_measured_else_fallback(bench, monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (bench.FALLBACK_HBM, "fallback")
    tf, kind = bench.tensor_peak_tf32()
    assert abs(tf - bench.FALLBACK_BF16 * 1.1 / 2.25) < 1e-9 and kind.startswith("fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6792.1,
                                                              "bf16_tflops": 2000.0}))
    assert bench.peaks() == (6792.1, "measured")
    tf, kind = bench.tensor_peak_tf32()
    assert abs(tf - 2000.0 * 1.1 / 2.25) < 1e-9 and kind.startswith("measured")


def test_both_arms_name_the_workload_alike(bench):
    one = bench.config_of("ols_dense_ar1", 1048576, 500, 5000, 1, 1)
    assert one["workload"].startswith("ols_dense_ar1 n=1048576 d=500 m=5000 s=1")
    assert one["parallelism"] == "single GPU"
    assert "2.10 GB" in one["l2"]
    assert bench.config_of("ols_dense_ar1", 1048576, 500, 5000, 1, 4)["parallelism"] == "replicas"


def test_reference_arm_runs_on_rank_zero_only(bench):
    """Under a 2-rank launch, the reference arm (the oracle on the host
    cores) runs and prints one JSON line on rank 0 only; rank 1 exits 0
    without work or output.  The line carries the contract's keys: impl,
    the same metric and workload as this library's arm, a cpu_baseline of
    kind oracle, and an e2e object with no host-device bytes."""
    import subprocess
    base = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
            "--warmup", "0", "--cpu-rows", "20000", "--ref-step-budget", "1"]
    outs = {}
    for rank in (1, 0):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
        p = subprocess.run(base, capture_output=True, text=True, env=env, timeout=600)
        assert p.returncode == 0, p.stderr[-2000:]
        outs[rank] = p.stdout.strip()
    assert outs[1] == ""
    lines = outs[0].splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["n_gpus"] == 2 and d["steps"] == 1 and d["higher_is_better"] is False
    assert d["config"]["workload"] == bench.config_of("ols_dense_ar1", 1048576, 500, 5000, 1,
                                                      2)["workload"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
