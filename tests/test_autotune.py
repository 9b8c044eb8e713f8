"""Autotuner: picks the fastest variant, records every candidate in its JSON cache, and
best_variant() reads it back (CPU, with a fake measurement); on a GPU it tunes N = 4096, where
the variants span radix 16 and radix 8."""
import json

import pytest


def test_tune_records_fastest(tmp_path, monkeypatch):
    from paper_2107_06147_gb300 import autotune, qtraj
    monkeypatch.setenv("QTRAJ_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    rates = {0: 10.0, 1: 12.0, 2: 11.0, 3: 9.0}
    rec = autotune.tune(4096, qtraj.FP32, measure_fn=lambda v: {"variant": v, "rate": rates[v]})
    assert rec["variant"] == 1
    assert autotune.best_variant(4096, qtraj.FP32) == 1
    assert autotune.best_variant(1024, qtraj.FP32) == 0          # not tuned -> default
    data = json.loads((tmp_path / "tune.json").read_text())
    assert len(data["N=4096,precision=fp32"]["candidates"]) == 4


@pytest.mark.gpu
def test_tune_on_gpu(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_06147_gb300 import autotune, build, qtraj
    build.build()
    monkeypatch.setenv("QTRAJ_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    rec = autotune.tune(4096, qtraj.FP32, steps=100)
    assert rec["variant"] in autotune.VARIANTS
    assert all(c["rate"] > 0 for c in rec["candidates"])
    assert {c["radix"] for c in rec["candidates"]} == {8, 16}
