"""Autotuner host logic: shape keys and the JSON cache (no GPU)."""
from paper_2201_13309_gb300 import autotune


def test_shape_key_buckets():
    k1 = autotune.shape_key("GB300", "rows", 2048, 401, 1001, "f32", "fp32")
    k2 = autotune.shape_key("GB300", "rows", 2048, 450, 1020, "f32", "fp32")
    k3 = autotune.shape_key("GB300", "rows", 2048, 600, 1001, "f32", "fp32")
    assert k1 == k2 and k1 != k3
    assert "W2048" in k1 and "K512" in k1 and "B1024" in k1


def test_cache_roundtrip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("DR_TUNE_CACHE", str(path))
    assert autotune.load_cache() == {}
    autotune.store_cache("a", {"tile_cols": 128, "bin_groups": 16, "ms": 1.0})
    autotune.store_cache("b", {"tile_cols": 64, "bin_groups": 8, "ms": 2.0})
    c = autotune.load_cache()
    assert c["a"]["bin_groups"] == 16 and c["b"]["tile_cols"] == 64
    path.write_text("not json")
    assert autotune.load_cache() == {}


def test_candidates_cover_both_kernels():
    assert all(tc % 8 == 0 for tc, _ in autotune.candidates("rows"))
    assert all((tc in (8, 16) or tc % 32 == 0) and tc * bg <= 512
               for tc, bg in autotune.candidates("pixels"))
