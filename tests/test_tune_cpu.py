"""Host logic of the autotuner's cache (no GPU): exact and nearest-shape lookup."""
import json


def test_lookup_exact_nearest_and_default(tmp_path, monkeypatch):
    from paper_1810_08142_gb300 import tune
    path = tmp_path / "cache.json"
    monkeypatch.setenv("LADDER_TUNE_CACHE", str(path))
    assert tune.lookup(4, 24, 96) == ("bf16x6", None)
    path.write_text(json.dumps({
        "10,120,480": {"mode": "bf16x6", "tuning": {"kc": 8, "s_pieces": 2, "ksplit": 5}},
        "34,400,1600": {"mode": "bf16x3", "tuning": {"kc": 16, "s_pieces": 4, "ksplit": 1}}}))
    assert tune.lookup(10, 120, 480) == ("bf16x6", {"kc": 8, "s_pieces": 2, "ksplit": 5})
    mode, t = tune.lookup(32, 380, 1500)      # nearest: the large shape, split not carried over
    assert mode == "bf16x3" and t == {"kc": 16, "s_pieces": 4}
