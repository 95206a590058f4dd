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


def test_select_needs_both_bounds():
    """The tuner keeps the fastest candidate within half of both the R and
    the E_L bound; with the energy bound off (etol_rel = 0) R alone decides."""
    from paper_1810_08142_gb300 import tune
    res = [{"mode": "bf16x3", "ms": 250.0, "err": 4e-6, "eerr": 3e-6},
           {"mode": "bf16x6", "ms": 350.0, "err": 4e-7, "eerr": 4e-7},
           {"mode": "ozaki", "ms": 860.0, "err": 3e-12, "eerr": 2e-14},
           {"mode": "ozaki", "ms": 1110.0, "err": 1e-13, "eerr": 5e-15}]
    assert tune.select(res, 1e-6, 1e-13)["ms"] == 860.0
    assert tune.select(res, 1e-6, 0.0)["ms"] == 350.0
    assert tune.select(res, 2e-5, 0.0)["ms"] == 250.0
    # nothing meets an energy bound below every candidate: the most accurate in E
    assert tune.select(res, 1e-6, 1e-17)["ms"] == 1110.0
    assert ("ozaki", {"oz_slices": 5}) in tune.candidates((0, 1))


def test_lookup_mode_reads_per_mode_entries(tmp_path, monkeypatch):
    from paper_1810_08142_gb300 import tune
    path = tmp_path / "cache.json"
    monkeypatch.setenv("LADDER_TUNE_CACHE", str(path))
    path.write_text(json.dumps({
        "34,400,1600": {"mode": "ozaki", "tuning": {"oz_slices": 5},
                        "by_mode": {"bf16x6": {"kc": 4, "flush_every": 128}, "ozaki": {"oz_slices": 5}}},
        "10,120,480": {"mode": "bf16x6", "tuning": {"kc": 8}}}))
    assert tune.lookup(34, 400, 1600) == ("ozaki", {"oz_slices": 5})
    assert tune.lookup_mode(34, 400, 1600, "bf16x6") == {"kc": 4, "flush_every": 128}
    assert tune.lookup_mode(10, 120, 480, "bf16x6") == {"kc": 8}      # older entries without by_mode
    assert tune.lookup_mode(10, 120, 480, "ozaki") is None
    assert tune.lookup_mode(4, 24, 96, "bf16x6") is None
