"""Autotuner table logic on the CPU: shape classes and lookups."""
import json

from paper_2010_08695_gb300 import autotune


def test_shape_class_buckets_by_powers_of_two():
    a = autotune.shape_class(1_000_000, 200_000, 10_000_000, 0, 43649)
    b = autotune.shape_class(1_050_000, 190_000, 10_400_000, 0, 45000)
    assert a == b == "s20-o18-m23-d15"
    assert autotune.shape_class(200_000, 1_000_000, 10_000_000, 1, 43649) == a


def test_lookup_reads_the_table(tmp_path, monkeypatch):
    path = tmp_path / "t.json"
    path.write_text(json.dumps({"s1-o1-m1-d1": {"warp_max_w": 64, "slice_min_w": 5}}))
    monkeypatch.setenv("RECEIPT_TUNING", str(path))
    monkeypatch.setattr(autotune, "_table", None)
    assert autotune.lookup("s1-o1-m1-d1")["slice_min_w"] == 5
    assert autotune.lookup("nope") is None
    monkeypatch.setattr(autotune, "_table", None)


def test_shipped_table_is_valid():
    with open(autotune.SHIPPED) as f:
        table = json.load(f)
    for key, rec in table.items():
        assert 0 < rec["warp_max_w"] <= 256 and rec["slice_min_w"] > 0


def test_coordinate_search_picks_the_fastest_setting():
    """The search visits every knob's candidates and keeps the fastest
    combination (a synthetic cost with a known optimum, no GPU)."""
    best = {"slice_ctas": 2, "slice_fetch": 4, "warp_max_w": 128, "slice_min_w": 98304,
            "P": 300, "range_max_n": -1, "dgm_frac_1024": 64}
    calls = []

    def cost(run, reps, **o):
        calls.append(o)
        return 1.0 + sum(o[k] != v for k, v in best.items())
    rec, times = autotune.search(lambda **o: None, 1_000_000, time_fn=cost)
    assert {k: rec[k] for k in best} == best and rec["ms"] == 1.0
    assert len(times) == len(calls)


def test_tuned_range_cap_follows_P():
    # the table's vertex cap was tuned with its own P: another P keeps
    # cap * P, and the special values stay
    import paper_2010_08695_gb300 as R
    rec = {"P": 200, "range_max_n": 6666}
    assert R._tuned_cap(rec, 200) == 6666
    assert R._tuned_cap(rec, 25) == 53328
    assert R._tuned_cap(rec, 400) == 3333
    assert R._tuned_cap({"P": 200, "range_max_n": -1}, 25) == -1
    assert R._tuned_cap({"P": 200, "range_max_n": 0}, 25) == 0
    assert R._tuned_cap({"range_max_n": 500}, 25) == 500
