"""CPU checks of the bench's roofline arithmetic: the dominant peel tier, its
algorithmic bytes per launch (4 B per wedge, 16 B per middle vertex, 16 B
per support atomic, 24 B per anchor), and the DRAM traffic figure, which is
reported only while the kernel sources match the ones it was captured on."""
import bench

STATS = {"ms_peel": [1.0, 2.0, 0.5, 10.0, 3.0], "peel_launches": [10, 10, 10, 10, 10],
         "peel_wedges": [5, 6, 7, 1000, 8], "peel_mids": [1, 1, 1, 10, 1],
         "peel_pairs": [2, 2, 2, 100, 2], "peel_anchors": [1, 1, 1, 2, 1]}


def test_roofline_of_the_busiest_tier():
    r = bench.roofline(STATS, 1000.0, "measured")
    assert r["kernel"] == "k_cd_update_slice" and r["launches"] == 10
    per_launch = (4 * 1000 + 16 * 10 + 16 * 100 + 24 * 2) / 10
    assert r["bytes_per_launch"] == per_launch
    launch_s = 10.0 / 1e3 / 10
    assert abs(r["launch_ms"] - launch_s * 1e3) < 1e-12
    assert abs(r["achieved"] - per_launch / launch_s / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1000.0) < 1e-12
    st = dict(STATS, ms_peel=[1.0, 20.0, 0.5, 10.0, 3.0])
    assert bench.roofline(st, 1000.0, "measured")["kernel"] == "k_cd_update_cta"


def test_traffic_only_for_the_captured_sources(monkeypatch):
    per_launch = (4 * 1000 + 16 * 10 + 16 * 100 + 24 * 2) / 10
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {
        "k_cd_update_slice": {"src": bench._src_digest(), "dram_per_alg_byte": 0.25}})
    assert bench.roofline(STATS, 1000.0, "measured")["traffic"] == int(0.25 * per_launch)
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {
        "k_cd_update_slice": {"src": "0" * 16, "dram_per_alg_byte": 0.25}})
    assert bench.roofline(STATS, 1000.0, "measured")["traffic"] is None
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {})
    assert bench.roofline(STATS, 1000.0, "measured")["traffic"] is None
