"""Host arithmetic of the benchmark line (no GPU): the emit's algorithmic
bytes are the stated formula of the tick's counters and leaf footprint, so
the line's `roofline.terms_per_launch` reproduce them; the committed DRAM
capture is read only while the emit kernel's sources hash to it, and is
scaled by results; an optional leg that raises is recorded, not lost."""
import pytest

import bench


def _stats(**kw):
    s = dict(n_objects=4_000_000, n_queries=400_000, n_results=0, n_bitmap_words=0,
             n_sub_intersecting=0, n_covering_runs=0, n_filter_loads=0, n_leaves=0,
             n_pairs=0, n_candidates=0)
    s.update(kw)
    return s


def test_emit_bytes_follow_the_stated_formula():
    s = _stats(n_results=1000, n_bitmap_words=70, n_sub_intersecting=40, n_covering_runs=9)
    fp = {"result_leaf_objects": 300, "tested_leaf_objects": 500}
    for elem, out in ((8, 1000), (4, 1000), (8, 12)):
        got = bench.phase_bytes(s, 10, 10, out, fp, elem)["emit"]
        assert got == elem * out + 4 * 70 + 20 * (40 + 9) + 4 * 300
    assert bench.PHASE_FORMULA["emit"] == \
        "out_elem_bytes*out_elems + 4*bitmap_words + 20*records + 4*result_leaf_objects"
    # the filter's bytes count the tested leaves' objects once, the rest per subquery / word
    assert bench.phase_bytes(s, 10, 10, 1000, fp, 8)["filter"] == 8 * 500 + 24 * 40 + 4 * 70


def test_traffic_capture_is_read_only_for_matching_sources_and_scaled_by_results(tmp_path, monkeypatch):
    cap = tmp_path / "traffic.txt"
    cap.write_text("# comment\nkernel=emit_kernel\nsource_hash=%s\ndram_bytes_per_launch=1000\nresults=100\n"
                   % bench.source_hash("emit_kernel"))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(cap))
    assert bench.read_traffic("emit_kernel", 250) == pytest.approx(2500.0)
    cap.write_text("kernel=emit_kernel\nsource_hash=0000000000000000\ndram_bytes_per_launch=1000\nresults=100\n")
    assert bench.read_traffic("emit_kernel", 250) is None
    assert bench.read_traffic("filter_kernel", 250) is None


def test_a_failing_optional_leg_is_recorded():
    def boom():
        raise RuntimeError("no link")
    r = bench.guarded("e2e", boom)
    assert "no link" in r["error"]
    assert bench.guarded("e2e", lambda: {"value": 1.0}) == {"value": 1.0}
