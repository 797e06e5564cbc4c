"""bench.py's roofline divides the DRAM bytes that ncu measured for one sweep
launch (kept in profiles/traffic.json) by the timed sweep.  The default
configuration must find its entry, or the line's roofline would silently be
null; and each entry must be a byte count below what a dense sweep would
move (48 B per triplet in FP64), since the filtered kernel moves only the
nonzero-dual bits and the nonzero duals."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(monkeypatch, argv):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    return bench, bench.parse()


def test_default_configuration_finds_its_traffic(monkeypatch):
    bench, args = _bench(monkeypatch, [])
    t = bench._profiled_traffic(args)
    assert isinstance(t, int) and t > 0


def test_precision_and_store_forms_find_their_traffic(monkeypatch):
    for argv in (["--precision", "fp32_refine"], ["--store", "sparse"]):
        bench, args = _bench(monkeypatch, argv)
        assert bench._profiled_traffic(args) is not None, argv


def test_other_workloads_have_no_traffic(monkeypatch):
    bench, args = _bench(monkeypatch, ["--workload", "planted60"])
    assert bench._profiled_traffic(args) is None


def test_traffic_entries_are_below_the_dense_sweep_bytes():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        t = json.load(fh)
    n = 1000
    dense = 48 * n * (n - 1) * (n - 2) // 6
    entries = {k: v for k, v in t.items() if k != "note"}
    assert entries
    for k, v in entries.items():
        assert k.startswith("chunglu1000/"), k
        assert isinstance(v, int) and 0 < v < dense, (k, v)
