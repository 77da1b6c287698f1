"""Host-side helpers of bench.py (no GPU): the stored-root loader, the
committed ncu traffic lookup with its kernel-source guard, and the headline
latency pick from the serving block."""
import importlib.util
import os

import numpy as np
import pytest

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def _make_roots():
    sp = importlib.util.spec_from_file_location("make_roots", os.path.join(HERE, "golden", "make_roots.py"))
    mod = importlib.util.module_from_spec(sp)
    sp.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,blocks,has_phi", [("oracle_root_181x61.txt", 1, True),
                                                 ("oracle_root_121x41_batch.txt", 2, False)])
def test_root_loader_matches_the_writer_script(name, blocks, has_phi):
    path = os.path.join(HERE, "golden", name)
    a, b = bench.load_roots(path), _make_roots().load(path)
    assert len(a) == len(b) == blocks
    for (ha, za, pa), (hb, zb, pb) in zip(a, b):
        assert ha == hb and np.array_equal(za, zb)
        assert (pa is not None) == has_phi and (pa is None or np.array_equal(pa, pb))
        assert za.shape == (ha["M"], ha["N"]) and ha["final_norm_inf"] < 1e-11


def test_traffic_lookup_and_source_guard(tmp_path, monkeypatch):
    b, note = bench.measured_traffic("k_pairs_x2r<2,256,2,0,1>")
    assert b is not None and 705_000 < b < 1.05 * 705_000, (b, note)   # algorithmic bytes 705 KB
    assert bench.measured_traffic("k_pairs_x2r<9,9,9,9,9>")[0] is None
    other = tmp_path / "pairs.cu"
    other.write_text("// a different kernel source\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(other))
    b2, note2 = bench.measured_traffic("k_pairs_x2r<2,256,2,0,1>")
    assert b2 is None and "changed" in note2


def test_headline_latency_is_the_mixed_block_at_its_saturated_rate():
    pt = lambda f, p50: {"rate_factor": f, "requests": 8, "latency_ms": {"p50": p50, "p99": 2 * p50}}
    serve = {"mixed": {"points": [pt("saturated", 900.0), pt(1.0, 100.0), pt(0.5, 10.0)]}}
    lat = bench.serve_latency(serve)
    assert lat["p50"] == 100.0 and lat["p99"] == 200.0 and "1.0 x" in lat["source"]
    assert bench.serve_latency(None) is None and bench.serve_latency({"fp64": {}}) is None
