"""CPU checks of bench.py's host-side bookkeeping (no GPU): the per-kernel source hashes that
decide whether a stored ncu traffic figure still describes the kernel, the traffic table's
keys, and the config object both bench arms print."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_sources_exist_and_hash_differs_per_storage():
    csrc = os.path.join(ROOT, "paper_2310_14746_gb300", "csrc")
    for storage, names in bench.KERNEL_SOURCES.items():
        for n in names:
            assert os.path.exists(os.path.join(csrc, n)), (storage, n)
    hashes = {s: bench.kernel_source_hash("stream_collide_d3q19_%s_two" % s) for s in bench.KERNEL_SOURCES}
    assert len(set(hashes.values())) == len(hashes)
    # the hash depends on the storage's sources only, not on the streaming pattern
    assert bench.kernel_source_hash("stream_collide_d3q19_f16_aa") == hashes["f16"]


def test_traffic_entries_name_bench_workloads():
    workloads = {("stream_collide_d3q19_%s_%s" % (w["storage"], w["pattern"]), w["n"]) for w in bench.WORKLOADS.values()}
    for (kname, n), e in bench.KERNEL_TRAFFIC_BYTES.items():
        assert (kname, n) in workloads, kname
        storage = kname.split("_")[3]
        bpl = 2 * 19 * {"f32": 4, "f16": 2, "bf16": 2, "f64": 8}[storage] + 4
        # DRAM traffic of a clean stream-collide launch is within a few percent of its algorithmic bytes
        assert 0.9 < e["bytes"] / (bpl * n ** 3) < 1.02, kname
        assert len(e["source_hash"]) == 16


def test_traffic_is_null_when_sources_changed(monkeypatch):
    key = ("stream_collide_d3q19_f32_two", 256)
    entry = dict(bench.KERNEL_TRAFFIC_BYTES[key])
    monkeypatch.setitem(bench.KERNEL_TRAFFIC_BYTES, key, dict(entry, source_hash="0" * 16))
    traffic, note = bench.kernel_traffic(*key)
    assert traffic is None and note.startswith("stale")
    assert bench.kernel_traffic("stream_collide_d3q19_f32_two", 128) == (None, "not captured")


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_both_arms_share_the_config_object(name):
    w = bench.WORKLOADS[name]
    c1 = bench.workload_config(w, 100, 1)
    assert c1 == bench.workload_config(w, 100, 1)
    assert c1["workload"] == w["desc"] and c1["cells"] == w["n"] ** 3
    assert c1["parallelism"] == "single" and bench.workload_config(w, 100, 4)["parallelism"] == "replicas"
