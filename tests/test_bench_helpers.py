"""Host-side helpers of the benchmark (no GPU): the whole-job throughput of
independent replicas, the search kernel's source hash and the committed
profile's DRAM traffic, which is reported only while the kernel source is
the one the counters were taken on."""
import importlib

import pytest


@pytest.fixture(scope="module")
def bench():
    return importlib.import_module("bench")


def test_replica_value(bench):
    # 3 replicas, 10 units each, slowest rank 20 ms -> 30 units / 0.02 s
    assert bench.replica_value(10, 3, 20.0) == pytest.approx(1500.0)
    assert bench.replica_value(5, 1, 1000.0) == pytest.approx(5.0)


def test_search_kernel_hash_is_stable(bench):
    h = bench.search_kernel_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    assert bench.search_kernel_hash() == h


def test_search_kernel_hash_covers_section_and_thresholds(bench, tmp_path, monkeypatch):
    """The hash changes with the search section's text and with the lookup
    thresholds defined outside it, and not with other code."""
    src = open(bench.KERNEL_SRC).read()
    h0 = bench.search_kernel_hash()

    def hash_of(text):
        f = tmp_path / "k.cu"
        f.write_text(text)
        monkeypatch.setattr(bench, "KERNEL_SRC", str(f))
        return bench.search_kernel_hash()

    assert hash_of(src) == h0
    coop = [ln for ln in src.splitlines() if ln.startswith("constexpr int32_t kCoopMin")]
    assert len(coop) == 1
    assert hash_of(src.replace(coop[0], coop[0].replace("=", "= 1 +"))) != h0
    a = src.index("// Steps A + B + C (Algorithms 3, 4, 5)") + 40
    assert hash_of(src[:a] + "\n// inside\n" + src[a:]) != h0
    b = src.index("// Step D (Algorithm 6)") + len("// Step D (Algorithm 6)")
    assert hash_of(src[:b] + "\n// elsewhere\n" + src[b:]) == h0


def write_profile(path, sha, traffic):
    import json
    path.write_text(json.dumps({"kernel_source_sha256_16": sha, "dram_bytes_per_launch": traffic,
                                "l2_sector_hit_rate_pct": 59.0}))


def test_profile_traffic_follows_the_source_hash(bench, tmp_path, monkeypatch):
    prof = tmp_path / "p.json"
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    write_profile(prof, bench.search_kernel_hash(), 123456789)
    assert bench.profile_traffic() == 123456789.0
    # counters taken on another version of the kernel are not reported
    write_profile(prof, "0" * 16, 123456789)
    assert bench.profile_traffic() is None
    # no profile at all
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "missing.json"))
    assert bench.profile_traffic() is None


def test_profile_traffic_rejects_malformed_values(bench, tmp_path, monkeypatch):
    prof = tmp_path / "p.json"
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    write_profile(prof, bench.search_kernel_hash(), "n/a")
    assert bench.profile_traffic() is None


def test_committed_profile_record_is_well_formed(bench):
    import json
    rec = json.load(open(bench.PROFILE))
    for k in ("kernel_source_sha256_16", "dram_bytes_read", "dram_bytes_write",
              "dram_bytes_per_launch", "l2_sector_hit_rate_pct", "gpu_time_ns", "command"):
        assert k in rec, k
    assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    assert "--clock-control none" in rec["command"] and "-c 1" in rec["command"]


def test_profile_record_garbage_is_none(bench, tmp_path, monkeypatch):
    prof = tmp_path / "p.json"
    prof.write_text("not json")
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench.profile_record() is None and bench.profile_traffic() is None
