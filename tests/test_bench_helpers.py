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


def write_profile(path, sha, traffic):
    path.write_text("# profile\n\n"
                    f"- kernel_source_sha256_16: `{sha}`\n"
                    f"- dram_bytes_per_launch: `{traffic}`\n")


def test_profile_traffic_follows_the_source_hash(bench, tmp_path, monkeypatch):
    prof = tmp_path / "p.md"
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    write_profile(prof, bench.search_kernel_hash(), 123456789)
    assert bench.profile_traffic() == 123456789.0
    # counters taken on another version of the kernel are not reported
    write_profile(prof, "0" * 16, 123456789)
    assert bench.profile_traffic() is None
    # no profile at all
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "missing.md"))
    assert bench.profile_traffic() is None


def test_profile_traffic_rejects_malformed_values(bench, tmp_path, monkeypatch):
    prof = tmp_path / "p.md"
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    write_profile(prof, bench.search_kernel_hash(), "n/a")
    assert bench.profile_traffic() is None
