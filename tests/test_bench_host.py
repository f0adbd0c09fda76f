"""Host-side logic of bench.py that needs no GPU: the captured-traffic
table (valid only for the captured sources and the launched kernel), the
workload names it is keyed by, and the CPU description of the baseline."""
import hashlib
import os
import platform
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sources_sha(rec):
    h = hashlib.sha1()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, "paper_0903_4044_gb300", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def test_traffic_needs_the_captured_kernel_and_sources():
    for (name, prec), rec in bench.MEASURED_TRAFFIC.items():
        assert bench.measured_traffic(name, prec, "bgk::some_other_kernel") is None
        got = bench.measured_traffic(name, prec, rec["kernel"])
        if _sources_sha(rec) == rec["sha1"]:
            assert got == rec["bytes"]
        else:
            assert got is None
    assert bench.measured_traffic("no_such_workload", "f64", "bgk::step_f64_kernel") is None


def test_traffic_keys_are_benchmark_workload_names():
    # the table is keyed by the names the benchmark's workloads carry
    names = {bench.workload(w)["name"] for w in ("cavity64", "cavity256", "shock")}
    for name, _ in bench.MEASURED_TRAFFIC:
        assert name in names, name


def test_cpu_model_names_the_architecture():
    m = bench.cpu_model()
    assert isinstance(m, str) and m.endswith(f"({platform.machine()})")
