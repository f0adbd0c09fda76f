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


def _args(**kw):
    import argparse

    d = dict(workload="cavity256", precision="f64", time_steps=None, checkpoint_every=100, persistent=False,
             gpus=1)
    d.update(kw)
    return argparse.Namespace(**d)


def test_both_arms_print_the_same_config():
    # the reference arm and the GPU arm build `config` from the same function
    # and the same resolved workload, so the driver can pair their lines
    for wl in ("cavity256", "cavity64", "shock", "adjoint", "shock3v", "batch"):
        a = _args(workload=wl)
        w = bench.resolve_workload(a)
        c = bench.config_for(a, w, 1)
        assert c == bench.config_for(_args(workload=wl), bench.resolve_workload(_args(workload=wl)), 1)
        assert "workload" in c and "l2" in c and "precision" in c
    d = bench.config_for(_args(), bench.resolve_workload(_args()), 1)
    assert d["workload"] == bench.CAVITY256_200
    assert d["cells"] == 256 * 256 and d["velocities"] == 48 * 48 and d["time_steps"] == 200


def test_default_workload_is_the_256_cavity():

    import inspect

    src = inspect.getsource(bench.main)
    assert 'default="cavity256"' in src
