"""The DRAM-traffic table that bench.py reads for the roofline's `traffic`
field: every 2D entry is keyed workload:precision:step kernel, records the
kernel it was captured on and the sha256 of the step sources, and its total is
its read plus its write bytes. (Whether the sha256 still matches the sources
is decided by bench.py at run time: a stale entry reads as null.)"""
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_entries_are_consistent():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert t
    for key, e in t.items():
        assert e["bytes_per_launch"] == e["read"] + e["write"], key
        assert re.fullmatch(r"[0-9a-f]{64}", e["step_source_sha256"]), key
        wl, prec, rest = key.split(":", 2)
        assert prec in ("fp32", "fp64", "bf16", "fp16"), key
        if not wl.endswith("3d"):
            assert rest in ("global", "pair", "staged32x8", "staged64x4"), key
            assert e["kernel"].startswith("k_step"), key

