"""The measurement records under profiles/: every ncu command they quote
leaves the GPU clocks alone, and the scatter pass's DRAM-traffic record is
read by bench.py only while it matches the kernel source it was taken on.
CPU only."""
import glob
import json
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _ncu_commands(text):
    """Each quoted ncu command, with its continuation lines joined."""
    joined = re.sub(r"\\\n\s*", " ", text)
    cmds = []
    for line in joined.splitlines():
        line = line.strip()
        if re.match(r"(\w+=\S+\s+)*ncu ", line):
            cmds.append(line)
        cmds += re.findall(r"`(ncu [^`]*)`", line)
    return cmds


def test_every_ncu_command_keeps_clock_control_off():
    files = glob.glob(os.path.join(ROOT, "profiles", "*.md")) + glob.glob(os.path.join(ROOT, "profiles", "*.json"))
    assert files
    seen = 0
    for path in files:
        text = open(path).read()
        if path.endswith(".json"):
            text = json.load(open(path)).get("command", "")
        for cmd in _ncu_commands(text):
            seen += 1
            assert "--clock-control none" in cmd, (os.path.basename(path), cmd)
    assert seen >= 5


def test_traffic_record_fields():
    rec = json.load(open(os.path.join(ROOT, "profiles", "radix_onesweep_traffic.json")))
    for key in ("dram_bytes_read", "dram_bytes_write", "keys", "dram_bytes_per_key", "algorithmic_bytes_per_key",
                "command", "sources_sha256"):
        assert key in rec, key
    per_key = (rec["dram_bytes_read"] + rec["dram_bytes_write"]) / rec["keys"]
    assert abs(per_key - rec["dram_bytes_per_key"]) < 1e-3
    # DRAM traffic of a key-only pass cannot fall far below the keys read once
    assert 8 <= rec["dram_bytes_per_key"] <= 2 * rec["algorithmic_bytes_per_key"]


def test_traffic_record_is_dropped_when_the_kernel_source_differs(monkeypatch):
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "radix_onesweep_traffic.json")))
    monkeypatch.setattr(bench, "sort_sources_sha", lambda: rec["sources_sha256"])
    assert bench._traffic_record() is not None
    monkeypatch.setattr(bench, "sort_sources_sha", lambda: "0" * 64)
    assert bench._traffic_record() is None
