"""The committed ncu summaries: each names the command that made it (ncu with
--clock-control none, after the same command run without ncu), and the DRAM
traffic table points at summaries that exist."""
import glob
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def test_every_summary_gives_its_command():
    files = sorted(glob.glob(os.path.join(PROF, "*.md")))
    assert files
    for f in files:
        text = open(f).read()
        assert "```" in text, f
        cmd = text.split("```")[1]
        assert "ncu " in cmd and "--clock-control none" in cmd, f
        assert "bench.py" in cmd, f
        # the plain run of the same command comes first
        assert cmd.index("> plain.log") < cmd.index("ncu "), f


def test_traffic_table_points_at_summaries():
    t = json.load(open(os.path.join(PROF, "traffic.json")))
    assert len(t["k_stage_sha1"]) == 40
    for k, v in t.items():
        if not isinstance(v, dict):
            continue
        assert v["bytes"] > 0, k
        md = [w for w in v["capture"].replace(",", " ").split() if w.startswith("profiles/")]
        assert md and all(os.path.exists(os.path.join(ROOT, p)) for p in md), k
