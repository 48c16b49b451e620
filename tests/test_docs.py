"""The design notes and profile summaries point at files that exist, and
every profile summary gives the command that produced it."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2008_12214_gb300")


def _exists(path):
    for base in (ROOT, PKG):
        if glob.glob(os.path.join(base, path)):
            return True
    return False


def test_design_references_exist():
    text = open(os.path.join(ROOT, "DESIGN.md")).read()
    paths = set(re.findall(r"`([A-Za-z0-9_./*-]+\.(?:py|cu|cuh|h|c|md|json|txt))`", text))
    missing = sorted(p for p in paths if "/" in p and not _exists(p))
    assert not missing, missing


def test_profile_summaries_state_their_command():
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(f).read()
        assert "Command" in text and ("bench.py" in text or "ncu" in text), f
