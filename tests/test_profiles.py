"""The profile summaries stay runnable: every `python bench.py ...` command they give parses with
the benchmark's own argument parser, every ncu command keeps --clock-control none, and every
summary names the command that made it."""
import glob
import os
import re
import shlex
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def bench_commands(text):
    """The bench.py argument lists in a summary (continuation lines joined, shell tails cut)."""
    text = text.replace("\\\n", " ")
    out = []
    for m in re.finditer(r"python bench\.py([^\n`]*)", text):
        args = shlex.split(m.group(1).split(">")[0].split("&&")[0])
        out.append(args)
    return out


def test_there_are_profiles():
    assert len(PROFILES) >= 4


@pytest.mark.parametrize("path", PROFILES, ids=[os.path.basename(p) for p in PROFILES])
def test_profile_commands_parse(path, monkeypatch):
    text = open(path).read()
    assert "Command" in text
    cmds = bench_commands(text)
    assert cmds, "no bench.py command"
    for args in cmds:
        monkeypatch.setattr(sys, "argv", ["bench.py"] + args)
        bench.parse()
    for line in text.replace("\\\n", " ").splitlines():
        if re.match(r"\s*ncu ", line):
            assert "--clock-control none" in line, line
