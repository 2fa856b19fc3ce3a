"""Every command recorded in a profile summary under profiles/ runs committed files only:
each `python <file>` names a file of this repository, each `python -m <module>` a module
of it, and every bench.py invocation parses with bench.py's own argument parser (so a
summary cannot keep a command whose script or flag has since gone)."""
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _commands(path):
    """Shell commands of the fenced code blocks of a summary (continuation lines joined)."""
    text = open(path, encoding="utf-8").read()
    out = []
    for block in re.findall(r"```[a-z]*\n(.*?)```", text, flags=re.S):
        joined = re.sub(r"\\\n\s*", " ", block)
        out += [line.strip() for line in joined.splitlines() if line.strip()]
    return out


def _python_invocations(cmd):
    """(script, args) or ('-m', module, args) for each `python ...` inside a command,
    including one wrapped by ncu."""
    toks = shlex.split(cmd)
    found = []
    for i, t in enumerate(toks):
        if t in ("python", "python3"):
            rest = toks[i + 1:]
            if rest and rest[0] == "-m":
                found.append(("-m", rest[1], rest[2:]))
            elif rest and rest[0] == "-c":
                continue
            elif rest:
                found.append((rest[0], rest[1:]))
    return found


SUMMARIES = sorted(f for f in os.listdir(PROFILES) if f.endswith(".md"))


def test_profiles_exist():
    assert SUMMARIES, "no profile summaries under profiles/"


@pytest.mark.parametrize("name", SUMMARIES)
def test_profile_commands_run_committed_files(name, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    for cmd in _commands(os.path.join(PROFILES, name)):
        if cmd.startswith("ncu"):
            assert "--clock-control none" in cmd, f"{name}: ncu without --clock-control none"
        for inv in _python_invocations(cmd):
            if inv[0] == "-m":
                mod = inv[1]
                rel = mod.replace(".", os.sep)
                assert (os.path.exists(os.path.join(ROOT, rel + ".py"))
                        or os.path.isdir(os.path.join(ROOT, rel))), f"{name}: no module {mod}"
                continue
            script, args = inv
            assert os.path.exists(os.path.join(ROOT, script)), f"{name}: no file {script}"
            if os.path.basename(script) == "bench.py":
                monkeypatch.setattr(sys, "argv", ["bench.py", *args])
                try:
                    bench.parse()
                except SystemExit as e:  # argparse rejects an unknown or malformed flag
                    pytest.fail(f"{name}: bench.py rejects {args} ({e})")
