"""The committed profile summaries are text, say how they were made, and every
ncu command in them leaves the GPU clocks alone (--clock-control none)."""
import os
import re

PROF = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")


def _files():
    return sorted(os.listdir(PROF))


def _commands(text):
    """Shell commands of a summary, continuation lines joined."""
    joined = re.sub(r"\\\n\s*", " ", text)
    out = []
    for line in joined.splitlines():
        for part in re.split(r"&&|;", line):
            part = part.strip()
            if part.startswith("ncu "):
                out.append(part)
    return out


def test_summaries_are_text():
    assert _files()
    for f in _files():
        assert f.endswith((".txt", ".md")), f
        assert os.path.getsize(os.path.join(PROF, f)) < 64 * 1024, f


def test_every_summary_gives_its_command():
    for f in _files():
        text = open(os.path.join(PROF, f)).read()
        assert "Command" in text, f
        assert _commands(text), f


def test_every_ncu_command_keeps_the_clocks():
    n = 0
    for f in _files():
        for cmd in _commands(open(os.path.join(PROF, f)).read()):
            if cmd.startswith("ncu -i "):
                continue  # reading a report back, no GPU involved
            assert "--clock-control none" in cmd, (f, cmd)
            n += 1
    assert n >= len(_files())
