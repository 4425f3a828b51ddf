"""The profile summaries are text only, each is listed in the index, and
every ncu command they quote keeps the clocks as they are."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def test_every_summary_is_indexed_and_text():
    index = open(os.path.join(PROF, "README.md")).read()
    for name in sorted(os.listdir(PROF)):
        assert name.endswith((".md", ".txt")), name
        if name != "README.md":
            assert "`%s`" % name in index, name


def test_ncu_commands_leave_the_clocks_alone():
    for name in sorted(os.listdir(PROF)):
        text = open(os.path.join(PROF, name)).read()
        for line in text.splitlines():
            if re.match(r"\s*ncu\s+--", line):  # a command line, not a title
                assert "--clock-control none" in line, (name, line)
