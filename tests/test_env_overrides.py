"""Environment overrides, on the host: DTE_PLAN gives committed types a
kernel plan (read once per process, so each case runs in a fresh
interpreter); an unknown name leaves the fixed rule."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SNIPPET = r"""
import paper_2402_12274_gb300 as dte
t = dte.Datatype.vector(64, 4, 8, dte.FLOAT32)
before = dte.dte_type_get_plan(t.h)
t.commit()
after = dte.dte_type_get_plan(t.h)
u = dte.Datatype.vector(64, 4, 8, dte.FLOAT32)
dte.dte_type_set_plan(u.h, dte.PLAN_CHUNK)
u.commit()
print(before, after, dte.dte_type_get_plan(u.h))
"""


def run(env_plan):
    env = dict(os.environ)
    env.pop("DTE_PLAN", None)
    if env_plan is not None:
        env["DTE_PLAN"] = env_plan
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    out = subprocess.run([sys.executable, "-c", SNIPPET], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    return [int(x) for x in out.stdout.split()]


@pytest.mark.parametrize("name,plan", [("segment", 3), ("chunk_wide", 2), ("bulk", 4)])
def test_env_plan_applies_at_commit(name, plan):
    import paper_2402_12274_gb300 as dte
    assert getattr(dte, "PLAN_" + name.upper()) == plan
    # auto before commit, the named plan after; an explicit plan is kept
    assert run(name) == [0, plan, 1]


def test_env_plan_unset_or_unknown_keeps_the_rule():
    assert run(None) == [0, 0, 1]
    assert run("fastest") == [0, 0, 1]
