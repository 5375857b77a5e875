"""VP_LOG: with level 1 every error message the library records is also
written to stderr ("vp: <object>: <message>"); unset, the library is silent.
Checked on the host through argument errors, which return before any device
work, in child processes (the level is read once per process)."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHILD = """
import ctypes
from paper_1604_03155_gb300 import vp
lib = vp.lib()
out = ctypes.c_void_p()
assert lib.vp_plan_create(ctypes.byref(out), 5, 32, vp.VP_LAPLACE, 0.0, 0.0) == vp.VP_ERR_INVALID_ARG
assert lib.vp_plan_load(ctypes.byref(out), b"/nonexistent/plan.vpplan") == vp.VP_ERR_INVALID_ARG
"""


def _run(level):
    env = dict(os.environ)
    env.pop("VP_LOG", None)
    if level is not None:
        env["VP_LOG"] = str(level)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return [ln for ln in r.stderr.splitlines() if ln.startswith("vp: ")]


def test_errors_are_logged_at_level_1():
    lines = _run(1)
    assert "vp: plan: d must be 2 or 3" in lines
    assert any(ln.startswith("vp: plan: cannot open: /nonexistent/plan.vpplan") for ln in lines)


def test_silent_by_default():
    assert _run(None) == []
    assert _run(0) == []
