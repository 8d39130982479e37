"""Host-side checks of bench.py's command line (no GPU needed)."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, timeout=300)


def test_reduced_ghost_depth_needs_the_fused_form():
    for form in ("3pass", "auto"):
        r = run("--form", form, "--ghost", "1")
        assert r.returncode == 2
        assert "--ghost 1 or 2 needs --form fused" in r.stderr


def test_ghost_depth_choices():
    r = run("--form", "fused", "--ghost", "4")
    assert r.returncode == 2 and "invalid choice" in r.stderr
