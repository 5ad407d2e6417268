"""The product path has no CPU fallback: without its CUDA library the binding
raises on the first call, and without a GPU a context cannot be created."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(code):
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)


def test_missing_library_raises():
    r = _run("import paper_2606_21883_b300 as M\n"
             "M.LIB_PATH = '/nonexistent/libmpwos.so'\n"
             "try:\n"
             "    M.lib()\n"
             "except RuntimeError as e:\n"
             "    print('raised:', e)\n")
    assert r.returncode == 0, r.stderr
    assert "raised:" in r.stdout and "no CPU fallback" in r.stdout


def test_context_needs_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _run("import paper_2606_21883_b300 as M\n"
             "try:\n"
             "    M.Context(0)\n"
             "    print('created')\n"
             "except Exception as e:\n"
             "    print('raised:', type(e).__name__)\n")
    assert r.returncode == 0, r.stderr
    assert "raised:" in r.stdout and "created" not in r.stdout
