"""The product path has no CPU fallback: the package never imports the
oracle (test infrastructure), and a missing library raises instead of
degrading.  Static and subprocess checks, no GPU."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2604_20731_gb300")


def _imports(path):
    tree = ast.parse(open(path).read())
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom) and node.module:
            yield node.module


def test_package_never_imports_the_oracle():
    for fn in os.listdir(PKG):
        if fn.endswith(".py"):
            mods = list(_imports(os.path.join(PKG, fn)))
            assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), (fn, mods)


def test_missing_library_raises():
    code = ("from paper_2604_20731_gb300 import _lib\n"
            "try:\n"
            "    _lib.load('/nonexistent/libadsgb.so')\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "else:\n"
            "    print('loaded')\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("raised:") and "not found" in out.stdout
