"""The product path has no CPU fallback: the binding refuses to load without the built
CUDA library, and no file of the package imports the oracle."""
import os
import re
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2110_15676_gb300")


def test_binding_without_library_raises_import_error():
    with tempfile.TemporaryDirectory() as d:
        pkg = os.path.join(d, "paper_2110_15676_gb300")
        os.makedirs(pkg)
        for f in ("__init__.py", "afc.py"):
            src = os.path.join(PKG, f)
            if os.path.exists(src):
                shutil.copy(src, pkg)
        os.makedirs(os.path.join(d, "include"))
        shutil.copy(os.path.join(ROOT, "include", "afc.h"), os.path.join(d, "include"))
        r = subprocess.run([sys.executable, "-c", "import paper_2110_15676_gb300.afc"], cwd=d,
                           capture_output=True, text=True, env={**os.environ, "PYTHONPATH": d})
        assert r.returncode != 0
        assert "ImportError" in r.stderr and "libafc.so is not built" in r.stderr


def test_package_does_not_import_the_oracle():
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b|from\s+\.\.?oracle\b)", re.M)
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                with open(os.path.join(dirpath, f), errors="replace") as fh:
                    text = fh.read()
                assert not pat.search(text), f
                assert "afc_oracle" not in text, f
