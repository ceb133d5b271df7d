"""The product path has no CPU fallback and never reaches the oracle: without
libsilu.so every call raises, and no library source imports, links or names
the oracle's module or shared library."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2111_09512_gb300")


def test_calls_raise_without_the_library():
    code = (
        "import paper_2111_09512_gb300 as s\n"
        "s.LIB_PATH = '/nonexistent/libsilu.so'\n"
        "s._lib = None\n"
        "try:\n"
        "    s.Context(device=-1)\n"
        "except s.SiluError as e:\n"
        "    print('raised', 'is not built' in str(e))\n"
        "else:\n"
        "    print('no error')\n")
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == "raised True"


def test_library_sources_do_not_reach_the_oracle():
    pat = re.compile(r"import\s+oracle|from\s+oracle|liboracle|oracle\.c|orc_")
    hits = []
    for d, _, files in os.walk(PKG):
        if "_build" in d:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                with open(os.path.join(d, f), encoding="utf-8") as fh:
                    for i, line in enumerate(fh, 1):
                        if pat.search(line):
                            hits.append(f"{f}:{i}: {line.strip()}")
    assert not hits, hits
