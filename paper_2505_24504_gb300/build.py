"""Build libjfnk.so for sm_103a from csrc/ with nvcc (in-tree, no cmake).

Each translation unit compiles in its own nvcc process (in parallel), then one
link step produces paper_2505_24504_gb300/libjfnk.so.  Objects go to
paper_2505_24504_gb300/_build/.  Rebuilds only when a source or header is newer
than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libjfnk.so")
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libjfnk.so")


def sources():
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cu", ".cpp")))


# Translation units compiled more than once with different defines: the DG
# operator kernels once per order k = 1..4 (in parallel).
VARIANTS = {"dg.cu": [("k%d" % (n - 1), ["-DJF_DG_NP1=%d" % n]) for n in (2, 3, 4, 5)]}


def _deps():
    files = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    files.append(os.path.join(ROOT, "include", "jfnk.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    objs = []
    cmds = []
    for s in sources():
        lang = ["-x", "cu"]   # every unit sees the device headers
        for tag, defs in VARIANTS.get(os.path.basename(s), [("", [])]):
            o = os.path.join(OUT, os.path.basename(s) + (("." + tag) if tag else "") + ".o")
            objs.append(o)
            cmds.append([cc, *ARCH, *FLAGS, *defs, *extra, *lang, "-c", s, "-o", o])
    with cf.ThreadPoolExecutor(max_workers=min(12, os.cpu_count() or 4)) as ex:
        res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), cmds))
    for c, r in zip(cmds, res):
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(c) + "\n" + r.stderr)
    tmp = LIB + ".tmp"
    link = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
