"""Build libsevennet.so in-tree for sm_103a with nvcc (no cmake, no torch).

Steps: generate csrc/cg_tables.cuh from gen_cg.py, compile every csrc/*.cu to
an object in parallel, link a shared library next to this file (lib/).
"""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libsevennet.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + INCLUDE, "-I" + CSRC]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    return r.returncode, " ".join(cmd), r.stdout


def build(verbose: bool = False, extra_flags=None, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    gen = os.path.join(CSRC, "gen_cg.py")
    cg = os.path.join(CSRC, "cg_tables.cuh")
    subprocess.run([sys.executable, gen, cg], check=True, stdout=subprocess.DEVNULL)
    nv = nvcc()
    flags = NVCC_FLAGS + ARCH + list(extra_flags or [])
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "sevennet.h"))
    newest_header = max(os.path.getmtime(h) for h in headers)
    jobs = []
    objs = []
    for src in sources():
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src[:-3] + ".o")
        objs.append(o)
        if (not force and os.path.exists(o) and os.path.getmtime(o) > os.path.getmtime(s)
                and os.path.getmtime(o) > newest_header and not extra_flags):
            continue
        jobs.append([nv] + flags + ["-c", s, "-o", o])
    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for rc, cmd, out in ex.map(_run, jobs):
            if verbose or rc:
                print(cmd)
                print(out)
            if rc:
                raise RuntimeError("nvcc failed")
    link = [nv, "-shared"] + ARCH + ["-o", LIB] + objs + ["-lpthread"]
    rc, cmd, out = _run(link)
    if verbose or rc:
        print(cmd)
        print(out)
    if rc:
        raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
