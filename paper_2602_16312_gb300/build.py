"""Builds libaggmg.so in-tree from csrc/ for sm_103a (nvcc + g++, no cmake).

Translation units compile in parallel; the block-size engines are split
across files so that the slowest unit bounds the build time.
"""
import os
import shutil
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
# AGG_BUILD_DIR / AGG_NVCC_FLAGS select another build folder and extra nvcc
# flags (used to compare tuning variants side by side)
OUT = os.environ.get("AGG_BUILD_DIR", os.path.join(HERE, "_build"))
LIB = os.path.join(OUT, "libaggmg.so")
EXTRA = os.environ.get("AGG_NVCC_FLAGS", "").split()
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile every translation unit and link libaggmg.so; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    cu, cpp = sources()
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(os.path.dirname(HERE), "include", "aggmg.h")]
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) > newest:
        return LIB
    jobs = []
    objs = []
    for f in cu:
        o = os.path.join(OUT, f + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", *EXTRA, "-Xcompiler", "-fPIC,-fopenmp",
               "-c", os.path.join(CSRC, f), "-o", o]
        jobs.append((f, cmd))
        objs.append(o)
    for f in cpp:
        o = os.path.join(OUT, f + ".o")
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-I/usr/local/cuda/include",
               "-c", os.path.join(CSRC, f), "-o", o]
        jobs.append((f, cmd))
        objs.append(o)
    t0 = time.time()
    procs = [(f, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)) for f, cmd in jobs]
    failed = []
    for f, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((f, out.decode(errors="replace")))
        elif verbose and out:
            sys.stderr.write(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(f"--- {f}\n{o}" for f, o in failed)
        raise RuntimeError(f"libaggmg build failed:\n{msg}")
    tmp = LIB + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    if verbose:
        sys.stderr.write(f"built {LIB} in {time.time() - t0:.1f} s\n")
    return LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv)
