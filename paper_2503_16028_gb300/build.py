"""Builds libsmcgm.so (sm_103a) in-tree from csrc/*.cu with nvcc.

One nvcc process per translation unit, run in parallel, then a shared-library
link.  Usage: python -m paper_2503_16028_gb300.build [--force]
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsmcgm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libsmcgm.so")
    return exe


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _newest_dep():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "smcgm.h")]
    return max(os.path.getmtime(f) for f in files if os.path.exists(f))


def build(force=False, verbose=False):
    """Compile (if stale) and return the path of libsmcgm.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_dep():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    exe = nvcc()
    # objects and the linked library go to a directory private to this build, so builds
    # started by several processes at once never link each other's half-written objects;
    # the finished library replaces the old one atomically (same file system)
    work = tempfile.mkdtemp(prefix="objs-", dir=BUILD)
    try:
        jobs = []
        for src in sources():
            obj = os.path.join(work, os.path.basename(src)[:-3] + ".o")
            jobs.append((src, obj, [exe] + ARCH + FLAGS + ["-c", src, "-o", obj]))
        with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            futs = {ex.submit(subprocess.run, cmd, capture_output=True, text=True): src for src, _, cmd in jobs}
            for f in cf.as_completed(futs):
                res = f.result()
                if res.returncode != 0:
                    raise RuntimeError("nvcc failed on %s:\n%s" % (futs[f], res.stderr[-4000:]))
                if verbose and res.stderr.strip():
                    print(res.stderr)
        tmp = os.path.join(work, os.path.basename(LIB))
        cmd = [exe] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + [o for _, o, _ in jobs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n" + res.stderr[-4000:])
        os.replace(tmp, LIB)
    finally:
        shutil.rmtree(work, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
