"""Build libins.so in-tree with nvcc for sm_103a (B300).

Usage: python -m paper_2604_18536_b300.build [--verbose]
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libins.so")
# translation units of the library (each compiled separately, in parallel, then linked)
SOURCES = ["ins_grid.cu", "ins_step.cu", "ins_vjp.cu", "ins_closure.cu", "ins_eddy.cu", "ins_noalloc.cu"]
NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC",
    "--expt-relaxed-constexpr",
]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _newest_source_mtime():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "ins.h"))
    return max(os.path.getmtime(f) for f in files if os.path.exists(f))


def up_to_date():
    return os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_source_mtime()


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    return r.returncode, r.stdout + r.stderr


def build(verbose=False, force=False):
    """Compile libins.so (skips when it is newer than every source)."""
    if not force and up_to_date():
        return LIB
    import shutil
    import tempfile
    from concurrent.futures import ThreadPoolExecutor
    OBJ = tempfile.mkdtemp(prefix="libins_build_")   # object files stay out of the tree
    extra = ["-Xptxas", "-v"] if verbose else []
    cmds, objs = [], []
    for src in SOURCES:
        obj = os.path.join(OBJ, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        cmds.append([nvcc()] + NVCC_FLAGS + extra + ["-c", "-o", obj, os.path.join(CSRC, src)])
    with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 1)) as ex:
        results = list(ex.map(_run, cmds))
    for (rc, out), src in zip(results, SOURCES):
        if rc != 0:
            raise RuntimeError("nvcc failed on %s:\n%s" % (src, out))
        if verbose:
            sys.stderr.write(out)
    rc, out = _run([nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", LIB + ".tmp"] + objs)
    if rc != 0:
        raise RuntimeError("link failed:\n" + out)
    os.replace(LIB + ".tmp", LIB)
    shutil.rmtree(OBJ, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    build(verbose="--verbose" in sys.argv, force=True)
    print(LIB)
