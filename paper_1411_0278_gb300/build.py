"""Build step: regenerate the pair-frame tables and compile libgbi.so for sm_103a.

The translation units are compiled in parallel with nvcc (one -gencode,
sm_103a only) and linked into ``_build/libgbi.so`` inside the package, where the
binding loads it.  Nothing is installed outside the source tree.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgbi.so")
SOURCES = ["gbi_api.cu", "common.cu", "solver.cu", "nearfield_api.cu", "trap_kernel.cu", "mlp_kernel.cu",
           "mlp_tc.cu", "flow.cu", "wall.cu", "periodic.cu"] + ["pairs_%s_%d.cu" % (p, t) for p in ("f32", "f64", "df") for t in (2, 3, 4)] + \
    ["pairs_f64_5.cu", "pairs_f64_40.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wno-deprecated-declarations",
         "-diag-suppress", "177"]


def nvcc():
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbi")


def _compile(src, verbose):
    obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc()] + FLAGS + ARCH + ["-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, res.stdout, res.stderr))
    return obj, res.stderr


def build(verbose=False):
    """Regenerate csrc/gbi_generated.cuh and (re)build _build/libgbi.so. Returns the path."""
    sys.path.insert(0, HERE)
    try:
        import gen_tables
    finally:
        sys.path.pop(0)
    gen_tables.emit(os.path.join(CSRC, "gbi_generated.cuh"))
    os.makedirs(OUT, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared"] + ARCH + objs + ["-o", tmp, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (res.stdout, res.stderr))
    os.replace(tmp, LIB)
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
