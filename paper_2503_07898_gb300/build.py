"""Build liblbm.so in-tree with nvcc for sm_103a.

Every translation unit is compiled in parallel to an object file under
``_build/`` and linked into ``liblbm.so`` next to this file.  Objects are
rebuilt when their source or any header in ``csrc/`` is newer.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2"]
SOURCES = ["api.cu", "dense.cu", "sparse.cu", "fields.cu", "multires.cu", "noalloc.cu", "closure.cu", "batch.cu"]
# The lattice-dependent sources are compiled a second time for D3Q27 (their
# code lands in namespace lbm::q27; the D3Q19 build in lbm::q19).
LATTICE_SOURCES = ["dense.cu", "sparse.cu", "fields.cu", "multires.cu"]
UNITS = [(src, [], src.replace(".cu", ".o")) for src in SOURCES] + \
        [(src, ["-DLBM_Q=27"], src.replace(".cu", "_q27.o")) for src in LATTICE_SOURCES]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm")


def _newest_header():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(os.path.dirname(HERE), "include", "lbm.h"))
    return max(os.path.getmtime(h) for h in hs if os.path.exists(h))


def _compile(nvcc, unit, verbose):
    src, defs, obj_name = unit
    obj = os.path.join(BUILD, obj_name)
    s = os.path.join(CSRC, src)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(s), _newest_header()):
        return obj, ""
    cmd = [nvcc] + ARCH + FLAGS + defs + ["-c", s, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr[-4000:]}")
    return obj, r.stderr


def build(verbose=False, force=False):
    """Compile and link liblbm.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(lambda u: _compile(nvcc, u, verbose), UNITS))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
