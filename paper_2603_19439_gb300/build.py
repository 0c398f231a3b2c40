"""Build libgrest.so in-tree with nvcc for sm_103a (GB300).

Every translation unit under csrc/ is compiled in parallel to an object file
under _build/, then linked into paper_2603_19439_gb300/libgrest.so.  The
library is rebuilt unless a stamp written by the last build of it matches the
sources, the headers, the flags and this machine's architecture: a library
copied in from elsewhere (another machine, another checkout) is never trusted
because of its modification time.
"""
import hashlib
import os
import platform
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libgrest.so")
SOURCES = ["scan.cu", "graph.cu", "spmm.cu", "dense.cu", "eig.cu", "rsvd.cu", "grest.cu", "noalloc.cu", "tc_gram.cu", "small.cu", "tc_gemm.cu", "refine.cu", "small32.cu", "central.cu", "serve.cu", "narrow_gram.cu", "group.cu", "group_update.cu", "group_dense.cu", "waitcheck.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-I", INCLUDE]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


STAMP = os.path.join(BUILD, "libgrest.stamp")


def _input_hash():
    """Hash of every source and header, the compiler flags and the machine."""
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            h.update(f.encode())
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS + SOURCES).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def _stamp_of(lib):
    """The input hash recorded for this very file (its size and mtime included)."""
    st = os.stat(lib)
    return f"{_input_hash()} {st.st_size} {st.st_mtime_ns}"


def build(force=False, verbose=False):
    """Compile and link libgrest.so; returns its path."""
    if not force and os.path.exists(LIB) and os.path.exists(STAMP):
        with open(STAMP) as fh:
            if fh.read().strip() == _stamp_of(LIB):
                return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(_stamp_of(LIB))
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
