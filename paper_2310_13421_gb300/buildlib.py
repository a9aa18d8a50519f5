"""Build libtpd.so in-tree (paper_2310_13421_gb300/_build/) for sm_103a.

Translation units compile in parallel: the two kernel files with nvcc, the
host-only C ABI and planner with g++.  A content hash of the sources decides
whether anything needs rebuilding.
"""
import concurrent.futures
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libtpd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["tpd_kernels_fixed_dec.cu", "tpd_kernels_fixed_com.cu", "tpd_kernels_batch_fixed.cu",
              "tpd_kernels_shapes_fixed.cu", "tpd_kernels_shapes_c64.cu", "tpd_kernels_shapes_f32.cu",
              "tpd_kernels_shapes_fx32.cu",
              "tpd_kernels_batch_ieee.cu", "tpd_kernels_c128.cu", "tpd_kernels_c64.cu", "tpd_noalloc.cu", "tpd_layout.cu",
              "tpd_sparse.cu", "tpd_weyl.cu", "tpd_gellmann.cu"]
CPP_SOURCES = ["tpd_api.cpp", "tpd_api_batched.cpp", "tpd_api_extra.cpp", "tpd_planner.cpp"]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _digest():
    h = hashlib.sha256()
    files = sorted(os.listdir(CSRC)) + ["../../include/tpd.h"]
    for f in files:
        p = os.path.normpath(os.path.join(CSRC, f))
        if os.path.isfile(p) and p.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(f.encode())
            with open(p, "rb") as fh:
                h.update(fh.read())
    h.update(" ".join(ARCH).encode())
    return h.hexdigest()


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n%s\n%s" % (" ".join(cmd), r.stdout))
    return r.stdout


def build(force=False, verbose=False):
    """Compile libtpd.so if its sources changed; return its path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "libtpd.stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == dig:
                return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I" + INCLUDE, "-I" + CSRC]
    jobs = []
    for src in CU_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append([nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                                     "-Xptxas", "-v" if verbose else "-O3"] + inc +
                    ["-c", os.path.join(CSRC, src), "-o", obj])
    for src in CPP_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I" + os.path.join(cuda, "include")] + inc +
                    ["-c", os.path.join(CSRC, src), "-o", obj])
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            print(o)
    objs = [os.path.join(BUILD, s + ".o") for s in CU_SOURCES + CPP_SOURCES]
    tmp = LIB + ".%d.tmp" % os.getpid()
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-lpthread", "-ldl"])
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
