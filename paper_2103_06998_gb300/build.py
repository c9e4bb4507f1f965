"""Compile the CUDA/C++ sources of the library into libadi_maxwell.so (in-tree).

nvcc for sm_103a only, translation units compiled in parallel, then linked
as one shared library next to this file.  Used by ``__graft_entry__.build()``
and by ``python -m paper_2103_06998_gb300.build``.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libadi_maxwell.so")
# (source, object name, extra flags): the step kernels are compiled twice, one
# element type per object, so the two halves build in parallel
SOURCES = [("adi_kernels.cu", "adi_kernels_f32", []), ("adi_kernels.cu", "adi_kernels_f64", ["-DADI_KERNELS_F64"]),
           ("adi_capi.cpp", "adi_capi", []), ("setup_host.cpp", "setup_host", []), ("adi_noalloc.cu", "adi_noalloc", []),
           ("adi_batch.cpp", "adi_batch", []), ("adi_net.cu", "adi_net", [])]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build(verbose=False, extra_flags=()):
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    nv = nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]
    common += list(extra_flags)

    def compile_one(entry):
        src, name, flags = entry
        obj = os.path.join(out_dir, name + ".o")
        cmd = [nv, "-c", os.path.join(CSRC, src), "-o", obj] + common + list(flags) + ARCH
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    tmp = LIB + ".tmp"
    cmd = [nv, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
