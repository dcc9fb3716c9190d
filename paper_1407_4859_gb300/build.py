"""Builds libadha.so in-tree from csrc/*.cu with nvcc for sm_103a (one -gencode, parallel compiles).

Float arithmetic in the kernels uses explicitly rounded intrinsics; the flags below (no FMA
contraction, no flush-to-zero, IEEE division and square root) keep any remaining plain operator
from being fused or approximated.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libadha.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-fmad=false", "-ftz=false",
              "-prec-div=true", "-prec-sqrt=true", "--expt-relaxed-constexpr"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libadha.so")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


# Headers of the kernels that fused runs specialise at run time (jit.cu): embedded into the
# library as text, under the names their #include lines use when compiled by the run-time compiler.
JIT_HEADERS = [("adha.h", os.path.join(HERE, "..", "include", "adha.h")),
               ("device_types.h", os.path.join(CSRC, "device_types.h")),
               ("ptx.cuh", os.path.join(CSRC, "ptx.cuh")),
               ("section_ops.cuh", os.path.join(CSRC, "section_ops.cuh")),
               ("fused_jit.cuh", os.path.join(CSRC, "fused_jit.cuh"))]
_DELIM = "ADHA_JIT_HEADER"


def _write_jit_headers(path):
    """Writes the C++ source that holds the run-time compiler's headers as string literals."""
    out = ["// Generated by build.py: the headers of the kernels specialised at run time.",
           "namespace adha {",
           "extern const int kJitHeaderCount = %d;" % len(JIT_HEADERS),
           "extern const char* const kJitHeaderNames[] = {%s};" % ", ".join('"%s"' % n for n, _ in JIT_HEADERS),
           "extern const char* const kJitHeaderText[] = {"]
    for _, p in JIT_HEADERS:
        text = open(p).read()
        if (")" + _DELIM + '"') in text:
            raise RuntimeError("%s contains the raw-string delimiter" % p)
        out.append('R"%s(%s)%s",' % (_DELIM, text, _DELIM))
    out += ["};", "}  // namespace adha", ""]
    body = "\n".join(out)
    if not os.path.exists(path) or open(path).read() != body:
        with open(path, "w") as f:
            f.write(body)


def build(force=False, verbose=False, ptxas_info=False):
    """Compile every csrc/*.cu and link libadha.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    jit_src = os.path.join(BUILD, "jit_headers.cpp")
    _write_jit_headers(jit_src)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu"))) + [jit_src]
    headers = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                     + glob.glob(os.path.join(HERE, "..", "include", "*.h")))
    cc = nvcc()
    libdir = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(cc))), "lib64")
    defs = ['-DADHA_CUDA_LIBDIR="%s"' % libdir]
    objs = []
    jobs = []
    for src in sources:
        obj = os.path.join(BUILD, os.path.splitext(os.path.basename(src))[0] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            cmd = [cc] + ARCH + NVCC_FLAGS + defs + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", src, "-o", obj]
            jobs.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if verbose or ptxas_info:
            print(" ".join(cmd))
            print(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), r.stdout + r.stderr))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".%d.tmp" % os.getpid()
        r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-ldl"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
