"""Build libqsim.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each .cu translation unit under csrc/ is compiled in parallel, then linked
into paper_1805_04708_gb300/libqsim.so.  Objects go to _build/ (git-ignored).
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqsim.so")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I" + INCLUDE, "-I" + CSRC,
         "-I" + BUILD]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _compile(src, verbose_ptxas=False):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + (["-Xptxas", "-v"] if verbose_ptxas else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


JIT_CORE = ("gatekind.h", "cplx.cuh", "tile_core.cuh")


def write_jit_core():
    """The device code that tile passes compiled at run time include, as one
    C++ string (kJitCore in _build/jit_core.inc): the headers in JIT_CORE
    with their #include and #pragma once lines dropped."""
    parts = []
    for name in JIT_CORE:
        with open(os.path.join(CSRC, name)) as f:
            for line in f:
                t = line.strip()
                if t.startswith('#include "') or t == "#pragma once":
                    continue
                parts.append(line)
    text = "".join(parts)
    assert ')QSJIT"' not in text
    out = os.path.join(BUILD, "jit_core.inc")
    body = 'static const char kJitCore[] = R"QSJIT(' + text + ')QSJIT";\n'
    if not os.path.exists(out) or open(out).read() != body:
        with open(out, "w") as f:
            f.write(body)


def build(force=False, verbose_ptxas=False, quiet=True):
    """Compile every csrc/*.cu for sm_103a and link libqsim.so.  Skips the
    work when the library is newer than every source and header."""
    os.makedirs(BUILD, exist_ok=True)
    write_jit_core()
    srcs = sources()
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(INCLUDE, "qsim.h"))
    if not force and not verbose_ptxas and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) < t for d in deps):
            return LIB
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        res = list(ex.map(lambda s: _compile(s, verbose_ptxas), srcs))
    if verbose_ptxas or not quiet:
        for (obj, err) in res:
            if err.strip():
                sys.stderr.write(err)
    objs = [o for o, _ in res]
    tmp = LIB + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv, quiet=False)
    print(LIB)
