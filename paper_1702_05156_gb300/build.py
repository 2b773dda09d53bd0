"""Build ``libdmsgm.so`` (sm_103a) in-tree with nvcc.

Each ``csrc/*.cu`` translation unit compiles in parallel to an object, then
the objects link into one shared library next to this file.  Nothing here
needs a GPU; nvcc cross-compiles for sm_103a.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdmsgm.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


# Per-unit flags: the RANSAC unit evaluates FP64 expressions exactly as
# written (no fused multiply-add), so its models and inlier counts are the
# values of the written operations, reproducible by any IEEE evaluation of
# the same expressions.
UNIT_FLAGS = {"dmsgm_homog_ransac.cu": ["-fmad=false"]}


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _fingerprint() -> str:
    """Hash of the kernel sources, the public headers and the compile flags.
    Paths enter relative to the repository root, so the same sources give the
    same fingerprint wherever the repository sits."""
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h"))):
        with open(p, "rb") as f:
            h.update(os.path.relpath(p, ROOT).encode())
            h.update(f.read())
    h.update(" ".join(ARCH + [f for f in FLAGS if f not in (INCLUDE, CSRC)]).encode())
    h.update(repr(sorted(UNIT_FLAGS.items())).encode())
    return h.hexdigest()


def kernel_fingerprint(tu: str) -> str:
    """Hash of one translation unit under csrc/, the repository headers it
    includes (transitively) and the compile flags: it changes exactly when the
    code compiled into that unit's kernels does, not when other units do."""
    seen, todo = [], [os.path.join(CSRC, tu)]
    while todo:
        p = todo.pop()
        if p in seen or not os.path.exists(p):
            continue
        seen.append(p)
        with open(p, "rb") as f:
            for line in f.read().decode(errors="replace").splitlines():
                line = line.strip()
                if line.startswith("#include \""):
                    name = line.split('"')[1]
                    todo += [os.path.join(d, name) for d in (CSRC, INCLUDE)]
    h = hashlib.sha256()
    for p in sorted(seen):
        with open(p, "rb") as f:
            h.update(os.path.relpath(p, ROOT).encode())
            h.update(f.read())
    h.update(" ".join(ARCH + [f for f in FLAGS if f not in (INCLUDE, CSRC)]).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile every .cu under csrc/ and link libdmsgm.so; returns its path."""
    fp = _fingerprint() + " ".join(extra_flags or [])
    stamp = os.path.join(BUILD, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read() == fp:
                return LIB
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def compile_one(src, obj):
        cmd = [NVCC, *ARCH, *FLAGS, *UNIT_FLAGS.get(os.path.basename(src), []),
               *(extra_flags or []), "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        logs = list(ex.map(compile_one, srcs, objs))
    if verbose:
        for lg in logs:
            if lg:
                print(lg, file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-ldl", "-lrt", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(fp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None))
