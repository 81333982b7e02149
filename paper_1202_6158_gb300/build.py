"""Build libditer.so (sm_103a) in-tree with nvcc.

Each translation unit of ``csrc/`` is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3``, then linked into
``paper_1202_6158_gb300/libditer.so`` against the shared CUDA runtime.
``build(debug=True)`` makes ``libditer_debug.so`` the same way with ``-DDI_DEBUG``:
the sweep kernels check the indices they compute (see include/diter.h).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libditer.so")
LIB_DEBUG = os.path.join(HERE, "libditer_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libditer")


def sources() -> list:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "diter.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra: tuple = (), debug: bool = False) -> str:
    """Compile (if stale) and return the path of libditer.so (libditer_debug.so with debug=True)."""
    lib = LIB_DEBUG if debug else LIB
    if debug:
        extra = (*extra, "-DDI_DEBUG")
    if not force and not _stale(lib):
        return lib
    nvcc = _nvcc()
    cuda_home = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    tmpdir = tempfile.mkdtemp(prefix="diter_build_", dir=HERE)
    try:
        common = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                  "--expt-relaxed-constexpr", *extra]
        procs = []
        objs = []
        for src in sources():
            obj = os.path.join(tmpdir, os.path.basename(src) + ".o")
            objs.append(obj)
            cmd = [*common, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        failed = []
        for src, p in procs:
            out, _ = p.communicate()
            if verbose or p.returncode != 0:
                sys.stderr.write(out.decode(errors="replace"))
            if p.returncode != 0:
                failed.append(src)
        if failed:
            raise RuntimeError("nvcc failed on: " + ", ".join(os.path.basename(f) for f in failed))
        out_tmp = os.path.join(tmpdir, os.path.basename(lib))
        link = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", out_tmp, *objs,
                "-Xlinker", "-rpath", "-Xlinker", os.path.join(cuda_home, "lib64")]
        if verbose:
            print(" ".join(link), file=sys.stderr)
        subprocess.run(link, check=True)
        os.replace(out_tmp, lib)
    finally:
        shutil.rmtree(tmpdir, ignore_errors=True)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv,
                extra=tuple(a for a in sys.argv[1:] if a.startswith("-X") or a.startswith("--resource"))))
