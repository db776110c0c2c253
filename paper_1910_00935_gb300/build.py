"""Build libmpm.so (the C-ABI library) for sm_103a with nvcc, in-tree.

    python -m paper_1910_00935_gb300.build [--force] [--polar-fp64]

Each translation unit is compiled in parallel; the objects are linked into
paper_1910_00935_gb300/_build/libmpm.so.  Only the sm_103a target is built.  The variant
with the fixed-corotated polar factor's refinement and adjoint in FP64 (MPM_POLAR_FP64=1)
goes to paper_1910_00935_gb300/_build_polar64/libmpm.so; load it with MPM_LIB.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmpm.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["kernels_3d_fcr.cu", "kernels_3d_fcr_det.cu", "kernels_3d_nh.cu", "kernels_3d_nh_det.cu",
           "kernels_3d_liq.cu", "kernels_3d_liq_det.cu", "kernels_3d_mixed.cu",
           "kernels_3d_mixed_det.cu", "kernels_2d.cu", "setup.cu", "controller.cu",
           "mass_spring.cu", "mpm_api.cu", "noalloc.cu", "peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "mpm.h"))
    return files


def needs_build(out_dir: str = OUT_DIR) -> bool:
    lib = os.path.join(out_dir, "libmpm.so")
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    objs = [os.path.join(out_dir, src.replace(".cu", ".o")) for src in SOURCES]
    return any(not os.path.exists(o) for o in objs) or any(os.path.getmtime(f) > t for f in _deps())


def variant_dir(tag: str) -> str:
    """Build folder of a named variant (`_build_<tag>` beside the default `_build`)."""
    return OUT_DIR if not tag else os.path.join(HERE, f"_build_{tag}")


# the library of the polar_fp64 variant (build(polar_fp64=True))
LIB_POLAR64 = os.path.join(variant_dir("polar64"), "libmpm.so")


def build(force: bool = False, verbose: bool = False, extra_flags=(), polar_fp64: bool = False,
          tag: str = "") -> str:
    """Compile and link libmpm.so; returns its path.  `tag` names a variant folder for
    builds with other `extra_flags` (e.g. another MPM_TILE); polar_fp64 is the variant
    `polar64` with -DMPM_POLAR_FP64=1."""
    if polar_fp64:
        tag = tag or "polar64"
        extra_flags = [*extra_flags, "-DMPM_POLAR_FP64=1"]
    out_dir = variant_dir(tag)
    lib = os.path.join(out_dir, "libmpm.so")
    if not force and not needs_build(out_dir):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [],
                polar_fp64="--polar-fp64" in sys.argv))
