"""Build libsrmc.so in-tree for sm_103a with nvcc.

The step kernel is compiled once per dimension D = 1..19 (-DSRMC_STEP_D=D) so
that per-path state stays in registers, and once per kind of strata
(-DSRMC_STEP_KIND: equal size, equal probability), of dynamics
(-DSRMC_STEP_DYN: Euler, exact, Euler with a non-diagonal sigma, also as a d x q
matrix with -DSRMC_STEP_Q=q) and of basis
(-DSRMC_STEP_BASIS=2: quadratic local polynomials, d <= 3) so that each kernel
carries only its own cell location, chain step and basis; the objects are
compiled in parallel and linked with the C-ABI translation unit into one shared
library under ``paper_2407_21085_gb300/_build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsrmc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
DIMS = range(1, 20)             # equal-size strata, Euler dynamics: d <= 19
NARROW_DIMS = range(1, 9)       # equal-probability strata, exact dynamics: d <= 8
LP2_DIMS = range(1, 4)          # quadratic local polynomials: d <= 3
DENSEQ_DIMS = range(1, 5)       # a d x q sigma with q != d: d, q <= 4


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsrmc")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-I", INCLUDE, "-Xcompiler",
                   "-fPIC,-ffp-contract=off", "--expt-relaxed-constexpr"]


def _cuda_include(nvcc: str) -> str:
    """The toolkit's include directory (NVRTC compiles user models against it)."""
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")


def _nvrtc_lib(nvcc: str) -> str:
    """The toolkit's NVRTC library (opened at run time for user models)."""
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for sub in ("lib64", "lib", os.path.join("targets", "sbsa-linux", "lib"),
                os.path.join("targets", "x86_64-linux", "lib")):
        cand = os.path.join(root, sub, "libnvrtc.so")
        if os.path.exists(cand):
            return cand
    return "libnvrtc.so"


def _embed_sources(out: str) -> str:
    """Write a unit holding the step-kernel sources as strings, which the
    library hands to NVRTC when it compiles a user model."""
    path = os.path.join(out, "rtc_sources.cu")
    lines = ["// generated by build.py: the step-kernel sources for run-time compilation"]
    for name, sym in (("srmc_device.cuh", "srmc_rtc_device_cuh"), ("srmc_step.cu", "srmc_rtc_step_cu")):
        with open(os.path.join(CSRC, name)) as fh:
            text = fh.read()
        body = ", ".join(str(b) for b in text.encode()) + ", 0"
        lines.append(f"extern const char {sym}[] = {{{body}}};")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    return path


def _sources():
    srcs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    srcs.append(os.path.join(INCLUDE, "srmc.h"))
    return srcs


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          out_dir: str | None = None, defines=()) -> str:
    """Compile and link libsrmc.so (into out_dir, default _build/, with extra
    -D defines for experiments on tuning constants)."""
    lib = LIB if out_dir is None else os.path.join(out_dir, "libsrmc.so")
    if out_dir is None and not force and not _stale():
        return LIB
    out = OUT_DIR if out_dir is None else out_dir
    os.makedirs(out, exist_ok=True)
    nvcc = _nvcc()
    extra_defs = [f"-D{d}" for d in defines]
    units = [(os.path.join(CSRC, "srmc_step.cu"), os.path.join(out, f"step_{tag}d{D}.o"),
              [f"-DSRMC_STEP_D={D}", f"-DSRMC_STEP_KIND={kind}"] + extra_defs)
             for kind, tag, dims in ((0, "", DIMS), (1, "prob_", NARROW_DIMS)) for D in dims]
    units += [(os.path.join(CSRC, "srmc_step.cu"), os.path.join(out, f"step_exact_d{D}.o"),
               [f"-DSRMC_STEP_D={D}", "-DSRMC_STEP_DYN=1"] + extra_defs) for D in NARROW_DIMS]
    units += [(os.path.join(CSRC, "srmc_step.cu"), os.path.join(out, f"step_dense_d{D}.o"),
               [f"-DSRMC_STEP_D={D}", "-DSRMC_STEP_DYN=2"] + extra_defs) for D in NARROW_DIMS]
    units += [(os.path.join(CSRC, "srmc_step.cu"), os.path.join(out, f"step_dense_d{D}_q{Q}.o"),
               [f"-DSRMC_STEP_D={D}", f"-DSRMC_STEP_Q={Q}", "-DSRMC_STEP_DYN=2"] + extra_defs)
              for D in DENSEQ_DIMS for Q in DENSEQ_DIMS if Q != D]
    units += [(os.path.join(CSRC, "srmc_step.cu"), os.path.join(out, f"step_quad_d{D}.o"),
               [f"-DSRMC_STEP_D={D}", "-DSRMC_STEP_BASIS=2"] + extra_defs) for D in LP2_DIMS]
    for name in sorted(os.listdir(CSRC)):
        if name.endswith(".cu") and name != "srmc_step.cu":
            units.append((os.path.join(CSRC, name), os.path.join(out, name[:-3] + ".o"),
                          extra_defs + [f'-DSRMC_CUDA_INCLUDE="{_cuda_include(nvcc)}"',
                                        f'-DSRMC_NVRTC_LIB="{_nvrtc_lib(nvcc)}"']))
    units.append((_embed_sources(out), os.path.join(out, "rtc_sources.o"), []))

    def compile_one(u):
        src, obj, extra = u
        cmd = [nvcc] + _flags() + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)} {extra}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    jobs = jobs or min(len(units), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = lib + f".{os.getpid()}.tmp"
    subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-ldl"], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
