"""Build step of the native library: nvcc for sm_103a, in-tree output.

``python -m paper_2502_08673_b300.build`` compiles csrc/*.cpp and csrc/*.cu
into paper_2502_08673_b300/libsatsampler.so (static CUDA runtime, -lineinfo, NVRTC for
the instance-compiled round kernel).  The text of the device headers that kernel's
program includes (relax.cuh, philox.cuh) is written into _build/jit_text.inc first, so
the run-time program and the nvcc-built kernels share one source.
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
LIB = PKG / "libsatsampler.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(CSRC.glob("*.cpp")) + sorted(CSRC.glob("*.cu"))


def needs_build() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    deps = sources() + sorted(CSRC.glob("*.hpp")) + sorted(CSRC.glob("*.cuh")) + [PKG.parent / "include" / "satsampler.h"]
    return any(p.stat().st_mtime > t for p in deps)


JIT_HEADERS = (("relax.cuh", "kRelaxCuh"), ("philox.cuh", "kPhiloxCuh"))


def write_jit_text(objdir: Path) -> None:
    parts = []
    for name, ident in JIT_HEADERS:
        text = (CSRC / name).read_text()
        if ")SATJIT" in text:
            raise ValueError(f"{name} holds the raw-string delimiter")
        parts.append(f'static const char {ident}[] = R"SATJIT({text})SATJIT";\n')
    out = objdir / "jit_text.inc"
    text = "".join(parts)
    if not out.exists() or out.read_text() != text:
        out.write_text(text)


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and not needs_build():
        return LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    objdir = PKG / "_build"
    objdir.mkdir(exist_ok=True)
    write_jit_text(objdir)
    objs = []
    for src in sources():
        obj = objdir / (src.stem + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3",
               "--expt-relaxed-constexpr", "-I", str(objdir), "-c", str(src), "-o", str(obj)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        objs.append(str(obj))
    tmp = LIB.with_suffix(".so.tmp")
    cuda_lib = Path(nvcc).resolve().parent.parent / "lib64"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", str(tmp), *objs, "-cudart", "static", "-lnvrtc",
                           "-Xlinker", f"-rpath,{cuda_lib}"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
