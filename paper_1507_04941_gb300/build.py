"""Build libsf.so in-tree with nvcc for sm_103a.

The kernel source that the runtime compiles per plan (csrc/kernels/
sf_kernels.cuh) and the parameter-block header are embedded into the library
as strings, so the shared object is self-contained.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsf.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _embed(out_path: str) -> None:
    def raw(name: str, path: str) -> str:
        text = open(path).read()
        if ")SFK\"" in text:
            raise RuntimeError(f"{path} contains the raw-string delimiter")
        return f'extern "C" const char *{name} = R"SFK({text})SFK";\n'
    body = "/* generated by paper_1507_04941_gb300/build.py: do not edit */\n"
    body += raw("sf_embedded_kernel_source", os.path.join(CSRC, "kernels", "sf_kernels.cuh"))
    body += raw("sf_embedded_abi_source", os.path.join(CSRC, "sf_kernel_abi.h"))
    tmp = out_path + ".tmp"
    with open(tmp, "w") as fh:
        fh.write(body)
    os.replace(tmp, out_path)


def _sources() -> list[str]:
    return [os.path.join(CSRC, "sf_runtime.cpp"), os.path.join(CSRC, "sf_aot.cu"),
            os.path.join(CSRC, "sf_noalloc.cu"), os.path.join(CSRC, "sf_server.cpp"),
            os.path.join(CSRC, "sf_local.cu"), os.path.join(CSRC, "sf_weighted.cu"),
            os.path.join(CSRC, "sf_probe.cu"), os.path.join(BUILD, "sf_embedded.cpp")]


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, "sf_runtime.cpp"), os.path.join(CSRC, "sf_aot.cu"),
             os.path.join(CSRC, "sf_noalloc.cu"), os.path.join(CSRC, "sf_server.cpp"),
             os.path.join(CSRC, "sf_local.cu"), os.path.join(CSRC, "sf_weighted.cu"),
             os.path.join(CSRC, "sf_probe.cu"), os.path.join(CSRC, "sf_kernel_abi.h"), os.path.join(CSRC, "kernels", "sf_kernels.cuh"),
             os.path.join(ROOT, "include", "sf.h"), os.path.abspath(__file__)]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library (skipped when it is newer than every input)."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    _embed(os.path.join(BUILD, "sf_embedded.cpp"))
    common = [nvcc, ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC]

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = common + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        return obj

    with ThreadPoolExecutor(max_workers=8) as ex:
        objs = list(ex.map(compile_one, _sources()))
    libdir = _cuda_lib_dir(nvcc)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, ARCH, "-shared", "-o", tmp] + objs + [
        "-cudart", "shared", "-L", libdir, "-lnvrtc", "-lpthread", "-Xlinker", f"-rpath,{libdir}"]
    if verbose:
        print(" ".join(cmd))
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
