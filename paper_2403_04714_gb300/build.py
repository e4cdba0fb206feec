"""Build the simulator's shared library (nvcc, sm_103a) in-tree.

    python -m paper_2403_04714_gb300.build

Each translation unit compiles in parallel, then nvcc links
paper_2403_04714_gb300/libgb300sim.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libgb300sim.so")
SOURCES = ["kernels.cu", "runtime.cpp", "compiler.cpp", "noalloc.cu", "server.cpp", "codegen.cpp", "jit.cpp", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(PKG), "include", "sim.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    out_dir = os.path.join(os.path.dirname(PKG), "_build", "obj")
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-lineinfo", *ARCH]

    def compile_one(src):
        obj = os.path.join(out_dir, src + ".o")
        cmd = [cc, *common, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    # the device runtime header and the ABI header are compiled into the
    # library as strings: NVRTC compiles them with the generated code
    emb = os.path.join(out_dir, "embedded_headers.cpp")
    with open(emb + ".tmp", "w") as f:
        f.write("namespace rtl {\n")
        for sym, name in (("kEmbeddedAbiHeader", "abi_device.h"), ("kEmbeddedRtHeader", "sim_rt.cuh")):
            text = open(os.path.join(CSRC, name)).read()
            assert ")RTLSIM_EMBED\"" not in text
            f.write(f"extern const char* const {sym};\nconst char* const {sym} = R\"RTLSIM_EMBED({text})RTLSIM_EMBED\";\n")
        f.write("}  // namespace rtl\n")
    os.replace(emb + ".tmp", emb)

    def compile_emb():
        obj = emb + ".o"
        subprocess.run([cc, *common, "-c", emb, "-o", obj], check=True, capture_output=True)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES) + 1) as ex:
        futs = [ex.submit(compile_one, s) for s in SOURCES] + [ex.submit(compile_emb)]
        objs = [f.result() for f in futs]
    tmp = f"{LIB}.tmp{os.getpid()}"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(cc))), "lib64")
    cmd = [cc, "-shared", *ARCH, *objs, "-o", tmp, "-lcudart", "-lnvrtc", "-lnvJitLink",
           "-Xlinker", f"-rpath,{cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
