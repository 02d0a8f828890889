"""Build libftgemm.so in-tree for sm_103a (nvcc, one -gencode, TUs in parallel)."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libftgemm.so")
SOURCES = ["ftgemm_host.cu", "ftgemm_k_nn.cu", "ftgemm_k_nt.cu", "ftgemm_k_tn.cu", "ftgemm_k_tt.cu",
           "ftgemm_kb_nn.cu", "ftgemm_kb_nt.cu", "ftgemm_kb_tn.cu", "ftgemm_kb_tt.cu",
           "ftgemm_k_split.cu", "ftgemm_k_split_tc.cu", "ftgemm_k_split_tcp.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def flags(verbose: bool = False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "ftgemm.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    procs = []
    for src in SOURCES:
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        cmd = [nvcc()] + flags(verbose) + ["-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((src, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    objs, failed = [], []
    for src, obj, pr in procs:
        out, _ = pr.communicate()
        if verbose or pr.returncode != 0:
            sys.stdout.write(out.decode(errors="replace"))
        if pr.returncode != 0:
            failed.append(src)
        objs.append(obj)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = LIB + f".tmp{os.getpid()}"
    exports = os.path.join(CSRC, "exports.map")   # only the ftgemm_* entry points are exported
    subprocess.run([nvcc()] + ARCH + ["-shared", "-Xlinker", "--version-script=" + exports, "-o", tmp] + objs,
                   check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
