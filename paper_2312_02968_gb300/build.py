"""Build the CUDA library libmondpm.so in-tree for sm_103a (nvcc, no cmake).

One translation unit per supported FFT-domain side plus the API unit are
compiled in parallel and linked into paper_2312_02968_gb300/_build/libmondpm.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmondpm.so")
SIZES = [16, 32, 48, 64, 96, 128, 192, 256, 384, 512]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "--expt-relaxed-constexpr"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _sources_digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(SRC)):
        with open(os.path.join(SRC, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    for hdr in ("mond_pm.h", "mond_fno.h"):
        with open(os.path.join(HERE, "..", "include", hdr), "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    stamp = os.path.join(OUT, "stamp")
    digest = _sources_digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == digest:
        return LIB
    nvcc = _nvcc()
    jobs = [([nvcc] + ARCH + FLAGS + ["-c", os.path.join(SRC, "mond_pm_api.cu"), "-o", os.path.join(OUT, "api.o")],
             os.path.join(OUT, "api.o")),
            ([nvcc] + ARCH + FLAGS + ["-c", os.path.join(SRC, "deposit_noalloc.cu"), "-o",
                                      os.path.join(OUT, "deposit_noalloc.o")], os.path.join(OUT, "deposit_noalloc.o")),
            ([nvcc] + ARCH + FLAGS + ["-c", os.path.join(SRC, "fno.cu"), "-o", os.path.join(OUT, "fno.o")],
             os.path.join(OUT, "fno.o")),
            ([nvcc] + ARCH + FLAGS + ["-c", os.path.join(SRC, "probe.cu"), "-o", os.path.join(OUT, "probe.o")],
             os.path.join(OUT, "probe.o"))]
    for n in SIZES:
        o = os.path.join(OUT, f"passes_{n}.o")
        jobs.append(([nvcc] + ARCH + FLAGS + [f"-DMOND_N={n}", "-c", os.path.join(SRC, "passes_inst.cu"), "-o", o], o))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        list(ex.map(run, [j[0] for j in jobs]))
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc] + ARCH + ["-shared", "-o", tmp] + [j[1] for j in jobs])
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=False))
