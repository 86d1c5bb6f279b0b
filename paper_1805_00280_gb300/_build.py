"""In-tree build of the native libraries of the package.

* ``lib/libn2v.so``   -- the CUDA sampler and its C ABI (nvcc, sm_103a only).
* ``graphs/libn2vgen.so`` -- the seeded input generators (gcc, host only).

Each library is rebuilt when its sources change or when the stamp was written
on another machine architecture (x86_64 build hosts vs aarch64 GPU hosts).
"""
from __future__ import annotations

import hashlib
import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
REPO = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
LIBN2V = os.path.join(LIBDIR, "libn2v.so")
# the same sources with the device self-checks compiled in (-DN2V_CHECKED), and with the
# step statistics (-DN2V_STATS)
LIBN2V_CHECKED = os.path.join(LIBDIR, "libn2v_checked.so")
LIBN2V_STATS = os.path.join(LIBDIR, "libn2v_stats.so")
GENDIR = os.path.join(PKG, "graphs")
LIBGEN = os.path.join(GENDIR, "libn2vgen.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _digest(paths: list[str], extra: str) -> str:
    h = hashlib.sha256(extra.encode())
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    h.update(platform.machine().encode())
    return h.hexdigest()


def _fresh(target: str, digest: str) -> bool:
    stamp = target + ".stamp"
    if not (os.path.exists(target) and os.path.exists(stamp)):
        return False
    with open(stamp) as f:
        return f.read().strip() == digest


def _stamp(target: str, digest: str) -> None:
    with open(target + ".stamp", "w") as f:
        f.write(digest + "\n")


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout)


def build_gen(verbose: bool = False) -> str:
    src = os.path.join(GENDIR, "n2v_gen.c")
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=c11", src, "-o", LIBGEN]
    d = _digest([src], " ".join(cmd))
    if not _fresh(LIBGEN, d):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        _run(cmd)
        _stamp(LIBGEN, d)
    return LIBGEN


def cuda_sources() -> tuple[list[str], list[str]]:
    cu = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    hdr = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))
    hdr.append(os.path.join(REPO, "include", "n2v.h"))
    return cu, hdr


def build_n2v(verbose: bool = False, extra_flags: list[str] | None = None, checked: bool = False,
              stats: bool = False) -> str:
    """Compile every .cu under csrc/ (in parallel) and link libn2v.so (checked: libn2v_checked.so,
    with the device self-checks; stats: libn2v_stats.so, with the step statistics)."""
    os.makedirs(LIBDIR, exist_ok=True)
    cu, hdr = cuda_sources()
    target = LIBN2V_CHECKED if checked else (LIBN2V_STATS if stats else LIBN2V)
    flags = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
             "-I", os.path.join(REPO, "include"), "-I", CSRC, "--expt-relaxed-constexpr"]
    if checked:
        flags.append("-DN2V_CHECKED")
    if stats:
        flags.append("-DN2V_STATS")
    flags += extra_flags or []
    d = _digest(cu + hdr, " ".join(flags))
    if _fresh(target, d):
        return target
    objdir = os.path.join(LIBDIR, "obj_checked" if checked else ("obj_stats" if stats else "obj"))
    os.makedirs(objdir, exist_ok=True)

    def one(src: str) -> str:
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [NVCC, *flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        _run(cmd)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(len(cu), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(one, cu))
    link = [NVCC, *ARCH, "-shared", "-o", target, *objs, "-lcudart"]
    if verbose:
        print(" ".join(link), file=sys.stderr)
    _run(link)
    _stamp(target, d)
    return target


def build_all(verbose: bool = False) -> None:
    """The generators, then the sampler library and its checked and stats twins, compiled side by side."""
    build_gen(verbose)
    with ThreadPoolExecutor(max_workers=3) as ex:
        for f in [ex.submit(build_n2v, verbose), ex.submit(build_n2v, verbose, None, True),
                  ex.submit(build_n2v, verbose, None, False, True)]:
            f.result()


if __name__ == "__main__":
    build_all(verbose=True)
