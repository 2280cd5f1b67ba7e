"""Build the CUDA library (libeg.so) in-tree with nvcc for sm_103a.

Translation units compile in parallel; the shared object is linked against
the shared CUDA runtime.  Nothing here imports torch.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libeg.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-Xptxas", "-O3"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libeg.so")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(INCLUDE, "eg.h"))
    return sorted(hs)


def _fingerprint(files=None) -> str:
    """SHA-256 over file names (not paths: the tree moves between machines),
    contents and compiler flags.  Default: every source and header."""
    h = hashlib.sha256()
    for p in (sources() + _headers()) if files is None else files:
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()


def _code_text(text: str) -> str:
    """C/C++/CUDA source without its comments and with runs of white space
    folded to one blank: what the compiler sees of it."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"' or c == "'":  # a literal, copied through (with escapes)
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def code_fingerprint_of(named_texts) -> str:
    """SHA-256 over (basename, code text) pairs and the compiler flags."""
    h = hashlib.sha256()
    for name, text in named_texts:
        h.update(name.encode())
        h.update(_code_text(text).encode())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()


def kernel_fingerprint(source: str) -> str:
    """Fingerprint of one translation unit (basename under csrc/) and the
    headers every unit includes, over their code without comments: it changes
    when that kernel's code does, not when a comment does."""
    files = [os.path.join(CSRC, source)] + _headers()
    return code_fingerprint_of((os.path.basename(p), open(p, encoding="utf-8").read()) for p in files)


LIB_CHECKED = os.path.join(HERE, "libeg_checked.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every .cu under csrc/ and link libeg.so; returns its path.
    checked=True builds the bounds-checked variant libeg_checked.so instead
    (EG_CHECKED: every computed index is tested before the access, a miss is
    reported in the status word; for tests, several times slower)."""
    lib = LIB_CHECKED if checked else LIB
    bdir = BUILD_CHECKED if checked else BUILD
    extra = ["-DEG_CHECKED"] if checked else []
    os.makedirs(bdir, exist_ok=True)
    stamp = os.path.join(bdir, "stamp")
    fp = _fingerprint() + ("-checked" if checked else "")
    if not force and os.path.exists(lib) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == fp:
                return lib
    nvcc = _nvcc()
    procs, objs = [], []
    for src in sources():
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{src}:\n{out.decode(errors='replace')}")
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=HERE)
    os.close(fd)
    cmd = [nvcc, *ARCH, "-shared", "-cudart=shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        os.unlink(tmp)
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(fp)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
