"""Build the CUDA library in-tree: csrc/*.cu -> lib/libtsm_gb300.so (sm_103a).

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into one shared object.  A hash of the sources, headers and flags is
kept beside the library so an unchanged tree is not rebuilt.
"""
import concurrent.futures
import glob
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIBNAME = "libtsm_gb300.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None:
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            exe = cand
    if exe is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return exe


def library_path():
    return os.path.join(LIBDIR, LIBNAME)


def _digest(extra_flags):
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h")))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS + extra_flags).encode())
    return h.hexdigest()


def source_digest(names=None):
    """sha256 of CUDA sources and public headers (names and contents): a
    profile taken on one tree is valid for another only if this matches.
    names: the basenames a kernel's translation unit is compiled from (the
    digest then also covers the compiler flags but not the checkout's include
    paths); None: every source."""
    h = hashlib.sha256()
    if names is None:
        files = sorted(glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h")))
    else:
        files = []
        for n in sorted(names):
            cand = [os.path.join(d, n) for d in (CSRC, INCLUDE) if os.path.exists(os.path.join(d, n))]
            files.append(cand[0] if cand else n)
    for f in files:
        h.update(os.path.basename(f).encode())
        if os.path.exists(f):
            with open(f, "rb") as fh:
                h.update(fh.read())
        else:
            h.update(b"<missing>")
    if names is not None:  # the flags, without the include paths (which differ between checkouts)
        flags = ARCH + FLAGS
        kept = [f for k, f in enumerate(flags) if f != "-I" and not (k > 0 and flags[k - 1] == "-I")]
        h.update(" ".join(kept).encode())
    return h.hexdigest()


def build(verbose=False, force=False, extra_flags=None, jobs=None):
    # TSM_NVCC_FLAGS adds compile definitions (variant builds for measurements)
    if extra_flags is None:
        extra_flags = os.environ.get("TSM_NVCC_FLAGS", "").split()
    extra_flags = list(extra_flags)
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    stamp = os.path.join(LIBDIR, LIBNAME + ".sha256")
    digest = _digest(extra_flags)
    if not force and os.path.exists(library_path()) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return library_path()
    exe = nvcc()
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [exe] + ARCH + FLAGS + extra_flags + ["-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), res.stderr))
        if verbose and res.stderr:
            sys.stderr.write(res.stderr)
        return obj

    workers = jobs or min(len(sources), os.cpu_count() or 4)
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, sources))
    tmp = library_path() + ".tmp"
    cmd = [exe] + ARCH + ["-shared", "-o", tmp] + objs
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), res.stderr))
    os.replace(tmp, library_path())
    with open(stamp, "w") as fh:
        fh.write(digest)
    return library_path()


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
