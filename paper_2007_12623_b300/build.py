"""Builds libstereo.so (the CUDA library behind include/stereo.h) in-tree for
sm_103a with nvcc.  `python -m paper_2007_12623_b300.build` or build()."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libstereo.so")
# the checked build: in-kernel index checks that record failures in a device
# error word instead of accessing memory (-DSTEREO_CHECKED), for tests
LIB_CHECKED = os.path.join(HERE, "libstereo_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cu", ".cuh"))] + [
        os.path.join(ROOT, "include", "stereo.h")]


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in sources())


def translation_units():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")]


def _deps(src: str, seen=None) -> set:
    """The file and every header it includes with quotes, transitively
    (csrc/ and include/)."""
    seen = set() if seen is None else seen
    if src in seen or not os.path.exists(src):
        return seen
    seen.add(src)
    with open(src) as f:
        for line in f:
            t = line.strip()
            if t.startswith("#include \""):
                name = t.split('"')[1]
                for d in (os.path.dirname(src), CSRC, os.path.join(ROOT, "include")):
                    cand = os.path.normpath(os.path.join(d, name))
                    if os.path.exists(cand):
                        _deps(cand, seen)
                        break
    return seen


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compiles the translation units (in parallel) whose object is older
    than one of its sources, and links libstereo.so (checked=True:
    libstereo_checked.so with -DSTEREO_CHECKED)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not needs_build(lib):
        return lib
    from concurrent.futures import ThreadPoolExecutor
    nvcc = os.environ.get("NVCC", "nvcc")
    bdir = os.path.join(ROOT, "_build", "stereo_checked" if checked else "stereo")
    os.makedirs(bdir, exist_ok=True)
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]
    if checked:
        flags.append("-DSTEREO_CHECKED")
    if verbose:
        flags.append("-Xptxas=-v")

    stamp = os.path.join(bdir, "flags.txt")
    same_flags = os.path.exists(stamp) and open(stamp).read() == " ".join(flags)

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        if not force and same_flags and os.path.exists(obj) and not verbose:
            t = os.path.getmtime(obj)
            if all(os.path.getmtime(d) <= t for d in _deps(src)):
                return obj
        r = subprocess.run([nvcc, *flags, "-c", "-o", obj, src], cwd=CSRC, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    tus = translation_units()
    with ThreadPoolExecutor(max_workers=min(8, len(tus))) as ex:
        objs = list(ex.map(compile_one, tus))
    with open(stamp, "w") as f:
        f.write(" ".join(flags))
    tmp = lib + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs], cwd=CSRC)
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> None:
    build(force=force)
    build(force=force, checked=True)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
