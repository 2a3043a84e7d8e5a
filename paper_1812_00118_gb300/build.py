"""Build liblbm.so (CUDA, sm_103a) in-tree with nvcc.

Compiles csrc/lbm_tables.cu once per (lattice, storage) pair plus
csrc/lbm_api.cu, in parallel, and links paper_1812_00118_gb300/_lib/liblbm.so.
Object files go to paper_1812_00118_gb300/_build/.  A rebuild happens only
when a source or header is newer than the library.

    python -m paper_1812_00118_gb300.build
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "liblbm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _units():
    units = [("lbm_api", os.path.join(CSRC, "lbm_api.cu"), [])]
    for lat in (0, 1):
        for st in range(4):
            units.append((f"lbm_tables_l{lat}_s{st}", os.path.join(CSRC, "lbm_tables.cu"),
                          [f"-DLBM_LAT={lat}", f"-DLBM_ST={st}"]))
    for extra in sorted(os.listdir(CSRC)):
        if extra.endswith(".cu") and extra not in ("lbm_api.cu", "lbm_tables.cu"):
            units.append((extra[:-3], os.path.join(CSRC, extra), []))
    return units


def _sources_mtime():
    newest = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            newest = max(newest, os.path.getmtime(os.path.join(d, f)))
    newest = max(newest, os.path.getmtime(os.path.abspath(__file__)))
    return newest


CHECKED_LIB = os.path.join(LIBDIR, "liblbm_checked.so")


def build(force=False, verbose=False, checked=False):
    """Compile and link; returns the path of liblbm.so.  With `checked`, the
    debugging variant liblbm_checked.so (LBM_CHECKED: the step kernels check
    their offsets against the population arrays; lbm_checked_status), built
    into its own object directory; the default build never includes it."""
    lib_path = CHECKED_LIB if checked else LIB
    obj_dir = BUILD + ("_checked" if checked else "")
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= _sources_mtime():
        return lib_path
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    extra = ["-DLBM_CHECKED"] if checked else []

    def compile_one(unit):
        name, src, defs = unit
        obj = os.path.join(obj_dir, name + ".o")
        cmd = [cc] + ARCH + FLAGS + extra + defs + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(f"compiled {name}", flush=True)
        return obj

    units = _units()
    with ThreadPoolExecutor(max_workers=min(len(units), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = lib_path + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
