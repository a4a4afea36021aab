"""Build step of libsawave.so: nvcc for sm_103a, one object per source compiled in parallel.

The library is built in-tree (paper_2511_18071_gb300/_build/libsawave.so) and
loaded by the ctypes binding in this package.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsawave.so")
# (source, object, defines): the persistent solve kernel and the batch kernel
# are compiled once per variant, so that the variants build in parallel
_SOLVE = [("f64_p2", "double", "WM_PERIODIC|WM_2D"), ("f64_p3", "double", "WM_PERIODIC|WM_3D"),
          ("f64_w2", "double", "WM_WALLS|WM_2D"), ("f32_p2", "float", "WM_PERIODIC|WM_2D"),
          ("f32_p3", "float", "WM_PERIODIC|WM_3D"), ("f32_w2", "float", "WM_WALLS|WM_2D")]
_BATCH = [("block_f64", "double", 0), ("block_f32", "float", 0), ("cluster_f64", "double", 1),
          ("cluster_f32", "float", 1)]
UNITS = ([("batch_kernel.cu", "batch_%s.o" % t, ["-DSW_TI=%s" % ti, "-DSW_CLUSTER=%d" % c,
                                                  "-DSW_NAME=batch_kernel_%s" % t]) for t, ti, c in _BATCH] +
         [("solve_kernel.cu", "solve_%s.o" % t, ["-DSW_TI=%s" % ti, "-DSW_WM=(%s)" % wm,
                                                  "-DSW_NAME=solve_kernel_%s" % t]) for t, ti, wm in _SOLVE] +
         [(f, f.replace(".cu", ".o"), []) for f in ("resident.cu", "streamed.cu", "setup.cu", "solver.cu", "driver.cu", "batch.cu",
                                                     "noalloc.cu")])
SOURCES = sorted({u[0] for u in UNITS})
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-Xcompiler", "-pthread", "--expt-relaxed-constexpr"]


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "sawave.h"))
    return files


def build(force=False, verbose=False):
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in _deps()):
            return LIB
    os.makedirs(OUT, exist_ok=True)
    nv = nvcc()

    newest = max(os.path.getmtime(d) for d in _deps())

    def comp(unit):
        src, objname, defs = unit
        obj = os.path.join(OUT, objname)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) > newest:
            return obj
        cmd = [nv] + ARCH + FLAGS + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s %s:\n%s%s" % (src, " ".join(defs), r.stdout, r.stderr))
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    # the slowest units first, all in parallel
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(UNITS), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(comp, UNITS))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nv] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
