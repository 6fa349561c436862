"""Build libhofem.so in-tree with nvcc for sm_103a (GB300).

Every translation unit under csrc/ is compiled in parallel to _build/*.o and linked
into lib/libhofem.so.  No CMake; only nvcc and the host compiler it drives.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libhofem.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libhofem")
    return exe


# Sources compiled more than once, each time with one macro: the sweep kernels' FP32 and
# FP64 instantiations (the longest compile) build in parallel with the host helpers.
PARTS = {"sweep.cu": ["HOFEM_SWEEP_PART=0", "HOFEM_SWEEP_PART=1", "HOFEM_SWEEP_PART=2"],
         "sweep_reg.cu": [f"HOFEM_REG_PART={k}" for k in range(15)] + ["HOFEM_REG_PART=100"]}


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def jobs():
    """(source, extra macro or None, object name) for every object of the library."""
    out = []
    for src in sources():
        base = os.path.basename(src)[:-3]
        parts = PARTS.get(os.path.basename(src))
        if parts:
            out += [(src, d, f"{base}_p{i}.o") for i, d in enumerate(parts)]
        else:
            out.append((src, None, base + ".o"))
    return out


def _compile(job, verbose=False, defines=()):
    src, part, name = job
    obj = os.path.join(BUILD, name)
    extra = [part] if part else []
    cmd = [nvcc(), *ARCH, *FLAGS, *[f"-D{d}" for d in (*defines, *extra)], "-c", src, "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    return obj, res.stderr


def build(verbose=False, force=False, lib=None, defines=()):
    """Compile and link; `lib` / `defines` build a variant library (tuning experiments)."""
    global BUILD
    target = lib or LIB
    if lib:
        BUILD = lib + ".objs"
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(os.path.dirname(target), exist_ok=True)
    srcs = sources()
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "hofem.h"))
    if not force and os.path.exists(target):
        lib_t = os.path.getmtime(target)
        if all(os.path.getmtime(d) <= lib_t for d in deps):
            return target
    todo = jobs()
    with cf.ThreadPoolExecutor(max_workers=min(max(os.cpu_count() or 1, 1), 16, len(todo))) as ex:
        results = list(ex.map(lambda j: _compile(j, verbose, defines), todo))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = target + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
