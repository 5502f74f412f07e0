"""Builds libbp4m.so in-tree: the CUDA kernels for sm_103a, the C-ABI layer and the host
graph builder.  Usage: python -m paper_2603_05381_gb300.build [--force] [--verbose]."""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbp4m.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SRCS = ["capi.cu", "kernels_decode.cu", "kernels_half.cu", "kernels_cluster.cu", "kernels_cluster_half.cu",
             "kernels_rw.cu", "kernels_misc.cu", "kernels_bbp.cu", "kernels_reg.cu"]
CXX_SRCS = ["host_graph.cpp"]
HEADERS = ["device.cuh", "decode_smem.cuh", "decode_stream.cuh", "decode_reg.cuh", "host_graph.h"]


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(cuda, "bin", "nvcc")
    return path if os.path.exists(path) else "nvcc"


def _commands():
    nvcc = _nvcc()
    # no floating-point contraction in host code: the graph builder must reproduce the plain
    # IEEE results of its expressions (merged probabilities, path sums)
    common_host = "-fPIC,-O2,-ffp-contract=off,-pthread"
    cmds = []
    for src in CUDA_SRCS:
        obj = os.path.join(BUILD, src + ".o")
        cmds.append((obj, src, [nvcc, "-c", os.path.join(CSRC, src), "-o", obj, *ARCH, "-O3",
                                "-lineinfo", "-std=c++17", "-I", INCLUDE, "-I", CSRC,
                                "-Xcompiler", common_host, "-Xptxas", "-v"]))
    for src in CXX_SRCS:
        obj = os.path.join(BUILD, src + ".o")
        cmds.append((obj, src, ["g++", "-c", os.path.join(CSRC, src), "-o", obj, "-O2", "-fPIC",
                                "-ffp-contract=off", "-std=c++17", "-pthread", "-I", INCLUDE, "-I", CSRC]))
    return cmds


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [os.path.join(CSRC, src)] + [os.path.join(CSRC, h) for h in HEADERS] + [
        os.path.join(INCLUDE, "bp4m.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compiles every translation unit (in parallel) and links the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    cmds = _commands()
    todo = [(obj, src, cmd) for (obj, src, cmd) in cmds if force or _stale(obj, src)]

    def run(item):
        obj, src, cmd = item
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, cmd, r

    logs = []
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(todo))) as ex:
        for src, cmd, r in ex.map(run, todo):
            logs.append((src, r.stdout + r.stderr))
            if r.returncode != 0:
                raise RuntimeError("compiling %s failed:\n%s\n%s" % (src, " ".join(cmd), r.stdout + r.stderr))
    with open(os.path.join(BUILD, "ptxas.log"), "a") as f:
        for src, text in logs:
            f.write("== %s\n%s\n" % (src, text))
    objs = [obj for (obj, _, _) in cmds]
    if force or todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [_nvcc(), "-shared", *ARCH, "-o", LIB, *objs, "-Xcompiler", "-pthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("linking failed:\n%s\n%s" % (" ".join(cmd), r.stdout + r.stderr))
    if verbose:
        for src, text in logs:
            print("==", src)
            print(text)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(LIB)
