"""Build libpqmc.so in-tree for sm_103a (nvcc + g++, translation units compiled in parallel)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpqmc.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["sweep.cu", "sweep_f64.cu", "sweep_f32.cu", "sweep_f32_256.cu", "sweep_f32_512.cu",
              "sweep_f32_dense.cu", "spread_f64.cu", "spread_f32.cu", "probe.cu"]
CPP_SOURCES = ["api.cpp", "model.cpp"]


def _cmds():
    os.makedirs(OUT_DIR, exist_ok=True)
    inc = ["-I" + CSRC, "-I" + os.path.join(os.path.dirname(HERE), "include"), "-I" + os.path.join(CUDA, "include")]
    cmds, objs = [], []
    for s in CU_SOURCES:
        o = os.path.join(OUT_DIR, s + ".o")
        cmds.append([NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "--expt-relaxed-constexpr", *inc, "-c", os.path.join(CSRC, s), "-o", o])
        objs.append(o)
    for s in CPP_SOURCES:
        o = os.path.join(OUT_DIR, s + ".o")
        cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", *inc, "-c", os.path.join(CSRC, s), "-o", o])
        objs.append(o)
    link = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", LIB, *objs,
            "-Xlinker", "-rpath," + os.path.join(CUDA, "lib64")]
    return cmds, link


def build(verbose=False):
    cmds, link = _cmds()
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    failed = []
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(" ".join(c) + "\n" + out)
        if p.returncode != 0:
            failed.append(c[-3])
    if failed:
        raise RuntimeError("compile failed: %s" % failed)
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        sys.stderr.write(" ".join(link) + "\n" + r.stdout)
        raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
