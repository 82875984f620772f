"""Compile the user-law test source against include/fdps_user_force.cuh."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "user_kernels", "user_laws.cu")
OUT = os.path.join(ROOT, "tests", "_build")


def compile_object() -> str:
    """nvcc -c only (no GPU, no link): the header template instantiates."""
    from paper_1601_03138_gb300 import build as B
    os.makedirs(OUT, exist_ok=True)
    obj = os.path.join(OUT, "user_laws.o")
    subprocess.run([B.nvcc(), *B.ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "include"), "-c", SRC, "-o", obj], check=True)
    return obj


def build_library() -> str:
    """Shared library of the user laws, linked to the FDPS library."""
    from paper_1601_03138_gb300 import build as B
    lib = B.build()
    os.makedirs(OUT, exist_ok=True)
    so = os.path.join(OUT, "libuser_laws.so")
    libdir = os.path.dirname(lib)
    subprocess.run([B.nvcc(), *B.ARCH, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "include"), SRC, "-o", so, "-L", libdir, "-lfdpsgpu",
                    "-Xlinker", "-rpath," + libdir, "-cudart", "shared"], check=True)
    return so
