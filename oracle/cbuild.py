"""Builds the CPU oracle's C helper library (test infrastructure only)."""
import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "gravity.c")
LIB = os.path.join(HERE, "_liboracle.so")


def build(force=False):
    if force or not os.path.exists(LIB) or os.path.getmtime(SRC) > os.path.getmtime(LIB):
        tmp = LIB + ".tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


def load():
    lib = ctypes.CDLL(build())
    f = lib.oracle_gravity_direct
    f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double,
                  ctypes.c_void_p]
    f.restype = None
    return lib
