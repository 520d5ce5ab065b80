"""Build the FP64 CPU oracle shared library (test infrastructure only).

The oracle is compiled with -ffp-contract=off so that no fused multiply-add changes
its rounding; it is single-threaded on purpose.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libaforacle.so")
SRC = os.path.join(HERE, "af_oracle.cpp")


def build_oracle(force: bool = False) -> str:
    """Compile oracle/af_oracle.cpp into oracle/_build/libaforacle.so if stale."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC)):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared",
           "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build_oracle(force=True))
