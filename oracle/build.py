"""Build the FP64 CPU oracle shared library (test infrastructure only).

The oracle is compiled with -ffp-contract=off so that no fused multiply-add changes
its rounding; it is single-threaded on purpose.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libaforacle.so")
SRC = os.path.join(HERE, "af_oracle.cpp")


def build_oracle(force: bool = False, defines: dict | None = None) -> str:
    """Compile oracle/af_oracle.cpp into oracle/_build/libaforacle.so if stale.

    ``defines`` builds a separate variant library with those preprocessor macros (the
    planted-mistake builds of the pin tests); the oracle itself takes none."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    path = LIB_PATH
    flags = []
    if defines:
        tag = "_".join(f"{k}-{v}" for k, v in sorted(defines.items())).replace(".", "p")
        path = os.path.join(BUILD_DIR, f"libaforacle_{tag}.so")
        flags = [f"-D{k}={v}" for k, v in sorted(defines.items())]
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared",
           *flags, "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


if __name__ == "__main__":
    print(build_oracle(force=True))
