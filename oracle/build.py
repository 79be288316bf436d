"""Builds the CPU oracle (test infrastructure) with the host C++ compiler.

Only tests/, __graft_entry__ and bench.py's cpu_baseline / reference legs use
the result.  `build(mutant=n)` builds a variant with one planted mistake for
the oracle's own mutation tests.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ash_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")


def lib_path(mutant: int = 0) -> str:
    name = "libash_oracle.so" if mutant == 0 else f"libash_oracle_mutant{mutant}.so"
    return os.path.join(OUT_DIR, name)


def build(mutant: int = 0, force: bool = False) -> str:
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    # -ffp-contract=off: float32 steps stay separately rounded on every host
    # (Arm compilers contract a * b + c into a fused multiply-add otherwise).
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", f"-DORACLE_MUTANT={mutant}", SRC,
           "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
