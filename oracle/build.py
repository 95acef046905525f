"""Compile the dense CPU oracle (TEST INFRASTRUCTURE ONLY).

Builds oracle/_build/libtdh_oracle.so from tdh_oracle.c with gcc.  OpenMP is used
when the compiler supports it.  -ffp-contract=off keeps the double-double arithmetic
free of fused multiply-adds, so the oracle gives the same bits on x86-64 and aarch64.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tdh_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libtdh_oracle.so")


def build(force=False, verbose=False):
    """Compile the oracle shared library if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", SRC,
            "-o", LIB + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if verbose:
            print(" ".join(cmd), res.stdout, res.stderr)
        if res.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            return LIB
    raise RuntimeError("oracle build failed:\n" + res.stderr)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
