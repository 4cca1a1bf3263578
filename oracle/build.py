"""Compile the oracle's C time loop (oracle/forward.c -> oracle/_oracle_forward.so).

Test infrastructure only.  Plain gcc, portable flags (x86_64 and aarch64), OpenMP when
the compiler supports it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def build(verbose=False):
    src = os.path.join(HERE, "forward.c")
    out = os.path.join(HERE, "_oracle_forward.so")
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math", "-ffp-contract=off", src, "-o", out, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=not verbose)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=not verbose)
    return out


if __name__ == "__main__":
    print(build(verbose=True))
