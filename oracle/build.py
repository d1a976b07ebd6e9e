"""Build the FP64 oracle shared library (test infrastructure only).

The oracle is plain C compiled with contraction of a*b+c into fused multiply-adds
switched off, so that every operation rounds exactly as written in the source.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rfi_oracle.c")
LIB = os.path.join(HERE, "_build", "librfi_oracle.so")


def compile_source(src: str, out: str) -> str:
    """Compile one C source file of the oracle into a shared library at `out`."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-Wall", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile rfi_oracle.c into oracle/_build/librfi_oracle.so; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    return compile_source(SRC, LIB)


if __name__ == "__main__":
    print(build(force=True))
