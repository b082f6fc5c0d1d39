"""Builds the exact CPU oracle (test infrastructure only).

Two builds of the same C source differ only in integer width: 128-bit limbs
(fast, used first) and 384-bit limbs (rerun when the 128-bit build reports an
overflow).  Output: oracle/libsg2v_oracle_nl2.so and oracle/libsg2v_oracle_nl6.so.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sg2v_oracle.c")
WIDTHS = (2, 6)


def lib_path(limbs: int) -> str:
    return os.path.join(HERE, f"libsg2v_oracle_nl{limbs}.so")


def build(force: bool = False, verbose: bool = False) -> None:
    for nl in WIDTHS:
        out = lib_path(nl)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
            continue
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", f"-DNL={nl}",
               "-Wall", "-Wextra", "-o", out, SRC]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
