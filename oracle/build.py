"""Compile the oracle's C sources (FP64 and a float instantiation) with gcc.

Building the checker is not using it: ``__graft_entry__.build()`` calls this so
that the test suite finds the shared objects ready.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "am_oracle.c")
TARGETS = {"f64": os.path.join(HERE, "_am_oracle_f64.so"),
           "f32": os.path.join(HERE, "_am_oracle_f32.so")}


def build(force: bool = False) -> dict:
    for kind, out in TARGETS.items():
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
            continue
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", out, SRC, "-lm"]
        if kind == "f32":
            cmd.insert(1, "-DORACLE_REAL_FLOAT")
        subprocess.run(cmd, check=True)
    return dict(TARGETS)


if __name__ == "__main__":
    print(build(force=True))
