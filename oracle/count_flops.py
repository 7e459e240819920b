"""Floating-point operations of one step of the FP64 oracle, per cell update.

TEST INFRASTRUCTURE: run by its test and by hand; the bench reads the JSON it
writes (flops_per_cell.json beside this file) as the algorithmic flop count of
the FP64 roofline.

count_flops.cpp compiles the unchanged oracle source with its scalar type
replaced by a counting one and runs one step (not the first) of a 64 x 64
periodic problem: the coupled model on a spinodal-like field, and the
Allen-Cahn model with a uniform velocity.  Two counts per cell:
  flops_per_cell           every +, -, *, / and sqrt the plain oracle performs
                           (it recomputes invariants, e.g. relaxation
                           coefficients for each direction);
  distinct_flops_per_cell  the same with each operation on the same operand
                           values counted once and identities (x * 0, x * 1,
                           x + 0, ...) left out: the method's own work, used as
                           the algorithmic flops of a step.

  python oracle/count_flops.py          # prints both models' counts
  python oracle/count_flops.py --write  # also rewrites flops_per_cell.json
"""
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
EXE = os.path.join(BUILD_DIR, "count_flops")
JSON_PATH = os.path.join(HERE, "flops_per_cell.json")


def build():
    os.makedirs(BUILD_DIR, exist_ok=True)
    src = os.path.join(HERE, "count_flops.cpp")
    deps = [src, os.path.join(HERE, "dugks_oracle.c"), os.path.join(HERE, "dugks_oracle.h")]
    if os.path.exists(EXE) and all(os.path.getmtime(d) <= os.path.getmtime(EXE) for d in deps):
        return EXE
    tmp = EXE + ".tmp.%d" % os.getpid()
    # -fpermissive: the C source assigns malloc's void * without a cast
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fpermissive", "-w", "-I", HERE, "-o", tmp, src], check=True)
    os.replace(tmp, EXE)
    return EXE


def count():
    exe = build()
    out = {}
    for flag, name in (("1", "coupled"), ("0", "allen-cahn")):
        res = subprocess.run([exe, flag], check=True, capture_output=True, text=True)
        out[name] = json.loads(res.stdout)
    return out


def stored():
    with open(JSON_PATH) as fh:
        return json.load(fh)


if __name__ == "__main__":
    counts = count()
    print(json.dumps(counts, indent=1))
    if "--write" in sys.argv:
        with open(JSON_PATH, "w") as fh:
            json.dump(counts, fh, indent=1)
            fh.write("\n")
