"""Build the FP64 CPU oracle (test infrastructure only) into oracle/_build/liboracle.so.

Plain gcc, no fast-math and no FMA contraction, so that every operation is the
IEEE double operation the source spells out.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["or_grid.c", "or_geom.c", "or_physics.c", "or_api.c", "or_adjoint.c"]
HEADERS = ["rt_oracle.h", "or_internal.h"]
OUT = os.path.join(HERE, "_build", "liboracle.so")


def build(force: bool = False, mutant: int = 0) -> str:
    """Build the oracle.  mutant > 0 builds a separate library with one planted
    mistake (OR_MUTANT in or_physics.c); only the test that shows the pins
    catch such mistakes loads it."""
    out = OUT if not mutant else os.path.join(HERE, "_build", "liboracle_m%d.so" % int(mutant))
    deps = [os.path.join(HERE, s) for s in SOURCES + HEADERS]
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in deps):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", "-Wall", "-Wno-unused-function", "-DOR_MUTANT=%d" % int(mutant), "-o", tmp]
    cmd += [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
