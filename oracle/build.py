"""Compile the CPU oracle (plain C, gcc) into oracle/_build/.

TEST INFRASTRUCTURE ONLY (see oracle.c).  ``mutant=k`` builds a copy with a
deliberately planted mistake, used only by the tests that show the oracle's
pins detect such mistakes.
"""

from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")


def lib_path(mutant: int = 0) -> str:
    name = "liborc.so" if mutant == 0 else f"liborc_mut{mutant}.so"
    return os.path.join(BUILD_DIR, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Build (if stale) and return the shared-library path."""
    out = lib_path(mutant)
    src = os.path.join(HERE, "oracle.c")
    hdr = os.path.join(HERE, "oracle.h")
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(src),
                                             os.path.getmtime(hdr))):
        return out
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
           "-fPIC", "-shared", f"-DORC_MUTANT={mutant}", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
