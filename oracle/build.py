"""Compile the oracle's C sources with the host compiler (test infrastructure).

The flags keep the arithmetic plain IEEE: no fast-math and no contraction of
a*b+c into fused multiply-adds, on x86-64 and aarch64 alike.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
SOURCES = ["rbsm_oracle.c", "shadow_map_oracle.c"]
LIB_NAME = "liboracle_rbsm.so"
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wextra"]


def lib_path():
    return os.path.join(BUILD_DIR, LIB_NAME)


def _stale(out, srcs):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force=False):
    """Build the oracle library if it is missing or older than its sources."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    out = lib_path()
    if force or _stale(out, srcs):
        tmp = out + ".tmp%d" % os.getpid()
        cmd = [os.environ.get("CC", "gcc")] + CFLAGS + srcs + ["-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
