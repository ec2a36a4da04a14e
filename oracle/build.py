"""Compile the CPU oracle into ``oracle/liboracle.so`` (plain g++, no fast-math).

Test infrastructure: the oracle is built by ``__graft_entry__.build()`` so the
checker exists on every machine the tests run on; building it is not using it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "oracle.cpp")
    hdr = os.path.join(HERE, "oracle.h")
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr)):
        return SO
    tmp = SO + ".tmp"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-fno-fast-math",
                    "-ffp-contract=off", "-o", tmp, src], check=True)
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force=True))
