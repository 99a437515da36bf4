"""Compile and run one microbenchmark: python -m paper_2201_10956_gb300.microbench NAME."""
import os
import subprocess
import sys

from paper_2201_10956_gb300 import build as B

HERE = os.path.dirname(os.path.abspath(__file__))


def main(argv):
    names = sorted(f[:-3] for f in os.listdir(HERE) if f.endswith(".cu"))
    if len(argv) != 1 or argv[0] not in names:
        sys.stderr.write("usage: python -m paper_2201_10956_gb300.microbench {%s}\n" % "|".join(names))
        return 2
    os.makedirs(B.BUILD, exist_ok=True)
    exe = os.path.join(B.BUILD, "mb_" + argv[0])
    src = os.path.join(HERE, argv[0] + ".cu")
    subprocess.check_call([B.nvcc(), *B.ARCH, "-O3", "-std=c++17", "-o", exe, src])
    return subprocess.call([exe])


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
