import os
import subprocess
import sys

from .. import build

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    exe = os.path.join(build.BUILD, "alu_peak")
    os.makedirs(build.BUILD, exist_ok=True)
    subprocess.run([build.nvcc(), *build.ARCH, "-O3", "-o", exe, os.path.join(HERE, "alu_peak.cu")], check=True)
    sys.exit(subprocess.run([exe]).returncode)


if __name__ == "__main__":
    main()
