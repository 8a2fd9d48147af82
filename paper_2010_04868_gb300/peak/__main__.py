import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    exe = os.path.join(tempfile.gettempdir(), "gb300_fp64_peak_%d" % os.getpid())
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                           os.path.join(HERE, "fp64_peak.cu")])
    try:
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        sys.stdout.write(out.stdout)
        return out.returncode
    finally:
        os.remove(exe)


if __name__ == "__main__":
    sys.exit(main())
