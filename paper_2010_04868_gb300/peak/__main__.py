"""FP64 and integer pipe rates of the current GPU: python -m paper_2010_04868_gb300.peak [--sweep]."""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    """Compile fp64_peak.cu for sm_103a, run it and print its JSON (one object per swept shape with --sweep)."""
    exe = os.path.join(tempfile.gettempdir(), "gb300_fp64_peak_%d" % os.getpid())
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                           os.path.join(HERE, "fp64_peak.cu")])
    try:
        out = subprocess.run([exe] + sys.argv[1:2], capture_output=True, text=True, timeout=300)
        sys.stdout.write(out.stdout)
        return out.returncode
    finally:
        os.remove(exe)


if __name__ == "__main__":
    sys.exit(main())
