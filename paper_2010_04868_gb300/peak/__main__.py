import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    """FP64 and integer pipe rates (default), or with --sync the level-loop and FP64-sharing probes."""
    src = "sync_probes.cu" if "--sync" in sys.argv[1:] else "fp64_peak.cu"
    exe = os.path.join(tempfile.gettempdir(), "gb300_%s_%d" % (src[:-3], os.getpid()))
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                           os.path.join(HERE, src)])
    try:
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        sys.stdout.write(out.stdout)
        return out.returncode
    finally:
        os.remove(exe)


if __name__ == "__main__":
    sys.exit(main())
