"""Register budgets the plain Jacobi kernels' speed rests on, checked from ptxas's own report.

The 2D radius-1 and 3D 7-point plain kernels are capped at 64 registers so that
4 CTAs of 256 threads stay resident per SM (3 resident CTAs measured ~6 % slower
on the 4096^2 5-point step); the cap must not cost spills. nvcc cross-compiles,
so this runs without a GPU.
"""
import os
import re
import shutil
import subprocess

import pytest

from paper_2010_04868_gb300 import build as B

# (dim, shape, radius) -> most registers allowed; shape 0 = star, 1 = box
BUDGET = {(2, 0, 1): 64, (2, 1, 1): 64, (3, 0, 1): 64, (2, 0, 2): 80}


def _ptxas_report(tmp_path):
    nvcc = B._nvcc()
    if shutil.which(nvcc) is None and not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = os.path.join(B.CSRC, "k_plain.cu")
    cmd = [nvcc] + B.ARCH + B.FLAGS + ["-Xptxas", "-v", "-c", src, "-o", str(tmp_path / "k_plain.o")]
    p = subprocess.run(cmd, capture_output=True, text=True)
    assert p.returncode == 0, p.stderr[-2000:]
    return p.stdout + p.stderr


def test_plain_jacobi_register_budgets(tmp_path):
    report = _ptxas_report(tmp_path)
    seen = {}
    kernel = None
    for line in report.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            kernel = m.group(1)
            continue
        if kernel is None or "k_jacobi_plainILi" not in kernel or "WArr" not in kernel:
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m:
            spill = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            t = re.search(r"k_jacobi_plainILi(\d)ELi(\d)ELi(\d)E", kernel)
            key = tuple(int(x) for x in t.groups())
            seen.setdefault(key, []).append((int(m.group(1)), spill))
            kernel = None
    for key, limit in BUDGET.items():
        assert key in seen, ("no ptxas report for", key)
        for regs, spill in seen[key]:
            assert regs <= limit, (key, regs, limit)
            assert spill == 0, (key, spill)
