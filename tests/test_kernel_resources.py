"""Register and local-memory use of the hot kernels, from the compiler's
resource report (`-Xptxas -v`), built exactly as the library is.

The partition merge runs five CTAs of 256 threads per SM, so it has at most
48 registers; everything else on the main path keeps its keys,
parameters and partition function out of local memory (an array indexed at
run time is placed there, and every access then goes through L1).  Runs on
the CPU: nvcc cross-compiles, nothing is launched.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2601_14400_gb300", "csrc")


def _report(src, tmp_path):
    from paper_2601_14400_gb300 import _build
    try:
        nvcc = _build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    cmd = [nvcc] + _build.ARCH + list(_build.NVCC_FLAGS)
    cmd += ["-Xptxas", "-v", "-c", os.path.join(CSRC, src), "-o", str(tmp_path / "k.o")]
    out = subprocess.run(cmd, capture_output=True, text=True, check=True).stderr
    names = subprocess.run([shutil.which("c++filt") or "c++filt"],
                           input="\n".join(re.findall(r"function '([^']+)'", out)),
                           capture_output=True, text=True).stdout.splitlines()
    res, i = {}, 0
    for line in out.splitlines():
        if "Compiling entry function" in line:
            cur = names[i]
            i += 1
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            res[cur] = tuple(int(v) for v in m.groups())
        m = re.search(r"Used (\d+) registers", line)
        if m:
            res[cur + " regs"] = int(m.group(1))
    return res


def _find(res, *parts):
    keys = [k for k in res if all(p in k for p in parts) and not k.endswith(" regs")]
    assert len(keys) == 1, (parts, keys)
    return keys[0]


def test_partition_kernels(tmp_path):
    res = _report("itpp_part.cu", tmp_path)
    for W in (1, 2):
        k = _find(res, f"k_part_scatter<{W}>")
        assert res[k] == (0, 0, 0), (k, res[k])
    # the staged merge: five CTAs of 256 per SM (48 registers), no local memory
    k = _find(res, "k_gate_part<1, 256>")
    assert res[k + " regs"] <= 48
    assert res[k] == (0, 0, 0), (k, res[k])
    k = _find(res, "k_gate_part<2, 256>")
    assert res[k + " regs"] <= 48
    assert res[k][1] <= 64 and res[k][2] <= 64, (k, res[k])   # a few spilled bytes at most


def test_select_streaming_kernels(tmp_path):
    res = _report("itpp_select.cu", tmp_path)
    for name in ("k_sel_hist", "k_sel_gather"):
        for W in (1, 2):
            k = _find(res, f"{name}<{W}>")
            assert res[k] == (0, 0, 0), (k, res[k])
