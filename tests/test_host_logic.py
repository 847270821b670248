"""CPU checks of the CUDA library's host-side logic and of its C ABI surface
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1302_4587_gb300", "csrc")


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "lm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lm_[a-z_]+)\s*\(", src)))


def test_library_loads_and_exports_every_declared_symbol():
    import paper_1302_4587_gb300 as lm
    lib = lm.load()
    declared = _declared_functions()
    assert "lm_match" in declared and "lm_batch_match" in declared and "lm_submit" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(lm.EXPORTS) | set(declared)
    nm = subprocess.run(["nm", "-D", "--defined-only", lm._build.LIB], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in nm.splitlines() if " T " in l}
    assert set(declared) <= exported
    # nothing beyond the header leaks out as an lm_ symbol
    assert {s for s in exported if s.startswith("lm_")} == set(declared)


def test_strerror_without_gpu():
    import paper_1302_4587_gb300 as lm
    assert lm.lm_strerror(lm.LM_OK) == "ok"
    assert "invalid" in lm.lm_strerror(lm.LM_EINVAL)
    assert lm.lm_strerror(999) == "unknown error"


def test_kernels_compile_for_sm103a():
    # -Xptxas -v report of the kernel translation unit (compile only, no GPU)
    out = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xptxas", "-v",
                          "-I" + CSRC, "-c", os.path.join(CSRC, "lm_kernels.cu"), "-o", os.devnull],
                         capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    for k in ("k_vertex", "k_sweep", "k_init"):
        assert k in out.stderr
