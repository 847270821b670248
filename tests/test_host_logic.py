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


def test_binding_structs_match_the_header(tmp_path):
    # every struct the binding passes through the C ABI has the header's field names,
    # order, offsets and sizes, as a C compiler lays them out from include/lm.h
    import paper_1302_4587_gb300 as lm
    structs = {"lm_config": lm.binding.LmConfig, "lm_stats": lm.binding.LmStats, "lm_tuning": lm.binding.LmTuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname}.{fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                         f'sizeof((({cname}*)0)->{fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    run = subprocess.run([str(exe)], capture_output=True, text=True, check=True)
    out = dict(l.split(" ", 1) for l in run.stdout.splitlines())  # name -> "size" or "offset size"
    for cname, py in structs.items():
        assert int(out[cname].split()[-1]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            off, size = (int(x) for x in out[f"{cname}.{fname}"].split())
            field = getattr(py, fname)
            assert (field.offset, field.size) == (off, size), (cname, fname)
    # and the header declares no field the binding lacks
    hdr = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "lm.h")).read(), flags=re.S)
    for cname, py in structs.items():
        body = re.search(r"typedef struct\s*\w*\s*\{([^}]*)\}\s*" + cname + ";", hdr).group(1)
        names = re.findall(r"(\w+)\s*(?:\[[^\]]*\])?\s*;", body)
        assert names == [f for f, _ in py._fields_], cname


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


def test_output_buffers_are_checked_before_any_call():
    # the library writes n 4-byte elements through an output pointer: the
    # binding refuses buffers that are short, of another element size,
    # strided or read-only instead of handing them over
    import numpy as np
    import torch
    from paper_1302_4587_gb300 import binding as B
    ok = np.empty(5, np.uint32)
    assert B._out(ok, 5, "mate")[1] is ok
    B._out(np.empty(6, np.int32), 5, "mate")  # longer is fine
    for bad in (np.empty(4, np.uint32), np.empty(5, np.int64), np.empty(10, np.uint32)[::2],
                np.frombuffer(bytes(20), np.uint32)):
        with pytest.raises(ValueError):
            B._out(bad, 5, "mate")
    t = torch.empty(5, dtype=torch.int32)
    assert B._out(t, 5, "mate")[1] is t
    for bad in (torch.empty(4, dtype=torch.int32), torch.empty(5, dtype=torch.int64),
                torch.empty(10, dtype=torch.int32)[::2]):
        with pytest.raises(ValueError):
            B._out(bad, 5, "mate")
    with pytest.raises(TypeError):
        B._out([0] * 5, 5, "mate")


def test_contraction_arguments_are_checked_before_any_call():
    import torch
    from paper_1302_4587_gb300 import binding as B
    i32 = lambda k: torch.zeros(k, dtype=torch.int32)
    f32 = lambda k: torch.zeros(k, dtype=torch.float32)
    for args in ((i32(2), i32(3), f32(2), i32(3)),                         # ev longer than eu
                 (i32(2), i32(2), torch.zeros(2, dtype=torch.float64), i32(3)),  # 8-byte weights
                 (i32(2), i32(2), f32(2), i32(2)),                         # mate shorter than n
                 (i32(4)[::2], i32(2), f32(2), i32(3))):                   # strided endpoints
        with pytest.raises(ValueError):
            B.lm_contract(None, 3, *args)
    with pytest.raises(ValueError):
        B.lm_contract(None, 3, i32(2), i32(2), f32(2), i32(3), vw=i32(2))  # vertex weights short


class _FakeLib:
    """Stands in for the CUDA library: records calls, fills out-parameters."""

    def __init__(self):
        self.calls = []

    def lm_graph_create(self, ctx, n, m, pu, pv, pw, mem, out):
        out._obj.value = 0x1000 + n
        self.calls.append(("create", n, m, mem))
        return 0

    def lm_graph_destroy(self, g):
        self.calls.append(("destroy", g.value))

    def lm_graph_info(self, g, n, m, b):
        n._obj.value, m._obj.value, b._obj.value = 9, 0, 0
        return 0

    def lm_match(self, ctx, g, seed, p, st):
        self.calls.append(("match", g.value, p))
        return 0

    def lm_batch_match(self, ctx, gs, count, seeds, mates, st):
        self.calls.append(("batch", count))
        return 0

    def lm_submit(self, ctx, g, seed, p, t):
        t._obj.value = 7
        return 0


def test_binding_marshals_graphs_and_outputs(monkeypatch):
    import numpy as np
    from paper_1302_4587_gb300 import binding as B
    fake = _FakeLib()
    monkeypatch.setattr(B, "load", lambda build=True: fake)
    eu, ev = np.array([0, 1], np.uint32), np.array([1, 2], np.uint32)
    h = B.lm_graph_create(None, 5, eu, ev, np.array([1, 2], np.float32))
    assert fake.calls[-1] == ("create", 5, 2, B.LM_HOST)
    mate = np.empty(5, np.uint32)
    assert B.lm_match(None, h, 1, mate) is mate
    assert fake.calls[-1] == ("match", h.value, mate.ctypes.data)
    with pytest.raises(ValueError):
        B.lm_match(None, h, 1, np.empty(4, np.uint32))
    job = B.BatchArgs([h, h], [1, 2], [mate, np.empty(6, np.uint32)])
    assert B.lm_batch_match(None, job)[0] is mate and fake.calls[-1] == ("batch", 2)
    with pytest.raises(ValueError):
        B.BatchArgs([h], [1], [np.empty(3, np.uint32)])
    assert B.lm_submit(None, h, 3, mate) == 7
    B.lm_graph_destroy(h)
    assert fake.calls[-1] == ("destroy", h.value)
    # a handle the binding no longer knows is sized through lm_graph_info (n = 9 here)
    with pytest.raises(ValueError):
        B.lm_match(None, h, 1, mate)
    B.lm_match(None, h, 1, np.empty(9, np.uint32))
