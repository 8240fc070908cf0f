"""The C-ABI library loads, exports every declared symbol, and its structs match ctypes.

CPU-only: nothing here launches device work.
"""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_1704_07458_gb300 as gb
from paper_1704_07458_gb300 import _native, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lobpcg.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _native.load()


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|void|const char\s*\*)\s+(lobpcg_\w+)\s*\(",
                                 txt, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(_native.EXPORTED) == names


def test_exported_symbols_are_only_the_abi(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True,
                         text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert syms == set(declared_functions())


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "lobpcg.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(lobpcg_options_t), offsetof(lobpcg_options_t, tau_ortho),
         offsetof(lobpcg_options_t, max_seconds), sizeof(lobpcg_stats_t));
  printf("%zu %zu\n", offsetof(lobpcg_stats_t, norm_a), offsetof(lobpcg_stats_t, ms_total));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    O, S = _native.lobpcg_options_t, _native.lobpcg_stats_t
    assert vals == [ctypes.sizeof(O), O.tau_ortho.offset, O.max_seconds.offset, ctypes.sizeof(S),
                    S.norm_a.offset, S.ms_total.offset]


def test_host_side_argument_errors_without_gpu(lib):
    """Argument validation happens before any device call."""
    assert gb.lobpcg_create.__name__ == "lobpcg_create"
    assert lib.lobpcg_gram_workspace(-1, 2, 2, 0, 0) == -1
    assert lib.lobpcg_gram(10, None, 1, 4, None, 4, 4, None, 4, 0, 0, None, 0, None) == gb.LOBPCG_ERR_ARG
    assert lib.lobpcg_update(10, None, 4, 4, None, 4, 4, 1.0, 0.0, None, 0, None, 4, 0, 0, None) == gb.LOBPCG_ERR_ARG
    assert lib.lobpcg_spmm(-1, None, None, None, None, 0, 1, None, 1, None, None, 0, None) == gb.LOBPCG_ERR_ARG
    assert lib.lobpcg_residual(0, None, None, None, 1, 1, 0, None, None, None, 1, 1.0, 1.0, None, None) == gb.LOBPCG_ERR_ARG
    assert lib.lobpcg_create(None, None, None) == gb.LOBPCG_ERR_ARG
    assert lib.lobpcg_get_stats(None, None) == gb.LOBPCG_ERR_ARG
    assert lib.lobpcg_last_error(None) == b"null handle"
    assert lib.lobpcg_wait_selftest(0, None) == gb.LOBPCG_ERR_ARG
    assert lib.lobpcg_set_operator_ex(None, 4, None, None, None, 0, gb.LOBPCG_F32, None, None,
                                      None, 0, None, gb.LOBPCG_F64, 0, 0) == gb.LOBPCG_ERR_ARG


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor: the attributes the binding inspects."""

    def __init__(self, dtype, contiguous=True):
        self.is_cuda = True
        self.dtype = dtype
        self._c = contiguous

    def is_contiguous(self):
        return self._c


def test_binding_marshals_and_refuses_misread_arrays():
    """Host arrays are converted to the ABI's int32 / float64; device tensors
    of another dtype, non-contiguous ones, and host / device mixes are refused
    before the library sees a pointer."""
    import numpy as np
    import torch
    H, D = gb.LOBPCG_MEM_HOST, gb.LOBPCG_MEM_DEVICE
    a = gb.Solver._arg(np.arange(5, dtype=np.int64), H, np.int32, "col")
    assert a.dtype == np.int32 and a.flags.c_contiguous
    b = gb.Solver._arg(torch.arange(6.0).reshape(2, 3).t(), H, np.float64, "X0")
    assert b.dtype == np.float64 and b.flags.c_contiguous and b.shape == (3, 2)
    assert gb.Solver._arg(None, D, np.float64, "x") is None
    ok = _FakeDeviceTensor("torch.int32")
    assert gb.Solver._arg(ok, D, np.int32, "col") is ok
    with pytest.raises(TypeError):
        gb.Solver._arg(_FakeDeviceTensor("torch.int64"), D, np.int32, "col")
    with pytest.raises(TypeError):
        gb.Solver._arg(_FakeDeviceTensor("torch.float32"), D, np.float64, "val")
    with pytest.raises(ValueError):
        gb.Solver._arg(_FakeDeviceTensor("torch.float64", contiguous=False), D, np.float64, "X0")
    with pytest.raises(ValueError):
        gb.Solver._arg(np.zeros(3), D, np.float64, "val")
    with pytest.raises(ValueError):
        gb.Solver._arg(_FakeDeviceTensor("torch.float64"), H, np.float64, "val")
    # shape checks run before any library call (no handle is needed for them)
    s = object.__new__(gb.Solver)
    s.h, s.n = None, 0
    with pytest.raises(ValueError):
        s.set_operator(np.array([0, 1, 2]), np.array([0, 1]), np.array([1.0]))
    with pytest.raises(ValueError):
        s.set_operator(np.array([0, 1, 2]), np.array([0, 1]), np.array([1.0, 1.0]),
                       b_diag=np.ones(3))
    with pytest.raises(ValueError):
        s.set_operator(np.array([0, 1, 2]), np.array([0, 1]), np.array([1.0, 1.0]),
                       b_csr=(np.array([0, 1]), np.array([0]), np.array([1.0])))


def test_binding_has_no_cpu_fallback():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1704_07458_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            txt = open(os.path.join(pkg, f)).read()
            assert "oracle" not in txt.replace("oracle-free", ""), f
            assert "scipy" not in txt, f
