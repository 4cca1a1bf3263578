"""Host-only checks of the C ABI: the built library loads, exports every entry point that
include/swimmer.h declares, and the Python binding's ctypes structs match the C layout.
No compute call is made (this runs without a GPU)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swimmer.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|size_t|char|void)\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_12007_gb300 import _lib

    if not os.path.exists(_lib.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("library not built and no nvcc")
        from paper_1910_12007_gb300.build import build

        build()
    return _lib


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["swimmer_init", "swimmer_destroy", "forward_batch", "loglik_batch", "tmcmc_stage"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.lib()
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert missing == []
    bound = {name for name, _, _ in lib.SIGNATURES}
    assert bound == set(_declared_functions())


def test_ctypes_structs_match_c_layout(tmp_path, lib):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "swimmer.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(swimmer_config), offsetof(swimmer_config, steps),
         offsetof(swimmer_config, precision), sizeof(tmcmc_state));
  printf("%zu %zu %zu\\n", offsetof(tmcmc_state, sigma), offsetof(tmcmc_state, q), offsetof(tmcmc_state, surr_loglik));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    c = [int(v) for v in out]
    C, S = lib.SwimmerConfigC, lib.TmcmcStateC
    assert c[0] == ctypes.sizeof(C)
    assert c[1] == C.steps.offset and c[2] == C.precision.offset
    assert c[3] == ctypes.sizeof(S)
    assert c[4] == S.sigma.offset and c[5] == S.q.offset and c[6] == S.surr_loglik.offset


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_1910_12007_gb300 import _lib

    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/libswimmer.so")
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.lib()


def test_seeded_inputs_are_deterministic():
    import numpy as np

    import synthetic

    a = synthetic.uniforms(7, synthetic.RESAMPLE, 3, 1000)
    b = synthetic.uniforms(7, synthetic.RESAMPLE, 3, 1000)
    assert np.array_equal(a, b)
    assert 0.0 <= a.min() and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.05
    z = synthetic.normals(7, synthetic.PROPOSAL, 0, 20000)
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1) < 0.03
    assert not np.array_equal(a, synthetic.uniforms(7, synthetic.RESAMPLE, 4, 1000))


def test_noalloc_binding_rejects_host_buffers_before_any_call(monkeypatch):
    """The allocation-free entry point's binding checks every buffer on the host: tensors that
    are not contiguous FP64 device memory are refused before the library is called."""
    torch = pytest.importorskip("torch")
    from paper_1910_12007_gb300 import _lib, api

    def no_library():
        raise AssertionError("the library must not be called")

    monkeypatch.setattr(_lib, "lib", no_library)
    monkeypatch.setattr(api, "lib", no_library)
    r = torch.zeros(8, dtype=torch.float64)
    with pytest.raises(TypeError):
        api.swimmer_kernel_eval_noalloc(1.0, 0.02, 1.0, r)
    with pytest.raises(TypeError):
        api.swimmer_kernel_eval_noalloc(1.0, 0.02, 1.0, r.float())
