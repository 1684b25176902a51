"""CPU checks of the C-ABI library: it builds, loads, exports every symbol
include/vqmc.h declares, and rejects bad arguments on the host before any
device work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_13308_gb300 import build
    build.build()
    from paper_2106_13308_gb300 import vqmc
    return vqmc.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "vqmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vqmc_[a-z_]+)\s*\(", src)))


def test_header_declares_binding_names():
    from paper_2106_13308_gb300 import vqmc
    assert _declared() == sorted(vqmc.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    from paper_2106_13308_gb300 import vqmc
    assert ctypes.sizeof(vqmc.Config) == 48
    assert ctypes.sizeof(vqmc.Instance) == 64
    assert ctypes.sizeof(vqmc.StepStats) == 48


def _cfg(vqmc, **kw):
    d = dict(n=10, h=8, max_batch=16, act=0, precision=1, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8,
             sampler=0, seed=1)
    d.update(kw)
    return vqmc.Config(**d)


def _inst(vqmc, n=10, row_ptr=None, col=None, w=None, kind=0):
    keep = []

    def p(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data_as(ctypes.c_void_p)

    if row_ptr is None:
        row_ptr = [0] * (n + 1)
        col, w = [], []
    inst = vqmc.Instance(kind, n, len(col), 0, p(row_ptr, np.int32), p(col, np.int32) if col else None,
                         p(w, np.int32) if w else None, None, None)
    return inst, keep


@pytest.mark.parametrize("bad", [dict(n=0), dict(h=0), dict(max_batch=0), dict(act=7), dict(precision=3)])
def test_create_rejects_bad_config(lib, bad):
    from paper_2106_13308_gb300 import vqmc
    cfg = _cfg(vqmc, **bad)
    inst, keep = _inst(vqmc, n=cfg.n if cfg.n > 0 else 10)
    h = ctypes.c_void_p()
    st = lib.vqmc_create(ctypes.byref(cfg), ctypes.byref(inst), ctypes.byref(h))
    assert st == vqmc.VQMC_ERR_INVALID_ARG and not h.value
    assert lib.vqmc_last_error()


def test_create_rejects_bad_instances(lib):
    from paper_2106_13308_gb300 import vqmc
    cfg = _cfg(vqmc)
    h = ctypes.c_void_p()
    # n mismatch
    inst, k1 = _inst(vqmc, n=11)
    assert lib.vqmc_create(ctypes.byref(cfg), ctypes.byref(inst), ctypes.byref(h)) == vqmc.VQMC_ERR_INVALID_ARG
    # lower-triangle entry
    rp = [0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1]
    inst, k2 = _inst(vqmc, row_ptr=rp, col=[1], w=[1])
    assert lib.vqmc_create(ctypes.byref(cfg), ctypes.byref(inst), ctypes.byref(h)) == vqmc.VQMC_ERR_INVALID_ARG
    assert b"upper triangle" in lib.vqmc_last_error()
    # bad kind
    inst, k3 = _inst(vqmc, kind=9)
    assert lib.vqmc_create(ctypes.byref(cfg), ctypes.byref(inst), ctypes.byref(h)) == vqmc.VQMC_ERR_INVALID_ARG


def test_create_rejects_bad_transverse_fields(lib):
    """alpha needs a float32 energy kind and finite alpha_i >= 0 (Sec. 2.4)."""
    from paper_2106_13308_gb300 import vqmc
    cfg = _cfg(vqmc)
    h = ctypes.c_void_p()
    for kind, a, msg in [(0, np.ones(10), b"float32"), (1, -np.ones(10), b">= 0"),
                         (1, np.full(10, np.nan), b">= 0")]:
        inst, keep = _inst(vqmc, kind=kind)
        al = np.ascontiguousarray(a, dtype=np.float32)
        inst.alpha = al.ctypes.data_as(ctypes.c_void_p)
        assert lib.vqmc_create(ctypes.byref(cfg), ctypes.byref(inst), ctypes.byref(h)) == vqmc.VQMC_ERR_INVALID_ARG
        assert msg in lib.vqmc_last_error() and not h.value


def test_null_context_calls_fail_cleanly(lib):
    from paper_2106_13308_gb300 import vqmc
    assert lib.vqmc_num_params(None) == 0
    assert lib.vqmc_sample(None, 1, None, 0, None, None, None) == vqmc.VQMC_ERR_INVALID_ARG
    assert lib.vqmc_step(None, 1, None, None) == vqmc.VQMC_ERR_INVALID_ARG
    assert lib.vqmc_check(None, None) == vqmc.VQMC_ERR_INVALID_ARG
    lib.vqmc_destroy(None)


def test_batch_rejects_bad_arguments(lib):
    from paper_2106_13308_gb300 import vqmc
    out = ctypes.c_void_p()
    cfg = (vqmc.Config * 1)(_cfg(vqmc))
    inst = (vqmc.Instance * 1)(vqmc.Instance(0, 10, 0, 0, None, None, None, None, None))
    assert lib.vqmc_batch_create(cfg, inst, 0, ctypes.byref(out)) == vqmc.VQMC_ERR_INVALID_ARG
    assert lib.vqmc_batch_create(None, inst, 1, ctypes.byref(out)) == vqmc.VQMC_ERR_INVALID_ARG
    assert lib.vqmc_batch_count(None) == 0
    assert not lib.vqmc_batch_member(None, 0)
    assert lib.vqmc_batch_step(None, None, None, None) == vqmc.VQMC_ERR_INVALID_ARG


def test_noalloc_source_calls_no_allocating_routine():
    """The allocation-free entry point's translation unit calls no
    cudaMalloc*/cudaFree* routine (comments aside) and takes its scratch from
    the file-scope __device__ array, whose address it looks up with
    cudaGetSymbolAddress."""
    import re
    src = open(os.path.join(ROOT, "paper_2106_13308_gb300", "csrc", "noalloc.cu")).read()
    code = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    code = re.sub(r"//[^\n]*", "", code)
    assert not re.search(r"\bcuda(Malloc|Free)\w*\s*\(", code)
    assert not re.search(r"\bcuMem(Alloc|Free)\w*\s*\(", code)
    assert re.search(r"static\s+__device__\s+__align__\(256\)", code)
    assert "cudaGetSymbolAddress" in code
