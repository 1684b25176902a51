"""GPU test of vqmc_logprob_noalloc, the allocation-free log-prob entry point
for callers that cannot allocate device memory at call time (memory owned by
another framework's pool, fixed-budget serving paths, or code that must not
let cudaMalloc synchronise the device).  Its scratch is a static 64 MiB device
array shared by all calls.

Called through the C ABI (ctypes) and compared with vqmc_logprob on two calls
in a row with different spins, at the tolerance the log-prob parity tests use
(relative 1e-5), and at the edge of the scratch limit: the largest batch whose
scratch (the size formula stated in include/vqmc.h) fits in the 64 MiB is
accepted and matches, and one padding step more (64 samples) is refused.
This file is named to be collected last, and it passes both alone in a fresh
process and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2106_13308_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vq():
    from paper_2106_13308_gb300 import build
    build.build()
    from paper_2106_13308_gb300 import vqmc
    vqmc.load_library()
    return vqmc


def _model(vq, n, h, B, precision, seed):
    e = inputs.erdos_renyi(n, 0.02, seed)
    inst = inputs.to_csr(n, e, inputs.int_weights(len(e), 1, 10, seed + 1))
    m = vq.VQMC(n, h, B, inst, precision=precision, seed=seed)
    m.set_params(torch.from_numpy(inputs.lively_params(n, h, seed + 2)))
    return m


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_noalloc_logprob_matches_logprob_on_two_calls(vq, precision):
    n, h, B = 300, 200, 300
    m = _model(vq, n, h, B, precision, 41)
    lib = vq.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (b, seed) in enumerate([(B, 42), (B - 77, 43)]):
        S = torch.from_numpy(inputs.spins(b, n, seed)).cuda()
        ref = m.logprob(S)
        out = torch.full((b,), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.vqmc_logprob_noalloc(m.ctx, b, ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      stream)
        assert st == vq.VQMC_OK, lib.vqmc_last_error()
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy().astype(np.float64), out.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(o)), call
        assert np.max(np.abs(o - r) / np.abs(r)) <= 1e-5, call
    assert m.check() == 0


def test_noalloc_rejects_batches_beyond_the_static_scratch(vq):
    n, h, B = 20000, 64, 2048  # the spin operand alone is ~82 MB in BF16
    m = _model(vq, n, h, B, "bf16", 51)
    lib = vq.load_library()
    S = torch.ones((B, n), dtype=torch.int8, device="cuda")
    out = torch.empty(B, dtype=torch.float32, device="cuda")
    st = lib.vqmc_logprob_noalloc(m.ctx, B, ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == vq.VQMC_ERR_UNSUPPORTED
    assert b"fixed limit" in lib.vqmc_last_error()
    # a batch that fits still works on the same context
    b = 256
    st = lib.vqmc_logprob_noalloc(m.ctx, b, ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == vq.VQMC_OK, lib.vqmc_last_error()
    ref = m.logprob(S[:b])
    torch.cuda.synchronize()
    r, o = ref.cpu().numpy().astype(np.float64), out[:b].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(o - r) / np.abs(r)) <= 1e-5


def _scratch_bytes(B, n, h, es):
    """The scratch a call needs, as include/vqmc.h states it."""
    r = lambda x: (x + 255) // 256 * 256  # noqa: E731
    p64 = lambda x: (x + 63) // 64 * 64  # noqa: E731
    return r(B * p64(n) * es) + r(B * p64(h) * es) + r(((n + 127) // 128) * p64(B) * 4)


def test_noalloc_at_the_edge_of_the_scratch_limit(vq):
    limit = 64 << 20
    n, h = 1000, 512
    B = 1
    while _scratch_bytes(B + 1, n, h, 2) <= limit:
        B += 1
    assert _scratch_bytes(B, n, h, 2) <= limit < _scratch_bytes(B + 64, n, h, 2)
    m = _model(vq, n, h, B + 64, "bf16", 61)
    lib = vq.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    S = torch.from_numpy(inputs.spins(B + 64, n, 62)).cuda()
    out = torch.full((B + 64,), float("nan"), dtype=torch.float32, device="cuda")
    st = lib.vqmc_logprob_noalloc(m.ctx, B, ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(out.data_ptr()), stream)
    assert st == vq.VQMC_OK, lib.vqmc_last_error()
    ref = m.logprob(S[:B])
    torch.cuda.synchronize()
    r, o = ref.cpu().numpy().astype(np.float64), out[:B].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(o - r) / np.abs(r)) <= 1e-5
    st = lib.vqmc_logprob_noalloc(m.ctx, B + 64, ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  stream)
    assert st == vq.VQMC_ERR_UNSUPPORTED
    assert m.check() == 0
