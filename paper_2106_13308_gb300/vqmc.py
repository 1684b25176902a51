"""Python binding of libvqmc (include/vqmc.h): argument marshalling only.

Every compute step runs in the CUDA library; this module converts torch
tensors to raw pointers and the current torch stream to a cudaStream_t.  The
functions carry the C names (``vqmc_create``, ``vqmc_sample``, ...); ``VQMC``
is a small convenience class over them and ``LogProb`` is the
``torch.autograd.Function`` whose backward is the library's hand-written
adjoint (``vqmc_logprob_backward``).

There is no CPU fallback: importing the library fails loudly when
``lib/libvqmc.so`` has not been built (``paper_2106_13308_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libvqmc.so")

VQMC_OK, VQMC_ERR_INVALID_ARG, VQMC_ERR_CUDA, VQMC_ERR_OOM = 0, 1, 2, 3
VQMC_ERR_NONFINITE, VQMC_ERR_TIMEOUT, VQMC_ERR_UNSUPPORTED = 4, 5, 6
ACT = {"relu": 0, "sigmoid": 1}
PREC = {"fp32": 0, "bf16": 1}
SAMPLER = {"auto": 0, "cuda_core": 1, "tensor_core": 2, "cuda_core_wide": 3}
SAMPLER_NAME = {v: k for k, v in SAMPLER.items()}
HAM = {"sparse_i32": 0, "sparse_f32": 1, "dense": 2}
DEVERR_TIMEOUT, DEVERR_NONFINITE = 1, 2

# Names declared in include/vqmc.h (the CPU test checks the library exports them).
EXPORTS = [
    "vqmc_create", "vqmc_destroy", "vqmc_num_params", "vqmc_set_params", "vqmc_get_params",
    "vqmc_params_device", "vqmc_params_updated", "vqmc_uniforms", "vqmc_sample", "vqmc_local_energy",
    "vqmc_logprob", "vqmc_logprob_backward", "vqmc_energy_stats", "vqmc_grad", "vqmc_adam", "vqmc_step",
    "vqmc_last_batch", "vqmc_iteration", "vqmc_check", "vqmc_save", "vqmc_load", "vqmc_timing_enable",
    "vqmc_timing_read", "vqmc_logprob_noalloc", "vqmc_last_error", "vqmc_batch_create", "vqmc_batch_destroy",
    "vqmc_batch_count", "vqmc_batch_member", "vqmc_batch_step", "vqmc_sr_gram", "vqmc_sr_direction",
    "vqmc_sr_step", "vqmc_graph_capture", "vqmc_graph_launch", "vqmc_batch_graph_capture",
    "vqmc_batch_graph_launch", "vqmc_batch_autotune", "vqmc_set_sample_offset", "vqmc_shard_sums",
    "vqmc_shard_apply", "vqmc_batch_schedule",
]
OPT = {"adam": 0, "sr": 1}
PARTS = ["sample", "energy", "stats", "grad", "adam"]


class VQMCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"vqmc status {status}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("h", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("act", ctypes.c_int32), ("precision", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("sampler", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class Instance(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("field", ctypes.c_void_p), ("J", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p)]


class StepStats(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("var", ctypes.c_double), ("min", ctypes.c_double),
                ("max", ctypes.c_double), ("iteration", ctypes.c_uint64), ("error_flags", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libvqmc.so and declares the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2106_13308_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    st = ctypes.c_int
    sig = {
        "vqmc_create": (st, [ctypes.POINTER(Config), ctypes.POINTER(Instance), ctypes.POINTER(P)]),
        "vqmc_destroy": (None, [P]),
        "vqmc_num_params": (I64, [P]),
        "vqmc_set_params": (st, [P, P, ctypes.c_int, P]),
        "vqmc_get_params": (st, [P, P, ctypes.c_int, P]),
        "vqmc_params_device": (P, [P]),
        "vqmc_params_updated": (st, [P, P]),
        "vqmc_uniforms": (st, [P, I32, U64, P, P]),
        "vqmc_sample": (st, [P, I32, P, U64, P, P, P]),
        "vqmc_local_energy": (st, [P, I32, P, P, P]),
        "vqmc_logprob": (st, [P, I32, P, P, P]),
        "vqmc_logprob_backward": (st, [P, I32, P, P, P, P]),
        "vqmc_energy_stats": (st, [P, I32, P, P, P, P]),
        "vqmc_grad": (st, [P, I32, P, P, P, P, P]),
        "vqmc_adam": (st, [P, P, P]),
        "vqmc_step": (st, [P, I32, P, ctypes.POINTER(StepStats)]),
        "vqmc_last_batch": (st, [P, ctypes.POINTER(P), ctypes.POINTER(P)]),
        "vqmc_iteration": (U64, [P]),
        "vqmc_check": (st, [P, ctypes.POINTER(ctypes.c_uint32)]),
        "vqmc_save": (st, [P, ctypes.c_char_p]),
        "vqmc_load": (st, [P, ctypes.c_char_p]),
        "vqmc_timing_enable": (st, [P, ctypes.c_int]),
        "vqmc_timing_read": (st, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "vqmc_logprob_noalloc": (st, [P, I32, P, P, P]),
        "vqmc_set_sample_offset": (st, [P, ctypes.c_uint32]),
        "vqmc_shard_sums": (st, [P, I32, P, P, ctypes.c_double, P, P, P]),
        "vqmc_shard_apply": (st, [P, P, P, ctypes.c_double, P, P, P]),
        "vqmc_last_error": (ctypes.c_char_p, []),
        "vqmc_batch_create": (st, [ctypes.POINTER(Config), ctypes.POINTER(Instance), I32, ctypes.POINTER(P)]),
        "vqmc_batch_destroy": (None, [P]),
        "vqmc_batch_count": (I32, [P]),
        "vqmc_batch_member": (P, [P, I32]),
        "vqmc_batch_step": (st, [P, ctypes.POINTER(I32), P, ctypes.POINTER(StepStats)]),
        "vqmc_sr_gram": (st, [P, I32, P, P, P]),
        "vqmc_sr_direction": (st, [P, I32, P, P, ctypes.c_float, P, P, P]),
        "vqmc_sr_step": (st, [P, I32, ctypes.c_float, ctypes.c_float, P, ctypes.POINTER(StepStats)]),
        "vqmc_graph_capture": (st, [P, I32, I32, I32, ctypes.c_float, ctypes.c_float, P]),
        "vqmc_graph_launch": (st, [P, P, ctypes.POINTER(StepStats)]),
        "vqmc_batch_graph_capture": (st, [P, ctypes.POINTER(I32), I32, P]),
        "vqmc_batch_graph_launch": (st, [P, P, ctypes.POINTER(StepStats)]),
        "vqmc_batch_autotune": (st, [P, ctypes.POINTER(I32), P, ctypes.POINTER(I32),
                                     ctypes.POINTER(ctypes.c_double)]),
        "vqmc_batch_schedule": (st, [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32),
                                     ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != VQMC_OK:
        raise VQMCError(status, _lib.vqmc_last_error().decode())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- C names

def vqmc_create(cfg: Config, inst: Instance) -> ctypes.c_void_p:
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.vqmc_create(ctypes.byref(cfg), ctypes.byref(inst), ctypes.byref(h)))
    return h


def vqmc_destroy(ctx):
    load_library().vqmc_destroy(ctx)


def vqmc_num_params(ctx) -> int:
    return int(load_library().vqmc_num_params(ctx))


def vqmc_set_params(ctx, theta: torch.Tensor, stream=None):
    if theta.is_cuda:
        _check(load_library().vqmc_set_params(ctx, _ptr(theta), 1, _stream(stream)))
    else:
        t = np.ascontiguousarray(theta.detach().numpy() if isinstance(theta, torch.Tensor) else theta,
                                 dtype=np.float32)
        _check(load_library().vqmc_set_params(ctx, t.ctypes.data_as(ctypes.c_void_p), 0, _stream(stream)))


def vqmc_get_params(ctx, out: torch.Tensor, stream=None):
    if out.is_cuda:
        _check(load_library().vqmc_get_params(ctx, _ptr(out), 1, _stream(stream)))
    else:
        assert out.dtype == torch.float32 and out.is_contiguous()
        _check(load_library().vqmc_get_params(ctx, ctypes.c_void_p(out.data_ptr()), 0, _stream(stream)))


def vqmc_params_updated(ctx, stream=None):
    _check(load_library().vqmc_params_updated(ctx, _stream(stream)))


def vqmc_uniforms(ctx, B: int, iteration: int, u: torch.Tensor, stream=None):
    _check(load_library().vqmc_uniforms(ctx, B, iteration, _ptr(u), _stream(stream)))


def vqmc_sample(ctx, B: int, u, iteration: int, s: torch.Tensor, logp=None, stream=None):
    _check(load_library().vqmc_sample(ctx, B, _ptr(u), iteration, _ptr(s), _ptr(logp), _stream(stream)))


def vqmc_local_energy(ctx, B: int, s: torch.Tensor, e: torch.Tensor, stream=None):
    _check(load_library().vqmc_local_energy(ctx, B, _ptr(s), _ptr(e), _stream(stream)))


def vqmc_logprob(ctx, B: int, s: torch.Tensor, logp: torch.Tensor, stream=None):
    _check(load_library().vqmc_logprob(ctx, B, _ptr(s), _ptr(logp), _stream(stream)))


def vqmc_logprob_noalloc(ctx, B: int, s: torch.Tensor, logp: torch.Tensor, stream=None):
    _check(load_library().vqmc_logprob_noalloc(ctx, B, _ptr(s), _ptr(logp), _stream(stream)))


def vqmc_logprob_backward(ctx, B: int, s, gout, grad, stream=None):
    _check(load_library().vqmc_logprob_backward(ctx, B, _ptr(s), _ptr(gout), _ptr(grad), _stream(stream)))


def vqmc_energy_stats(ctx, B: int, e, stats, coef=None, stream=None):
    _check(load_library().vqmc_energy_stats(ctx, B, _ptr(e), _ptr(stats), _ptr(coef), _stream(stream)))


def vqmc_grad(ctx, B: int, s, e, grad, stats=None, stream=None):
    _check(load_library().vqmc_grad(ctx, B, _ptr(s), _ptr(e), _ptr(grad), _ptr(stats), _stream(stream)))


def vqmc_adam(ctx, grad, stream=None):
    _check(load_library().vqmc_adam(ctx, _ptr(grad), _stream(stream)))


def vqmc_step(ctx, B: int, out: StepStats | None = None, stream=None):
    _check(load_library().vqmc_step(ctx, B, _stream(stream), ctypes.byref(out) if out is not None else None))


def vqmc_set_sample_offset(ctx, b0: int):
    _check(load_library().vqmc_set_sample_offset(ctx, int(b0)))


def vqmc_shard_sums(ctx, B: int, s, e, shift: float, sums, scalars, stream=None):
    _check(load_library().vqmc_shard_sums(ctx, B, _ptr(s), _ptr(e), float(shift), _ptr(sums), _ptr(scalars),
                                          _stream(stream)))


def vqmc_shard_apply(ctx, sums, scalars, shift: float, grad=None, stats=None, stream=None):
    _check(load_library().vqmc_shard_apply(ctx, _ptr(sums), _ptr(scalars), float(shift), _ptr(grad), _ptr(stats),
                                           _stream(stream)))


def vqmc_sr_gram(ctx, B: int, s, gram, stream=None):
    _check(load_library().vqmc_sr_gram(ctx, B, _ptr(s), _ptr(gram), _stream(stream)))


def vqmc_sr_direction(ctx, B: int, s, e, lam: float, delta, stats=None, stream=None):
    _check(load_library().vqmc_sr_direction(ctx, B, _ptr(s), _ptr(e), float(lam), _ptr(delta), _ptr(stats),
                                            _stream(stream)))


def vqmc_sr_step(ctx, B: int, lr: float, lam: float, out: StepStats | None = None, stream=None):
    _check(load_library().vqmc_sr_step(ctx, B, float(lr), float(lam), _stream(stream),
                                       ctypes.byref(out) if out is not None else None))


def vqmc_graph_capture(ctx, B: int, steps: int, optimizer: str = "adam", sr_lr: float = 0.1,
                       sr_lambda: float = 1e-3, stream=None):
    _check(load_library().vqmc_graph_capture(ctx, B, steps, OPT[optimizer], float(sr_lr), float(sr_lambda),
                                             _stream(stream)))


def vqmc_graph_launch(ctx, out: StepStats | None = None, stream=None):
    _check(load_library().vqmc_graph_launch(ctx, _stream(stream), ctypes.byref(out) if out is not None else None))


def vqmc_check(ctx) -> int:
    f = ctypes.c_uint32()
    st = load_library().vqmc_check(ctx, ctypes.byref(f))
    if st not in (VQMC_OK, VQMC_ERR_TIMEOUT, VQMC_ERR_NONFINITE):
        _check(st)
    return int(f.value)


def vqmc_timing_enable(ctx, enable: bool):
    _check(load_library().vqmc_timing_enable(ctx, 1 if enable else 0))


def vqmc_timing_read(ctx):
    """({part: ms summed over recorded steps}, steps, kernel launches)."""
    ms = (ctypes.c_double * len(PARTS))()
    steps, launches = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().vqmc_timing_read(ctx, ms, ctypes.byref(steps), ctypes.byref(launches)))
    return dict(zip(PARTS, list(ms))), int(steps.value), int(launches.value)


def vqmc_save(ctx, path: str):
    _check(load_library().vqmc_save(ctx, path.encode()))


def vqmc_load(ctx, path: str):
    _check(load_library().vqmc_load(ctx, path.encode()))


# --------------------------------------------------------------- wrapper

class _DeviceArray:
    """Exposes a raw device pointer through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int, typestr: str = "<f4"):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _describe(n, h, max_batch, instance, act, precision, lr, beta1, beta2, eps, seed, sampler, keep):
    """The C structures of one problem; keep receives the host arrays they point into."""
    cfg = Config(int(n), int(h), int(max_batch), ACT[act], PREC[precision], lr, beta1, beta2, eps, SAMPLER[sampler],
                 int(seed) & (2 ** 64 - 1))

    def arr(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data_as(ctypes.c_void_p)

    kind = instance["kind"]
    alpha = arr(instance.get("alpha"), np.float32)
    if kind == "dense":
        inst = Instance(HAM["dense"], int(n), 0, 0, None, None, None, arr(instance.get("field"), np.float32),
                        arr(instance["J"], np.float32), alpha)
    else:
        wdt = np.int32 if kind == "sparse_i32" else np.float32
        inst = Instance(HAM[kind], int(n), int(len(instance["col"])), 0, arr(instance["row_ptr"], np.int32),
                        arr(instance["col"], np.int32), arr(instance["w"], wdt), arr(instance.get("field"), wdt),
                        None, alpha)
    return cfg, inst


class VQMC:
    """One GPU context: model, instance, optimiser and workspaces.

    ``instance`` is a dict as produced by ``paper_2106_13308_gb300.inputs``
    (kind sparse_i32 / sparse_f32 with row_ptr, col, w[, field]; or dense with
    J[, field]; float kinds may add the transverse field ``alpha``)."""

    def __init__(self, n, h, max_batch, instance, act="relu", precision="bf16", lr=1e-2, beta1=0.9,
                 beta2=0.999, eps=1e-8, seed=0, sampler="auto", _ctx=None):
        load_library()
        self.n, self.h, self.max_batch = int(n), int(h), int(max_batch)
        self.act, self.precision = act, precision
        self.kind = instance["kind"]
        self._owned = _ctx is None
        if _ctx is None:
            keep = []
            cfg, inst = _describe(n, h, max_batch, instance, act, precision, lr, beta1, beta2, eps, seed, sampler,
                                  keep)
            self.ctx = vqmc_create(cfg, inst)
        else:  # a member of a VQMCBatch, owned by the batch
            self.ctx = _ctx
        self.d = vqmc_num_params(self.ctx)
        self.e_dtype = torch.int32 if self.kind == "sparse_i32" else torch.float32

    def close(self):
        if getattr(self, "ctx", None):
            if self._owned:
                vqmc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # parameters
    def set_params(self, theta):
        vqmc_set_params(self.ctx, torch.as_tensor(theta))

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.d, dtype=torch.float32)
        vqmc_get_params(self.ctx, out)
        return out

    def params_view(self) -> torch.Tensor:
        """Zero-copy CUDA view of the master theta (valid while the context lives)."""
        ptr = load_library().vqmc_params_device(self.ctx)
        return torch.as_tensor(_DeviceArray(ptr, self.d), device="cuda")

    # the path
    def uniforms(self, B, iteration):
        u = torch.empty((B, self.n), dtype=torch.float32, device="cuda")
        vqmc_uniforms(self.ctx, B, iteration, u)
        return u

    def sample(self, B, u=None, iteration=0):
        s = torch.empty((B, self.n), dtype=torch.int8, device="cuda")
        lp = torch.empty(B, dtype=torch.float32, device="cuda")
        vqmc_sample(self.ctx, B, u, iteration, s, lp)
        return s, lp

    def local_energy(self, s):
        B = s.shape[0]
        e = torch.empty(B, dtype=self.e_dtype, device="cuda")
        vqmc_local_energy(self.ctx, B, s, e)
        return e

    def logprob(self, s):
        B = s.shape[0]
        lp = torch.empty(B, dtype=torch.float32, device="cuda")
        vqmc_logprob(self.ctx, B, s, lp)
        return lp

    def logprob_backward(self, s, gout):
        g = torch.empty(self.d, dtype=torch.float32, device="cuda")
        vqmc_logprob_backward(self.ctx, s.shape[0], s, gout.contiguous().float(), g)
        return g

    def energy_stats(self, e):
        stats = torch.empty(4, dtype=torch.float64, device="cuda")
        coef = torch.empty(e.shape[0], dtype=torch.float32, device="cuda")
        vqmc_energy_stats(self.ctx, e.shape[0], e, stats, coef)
        return stats, coef

    def grad(self, s, e):
        g = torch.empty(self.d, dtype=torch.float32, device="cuda")
        stats = torch.empty(4, dtype=torch.float64, device="cuda")
        vqmc_grad(self.ctx, s.shape[0], s, e, g, stats)
        return g, stats

    def adam(self, g):
        vqmc_adam(self.ctx, g)

    def step(self, B, out: StepStats | None = None):
        vqmc_step(self.ctx, B, out)
        return out

    # sampling parallelism: one shard of a batch spread over several GPUs
    def set_sample_offset(self, b0):
        vqmc_set_sample_offset(self.ctx, b0)

    def shard_sums(self, B, shift=0.0, s=None, e=None):
        """(sums float32 [2d], scalars float64 [3]) of this shard; with s = None
        the shard's samples are drawn (internal Philox, sample offset)."""
        sums = torch.empty(2 * self.d, dtype=torch.float32, device="cuda")
        scal = torch.empty(3, dtype=torch.float64, device="cuda")
        vqmc_shard_sums(self.ctx, B, s, e, shift, sums, scal)
        return sums, scal

    def shard_apply(self, sums, scalars, shift=0.0):
        """Gradient from the all-ranks sums, one Adam step; returns (grad, stats)."""
        g = torch.empty(self.d, dtype=torch.float32, device="cuda")
        stats = torch.empty(2, dtype=torch.float64, device="cuda")
        vqmc_shard_apply(self.ctx, sums.contiguous(), scalars.contiguous(), shift, g, stats)
        return g, stats

    # stochastic reconfiguration (FP32 contexts)
    def sr_gram(self, s):
        B = s.shape[0]
        G = torch.empty((B, B), dtype=torch.float32, device="cuda")
        vqmc_sr_gram(self.ctx, B, s, G)
        return G

    def sr_direction(self, s, e, lam=1e-3):
        delta = torch.empty(self.d, dtype=torch.float32, device="cuda")
        stats = torch.empty(4, dtype=torch.float64, device="cuda")
        vqmc_sr_direction(self.ctx, s.shape[0], s, e, lam, delta, stats)
        return delta, stats

    def sr_step(self, B, lr=0.1, lam=1e-3, out: StepStats | None = None):
        vqmc_sr_step(self.ctx, B, lr, lam, out)
        return out

    # captured iterations (one CUDA graph launch each)
    def graph_capture(self, B, steps=1, optimizer="adam", sr_lr=0.1, sr_lambda=1e-3, stream=None):
        vqmc_graph_capture(self.ctx, B, steps, optimizer, sr_lr, sr_lambda, stream)

    def graph_launch(self, out: StepStats | None = None, stream=None):
        vqmc_graph_launch(self.ctx, out, stream)
        return out

    def last_batch(self, B):
        ps, pe = ctypes.c_void_p(), ctypes.c_void_p()
        _check(load_library().vqmc_last_batch(self.ctx, ctypes.byref(ps), ctypes.byref(pe)))
        s = torch.as_tensor(_DeviceArray(ps.value, B * self.n, "|i1"), device="cuda").view(B, self.n)
        e = torch.as_tensor(_DeviceArray(pe.value, B, "<i4" if self.e_dtype == torch.int32 else "<f4"),
                            device="cuda")
        return s, e

    @property
    def iteration(self) -> int:
        return int(load_library().vqmc_iteration(self.ctx))

    def check(self) -> int:
        return vqmc_check(self.ctx)

    def timing_enable(self, enable=True):
        vqmc_timing_enable(self.ctx, enable)

    def timing_read(self):
        return vqmc_timing_read(self.ctx)

    def save(self, path):
        vqmc_save(self.ctx, path)

    def load(self, path):
        vqmc_load(self.ctx, path)


class LogProb(torch.autograd.Function):
    """log pi_theta(s) with the library's adjoint as backward.

    ``theta`` must be ``model.params_view()`` (the context's own parameters):
    forward reads the weight copies the context keeps in sync with it, and
    backward returns sum_b grad_out[b] * grad_theta log pi(s_b), recomputing
    the hidden activations instead of saving them."""

    @staticmethod
    def forward(ctx, theta, spins, model: VQMC):
        ctx.model = model
        ctx.save_for_backward(spins)
        return model.logprob(spins)

    @staticmethod
    def backward(ctx, grad_out):
        (spins,) = ctx.saved_tensors
        g = ctx.model.logprob_backward(spins, grad_out)
        return g, None, None


class VQMCBatch:
    """Independent problems stepped together (vqmc_batch_*).  ``problems`` is
    a list of dicts with the keyword arguments of VQMC (n, h, max_batch,
    instance, and optionally act, precision, lr, beta1, beta2, eps, seed,
    sampler); ``members[i]`` is a VQMC view of problem i, owned by the batch."""

    def __init__(self, problems):
        lib = load_library()
        keep, cfgs, insts = [], [], []
        defaults = dict(act="relu", precision="bf16", lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, seed=0,
                        sampler="auto")
        self.problems = [dict(defaults, **p) for p in problems]
        for p in self.problems:
            cfg, inst = _describe(p["n"], p["h"], p["max_batch"], p["instance"], p["act"], p["precision"], p["lr"],
                                  p["beta1"], p["beta2"], p["eps"], p["seed"], p["sampler"], keep)
            cfgs.append(cfg)
            insts.append(inst)
        count = len(cfgs)
        ca, ia = (Config * count)(*cfgs), (Instance * count)(*insts)
        h = ctypes.c_void_p()
        _check(lib.vqmc_batch_create(ca, ia, count, ctypes.byref(h)))
        self.handle = h
        self.members = [VQMC(p["n"], p["h"], p["max_batch"], p["instance"], act=p["act"], precision=p["precision"],
                             _ctx=ctypes.c_void_p(lib.vqmc_batch_member(h, i))) for i, p in enumerate(self.problems)]

    def __len__(self):
        return len(self.members)

    def step(self, B, out=None, stream=None):
        """One iteration of every member, member i with B[i] samples (or B for all)."""
        count = len(self.members)
        bs = list(B) if hasattr(B, "__len__") else [int(B)] * count
        arr = (ctypes.c_int32 * count)(*bs)
        outp = None
        if out is not None:
            assert len(out) == count
            outp = out
        _check(_lib.vqmc_batch_step(self.handle, arr, _stream(stream), outp))

    def _bs(self, B):
        count = len(self.members)
        bs = list(B) if hasattr(B, "__len__") else [int(B)] * count
        return (ctypes.c_int32 * count)(*bs)

    def graph_capture(self, B, steps=1, stream=None):
        """Captures `steps` batched iterations as one CUDA graph."""
        _check(_lib.vqmc_batch_graph_capture(self.handle, self._bs(B), steps, _stream(stream)))

    def graph_launch(self, out=None, stream=None):
        _check(_lib.vqmc_batch_graph_launch(self.handle, _stream(stream), out))

    def autotune(self, B, stream=None):
        """Chooses each member's sampler layout (timed alone) and the schedule
        (streams, member assignment) by timing graph replays; returns
        (streams, ms per batched iteration)."""
        s, ms = ctypes.c_int32(), ctypes.c_double()
        _check(_lib.vqmc_batch_autotune(self.handle, self._bs(B), _stream(stream), ctypes.byref(s), ctypes.byref(ms)))
        return int(s.value), float(ms.value)

    def schedule(self):
        """(streams in use, [stream of each member], [sampler of each member],
        [ms of one iteration of each member alone, from the last autotune])."""
        k = len(self)
        used = ctypes.c_int32()
        st = (ctypes.c_int32 * k)()
        sm = (ctypes.c_int32 * k)()
        ms = (ctypes.c_double * k)()
        _check(_lib.vqmc_batch_schedule(self.handle, ctypes.byref(used), st, sm, ms))
        return int(used.value), list(st), [SAMPLER_NAME[x] for x in sm], list(ms)

    def close(self):
        if getattr(self, "handle", None):
            for m in self.members:
                m.ctx = None
            _lib.vqmc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
