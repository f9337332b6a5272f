"""Thin ctypes binding of libhmpcg (include/hmpcg.h).

Argument marshalling only: every step of the method runs in the CUDA kernels of
libhmpcg.so.  Torch supplies device memory and streams.  Importing this module
fails loudly when the shared library has not been built; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhmpcg.so")

OK, NOT_CONVERGED = 0, 1
E_INVALID, E_SHAPE, E_CUDA, E_BREAKDOWN, E_NAN, E_TIMEOUT, E_NOMEM = -1, -2, -3, -4, -5, -6, -7
F32, BF16, FP8E4M3 = 0, 1, 2
PRE_NONE, PRE_JACOBI, PRE_SVDH, PRE_LEARNED = 0, 1, 2, 3
BC_DIRICHLET, BC_NEUMANN = 0, 1
FACE_INV_RHO, FACE_RHO = 0, 1


class HmpcgError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


class Config(C.Structure):
    _fields_ = [("max_n", C.c_int64), ("max_batch", C.c_int32), ("max_nrhs", C.c_int32),
                ("leaf", C.c_int32), ("rank", C.c_int32), ("d_model", C.c_int32),
                ("n_layers", C.c_int32), ("n_heads", C.c_int32), ("d_mlp", C.c_int32)]


class SystemStruct(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("dims", C.c_int32 * 3), ("n", C.c_int64),
                ("diag", C.c_void_p), ("wplus", C.c_void_p * 3),
                ("diag32", C.c_void_p), ("wplus32", C.c_void_p * 3),
                ("rho", C.c_void_p), ("perm", C.c_void_p)]


class Factors(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dtype", C.c_int32), ("leaf", C.c_int32),
                ("rank", C.c_int32), ("n", C.c_int64), ("packed", C.c_void_p),
                ("scales", C.c_void_p)]


class SolveOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_iter", C.c_int32), ("recompute_every", C.c_int32),
                ("fallback", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("rel_res_true", C.c_double),
                ("ms_solve", C.c_float), ("fallback", C.c_int32)]


EXPORTS = {
    "hmpcg_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Config), C.c_void_p, C.c_int64, C.c_void_p]),
    "hmpcg_destroy": (C.c_int, [C.c_void_p]),
    "hmpcg_weight_count": (C.c_int64, [C.POINTER(Config)]),
    "hmpcg_status_string": (C.c_char_p, [C.c_int]),
    "hmpcg_system_bytes": (C.c_int64, [C.c_int32, C.POINTER(C.c_int32)]),
    "hmpcg_system_layout": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), C.c_void_p, C.POINTER(SystemStruct)]),
    "hmpcg_assemble": (C.c_int, [C.c_void_p, C.POINTER(SystemStruct), C.c_int32, C.c_int32, C.c_void_p]),
    "hmpcg_spmv": (C.c_int, [C.POINTER(SystemStruct), C.c_void_p, C.c_void_p, C.c_void_p]),
    "hmpcg_apply": (C.c_int, [C.c_void_p, C.POINTER(Factors), C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "hmpcg_solve": (C.c_int, [C.c_void_p, C.POINTER(SystemStruct), C.POINTER(Factors), C.c_void_p, C.c_void_p,
                              C.POINTER(SolveOpts), C.POINTER(SolveInfo), C.c_void_p]),
    "hmpcg_infer_factors": (C.c_int, [C.c_void_p, C.POINTER(SystemStruct), C.c_int32, C.c_void_p, C.c_int32,
                                      C.c_void_p, C.c_void_p]),
    "hmpcg_packed_width": (C.c_int64, [C.c_int64, C.c_int32, C.c_int32, C.c_int32]),
    "hmpcg_set_infer_mode": (C.c_int, [C.c_void_p, C.c_int32]),
    "hmpcg_set_train_probes": (C.c_int, [C.c_void_p, C.c_int32, C.c_float, C.c_int32]),
    "hmpcg_set_train_loss": (C.c_int, [C.c_void_p, C.c_int32]),
    "hmpcg_set_highways": (C.c_int, [C.c_void_p, C.c_int32]),
    "hmpcg_train_step": (C.c_int, [C.c_void_p, C.POINTER(SystemStruct), C.c_int32, C.c_int32, C.c_float,
                                   C.c_uint64, C.POINTER(C.c_float), C.c_void_p]),
    "hmpcg_get_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "hmpcg_get_grads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "hmpcg_apply_noalloc": (C.c_int, [C.POINTER(Factors), C.c_void_p, C.c_void_p, C.c_void_p]),
    "hmpcg_selftest_wait": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "hmpcg_gemm_bf16": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                  C.c_void_p, C.c_int32, C.c_void_p]),
    "hmpcg_solve_batch": (C.c_int, [C.c_void_p, C.POINTER(SystemStruct), C.POINTER(Factors),
                                    C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int32,
                                    C.POINTER(SolveOpts), C.POINTER(SolveInfo), C.c_void_p]),
    "hmpcg_autotune_batch": (C.c_int, [C.c_void_p, C.POINTER(SystemStruct), C.POINTER(Factors),
                                       C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int32,
                                       C.POINTER(SolveOpts), C.POINTER(C.c_int32), C.c_void_p]),
}


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libhmpcg.so is not built ({path}); run __graft_entry__.build() "
                          "or python -m paper_2605_13343_gb300.build")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def status_string(code):
    return lib().hmpcg_status_string(int(code)).decode()


def _check(code, what, allow=(OK,)):
    if code not in allow:
        raise HmpcgError(code, what)
    return code


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return C.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ systems
class System:
    """One assembled system: a caller-owned device buffer carved by hmpcg_system_layout."""

    def __init__(self, dims, device="cuda"):
        self.dims = tuple(int(d) for d in dims)
        nd = len(self.dims)
        arr = (C.c_int32 * 3)(*(list(self.dims) + [1] * (3 - nd)))
        nbytes = lib().hmpcg_system_bytes(nd, arr)
        if nbytes <= 0:
            raise HmpcgError(E_SHAPE, f"grid {dims}")
        self.buf = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device)
        base = (self.buf.data_ptr() + 255) // 256 * 256
        self.struct = SystemStruct()
        _check(lib().hmpcg_system_layout(nd, arr, C.c_void_p(base), C.byref(self.struct)), "system_layout")
        self.n = int(self.struct.n)

    def _view(self, ptr, dtype, count=None):
        count = self.n if count is None else count
        off = ptr - self.buf.data_ptr()
        esz = torch.empty(0, dtype=dtype).element_size()
        return self.buf[off:off + count * esz].view(dtype)

    @property
    def diag(self):
        return self._view(self.struct.diag, torch.float64)

    def wplus(self, a):
        return self._view(self.struct.wplus[a], torch.float64)

    @property
    def diag32(self):
        return self._view(self.struct.diag32, torch.float32)

    def wplus32(self, a):
        return self._view(self.struct.wplus32[a], torch.float32)

    @property
    def rho(self):
        return self._view(self.struct.rho, torch.float64)

    @property
    def perm(self):
        return self._view(self.struct.perm, torch.int32)


def systems_array(systems):
    arr = (SystemStruct * len(systems))()
    for i, s in enumerate(systems):
        arr[i] = s.struct
    return arr


def assemble(rho_lex, system, bc=BC_DIRICHLET, face=FACE_INV_RHO, stream=None):
    """hmpcg_assemble: density (device FP64, lexicographic) -> Morton-order operator."""
    assert rho_lex.dtype == torch.float64 and rho_lex.numel() == system.n
    _check(lib().hmpcg_assemble(_ptr(rho_lex), C.byref(system.struct), bc, face, _stream(stream)),
           "assemble")
    return system


def spmv(system, x, y, stream=None):
    """hmpcg_spmv: y = A x with the FP32 mirror."""
    assert x.dtype == torch.float32 and y.dtype == torch.float32
    _check(lib().hmpcg_spmv(C.byref(system.struct), _ptr(x), _ptr(y), _stream(stream)), "spmv")
    return y


def packed_width(n, leaf, rank, kind):
    return int(lib().hmpcg_packed_width(n, leaf, rank, kind))


_DT = {torch.float32: F32, torch.bfloat16: BF16, torch.float8_e4m3fn: FP8E4M3}


def factors(kind, packed, n, leaf, rank, scales=None):
    """hmpcg_factors struct for a packed device tensor (keeps references alive)."""
    f = Factors()
    f.kind = kind
    f.dtype = _DT[packed.dtype]
    f.leaf, f.rank, f.n = leaf, rank, n
    f.packed = packed.data_ptr()
    f.scales = scales.data_ptr() if scales is not None else None
    f._keep = (packed, scales)
    return f


# ------------------------------------------------------------------ context
class Context:
    def __init__(self, max_n, leaf=64, rank=16, d_model=0, n_layers=0, n_heads=0, d_mlp=0,
                 max_batch=1, max_nrhs=1, weights=None, stream=None):
        self.cfg = Config(max_n=max_n, max_batch=max_batch, max_nrhs=max_nrhs, leaf=leaf, rank=rank,
                          d_model=d_model, n_layers=n_layers, n_heads=n_heads, d_mlp=d_mlp)
        h = C.c_void_p()
        wp, wn = None, 0
        if weights is not None:
            import numpy as np
            self._w = np.ascontiguousarray(weights, dtype=np.float32)
            wp, wn = self._w.ctypes.data_as(C.c_void_p), self._w.size
        _check(lib().hmpcg_create(C.byref(h), C.byref(self.cfg), wp, wn, _stream(stream)), "create")
        self.h = h

    def weight_count(self):
        return int(lib().hmpcg_weight_count(C.byref(self.cfg)))

    def close(self):
        if self.h:
            lib().hmpcg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def weight_count(**cfg):
    c = Config(**cfg)
    return int(lib().hmpcg_weight_count(C.byref(c)))


def apply(ctx, f, r, z, nrhs=1, stream=None):
    """hmpcg_apply: z = M r (FP32, node-major)."""
    assert r.dtype == torch.float32 and z.dtype == torch.float32
    _check(lib().hmpcg_apply(ctx.h, C.byref(f), _ptr(r), _ptr(z), nrhs, _stream(stream)), "apply")
    return z


def apply_noalloc(f, r, z, stream=None):
    """hmpcg_apply_noalloc: z = M r with the library's fixed scratch array (no context,
    no allocation); for callers that cannot allocate device memory."""
    assert r.dtype == torch.float32 and z.dtype == torch.float32
    _check(lib().hmpcg_apply_noalloc(C.byref(f), _ptr(r), _ptr(z), _stream(stream)), "apply_noalloc")
    return z


def solve(ctx, system, f, b, x, rtol=1e-6, max_iter=0, recompute_every=10, stream=None,
          info=True, allow=(OK, NOT_CONVERGED)):
    """hmpcg_solve: PCG in one persistent kernel.  Returns a SolveInfo (info=True)."""
    assert b.dtype == torch.float64 and x.dtype == torch.float64
    o = SolveOpts(rtol=rtol, max_iter=max_iter, recompute_every=recompute_every)
    inf = SolveInfo() if info else None
    rc = lib().hmpcg_solve(ctx.h, C.byref(system.struct), C.byref(f) if f is not None else None,
                           _ptr(b), _ptr(x), C.byref(o), C.byref(inf) if info else None, _stream(stream))
    _check(rc, "solve", allow=allow)
    return inf


def _batch_args(systems, facs, bs, xs):
    n = len(systems)
    assert len(bs) == n and len(xs) == n and (facs is None or len(facs) == n)
    sysarr = systems_array(systems)
    facarr = None
    if facs is not None:
        facarr = (Factors * n)()
        for i, f in enumerate(facs):
            facarr[i] = f
    for t in list(bs) + list(xs):
        assert t.dtype == torch.float64 and t.is_cuda
    barr = (C.c_void_p * n)(*[t.data_ptr() for t in bs])
    xarr = (C.c_void_p * n)(*[t.data_ptr() for t in xs])
    return sysarr, facarr, barr, xarr


def solve_batch(ctx, systems, facs, bs, xs, rtol=1e-6, max_iter=0, recompute_every=10, stream=None,
                info=True, allow=(OK, NOT_CONVERGED), fallback=False):
    """hmpcg_solve_batch: independent systems of uneven size, one persistent cluster launch per
    cluster size.  facs: list of Factors (same kind and dtype) or None.  Returns the list of
    per-system SolveInfo (info=True)."""
    sysarr, facarr, barr, xarr = _batch_args(systems, facs, bs, xs)
    o = SolveOpts(rtol=rtol, max_iter=max_iter, recompute_every=recompute_every, fallback=int(fallback))
    n = len(systems)
    infos = (SolveInfo * n)() if info else None
    rc = lib().hmpcg_solve_batch(ctx.h, sysarr, facarr, barr, xarr, n, C.byref(o), infos, _stream(stream))
    _check(rc, "solve_batch", allow=allow)
    return list(infos) if info else None


def autotune_batch(ctx, systems, facs, bs, xs, rtol=1e-6, max_iter=0, recompute_every=10, stream=None):
    """hmpcg_autotune_batch: time each cluster size per distinct n, keep the fastest in the
    context; returns the chosen cluster size of every system."""
    sysarr, facarr, barr, xarr = _batch_args(systems, facs, bs, xs)
    o = SolveOpts(rtol=rtol, max_iter=max_iter, recompute_every=recompute_every)
    n = len(systems)
    out = (C.c_int32 * n)()
    _check(lib().hmpcg_autotune_batch(ctx.h, sysarr, facarr, barr, xarr, n, C.byref(o), out, _stream(stream)),
           "autotune_batch")
    return list(out)


def infer_factors(ctx, systems, packed, scales=None, stream=None):
    """hmpcg_infer_factors: learned factors of len(systems) same-grid systems."""
    arr = systems_array(systems)
    _check(lib().hmpcg_infer_factors(ctx.h, arr, len(systems), _ptr(packed), _DT[packed.dtype],
                                     _ptr(scales), _stream(stream)), "infer_factors")
    return packed


INFER_LAYERED, INFER_FUSED = 0, 1


def set_infer_mode(ctx, mode):
    """hmpcg_set_infer_mode: INFER_FUSED (default) or INFER_LAYERED kernels for infer_factors."""
    _check(lib().hmpcg_set_infer_mode(ctx.h, int(mode)), "set_infer_mode")


PROBES_RADEMACHER, PROBES_GAUSSIAN_SMOOTHED = 0, 1


def set_train_probes(ctx, kind, omega=0.6, steps=2):
    """hmpcg_set_train_probes: Rademacher, or the paper's smoothed Gaussian probes."""
    _check(lib().hmpcg_set_train_probes(ctx.h, int(kind), float(omega), int(steps)), "set_train_probes")


LOSS_COSINE, LOSS_SAI = 0, 1


def set_train_loss(ctx, kind):
    """hmpcg_set_train_loss: LOSS_COSINE (Eq. 7, default) or the LOSS_SAI ablation."""
    _check(lib().hmpcg_set_train_loss(ctx.h, int(kind)), "set_train_loss")


def set_highways(ctx, on):
    """hmpcg_set_highways: highway channels on (default) or held at zero (ablation)."""
    _check(lib().hmpcg_set_highways(ctx.h, int(bool(on))), "set_highways")


def train_step(ctx, systems, n_probes, lr, step_seed, want_loss=True, stream=None):
    """hmpcg_train_step: one AdamW step of the cosine-Hutchinson objective."""
    arr = systems_array(systems)
    loss = C.c_float(0.0)
    _check(lib().hmpcg_train_step(ctx.h, arr, len(systems), n_probes, lr, step_seed,
                                  C.byref(loss) if want_loss else None, _stream(stream)), "train_step")
    return loss.value if want_loss else None


def get_grads(ctx, count):
    import numpy as np
    g = np.empty(count, dtype=np.float32)
    _check(lib().hmpcg_get_grads(ctx.h, g.ctypes.data_as(C.c_void_p), count), "get_grads")
    return g


def get_weights(ctx, count):
    import numpy as np
    w = np.empty(count, dtype=np.float32)
    _check(lib().hmpcg_get_weights(ctx.h, w.ctypes.data_as(C.c_void_p), count), "get_weights")
    return w


def selftest_wait(flag, status, max_iters, stream=None):
    """hmpcg_selftest_wait: bounded wait on a device int32 flag; status (device int32) receives
    OK once the flag is set, else E_TIMEOUT after max_iters polls."""
    assert flag.dtype == torch.int32 and status.dtype == torch.int32
    _check(lib().hmpcg_selftest_wait(_ptr(flag), _ptr(status), int(max_iters), _stream(stream)), "selftest_wait")


def gemm_bf16(a, b, bias=None, act=0, out=None, stream=None):
    """hmpcg_gemm_bf16: C = A B^T (+ bias, GELU) on the tcgen05 GEMM; A, B BF16."""
    assert a.dtype == torch.bfloat16 and b.dtype == torch.bfloat16
    m, k = a.shape
    n = b.shape[0]
    if out is None:
        out = torch.empty(m, n, dtype=torch.float32, device=a.device)
    _check(lib().hmpcg_gemm_bf16(_ptr(a), _ptr(b), _ptr(out), m, n, k, _ptr(bias), act, _stream(stream)),
           "gemm_bf16")
    return out
