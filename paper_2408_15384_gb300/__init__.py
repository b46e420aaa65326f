"""paper_2408_15384_gb300 -- Python binding of libmm, the GB300 (sm_103a) dense
product C = A*B in plain FP64, FP64-accuracy and FP32-accuracy emulation,
grouped and served.

The binding only marshals arguments: every step of the computation runs in the
library's CUDA kernels, and nothing here falls back to the CPU or to torch
arithmetic. Operands are torch CUDA float64 tensors (row-major, unit column
stride) or, for the host entry point, numpy float64 arrays.
"""
from __future__ import annotations

import ctypes
import os

from . import _lib

FP64 = 0
FP64_EMU = 1
FP32_EMU = 2
PRECISIONS = {"fp64": FP64, "fp64_emu": FP64_EMU, "fp32_emu": FP32_EMU}

OK, PENDING = 0, 1
INVALID_ARG, BUDGET, NONFINITE, CUDA_ERROR, TIMEOUT, NOT_FOUND = 2, 3, 4, 5, 6, 7
OPT_SLICES, OPT_TIMEOUT_MS, OPT_AUTOTUNE, OPT_SERVE_MAX_BATCH, OPT_SERVE_STREAMS, OPT_FP64_KERNEL = 1, 2, 3, 4, 5, 6
OPT_PROFILE = 7
OPT_CTA_PAIR = 8
OPT_TILE_N = 9
OPT_INT8_SLICES = 11
OPT_FP64_SCHEME = 12
CRT_BASE = 16   # decision code of the modular form: CRT_BASE + N
KERNEL_SLICE_GEMM, KERNEL_SPLIT, KERNEL_FP64_GEMM, KERNEL_REBUILD = 0, 1, 2, 3


class MMError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib.load().mm_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status})" if what else f"{msg} (status {status})")


def _check(rc: int, what: str):
    if rc != OK:
        raise MMError(rc, what)


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _mat(t, name):
    """(pointer, rows, cols, ld) of a row-major float64 CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.dim() != 2 or not t.is_cuda:
        raise TypeError(f"{name} must be a 2-D torch.float64 CUDA tensor")
    if t.numel() == 0:
        return t.data_ptr(), t.shape[0], t.shape[1], max(t.shape[1], 1)
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError(f"{name} must have unit column stride (row-major)")
    ld = t.stride(0) if t.shape[0] > 1 else max(t.shape[1], 1)
    return t.data_ptr(), t.shape[0], t.shape[1], max(ld, t.shape[1], 1)


class Handle:
    """An mm_handle on one CUDA device (mm_create / mm_destroy)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        _check(self.lib.mm_create(ctypes.byref(h), int(device), int(budget_bytes)), "mm_create")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _check(self.lib.mm_destroy(self.h), "mm_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- GEMM
    def gemm(self, A, B, C=None, precision=FP64_EMU, stream=None):
        """C <- A @ B on the device (asynchronous on `stream`); returns C."""
        import torch
        pa, m, k, lda = _mat(A, "A")
        pb, kb, n, ldb = _mat(B, "B")
        if kb != k:
            raise ValueError("inner dimensions differ")
        if C is None:
            C = torch.empty((m, n), dtype=torch.float64, device=A.device)
        pc, mc, nc, ldc = _mat(C, "C")
        if (mc, nc) != (m, n):
            raise ValueError("C has the wrong shape")
        _check(self.lib.mm_gemm(self.h, m, n, k, pa, lda, pb, ldb, pc, ldc, _prec(precision),
                                _stream_handle(stream)), "mm_gemm")
        return C

    def gemm_host(self, A, B, C=None, precision=FP64_EMU, stream=0):
        """Host (numpy) operands: copies in, computes, copies out, synchronises."""
        import numpy as np
        A = np.asarray(A)
        B = np.asarray(B)
        for name, x in (("A", A), ("B", B)):
            if x.dtype != np.float64 or x.ndim != 2 or x.strides[1] not in (8, 0) and x.shape[1] > 1:
                raise TypeError(f"{name} must be a row-major 2-D float64 array")
        m, k = A.shape
        k2, n = B.shape
        if k2 != k:
            raise ValueError("inner dimensions differ")
        if C is None:
            C = np.empty((m, n), dtype=np.float64)
        lda = A.strides[0] // 8 if m > 1 else max(k, 1)
        ldb = B.strides[0] // 8 if k > 1 else max(n, 1)
        ldc = C.strides[0] // 8 if m > 1 else max(n, 1)
        _check(self.lib.mm_gemm_host(self.h, m, n, k, A.ctypes.data, max(lda, k, 1), B.ctypes.data, max(ldb, n, 1),
                                     C.ctypes.data, max(ldc, n, 1), _prec(precision), int(stream)), "mm_gemm_host")
        return C

    def sync(self, stream=None) -> int:
        """Wait for the stream; return (and clear) the device status of the work queued on it (0 = ok)."""
        return self.lib.mm_sync(self.h, _stream_handle(stream))

    @staticmethod
    def problem_array(problems):
        """The mm_problem array of a list of (A, B, C) CUDA tensors, reusable
        across grouped calls on the same tensors."""
        arr = (_lib.Problem * len(problems))()
        for i, (A, B, C) in enumerate(problems):
            pa, m, k, lda = _mat(A, "A")
            pb, _, n, ldb = _mat(B, "B")
            pc, _, _, ldc = _mat(C, "C")
            arr[i] = _lib.Problem(m, n, k, pa, lda, pb, ldb, pc, ldc)
        return arr

    def grouped(self, problems, precision=FP64_EMU, stream=None):
        """problems: list of (A, B, C) CUDA tensors, or an array from
        problem_array; one grouped launch."""
        arr = problems if isinstance(problems, ctypes.Array) else self.problem_array(problems)
        _check(self.lib.mm_gemm_grouped(self.h, len(arr), arr, _prec(precision), _stream_handle(stream)),
               "mm_gemm_grouped")

    # ------------------------------------------------------------- serving
    def serve_submit(self, A, B, C, precision=FP64_EMU, tag: int = 0) -> int:
        pa, m, k, lda = _mat(A, "A")
        pb, _, n, ldb = _mat(B, "B")
        pc, _, _, ldc = _mat(C, "C")
        req = _lib.Request(_lib.Problem(m, n, k, pa, lda, pb, ldb, pc, ldc), _prec(precision), tag)
        t = ctypes.c_uint64()
        _check(self.lib.mm_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t)), "mm_serve_submit")
        return t.value

    def serve_poll(self, ticket: int):
        """(status, ReqStatus or None)."""
        st = _lib.ReqStatus()
        rc = self.lib.mm_serve_poll(self.h, ticket, ctypes.byref(st))
        return rc, (st if rc != PENDING else None)

    def serve_drain(self):
        _check(self.lib.mm_serve_drain(self.h), "mm_serve_drain")

    def serve_bench(self, count, dim_lo=64, dim_hi=4096, fp64_share=0.5, rate_per_s=0.0, seed=5, slots=64,
                    sample_every=0, max_samples=64, sample_cap=1 << 24):
        """Run a seeded request stream through the serving calls (mm_serve_bench).
        Returns (result dict, list of sample dicts with their C as numpy arrays)."""
        import numpy as np
        load = _lib.ServeLoad(count, dim_lo, dim_hi, fp64_share, rate_per_s, seed, slots, sample_every)
        res = _lib.ServeLoadResult()
        samples = (_lib.ServeSample * max(max_samples, 1))()
        host = np.zeros(sample_cap if sample_every else 1, dtype=np.float64)
        ns = ctypes.c_int64()
        _check(self.lib.mm_serve_bench(self.h, ctypes.byref(load), ctypes.byref(res), samples, max_samples,
                                       ctypes.byref(ns), host.ctypes.data, host.size), "mm_serve_bench")
        out = {f: getattr(res, f) for f, _ in _lib.ServeLoadResult._fields_}
        smp = []
        for i in range(ns.value):
            sm = samples[i]
            C = host[sm.host_offset: sm.host_offset + sm.m * sm.n].reshape(sm.m, sm.n).copy()
            smp.append({"index": sm.index, "m": sm.m, "n": sm.n, "k": sm.k, "precision": sm.precision,
                        "slot": sm.slot, "C": C})
        return out, smp

    # ------------------------------------------------------- configuration
    def set_option(self, opt: int, value: int):
        _check(self.lib.mm_set_option(self.h, opt, int(value)), "mm_set_option")

    def get_option(self, opt: int) -> int:
        v = ctypes.c_int64()
        _check(self.lib.mm_get_option(self.h, opt, ctypes.byref(v)), "mm_get_option")
        return v.value

    def stats(self) -> int:
        v = ctypes.c_uint64()
        _check(self.lib.mm_stats(self.h, ctypes.byref(v)), "mm_stats")
        return v.value

    def profile_read(self, kernel: int, reset: bool = False):
        """(device ms summed over the launches of `kernel`, launch count)."""
        ms, n = ctypes.c_double(), ctypes.c_uint64()
        _check(self.lib.mm_profile_read(self.h, kernel, ctypes.byref(ms), ctypes.byref(n), int(reset)),
               "mm_profile_read")
        return ms.value, n.value

    # ----------------------------------------------------------- autotuner
    def tune_save(self, path: str):
        _check(self.lib.mm_tune_save(self.h, os.fsencode(path)), "mm_tune_save")

    def tune_load(self, path: str):
        _check(self.lib.mm_tune_load(self.h, os.fsencode(path)), "mm_tune_load")

    def tune_lookup(self, precision: int, a: int, b: int, c: int = 0, grouped: bool = False):
        """(bn, cg, kern) tuned for the bucket, or None."""
        bn, cg, kern = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rc = self.lib.mm_tune_lookup(self.h, int(grouped), precision, a, b, c, ctypes.byref(bn), ctypes.byref(cg),
                                     ctypes.byref(kern))
        if rc == NOT_FOUND:
            return None
        _check(rc, "mm_tune_lookup")
        return bn.value, cg.value, kern.value

    def debug_wait_timeout(self, timeout_ms: int, stream=None) -> int:
        """Status of a bounded device wait that is made to run out (MM_ERR_TIMEOUT expected)."""
        return self.lib.mm_debug_wait_timeout(self.h, int(timeout_ms), _stream_handle(stream))

    def peak_fp64(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(self.lib.mm_peak_fp64(self.h, ctypes.byref(a), ctypes.byref(b)), "mm_peak_fp64")
        return a.value, b.value

    # --------------------------------------------------------- diagnostics
    def debug_slices(self, X, which: int, precision=FP64_EMU, s: int = 5, stream=None):
        """(exps int32, slices uint16 [S][vectors][k]) for A (which=0) or B (which=1)."""
        import torch
        px, rows, cols, ldx = _mat(X, "X")
        S = s if _prec(precision) == FP64_EMU else 3
        nvec, klen = (rows, cols) if which == 0 else (cols, rows)
        exps = torch.zeros(nvec, dtype=torch.int32, device=X.device)
        sl = torch.zeros((S, nvec, klen), dtype=torch.int16, device=X.device)
        rc = self.lib.mm_debug_slices(self.h, which, _prec(precision), s, rows, cols, px, ldx, exps.data_ptr(),
                                      sl.data_ptr(), _stream_handle(stream))
        if rc not in (OK, 4):
            raise MMError(rc, "mm_debug_slices")
        return exps, sl, rc

    def debug_levels_int8(self, A, B, s: int, stream=None):
        """Level products of the INT8 digit form as int64 [s][m][n]."""
        import torch
        pa, m, k, lda = _mat(A, "A")
        pb, _, n, ldb = _mat(B, "B")
        L = torch.empty((s, m, n), dtype=torch.int64, device=A.device)
        _check(self.lib.mm_debug_level_products_int8(self.h, m, n, k, pa, lda, pb, ldb, s, L.data_ptr(),
                                                     _stream_handle(stream)), "mm_debug_level_products_int8")
        return L

    def debug_slice_count(self, A, B, stream=None):
        """(s, alpha_min, beta_min) as the device decides them for A*B."""
        pa, m, k, lda = _mat(A, "A")
        pb, _, n, ldb = _mat(B, "B")
        s = ctypes.c_int(0)
        a = ctypes.c_float(0.0)
        b = ctypes.c_float(0.0)
        rc = self.lib.mm_debug_slice_count(self.h, m, n, k, pa, lda, pb, ldb, ctypes.byref(s), ctypes.byref(a),
                                           ctypes.byref(b), _stream_handle(stream))
        _check(rc, "mm_debug_slice_count")
        return s.value, a.value, b.value

    def debug_crt_residues(self, X, which: int, N: int, bits: int, stream=None):
        """(exps int32, residues uint16 [N][vectors][k] as bfloat16 bits) of the
        modular form for A (which=0) or B (which=1), N moduli, b-bit integers."""
        import torch
        px, rows, cols, ldx = _mat(X, "X")
        nvec, klen = (rows, cols) if which == 0 else (cols, rows)
        exps = torch.zeros(nvec, dtype=torch.int32, device=X.device)
        pl = torch.zeros((N, nvec, klen), dtype=torch.int16, device=X.device)
        rc = self.lib.mm_debug_crt_residues(self.h, which, N, bits, rows, cols, px, ldx, exps.data_ptr(),
                                            pl.data_ptr(), _stream_handle(stream))
        if rc not in (OK, 4):
            raise MMError(rc, "mm_debug_crt_residues")
        return exps, pl, rc

    def debug_crt_rebuild(self, res, E, F, N: int, bits: int, stream=None):
        """The modular form's rebuild pass alone: C (m x n float64) from
        residue bytes res (uint8 [N][m][n], device), row exponents E (int32 m)
        and column exponents F (int32 n), N moduli, b = bits."""
        import torch
        if res.dtype != torch.uint8 or res.dim() != 3 or res.shape[0] != N:
            raise ValueError("res must be uint8 [N][m][n]")
        _, m, n = res.shape
        n8 = (n + 7) // 8
        # the slice GEMM's layout: per plane, blocks of 8 columns of the rows' 8-byte records
        pad = torch.zeros((N, m, 8 * n8), dtype=torch.uint8, device=res.device)
        pad[:, :, :n] = res
        lay = pad.reshape(N, m, n8, 8).permute(0, 2, 1, 3).contiguous()
        E = E.to(device=res.device, dtype=torch.int32).contiguous()
        F = F.to(device=res.device, dtype=torch.int32).contiguous()
        C = torch.empty((m, n), dtype=torch.float64, device=res.device)
        rc = self.lib.mm_debug_crt_rebuild(self.h, m, n, N, bits, lay.data_ptr(), E.data_ptr(), F.data_ptr(),
                                           C.data_ptr(), n, _stream_handle(stream))
        if rc != OK:
            raise MMError(rc, "mm_debug_crt_rebuild")
        return C

    def debug_fp64_product(self, A, B, C=None, residues=True, stream=None):
        """One automatic FP64-accuracy product as mm_gemm runs it: (C, code,
        bits, alpha_min, beta_min, residues uint8 [N][m][n] or None)."""
        import torch
        pa, m, k, lda = _mat(A, "A")
        pb, _, n, ldb = _mat(B, "B")
        if C is None:
            C = torch.empty((m, n), dtype=torch.float64, device=A.device)
        pc, _, _, ldc = _mat(C, "C")
        res = torch.zeros((14 * m * n if residues else 1,), dtype=torch.uint8, device=A.device)
        code, bits = ctypes.c_int(0), ctypes.c_int(0)
        a, b = ctypes.c_float(0.0), ctypes.c_float(0.0)
        rc = self.lib.mm_debug_fp64_product(self.h, m, n, k, pa, lda, pb, ldb, pc, ldc,
                                            res.data_ptr() if residues else None,
                                            ctypes.byref(code), ctypes.byref(bits), ctypes.byref(a), ctypes.byref(b),
                                            _stream_handle(stream))
        if rc not in (OK, 4):
            raise MMError(rc, "mm_debug_fp64_product")
        N = code.value - CRT_BASE
        r = res[: N * m * n].view(N, m, n) if (N > 0 and residues) else None
        return C, code.value, bits.value, a.value, b.value, r

    def debug_levels(self, A, B, s: int, stream=None):
        """Level products L_d (d = 2..s+1) as int64 [s][m][n]."""
        import torch
        pa, m, k, lda = _mat(A, "A")
        pb, _, n, ldb = _mat(B, "B")
        L = torch.empty((s, m, n), dtype=torch.int64, device=A.device)
        _check(self.lib.mm_debug_level_products(self.h, m, n, k, pa, lda, pb, ldb, s, L.data_ptr(),
                                                _stream_handle(stream)), "mm_debug_level_products")
        return L


def slice_count_rule(k: int, alpha_min: float, beta_min: float) -> int:
    """The automatic FP64-accuracy slice count for inner dimension k and the
    smallest row / column spreads (8: the plain FP64 kernel)."""
    return _lib.load().mm_slice_count_rule(int(k), float(alpha_min), float(beta_min))


def crt_rule(k: int, alpha_min: float, beta_min: float):
    """(N, b) of the modular form for inner dimension k and the smallest spreads
    (N = 0: it does not fit)."""
    b = ctypes.c_int(0)
    N = _lib.load().mm_crt_rule(int(k), float(alpha_min), float(beta_min), ctypes.byref(b))
    return N, b.value


def fill_uniform(X, seed: int, stream_id: int, scale_mode: int = 0, exp_stream_id: int = 0, stream=None):
    """Device-side fill with the seeded generator of the inputs module."""
    px, rows, cols, ld = _mat(X, "X")
    _check(_lib.load().mm_fill_uniform(px, rows, cols, ld, seed, stream_id, scale_mode, exp_stream_id,
                                       _stream_handle(stream)), "mm_fill_uniform")
    return X
