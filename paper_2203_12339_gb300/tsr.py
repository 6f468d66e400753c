"""Python binding of libtsr (the C ABI in include/tsr.h).

Argument marshalling only: each function checks shapes/dtypes, allocates the
outputs with PyTorch on the current CUDA device, and calls the library entry
point of the same name on the current stream.  Every step of the computation
runs in the library's CUDA kernels; if the library is missing this module
raises instead of computing anything another way.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtsr.so")

TSR_FP32, TSR_BF16, TSR_BF16X3 = 0, 1, 2
PRECISIONS = {"fp32": TSR_FP32, "bf16": TSR_BF16, "bf16x3": TSR_BF16X3}
STATUS_NAMES = {0: "TSR_OK", -1: "TSR_ERR_INVALID_ARG", -2: "TSR_ERR_CUDA", -3: "TSR_ERR_OOM",
                -4: "TSR_ERR_TIMEOUT", -5: "TSR_ERR_UNSUPPORTED"}

_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGNATURES = {
    "tsr_last_error": (ctypes.c_char_p, []),
    "tsr_version": (_I, []),
    "tsr_stream_status": (_I, [_P]),
    "tsr_kernel_launches": (ctypes.c_uint64, []),
    "tsr_selftest_bounded_wait": (_I, [ctypes.c_uint, _P]),
    "tsr_fit_pca_basis": (_I, [_I, _P, _P, _D, _I, _D, _I, _P, ctypes.POINTER(_P), _P]),
    "tsr_basis_create": (_I, [_I, _I, _D, _P, ctypes.POINTER(_P)]),
    "tsr_basis_table": (_I, [_P, _P, _P]),
    "tsr_basis_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "tsr_basis_far_series": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "tsr_kernel_timing": (_I, [_I]),
    "tsr_kernel_timing_read": (_I, [ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "tsr_basis_destroy": (None, [_P]),
    "tsr_project_material": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P]),
    "tsr_project_material_backward": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
    "tsr_precompute_transfer": (_I, [_P, _I, _P, _P, _P, _I, _I, _P, _P]),
    "tsr_precompute_transfer_batched": (_I, [_P, _I, _P, _P, _P, _P, _I, _I, _P, _P]),
    "tsr_batch_plan_create": (_I, [_P, _I, _P, _I, _I, ctypes.POINTER(_P)]),
    "tsr_batch_plan_autotune": (_I, [_P, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_float)]),
    "tsr_precompute_transfer_plan": (_I, [_P, _P, _P, _P, _P, _P]),
    "tsr_batch_plan_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "tsr_batch_plan_destroy": (None, [_P]),
    "tsr_haar_forward": (_I, [_P, _I, _I, _P, _P]),
    "tsr_haar_inverse": (_I, [_P, _I, _I, _P, _P]),
    "tsr_wavelet_compress": (_I, [_P, _I, _I, _I, _D, ctypes.POINTER(_P), _P]),
    "tsr_haar_compress": (_I, [_P, _I, _I, _I, _D, ctypes.POINTER(_P), _P]),
    "tsr_haar_compress_energy": (_I, [_P, _I, _I, _I, _D, ctypes.POINTER(_P), _P]),
    "tsr_compress": (_I, [_P, _I, _I, _I, _I, _I, _D, ctypes.POINTER(_P), _P]),
    "tsr_fresnel_output": (_I, [_I, _P, _I, _P, _P, _P, _P]),
    "tsr_fresnel_output_backward": (_I, [_I, _P, _I, _P, _P, _P, _P, _P, _P]),
    "tsr_sh_transfer": (_I, [_I, _P, _I, _D, _P, _P]),
    "tsr_visibility_transfer": (_I, [_I, _P, _P, _I, _P, _I, _I, _D, ctypes.c_float, _P, _P]),
    "tsr_cdf97_forward": (_I, [_P, _I, _I, _P, _P]),
    "tsr_cdf97_inverse": (_I, [_P, _I, _I, _P, _P]),
    "tsr_cdf97_inverse_transpose": (_I, [_P, _I, _I, _P, _P]),
    "tsr_haar_recompress": (_I, [_P, _P, _P]),
    "tsr_compressed_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                 ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_I)]),
    "tsr_compressed_export": (_I, [_P, _P, _P, _P, _P]),
    "tsr_compressed_destroy": (None, [_P]),
    "tsr_relight": (_I, [_P, _I, _P, _P, _P, _P]),
    "tsr_relight_backward": (_I, [_P, _I, _P, _P, _P, _P, _P, _P]),
    "tsr_relight_noalloc": (_I, [_P, _I, _P, _P, _P, _P]),
    "tsr_relight_many": (_I, [_I, _P, _I, _P, _P, _P, _P]),
    "tsr_haar_compress_batched": (_I, [_I, _P, _P, _I, _I, _D, _P, _P]),
    "tsr_compressed_save": (_I, [_P, ctypes.c_char_p]),
    "tsr_fault_inject": (_I, [_I, _I]),
    "tsr_compressed_load": (_I, [ctypes.c_char_p, ctypes.POINTER(_P)]),
    "tsr_haar_recompress_batched": (_I, [_I, _P, _P, _P, _P]),
}


class TsrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """The loaded libtsr.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                                   "(there is no fallback implementation)")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
        return _lib


def _check(status: int) -> None:
    if status != 0:
        raise TsrError(status, lib().tsr_last_error().decode(errors="replace"))


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _dev(t: torch.Tensor, dtype: torch.dtype, shape: tuple | None = None, name: str = "tensor") -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.contiguous()


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def stream_status() -> None:
    """Synchronise the current stream and raise if a kernel gave up a bounded wait."""
    _check(lib().tsr_stream_status(_stream()))


def kernel_timing(enable: bool) -> None:
    """tsr_kernel_timing: bracket each launch of the transfer's tensor-core kernel with CUDA events."""
    _check(lib().tsr_kernel_timing(1 if enable else 0))


def kernel_timing_read():
    """tsr_kernel_timing_read: (total ms, launches) of the timed kernel launches since the last read."""
    ms, n = _D(), _I()
    _check(lib().tsr_kernel_timing_read(ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def kernel_launches() -> int:
    """Kernel launches made by the library so far in this process."""
    return int(lib().tsr_kernel_launches())


FAULT_KINDS = {"alloc": 1, "cuda": 2, "timeout": 3}


def fault_inject(kind: str, n: int = 1) -> None:
    """tsr_fault_inject: the next n occurrences of `kind` ("alloc", "cuda", "timeout") fail on the host."""
    _check(lib().tsr_fault_inject(FAULT_KINDS[kind], n))


def selftest_bounded_wait(limit: int = 1000) -> None:
    """Run the bounded-wait diagnostic kernel (a wait that nothing ends); see include/tsr.h."""
    _check(lib().tsr_selftest_bounded_wait(int(limit), _stream()))


# ---------------------------------------------------------------- basis
class Basis:
    """Radial PCA basis f_k on the grid r_m = r_max m/(n_r-1) (owned by the library)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        K, n_r, r_max = _I(), _I(), _D()
        _check(lib().tsr_basis_info(self._h, ctypes.byref(K), ctypes.byref(n_r), ctypes.byref(r_max)))
        self.K, self.n_r, self.r_max = K.value, n_r.value, r_max.value

    @property
    def handle(self):
        return self._h

    def far_series(self):
        """tsr_basis_far_series: (relative error of the 12-term far-field series, used by BF16)."""
        err, used = _D(), _I()
        _check(lib().tsr_basis_far_series(self._h, ctypes.byref(err), ctypes.byref(used)))
        return err.value, bool(used.value)

    def table(self) -> torch.Tensor:
        f = torch.empty((self.K, self.n_r), dtype=torch.float64, device="cuda")
        _check(lib().tsr_basis_table(self._h, _ptr(f), _stream()))
        return f

    def close(self):
        if self._h:
            lib().tsr_basis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fit_pca_basis(sigma_a: torch.Tensor, sigma_s: torch.Tensor, eta: float = 1.3, n_r: int = 1024,
                  r_max: float = 40.0, K: int = 12) -> tuple[Basis, torch.Tensor]:
    """tsr_fit_pca_basis: returns the basis and the singular values (FP64, descending)."""
    sa = _dev(sigma_a, torch.float64, name="sigma_a")
    ss = _dev(sigma_s, torch.float64, sa.shape, name="sigma_s")
    n_mat = sa.numel()
    sv = torch.empty(min(n_mat, n_r), dtype=torch.float64, device=sa.device)
    h = _P()
    _check(lib().tsr_fit_pca_basis(n_mat, _ptr(sa), _ptr(ss), float(eta), n_r, float(r_max), K, _ptr(sv),
                                   ctypes.byref(h), _stream()))
    return Basis(h), sv


def basis_create(f, r_max: float = 40.0) -> Basis:
    """tsr_basis_create from a host table f[K][n_r] (FP64)."""
    ft = torch.as_tensor(f, dtype=torch.float64).contiguous().cpu()
    K, n_r = ft.shape
    h = _P()
    _check(lib().tsr_basis_create(K, n_r, float(r_max), ctypes.c_void_p(ft.data_ptr()), ctypes.byref(h)))
    return Basis(h)


def project_material(basis: Basis, sigma_a: torch.Tensor, sigma_s: torch.Tensor, eta: torch.Tensor,
                     jacobian: bool = False):
    """tsr_project_material: returns (g f64 [n,3,K], g32 f32 [n,3,K], dg f64 [n,3,K,3] or None)."""
    sa = _dev(sigma_a, torch.float64, name="sigma_a")
    n = sa.shape[0]
    sa = _dev(sa, torch.float64, (n, 3), "sigma_a")
    ss = _dev(sigma_s, torch.float64, (n, 3), "sigma_s")
    et = _dev(eta, torch.float64, (n,), "eta")
    g = torch.empty((n, 3, basis.K), dtype=torch.float64, device=sa.device)
    g32 = torch.empty((n, 3, basis.K), dtype=torch.float32, device=sa.device)
    dg = torch.empty((n, 3, basis.K, 3), dtype=torch.float64, device=sa.device) if jacobian else None
    _check(lib().tsr_project_material(basis.handle, n, _ptr(sa), _ptr(ss), _ptr(et), _ptr(g), _ptr(g32), _ptr(dg),
                                      _stream()))
    return g, g32, dg


def project_material_backward(basis: Basis, sigma_a, sigma_s, eta, dLdg: torch.Tensor):
    """tsr_project_material_backward: returns (dsigma_a [n,3], dsigma_s [n,3], deta [n]) in FP32."""
    n = sigma_a.shape[0]
    sa = _dev(sigma_a, torch.float64, (n, 3), "sigma_a")
    ss = _dev(sigma_s, torch.float64, (n, 3), "sigma_s")
    et = _dev(eta, torch.float64, (n,), "eta")
    dg = _dev(dLdg, torch.float32, (n, 3, basis.K), "dLdg")
    dsa = torch.empty((n, 3), dtype=torch.float32, device=sa.device)
    dss = torch.empty((n, 3), dtype=torch.float32, device=sa.device)
    de = torch.empty((n,), dtype=torch.float32, device=sa.device)
    _check(lib().tsr_project_material_backward(basis.handle, n, _ptr(sa), _ptr(ss), _ptr(et), _ptr(dg), _ptr(dsa),
                                               _ptr(dss), _ptr(de), _stream()))
    return dsa, dss, de


# ---------------------------------------------------------------- transfer
def precompute_transfer(basis: Basis, pos: torch.Tensor, area: torch.Tensor, T: torch.Tensor,
                        precision: str = "bf16", out: torch.Tensor | None = None) -> torch.Tensor:
    """tsr_precompute_transfer: M[k][j][o] = sum_i A_i f_k(|x_o-x_i|) T[j][i]; pos is [3][N] FP32."""
    N = pos.shape[1]
    p = _dev(pos, torch.float32, (3, N), "pos")
    a = _dev(area, torch.float32, (N,), "area")
    J = T.shape[0]
    t = _dev(T, torch.float32, (J, N), "T")
    M = out if out is not None else torch.empty((basis.K, J, N), dtype=torch.float32, device=p.device)
    _dev(M, torch.float32, (basis.K, J, N), "out")
    _check(lib().tsr_precompute_transfer(basis.handle, N, _ptr(p), _ptr(a), _ptr(t), J, PRECISIONS[precision],
                                         _ptr(M), _stream()))
    return M


def precompute_transfer_batched(basis: Basis, offsets, pos: torch.Tensor, area: torch.Tensor, T: torch.Tensor,
                                precision: str = "bf16", out: torch.Tensor | None = None) -> torch.Tensor:
    """tsr_precompute_transfer_batched over meshes concatenated along the vertex axis (offsets on the host)."""
    off = torch.as_tensor(offsets, dtype=torch.int64).contiguous().cpu()
    n_mesh = off.numel() - 1
    total = int(off[-1])
    p = _dev(pos, torch.float32, (3, total), "pos")
    a = _dev(area, torch.float32, (total,), "area")
    J = T.shape[0]
    t = _dev(T, torch.float32, (J, total), "T")
    M = out if out is not None else torch.empty((basis.K, J, total), dtype=torch.float32, device=p.device)
    _check(lib().tsr_precompute_transfer_batched(basis.handle, n_mesh, ctypes.c_void_p(off.data_ptr()), _ptr(p),
                                                 _ptr(a), _ptr(t), J, PRECISIONS[precision], _ptr(M), _stream()))
    return M


class BatchPlan:
    """Plan of a batched transfer (unit and mesh tables on the device; owned by the library)."""

    def __init__(self, basis: Basis, offsets, J: int, precision: str = "bf16"):
        self.offsets = torch.as_tensor(offsets, dtype=torch.int64).contiguous().cpu()
        self.basis, self.J = basis, J
        self.total = int(self.offsets[-1])
        h = _P()
        _check(lib().tsr_batch_plan_create(basis.handle, self.offsets.numel() - 1, ctypes.c_void_p(self.offsets.data_ptr()),
                                           J, PRECISIONS[precision], ctypes.byref(h)))
        self._h = h

    def _args(self, pos, area, T, out):
        p = _dev(pos, torch.float32, (3, self.total), "pos")
        a = _dev(area, torch.float32, (self.total,), "area")
        t = _dev(T, torch.float32, (self.J, self.total), "T")
        M = out if out is not None else torch.empty((self.basis.K, self.J, self.total), dtype=torch.float32,
                                                    device=p.device)
        return p, a, t, M

    def autotune(self, pos, area, T, out=None) -> float:
        """tsr_batch_plan_autotune: returns the best time (ms) and keeps that generator configuration."""
        p, a, t, M = self._args(pos, area, T, out)
        best = ctypes.c_float()
        _check(lib().tsr_batch_plan_autotune(self._h, _ptr(p), _ptr(a), _ptr(t), _ptr(M), _stream(), ctypes.byref(best)))
        return best.value

    def run(self, pos, area, T, out=None) -> torch.Tensor:
        """tsr_precompute_transfer_plan (enqueue only; capturable in a CUDA graph)."""
        p, a, t, M = self._args(pos, area, T, out)
        _check(lib().tsr_precompute_transfer_plan(self._h, _ptr(p), _ptr(a), _ptr(t), _ptr(M), _stream()))
        return M

    def info(self):
        n, gen, par = _I(), _I(), _I()
        _check(lib().tsr_batch_plan_info(self._h, ctypes.byref(n), ctypes.byref(gen), ctypes.byref(par)))
        return {"units": n.value, "generator": "series" if gen.value == 0 else "table",
                "param": par.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().tsr_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- wavelet / compression
def chart_side(nu: int) -> int:
    P = 1
    while P < nu:
        P *= 2
    return P


def haar_forward(X: torch.Tensor, nu: int) -> torch.Tensor:
    """tsr_haar_forward: X [rows][10 nu^2 + 2] -> Xw [rows][10 P^2 + 2]."""
    N = 10 * nu * nu + 2
    x = _dev(X, torch.float32, name="X").reshape(-1, N)
    P = chart_side(nu)
    Xw = torch.empty((x.shape[0], 10 * P * P + 2), dtype=torch.float32, device=x.device)
    _check(lib().tsr_haar_forward(_ptr(x), x.shape[0], nu, _ptr(Xw), _stream()))
    return Xw.reshape(X.shape[:-1] + (10 * P * P + 2,))


def haar_inverse(Xw: torch.Tensor, nu: int) -> torch.Tensor:
    """tsr_haar_inverse: Xw [rows][10 P^2 + 2] -> X [rows][10 nu^2 + 2]."""
    P = chart_side(nu)
    x = _dev(Xw, torch.float32, name="Xw").reshape(-1, 10 * P * P + 2)
    X = torch.empty((x.shape[0], 10 * nu * nu + 2), dtype=torch.float32, device=x.device)
    _check(lib().tsr_haar_inverse(_ptr(x), x.shape[0], nu, _ptr(X), _stream()))
    return X.reshape(Xw.shape[:-1] + (10 * nu * nu + 2,))


def _chart_op(fn, x_in: torch.Tensor, n_in: int, n_out: int, nu: int) -> torch.Tensor:
    x = _dev(x_in, torch.float32, name="input").reshape(-1, n_in)
    y = torch.empty((x.shape[0], n_out), dtype=torch.float32, device=x.device)
    _check(fn(_ptr(x), x.shape[0], nu, _ptr(y), _stream()))
    return y.reshape(x_in.shape[:-1] + (n_out,))


def cdf97_forward(X: torch.Tensor, nu: int) -> torch.Tensor:
    """tsr_cdf97_forward: X [rows][10 nu^2 + 2] -> Xw [rows][10 P^2 + 2] (CDF 9/7 pyramid per chart)."""
    P = chart_side(nu)
    return _chart_op(lib().tsr_cdf97_forward, X, 10 * nu * nu + 2, 10 * P * P + 2, nu)


def cdf97_inverse(Xw: torch.Tensor, nu: int) -> torch.Tensor:
    """tsr_cdf97_inverse: the synthesis, Xw [rows][10 P^2 + 2] -> X [rows][10 nu^2 + 2]."""
    P = chart_side(nu)
    return _chart_op(lib().tsr_cdf97_inverse, Xw, 10 * P * P + 2, 10 * nu * nu + 2, nu)


def cdf97_inverse_transpose(X: torch.Tensor, nu: int) -> torch.Tensor:
    """tsr_cdf97_inverse_transpose: the transpose of the synthesis, X [rows][N] -> [rows][10 P^2 + 2]."""
    P = chart_side(nu)
    return _chart_op(lib().tsr_cdf97_inverse_transpose, X, 10 * nu * nu + 2, 10 * P * P + 2, nu)


class Compressed:
    """Compressed wavelet transfer (CSR over wavelet rows; owned by the library)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        K, J, nu, n_rows = _I(), _I(), _I(), _I()
        nnz = ctypes.c_int64()
        _check(lib().tsr_compressed_info(self._h, ctypes.byref(K), ctypes.byref(J), ctypes.byref(nu),
                                         ctypes.byref(nnz), ctypes.byref(n_rows)))
        self.K, self.J, self.nu, self.nnz, self.n_rows = K.value, J.value, nu.value, nnz.value, n_rows.value

    @property
    def handle(self):
        return self._h

    @property
    def n(self) -> int:
        return 10 * self.nu * self.nu + 2

    def export(self):
        """(row_ptr int64 [n_rows+1], col int32 [nnz], val f32 [nnz]) on the device."""
        row_ptr = torch.empty(self.n_rows + 1, dtype=torch.int64, device="cuda")
        col16 = torch.empty(self.nnz, dtype=torch.int16, device="cuda")
        val = torch.empty(self.nnz, dtype=torch.float32, device="cuda")
        _check(lib().tsr_compressed_export(self._h, _ptr(row_ptr), _ptr(col16), _ptr(val), _stream()))
        col = col16.to(torch.int32) & 0xFFFF
        return row_ptr, col, val

    def save(self, path: str) -> None:
        """tsr_compressed_save: write the handle to `path`."""
        _check(lib().tsr_compressed_save(self._h, os.fsencode(path)))

    @staticmethod
    def load(path: str) -> "Compressed":
        """tsr_compressed_load: a new handle on the current device from a file written by save()."""
        h = _P()
        _check(lib().tsr_compressed_load(os.fsencode(path), ctypes.byref(h)))
        return Compressed(h)

    def close(self):
        if self._h:
            lib().tsr_compressed_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wavelet_compress(Mw: torch.Tensor, nu: int, p: float) -> Compressed:
    """tsr_wavelet_compress from wavelet coefficients Mw [K][J][10 P^2 + 2]."""
    K, J, NW = Mw.shape
    m = _dev(Mw, torch.float32, name="Mw")
    h = _P()
    _check(lib().tsr_wavelet_compress(_ptr(m), K, J, nu, float(p), ctypes.byref(h), _stream()))
    return Compressed(h)


def haar_compress(M: torch.Tensor, nu: int, p: float, out: Compressed | None = None) -> Compressed:
    """tsr_haar_compress: forward Haar of M [K][J][N] then the top-p keep rule.

    With ``out`` (a handle of the same K, J, nu and p) the result is written into
    it by tsr_haar_recompress, without allocating a new handle."""
    K, J, N = M.shape
    m = _dev(M, torch.float32, (K, J, 10 * nu * nu + 2), "M")
    if out is not None:
        if (out.K, out.J, out.nu) != (K, J, nu):
            raise ValueError("out handle has different K, J or nu")
        _check(lib().tsr_haar_recompress(_ptr(m), out.handle, _stream()))
        return out
    h = _P()
    _check(lib().tsr_haar_compress(_ptr(m), K, J, nu, float(p), ctypes.byref(h), _stream()))
    return Compressed(h)


def _offsets_host(offsets):
    import numpy as np
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    return offs, offs.ctypes.data_as(ctypes.c_void_p)


def haar_compress_batched(M: torch.Tensor, offsets, p: float) -> list:
    """tsr_haar_compress_batched: M [K][J][total] (a batched transfer) -> one Compressed per mesh."""
    K, J, total = M.shape
    m = _dev(M, torch.float32, name="M")
    offs, op = _offsets_host(offsets)
    n = len(offs) - 1
    if offs[-1] != total:
        raise ValueError(f"offsets end at {offs[-1]}, M has {total} columns")
    hs = (ctypes.c_void_p * n)()
    _check(lib().tsr_haar_compress_batched(n, op, _ptr(m), K, J, float(p), ctypes.cast(hs, ctypes.c_void_p),
                                           _stream()))
    return [Compressed(ctypes.c_void_p(h)) for h in hs]


def haar_recompress_batched(M: torch.Tensor, offsets, comps) -> None:
    """tsr_haar_recompress_batched: refill the per-mesh handles from a new batched M [K][J][total]."""
    m = _dev(M, torch.float32, name="M")
    offs, op = _offsets_host(offsets)
    comps = list(comps)
    if len(comps) != len(offs) - 1:
        raise ValueError("one handle per mesh")
    hs = (ctypes.c_void_p * len(comps))(*[c.handle.value for c in comps])
    _check(lib().tsr_haar_recompress_batched(len(comps), op, _ptr(m), ctypes.cast(hs, ctypes.c_void_p), _stream()))


def haar_compress_energy(M: torch.Tensor, nu: int, energy: float) -> Compressed:
    """tsr_haar_compress_energy: forward Haar of M [K][J][N], then per (k, j) the fewest largest
    coefficients holding at least `energy` of the row's energy (the poles always kept)."""
    K, J, N = M.shape
    m = _dev(M, torch.float32, (K, J, 10 * nu * nu + 2), "M")
    h = _P()
    _check(lib().tsr_haar_compress_energy(_ptr(m), K, J, nu, float(energy), ctypes.byref(h), _stream()))
    return Compressed(h)


WAVELETS = {"haar": 0, "cdf97": 1}
KEEP_RULES = {"top": 0, "energy": 1}


def compress(M: torch.Tensor, nu: int, wavelet: str = "haar", rule: str = "top", param: float = 0.1) -> Compressed:
    """tsr_compress: Step 2 with the Haar or CDF 9/7 spatial wavelet and the top-fraction or energy keep rule."""
    K, J, N = M.shape
    m = _dev(M, torch.float32, (K, J, 10 * nu * nu + 2), "M")
    h = _P()
    _check(lib().tsr_compress(_ptr(m), K, J, nu, WAVELETS[wavelet], KEEP_RULES[rule], float(param), ctypes.byref(h),
                              _stream()))
    return Compressed(h)


# ---------------------------------------------------------------- Fresnel factors
def fresnel_output(B: torch.Tensor, eta: torch.Tensor, cos_o: torch.Tensor, out: torch.Tensor | None = None):
    """tsr_fresnel_output: (1/pi) F_t(eta_e, cos_o) B for B [E][3][N], eta [E] FP64, cos_o [N] FP32."""
    E, _, N = B.shape
    b = _dev(B, torch.float32, (E, 3, N), "B")
    e = _dev(eta, torch.float64, (E,), "eta")
    c = _dev(cos_o, torch.float32, (N,), "cos_o")
    o = out if out is not None else torch.empty_like(b)
    _check(lib().tsr_fresnel_output(E, _ptr(e), N, _ptr(c), _ptr(b), _ptr(o), _stream()))
    return o


def fresnel_output_backward(B: torch.Tensor, eta: torch.Tensor, cos_o: torch.Tensor, dBout: torch.Tensor):
    """tsr_fresnel_output_backward: returns (dL/dB [E][3][N] FP32, dL/deta [E] FP32)."""
    E, _, N = B.shape
    b = _dev(B, torch.float32, (E, 3, N), "B")
    e = _dev(eta, torch.float64, (E,), "eta")
    c = _dev(cos_o, torch.float32, (N,), "cos_o")
    g = _dev(dBout, torch.float32, (E, 3, N), "dBout")
    dB = torch.empty_like(b)
    deta = torch.empty(E, dtype=torch.float32, device=b.device)
    _check(lib().tsr_fresnel_output_backward(E, _ptr(e), N, _ptr(c), _ptr(b), _ptr(g), _ptr(dB), _ptr(deta),
                                             _stream()))
    return dB, deta


def visibility_transfer(pos: torch.Tensor, normals: torch.Tensor, tris: torch.Tensor, J: int, S: int = 256,
                        eta: float = 0.0, eps: float = 1e-3) -> torch.Tensor:
    """tsr_visibility_transfer: self-shadowed T [J][N] for positions/normals [3][N] and triangles [F][3] int32."""
    N = pos.shape[1]
    p = _dev(pos, torch.float32, (3, N), "pos")
    n = _dev(normals, torch.float32, (3, N), "normals")
    t = _dev(tris, torch.int32, (tris.shape[0], 3), "tris")
    T = torch.empty((J, N), dtype=torch.float32, device=p.device)
    _check(lib().tsr_visibility_transfer(N, _ptr(p), _ptr(n), t.shape[0], _ptr(t), J, S, float(eta), float(eps),
                                         _ptr(T), _stream()))
    return T


def sh_transfer(normals: torch.Tensor, J: int, eta: float = 1.0) -> torch.Tensor:
    """tsr_sh_transfer: T [J][N] for unit normals [3][N] with the incident Fresnel factor at eta folded in."""
    N = normals.shape[1]
    n = _dev(normals, torch.float32, (3, N), "normals")
    T = torch.empty((J, N), dtype=torch.float32, device=n.device)
    _check(lib().tsr_sh_transfer(N, _ptr(n), J, float(eta), _ptr(T), _stream()))
    return T


# ---------------------------------------------------------------- relight
def relight(comp: Compressed, g: torch.Tensor, light: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """tsr_relight: g [E][3][K] FP32, light [J] FP32 -> B [E][3][N]."""
    E = g.shape[0]
    gg = _dev(g, torch.float32, (E, 3, comp.K), "g")
    ll = _dev(light, torch.float32, (comp.J,), "light")
    B = out if out is not None else torch.empty((E, 3, comp.n), dtype=torch.float32, device=gg.device)
    _check(lib().tsr_relight(comp.handle, E, _ptr(gg), _ptr(ll), _ptr(B), _stream()))
    return B


def relight_many(comps, g: torch.Tensor, light: torch.Tensor, out: torch.Tensor | None = None):
    """tsr_relight_many: g [n_copy][E][3][K] FP32, light [J] -> list of B_i [E][3][N_i], views of one
    buffer (the copies' blocks back to back, returned as `out` when given)."""
    comps = list(comps)
    n = len(comps)
    if n == 0:
        return []
    K, J = comps[0].K, comps[0].J
    E = g.shape[1] if g.dim() == 4 else 0
    gg = _dev(g, torch.float32, (n, E, 3, K), "g")
    ll = _dev(light, torch.float32, (J,), "light")
    sizes = [E * 3 * c.n for c in comps]
    total = sum(sizes)
    if out is None:
        out = torch.empty(total, device=gg.device, dtype=torch.float32)
    out = _dev(out, torch.float32, (total,), "out")
    handles = (ctypes.c_void_p * n)(*[c.handle.value for c in comps])
    _check(lib().tsr_relight_many(n, ctypes.cast(handles, ctypes.c_void_p), E, _ptr(gg), _ptr(ll), _ptr(out),
                                  _stream()))
    views, o = [], 0
    for c, sz in zip(comps, sizes):
        views.append(out[o:o + sz].view(E, 3, c.n))
        o += sz
    return views


def relight_backward(comp: Compressed, g: torch.Tensor, light: torch.Tensor, dLdB: torch.Tensor):
    """tsr_relight_backward: returns (dg [E][3][K], dl [J])."""
    E = g.shape[0]
    gg = _dev(g, torch.float32, (E, 3, comp.K), "g")
    ll = _dev(light, torch.float32, (comp.J,), "light")
    db = _dev(dLdB, torch.float32, (E, 3, comp.n), "dLdB")
    dg = torch.empty_like(gg)
    dl = torch.empty_like(ll)
    _check(lib().tsr_relight_backward(comp.handle, E, _ptr(gg), _ptr(ll), _ptr(db), _ptr(dg), _ptr(dl), _stream()))
    return dg, dl


def relight_noalloc(comp: Compressed, g: torch.Tensor, light: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
    """tsr_relight_noalloc: tsr_relight into a caller-provided B [E][3][N], with the
    library's fixed device scratch instead of an allocation (see include/tsr.h)."""
    E = g.shape[0]
    gg = _dev(g, torch.float32, (E, 3, comp.K), "g")
    ll = _dev(light, torch.float32, (comp.J,), "light")
    _dev(out, torch.float32, (E, 3, comp.n), "out")
    if not out.is_contiguous():
        raise ValueError("out must be contiguous")
    _check(lib().tsr_relight_noalloc(comp.handle, E, _ptr(gg), _ptr(ll), _ptr(out), _stream()))
    return out
