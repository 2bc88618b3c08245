"""Thin ctypes binding of the sm_103a TDDFT-ris library (include/ris.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Arrays may be numpy arrays (host) or CUDA torch tensors (device);
the library tells them apart.  There is no CPU fallback: if the library
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libris.so")

RIS_OK = 0
STATUS = {0: "RIS_OK", -1: "RIS_ERR_ARG", -2: "RIS_ERR_OOM", -3: "RIS_ERR_METRIC_NOT_PD",
          -4: "RIS_ERR_NOT_CONVERGED", -5: "RIS_ERR_CUDA", -6: "RIS_ERR_TIMEOUT",
          -7: "RIS_ERR_STATE", -8: "RIS_ERR_DEGENERATE"}
FP64, MIXED = 0, 1

EXPORTS = ["ris_options_default", "ris_create", "ris_build_aux", "ris_build_B", "ris_excite",
           "ris_apply", "ris_excite_guess", "ris_trim", "ris_zvector", "ris_phase_align", "ris_time_coupling", "ris_get_mo_window", "ris_debug_gemm_tf32x3", "ris_debug_gemm_f64emu", "ris_debug_gemm_ff", "ris_debug_sym_eig", "ris_debug_sym_eig_f32", "ris_debug_dgemm",
           "ris_gemm_tf32x3_noalloc", "ris_debug_alloc_count", "ris_debug_peak_probe",
           "ris_gradient", "ris_nac", "ris_get_dims", "ris_get_stats", "ris_debug_boys",
           "ris_last_error", "ris_destroy"]


class RisError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("rpa", ctypes.c_int), ("cx", ctypes.c_double),
                ("conv_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("max_subspace", ctypes.c_int), ("screen_thr", ctypes.c_double),
                ("mem_budget", ctypes.c_size_t), ("occ_block", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("profile", ctypes.c_int), ("mixed_tol", ctypes.c_double), ("refine", ctypes.c_int),
                ("precond", ctypes.c_int), ("mo_window", ctypes.c_double),
                ("deriv_prefetch", ctypes.c_int), ("emu_f64", ctypes.c_int),
                ("eig_fp32", ctypes.c_int), ("stream", ctypes.c_int), ("stream_block", ctypes.c_int),
                ("subspace_ff", ctypes.c_int)]


class Shell(ctypes.Structure):
    _fields_ = [("atom", ctypes.c_int), ("l", ctypes.c_int), ("exponent", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libris.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i, d = ctypes.c_int, ctypes.c_double
    L.ris_options_default.argtypes = [ctypes.POINTER(Options)]
    L.ris_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Options)]
    L.ris_build_aux.argtypes = [P, i, P, i, P, i, P, i, P]
    L.ris_build_B.argtypes = [P, i, i, i, P, P]
    L.ris_excite.argtypes = [P, i, P, P, P]
    L.ris_excite_guess.argtypes = [P, i, P, P, P, P]
    L.ris_trim.argtypes = [P]
    L.ris_zvector.argtypes = [P, i, P, P]
    L.ris_phase_align.argtypes = [P, i, P, P, P]
    L.ris_time_coupling.argtypes = [P, i, P, P, P]
    L.ris_get_mo_window.argtypes = [P, P, P, P]
    L.ris_apply.argtypes = [P, i, P, P, P]
    L.ris_gradient.argtypes = [P, i, P, i, P, P, P]
    L.ris_nac.argtypes = [P, i, P, i, P, P, P, P, P]
    L.ris_get_dims.argtypes = [P] + [ctypes.POINTER(i)] * 6
    L.ris_get_stats.argtypes = [P, ctypes.POINTER(d), i]
    L.ris_debug_boys.argtypes = [i, P, P, P]
    L.ris_debug_gemm_tf32x3.argtypes = [i, i, i, P, P, P]
    L.ris_debug_gemm_f64emu.argtypes = [i, i, i, P, P, P]
    L.ris_debug_gemm_ff.argtypes = [i, i, i, i, ctypes.c_double, P, P, ctypes.c_double, P,
                                    ctypes.POINTER(i)]
    L.ris_debug_sym_eig.argtypes = [i, i, P, P, P]
    L.ris_debug_sym_eig_f32.argtypes = [i, i, P, P, P]
    d = ctypes.c_double
    L.ris_debug_dgemm.argtypes = [i, i, i, i, i, d, P, i, P, i, d, P, i]
    L.ris_gemm_tf32x3_noalloc.argtypes = [i, i, i, P, P, P, P]
    L.ris_debug_alloc_count.argtypes = []
    L.ris_debug_peak_probe.argtypes = [i, i, P, P]
    L.ris_last_error.argtypes = [P]
    L.ris_last_error.restype = ctypes.c_char_p
    L.ris_destroy.argtypes = [P]
    for f in EXPORTS:
        if f not in ("ris_last_error", "ris_destroy", "ris_debug_alloc_count"):
            getattr(L, f).restype = ctypes.c_int
    L.ris_debug_alloc_count.restype = ctypes.c_longlong
    L.ris_destroy.restype = None
    _lib = L
    return L


def _ptr(a) -> Optional[int]:
    """Raw address of a numpy array or torch tensor (contiguous, float64/int32)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensors must be contiguous"
        return a.data_ptr()
    raise TypeError(type(a))


def _shells(arr) -> ctypes.Array:
    if isinstance(arr, ctypes.Array):
        return arr
    n = len(arr)
    out = (Shell * n)()
    for k in range(n):
        out[k].atom = int(arr["atom"][k])
        out[k].l = int(arr["l"][k])
        out[k].exponent = float(arr["exp"][k])
    return out


def options(**kw) -> Options:
    o = Options()
    load().ris_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Context:
    """One ris_ctx (one CUDA stream).  Methods mirror the C ABI."""

    def __init__(self, **opts):
        self.L = load()
        self.opt = options(**opts)
        h = ctypes.c_void_p()
        self._check(self.L.ris_create(ctypes.byref(h), ctypes.byref(self.opt)), None)
        self.h = h
        self.natm = self.nocc = self.nvir = 0

    def _check(self, st: int, h=...):
        if st != RIS_OK:
            hh = self.h if h is ... else h
            msg = self.L.ris_last_error(hh).decode() if hh else ""
            raise RisError(st, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.ris_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_aux(self, coords, shells, aux_j, aux_k):
        c = np.ascontiguousarray(coords, dtype=np.float64) if isinstance(coords, np.ndarray) else coords
        s, j, k = _shells(shells), _shells(aux_j), _shells(aux_k)
        self.natm = int(c.shape[0])
        self._check(self.L.ris_build_aux(self.h, self.natm, _ptr(c), len(s), ctypes.addressof(s),
                                         len(j), ctypes.addressof(j), len(k), ctypes.addressof(k)))

    def build_B(self, C, mo_energy, nocc: int):
        if isinstance(C, np.ndarray):
            C = np.ascontiguousarray(C, dtype=np.float64)
            mo_energy = np.ascontiguousarray(mo_energy, dtype=np.float64)
        nao, nmo = C.shape
        self._check(self.L.ris_build_B(self.h, nao, nmo, int(nocc), _ptr(C), _ptr(mo_energy)))
        self.first_occ, self.nocc, self.nvir = self.mo_window()

    def mo_window(self):
        """(first active occupied MO, active nocc, active nvir) after build_B."""
        v = [ctypes.c_int() for _ in range(3)]
        self._check(self.L.ris_get_mo_window(self.h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def excite(self, nstates: int, out=None):
        """Returns (omega, X[, Y]) as numpy arrays, or fills `out` (omega, X, Y)
        tensors/arrays in place (host or device)."""
        rpa = bool(self.opt.rpa)
        if out is None:
            om = np.zeros(nstates)
            X = np.zeros((nstates, self.nocc, self.nvir))
            Y = np.zeros_like(X) if rpa else None
        else:
            om, X, Y = out
        self._check(self.L.ris_excite(self.h, int(nstates), _ptr(om), _ptr(X), _ptr(Y)))
        return (om, X, Y) if rpa else (om, X)

    def excite_guess(self, nstates: int, guess, out=None):
        """ris_excite seeded with guess vectors [nstates][nocc][nvir]."""
        rpa = bool(self.opt.rpa)
        if out is None:
            om = np.zeros(nstates)
            X = np.zeros((nstates, self.nocc, self.nvir))
            Y = np.zeros_like(X) if rpa else None
        else:
            om, X, Y = out
        self._check(self.L.ris_excite_guess(self.h, int(nstates), _ptr(guess), _ptr(om), _ptr(X),
                                            _ptr(Y)))
        return (om, X, Y) if rpa else (om, X)

    def apply(self, X, out=None, out2=None):
        """TDA: A X.  RPA: ((A+B) X, (A-B) X)."""
        rpa = bool(self.opt.rpa)
        if out is None:
            out = np.zeros_like(X)
            out2 = np.zeros_like(X) if rpa else None
        self._check(self.L.ris_apply(self.h, int(X.shape[0]), _ptr(X), _ptr(out), _ptr(out2)))
        return (out, out2) if rpa else out

    def gradient(self, states: Sequence[int], X=None, Y=None, out=None):
        st = np.ascontiguousarray(states, dtype=np.int32)
        nx = 0 if X is None else int(X.shape[0])
        g = np.zeros((len(st), self.natm, 3)) if out is None else out
        self._check(self.L.ris_gradient(self.h, len(st), _ptr(st), nx, _ptr(X), _ptr(Y), _ptr(g)))
        return g

    def nac(self, pairs, X=None, Y=None, omega=None, out=None, numerator=None):
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        nx = 0 if X is None else int(X.shape[0])
        n = np.zeros((len(pr), self.natm, 3)) if out is None else out
        self._check(self.L.ris_nac(self.h, len(pr), _ptr(pr), nx, _ptr(X), _ptr(Y), _ptr(omega),
                                   _ptr(n), _ptr(numerator)))
        return n

    def zvector(self, rhs, out=None):
        """Solve (A+B) Z = rhs (ris_zvector); rhs [n][nocc][nvir], host or device."""
        Z = np.zeros(rhs.shape) if out is None else out
        self._check(self.L.ris_zvector(self.h, int(rhs.shape[0]), _ptr(rhs), _ptr(Z)))
        return Z

    def phase_align(self, X_prev, X_out=None):
        """Align the current states' phases with X_prev (ris_phase_align); returns the signs."""
        ns = int(X_prev.shape[0])
        sign = np.zeros(ns, dtype=np.int32)
        self._check(self.L.ris_phase_align(self.h, ns, _ptr(X_prev), _ptr(sign), _ptr(X_out)))
        return sign

    def time_coupling(self, nac, velocity, out=None):
        """T_IJ = d_IJ . v for each coupling (ris_time_coupling); nac
        [npair][natm][3], velocity [natm][3], host or device."""
        npair = int(nac.shape[0])
        T = np.zeros(npair) if out is None else out
        if isinstance(nac, np.ndarray):
            nac = np.ascontiguousarray(nac, dtype=np.float64)
        if isinstance(velocity, np.ndarray):
            velocity = np.ascontiguousarray(velocity, dtype=np.float64)
        self._check(self.L.ris_time_coupling(self.h, npair, _ptr(nac), _ptr(velocity), _ptr(T)))
        return T

    def trim(self):
        """Release every device buffer of the context (ris_trim)."""
        self._check(self.L.ris_trim(self.h))

    def dims(self):
        v = [ctypes.c_int() for _ in range(6)]
        self._check(self.L.ris_get_dims(self.h, *[ctypes.byref(x) for x in v]))
        keys = ["natm", "nao", "nocc", "nauxJ", "nauxK", "npairs"]
        return {k: x.value for k, x in zip(keys, v)}

    STAT_KEYS = {0: "aux_ms", 1: "B_ms", 2: "excite_ms", 3: "deriv_ms", 4: "n_products",
                 5: "n_iter", 15: "launches", 16: "gemm_ms", 17: "gemm_flops", 18: "int3c_ms",
                 19: "int3c_triples", 20: "int3c_deriv_ms", 21: "int3c_deriv_triples",
                 22: "contract_ms", 23: "contract_bytes", 24: "eig_ms", 25: "eig_calls",
                 26: "tc_gemm_ms", 27: "tc_gemm_flops", 6: "refine_products",
                 28: "bytes_held", 29: "bytes_peak", 7: "residual_max", 30: "emu_gemm_ms",
                 31: "emu_gemm_flops", 32: "ff_gemm_ms", 33: "ff_gemm_flops"}

    def stats(self):
        out = (ctypes.c_double * 34)()
        self._check(self.L.ris_get_stats(self.h, out, 34))
        return {k: out[i] for i, k in self.STAT_KEYS.items()}


def debug_boys(m, T):
    """F_m(T) from the library's device Boys function (torch CUDA tensors)."""
    import torch
    m_t = torch.as_tensor(np.asarray(m, dtype=np.int32), device="cuda")
    T_t = torch.as_tensor(np.asarray(T, dtype=np.float64), device="cuda")
    out = torch.empty_like(T_t)
    st = load().ris_debug_boys(int(T_t.numel()), m_t.data_ptr(), T_t.data_ptr(), out.data_ptr())
    if st != 0:
        raise RisError(st, "ris_debug_boys failed")
    return out.cpu().numpy()


def debug_gemm_tf32x3(A, B):
    """C = A B^T through the library's 3xTF32 tcgen05 GEMM (numpy in/out)."""
    import torch
    A_t = torch.as_tensor(np.ascontiguousarray(A, dtype=np.float64), device="cuda")
    B_t = torch.as_tensor(np.ascontiguousarray(B, dtype=np.float64), device="cuda")
    M, K = A_t.shape
    N = B_t.shape[0]
    C_t = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    st = load().ris_debug_gemm_tf32x3(M, N, K, A_t.data_ptr(), B_t.data_ptr(), C_t.data_ptr())
    torch.cuda.synchronize()
    if st != 0:
        raise RisError(st, "ris_debug_gemm_tf32x3 failed")
    return C_t.cpu().numpy()


def debug_gemm_f64emu(A, B):
    """C = A B^T through the library's FP64-emulating tensor-core GEMM
    (numpy in/out)."""
    import torch
    A_t = torch.as_tensor(np.ascontiguousarray(A, dtype=np.float64), device="cuda")
    B_t = torch.as_tensor(np.ascontiguousarray(B, dtype=np.float64), device="cuda")
    M, K = A_t.shape
    N = B_t.shape[0]
    C_t = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    st = load().ris_debug_gemm_f64emu(M, N, K, A_t.data_ptr(), B_t.data_ptr(), C_t.data_ptr())
    torch.cuda.synchronize()
    if st != 0:
        raise RisError(st, "ris_debug_gemm_f64emu failed")
    return C_t.cpu().numpy()


def debug_gemm_ff(A, B, transB=True, alpha=1.0, beta=0.0, C=None):
    """C = alpha A op(B) + beta C through the library's double-FP32 GEMM
    (numpy in/out); op(B) = B^T (B [N][K]) when transB, else B ([K][N]).
    Returns (C, kind) with kind 1 (long-K kernel) or 2 (short-K kernel)."""
    import torch
    A_t = torch.as_tensor(np.ascontiguousarray(A, dtype=np.float64), device="cuda")
    B_t = torch.as_tensor(np.ascontiguousarray(B, dtype=np.float64), device="cuda")
    M, K = A_t.shape
    N = B_t.shape[0] if transB else B_t.shape[1]
    if (B_t.shape[1] if transB else B_t.shape[0]) != K:
        raise ValueError("debug_gemm_ff: inner dimensions differ")
    if C is None:
        C_t = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    else:
        C_t = torch.as_tensor(np.ascontiguousarray(C, dtype=np.float64), device="cuda").clone()
    kind = ctypes.c_int(-1)
    st = load().ris_debug_gemm_ff(int(bool(transB)), M, N, K, float(alpha), A_t.data_ptr(),
                                  B_t.data_ptr(), float(beta), C_t.data_ptr(), ctypes.byref(kind))
    torch.cuda.synchronize()
    if st != 0:
        raise RisError(st, f"ris_debug_gemm_ff failed (shape kind {kind.value})")
    return C_t.cpu().numpy(), kind.value


def gemm_tf32x3_noalloc(A_t, B_t, C_t, stream=None) -> int:
    """C_t = A_t B_t^T through the allocation-free entry point; returns the
    status code.  A_t [M][K], B_t [N][K], C_t [M][N]: contiguous float64 CUDA
    tensors on the current device (ValueError otherwise).  stream: a raw
    cudaStream_t, default torch's current stream on that device."""
    import torch
    dev = torch.cuda.current_device()
    for name, t in (("A", A_t), ("B", B_t), ("C", C_t)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
            raise ValueError(f"{name} must be a float64 CUDA tensor")
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
        if t.dim() != 2 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous matrix")
    M, K = A_t.shape
    N = B_t.shape[0]
    if B_t.shape[1] != K or tuple(C_t.shape) != (M, N):
        raise ValueError(f"shapes A {tuple(A_t.shape)}, B {tuple(B_t.shape)}, C {tuple(C_t.shape)} "
                         "do not form C = A B^T")
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    return load().ris_gemm_tf32x3_noalloc(int(M), int(N), int(K), A_t.data_ptr(), B_t.data_ptr(),
                                          C_t.data_ptr(), stream)


PROBE_KINDS = {"fp64_fma": 0, "fp32_fma": 1, "fp64_mma_sync": 2, "tf32_tcgen05": 3,
               "f16_tcgen05": 4}


def debug_peak_probe(kind: str, reps: int = 3):
    """Measured rate (TFLOP/s, ms of the best run) of one arithmetic pipe of
    the current device (ris_debug_peak_probe)."""
    r = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    st = load().ris_debug_peak_probe(PROBE_KINDS[kind], int(reps), ctypes.addressof(r),
                                     ctypes.addressof(ms))
    if st != 0:
        raise RisError(st, f"ris_debug_peak_probe({kind}) failed")
    return r.value, ms.value


def debug_alloc_count() -> int:
    """Device allocations the library has made since it was loaded."""
    return int(load().ris_debug_alloc_count())


def debug_dgemm(A, B, C, transA=False, transB=False, alpha=1.0, beta=0.0):
    """C = alpha op(A) op(B) + beta C with the library's FP64 GEMM (numpy in, numpy out)."""
    import torch
    A_t = torch.as_tensor(np.ascontiguousarray(A, dtype=np.float64), device="cuda")
    B_t = torch.as_tensor(np.ascontiguousarray(B, dtype=np.float64), device="cuda")
    C_t = torch.as_tensor(np.ascontiguousarray(C, dtype=np.float64), device="cuda")
    m = A_t.shape[1] if transA else A_t.shape[0]
    k = A_t.shape[0] if transA else A_t.shape[1]
    n = B_t.shape[0] if transB else B_t.shape[1]
    st = load().ris_debug_dgemm(int(transA), int(transB), m, n, k, float(alpha), A_t.data_ptr(),
                                A_t.shape[1], B_t.data_ptr(), B_t.shape[1], float(beta),
                                C_t.data_ptr(), C_t.shape[1])
    if st != 0:
        raise RisError(st, "ris_debug_dgemm failed")
    return C_t.cpu().numpy()


def debug_sym_eig(H, k, fp32=False):
    """Lowest k eigenpairs of symmetric H via the device subspace eigensolver
    (fp32: its FP32 form with FP64 Rayleigh quotients)."""
    import torch
    H_t = torch.as_tensor(np.ascontiguousarray(H, dtype=np.float64), device="cuda")
    m = H_t.shape[0]
    w = torch.zeros(k, dtype=torch.float64, device="cuda")
    V = torch.zeros((k, m), dtype=torch.float64, device="cuda")
    fn = load().ris_debug_sym_eig_f32 if fp32 else load().ris_debug_sym_eig
    st = fn(int(m), int(k), H_t.data_ptr(), w.data_ptr(), V.data_ptr())
    if st != 0:
        raise RisError(st, "ris_debug_sym_eig failed")
    return w.cpu().numpy(), V.cpu().numpy()
