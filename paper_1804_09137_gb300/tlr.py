"""Thin Python binding of libtlr (include/tlr.h): argument marshalling only.

Every step of the likelihood runs in the CUDA library; this module passes
device pointers of float64 torch tensors and the current CUDA stream.  It
fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtlr.so")

TLR_OK, TLR_ERR_NOT_SPD, TLR_ERR_RANK_CAP, TLR_ERR_OOM, TLR_ERR_CUDA, TLR_ERR_TIMEOUT, TLR_ERR_STATE, \
    TLR_ERR_NUMERIC = range(8)
ERR_NAMES = {1: "not SPD", 2: "rank cap exceeded", 3: "out of memory", 4: "CUDA error", 5: "device wait timed out",
             6: "call out of order", 7: "non-finite value in a recompression"}


class TlrOpts(C.Structure):
    _fields_ = [("nb", C.c_int), ("eps", C.c_double), ("rank_cap", C.c_int), ("truncate_at_cap", C.c_int),
                ("order", C.c_int), ("dense_rank", C.c_int), ("inv_scale", C.c_double), ("metric", C.c_int),
                ("radius", C.c_double), ("precision", C.c_int)]


class TlrTheta(C.Structure):
    _fields_ = [("sigma2", C.c_double), ("beta", C.c_double), ("nu", C.c_double)]


class TlrError(RuntimeError):
    def __init__(self, name, code, info=None):
        self.code = code
        self.info = info
        what = ERR_NAMES.get(code, f"invalid argument {-code}" if code < 0 else f"error {code}")
        super().__init__(f"{name}: {what}" + (f" (info {info})" if info is not None else ""))


_lib = None

EXPORTS = ["tlr_create", "tlr_destroy", "tlr_matern_generate", "tlr_compress", "tlr_potrf", "tlr_loglik",
           "tlr_loglik_grad", "tlr_predict", "tlr_sample", "tlr_status", "tlr_rank_stats", "tlr_shape",
           "tlr_get_tile", "tlr_get_perm", "tlr_tile_counts", "tlr_launch_count", "tlr_profile", "tlr_inverse_stats", "tlr_memory", "tlr_profile_phases", "tlr_loglik_dense_noalloc",
           "tlr_loglik_grad_batched", "tlr_predict_var",
           "tlr_profile_read", "tlr_gemm_tc", "tlr_profile_read_tc"]


def lib():
    """Load libtlr.so (built by paper_1804_09137_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build() first")
    L = C.CDLL(LIB_PATH)
    vp, i64, d = C.c_void_p, C.c_int64, C.c_double
    L.tlr_create.argtypes = [i64, vp, vp, C.POINTER(TlrOpts), vp, C.POINTER(vp)]
    L.tlr_destroy.argtypes = [vp]
    L.tlr_matern_generate.argtypes = [vp, TlrTheta, vp]
    L.tlr_compress.argtypes = [vp, d, vp]
    L.tlr_potrf.argtypes = [vp, vp]
    L.tlr_loglik.argtypes = [vp, vp, vp, vp]
    L.tlr_loglik_grad.argtypes = [vp, vp, vp, vp, vp]
    L.tlr_predict.argtypes = [vp, vp, i64, vp, vp, vp, vp]
    L.tlr_predict_var.argtypes = [vp, i64, vp, vp, vp, vp]
    L.tlr_sample.argtypes = [vp, vp, vp, vp]
    L.tlr_status.argtypes = [vp, C.POINTER(i64)]
    L.tlr_rank_stats.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(d), C.POINTER(C.c_int), C.POINTER(i64)]
    L.tlr_shape.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.tlr_get_tile.argtypes = [vp, C.c_int, C.c_int, vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_int), vp]
    L.tlr_get_perm.argtypes = [vp, vp, vp]
    L.tlr_tile_counts.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    L.tlr_launch_count.argtypes = [C.POINTER(i64)]
    L.tlr_inverse_stats.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(d), C.POINTER(C.c_int), C.POINTER(i64)]
    L.tlr_memory.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    L.tlr_profile.argtypes = [C.c_int]
    L.tlr_loglik_grad_batched.argtypes = [C.c_int, C.POINTER(i64), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                          C.POINTER(TlrTheta), C.POINTER(TlrOpts), vp, vp, C.POINTER(C.c_int),
                                          C.c_int, vp]
    L.tlr_loglik_dense_noalloc.argtypes = [i64, vp, vp, vp, TlrTheta, vp, vp]
    L.tlr_profile_phases.argtypes = [C.c_char_p, i64]
    L.tlr_profile_read.argtypes = [C.POINTER(i64), C.POINTER(d), C.POINTER(d)]
    L.tlr_profile_read_tc.argtypes = [C.POINTER(i64), C.POINTER(d), C.POINTER(d)]
    ci = C.c_int
    L.tlr_gemm_tc.argtypes = [ci, ci, ci, vp, ci, ci, vp, ci, ci, vp, ci, d, d, ci, vp]
    for name in EXPORTS:
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(t: torch.Tensor):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(name, rc):
    if rc != TLR_OK:
        raise TlrError(name, rc)


class Handle:
    """Owns one tlr_handle (tile storage on the current CUDA device)."""

    def __init__(self, x: torch.Tensor, y: torch.Tensor, nb: int, eps: float = 1e-9, rank_cap: int = 0,
                 truncate_at_cap: bool = False, order: bool = True, dense_rank: int = 0, inv_scale: float = 0.0,
                 radius: float | None = None, precision: int = 0):
        """radius: None for Euclidean distances; a sphere radius for great-circle distances (eq. 6) with
        x = longitude and y = latitude in degrees.  precision: 0 tensor-core contractions on 6 bf16 slices
        (default), 1 double-float on the CUDA cores, 4..6 tensor cores with that many slices."""
        L = lib()
        self._opts = TlrOpts(int(nb), float(eps), int(rank_cap), int(bool(truncate_at_cap)), int(bool(order)),
                             int(dense_rank), float(inv_scale), 0 if radius is None else 1,
                             0.0 if radius is None else float(radius), int(precision))
        h = C.c_void_p()
        _check("tlr_create", L.tlr_create(int(x.numel()), _ptr(x), _ptr(y), C.byref(self._opts), _stream(),
                                          C.byref(h)))
        self._h = h
        self.n = int(x.numel())
        self.eps = float(eps)
        self.dev = x.device
        nt, nbo = C.c_int(), C.c_int()
        L.tlr_shape(h, C.byref(nt), C.byref(nbo))
        self.nt, self.nb = nt.value, nbo.value

    def close(self):
        if getattr(self, "_h", None):
            lib().tlr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # pipeline -----------------------------------------------------------
    def matern_generate(self, theta):
        s2, b, nu = (float(v) for v in theta)
        _check("tlr_matern_generate", lib().tlr_matern_generate(self._h, TlrTheta(s2, b, nu), _stream()))

    def compress(self, eps=None):
        _check("tlr_compress", lib().tlr_compress(self._h, float(self.eps if eps is None else eps), _stream()))

    def potrf(self):
        _check("tlr_potrf", lib().tlr_potrf(self._h, _stream()))

    def factor(self, theta, eps=None):
        self.matern_generate(theta)
        self.compress(eps)
        self.potrf()

    def loglik(self, z: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        out = torch.empty(3, dtype=torch.float64, device=self.dev) if out is None else out
        _check("tlr_loglik", lib().tlr_loglik(self._h, _ptr(z), _ptr(out), _stream()))
        return out

    def loglik_grad(self, z: torch.Tensor, ll=None, grad=None):
        ll = torch.empty(1, dtype=torch.float64, device=self.dev) if ll is None else ll
        grad = torch.empty(3, dtype=torch.float64, device=self.dev) if grad is None else grad
        _check("tlr_loglik_grad", lib().tlr_loglik_grad(self._h, _ptr(z), _ptr(ll), _ptr(grad), _stream()))
        return ll, grad

    def predict(self, z_obs, x_new, y_new, out=None):
        m = int(x_new.numel())
        out = torch.empty(m, dtype=torch.float64, device=self.dev) if out is None else out
        _check("tlr_predict", lib().tlr_predict(self._h, _ptr(z_obs), m, _ptr(x_new), _ptr(y_new), _ptr(out),
                                                _stream()))
        return out

    def predict_var(self, x_new, y_new, out=None):
        """Prediction variance sigma2 - Sigma_12 Sigma_22^{-1} Sigma_21 (diagonal) at the new points."""
        m = int(x_new.numel())
        out = torch.empty(m, dtype=torch.float64, device=self.dev) if out is None else out
        _check("tlr_predict_var", lib().tlr_predict_var(self._h, m, _ptr(x_new), _ptr(y_new), _ptr(out), _stream()))
        return out

    def sample(self, e, out=None):
        out = torch.empty_like(e) if out is None else out
        _check("tlr_sample", lib().tlr_sample(self._h, _ptr(e), _ptr(out), _stream()))
        return out

    def status(self):
        info = C.c_int64()
        rc = lib().tlr_status(self._h, C.byref(info))
        return rc, info.value

    def check(self):
        rc, info = self.status()
        if rc != TLR_OK:
            raise TlrError("device", rc, info)

    def get_tile(self, i, j):
        """Tile (i, j) in sorted point order: (A, None) if dense (or diagonal), else (U, V)."""
        U = torch.zeros(self.nb * self.nb, dtype=torch.float64, device=self.dev)
        V = torch.zeros_like(U)
        k, dense = C.c_int(), C.c_int()
        _check("tlr_get_tile", lib().tlr_get_tile(self._h, int(i), int(j), _ptr(U), _ptr(V), C.byref(k),
                                                  C.byref(dense), _stream()))
        if dense.value:
            return U.view(self.nb, self.nb).T, None
        kk = k.value
        return U[: self.nb * kk].view(kk, self.nb).T, V[: self.nb * kk].view(kk, self.nb).T

    def tile_counts(self):
        a, b = C.c_int64(), C.c_int64()
        _check("tlr_tile_counts", lib().tlr_tile_counts(self._h, C.byref(a), C.byref(b)))
        return {"lowrank": a.value, "dense": b.value}

    def inverse_stats(self):
        kmin, kmax, kmean, nd = C.c_int(), C.c_int(), C.c_double(), C.c_int64()
        _check("tlr_inverse_stats", lib().tlr_inverse_stats(self._h, C.byref(kmin), C.byref(kmean), C.byref(kmax),
                                                            C.byref(nd)))
        return {"kmin": kmin.value, "kmean": kmean.value, "kmax": kmax.value, "dense": nd.value}

    def memory(self):
        """Device bytes held by the handle: total, low-rank arenas, their used part, workspaces."""
        v = [C.c_int64() for _ in range(4)]
        _check("tlr_memory", lib().tlr_memory(self._h, *[C.byref(x) for x in v]))
        return dict(zip(("total", "arenas", "arena_used", "workspace"), (x.value for x in v)))

    def get_perm(self):
        p = torch.zeros(self.n, dtype=torch.int32, device=self.dev)
        _check("tlr_get_perm", lib().tlr_get_perm(self._h, C.c_void_p(p.data_ptr()), _stream()))
        return p

    def rank_stats(self):
        kmin, kmax, kmean, nbytes = C.c_int(), C.c_int(), C.c_double(), C.c_int64()
        _check("tlr_rank_stats", lib().tlr_rank_stats(self._h, C.byref(kmin), C.byref(kmean), C.byref(kmax),
                                                      C.byref(nbytes)))
        return {"kmin": kmin.value, "kmean": kmean.value, "kmax": kmax.value, "bytes": nbytes.value}


def gemm_tc(A: torch.Tensor, B: torch.Tensor, Cm: torch.Tensor, tA=False, tB=False, alpha=1.0, beta=0.0,
            slices=6):
    """Cm = beta Cm + alpha op(A) op(B) on the tensor cores.  A, B, Cm: column-major (Fortran-ordered: .T is
    contiguous) float64 CUDA tensors with BLAS shapes (op(A) m x k, op(B) k x n, Cm m x n)."""
    m, n = Cm.shape
    k = A.shape[0] if tA else A.shape[1]
    for t in (A, B, Cm):
        if not (t.is_cuda and t.dtype == torch.float64 and t.T.is_contiguous()):
            raise ValueError("expected column-major float64 CUDA tensors")
    vp = lambda t: C.c_void_p(t.data_ptr())
    _check("tlr_gemm_tc", lib().tlr_gemm_tc(m, n, k, vp(A), A.shape[0], int(tA), vp(B), B.shape[0], int(tB), vp(Cm),
                                            Cm.shape[0], float(alpha), float(beta), int(slices), _stream()))
    return Cm


def launch_count() -> int:
    c = C.c_int64()
    _check("tlr_launch_count", lib().tlr_launch_count(C.byref(c)))
    return c.value


def profile(enable: bool):
    _check("tlr_profile", lib().tlr_profile(int(bool(enable))))


def profile_read():
    n, ms, fl = C.c_int64(), C.c_double(), C.c_double()
    _check("tlr_profile_read", lib().tlr_profile_read(C.byref(n), C.byref(ms), C.byref(fl)))
    return {"launches": n.value, "ms": ms.value, "flops": fl.value}


def profile_read_tc():
    """Tensor-core GEMM launches, their device time (ms) and bf16 MMA flops since profile(True)."""
    n, ms, fl = C.c_int64(), C.c_double(), C.c_double()
    _check("tlr_profile_read_tc", lib().tlr_profile_read_tc(C.byref(n), C.byref(ms), C.byref(fl)))
    return {"launches": n.value, "ms": ms.value, "flops": fl.value}


def profile_phases() -> dict:
    import json

    buf = C.create_string_buffer(1 << 16)
    _check("tlr_profile_phases", lib().tlr_profile_phases(buf, len(buf)))
    return json.loads(buf.value.decode())


def loglik_grad_batched(xs, ys, zs, thetas, opts, nworkers: int = 8):
    """l and dl/dtheta of independent regions (lists of float64 CUDA tensors, thetas, TlrOpts).

    Returns (ll (R,), grad (R, 3), status list)."""
    R = len(xs)
    dev = xs[0].device
    n = (C.c_int64 * R)(*[int(t.numel()) for t in xs])
    px = (C.c_void_p * R)(*[_ptr(t).value for t in xs])
    py = (C.c_void_p * R)(*[_ptr(t).value for t in ys])
    pz = (C.c_void_p * R)(*[_ptr(t).value for t in zs])
    th = (TlrTheta * R)(*[TlrTheta(*[float(v) for v in t]) for t in thetas])
    op = (TlrOpts * R)(*opts)
    ll = torch.empty(R, dtype=torch.float64, device=dev)
    grad = torch.empty(R, 3, dtype=torch.float64, device=dev)
    st = (C.c_int * R)()
    _check("tlr_loglik_grad_batched", lib().tlr_loglik_grad_batched(R, n, px, py, pz, th, op, _ptr(ll), _ptr(grad),
                                                                    st, int(nworkers), _stream()))
    return ll, grad, list(st)
