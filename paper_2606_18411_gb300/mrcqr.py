"""Python binding of the MRCQR C ABI: argument marshalling only.

Matrices are torch CUDA float64 tensors in column-major layout, i.e. a
tensor ``A`` of shape (m, n) with ``A.stride() == (1, lda)``; use
``empty_colmajor`` / ``to_colmajor`` to make them.  Every computation runs in
libmrcqr.so on the tensors' device, on torch's current stream unless a
stream is passed."""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import PREC, PREC_NAME, MrcqrError, Opts, Stats, check

__all__ = ["factor", "factor_ex", "last_status", "factor_batched", "signs", "sample_rows", "sketch", "sketch_qr",
           "cholqr_precond", "empty_colmajor", "to_colmajor", "version", "PREC", "PREC_NAME", "MrcqrError"]


_selector_state = {"loaded": False}


def _prec(p) -> int:
    v = PREC[p.lower()] if isinstance(p, str) else int(p)
    if v == PREC["auto"] and not _selector_state["loaded"]:
        # the automatic choice needs selector weights: the shipped ones unless the caller set others
        from . import selector
        selector.load_into_library()
    return v


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def empty_colmajor(m: int, n: int, device=None, ld: int | None = None) -> torch.Tensor:
    ld = m if ld is None else ld
    return torch.empty((n, ld), dtype=torch.float64, device=device or "cuda").t()[:m]


def to_colmajor(x, device=None, ld: int | None = None) -> torch.Tensor:
    """Column-major float64 copy of an (m, n) array or tensor on the device."""
    t = torch.as_tensor(x, dtype=torch.float64)
    m, n = t.shape
    out = empty_colmajor(m, n, device=device or "cuda", ld=ld)
    out.copy_(t)
    return out


def _ld(t: torch.Tensor, name: str) -> int:
    """Leading dimension of a column-major (m, n) CUDA float64 tensor."""
    if t.dtype != torch.float64 or not t.is_cuda or t.dim() != 2:
        raise ValueError(f"{name} must be a 2-D CUDA float64 tensor")
    if t.stride(0) != 1 and t.shape[0] > 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    return max(t.stride(1), t.shape[0]) if t.shape[1] == 1 else t.stride(1)


def version() -> int:
    return _lib.load().mrcqr_version()


def factor_ex(A: torch.Tensor, Q: torch.Tensor, R: torch.Tensor, prec="fp64", seed: int = 0, s_factor: int = 2,
              check_ortho: bool = True, escalate: bool = True, tol: float = 1e-13, stats_device=None,
              sketch_variant: int = 0, fp64_products: int = 0, transform="dct", stream=None) -> None:
    """Enqueue MRCQR of A into Q (m x n) and R (n x n); asynchronous.  transform: "dct" (default),
    "rfft" (the paper's real-FFT sketch) or "rfft_reim" (real and imaginary parts)."""
    m, n = A.shape
    o = Opts(s_factor=s_factor, check=int(check_ortho), escalate=int(escalate), sketch_variant=sketch_variant,
             ortho_tol=tol, stats_device=stats_device.data_ptr() if stats_device is not None else None,
             fp64_products=fp64_products, transform=_transform(transform))
    rc = _lib.load().mrcqr_factor_ex(m, n, A.data_ptr(), _ld(A, "A"), Q.data_ptr(), _ld(Q, "Q"), R.data_ptr(),
                                     _ld(R, "R"), _prec(prec), seed, ctypes.byref(o), _stream(stream))
    check(rc, "mrcqr_factor_ex")


def factor(A: torch.Tensor, prec="fp64", seed: int = 0, stream=None, **kw):
    """Q, R = MRCQR(A); returns column-major tensors (asynchronous)."""
    m, n = A.shape
    Q = empty_colmajor(m, n, device=A.device)
    R = empty_colmajor(n, n, device=A.device)
    if kw:
        factor_ex(A, Q, R, prec=prec, seed=seed, stream=stream, **kw)
    else:
        check(_lib.load().mrcqr_factor(m, n, A.data_ptr(), _ld(A, "A"), Q.data_ptr(), _ld(Q, "Q"), R.data_ptr(),
                                       _prec(prec), seed, _stream(stream)), "mrcqr_factor")
    return Q, R


def last_status(stream=None) -> dict:
    st = Stats()
    check(_lib.load().mrcqr_get_last_status(_stream(stream), ctypes.byref(st)), "mrcqr_get_last_status")
    return st.as_dict()


def factor_batched(As, Qs, Rs, precs, seeds, status: torch.Tensor, stream=None) -> None:
    """Enqueue MRCQR of every A_i (lists of column-major tensors)."""
    cnt = len(As)
    arr = lambda ct, vals: (ct * cnt)(*vals)
    m = arr(ctypes.c_int64, [a.shape[0] for a in As])
    n = arr(ctypes.c_int64, [a.shape[1] for a in As])
    lda = arr(ctypes.c_int64, [_ld(a, "A") for a in As])
    ldq = arr(ctypes.c_int64, [_ld(q, "Q") for q in Qs])
    pa = arr(ctypes.c_void_p, [a.data_ptr() for a in As])
    pq = arr(ctypes.c_void_p, [q.data_ptr() for q in Qs])
    pr = arr(ctypes.c_void_p, [r.data_ptr() for r in Rs])
    pp = arr(ctypes.c_int, [_prec(p) for p in precs])
    ps = arr(ctypes.c_uint64, [int(s) for s in seeds])
    if status.dtype != torch.int32 or not status.is_cuda or status.numel() < cnt:
        raise ValueError("status must be a CUDA int32 tensor with >= count entries")
    rc = _lib.load().mrcqr_factor_batched(cnt, m, n, pa, lda, pq, ldq, pr, pp, ps, status.data_ptr(),
                                          _stream(stream))
    check(rc, "mrcqr_factor_batched")


def round_to(prec, x: torch.Tensor, stream=None) -> torch.Tensor:
    """fl_p(x) as the tensor-core sketch computes it, widened to float64."""
    x = x.contiguous()
    y = torch.empty_like(x)
    check(_lib.load().mrcqr_round(_prec(prec), x.numel(), x.data_ptr(), y.data_ptr(), _stream(stream)), "mrcqr_round")
    return y


class BatchedPlan:
    """Reusable batched MRCQR over fixed buffers (mrcqr_batched_plan_*)."""

    def __init__(self, As, Qs, Rs, precs, seeds, status: torch.Tensor, use_graph: bool = False,
                 autotune: bool = False, check_ortho: bool = True, escalate: bool = True, tol: float = 1e-13,
                 rows_per_split: int = 0, rows_per_chunk: int = 0, fp64_products: int = 0, transform="dct",
                 oz_per_problem: int = 0):
        cnt = len(As)
        arr = lambda ct, vals: (ct * cnt)(*vals)
        self._keep = dict(
            m=arr(ctypes.c_int64, [a.shape[0] for a in As]), n=arr(ctypes.c_int64, [a.shape[1] for a in As]),
            lda=arr(ctypes.c_int64, [_ld(a, "A") for a in As]), ldq=arr(ctypes.c_int64, [_ld(q, "Q") for q in Qs]),
            pa=arr(ctypes.c_void_p, [a.data_ptr() for a in As]), pq=arr(ctypes.c_void_p, [q.data_ptr() for q in Qs]),
            pr=arr(ctypes.c_void_p, [r.data_ptr() for r in Rs]), pp=arr(ctypes.c_int, [_prec(p) for p in precs]),
            ps=arr(ctypes.c_uint64, [int(s) for s in seeds]))
        if status.dtype != torch.int32 or not status.is_cuda or status.numel() < cnt:
            raise ValueError("status must be a CUDA int32 tensor with >= count entries")
        o = _lib.BatchedOpts(use_graph=int(use_graph), autotune=int(autotune), check=int(check_ortho),
                             escalate=int(escalate), ortho_tol=tol, rows_per_split=rows_per_split,
                             rows_per_chunk=rows_per_chunk, fp64_products=int(fp64_products),
                             transform=_transform(transform), oz_per_problem=int(oz_per_problem))
        self._plan = ctypes.c_void_p()
        k = self._keep
        check(_lib.load().mrcqr_batched_plan_create(cnt, k["m"], k["n"], k["pa"], k["lda"], k["pq"], k["ldq"],
                                                     k["pr"], k["pp"], k["ps"], status.data_ptr(), ctypes.byref(o),
                                                     ctypes.byref(self._plan)), "mrcqr_batched_plan_create")

    def execute(self, stream=None) -> None:
        check(_lib.load().mrcqr_batched_plan_execute(self._plan, _stream(stream)), "mrcqr_batched_plan_execute")

    def info(self) -> dict:
        a, b, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        k = ctypes.c_int32()
        check(_lib.load().mrcqr_batched_plan_info(self._plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(k),
                                                   ctypes.byref(w)), "mrcqr_batched_plan_info")
        return {"rows_per_split": a.value, "rows_per_chunk": b.value, "kernels_per_execute": k.value,
                "workspace_bytes": w.value}

    def close(self) -> None:
        if self._plan:
            _lib.load().mrcqr_batched_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def signs(m: int, seed: int, device="cuda", stream=None) -> torch.Tensor:
    d = torch.empty(m, dtype=torch.float64, device=device)
    check(_lib.load().mrcqr_signs(m, seed, d.data_ptr(), _stream(stream)), "mrcqr_signs")
    return d


def sample_rows(m: int, s: int, seed: int, device="cuda", stream=None) -> torch.Tensor:
    idx = torch.empty(s, dtype=torch.int32, device=device)
    check(_lib.load().mrcqr_sample_rows(m, s, seed, idx.data_ptr(), _stream(stream)), "mrcqr_sample_rows")
    return idx


TRANSFORMS = {"dct": 0, "rfft": 1, "rfft_reim": 2}


def _transform(t) -> int:
    if isinstance(t, str):
        if t not in TRANSFORMS:
            raise ValueError(f"unknown transform {t!r}")
        return TRANSFORMS[t]
    return int(t)


def sample_transform_rows(m: int, c: int, transform="rfft", seed: int = 0, device="cuda",
                          stream=None) -> torch.Tensor:
    """c sampled rows (DCT) or bins (real FFT); rfft_reim returns 2c words, the Im rows with bit 31 set."""
    tf = _transform(transform)
    idx = torch.empty(2 * c if tf == 2 else c, dtype=torch.int32, device=device)
    check(_lib.load().mrcqr_sample_transform_rows(m, c, tf, seed, idx.data_ptr(), _stream(stream)),
          "mrcqr_sample_transform_rows")
    return idx


def sketch_transform(A: torch.Tensor, c: int, transform="rfft", prec="fp64", seed: int = 0, variant: int = 0,
                     stream=None) -> torch.Tensor:
    """Y of the given transform: c x n (2c x n for rfft_reim, Re rows first)."""
    m, n = A.shape
    tf = _transform(transform)
    Y = empty_colmajor(2 * c if tf == 2 else c, n, device=A.device)
    check(_lib.load().mrcqr_sketch_transform(m, n, A.data_ptr(), _ld(A, "A"), c, tf, _prec(prec), seed, variant,
                                             Y.data_ptr(), _stream(stream)), "mrcqr_sketch_transform")
    return Y


REGIME_METHODS = {"probe": 0, "onenorm": 1}


def regime_estimate(A: torch.Tensor, method="probe", seed: int = 0, out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """Device tensor [kappa estimate, regime (0 fp16, 1 fp32, 2 fp64), q or ||A^T A||_1, 0 or est
    ||(A^T A)^-1||_1] from the CholQR probe or the block 1-norm estimate (Sec. II-C)."""
    m, n = A.shape
    o = out if out is not None else torch.empty(4, dtype=torch.float64, device=A.device)
    check(_lib.load().mrcqr_regime_estimate(m, n, A.data_ptr(), _ld(A, "A"), REGIME_METHODS[method], seed,
                                            o.data_ptr(), _stream(stream)), "mrcqr_regime_estimate")
    return o


def sketch(A: torch.Tensor, s: int, prec="fp64", seed: int = 0, variant: int = 0, stream=None) -> torch.Tensor:
    """Y = sqrt(m/s) P F D A in precision prec (variant 0 auto, 1 SIMT, 2 tensor-core dense rows,
    3 emulated FP64 sliced per work item, 4 four-step transform, 5 emulated FP64 from digit planes)."""
    m, n = A.shape
    Y = empty_colmajor(s, n, device=A.device)
    check(_lib.load().mrcqr_sketch_ex(m, n, A.data_ptr(), _ld(A, "A"), s, _prec(prec), seed, variant, Y.data_ptr(),
                                      _stream(stream)), "mrcqr_sketch_ex")
    return Y


def last_sketch_variant() -> int:
    return _lib.load().mrcqr_last_sketch_variant()


def sketch_qr(Y: torch.Tensor, prec="fp64", stream=None) -> torch.Tensor:
    s, n = Y.shape
    if _ld(Y, "Y") != s:
        raise ValueError("Y must be packed (ld == s)")
    Rs = empty_colmajor(n, n, device=Y.device)
    check(_lib.load().mrcqr_sketch_qr(n, s, Y.data_ptr(), _prec(prec), Rs.data_ptr(), _stream(stream)),
          "mrcqr_sketch_qr")
    return Rs


def cholqr_precond(A: torch.Tensor, Rs: torch.Tensor, stream=None):
    m, n = A.shape
    if _ld(Rs, "Rs") != n:
        raise ValueError("Rs must be packed (ld == n)")
    Q = empty_colmajor(m, n, device=A.device)
    R = empty_colmajor(n, n, device=A.device)
    check(_lib.load().mrcqr_cholqr_precond(m, n, A.data_ptr(), _ld(A, "A"), Rs.data_ptr(), Q.data_ptr(),
                                           _ld(Q, "Q"), R.data_ptr(), _ld(R, "R"), _stream(stream)),
          "mrcqr_cholqr_precond")
    return Q, R


def cholqr2(A: torch.Tensor, stream=None):
    """Q, R = CholQR2(A) (asynchronous; status through last_status)."""
    m, n = A.shape
    Q = empty_colmajor(m, n, device=A.device)
    R = empty_colmajor(n, n, device=A.device)
    check(_lib.load().mrcqr_cholqr2(m, n, A.data_ptr(), _ld(A, "A"), Q.data_ptr(), _ld(Q, "Q"), R.data_ptr(),
                                    _ld(R, "R"), _stream(stream)), "mrcqr_cholqr2")
    return Q, R


def finalize_q(W: torch.Tensor, X: torch.Tensor, fp64_products: int = 0, stream=None) -> torch.Tensor:
    """Q = W X with X upper triangular (the upper triangle of X is read); W is overwritten."""
    m, n = W.shape
    check(_lib.load().mrcqr_finalize_q(m, n, W.data_ptr(), _ld(W, "W"), X.data_ptr(), _ld(X, "X"),
                                       int(fp64_products), _stream(stream)), "mrcqr_finalize_q")
    return W


def gram(W: torch.Tensor, fp64_products: int = 0, stream=None) -> torch.Tensor:
    """Upper triangle of W^T W (strictly lower triangle zero), n x n column-major."""
    m, n = W.shape
    G = empty_colmajor(n, n, device=W.device)
    check(_lib.load().mrcqr_gram(m, n, W.data_ptr(), _ld(W, "W"), G.data_ptr(), int(fp64_products),
                                 _stream(stream)), "mrcqr_gram")
    return G


def trsm(A: torch.Tensor, R: torch.Tensor, fp64_products: int = 0, stream=None) -> torch.Tensor:
    """W = A R^{-1} (R upper triangular; its upper triangle is read), column-major m x n."""
    m, n = A.shape
    W = empty_colmajor(m, n, device=A.device)
    check(_lib.load().mrcqr_trsm(m, n, A.data_ptr(), _ld(A, "A"), R.data_ptr(), _ld(R, "R"), W.data_ptr(),
                                 _ld(W, "W"), int(fp64_products), _stream(stream)), "mrcqr_trsm")
    return W
