"""ctypes wrapper of the CPU FP64 oracle (``bn_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark are the only users.  Nothing in the product package imports
this module, and this module imports nothing from the product package.

``build()`` compiles ``bn_oracle.c`` with gcc (OpenMP when available) into
``oracle/_build/libbnoracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bn_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libbnoracle.so")
_lib = None

_u8p = C.POINTER(C.c_uint8)
_u32p = C.POINTER(C.c_uint32)
_i64p = C.POINTER(C.c_int64)
_f64p = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle; returns the path of the shared library."""
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _OUT + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_OUT + ".tmp", _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_num_threads.restype = C.c_int
        L.orc_num_families.restype = C.c_int64
        L.orc_num_families.argtypes = [C.c_int, C.c_int]
        L.orc_family_list.restype = C.c_int64
        L.orc_family_list.argtypes = [C.c_int, C.c_int, C.c_int, _u32p]
        L.orc_family_cells.restype = C.c_int64
        L.orc_family_cells.argtypes = [C.c_int, _u8p, C.c_int, C.c_uint32]
        L.orc_family_counts.restype = None
        L.orc_family_counts.argtypes = [C.c_int, C.c_int, _u8p, _u8p, C.c_int, C.c_uint32, _i64p]
        L.orc_bdeu.restype = C.c_double
        L.orc_bdeu.argtypes = [C.c_int, C.c_int64, _i64p, C.c_double]
        L.orc_family_score.restype = C.c_double
        L.orc_family_score.argtypes = [C.c_int, C.c_int, _u8p, _u8p, C.c_double, _f64p,
                                       C.c_int, C.c_uint32]
        L.orc_scores.restype = C.c_int
        L.orc_scores.argtypes = [C.c_int, C.c_int, C.c_int, _u8p, _u8p, C.c_double, _f64p,
                                 _u32p, _f64p]
        L.orc_upzeta.restype = C.c_int
        L.orc_upzeta.argtypes = [C.c_int, C.c_int, _f64p, _f64p]
        L.orc_downzeta.restype = C.c_int
        L.orc_downzeta.argtypes = [C.c_int, C.c_int, _f64p, _f64p]
        L.orc_forward.restype = None
        L.orc_forward.argtypes = [C.c_int, _f64p, _f64p]
        L.orc_backward.restype = None
        L.orc_backward.argtypes = [C.c_int, _f64p, _f64p]
        L.orc_edge_posteriors.restype = C.c_int
        L.orc_edge_posteriors.argtypes = [C.c_int, C.c_int, C.c_int, _u8p, _u8p, C.c_double,
                                          _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p,
                                          _f64p, _u32p]
        L.orc_edge_posteriors_ext.restype = C.c_int
        L.orc_edge_posteriors_ext.argtypes = [C.c_int, C.c_int, C.c_int, _u8p, _u8p,
                                              C.c_double, _f64p, _f64p, _f64p, _f64p, _f64p,
                                              _f64p, _f64p, _f64p, _f64p, _f64p, _u32p]
        L.orc_feature_posterior.restype = C.c_int
        L.orc_feature_posterior.argtypes = [C.c_int, C.c_int, C.c_int, _u8p, _u8p, C.c_double,
                                            _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


def _prep(data, arity):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    arity = np.ascontiguousarray(arity, dtype=np.uint8)
    if data.ndim != 2:
        data = data.reshape(0, arity.shape[0])
    return data, arity


def num_threads() -> int:
    return int(lib().orc_num_threads())


def num_families(n: int, d: int) -> int:
    return int(lib().orc_num_families(n, d))


def family_list(n: int, d: int, i: int) -> np.ndarray:
    K = num_families(n, d)
    out = np.zeros(K, dtype=np.uint32)
    lib().orc_family_list(n, d, i, _p(out, _u32p))
    return out


def family_counts(data, arity, i: int, mask: int) -> np.ndarray:
    data, arity = _prep(data, arity)
    n = arity.shape[0]
    cells = int(lib().orc_family_cells(n, _p(arity, _u8p), i, mask))
    out = np.zeros(cells, dtype=np.int64)
    lib().orc_family_counts(n, data.shape[0], _p(data, _u8p), _p(arity, _u8p), i, mask,
                            _p(out, _i64p))
    return out


def family_score(data, arity, i: int, mask: int, ess: float = 1.0, log_rho=None) -> float:
    data, arity = _prep(data, arity)
    lr = None if log_rho is None else np.ascontiguousarray(log_rho, dtype=np.float64)
    return float(lib().orc_family_score(arity.shape[0], data.shape[0], _p(data, _u8p),
                                        _p(arity, _u8p), ess, _p(lr, _f64p), i, mask))


def scores(data, arity, d: int, ess: float = 1.0, log_rho=None):
    """(masks, logB), each shaped (n, K), families in canonical order."""
    data, arity = _prep(data, arity)
    n = arity.shape[0]
    K = num_families(n, d)
    masks = np.zeros((n, K), dtype=np.uint32)
    logB = np.zeros((n, K), dtype=np.float64)
    lr = None if log_rho is None else np.ascontiguousarray(log_rho, dtype=np.float64)
    rc = lib().orc_scores(n, d, data.shape[0], _p(data, _u8p), _p(arity, _u8p), ess,
                          _p(lr, _f64p), _p(masks, _u32p), _p(logB, _f64p))
    if rc:
        raise ValueError(f"oracle scores: error {rc}")
    return masks, logB


def upzeta(n: int, d: int, s) -> np.ndarray:
    s = np.ascontiguousarray(s, dtype=np.float64)
    t = np.empty_like(s)
    if lib().orc_upzeta(n, d, _p(s, _f64p), _p(t, _f64p)):
        raise MemoryError
    return t


def downzeta(n: int, d: int, s) -> np.ndarray:
    s = np.ascontiguousarray(s, dtype=np.float64)
    t = np.empty_like(s)
    if lib().orc_downzeta(n, d, _p(s, _f64p), _p(t, _f64p)):
        raise MemoryError
    return t


def forward(n: int, A) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    F = np.empty(1 << n)
    lib().orc_forward(n, _p(A, _f64p), _p(F, _f64p))
    return F


def backward(n: int, A) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    R = np.empty(1 << n)
    lib().orc_backward(n, _p(A, _f64p), _p(R, _f64p))
    return R


def _f64_or_none(a, size: int):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.shape[0] != size:
        raise ValueError(f"expected {size} values, got {a.shape[0]}")
    return a


def edge_posteriors(data, arity, d: int, ess: float = 1.0, log_rho=None,
                    stages: bool = False, log_q=None, log_w=None) -> dict:
    """Run Algorithm 1.  Returns {'post': (n, n), 'log_PD': float} and, with
    ``stages``, also 'A' (n, 2^n), 'F', 'R' (2^n), 'Gamma', 'logB', 'masks'
    (n, K); ``stages`` may also name a subset of these, e.g. ("F", "R").
    log_q (n, n): log q_i(S) by |S| (Eq. 4, 7, 12); log_w (n, K): per family
    log weights added to log B (a general rho_i(G))."""
    data, arity = _prep(data, arity)
    n = arity.shape[0]
    K = num_families(n, d)
    N = 1 << n
    post = np.zeros((n, n))
    lpd = np.zeros(1)
    lr = None if log_rho is None else np.ascontiguousarray(log_rho, dtype=np.float64)
    st = {}
    if stages:
        make = dict(A=lambda: np.empty((n, N)), F=lambda: np.empty(N), R=lambda: np.empty(N),
                    Gamma=lambda: np.empty((n, K)), logB=lambda: np.empty((n, K)),
                    masks=lambda: np.empty((n, K), dtype=np.uint32))
        names = make if stages is True else stages
        st = {k: make[k]() for k in names}
    lq = _f64_or_none(log_q, n * n)
    lw = _f64_or_none(log_w, n * K)
    rc = lib().orc_edge_posteriors_ext(
        n, d, data.shape[0], _p(data, _u8p), _p(arity, _u8p), ess, _p(lr, _f64p),
        _p(lq, _f64p), _p(lw, _f64p),
        _p(post, _f64p), _p(lpd, _f64p), _p(st.get("A"), _f64p), _p(st.get("F"), _f64p),
        _p(st.get("R"), _f64p), _p(st.get("Gamma"), _f64p), _p(st.get("logB"), _f64p),
        _p(st.get("masks"), _u32p))
    if rc:
        raise ValueError(f"oracle edge_posteriors: error {rc}")
    out = dict(post=post, log_PD=float(lpd[0]))
    out.update(st)
    return out


def feature_posterior(data, arity, d: int, log_f, ess: float = 1.0, log_rho=None,
                      log_q=None, log_w=None) -> tuple[float, float]:
    """P(f | D) and log P(f, D) of the modular feature with log f_i(G) =
    log_f[i, f] (n, K; -inf where f_i(G) = 0), Eqs. 5-9."""
    data, arity = _prep(data, arity)
    n = arity.shape[0]
    K = num_families(n, d)
    lf = _f64_or_none(log_f, n * K)
    lq = _f64_or_none(log_q, n * n)
    lw = _f64_or_none(log_w, n * K)
    lr = None if log_rho is None else np.ascontiguousarray(log_rho, dtype=np.float64)
    p = np.zeros(1)
    lpfd = np.zeros(1)
    rc = lib().orc_feature_posterior(n, d, data.shape[0], _p(data, _u8p), _p(arity, _u8p), ess,
                                     _p(lr, _f64p), _p(lq, _f64p), _p(lw, _f64p), _p(lf, _f64p),
                                     _p(p, _f64p), _p(lpfd, _f64p))
    if rc:
        raise ValueError(f"oracle feature_posterior: error {rc}")
    return float(p[0]), float(lpfd[0])
