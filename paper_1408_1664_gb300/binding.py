"""Thin ctypes binding of the C ABI in ``include/bnedge.h``.

Only argument marshalling happens here: every step of the computation runs
in the CUDA kernels of ``_build/libbnedge.so``.  Loading fails loudly when the
library has not been built (there is no CPU fallback).  Functions carry the C
names (``bn_ctx_create``, ``bn_edge_posteriors``, ...); ``Context`` wraps them
for numpy / torch callers.  Device pointers and CUDA streams may be given as
integers or as torch tensors / streams (``data_ptr()`` / ``cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

BN_OK, BN_EINVAL, BN_ENOMEM, BN_EAGAIN, BN_ETIMEOUT = 0, -1, -2, -3, -4
BN_EDEVICE_TIMEOUT, BN_ECUDA, BN_ECANCELED, BN_ENOTFOUND = -5, -6, -7, -8
BN_FP64, BN_FP32_SHIFTED = 0, 1
PRECISIONS = {"fp64": BN_FP64, "fp32": BN_FP32_SHIFTED}
BN_SHARD_DIVIDE_A = 1
(BN_STAGE_LOGB, BN_STAGE_MASKS, BN_STAGE_SHIFT, BN_STAGE_A, BN_STAGE_F, BN_STAGE_RC,
 BN_STAGE_GAMMA) = range(1, 8)


class BnError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {bn_strerror(code)} ({code})")


class bn_ctx_opts(C.Structure):
    _fields_ = [("device", C.c_int32), ("slots", C.c_int32), ("mem_budget", C.c_uint64),
                ("fail_alloc_after", C.c_int32), ("flags", C.c_int32)]


class bn_job_desc(C.Structure):
    _fields_ = [("n", C.c_int32), ("d", C.c_int32), ("m", C.c_int32), ("precision", C.c_int32),
                ("data", C.c_void_p), ("arity", C.c_void_p), ("ess", C.c_double),
                ("log_rho", C.c_void_p), ("data_on_device", C.c_int32), ("reserved", C.c_int32),
                ("log_q", C.c_void_p), ("log_w", C.c_void_p)]


class bn_stats(C.Structure):
    _fields_ = [("ms_scores", C.c_double), ("ms_upzeta", C.c_double),
                ("ms_forward", C.c_double), ("ms_backward", C.c_double),
                ("ms_gamma_p1", C.c_double), ("ms_gamma_p2", C.c_double),
                ("ms_edges", C.c_double), ("ms_total", C.c_double), ("cells", C.c_double),
                ("alg_bytes", C.c_double), ("kernels", C.c_int32), ("precision", C.c_int32),
                ("ms_upzeta_sums", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
EXPORTS = ["bn_ctx_create", "bn_ctx_destroy", "bn_num_families", "bn_scores",
           "bn_edge_posteriors", "bn_edge_posteriors_async", "bn_submit", "bn_poll", "bn_wait",
           "bn_cancel", "bn_job_stats", "bn_stats_history", "bn_strerror",
           "bn_edge_posteriors_static", "bn_job_footprint", "bn_batch_create",
           "bn_batch_run", "bn_batch_results", "bn_batch_describe", "bn_batch_destroy",
           "bn_feature_posterior", "bn_batch_upload", "bn_batch_download",
           "bn_shard_create", "bn_shard_prepare", "bn_shard_level", "bn_shard_exchange_bytes",
           "bn_shard_pack", "bn_shard_unpack", "bn_shard_finish", "bn_shard_destroy",
           "bn_shard_bytes"]


# Test hooks: exported only by the testing build (BN_TESTING).
TEST_EXPORTS = ["bn_debug_stage", "bn_debug_counts", "bn_debug_batch_drop", "bn_debug_bounds",
                "bn_debug_explog", "bn_debug_copy_wait"]


def testing_build() -> bool:
    """The testing build of the library (with the BN_TESTING hooks) is loaded
    when the environment sets BN_TESTING=1; the test suite does."""
    return os.environ.get("BN_TESTING") == "1"


def checked_build() -> bool:
    """The BN_CHECK_BOUNDS debug build (index checks in the kernels, plus the
    test hooks) is loaded when the environment sets BN_CHECK_BOUNDS=1."""
    return os.environ.get("BN_CHECK_BOUNDS") == "1"


def asan_build() -> bool:
    """The host-sanitizer build (the process must preload libasan and
    libubsan) is loaded when the environment sets BN_ASAN=1."""
    return os.environ.get("BN_ASAN") == "1"


def library_path() -> str:
    if asan_build():
        return _build.LIB_ASAN
    if checked_build():
        return _build.LIB_CHECKED
    return _build.LIB_TESTING if testing_build() else _build.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Load the CUDA library (building it first only when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing:
        if asan_build():
            _build.build_asan()
        elif checked_build():
            _build.build_checked()
        else:
            _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build()); there is no CPU fallback")
    L = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "bn_ctx_create": (C.c_int, [C.POINTER(P), C.POINTER(bn_ctx_opts)]),
        "bn_ctx_destroy": (C.c_int, [P]),
        "bn_num_families": (C.c_int64, [C.c_int32, C.c_int32]),
        "bn_job_footprint": (C.c_int, [C.POINTER(bn_job_desc), C.POINTER(C.c_uint64)]),
        "bn_scores": (C.c_int, [P, C.POINTER(bn_job_desc), P, P]),
        "bn_edge_posteriors": (C.c_int, [P, C.POINTER(bn_job_desc), P, P]),
        "bn_edge_posteriors_async": (C.c_int, [P, C.POINTER(bn_job_desc), P, P, P]),
        "bn_edge_posteriors_static": (C.c_int, [C.POINTER(bn_job_desc), P, P, P]),
        "bn_submit": (C.c_int, [P, C.POINTER(bn_job_desc), C.POINTER(C.c_uint64)]),
        "bn_poll": (C.c_int, [P, C.c_uint64, P, P]),
        "bn_wait": (C.c_int, [P, C.c_uint64, C.c_double, P, P]),
        "bn_cancel": (C.c_int, [P, C.c_uint64]),
        "bn_job_stats": (C.c_int, [P, C.c_uint64, C.POINTER(bn_stats)]),
        "bn_stats_history": (C.c_int, [P, C.POINTER(bn_stats), C.c_int32,
                                       C.POINTER(C.c_int32)]),
        "bn_strerror": (C.c_char_p, [C.c_int]),
        "bn_batch_create": (C.c_int, [P, C.POINTER(bn_job_desc), C.c_int32, C.POINTER(P)]),
        "bn_batch_run": (C.c_int, [P, P]),
        "bn_batch_results": (C.c_int, [P, C.c_int32, P, P]),
        "bn_batch_describe": (C.c_int, [P, C.c_char_p, C.c_size_t]),
        "bn_batch_upload": (C.c_int, [P, C.POINTER(bn_job_desc), C.c_int32, P]),
        "bn_batch_download": (C.c_int, [P, P, P]),
        "bn_batch_destroy": (C.c_int, [P]),
        "bn_debug_stage": (C.c_int, [P, C.c_int32, P, C.c_size_t]),
        "bn_debug_counts": (C.c_int, [P, C.POINTER(bn_job_desc), C.c_int32, C.c_uint32, P,
                                      C.c_int64]),
        "bn_feature_posterior": (C.c_int, [P, C.POINTER(bn_job_desc), P, P, P]),
        "bn_debug_batch_drop": (C.c_int, [P, C.c_int32, C.c_uint64]),
        "bn_debug_bounds": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "bn_debug_explog": (C.c_int, [P, C.c_int64, P]),
        "bn_debug_copy_wait": (C.c_int, [C.c_uint32, C.POINTER(C.c_int32)]),
        "bn_shard_create": (C.c_int, [P, C.POINTER(bn_job_desc), C.c_int32, C.c_int32, C.c_int32,
                                      C.POINTER(P)]),
        "bn_shard_bytes": (C.c_int, [P, C.POINTER(C.c_uint64)]),
        "bn_shard_prepare": (C.c_int, [P, P]),
        "bn_shard_level": (C.c_int, [P, C.c_int32, C.c_int32, P]),
        "bn_shard_exchange_bytes": (C.c_int, [P, C.c_int32, C.POINTER(C.c_uint64)]),
        "bn_shard_pack": (C.c_int, [P, C.c_int32, C.c_int32, P, P]),
        "bn_shard_unpack": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, P, P]),
        "bn_shard_finish": (C.c_int, [P, P, P, P]),
        "bn_shard_destroy": (C.c_int, [P]),
    }
    for name, (res, args) in sig.items():
        if name in TEST_EXPORTS and not hasattr(L, name):
            continue                                   # release build
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(x) -> int | None:
    """Address of a numpy array, a torch tensor or an integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "cuda_stream"):
        return int(x.cuda_stream)
    raise TypeError(f"cannot take the address of {type(x)}")


# ---- C-named entry points ------------------------------------------------

def bn_strerror(code: int) -> str:
    if _lib is None:
        return {0: "ok", -1: "invalid argument", -2: "out of memory"}.get(code, f"error {code}")
    return _lib.bn_strerror(code).decode()


def bn_num_families(n: int, d: int) -> int:
    return int(load().bn_num_families(n, d))


def bn_job_footprint(job: "Job") -> int:
    out = C.c_uint64()
    rc = load().bn_job_footprint(C.byref(job.desc), C.byref(out))
    if rc:
        raise BnError(rc, "bn_job_footprint")
    return int(out.value)


BN_CTX_NO_AUTOTUNE = 1
BN_CTX_CLUSTER_STEP3 = 2
BN_CTX_GRAPH_BATCH = 4


def bn_ctx_create(device: int = 0, slots: int = 4, mem_budget: int = 0,
                  fail_alloc_after: int = -1, flags: int = 0) -> int:
    h = C.c_void_p()
    opts = bn_ctx_opts(device, slots, mem_budget, fail_alloc_after, flags)
    rc = load().bn_ctx_create(C.byref(h), C.byref(opts))
    if rc:
        raise BnError(rc, "bn_ctx_create")
    return h.value


def bn_ctx_destroy(ctx: int) -> int:
    return load().bn_ctx_destroy(ctx)


class Job:
    """A bn_job_desc plus the arrays it points to (kept alive with it)."""

    def __init__(self, data, arity, d: int, ess: float = 1.0, log_rho=None,
                 precision: str | int = "fp64", m: int | None = None, log_q=None, log_w=None):
        self.arity = np.ascontiguousarray(arity, dtype=np.uint8)
        n = int(self.arity.shape[0])
        on_dev = not isinstance(data, np.ndarray)
        if on_dev:
            self.data = data
            if m is None:
                m = int(data.numel()) // n if hasattr(data, "numel") else None
            if m is None:
                raise ValueError("m is required for a device pointer")
        else:
            self.data = np.ascontiguousarray(data, dtype=np.uint8).reshape(-1, n)
            m = int(self.data.shape[0])
        self.log_rho = None if log_rho is None else np.ascontiguousarray(log_rho, np.float64)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.n, self.d, self.m = n, int(d), int(m)
        self.log_q = None if log_q is None else np.ascontiguousarray(log_q, np.float64).reshape(-1)
        self.log_w = None if log_w is None else np.ascontiguousarray(log_w, np.float64).reshape(-1)
        self.desc = bn_job_desc(n, int(d), int(m), prec,
                                _ptr(self.data) if m > 0 else None, _ptr(self.arity),
                                float(ess), _ptr(self.log_rho), 1 if on_dev else 0, 0,
                                _ptr(self.log_q), _ptr(self.log_w))


def bn_edge_posteriors(ctx: int, job: Job, post: np.ndarray | None = None):
    n = job.n
    post = np.zeros((n, n)) if post is None else post
    lpd = np.zeros(1)
    rc = load().bn_edge_posteriors(ctx, C.byref(job.desc), _ptr(post), _ptr(lpd))
    if rc:
        raise BnError(rc, "bn_edge_posteriors")
    return post, float(lpd[0])


def bn_edge_posteriors_async(ctx: int, job: Job, post_dev, log_PD_dev=None, stream=None) -> None:
    rc = load().bn_edge_posteriors_async(ctx, C.byref(job.desc), _ptr(post_dev),
                                         _ptr(log_PD_dev), _ptr(stream))
    if rc:
        raise BnError(rc, "bn_edge_posteriors_async")


def bn_edge_posteriors_static(job: Job, post_dev, log_PD_dev=None, stream=None) -> None:
    """No-allocation variant: all intermediates in the library's fixed device
    scratch array (for callers that cannot allocate device memory)."""
    rc = load().bn_edge_posteriors_static(C.byref(job.desc), _ptr(post_dev), _ptr(log_PD_dev),
                                          _ptr(stream))
    if rc:
        raise BnError(rc, "bn_edge_posteriors_static")


def bn_feature_posterior(ctx: int, job: Job, log_f) -> tuple[float, float]:
    """P(f | D) and log P(f, D) of the modular feature log_f (n, K)."""
    lf = np.ascontiguousarray(log_f, dtype=np.float64).reshape(-1)
    if lf.shape[0] != job.n * bn_num_families(job.n, job.d):
        raise ValueError("log_f must hold n * K values")
    p = np.zeros(1)
    lpfd = np.zeros(1)
    rc = load().bn_feature_posterior(ctx, C.byref(job.desc), _ptr(lf), _ptr(p), _ptr(lpfd))
    if rc:
        raise BnError(rc, "bn_feature_posterior")
    return float(p[0]), float(lpfd[0])


def bn_scores(ctx: int, job: Job):
    K = bn_num_families(job.n, job.d)
    masks = np.zeros((job.n, K), dtype=np.uint32)
    logB = np.zeros((job.n, K))
    rc = load().bn_scores(ctx, C.byref(job.desc), _ptr(masks), _ptr(logB))
    if rc:
        raise BnError(rc, "bn_scores")
    return masks, logB


def bn_submit(ctx: int, job: Job) -> int:
    jid = C.c_uint64()
    rc = load().bn_submit(ctx, C.byref(job.desc), C.byref(jid))
    if rc:
        raise BnError(rc, "bn_submit")
    return int(jid.value)


def bn_poll(ctx: int, job_id: int, n: int):
    """(rc, post, log_PD); rc is BN_OK, BN_EAGAIN or an error code."""
    post = np.zeros((n, n))
    lpd = np.zeros(1)
    rc = load().bn_poll(ctx, job_id, _ptr(post), _ptr(lpd))
    return rc, post, float(lpd[0])


def bn_wait(ctx: int, job_id: int, n: int, timeout_s: float = 60.0):
    post = np.zeros((n, n))
    lpd = np.zeros(1)
    rc = load().bn_wait(ctx, job_id, float(timeout_s), _ptr(post), _ptr(lpd))
    return rc, post, float(lpd[0])


def bn_cancel(ctx: int, job_id: int) -> int:
    return int(load().bn_cancel(ctx, job_id))


def bn_job_stats(ctx: int, job_id: int = 0) -> dict:
    st = bn_stats()
    rc = load().bn_job_stats(ctx, job_id, C.byref(st))
    if rc:
        raise BnError(rc, "bn_job_stats")
    return st.as_dict()


def bn_stats_history(ctx: int, max_entries: int = 32) -> list:
    arr = (bn_stats * max_entries)()
    cnt = C.c_int32()
    rc = load().bn_stats_history(ctx, arr, max_entries, C.byref(cnt))
    if rc:
        raise BnError(rc, "bn_stats_history")
    return [arr[k].as_dict() for k in range(cnt.value)]


def bn_debug_stage(ctx: int, stage: int, shape, dtype) -> np.ndarray:
    out = np.zeros(shape, dtype=dtype)
    rc = load().bn_debug_stage(ctx, stage, _ptr(out), out.nbytes)
    if rc:
        raise BnError(rc, "bn_debug_stage")
    return out


def bn_debug_bounds() -> tuple[int, int]:
    """(line, unit) of the first failing index check of the BN_CHECK_BOUNDS
    build since the last call; (0, 0) when none failed, (-1, 0) in the other
    builds."""
    line, unit = C.c_int32(), C.c_int32()
    rc = load().bn_debug_bounds(C.byref(line), C.byref(unit))
    if rc:
        raise BnError(rc, "bn_debug_bounds")
    return int(line.value), int(unit.value)


def bn_debug_counts(ctx: int, job: Job, i: int, mask: int, cells: int) -> np.ndarray:
    out = np.zeros(cells, dtype=np.int64)
    rc = load().bn_debug_counts(ctx, C.byref(job.desc), i, mask, _ptr(out), cells)
    if rc:
        raise BnError(rc, "bn_debug_counts")
    return out


class Batch:
    """Owns one bn_batch: many independent jobs replayed as one CUDA graph."""

    def __init__(self, ctx: int, jobs: list):
        self.jobs = list(jobs)
        arr = (bn_job_desc * len(self.jobs))(*[j.desc for j in self.jobs])
        self._arr = arr
        h = C.c_void_p()
        rc = load().bn_batch_create(ctx, arr, len(self.jobs), C.byref(h))
        if rc:
            raise BnError(rc, "bn_batch_create")
        self.h = h.value

    def run(self, stream=None) -> None:
        rc = load().bn_batch_run(self.h, _ptr(stream))
        if rc:
            raise BnError(rc, "bn_batch_run")

    def upload(self, jobs: list, stream=None) -> None:
        """New data for every job (same shapes as at creation)."""
        self._up = list(jobs)
        arr = (bn_job_desc * len(self._up))(*[j.desc for j in self._up])
        self._up_arr = arr
        rc = load().bn_batch_upload(self.h, arr, len(self._up), _ptr(stream))
        if rc:
            raise BnError(rc, "bn_batch_upload")

    def download(self):
        """Every job's posteriors (a list of n x n arrays) and log P(D)s."""
        sizes = [j.n * j.n for j in self.jobs]
        flat = np.zeros(sum(sizes))
        lpd = np.zeros(len(self.jobs))
        rc = load().bn_batch_download(self.h, _ptr(flat), _ptr(lpd))
        if rc:
            raise BnError(rc, "bn_batch_download")
        out, o = [], 0
        for j, sz in zip(self.jobs, sizes):
            out.append(flat[o:o + sz].reshape(j.n, j.n))
            o += sz
        return out, lpd

    def describe(self) -> str:
        buf = C.create_string_buffer(1 << 14)
        rc = load().bn_batch_describe(self.h, buf, len(buf))
        if rc:
            raise BnError(rc, "bn_batch_describe")
        return buf.value.decode()

    def results(self, k: int):
        n = self.jobs[k].n
        post = np.zeros((n, n))
        lpd = np.zeros(1)
        rc = load().bn_batch_results(self.h, k, _ptr(post), _ptr(lpd))
        if rc:
            raise BnError(rc, "bn_batch_results")
        return post, float(lpd[0])

    def close(self):
        if self.h:
            load().bn_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Shard:
    """Owns one bn_shard: rank `rank` of a job split over `world` ranks
    (include/bnedge.h, "Shards").  Buffers are device tensors or addresses;
    `stream` a torch stream or a cudaStream_t address (None = the context's
    stream)."""

    def __init__(self, ctx: int, job: Job, rank: int, world: int, divide_a: bool = False):
        self.job, self.rank, self.world = job, int(rank), int(world)
        h = C.c_void_p()
        rc = load().bn_shard_create(ctx, C.byref(job.desc), self.rank, self.world,
                                    BN_SHARD_DIVIDE_A if divide_a else 0, C.byref(h))
        if rc:
            raise BnError(rc, "bn_shard_create")
        self.h = h.value
        # tile levels of the step-3 sweeps: n - 4 (FP32) or n - 3 (FP64)
        self.levels = job.n - (4 if job.desc.precision == PRECISIONS["fp32"] else 3)

    def _call(self, name, *args):
        rc = getattr(load(), name)(self.h, *args)
        if rc:
            raise BnError(rc, name)

    def prepare(self, stream=None) -> None:
        self._call("bn_shard_prepare", _ptr(stream))

    def level(self, sweep: int, hl: int, stream=None) -> None:
        self._call("bn_shard_level", sweep, hl, _ptr(stream))

    def bytes(self) -> int:
        """Device bytes the shard holds."""
        b = C.c_uint64()
        self._call("bn_shard_bytes", C.byref(b))
        return int(b.value)

    def exchange_bytes(self, hl: int) -> int:
        b = C.c_uint64()
        self._call("bn_shard_exchange_bytes", hl, C.byref(b))
        return int(b.value)

    def pack(self, sweep: int, hl: int, buf, stream=None) -> None:
        self._call("bn_shard_pack", sweep, hl, _ptr(buf), _ptr(stream))

    def unpack(self, sweep: int, hl: int, src: int, buf, stream=None) -> None:
        self._call("bn_shard_unpack", sweep, hl, src, _ptr(buf), _ptr(stream))

    def finish(self, post_dev, log_PD_dev=None, stream=None) -> None:
        self._call("bn_shard_finish", _ptr(post_dev), _ptr(log_PD_dev), _ptr(stream))

    def close(self):
        if self.h:
            load().bn_shard_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Context:
    """Owns one bn_ctx."""

    def __init__(self, device: int = 0, slots: int = 4, mem_budget: int = 0,
                 fail_alloc_after: int = -1, autotune: bool = True,
                 cluster_step3: bool = False, graph_batch: bool = False):
        flags = ((0 if autotune else BN_CTX_NO_AUTOTUNE)
                 | (BN_CTX_CLUSTER_STEP3 if cluster_step3 else 0)
                 | (BN_CTX_GRAPH_BATCH if graph_batch else 0))
        self.h = bn_ctx_create(device, slots, mem_budget, fail_alloc_after, flags)

    def close(self):
        if self.h:
            bn_ctx_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def edge_posteriors(self, data, arity, d, ess=1.0, log_rho=None, precision="fp64"):
        return bn_edge_posteriors(self.h, Job(data, arity, d, ess, log_rho, precision))

    def scores(self, data, arity, d, ess=1.0, log_rho=None):
        return bn_scores(self.h, Job(data, arity, d, ess, log_rho))

    def stats(self, job_id: int = 0) -> dict:
        return bn_job_stats(self.h, job_id)
