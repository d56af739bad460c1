"""Thin ctypes binding of libbie2d (include/bie2d.h): argument marshalling only.

Every function here forwards to the C ABI of the same name; all arithmetic runs
in the CUDA kernels of the library.  Arrays may be torch tensors (CUDA or CPU)
or numpy arrays: their data pointers are passed as is, and the library tells
host from device memory.  The library must have been built
(``paper_1507_05925_gb300.build.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

OK, WARN_NONNEUTRAL, WARN_NOT_CONVERGED = 0, 1, 2
ERR_INVALID, ERR_OUTSIDE, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM = -1, -2, -3, -4, -5
LAPLACE, STOKES = 0, 1
FP64, MIXED, MIXED_FF = 0, 1, 2
PRECOND_BLOCK_JACOBI, PRECOND_NONE = 0, 1


class BieGeometry(ctypes.Structure):
    _fields_ = [("n_bodies", ctypes.c_int32), ("body_start", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("dx", ctypes.c_void_p), ("dy", ctypes.c_void_p),
                ("ddx", ctypes.c_void_p), ("ddy", ctypes.c_void_p),
                ("interior_pt", ctypes.c_void_p)]


class BieOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("restart", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("formulation", ctypes.c_int32), ("max_refine", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("fmm_order", ctypes.c_int32), ("precond", ctypes.c_int32)]


class BieInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("matvecs_fp64", ctypes.c_int32), ("matvecs_fp32", ctypes.c_int32),
                ("matvecs_ff", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("constraint_residual", ctypes.c_double),
                ("net_load", ctypes.c_double), ("fp32_error", ctypes.c_double),
                ("precond_fallbacks", ctypes.c_int32), ("graph_replay", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BieRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("geom", BieGeometry), ("load", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("density", ctypes.c_void_p), ("opts", BieOpts)]


class BieProfileCounters(ctypes.Structure):
    _fields_ = [("launches", (ctypes.c_int64 * 2) * 3), ("ms", (ctypes.c_double * 2) * 3),
                ("pairs", (ctypes.c_double * 2) * 3), ("kernel_launches", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for p, pn in ((0, "fp64"), (1, "fp32"), (2, "ff")):
            for k, kn in ((0, "laplace"), (1, "stokes")):
                out[f"{kn}_{pn}"] = dict(launches=int(self.launches[p][k]), ms=float(self.ms[p][k]),
                                         pairs=float(self.pairs[p][k]))
        out["kernel_launches"] = int(self.kernel_launches)
        return out


_LIB = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libbie2d.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libbie2d.so is not built ({path}); call paper_1507_05925_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.bie_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.c_size_t]
    lib.bie_create.restype = i32
    lib.bie_destroy.argtypes = [vp]
    lib.bie_destroy.restype = None
    lib.bie_last_error.argtypes = [vp]
    lib.bie_last_error.restype = ctypes.c_char_p
    for name in ("elastance_solve", "mobility_solve"):
        f = getattr(lib, name)
        f.argtypes = [vp, ctypes.POINTER(BieGeometry), vp, vp, vp, ctypes.POINTER(BieOpts),
                      ctypes.POINTER(BieInfo), vp]
        f.restype = i32
    for name in ("elastance_solve_batch", "mobility_solve_batch"):
        f = getattr(lib, name)
        f.argtypes = [vp, i32, ctypes.POINTER(BieGeometry), ctypes.POINTER(vp), ctypes.POINTER(vp),
                      ctypes.POINTER(BieOpts), ctypes.POINTER(BieInfo), ctypes.POINTER(i32), vp]
        f.restype = i32
    lib.apply_operator.argtypes = [vp, ctypes.POINTER(BieGeometry), i32, i32, vp, vp, vp]
    lib.apply_operator.restype = i32
    lib.apply_operator_fmm.argtypes = [vp, ctypes.POINTER(BieGeometry), i32, i32, vp, vp, vp]
    lib.apply_operator_fmm.restype = i32
    lib.bie_test_log.argtypes = [vp, vp, ctypes.c_int64, vp]
    lib.bie_test_log.restype = i32
    lib.apply_operator_fmm_prec.argtypes = [vp, ctypes.POINTER(BieGeometry), i32, i32, i32, vp, vp, vp]
    lib.apply_operator_fmm_prec.restype = i32
    lib.apply_operator_noalloc.argtypes = [ctypes.POINTER(BieGeometry), i32, i32, vp, vp, vp]
    lib.apply_operator_noalloc.restype = i32
    lib.bie_workspace_bytes.argtypes = [i32, i32, i32, i32]
    lib.bie_workspace_bytes.restype = ctypes.c_size_t
    lib.bie_server_create.argtypes = [ctypes.POINTER(vp), i32, i32, ctypes.c_size_t]
    lib.bie_server_create.restype = i32
    lib.bie_server_submit.argtypes = [vp, ctypes.POINTER(BieRequest), ctypes.POINTER(ctypes.c_int64)]
    lib.bie_server_submit.restype = i32
    lib.bie_server_wait.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(BieInfo), ctypes.POINTER(ctypes.c_double)]
    lib.bie_server_wait.restype = i32
    lib.bie_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t)]
    lib.bie_server_stats.restype = i32
    lib.bie_server_batching.argtypes = [vp, i32, i32, ctypes.POINTER(ctypes.c_int64)]
    lib.bie_server_batching.restype = i32
    lib.bie_server_destroy.argtypes = [vp]
    lib.bie_server_destroy.restype = None
    lib.bie_tune.argtypes = [vp, ctypes.POINTER(BieGeometry), i32, i32, ctypes.POINTER(i32),
                             ctypes.POINTER(ctypes.c_double), vp]
    lib.bie_tune.restype = i32
    lib.bie_tune_fmm.argtypes = [vp, ctypes.POINTER(BieGeometry), i32, vp, ctypes.POINTER(BieOpts),
                                 ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double), vp]
    lib.bie_tune_fmm.restype = i32
    lib.bie_tune_clear.argtypes = []
    lib.bie_tune_clear.restype = None
    lib.bie_profile.argtypes = [vp, i32, ctypes.POINTER(BieProfileCounters)]
    lib.bie_profile.restype = i32
    lib.bie_small_batch_path.argtypes = [i32]
    lib.bie_small_batch_path.restype = None
    lib.bie_measure_alu_peaks.argtypes = [i32, ctypes.POINTER(dbl)]
    lib.bie_measure_alu_peaks.restype = i32
    lib.bie_test_arm_barrier_timeout.argtypes = [i32, ctypes.c_longlong]
    lib.bie_test_arm_barrier_timeout.restype = None
    lib.bie_test_precond_pivot_floor.argtypes = [dbl]
    lib.bie_test_precond_pivot_floor.restype = None
    _ = dbl
    _LIB = lib
    return lib


def declared_symbols() -> list[str]:
    """Function names declared in include/bie2d.h."""
    with open(os.path.join(_build.INCLUDE, "bie2d.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^\s*(?:int|void|size_t|const char\*)\s+\**(\w+)\s*\(", text, flags=re.M)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def _check_dtypes(geom):
    for k in ("x", "y", "dx", "dy", "ddx", "ddy"):
        dt = str(geom[k].dtype)
        if "float64" not in dt:
            raise TypeError(f"geometry[{k!r}] must be float64, got {dt}")
    if "int32" not in str(geom["body_start"].dtype):
        raise TypeError("geometry['body_start'] must be int32")


def make_geometry(geom) -> tuple[BieGeometry, list]:
    """Build the C geometry struct from a dict of arrays; returns (struct, keepalive)."""
    _check_dtypes(geom)
    keep = [geom[k] for k in ("body_start", "x", "y", "dx", "dy", "ddx", "ddy")]
    ipt = geom.get("interior_pt")
    if ipt is not None:
        keep.append(ipt)
    g = BieGeometry(int(geom["body_start"].shape[0]) - 1, _ptr(geom["body_start"]),
                    _ptr(geom["x"]), _ptr(geom["y"]), _ptr(geom["dx"]), _ptr(geom["dy"]),
                    _ptr(geom["ddx"]), _ptr(geom["ddy"]), _ptr(ipt))
    return g, keep


def make_opts(tol=1e-12, max_iter=500, restart=50, precision=FP64, formulation=0,
              max_refine=8, inner_tol=1e-6, fmm_order=0, precond=0) -> BieOpts:
    return BieOpts(tol, max_iter, restart, precision, formulation, max_refine, inner_tol, fmm_order, precond)


class Context:
    """Owns a bie_ctx (device workspace) on one CUDA device."""

    def __init__(self, device: int = 0, workspace_cap_bytes: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        rc = self.lib.bie_create(ctypes.byref(h), device, workspace_cap_bytes)
        if rc != OK:
            raise RuntimeError(f"bie_create failed with status {rc}")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.bie_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self.lib.bie_last_error(self.handle).decode()

    def profile(self, enable: bool) -> dict:
        """bie_profile: returns the pair-sum timing counters so far, then (re)starts or stops timing."""
        c = BieProfileCounters()
        rc = self.lib.bie_profile(self.handle, 1 if enable else 0, ctypes.byref(c))
        if rc != OK:
            raise RuntimeError(f"bie_profile failed with status {rc}")
        return c.as_dict()


def elastance_solve(ctx: Context, geom, q, phi, density=None, opts: BieOpts | None = None, stream=None):
    """elastance_solve of include/bie2d.h; returns (status, info dict)."""
    g, keep = make_geometry(geom)
    info = BieInfo()
    rc = ctx.lib.elastance_solve(ctx.handle, ctypes.byref(g), _ptr(q), _ptr(phi), _ptr(density),
                                 ctypes.byref(opts) if opts is not None else None, ctypes.byref(info),
                                 _stream_ptr(stream))
    del keep
    return rc, info.as_dict()


def mobility_solve(ctx: Context, geom, FT, UW, density=None, opts: BieOpts | None = None, stream=None):
    """mobility_solve of include/bie2d.h; returns (status, info dict)."""
    g, keep = make_geometry(geom)
    info = BieInfo()
    rc = ctx.lib.mobility_solve(ctx.handle, ctypes.byref(g), _ptr(FT), _ptr(UW), _ptr(density),
                                ctypes.byref(opts) if opts is not None else None, ctypes.byref(info),
                                _stream_ptr(stream))
    del keep
    return rc, info.as_dict()


def _solve_batch(fn, ctx: Context, geoms, loads, outs, opts, stream):
    if not (len(geoms) == len(loads) == len(outs)) or len(geoms) == 0:
        raise ValueError("geoms, loads and outs must be non-empty lists of one length")
    P = len(geoms)
    built = [make_geometry(g) for g in geoms]
    arr = (BieGeometry * P)(*[b[0] for b in built])
    pl = (ctypes.c_void_p * P)(*[_ptr(x) for x in loads])
    po = (ctypes.c_void_p * P)(*[_ptr(x) for x in outs])
    infos = (BieInfo * P)()
    status = (ctypes.c_int32 * P)()
    rc = fn(ctx.handle, P, arr, pl, po, ctypes.byref(opts) if opts is not None else None,
            infos, status, _stream_ptr(stream))
    del built
    return rc, [i.as_dict() for i in infos], list(status)


def elastance_solve_batch(ctx: Context, geoms, qs, phis, opts: BieOpts | None = None, stream=None):
    """elastance_solve_batch of include/bie2d.h: lists of geometries, charges and
    potential outputs, solved together; returns (status of the batch, per-problem
    info dicts, per-problem statuses)."""
    return _solve_batch(ctx.lib.elastance_solve_batch, ctx, geoms, qs, phis, opts, stream)


def mobility_solve_batch(ctx: Context, geoms, FTs, UWs, opts: BieOpts | None = None, stream=None):
    """mobility_solve_batch of include/bie2d.h; returns (status of the batch,
    per-problem info dicts, per-problem statuses)."""
    return _solve_batch(ctx.lib.mobility_solve_batch, ctx, geoms, FTs, UWs, opts, stream)


def tune(ctx: Context, geom, kind: int, precision: int, splits: int = 0, stream=None):
    """bie_tune of include/bie2d.h: time the pair-sum grid on this geometry and keep
    the fastest split count for its shape (splits > 0: install that count
    untimed); returns (status, splits, ms)."""
    g, keep = make_geometry(geom)
    S = ctypes.c_int32(splits)
    ms = ctypes.c_double()
    rc = ctx.lib.bie_tune(ctx.handle, ctypes.byref(g), kind, precision, ctypes.byref(S), ctypes.byref(ms),
                          _stream_ptr(stream))
    del keep
    return rc, int(S.value), float(ms.value)


def test_arm_barrier_timeout(skip_cta: int, spins: int) -> None:
    """bie_test_arm_barrier_timeout: the next fused Arnoldi step skips CTA skip_cta
    and its barrier waits give up after `spins` polls (spins <= 0 disarms)."""
    load().bie_test_arm_barrier_timeout(skip_cta, spins)


def test_precond_pivot_floor(floor: float) -> None:
    """bie_test_precond_pivot_floor: block-Jacobi pivots below floor count as bad (<= 0: default)."""
    load().bie_test_precond_pivot_floor(floor)


test_arm_barrier_timeout.__test__ = False  # hooks, not tests: pytest must not collect them
test_precond_pivot_floor.__test__ = False


def small_batch_path(enable: bool) -> None:
    """bie_small_batch_path: one-launch solves of batches of small problems on or off."""
    load().bie_small_batch_path(1 if enable else 0)


def measure_alu_peaks(device: int = 0) -> dict:
    """bie_measure_alu_peaks: measured FP32 (FFMA, FFMA2), MUFU and FP64 rates of a device."""
    out = (ctypes.c_double * 4)()
    rc = load().bie_measure_alu_peaks(device, out)
    if rc != OK:
        raise RuntimeError(f"bie_measure_alu_peaks failed with status {rc}")
    return {"fp32_ffma_tflops": out[0], "fp32_ffma2_tflops": out[1], "mufu_rcp_tops": out[2],
            "fp64_dfma_tflops": out[3]}


def tune_fmm(ctx: Context, geom, kind: int, load, opts: BieOpts, stream=None):
    """bie_tune_fmm of include/bie2d.h: time whole FMM solves over leaf populations
    and inner orders, keep the fastest converged schedule for this shape;
    returns (status, leaf_nodes, inner_order, ms)."""
    g, keep = make_geometry(geom)
    leaf, inner, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    rc = ctx.lib.bie_tune_fmm(ctx.handle, ctypes.byref(g), kind, _ptr(load), ctypes.byref(opts), ctypes.byref(leaf),
                              ctypes.byref(inner), ctypes.byref(ms), _stream_ptr(stream))
    del keep
    return rc, int(leaf.value), int(inner.value), float(ms.value)


def tune_clear() -> None:
    """bie_tune_clear: forget every tuned split count."""
    load().bie_tune_clear()


def apply_operator(ctx: Context, geom, kind: int, precision: int, inp, out, stream=None) -> int:
    """apply_operator of include/bie2d.h: out = (1/2 I + K + L) inp; returns status."""
    g, keep = make_geometry(geom)
    rc = ctx.lib.apply_operator(ctx.handle, ctypes.byref(g), kind, precision, _ptr(inp), _ptr(out),
                                _stream_ptr(stream))
    del keep
    return rc


def apply_operator_noalloc(geom, kind: int, precision: int, inp, out, stream=None) -> int:
    """apply_operator_noalloc of include/bie2d.h (no context, no allocation; device arrays only)."""
    lib = load()
    g, keep = make_geometry(geom)
    rc = lib.apply_operator_noalloc(ctypes.byref(g), kind, precision, _ptr(inp), _ptr(out), _stream_ptr(stream))
    del keep
    return rc


def workspace_bytes(kind: int, n_bodies: int, n_nodes: int, restart: int = 0) -> int:
    """bie_workspace_bytes of include/bie2d.h."""
    return int(load().bie_workspace_bytes(kind, n_bodies, n_nodes, restart))


class Server:
    """bie_server: continuous batching of solve requests on one GPU."""

    def __init__(self, device: int = 0, workers: int = 4, hbm_cap_bytes: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        rc = self.lib.bie_server_create(ctypes.byref(h), device, workers, hbm_cap_bytes)
        if rc != OK:
            raise RuntimeError(f"bie_server_create failed with status {rc}")
        self.handle = h
        self._keep = {}

    def submit(self, kind: int, geom, load, out, density=None, opts: BieOpts | None = None) -> int:
        """Queue a request; returns its ticket (raises on a rejected request)."""
        g, keep = make_geometry(geom)
        req = BieRequest(kind, g, _ptr(load), _ptr(out), _ptr(density), opts if opts is not None else BieOpts())
        t = ctypes.c_int64()
        rc = self.lib.bie_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t))
        if rc != OK:
            return rc if rc < 0 else OK
        self._keep[t.value] = (keep, load, out, density)
        return int(t.value)

    def wait(self, ticket: int):
        """Block until the request completes; returns (status, info dict, seconds)."""
        info = BieInfo()
        sec = ctypes.c_double()
        rc = self.lib.bie_server_wait(self.handle, ticket, ctypes.byref(info), ctypes.byref(sec))
        self._keep.pop(ticket, None)
        return rc, info.as_dict(), sec.value

    def batching(self, max_batch: int = 0, max_request_nodes: int = 0) -> int:
        """bie_server_batching: set the batch limits (0 = unchanged); returns the
        number of batched solves run so far."""
        b = ctypes.c_int64()
        rc = self.lib.bie_server_batching(self.handle, max_batch, max_request_nodes, ctypes.byref(b))
        if rc != OK:
            raise ValueError(f"bie_server_batching failed with status {rc}")
        return int(b.value)

    def stats(self) -> dict:
        c, i, p = ctypes.c_int64(), ctypes.c_size_t(), ctypes.c_size_t()
        self.lib.bie_server_stats(self.handle, ctypes.byref(c), ctypes.byref(i), ctypes.byref(p))
        return dict(completed=c.value, inflight_bytes=i.value, peak_inflight_bytes=p.value)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.bie_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def apply_operator_fmm(ctx: Context, geom, kind: int, order: int, inp, out, stream=None) -> int:
    """apply_operator_fmm of include/bie2d.h: the operator with FMM pair sums of the given order."""
    g, keep = make_geometry(geom)
    rc = ctx.lib.apply_operator_fmm(ctx.handle, ctypes.byref(g), kind, order, _ptr(inp), _ptr(out),
                                    _stream_ptr(stream))
    del keep
    return rc


def test_log(x, out, stream=None) -> int:
    """bie_test_log: out[:n] = the output sums' table-driven log of x, out[n:] = CUDA's log."""
    return load().bie_test_log(_ptr(x), _ptr(out), int(x.numel()), _stream_ptr(stream))


test_log.__test__ = False


def apply_operator_fmm_prec(ctx: Context, geom, kind: int, order: int, precision: int, inp, out,
                            stream=None) -> int:
    """apply_operator_fmm_prec of include/bie2d.h: the FMM operator in a solve precision's arithmetic."""
    g, keep = make_geometry(geom)
    rc = ctx.lib.apply_operator_fmm_prec(ctx.handle, ctypes.byref(g), kind, order, precision, _ptr(inp),
                                         _ptr(out), _stream_ptr(stream))
    del keep
    return rc
