"""ctypes binding of libsfhad's C ABI (include/sfhad.h).

Argument marshalling only: every function here forwards to the C entry point
of the same name and raises :class:`SfhError` on a non-OK status.  The
library must have been built (``python -m paper_2306_11665_gb300.build`` or
``__graft_entry__.build()``); loading fails loudly otherwise -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# SFH_LIB_VARIANT=debug loads the bounds-checked debug build instead
LIB_VARIANT = os.environ.get("SFH_LIB_VARIANT", "")
if LIB_VARIANT not in ("", "release", "debug"):
    raise RuntimeError(f"SFH_LIB_VARIANT must be 'release' or 'debug', got {LIB_VARIANT!r}")
LIB_PATH = os.path.join(HERE, "libsfhad_debug.so" if LIB_VARIANT == "debug" else "libsfhad.so")

# enums (mirror include/sfhad.h)
SFH_OK, SFH_EINVAL, SFH_ENOMEM, SFH_ECUDA, SFH_EDOMAIN = 0, 1, 2, 3, 4
SFH_EBUSY, SFH_ENOTREADY, SFH_ETIMEOUT, SFH_EUNSUPPORTED, SFH_EBOUNDS = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "SFH_OK", 1: "SFH_EINVAL", 2: "SFH_ENOMEM", 3: "SFH_ECUDA", 4: "SFH_EDOMAIN",
                5: "SFH_EBUSY", 6: "SFH_ENOTREADY", 7: "SFH_ETIMEOUT", 8: "SFH_EUNSUPPORTED",
                9: "SFH_EBOUNDS"}
SFH_BUILD_DEBUG = 1
SFH_NODES_GLL, SFH_NODES_GAUSS = 0, 1
SFH_FLUX_BURGERS, SFH_FLUX_EULER_RANOCHA, SFH_FLUX_EULER_CHANDRASHEKAR = 0, 1, 2
SFH_FP64, SFH_FP32_KAHAN, SFH_FP32_MIXED = 0, 1, 2
SFH_BASIS_LEGENDRE, SFH_BASIS_LAGRANGE_GLL, SFH_BASIS_LAGRANGE_GAUSS = 0, 1, 2
SFH_REQ_RESIDUAL, SFH_REQ_VJP = 0, 1
SFH_FAULT_CREATE_ALLOC, SFH_FAULT_DROP_TILE, SFH_FAULT_STALL_ADMISSION = 1, 2, 3


class SfhError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("timeout_ms", ctypes.c_int), ("n_workers", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("p", ctypes.c_int), ("nodes", ctypes.c_int), ("prec", ctypes.c_int),
                ("n_elem", ctypes.c_int64), ("u", ctypes.c_void_p), ("Ja", ctypes.c_void_p),
                ("lambda_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("flux", ctypes.c_int)]

    def __init__(self, *args, **kw):
        # the flux field comes last; a request built without it is Ranocha's
        if len(args) < len(self._fields_):
            kw.setdefault("flux", SFH_FLUX_EULER_RANOCHA)
        super().__init__(*args, **kw)


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("t_submit_ns", ctypes.c_uint64), ("t_admit_ns", ctypes.c_uint64),
                ("t_start_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64)]


class ServeStats(ctypes.Structure):
    _fields_ = [("tiles", ctypes.c_uint64 * 4), ("busy_ns", ctypes.c_uint64 * 4), ("claim_ns", ctypes.c_uint64)]


_lib = None
vp, i64, dp, ip = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "sfh_create": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)],
    "sfh_destroy": [vp],
    "sfh_volume_residual": [vp, i64, vp, vp, vp, ctypes.c_int, vp],
    "sfh_volume_residual_modal": [vp, ctypes.c_int, i64, vp, vp, vp, ctypes.c_int, vp],
    "sfh_basis_table": [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp],
    "sfh_vjp_modal": [vp, ctypes.c_int, i64, vp, vp, vp, vp, vp],
    "sfh_surface_hadamard": [vp, i64, vp, vp, vp, vp, vp, vp],
    "sfh_vjp": [vp, i64, vp, vp, vp, vp, vp],
    "sfh_check": [vp, vp],
    "sfh_volume_residual_host": [vp, i64, vp, vp, vp, ctypes.c_int],
    "sfh_ctx_info": [vp, ip, ip, ip, ip, ip, ip],
    "sfh_volume_residual_host_noalloc": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, vp, vp, vp,
                                         ctypes.c_int, vp],
    "sfh_operator_tables": [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp],
    "sfh_peak_fma": [ctypes.c_int, dp, dp],
    "sfh_entropy_residual": [vp, i64, vp, vp, vp, ctypes.c_int, vp, vp],
    "sfh_fig1_hadamard": [ctypes.c_int, i64, vp, vp, ctypes.c_int, vp],
    "sfh_selftest_bounded_wait": [ctypes.c_int64, ctypes.c_void_p, dp],
    "sfh_selftest_bounds": [ctypes.c_void_p],
    "sfh_bind_metric": [vp, ctypes.c_int64, ctypes.c_void_p],
    "sfh_volume_residual_host_bound": [vp, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "sfh_build_flags": [],
    "sfh_server_create": [ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)],
    "sfh_serve_submit": [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)],
    "sfh_serve_poll": [vp, ctypes.c_uint64, ctypes.POINTER(Result)],
    "sfh_serve_drain": [vp, ctypes.c_int],
    "sfh_serve_stats": [vp, ctypes.POINTER(ServeStats)],
    "sfh_serve_replay": [vp, ctypes.c_int, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(Result), ctypes.c_int],
    "sfh_server_destroy": [vp],
    "sfh_serial_replay": [ctypes.c_int, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(Result), ctypes.c_int],
    "sfh_serve_inject_fault": [vp, ctypes.c_int, ctypes.c_int],
}


def lib():
    """The loaded libsfhad (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsfhad is not built ({LIB_PATH} missing); run "
                               "`python -m paper_2306_11665_gb300.build` first")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.sfh_last_error.argtypes = []
        L.sfh_last_error.restype = ctypes.c_char_p
        L.sfh_version.argtypes = []
        L.sfh_version.restype = ctypes.c_int
        _lib = L
    return _lib


def sfh_last_error() -> str:
    return lib().sfh_last_error().decode()


def sfh_version() -> int:
    return lib().sfh_version()


def _call(name, *args, ok=(SFH_OK,)):
    st = getattr(lib(), name)(*args)
    if st not in ok:
        raise SfhError(st, name, sfh_last_error())
    return st


def sfh_create(d: int, p: int, nodes: int, nvar: int, flux: int) -> int:
    out = vp()
    _call("sfh_create", d, p, nodes, nvar, flux, ctypes.byref(out))
    return out.value


def sfh_destroy(ctx: int) -> None:
    _call("sfh_destroy", ctx)


def sfh_volume_residual(ctx: int, n_elem: int, u: int, Ja: int, r: int, prec: int, stream: int = 0) -> None:
    _call("sfh_volume_residual", ctx, n_elem, u, Ja, r, prec, stream)


def sfh_volume_residual_modal(ctx: int, basis: int, n_elem: int, u_hat: int, Ja: int, r_hat: int, prec: int,
                              stream: int = 0) -> None:
    _call("sfh_volume_residual_modal", ctx, basis, n_elem, u_hat, Ja, r_hat, prec, stream)


def sfh_vjp_modal(ctx: int, basis: int, n_elem: int, u_hat: int, Ja: int, lam_hat: int, grad_hat: int,
                  stream: int = 0) -> None:
    _call("sfh_vjp_modal", ctx, basis, n_elem, u_hat, Ja, lam_hat, grad_hat, stream)


def sfh_surface_hadamard(ctx: int, n_elem: int, u: int, u_face: int, nJ_face: int, r_vol: int, r_face: int,
                         stream: int = 0) -> None:
    _call("sfh_surface_hadamard", ctx, n_elem, u, u_face, nJ_face, r_vol, r_face, stream)


def sfh_basis_table(p: int, nodes: int, basis: int):
    import numpy as np
    V = np.zeros((p + 1, p + 1))
    _call("sfh_basis_table", p, nodes, basis, V.ctypes.data_as(dp))
    return V


def sfh_vjp(ctx: int, n_elem: int, u: int, Ja: int, lam: int, grad_u: int, stream: int = 0) -> None:
    _call("sfh_vjp", ctx, n_elem, u, Ja, lam, grad_u, stream)


def sfh_check(ctx: int, stream: int = 0) -> int:
    """Returns the status (SFH_OK or SFH_EDOMAIN); raises on other errors."""
    return _call("sfh_check", ctx, stream, ok=(SFH_OK, SFH_EDOMAIN))


def sfh_volume_residual_host(ctx: int, n_elem: int, u_host: int, Ja_host: int, r_host: int, prec: int) -> int:
    return _call("sfh_volume_residual_host", ctx, n_elem, u_host, Ja_host, r_host, prec, ok=(SFH_OK, SFH_EDOMAIN))


def sfh_volume_residual_host_noalloc(d: int, p: int, nodes: int, flux: int, n_elem: int, u_host: int,
                                     Ja_host: int, r_host: int, prec: int, stream: int = 0) -> int:
    """Context-free, allocation-free host-buffer residual (returns the status;
    SFH_OK or SFH_EDOMAIN; raises on other errors)."""
    return _call("sfh_volume_residual_host_noalloc", d, p, nodes, flux, n_elem, u_host, Ja_host, r_host, prec, stream,
                 ok=(SFH_OK, SFH_EDOMAIN))


def sfh_ctx_info(ctx: int) -> dict:
    vals = [ctypes.c_int() for _ in range(6)]
    _call("sfh_ctx_info", ctx, *[ctypes.byref(v) for v in vals])
    return dict(zip(("d", "p", "nodes", "nvar", "flux", "n_nodes"), (v.value for v in vals)))


def sfh_operator_tables(p: int, nodes: int):
    import numpy as np
    n = p + 1
    xi, w, D, Q1 = np.zeros(n), np.zeros(n), np.zeros((n, n)), np.zeros((n, n))
    c = lambda a: a.ctypes.data_as(dp)  # noqa: E731
    _call("sfh_operator_tables", p, nodes, c(xi), c(w), c(D), c(Q1))
    return xi, w, D, Q1


def sfh_entropy_residual(ctx: int, n_elem: int, u: int, Ja: int, r: int, r_prec: int, out: int, stream: int = 0):
    _call("sfh_entropy_residual", ctx, n_elem, u, Ja, r, r_prec, out, stream)


def sfh_fig1_hadamard(p: int, n_elem: int, c: int, y: int, dense: bool, stream: int = 0):
    _call("sfh_fig1_hadamard", p, n_elem, c, y, 1 if dense else 0, stream)


def sfh_peak_fma(prec: int):
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _call("sfh_peak_fma", prec, ctypes.byref(tf), ctypes.byref(ms))
    return tf.value, ms.value


def sfh_bind_metric(ctx: int, n_elem: int, Ja_host: int):
    _call("sfh_bind_metric", ctx, n_elem, Ja_host)


def sfh_volume_residual_host_bound(ctx: int, n_elem: int, u_host: int, r_host: int, prec: int) -> int:
    return _call("sfh_volume_residual_host_bound", ctx, n_elem, u_host, r_host, prec, ok=(SFH_OK, SFH_EDOMAIN))


def sfh_build_flags() -> int:
    return lib().sfh_build_flags()


def sfh_selftest_bounds(stream: int = 0) -> int:
    """Status of the debug build's bounds self-test (SFH_OK or, in the release
    library, SFH_EUNSUPPORTED)."""
    return _call("sfh_selftest_bounds", stream, ok=(SFH_OK, SFH_EUNSUPPORTED))


def sfh_selftest_bounded_wait(limit_us: int, stream: int = 0):
    """Runs the bounded-wait self-test; returns (status, elapsed_us).  The
    expected status is SFH_ETIMEOUT."""
    el = ctypes.c_double()
    st = _call("sfh_selftest_bounded_wait", limit_us, stream, ctypes.byref(el), ok=(SFH_OK, SFH_ETIMEOUT))
    return st, el.value


def sfh_server_create(hbm_budget_bytes: int, max_inflight: int, timeout_ms: int, n_workers: int = 0) -> int:
    opts = ServerOpts(hbm_budget_bytes, max_inflight, timeout_ms, n_workers)
    out = vp()
    _call("sfh_server_create", ctypes.byref(opts), ctypes.byref(out))
    return out.value


def sfh_serve_submit(srv: int, req: Request) -> int:
    t = ctypes.c_uint64()
    _call("sfh_serve_submit", srv, ctypes.byref(req), ctypes.byref(t))
    return t.value


def sfh_serve_poll(srv: int, ticket: int):
    """Result (done) or None (not ready)."""
    res = Result()
    st = _call("sfh_serve_poll", srv, ticket, ctypes.byref(res), ok=(SFH_OK, SFH_ENOTREADY))
    return res if st == SFH_OK else None


def sfh_serve_replay(srv: int, reqs, arrival_s, timeout_ms: int):
    """Replay requests (a list of Request) at the given arrival times; returns the Results."""
    n = len(reqs)
    R = (Request * n)(*reqs)
    T = (ctypes.c_double * n)(*arrival_s)
    out = (Result * n)()
    _call("sfh_serve_replay", srv, n, R, T, out, timeout_ms)
    return list(out)


def sfh_serial_replay(reqs, arrival_s, timeout_ms: int):
    """The serving baseline: the requests as plain FIFO launches on one stream,
    each enqueued at its arrival time; returns the Results."""
    n = len(reqs)
    R = (Request * n)(*reqs)
    T = (ctypes.c_double * n)(*arrival_s)
    out = (Result * n)()
    _call("sfh_serial_replay", n, R, T, out, timeout_ms)
    return list(out)


def sfh_serve_inject_fault(srv, kind: int, arg: int) -> None:
    """Test hook: host-side fault injection into the server (header)."""
    _call("sfh_serve_inject_fault", srv, kind, arg)


def sfh_serve_drain(srv: int, timeout_ms: int) -> None:
    _call("sfh_serve_drain", srv, timeout_ms)


def sfh_serve_stats(srv: int) -> dict:
    """Serving-kernel counters: per class (fp64, fp32k, mixed, vjp) tiles and
    busy seconds, and the seconds CTAs spent claiming tiles."""
    st = ServeStats()
    _call("sfh_serve_stats", srv, ctypes.byref(st))
    names = ("fp64", "fp32k", "fp32mix", "vjp")
    return {"tiles": {n: int(st.tiles[k]) for k, n in enumerate(names)},
            "busy_s": {n: st.busy_ns[k] * 1e-9 for k, n in enumerate(names)},
            "claim_s": st.claim_ns * 1e-9}


def sfh_server_destroy(srv: int) -> None:
    _call("sfh_server_destroy", srv)
