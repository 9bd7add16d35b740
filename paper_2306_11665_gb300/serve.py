"""Thin wrapper of the serving ABI (sfh_server_*): resident device arrays in,
tickets out.  All scheduling happens in the library (host admission thread +
persistent kernel)."""
from __future__ import annotations

import torch

from . import _abi as A


class Server:
    def __init__(self, hbm_budget_bytes: int = 40 << 30, max_inflight: int = 32, timeout_ms: int = 20000,
                 n_workers: int = 0):
        self.handle = A.sfh_server_create(hbm_budget_bytes, max_inflight, timeout_ms, n_workers)
        self._keep = {}

    def submit(self, kind: int, p: int, nodes: int, prec: int, u: torch.Tensor, Ja: torch.Tensor,
               out: torch.Tensor, lam: torch.Tensor | None = None, sync: bool = True,
               flux: int = A.SFH_FLUX_EULER_RANOCHA) -> int:
        """Queue one request; the tensors must stay alive and unchanged until it
        is done.  The server's kernel is not ordered after torch's streams, so
        by default the current stream is synchronized first (work that wrote
        the inputs, or that still uses `out`, completes before the queueing)."""
        if sync:
            torch.cuda.current_stream(u.device).synchronize()
        req = A.Request(kind, p, nodes, prec, u.shape[0], u.data_ptr(), Ja.data_ptr(),
                        lam.data_ptr() if lam is not None else None, out.data_ptr(), flux)
        t = A.sfh_serve_submit(self.handle, req)
        self._keep[t] = (u, Ja, out, lam)
        return t

    def poll(self, ticket: int):
        """The request's Result once it is done, else None."""
        res = A.sfh_serve_poll(self.handle, ticket)
        if res is not None:
            self._keep.pop(ticket, None)
        return res

    def drain(self, timeout_ms: int = 20000) -> None:
        A.sfh_serve_drain(self.handle, timeout_ms)

    def close(self) -> None:
        if getattr(self, "handle", None):
            A.sfh_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
