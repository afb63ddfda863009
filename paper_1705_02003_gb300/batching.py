"""Batching layer: many samples with uneven iteration counts through one GPU.

``solve_stream`` runs the continuous ensemble batching of ens_solve_stream
(frozen lanes take the next queued sample; the drained pool is re-packed).
``autotune`` picks the ensemble size S for a fixed lane capacity, and
``autotune_chunk`` the trips per launch between harvests for that S, by timing
each candidate on a bounded sample of the workload.
"""
from __future__ import annotations

import torch

from . import ens


def solve_stream(h: ens.Handle, prob: ens.Problem, xi: torch.Tensor, S: int, E: int, rtol: float, maxit: int,
                 chunk: int = 64, order: torch.Tensor | None = None, weights: torch.Tensor | None = None,
                 work: torch.Tensor | None = None, want_qoi: bool = True):
    """Solve every row of xi [M][N] (device f64); returns per-sample tensors."""
    M = xi.shape[0]
    dev = xi.device
    iters = torch.empty(M, dtype=torch.int32, device=dev)
    status = torch.empty(M, dtype=torch.int32, device=dev)
    relres = torch.empty(M, dtype=torch.float64, device=dev)
    qoi = torch.empty(M, dtype=torch.float64, device=dev) if want_qoi else None
    ens.ens_solve_stream(h, prob, S, E, xi.contiguous(), order, rtol, maxit, chunk, iters, status, relres, qoi=qoi,
                         w=weights, work=work)
    return dict(iters=iters, status=status, relres=relres, qoi=qoi)


def _time_stream(h, prob, xi, S, E, rtol, maxit, chunk, stream):
    work = torch.empty(ens.ens_stream_workspace_size(prob, S, E), dtype=torch.uint8, device=xi.device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    solve_stream(h, prob, xi, S, E, rtol, maxit, chunk=chunk, work=work, want_qoi=False)
    e1.record(stream)
    torch.cuda.synchronize()
    del work
    return e0.elapsed_time(e1) / 1e3


def autotune(h: ens.Handle, prob: ens.Problem, xi: torch.Tensor, lanes: int, rtol: float, maxit: int,
             chunk: int = 64, candidates=(8, 16, 32, 64), stream=None):
    """Time solve_stream on xi for each S with E = lanes / S; return (best S, {S: seconds})."""
    stream = torch.cuda.current_stream() if stream is None else stream
    times = {}
    for S in candidates:
        if lanes % S:
            continue
        times[S] = _time_stream(h, prob, xi, S, lanes // S, rtol, maxit, chunk, stream)
    best = min(times, key=times.get)
    return best, times


def autotune_chunk(h: ens.Handle, prob: ens.Problem, xi: torch.Tensor, lanes: int, S: int, rtol: float,
                   maxit: int, candidates=(16, 32, 64, 128), stream=None):
    """The trips per launch between harvests and re-packs for a given S (any
    chunk gives the same per-sample results; it trades host round trips
    against lanes idling until the next harvest).  Returns (best, {chunk: s})."""
    stream = torch.cuda.current_stream() if stream is None else stream
    times = {c: _time_stream(h, prob, xi, S, lanes // S, rtol, maxit, c, stream) for c in candidates}
    best = min(times, key=times.get)
    return best, times
