"""Serving front end: a seeded request mix and an open-loop driver for the continuous-batching
server of libstencil (stencil_server_*), plus the plain per-grid path it is compared with.

The request mix follows the serving configuration: grid sizes n log-uniform in [32, 192]
(rounded to a multiple of 8 so that one input template per kind and size can be kept in
page-locked memory; with round_to=1 the sizes are not rounded, and an input of a ragged size
is the leading n^3 block of the template of the next multiple of 8), kinds uniform over
{1D cross-correlation of n^3 cells, 3D heat equation, 8-field MHD system}, 10..50 steps each,
FP32, Poisson arrivals.  Latency is
measured open-loop: from a request's scheduled arrival time to the moment its result is in
host memory.

Every step of every request runs in the library's CUDA kernels; this module only generates
inputs, submits, polls and times.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import _lib as L
from . import synth

KINDS = (L.STENCIL_XCORR, L.STENCIL_DIFFUSION, L.STENCIL_MHD8)
KIND_NAMES = {L.STENCIL_XCORR: "xcorr1d", L.STENCIL_DIFFUSION: "heat3d", L.STENCIL_MHD8: "mhd8"}
SEED_SERVE = 2406089235
# 1D cross-correlation weights for serving: one forward-Euler diffusion step with dt = 0.1 (dx = 1),
# i.e. delta + 0.1 * (6th-order 2nd-derivative weights); stable over any number of sweeps.
XC_WEIGHTS = tuple([0.1 * c for c in (1 / 90, -3 / 20, 3 / 2)] + [1.0 + 0.1 * (-49 / 18)] +
                   [0.1 * c for c in (3 / 2, -3 / 20, 1 / 90)])


@dataclass
class Request:
    index: int
    kind: int
    n: int
    nsteps: int
    arrival: float = 0.0          # scheduled arrival, seconds from the start of the run
    ticket: int = 0
    done_at: float = math.nan     # seconds from the start
    out: list = field(default_factory=list)

    @property
    def nfields(self):
        return 8 if self.kind == L.STENCIL_MHD8 else 1

    @property
    def cells(self):
        return self.n ** 3

    @property
    def shape(self):
        return (self.n ** 3,) if self.kind == L.STENCIL_XCORR else (self.n, self.n, self.n)

    def work(self):
        """Cell updates (MHD counted per RK substep, as the paper's Table 3)."""
        return self.cells * self.nsteps * (3 if self.kind == L.STENCIL_MHD8 else 1)


def make_requests(count=1024, seed=SEED_SERVE, nmin=32, nmax=192, smin=10, smax=50, round_to=8):
    u = synth.uniform(seed, 1, count, math.log(nmin), math.log(nmax))
    n = np.clip(np.round(np.exp(u) / round_to) * round_to, nmin, nmax).astype(int)
    kinds = synth.integers(seed, 2, count, 0, 2)
    steps = synth.integers(seed, 3, count, smin, smax)
    return [Request(i, KINDS[int(kinds[i])], int(n[i]), int(steps[i])) for i in range(count)]


def poisson_arrivals(reqs, rate_per_s, seed=SEED_SERVE):
    gaps = -np.log(np.maximum(synth.uniform(seed, 4, len(reqs)), 1e-300)) / rate_per_s
    t = np.cumsum(gaps) - gaps[0]
    for r, a in zip(reqs, t):
        r.arrival = float(a)
    return reqs


def request_params(kind, n, nsteps=1):
    """stencil_request for one problem of the serving mix."""
    q = L.stencil_request()
    q.kind = kind
    q.nsteps = nsteps
    if kind == L.STENCIL_XCORR:
        q.dims[0], q.dims[1], q.dims[2] = n ** 3, 1, 1
        for j, w in enumerate(XC_WEIGHTS):
            q.coeffs[j] = w
    else:
        q.dims[0] = q.dims[1] = q.dims[2] = n
        q.params = L.heat_params(n) if kind == L.STENCIL_DIFFUSION else L.mhd_params(n)
    return q


class Templates:
    """One page-locked FP32 input template per (kind, n), generated on first use."""

    def __init__(self, pinned=True):
        self.pinned = pinned
        self.cache = {}

    def get(self, kind, n):
        key = (kind, n)
        if key not in self.cache and n % 8:
            import torch
            m = (n + 7) // 8 * 8
            base = self.get(kind, m)
            ts = []
            for t in base:
                blk = t[:n ** 3] if kind == L.STENCIL_XCORR else t.view(m, m, m)[:n, :n, :n]
                c = blk.contiguous().clone()
                ts.append(c.pin_memory() if self.pinned else c)
            self.cache[key] = ts
        if key not in self.cache:
            import torch
            if kind == L.STENCIL_XCORR:
                arrs = [synth.uniform(SEED_SERVE + n, 5, n ** 3, -1.0, 1.0)]
            elif kind == L.STENCIL_DIFFUSION:
                arrs = [synth.heat_field(n, seed=SEED_SERVE + n)]
            else:
                arrs = list(synth.mhd_fields(n, seed=SEED_SERVE + n))
            ts = []
            for a in arrs:
                t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel())
                ts.append(t.pin_memory() if self.pinned else t)
            self.cache[key] = ts
        return self.cache[key]


class OutputPool:
    """Page-locked output buffers recycled by size."""

    def __init__(self):
        self.free = {}

    def take(self, nelem, count):
        import torch
        lst = self.free.setdefault(nelem, [])
        out = []
        for _ in range(count):
            out.append(lst.pop() if lst else torch.empty(nelem, dtype=torch.float32).pin_memory())
        return out

    def give(self, bufs):
        for b in bufs:
            self.free.setdefault(b.numel(), []).append(b)


def serve(reqs, templates, budget_bytes=120 * 10 ** 9, max_active=4096, keep_outputs=False, time_limit=600.0,
          stream=None):
    """Open-loop run: submit each request at its arrival time, drive the server until all are
    done.  Returns (wall seconds, peak bytes, server cell updates)."""
    server = L.stencil_server_create(budget_bytes, max_active, stream)
    pool = OutputPool()
    inflight = {}
    order = sorted(reqs, key=lambda r: r.arrival)
    i = 0
    t0 = time.perf_counter()
    try:
        while i < len(order) or inflight:
            now = time.perf_counter() - t0
            if now > time_limit:
                raise RuntimeError(f"serving run exceeded {time_limit} s")
            while i < len(order) and order[i].arrival <= now:
                r = order[i]
                ins = templates.get(r.kind, r.n)
                r.out = pool.take(r.cells, r.nfields)
                r.ticket = L.stencil_server_submit(server, request_params(r.kind, r.n, r.nsteps), [t.data_ptr() for t in ins],
                                                   [t.data_ptr() for t in r.out])
                inflight[r.ticket] = r
                i += 1
            # the server steps every active request by one
            pend, act, _ = L.stencil_server_progress(server)
            now = time.perf_counter() - t0
            for tk in list(inflight):
                if L.stencil_server_poll(server, tk) == L.STENCIL_REQ_DONE:
                    r = inflight.pop(tk)
                    r.done_at = now
                    if not keep_outputs:
                        pool.give(r.out)
                        r.out = []
            if not inflight and i < len(order):
                time.sleep(max(0.0, order[i].arrival - (time.perf_counter() - t0)))
        wall = time.perf_counter() - t0
        L.stencil_server_sync(server)
        used, peak, updates = L.stencil_server_stats(server)
    finally:
        L.stencil_server_destroy(server)
    return wall, peak, updates


def latency_stats(reqs):
    lat = np.array([r.done_at - r.arrival for r in reqs])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}


def serve_per_grid(reqs, templates, storage=L.STENCIL_F64):
    """The plain path: each request alone, in arrival order, through its own plan
    (stencil_create, upload, stencil_step(nsteps), download).  Returns wall seconds."""
    import torch
    t0 = time.perf_counter()
    for r in sorted(reqs, key=lambda r: r.arrival):
        ins = templates.get(r.kind, r.n)
        compute = storage if storage != L.STENCIL_BF16 else L.STENCIL_F32
        if r.kind == L.STENCIL_XCORR:
            p = L.Plan(1, (r.n ** 3,), 3, 1, L.STENCIL_BC_PERIODIC, L.STENCIL_XCORR, storage, compute,
                       coeffs=np.array(XC_WEIGHTS))
        elif r.kind == L.STENCIL_DIFFUSION:
            p = L.Plan(3, (r.n,) * 3, 3, 1, L.STENCIL_BC_PERIODIC, L.STENCIL_DIFFUSION, storage, compute,
                       params=L.heat_params(r.n))
        else:
            p = L.Plan(3, (r.n,) * 3, 3, 8, L.STENCIL_BC_PERIODIC, L.STENCIL_MHD8, storage, compute,
                       params=L.mhd_params(r.n))
        a, b = p.alloc(), p.alloc()
        for t, src in zip(a, ins):
            p.interior(t).copy_(src.view(r.shape).to(p.torch_dtype))
        p.step(a, b, r.nsteps)
        r.out = [p.interior(t).float().cpu() for t in b]
        r.done_at = time.perf_counter() - t0
        p.close()
        del a, b
    torch.cuda.synchronize()
    return time.perf_counter() - t0
