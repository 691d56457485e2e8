"""Continuous-batching server (stencil_server_*).

* Each result is the same alone and in the mix: a staggered mix of small problems of all
  three kinds runs through one server; every problem is then run alone through a fresh
  server (bit-identical expected) and through the plain per-grid plan path (FP32, within the
  FP32 tolerance), and heat / cross-correlation results are checked against the FP64 oracle.
* Admission respects the HBM budget: with a budget that holds only part of the mix, the
  peak never exceeds it and every problem still completes.
* Malformed requests are rejected with STENCIL_EINVAL.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_close, oracle_mhd_params
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import serving

pytestmark = pytest.mark.gpu


def _mix():
    spec = [(L.STENCIL_MHD8, 16, 3), (L.STENCIL_DIFFUSION, 24, 7), (L.STENCIL_XCORR, 16, 9),
            (L.STENCIL_DIFFUSION, 32, 4), (L.STENCIL_MHD8, 24, 2), (L.STENCIL_XCORR, 24, 5),
            (L.STENCIL_DIFFUSION, 16, 11), (L.STENCIL_MHD8, 8, 5), (L.STENCIL_XCORR, 32, 3),
            (L.STENCIL_DIFFUSION, 40, 2), (L.STENCIL_MHD8, 32, 1), (L.STENCIL_XCORR, 8, 12),
            # sizes that are not multiples of 4: scalar x-image stores in the batched heat kernel
            (L.STENCIL_DIFFUSION, 21, 3), (L.STENCIL_MHD8, 13, 2), (L.STENCIL_XCORR, 11, 4)]
    reqs = [serving.Request(i, k, n, s) for i, (k, n, s) in enumerate(spec)]
    for i, r in enumerate(reqs):
        r.arrival = 0.002 * (i % 4)  # some arrive while others are already stepping
    return reqs


def _alone(r, templates):
    rr = serving.Request(0, r.kind, r.n, r.nsteps)
    serving.serve([rr], templates, keep_outputs=True)
    return [t.numpy().copy() for t in rr.out]


def test_results_same_alone_and_in_the_mix(cuda_lib):
    templates = serving.Templates(pinned=True)
    reqs = _mix()
    serving.serve(reqs, templates, keep_outputs=True)
    for r in reqs:
        mixed = [t.numpy().copy() for t in r.out]
        alone = _alone(r, templates)
        for q in range(r.nfields):
            assert np.array_equal(mixed[q], alone[q]), (serving.KIND_NAMES[r.kind], r.n, q)
        # plain per-grid path in FP32
        plain = [serving.Request(0, r.kind, r.n, r.nsteps)]
        serving.serve_per_grid(plain, templates, storage=L.STENCIL_F32)
        for q in range(r.nfields):
            assert_close(mixed[q], plain[0].out[q].numpy().ravel(), 1e-5, f"{serving.KIND_NAMES[r.kind]} n={r.n}")
        # FP64 oracle for the linear kinds
        ins = [t.numpy().astype(np.float64) for t in templates.get(r.kind, r.n)]
        if r.kind == L.STENCIL_XCORR:
            ref = oracle.xcorr1d(ins[0], np.array(serving.XC_WEIGHTS), r.nsteps)
            assert_close(mixed[0], ref, 1e-5, "xcorr vs oracle")
        elif r.kind == L.STENCIL_DIFFUSION:
            par = L.heat_params(r.n)
            h = (par.dx[0], par.dx[1], par.dx[2])
            ref = oracle.diffusion(ins[0].reshape(r.shape), par.dt, par.alpha, h, r.nsteps)
            assert_close(mixed[0], ref.ravel(), 1e-5, "heat vs oracle")
        else:
            par = L.mhd_params(r.n)
            ref = oracle.mhd_rk3(np.stack([a.reshape(r.shape) for a in ins]), oracle_mhd_params(par), par.dt,
                                 r.nsteps)
            for q in range(8):
                assert_close(mixed[q], ref[q].ravel(), 1e-5, f"mhd field {q} vs oracle")


def test_admission_respects_budget(cuda_lib):
    templates = serving.Templates(pinned=True)
    reqs = [serving.Request(i, L.STENCIL_MHD8, 24, 3) for i in range(6)]
    for r in reqs:
        r.arrival = 0.0
    one = 2 * 8 * 4 * (24 + 8) * 30 * 30 + 16 * 4 * 24 ** 3  # rough size of one problem
    budget = int(2.5 * one)
    wall, peak, updates = serving.serve(reqs, templates, budget_bytes=budget)
    assert peak <= budget
    assert all(np.isfinite(r.done_at) for r in reqs)
    assert updates == sum(r.cells * r.nsteps for r in reqs)


def test_malformed_requests_rejected(cuda_lib):
    server = L.stencil_server_create(10 ** 9, 16)
    try:
        x = torch.zeros(512, dtype=torch.float32).pin_memory()
        q = serving.request_params(L.STENCIL_DIFFUSION, 8, 2)
        q.dims[0] = 5  # below 2r+1
        with pytest.raises(L.StencilError) as e:
            L.stencil_server_submit(server, q, [x.data_ptr()], [x.data_ptr()])
        assert e.value.status == L.STENCIL_EINVAL
        q = serving.request_params(L.STENCIL_DIFFUSION, 8)
        q.nsteps = 0
        with pytest.raises(L.StencilError):
            L.stencil_server_submit(server, q, [x.data_ptr()], [x.data_ptr()])
        big = serving.request_params(L.STENCIL_MHD8, 400, 2)  # more than the whole budget
        with pytest.raises(L.StencilError):
            L.stencil_server_submit(server, big, [x.data_ptr()] * 8, [x.data_ptr()] * 8)
    finally:
        L.stencil_server_destroy(server)


def test_cancel_pending_and_active(cuda_lib):
    # a cancelled problem leaves the queue (pending) or the batch (active), its memory returns to
    # the pool, its host output is never written, and the other problems still finish correctly
    n, steps = 16, 6
    templates = serving.Templates(pinned=True)
    src = templates.get(L.STENCIL_DIFFUSION, n)[0]
    outs = [torch.full((n ** 3,), -7.0, dtype=torch.float32).pin_memory() for _ in range(4)]
    server = L.stencil_server_create(10 ** 9, 2)  # two slots: requests 2 and 3 wait
    try:
        q = serving.request_params(L.STENCIL_DIFFUSION, n, steps)
        tickets = [L.stencil_server_submit(server, q, [src.data_ptr()], [o.data_ptr()]) for o in outs]
        L.stencil_server_cancel(server, tickets[3])  # pending
        assert L.stencil_server_poll(server, tickets[3]) == L.STENCIL_REQ_CANCELLED
        L.stencil_server_progress(server)  # admits 0 and 1, one step each
        assert L.stencil_server_poll(server, tickets[0]) == L.STENCIL_REQ_ACTIVE
        L.stencil_server_cancel(server, tickets[0])  # active
        assert L.stencil_server_poll(server, tickets[0]) == L.STENCIL_REQ_CANCELLED
        with pytest.raises(L.StencilError) as e:
            L.stencil_server_cancel(server, tickets[0])
        assert e.value.status == L.STENCIL_EINVAL
        for _ in range(200):
            L.stencil_server_progress(server)
            if all(L.stencil_server_poll(server, t) == L.STENCIL_REQ_DONE for t in (tickets[1], tickets[2])):
                break
        L.stencil_server_sync(server)
        assert L.stencil_server_poll(server, tickets[1]) == L.STENCIL_REQ_DONE
        assert L.stencil_server_poll(server, tickets[2]) == L.STENCIL_REQ_DONE
        used, _, done = L.stencil_server_stats(server)
        assert used == 0
        assert done == 2 * n ** 3 * steps
        for i in (0, 3):
            assert torch.all(outs[i] == -7.0)
        par = L.heat_params(n)
        ref = oracle.diffusion(src.numpy().astype(np.float64).reshape(n, n, n), par.dt, par.alpha,
                               (par.dx[0], par.dx[1], par.dx[2]), steps)
        for i in (1, 2):
            assert_close(outs[i].numpy(), ref.ravel(), 1e-5, f"request {i}")
        with pytest.raises(L.StencilError):
            L.stencil_server_cancel(server, tickets[1])  # done
    finally:
        L.stencil_server_destroy(server)
