"""Continuous-batching reconstruction server over the library's job API.

Requests (scan description + compressed data + iteration budget) arrive over
time. The server admits a request as soon as its device memory fits in the HBM
budget next to the jobs already running, keeps every admitted job's data and
solver state on the device, and advances all running jobs together: each
mpi_ffl_job_step call is one iteration of Eq. (26) for every job, issued as one
launch per kernel kind for the jobs on the full-GEMM path. Finished jobs are
retired (their result copied out, their memory released) and waiting requests
take their place, so requests that arrive while others run join the batch.
Latency is measured per request from arrival to result.
"""

import ctypes as C
import dataclasses
import time
from concurrent.futures import ThreadPoolExecutor

import torch

from . import _lib
from ._lib import check
from .operator import FFLOperator


JobStatus = _lib.JobStatus


def _declare(lib):
    """The job prototypes are declared by _lib.load(); kept for callers that import it."""
    return lib


@dataclasses.dataclass
class Request:
    """One reconstruction request: a scan description (FFLOperator keyword args),
    its compressed data (float32 [M, N_z, n_bins, 2], on the device or the host),
    and the solve settings."""

    geometry: dict
    data: torch.Tensor
    iters: int = 100
    stop_rel: float = 0.0
    lam: float = -1.0
    tau: float = 0.0
    n_power: int = 20
    arrival: float = 0.0            # seconds after the start of the run
    name: str = ""
    # filled in by the server
    admitted: float = None
    finished: float = None
    result: torch.Tensor = None
    status: dict = None

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


class Job:
    """A running request: handle, device data and the library job. Created on its
    own stream (handle tables, data copy, power iteration) so that preparing a new
    request overlaps the running batch."""

    def __init__(self, req, path, precision=None):
        lib = _lib.load()
        _declare(lib)
        self.req = req
        self.prep_stream = torch.cuda.Stream()
        with torch.cuda.stream(self.prep_stream):
            self.op = FFLOperator(**req.geometry)
            self.op.set_path(path)
            if precision is not None:
                self.op.set_precision(precision)
            self.b = req.data.to(self.op.device, non_blocking=True).contiguous()
            p = _lib.SolveParams(int(req.iters), float(req.lam), float(req.tau), int(req.n_power), C.c_uint64(1234),
                                 1, float(req.stop_rel), 0.0)
            h = C.c_void_p()
            check(lib.mpi_ffl_job_create(self.op._h, C.c_void_p(self.b.data_ptr()), None, C.byref(p), C.byref(h),
                                         C.c_void_p(self.prep_stream.cuda_stream)), self.op._h)
        self.ready = torch.cuda.Event()
        self.ready.record(self.prep_stream)
        self.h = h
        self.lib = lib
        self.steps = 0

    def finish(self, stream):
        st = JobStatus()
        rc = self.lib.mpi_ffl_job_status(self.h, C.byref(st), C.c_void_p(stream.cuda_stream))
        with torch.cuda.stream(stream):
            x = self.op.new_volume()
        check(self.lib.mpi_ffl_job_result(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(stream.cuda_stream)))
        self.req.status = dict(iters_done=st.iters_done, stopped=st.stopped, residual_first=st.residual_first,
                               residual_last=st.residual_last, tau=st.tau, lam=st.lambda_, rc=rc)
        return x

    def release(self):
        self.lib.mpi_ffl_job_destroy(self.h)
        self.h = None
        self.op.close()


def estimate_job_bytes(op):
    """Device bytes of a job besides its handle: 4 volumes, 2 data vectors, history."""
    s = op.sizes
    return 4 * (4 * s.n_vox + 2 * s.n_data) + 8 * 1024


def estimate_request_bytes(geometry):
    """Device bytes a request will hold (handle workspace + job state), from its sizes."""
    nx, nz, m = geometry["nx"], geometry["nz"], geometry["n_angles"]
    S, P, Q, A = geometry["S"], geometry["P"], geometry.get("Q", 8), geometry.get("A", 6.0)
    K = geometry["k_max"] - geometry["k_min"] + 1
    nb = K * (2 * geometry["half_width"] + 1)
    ne = (nx - 1) * Q + 2 * int(-(-A * Q // 1)) + 1
    nvox, nproj, nfine, ndata = nz * nx * nx, m * nz * nx, m * nz * ne, 2 * m * nz * nb
    handle = 4 * (3 * nvox + nproj + nfine + 2 * ndata) + 4 * 4 * nvox + 4 * 2 * S * P * 12 + (8 << 20)
    return handle + 4 * (4 * nvox + 2 * ndata)


class ReconServer:
    """Continuous batching of reconstructions within an HBM budget.

    run(requests) replays the requests at their arrival times (seconds from the
    start of the run) and returns them with admitted/finished times, results and
    solver status filled in.
    """

    def __init__(self, hbm_budget_bytes=150 * 2**30, path="full_gemm", max_active=64, poll_every=1,
                 keep_results=True, prepare_workers=4, precision=None):
        self.prepare_workers = prepare_workers
        self.precision = precision  # PREC_* for the jobs' handles, None = the path's default
        self.budget = int(hbm_budget_bytes)
        self.path = path
        self.max_active = max_active
        self.poll_every = max(1, poll_every)
        self.keep_results = keep_results
        self.stream = torch.cuda.Stream()
        self.release_pool = ThreadPoolExecutor(max_workers=1)
        self.peak_bytes = 0
        self.steps = 0

    def run(self, requests):
        lib = _lib.load()
        _declare(lib)
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            r.est_bytes = estimate_request_bytes(r.geometry)
        waiting = []      # arrived, not yet admitted
        preparing = []    # admitted, handle and job being built by a worker thread
        active = []
        done = []
        in_use = 0
        flags_host = torch.empty(3 * self.max_active, dtype=torch.int32).pin_memory()
        dev = torch.cuda.current_device()

        def prepare(req):
            torch.cuda.set_device(dev)
            return Job(req, self.path, self.precision)

        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        steps_since_poll = 0
        with ThreadPoolExecutor(max_workers=self.prepare_workers) as pool:
            while pending or waiting or preparing or active:
                t = now()
                while pending and pending[0].arrival <= t:
                    waiting.append(pending.pop(0))
                # admit in arrival order while memory and slots allow
                while (waiting and len(active) + len(preparing) < self.max_active
                       and in_use + waiting[0].est_bytes <= self.budget):
                    r = waiting.pop(0)
                    r.admitted = now()
                    in_use += r.est_bytes
                    preparing.append(pool.submit(prepare, r))
                self.peak_bytes = max(self.peak_bytes, in_use)
                still = []
                for f in preparing:
                    if f.done():
                        job = f.result()
                        self.stream.wait_event(job.ready)
                        active.append(job)
                    else:
                        still.append(f)
                preparing = still
                if not active:
                    if waiting and not pending and not preparing and in_use == 0:
                        raise RuntimeError("a request does not fit the HBM budget on its own")
                    time.sleep(0.0005)
                    continue
                arr = (C.c_void_p * len(active))(*[j.h for j in active])
                check(lib.mpi_ffl_job_step(arr, len(active), C.c_void_p(self.stream.cuda_stream)))
                self.steps += 1
                for j in active:
                    j.steps += 1
                steps_since_poll += 1
                budget_done = any(j.steps >= j.req.iters for j in active)
                if steps_since_poll >= self.poll_every or budget_done:
                    steps_since_poll = 0
                    arr = (C.c_void_p * len(active))(*[j.h for j in active])
                    check(lib.mpi_ffl_job_poll(arr, len(active), C.c_void_p(flags_host.data_ptr()),
                                               C.c_void_p(self.stream.cuda_stream)))
                    self.stream.synchronize()
                    fl = flags_host[: 3 * len(active)].view(-1, 3).tolist()
                    keep = []
                    for j, (stop, _, frozen) in zip(active, fl):
                        if stop != 0 or frozen != 0 or j.steps >= j.req.iters:
                            x = j.finish(self.stream)
                            j.req.finished = now()
                            if self.keep_results:
                                j.req.result = x
                            in_use -= j.req.est_bytes
                            done.append(j.req)
                            self.release_pool.submit(j.release)
                        else:
                            keep.append(j)
                    active = keep
        self.release_pool.shutdown(wait=True)
        self.release_pool = ThreadPoolExecutor(max_workers=1)
        return done


def percentile(values, q):
    v = sorted(values)
    if not v:
        return None
    k = (len(v) - 1) * q / 100.0
    lo = int(k)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


def run_sequential(requests, path="staged"):
    """Baseline: one request at a time, in arrival order, with mpi_ffl_solve."""
    out = []
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.arrival):
        while time.perf_counter() - t0 < r.arrival:
            time.sleep(0.001)
        op = FFLOperator(**r.geometry)
        op.set_path(path)
        b = r.data.to(op.device).contiguous()
        x, rep = op.solve(b, iters=r.iters, lam=r.lam, tau=r.tau, n_power=r.n_power, stop_rel=r.stop_rel)
        torch.cuda.synchronize()
        r.finished = time.perf_counter() - t0
        r.result = x
        r.status = rep
        op.close()
        out.append(r)
    return out
