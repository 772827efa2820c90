"""Throughput of the compressed 3D FFL-MPI operator: A + A^T pairs per second.

One step = one application of A followed by one of A^T (the hot loop of the
regularised solve) on the in-vivo-scale workload: a 256x256x128 volume, 36 FFL
angles, 128 lines x 512 drive periods x 128 samples per angle (302M time
samples), harmonics 1..16 kept at +-4 bins. Inputs are synthetic (a seeded
mouse-like phantom). Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--path staged|fused|line_gemm|full_gemm] [--workload invivo|phantom|tiny]
                  [--serving-requests 64] [--recon-iters 100] [--no-cpu-baseline] [--quick]

The headline `value` is the full-GEMM path (the operator with S D F V E H
precomputed per trajectory, on tensor cores in split bf16 with FP32 accuracy);
`paths` reports every evaluation path of the same operator, `recon` seconds per
reconstruction, `serving` the continuous-batching run of the serving workload
against one-at-a-time plain FP32.

K defaults to 3000 pairs, about a second of device time, so that the 200 ms clock
samples fall inside the timed region; the other paths take at most 20 steps each.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (a subset of angles), scaled to pairs/s.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from phantoms import config, phantom_for  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
METRIC = "A+A^T pairs/s at 256^2x128, 36 angles"


def workload_desc(cfg):
    return (f"{cfg['name']}: {cfg['nx']}x{cfg['nx']}x{cfg['nz']} volume, {cfg['n_angles']} angles, "
            f"{cfg['nz']} lines x {cfg['P']} periods x {cfg['S']} samples per angle, "
            f"harmonics {cfg['k_min']}..{cfg['k_max']} at +-{cfg['half_width']} bins, Q={cfg['Q']}, "
            f"FWHM {cfg['fwhm']} vox")


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.perf_counter()  # nvidia-smi takes a moment to start: wait for its first line
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.first = len(self.lines)  # samples taken before the timed region are not counted
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "first", 0):]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle (CPU)

def oracle_pair_seconds(cfg, x, n_angles_sample):
    """Time A+A^T of the oracle restricted to a few angles; returns (seconds per full pair, sample text)."""
    from oracle import Setup, operator

    st = Setup.from_config(cfg)
    rng = np.random.default_rng(5)
    t0 = time.perf_counter()
    for m in range(n_angles_sample):
        fs = operator.forward_stages(x, st, angles=np.array([m]))
        y = fs["data"] + 0.01 * (rng.standard_normal(fs["data"].shape) + 1j * rng.standard_normal(fs["data"].shape))
        operator.adjoint_stages(y, st, angles=np.array([m]))
    dt = time.perf_counter() - t0
    per_pair = dt / n_angles_sample * cfg["n_angles"]
    return per_pair, f"A+A^T of {n_angles_sample} of {cfg['n_angles']} angles, scaled by {cfg['n_angles']}/{n_angles_sample}"


def oracle_recon_seconds(power_iters=50):
    """Seconds per reconstruction of the FP64 oracle (power iteration for tau, then the
    workload's iterations of Eq. (26)): measured in full on the tiny workload, and
    extrapolated on the phantom-scale one from the measured time of A+A^T on one angle
    x angles x (power iterations + solve iterations)."""
    from oracle import Setup, operator, solver
    from oracle.data import make_data

    out = {}
    cfg = config("tiny")
    st = Setup.from_config(cfg)
    b, _ = make_data(st, phantom_for(cfg), noise=cfg["noise"], seed=cfg["seed"])
    shape = (st.nz, st.nx, st.nx)
    t0 = time.perf_counter()
    ata = solver.power_norm(lambda v: operator.adjoint(operator.forward(v, st), st), shape, n_iter=power_iters)
    lam = solver.default_lambda(ata, shape)
    solver.solve(lambda v: operator.forward(v, st), lambda r: operator.adjoint(r, st), b, shape,
                 solver.step_size(ata, lam, shape), lam, cfg["iters"])
    out["tiny"] = {"s_per_recon": time.perf_counter() - t0, "iters": cfg["iters"], "power_iters": power_iters,
                   "how": "measured"}
    cfg = config("phantom")
    per_pair, _ = oracle_pair_seconds(cfg, phantom_for(cfg).astype(np.float64), 1)
    out["phantom"] = {"s_per_recon": per_pair * (power_iters + cfg["iters"]), "iters": cfg["iters"],
                      "power_iters": power_iters,
                      "how": "extrapolated: A+A^T of one angle measured, x angles x (power + solve iterations)"}
    return out


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def over_ranks(values_ms, dist, device="cuda"):
    """Each timing (ms) maximised over the ranks of the process group (the slowest rank
    sets the job's time); unchanged without one."""
    if dist is None:
        return [float(v) for v in values_ms]
    import torch

    t = torch.tensor([float(v) for v in values_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def aux_steps(args):
    """Steps for the secondary measurements (other paths, dual drive, tensor PSF)."""
    return max(3, min(args.steps, 40) // 2)


def whole_job_rate(units_per_rank, world, max_ms):
    """Units every rank processed, divided by the slowest rank's time (per second)."""
    return units_per_rank * world / (max_ms / 1e3)


def run_reference(args, cfg, rank):
    """The reference arm: the FP64 oracle on the host cores. One step is A + A^T
    restricted to one FFL angle (angles taken in turn), 1/M of a full pair, so that K
    steps run in seconds; the value is full pairs per second, 1 / (M x median time
    per step)."""
    if rank != 0:
        return
    from oracle import Setup, operator

    x = phantom_for(cfg).astype(np.float64)
    st = Setup.from_config(cfg)
    rng = np.random.default_rng(5)
    M = cfg["n_angles"]

    def angle_step(m):
        fs = operator.forward_stages(x, st, angles=np.array([m]))
        y = fs["data"] + 0.01 * (rng.standard_normal(fs["data"].shape) + 1j * rng.standard_normal(fs["data"].shape))
        operator.adjoint_stages(y, st, angles=np.array([m]))

    for w in range(args.warmup):  # caches and FFT plans
        angle_step(w % M)
    times = []
    t_run = time.perf_counter()
    for k in range(args.steps):
        t0 = time.perf_counter()
        angle_step(k % M)
        times.append(time.perf_counter() - t0)
    t_run = time.perf_counter() - t_run
    per_step = statistics.median(times)
    value = 1.0 / (per_step * M)
    sample = (f"each step is A+A^T of one of the {M} angles (angles in turn, 1/{M} of a pair); "
              f"value = 1 / ({M} x median step time), an extrapolation from the measured per-angle time")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(cfg), "step": f"A+A^T restricted to one FFL angle (1/{M} of a pair)"},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores(), "kind": "oracle", "sample": sample,
                         "measured_s_per_angle_step": per_step, "wall_s_timed_steps": t_run},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU

ALGO_BYTES = {
    # compulsory HBM bytes per launch: inputs read once, outputs written once
    "project": lambda d: 4 * (d["nvox"] + d["nproj"]),
    "backproject": lambda d: 4 * (d["nvox"] + d["nproj"]),
    "psf_fwd": lambda d: 4 * (d["nproj"] + d["nfine"]),
    "psf_adj": lambda d: 4 * (d["nproj"] + d["nfine"]),
    "resample_fwd": lambda d: 4 * (d["nfine"] + d["nsig"]),
    "resample_adj": lambda d: 4 * (d["nfine"] + d["nsig"]),
    "dft_fwd": lambda d: 4 * (d["nsig"] + d["ndata"]),
    "dft_adj": lambda d: 4 * (d["nsig"] + d["ndata"]),
    "tc_fwd": lambda d: 4 * (d["nfine"] + d["ndata"]),
    "tc_adj": lambda d: 4 * (d["nfine"] + d["ndata"]),
    # the slice-interleaving pass: reads the volume, writes its interleaved copy
    "transpose": lambda d: 8 * d["nvox"],
    # the full-GEMM path applies W H to projections, the line-GEMM path W to fine rows
    "gemm_fwd": lambda d: 4 * ((d["nproj"] if d["path"].startswith("full_gemm") else d["nfine"]) + d["ndata"]),
    "gemm_adj": lambda d: 4 * ((d["nproj"] if d["path"].startswith("full_gemm") else d["nfine"]) + d["ndata"]),
}

# Shared-memory bytes the projector pair reads per launch: two interpolation taps of
# 4 bytes for every (angle, ray, march step, slice) sample, M N N N_z = M n_vox samples. Both
# kernels stage their operand in shared memory and are bound by its bandwidth, held
# against the bandwidth the library's probe kernel measures.
SMEM_BYTES = {
    "project": lambda d: 8 * d["M"] * d["nvox"],
    "backproject": lambda d: 8 * d["M"] * d["nvox"],
}

# DRAM bytes (read + write) per launch from one ncu capture of each kernel (cold
# caches, 256^2x128, 36 angles, --set full, one launch). Reported only for that
# workload and only while the kernel is the one that was captured.
DRAM_TRAFFIC = {
    "project": 33_579_008 + 0,          # reads the interleaved copy once; its GEMM operand stays in L2
    "backproject": 4_736_000 + 0,       # reads the projections; the volume it writes stays in L2
    "transpose": 33_564_672 + 418_048,  # interleave pass: most of its writes stay in L2
}


def use_path(op, key):
    """Select an evaluation path by key ('full_gemm', 'full_gemm_tf32', ...) with its
    precision set explicitly (set_path keeps TF32 between the two GEMM paths)."""
    from paper_2511_06627_gb300 import PREC_BF16X3, PREC_TF32

    tf32 = key.endswith("_tf32")
    p = key[: -len("_tf32")] if tf32 else key
    op.set_path(p)
    if p in ("line_gemm", "full_gemm"):
        op.set_precision(PREC_TF32 if tf32 else PREC_BF16X3)


def bf16_peak_tflops():
    try:
        with open(PEAKS_PATH) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def smem_peak_gbs():
    """Shared-memory read bandwidth of this GPU in GB/s, measured by the library's probe
    kernel (conflict-free 16-byte loads on every SM, CUDA events)."""
    import ctypes as C

    import torch

    from paper_2511_06627_gb300 import _lib

    lib = _lib.load()
    v = C.c_double(0.0)
    rc = lib.mpi_ffl_probe_smem_bandwidth(C.byref(v), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != _lib.OK:
        raise RuntimeError(f"shared-memory probe failed: {rc}")
    return v.value


def kernel_rooflines(prof, d, hbm, sm_peak):
    """Per kernel kind of the timed region: achieved algorithmic HBM GB/s against the
    measured copy peak; for the projector pair also the shared-memory roofline against
    the measured shared-memory bandwidth; for the GEMMs the tensor rate (3 products of
    2 M N K flops, and the method's own single product) against the peak of the operand
    type (measured bf16; tf32 from it by the nominal ratio)."""
    bf16, _ = bf16_peak_tflops()
    nz = d["nvox"] // (d["N"] * d["N"])
    nseg = d["M"] * nz
    rows_k = d["N"] if d["path"].startswith("full_gemm") else d["nfine"] // nseg
    # tf32 operands: the measured bf16 peak times the nominal tf32/bf16 ratio (1.1 / 2.25 PFLOP/s)
    tensor_peak = bf16 * (1.1 / 2.25) if d["path"].endswith("_tf32") else bf16
    out = {}
    for k, (t_ms, n) in prof.items():
        if n <= 0 or k not in ALGO_BYTES:
            continue
        sec = t_ms / n / 1e3
        e = {"ms_per_launch": t_ms / n, "hbm_frac": ALGO_BYTES[k](d) / sec / 1e9 / hbm}
        if k in SMEM_BYTES:
            e["smem_frac"] = SMEM_BYTES[k](d) / sec / 1e9 / sm_peak
        if k in ("gemm_fwd", "gemm_adj"):
            flops = 3 * 2 * nseg * (d["ndata"] // nseg) * rows_k
            e["tensor_tflops"] = flops / sec / 1e12
            e["tensor_frac"] = e["tensor_tflops"] / tensor_peak
            e["method_tensor_frac"] = e["tensor_frac"] / 3  # one product of the method's 2 M N K
        out[k] = {kk: round(vv, 5) for kk, vv in e.items()}
    return out


def detection_bench(cfg_name="phantom", amounts=(5.0, 10.0, 25.0, 50.0), noise=0.2, seed=3, w_true=3.3):
    """Sensitivity series (Gaussian samples of the given amounts on the middle slice,
    five void boxes). The data carry the scan nonidealities the solve does not model
    (per-angle gains U(0.95, 1.05) and a PSF width of 3.3 voxels against the model's 3)
    and complex Gaussian noise at `noise` x max |b| (seeded), so the void boxes hold
    reconstruction noise as the paper's scans do. The configuration's iterations of
    Eq. (26) on the full-GEMM path, then the detection-limit analysis on the GPU; the
    oracle's analysis of the same volume checks it."""
    import time

    import torch

    from oracle import detection
    from paper_2511_06627_gb300 import FFLOperator
    from paper_2511_06627_gb300.operator import box_stats, detection_limit
    from phantoms.generators import sensitivity_series

    cfg = config(cfg_name)
    vol, sboxes, vboxes = sensitivity_series(cfg["nx"], cfg["nz"], list(amounts), seed=seed)
    rng = np.random.default_rng(seed)
    truth = FFLOperator.from_config(cfg, fwhm=w_true, gains=rng.uniform(0.95, 1.05, cfg["n_angles"]))
    truth.set_path("full_gemm")
    b = truth.forward(torch.from_numpy(vol).cuda()).clone()
    truth.close()
    op = FFLOperator.from_config(cfg)
    op.set_path("full_gemm")
    sigma = noise * float(b.abs().max())
    b += torch.from_numpy((sigma / np.sqrt(2) * rng.standard_normal(b.shape)).astype(np.float32)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, rep = op.solve(b, iters=cfg["iters"])
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    values = box_stats(x, sboxes)[:, 1]
    nz_ = box_stats(x, vboxes, pooled=True)[0, 2]
    res = detection_limit(list(amounts), values, nz_)
    t2 = time.perf_counter()
    ref = detection.analyse(x.cpu().numpy(), sboxes, list(amounts), vboxes)
    op.close()
    return {"limit": res["limit"], "slope": res["slope"], "intercept": res["intercept"], "noise_mad": nz_,
            "amounts": list(amounts), "sample_values": [float(v) for v in values],
            "solve_s": t1 - t0, "analysis_ms": (t2 - t1) * 1e3, "iters": cfg["iters"],
            "limit_rel_diff_vs_oracle_analysis": abs(res["limit"] - ref["limit"]) / abs(ref["limit"]),
            "workload": f"{cfg['nx']}^2 x {cfg['nz']}, {cfg['n_angles']} angles, noise {noise} x max|b|, "
                        f"unmodelled gains U(0.95, 1.05) and PSF width {w_true} (model {cfg['fwhm']})",
            "note": "sample value = ROI mean over its box; noise = pooled mean absolute deviation of 5 void boxes; "
                    "limit where the least-squares line reaches 3 x noise"}


def calibration_bench(iters=200, seed=62, w_true=3.3):
    """The calibration workload: the phantom-scale scan with unknown per-angle gains
    U(0.95, 1.05) and PSF width (3.3 voxels, model started at 3), data b = A(g, w) x of
    the phantom; `iters` iterations of the joint volume + calibration fit (autograd.calibrate:
    projected gradient on x, Adam on gains and width) on the line-GEMM path. Reports the
    time per iteration and the recovered parameters (gains compared after dividing by
    their mean: the volume and the gains share one scale)."""
    import torch

    from paper_2511_06627_gb300 import FFLOperator
    from paper_2511_06627_gb300.autograd import calibrate

    cfg = config("phantom")
    keys = ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm", "k_min", "k_max", "half_width")
    geom = {k: cfg[k] for k in keys}
    M = cfg["n_angles"]
    rng = np.random.default_rng(seed)
    g_true = rng.uniform(0.95, 1.05, M)
    x = torch.from_numpy(phantom_for(cfg)).cuda()
    truth = FFLOperator(**{**geom, "fwhm": w_true}, gains=g_true)
    truth.set_path("full_gemm")
    b = truth.forward(x).clone()
    truth.close()
    # the line-GEMM path: W holds no PSF, so a new width only replaces the PSF taps
    op = FFLOperator(**geom)
    op.set_path("line_gemm")
    calibrate(op, b, iters=2, gains0=[1.0] * M, fwhm0=cfg["fwhm"])  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, gj, wj, hist = calibrate(op, b, iters=iters, gains0=[1.0] * M, fwhm0=cfg["fwhm"])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    gj = gj.cpu().numpy().astype(np.float64)
    wj = float(wj.cpu().numpy()[0])
    op.close()
    gn_true = g_true / g_true.mean()
    return {"iters": iters, "ms_per_iteration": dt / iters * 1e3, "loss_ratio": hist[-1] / hist[0],
            "gain_max_abs_error": float(np.max(np.abs(gj / gj.mean() - gn_true))),
            "gain_max_abs_error_at_start": float(np.max(np.abs(1.0 - gn_true))),
            "fwhm": wj, "fwhm_true": w_true, "fwhm_at_start": cfg["fwhm"],
            "workload": f"{cfg['nx']}^2 x {cfg['nz']}, {M} angles, {M} gains + 1 PSF width unknown",
            "note": "wall time per iteration of forward, backward (A^T and the parameter gradients) and the "
                    "updates, with the host reading the loss each iteration"}


def _timed_pairs(op, x, b, xa, steps, flush, stream):
    """Time `steps` A+A^T pairs (CUDA events per step, L2 flushed between steps); returns ms."""
    import torch

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        op.forward(x, out=b)
        op.adjoint(b, out=xa)
        ends[k].record(stream)
    torch.cuda.synchronize()
    return sum(s_.elapsed_time(e) for s_, e in zip(starts, ends))


def serving_bench(n_requests, iters, seed=0):
    """The serving workload: a Poisson stream of mixed reconstruction requests.

    Requests follow the serving recipe (64^3 .. 256^2x128 volumes, 8-36 angles,
    harmonics 1..K, K in 8..16); data are b = A x + complex Gaussian noise (0.5 % of
    max |b|) from seeded phantoms, computed on the GPU before the run. Each job runs 100
    iterations or stops when its residual changes by at most 1e-3. The sequential
    plain-FP32 baseline solves one request at a time with the staged FP32 path; the
    arrival rate is 1.5x its measured throughput and its latencies follow from its
    measured per-request service times (single FIFO server). The batched server then
    replays the same arrivals live.
    """
    import torch

    from paper_2511_06627_gb300 import FFLOperator
    from paper_2511_06627_gb300.serving import ReconServer, Request, percentile
    from phantoms.configs import serving_mix

    mix = serving_mix(seed=seed, n_requests=n_requests)
    keys = ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm", "k_min", "k_max", "half_width")
    phantoms = {}
    reqs = []
    gen = torch.Generator(device="cuda").manual_seed(seed)
    for i, c in enumerate(mix):
        g = {k: c[k] for k in keys}
        key = (c["nx"], c["nz"])
        if key not in phantoms:
            phantoms[key] = torch.from_numpy(phantom_for(c, seed=seed)).cuda()
        op = FFLOperator(**g)
        op.set_path("line_gemm")
        b = op.forward(phantoms[key])
        sig = 0.005 * float(b.abs().max())
        b += sig * torch.randn(b.shape, device="cuda", generator=gen)
        torch.cuda.synchronize()
        op.close()
        reqs.append(Request(geometry=g, data=b, iters=iters, n_power=20, stop_rel=1e-3, name=f"req{i}"))
    # sequential plain FP32: measured service time per request (handle set-up + solve)
    service, seq_x, seq_iters = [], {}, []
    for r in reqs:
        t0 = time.perf_counter()
        op = FFLOperator(**r.geometry)
        xs_, rep = op.solve(r.data, iters=r.iters, n_power=r.n_power, stop_rel=r.stop_rel)
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t0)
        seq_x[r.name] = xs_.cpu()
        seq_iters.append(rep["iters_done"])
        op.close()
    rate = 1.5 / (sum(service) / len(service))
    rng = np.random.default_rng(seed + 1)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    arrivals -= arrivals[0]
    t_free, seq_lat = 0.0, []
    for a, s_ in zip(arrivals, service):
        start = max(a, t_free)
        t_free = start + s_
        seq_lat.append(t_free - a)
    seq_makespan = t_free
    for r, a in zip(reqs, arrivals):
        r.arrival = float(a)
    server = ReconServer(hbm_budget_bytes=150 * 2**30, path="full_gemm", max_active=64, poll_every=4,
                         keep_results=True)
    t0 = time.perf_counter()
    done = server.run(reqs)
    makespan = time.perf_counter() - t0
    lat = [r.latency for r in done]
    # capacity: the same requests all present at t = 0
    import copy

    sat = [copy.copy(r) for r in reqs]
    for r in sat:
        r.arrival, r.admitted, r.finished, r.result, r.status = 0.0, None, None, None, None
    sat_server = ReconServer(hbm_budget_bytes=150 * 2**30, path="full_gemm", max_active=64, poll_every=4,
                             keep_results=False)
    t1 = time.perf_counter()
    sat_done = sat_server.run(sat)
    sat_makespan = time.perf_counter() - t1
    # each batched result against the same request solved alone on the plain FP32 path
    diffs = []
    for r in done:
        a_ = r.result.double().cpu()
        b_ = seq_x[r.name].double()
        diffs.append(float((a_ - b_).norm() / max(float(b_.norm()), 1e-300)))
        r.result = None
    return {
        "requests": len(reqs), "iters_per_request": iters, "arrival_rate_per_s": rate,
        "batched": {"recons_per_s": len(done) / makespan, "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
                    "path": "full_gemm (bf16 hi+lo tensor cores), continuous batching", "peak_hbm_bytes": server.peak_bytes,
                    "batched_steps": server.steps,
                    "iters_done_mean": float(np.mean([r.status["iters_done"] for r in done])),
                    "max_rel_l2_vs_sequential": max(diffs), "median_rel_l2_vs_sequential": float(np.median(diffs))},
        "sequential_plain_fp32": {"recons_per_s": len(reqs) / seq_makespan, "p50_s": percentile(seq_lat, 50),
                                  "p99_s": percentile(seq_lat, 99),
                                  "iters_done_mean": float(np.mean(seq_iters)),
                                  "note": "staged FP32 path, one request at a time; latencies from measured service "
                                          "times under the same arrivals"},
        "saturated": {"batched_recons_per_s": len(sat_done) / sat_makespan,
                      "sequential_plain_fp32_recons_per_s": len(reqs) / sum(service),
                      "note": "all requests present at t = 0: the batched server's makespan vs the sum of the "
                              "sequential service times"},
        "stop_rule": "100 iterations, or earlier when the FP64 residual changes by <= 1e-3 between iterations",
        "hbm_budget_bytes": 150 * 2**30,
    }


def run_ours(args, cfg, rank, world, local_rank):
    import torch

    from paper_2511_06627_gb300 import FFLOperator

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    # headline: the full-GEMM path with bf16 hi+lo operands (tf32 hi+lo is reported
    # beside it under "paths")
    path = args.path or ("staged" if args.plain else "full_gemm")
    op = FFLOperator.from_config(cfg)
    use_path(op, path)
    sz = op.sizes
    dims = dict(nvox=sz.n_vox, nproj=sz.n_proj, nfine=sz.n_fine, nsig=sz.n_sig, ndata=sz.n_data, M=op.n_angles,
                N=op.nx)
    x_np = phantom_for(cfg)
    x_host = torch.from_numpy(x_np).pin_memory()
    x = x_host.cuda()
    b = op.new_data()
    xa = op.new_volume()
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream()

    def step():
        op.forward(x, out=b)
        op.adjoint(b, out=xa)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # ---- timed region: K steps, L2 flushed between steps (outside the events)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = op.launch_count()
    with ClockSampler(local_rank) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
        launches = op.launch_count() - launches0
        ms = sum(s_.elapsed_time(e) for s_, e in zip(starts, ends))
        # the same K steps again with the library's CUDA events around every launch (on
        # the launching stream): per-kernel durations for the shares and the rooflines.
        # The events cost a little time, so the headline comes from the pass above.
        op.profile(True)
        op.profile_read()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
        prof = op.profile_read()
        op.profile(False)
        ms_prof = sum(s_.elapsed_time(e) for s_, e in zip(starts, ends))
    (ms,) = over_ranks([ms], dist)
    if dist:
        dist.barrier()
    pairs = args.steps * world
    value = whole_job_rate(args.steps, world, ms)

    # ---- end to end through the public API with host buffers: forward reads a pinned
    # host volume and adjoint writes a pinned host volume; the library stages both. Two
    # handles on two streams take alternate steps, so one step's copies overlap the
    # other's kernels (the way a stream of volumes is fed); each handle also copies its
    # next input on its own stream.
    ops = [op, FFLOperator.from_config(cfg)]
    use_path(ops[1], path)
    streams = [stream, torch.cuda.Stream()]
    bufs = [b, ops[1].new_data()]
    outs = [torch.empty(op.vol_shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    for o in ops:
        o.set_host_overlap(True)

    def e2e_step(k):
        i = k % 2
        with torch.cuda.stream(streams[i]):
            ops[i].forward(x_host, out=bufs[i])
            ops[i].adjoint(bufs[i], out=outs[i])

    def e2e_time(step_fn, n):
        ta = torch.cuda.Event(enable_timing=True)
        tb = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ta.record(streams[0])
        for k in range(n):
            step_fn(k)
        tb.record(streams[0])
        torch.cuda.synchronize()
        return ta.elapsed_time(tb)

    # one handle, one stream: each step's copies in series with its kernels except the
    # next input copy, which the handle overlaps
    e2e_step(0)
    e2e_serial_ms = e2e_time(lambda k: e2e_step(0), args.steps)
    for k in range(4):
        e2e_step(k)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(streams[0])
    streams[1].wait_event(e0)
    for k in range(args.steps):
        e2e_step(k)
    streams[0].wait_stream(streams[1])
    e1.record(streams[0])
    torch.cuda.synchronize()
    for o in ops:
        o.set_host_overlap(False)
    ops[1].close()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms, e2e_serial_ms = over_ranks([e2e_ms, e2e_serial_ms], dist)

    # ---- roofline of the dominant kernel (times measured inside the timed region)
    hbm, src = peaks()
    sm_peak = smem_peak_gbs()
    top = max((k for k in prof if prof[k][1] > 0 and k != "solver"), key=lambda k: prof[k][0])
    per_launch_ms = prof[top][0] / prof[top][1]
    algo = ALGO_BYTES[top](dict(dims, path=path))
    achieved = algo / (per_launch_ms / 1e3) / 1e9
    traffic = DRAM_TRAFFIC.get(top) if args.workload == "invivo" and path.startswith("full_gemm") else None
    roofline = {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic,
                "peak_source": f"{src}: hbm_gbs of MEASURED_PEAKS.json (STREAM-style copy)",
                "algorithmic_bytes_per_launch": algo, "avg_launch_ms": per_launch_ms}
    if top in SMEM_BYTES:
        sm_bytes = SMEM_BYTES[top](dims)
        sm_ach = sm_bytes / (per_launch_ms / 1e3) / 1e9
        roofline["smem"] = {"achieved": sm_ach, "peak": sm_peak, "unit": "GB/s", "frac": sm_ach / sm_peak,
                            "bytes_per_launch": sm_bytes,
                            "peak_source": "measured: mpi_ffl_probe_smem_bandwidth (conflict-free 16-byte loads)"}
        roofline["note"] = ("the projector pair reads each voxel once from HBM but every interpolation tap from "
                            "shared memory: it is bound on chip by shared-memory bandwidth (see smem), not by HBM")
    kernel_share = {k: round(v[0] / max(ms_prof, 1e-9), 4) for k, v in prof.items() if v[1] > 0}
    kernel_roof = {path: kernel_rooflines(prof, dict(dims, path=path), hbm, sm_peak)}
    kernel_ms = {k: round(v[0] / v[1], 4) for k, v in prof.items() if v[1] > 0}

    # ---- the other evaluation paths of the same operator (same inputs, same timing rules)
    paths = {path: {"pairs_per_s": value, "ms_per_pair": ms / args.steps}}
    if not args.quick:
        for key in ("staged", "fused", "line_gemm", "full_gemm", "line_gemm_tf32", "full_gemm_tf32"):
            if key in paths:
                continue
            try:
                use_path(op, key)
            except Exception as exc:  # shape not taken by that path
                paths[key] = {"unsupported": str(exc)}
                continue
            for _ in range(2):
                step()
            pm = _timed_pairs(op, x, b, xa, aux_steps(args), flush, stream)
            n = aux_steps(args)
            paths[key] = {"pairs_per_s": n / (pm / 1e3), "ms_per_pair": pm / n}
            # the same steps with the library's per-launch events: every kernel's roofline
            op.profile(True)
            op.profile_read()
            _timed_pairs(op, x, b, xa, n, flush, stream)
            kernel_roof[key] = kernel_rooflines(op.profile_read(), dict(dims, path=key), hbm, sm_peak)
            op.profile(False)
        use_path(op, path)
    plain = paths.get("staged", {}).get("pairs_per_s")

    result = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f32" if path == "staged" else
                  "f32 (line stage on tensor cores as %s hi+lo, 3 products, f32 acc)"
                  % ("tf32" if path.endswith("_tf32") else "bf16")),
        "data": "synthetic",
        "config": {"workload": workload_desc(cfg), "path": path,
                   "l2": "flushed (256 MB write) between timed steps",
                   "step": "b = A x then x' = A^T b, inputs resident in HBM"},
        # HBM roofline of the dominant kernel on its algorithmic bytes (inputs read once,
        # outputs written once) against the measured copy peak; for the projector pair
        # the shared-memory roofline against the measured shared-memory bandwidth beside it
        "roofline": roofline,
        "kernel_time_share": kernel_share,
        "profiled_ms_per_step": ms_prof / args.steps,
        "kernel_ms_per_launch": kernel_ms,
        "kernel_roofline": kernel_roof,
        "paths": paths,
        "speedup_vs_plain_fp32": (value / plain) if plain else None,
        "e2e": {"value": pairs / (e2e_ms / 1e3), "unit": "pairs/s", "h2d_bytes_per_step": 4 * sz.n_vox,
                "d2h_bytes_per_step": 4 * sz.n_vox,
                "how": "forward(pinned host x) + adjoint(-> pinned host x') through the C ABI, which stages host "
                       "buffers; two handles on two streams take alternate steps",
                "serial_value": pairs / (e2e_serial_ms / 1e3),
                "serial_how": "the same calls on one handle and one stream"},
        "clocks": clk.summary(),
        "gpu_launches": int(launches),
        "wall_s_timed_region": t_wall,
    }
    if args.recon_iters > 0:
        # seconds per reconstruction (Eq. (26), 100 iterations, lambda by default rule) on b = A x
        bd = op.forward(x).clone()
        rec = {}
        xs = {}
        runs = [path, "staged"] if path != "staged" else ["staged"]
        if path.endswith("gemm"):
            runs.append(path + "_tf32")
        elif path.endswith("_tf32"):
            runs.append(path[: -len("_tf32")])
        for p in runs:
            use_path(op, p)
            ata = op.power_norm(20, 1234)
            torch.cuda.synchronize()
            r0 = torch.cuda.Event(enable_timing=True)
            r1 = torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            xr, _ = op.solve(bd, iters=args.recon_iters, ata_norm=ata, report=False)
            r1.record(stream)
            torch.cuda.synchronize()
            xs[p] = xr
            rec[p] = {"s_per_recon": r0.elapsed_time(r1) / 1e3, "iters": args.recon_iters}
        if "staged" in xs:
            ref_x = xs["staged"].double()
            rec["rel_l2_vs_staged_fp32"] = {p: float((xs[p].double() - ref_x).norm() / ref_x.norm())
                                            for p in xs if p != "staged"}
        rec["note"] = "tau from a 20-step power iteration done before the timed solve"
        # the tiny and phantom-scale workloads, timed like the oracle's s/recon: the
        # 50-step power iteration for tau, then the workload's iterations of Eq. (26)
        small = {}
        for wname in ("tiny", "phantom"):
            cw = config(wname)
            ow = FFLOperator.from_config(cw)
            xw = torch.from_numpy(phantom_for(cw)).cuda()
            bw = ow.forward(xw).clone()
            small[wname] = {"iters": cw["iters"], "power_iters": 50}
            for p in ("full_gemm", "staged"):
                use_path(ow, p)
                ow.solve(bw, iters=2, n_power=2, report=False)
                torch.cuda.synchronize()
                r0 = torch.cuda.Event(enable_timing=True)
                r1 = torch.cuda.Event(enable_timing=True)
                r0.record(stream)
                ow.solve(bw, iters=cw["iters"], n_power=50, report=False)
                r1.record(stream)
                torch.cuda.synchronize()
                small[wname][p] = r0.elapsed_time(r1) / 1e3
            ow.close()
        rec["s_per_recon_smaller_workloads"] = small
        result["recon"] = rec
        use_path(op, path)
    if not args.quick:
        # dual-drive acquisition (Sec. 3.1): the x-drive scan on the headline path plus the
        # z-drive scan (FP32, resampling fused with the band DFT); one step is
        # [A; A_z] x then A^T b + A_z^T b_z
        bz = op.new_data()
        xz = op.new_volume()

        def dual_step():
            op.forward(x, out=b)
            op.forward_zdrive(x, out=bz)
            op.adjoint(b, out=xa)
            op.adjoint_zdrive(bz, out=xz)
            xa.add_(xz)

        for _ in range(2):
            dual_step()
        n_dual = aux_steps(args)
        d_starts = [torch.cuda.Event(enable_timing=True) for _ in range(n_dual)]
        d_ends = [torch.cuda.Event(enable_timing=True) for _ in range(n_dual)]
        for k in range(n_dual):
            flush.zero_()
            d_starts[k].record(stream)
            dual_step()
            d_ends[k].record(stream)
        torch.cuda.synchronize()
        dual_ms = sum(s_.elapsed_time(e) for s_, e in zip(d_starts, d_ends)) / n_dual
        z_ms = {}
        for name, fn in (("forward_zdrive", lambda: op.forward_zdrive(x, out=bz)),
                         ("adjoint_zdrive", lambda: op.adjoint_zdrive(bz, out=xz))):
            z0 = torch.cuda.Event(enable_timing=True)
            z1 = torch.cuda.Event(enable_timing=True)
            flush.zero_()
            z0.record(stream)
            fn()
            z1.record(stream)
            torch.cuda.synchronize()
            z_ms[name] = z0.elapsed_time(z1)
        # reconstruction from both scans: Eq. (26) on [A; A_z] (mpi_ffl_set_scans)
        op.set_scans("xz")
        b_xz = torch.cat([b, bz]).contiguous()
        op.solve(b_xz, iters=2)
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        flush.zero_()
        r0.record(stream)
        op.solve(b_xz, iters=100, report=False)
        r1.record(stream)
        torch.cuda.synchronize()
        recon_xz_s = r0.elapsed_time(r1) / 1e3
        op.set_scans("x")
        result["dual_drive"] = {"pairs_per_s": 1e3 / dual_ms, "ms_per_pair": dual_ms, "z_drive_ms": z_ms,
                                "recon_both_scans_s_per_100_iters": recon_xz_s,
                                "x_drive_path": path, "z_drive_path": "FP32, E_z V_z B fused with S D F",
                                "step": "[A; A_z] x then A^T b + A_z^T b_z"}
        # tensor PSF (Appendix B, Eq. (31)): every line reads every slice of its projection;
        # A and A^T run as per-line (per-slice) split-K GEMMs on the bf16 hi+lo operands
        op.set_psf_model("tensor")
        for _ in range(2):
            op.forward(x, out=b)
            op.adjoint(b, out=xa)
        n_ten = aux_steps(args)
        ten_ms = _timed_pairs(op, x, b, xa, n_ten, flush, stream) / n_ten
        op.profile(True)
        op.profile_read()
        _timed_pairs(op, x, b, xa, n_ten, flush, stream)
        tprof = op.profile_read()
        op.profile(False)
        t_ms, t_n = tprof["tensor"]
        nz_ = dims["nvox"] // (dims["N"] * dims["N"])
        R_ = dims["ndata"] // (dims["M"] * nz_)
        flops = 2.0 * dims["M"] * nz_ * (nz_ * dims["N"]) * R_  # one direction, FP32 contraction
        sec = t_ms / max(t_n, 1) / 1e3
        peak, peak_src = bf16_peak_tflops()
        # issued MMA work: J = 128 // M8 lines of one trajectory share a problem (rows M8 J,
        # M8 = M rounded up to 8, in 128-row tiles) and its window spans N_z + step (J - 1)
        # slices
        step_ = 2 if cfg["zigzag"] else 1
        M8_ = (dims["M"] + 7) // 8 * 8
        J_ = max(1, min(128 // M8_, (nz_ + step_ - 1) // step_))
        issue_factor = (128 * ((M8_ * J_ + 127) // 128) / (dims["M"] * J_)) * (nz_ + step_ * (J_ - 1)) / nz_
        result["tensor_psf"] = {
            "pairs_per_s": 1e3 / ten_ms, "ms_per_pair": ten_ms,
            "stage_ms_per_launch": round(t_ms / max(t_n, 1), 4),
            "tensor_tflops": round(3 * flops / sec / 1e12, 2),
            "tensor_frac": round(3 * flops / sec / 1e12 / peak, 4),
            "issued_frac": round(3 * flops * issue_factor / sec / 1e12 / peak, 4),
            "peak": f"{peak} TFLOP/s bf16 ({peak_src})",
            "note": "stage = coil weighting + padding, per-line (per-slice) GEMMs over all slices (3 bf16 "
                    "products of 2 M N_z (N_z N) 2n_b flops), sum of the K splits; issued counts the 128-row "
                    "MMA tiles that hold J lines x M8 angles and the window's step (J - 1) extra slices"}
        op.set_psf_model("collinear")
        # detection limit (Sec. 4.2, Fig. 5) of a synthetic sensitivity series at the
        # phantom scale: reconstruction with Eq. (26), box statistics on the GPU, line fit
        result["detection_limit"] = detection_bench(cfg_name="phantom")
        # joint volume + calibration fit (the differentiation pattern) at the phantom scale
        result["calibration"] = calibration_bench()
        # compression analysis (Appendix A, Eq. (30)) on the phantom's time signal
        Ks = [k for k in (1, 2, 4, 8, 16) if op.k_min <= k <= op.k_max]
        ws = [w for w in (0, 1, 2, 4) if w <= op.half_width]
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        table = op.information_retained(x, Ks, ws)
        c1.record(stream)
        torch.cuda.synchronize()
        result["compression_analysis"] = {
            "information_retained": {f"K={K}": {f"w={w}": round(float(table[a, c]), 6) for c, w in enumerate(ws)}
                                     for a, K in enumerate(Ks)},
            "ms": c0.elapsed_time(c1),
            "note": "I(s, S) of Eq. (30) over all segments, harmonics 1..K, |delta| <= w, each bin with its conjugate"}
    if args.serving_requests > 0 and world == 1:
        result["serving"] = serving_bench(args.serving_requests, args.serving_iters)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline_leg(cfg, x_np, op, args)
    if rank == 0:
        print(json.dumps(result), flush=True)
    op.close()
    if dist:
        dist.destroy_process_group()


def cpu_baseline_leg(cfg, x_np, op, args):
    """The FP64 oracle timed on the host cores on a bounded sample (a subset of the
    angles), plus the error of every GPU evaluation path against the oracle on sampled
    angles: theta = 0 (row-marched) and the first angle past 90 degrees (column-marched),
    each with A x on the phantom and A^T y for random y on that angle alone; the worst
    of the angles is reported. Per stage: the staged path's own intermediates."""
    import torch

    from oracle import Setup, operator

    xo = x_np.astype(np.float64)
    nang = max(1, min(cfg["n_angles"], args.oracle_angles))
    per, text = oracle_pair_seconds(cfg, xo, nang)
    st = Setup.from_config(cfg)
    M = st.n_angles
    sample = sorted({0, min(M - 1, M // 2 + 1)})
    rng = np.random.default_rng(9)
    refs = {}
    for m in sample:
        fs = operator.forward_stages(xo, st, angles=np.array([m]))
        y = rng.standard_normal(fs["data"][0].shape) + 1j * rng.standard_normal(fs["data"][0].shape)
        y_full = np.zeros(st.data_shape, dtype=np.complex128)
        y_full[m] = y
        refs[m] = dict(stages=fs, ref_b=fs["data"][0],
                       ref_x=operator.adjoint_stages(y[None], st, angles=np.array([m]))["vol"],
                       y_dev=torch.from_numpy(np.stack([y_full.real, y_full.imag], -1).astype(np.float32)).cuda())
    x_dev = torch.from_numpy(x_np).cuda()
    errs = {}
    for key in ("staged", "fused", "line_gemm", "full_gemm", "line_gemm_tf32", "full_gemm_tf32"):
        try:
            use_path(op, key)
        except Exception:
            continue
        b_all = op.forward(x_dev).cpu().numpy().astype(np.float64)
        ef, ea = 0.0, 0.0
        for m, r in refs.items():
            got_b = b_all[m, ..., 0] + 1j * b_all[m, ..., 1]
            xx = op.adjoint(r["y_dev"]).cpu().numpy().astype(np.float64)
            ef = max(ef, float(np.linalg.norm(got_b - r["ref_b"]) / np.linalg.norm(r["ref_b"])))
            ea = max(ea, float(np.linalg.norm(xx - r["ref_x"]) / np.linalg.norm(r["ref_x"])))
        errs[key] = {"forward_rel_l2": ef, "adjoint_rel_l2": ea}
    # the z-drive scan (staged FP32) on the same sampled angles
    from oracle import zdrive

    bz_all = op.forward_zdrive(x_dev).cpu().numpy().astype(np.float64)
    ezf, eza = 0.0, 0.0
    for m, r in refs.items():
        ref_bz = zdrive.forward_stages_z(xo, st, angles=np.array([m]))["data"][0]
        ezf = max(ezf, float(np.linalg.norm(bz_all[m, ..., 0] + 1j * bz_all[m, ..., 1] - ref_bz) /
                             np.linalg.norm(ref_bz)))
        y_m = r["y_dev"][m].cpu().numpy().astype(np.float64)
        ref_xz = zdrive.adjoint_stages_z((y_m[..., 0] + 1j * y_m[..., 1])[None], st, angles=np.array([m]))["vol"]
        xz = op.adjoint_zdrive(r["y_dev"]).cpu().numpy().astype(np.float64)
        eza = max(eza, float(np.linalg.norm(xz - ref_xz) / np.linalg.norm(ref_xz)))
    errs["z_drive"] = {"forward_rel_l2": ezf, "adjoint_rel_l2": eza}
    # the tensor PSF (full-GEMM path, bf16 hi+lo) on the first sampled angle
    from oracle import tensor_psf

    use_path(op, "full_gemm")
    op.set_psf_model("tensor")
    bt_all = op.forward(x_dev).cpu().numpy().astype(np.float64)
    m0 = sample[-1]
    r = refs[m0]
    ref_bt = tensor_psf.forward_stages(xo, st, None, angles=np.array([m0]))["data"][0]
    etf = float(np.linalg.norm(bt_all[m0, ..., 0] + 1j * bt_all[m0, ..., 1] - ref_bt) / np.linalg.norm(ref_bt))
    y_m = r["y_dev"][m0].cpu().numpy().astype(np.float64)
    ref_xt = tensor_psf.adjoint_stages((y_m[..., 0] + 1j * y_m[..., 1])[None], st, None, angles=np.array([m0]))["vol"]
    xt = op.adjoint(r["y_dev"]).cpu().numpy().astype(np.float64)
    errs["tensor_psf"] = {"forward_rel_l2": etf, "adjoint_rel_l2": float(np.linalg.norm(xt - ref_xt) /
                                                                             np.linalg.norm(ref_xt)),
                          "angles": [int(m0)]}
    op.set_psf_model("collinear")
    # per stage: the staged FP32 path's own intermediates against the oracle's
    op.set_path("staged")
    stages = {}
    cur = x_dev
    for k, name in enumerate(("proj", "fine", "sig", "data")):
        cur = op.apply_stage(k, cur)
        worst = 0.0
        for m, r in refs.items():
            got = cur[m].cpu().numpy().astype(np.float64)
            ref = r["stages"][name][0]
            if name == "data":
                got = got[..., 0] + 1j * got[..., 1]
            worst = max(worst, float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
        stages[name] = worst
    del cur
    return {"value": 1.0 / per, "unit": "pairs/s", "cores": cores(), "kind": "oracle", "sample": text,
            "s_per_recon": oracle_recon_seconds(),
            "gpu_error_vs_oracle": errs,
            "staged_error_per_stage": stages,
            "error_sample": f"angles {sample}: A x on the phantom and A^T y for random y on each angle alone, "
                            "worst angle; per stage: P, H, E V B, S D F of the staged path chained from x"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 3000 A+A^T pairs, about a second, so that the clock "
                         "sampler sees the load; 20 oracle samples with --impl reference)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default=None,
                    choices=["staged", "fused", "line_gemm", "full_gemm", "line_gemm_tf32", "full_gemm_tf32"])
    ap.add_argument("--workload", default="invivo", choices=["invivo", "phantom", "tiny"])
    ap.add_argument("--oracle-angles", type=int, default=1)
    ap.add_argument("--recon-iters", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=64)
    ap.add_argument("--serving-iters", type=int, default=100)
    ap.add_argument("--plain", action="store_true", help="time the staged FP32 path as the headline")
    ap.add_argument("--quick", action="store_true", help="skip the other evaluation paths")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = config(args.workload)
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else 3000
    if args.impl == "reference":
        run_reference(args, cfg, rank)
        return
    run_ours(args, cfg, rank, world, local_rank)


if __name__ == "__main__":
    main()
