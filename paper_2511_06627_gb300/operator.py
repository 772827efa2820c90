"""Python front end of the library: argument marshalling around the C ABI.

Every step of A, A^T and the solve runs in the library's CUDA kernels; PyTorch
only supplies device memory and the current stream. Tensors are float32 on the
handle's CUDA device: volumes [N_z, N, N] (x fastest), data [M, N_z, n_bins, 2]
(complex interleaved, bins k-major with delta ascending).
"""

import ctypes as C
import math

import numpy as np
import torch

from . import _lib
from ._lib import check


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class FFLOperator:
    """A handle on the compressed 3D FFL-MPI operator of one scan description.

    Parameters follow include/mpi_ffl.h: volume nx x nx x nz, n_angles FFL angles
    (default m*pi/M), S samples per drive period, P periods per raster line,
    drive amplitude A (voxels) and phase phi0, zig-zag raster, fine-grid factor Q,
    PSF FWHM (voxels), kept harmonics k_min..k_max with half-width `half_width`.
    """

    def __init__(self, nx, nz, n_angles, S, P, A=6.0, phi0=0.0, zigzag=1, Q=8, fwhm=2.0,
                 k_min=1, k_max=8, half_width=2, angles=None, gains=None, d_gamma=None,
                 precision=_lib.PREC_FP32, path=None):
        lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("FFLOperator needs a CUDA device")
        self.nx, self.nz, self.n_angles = nx, nz, n_angles
        self._ang = None if angles is None else (C.c_double * n_angles)(*[float(a) for a in angles])
        self._gain = None if gains is None else (C.c_float * n_angles)(*[float(g) for g in gains])
        geom = _lib.Geometry(nx, nx, nz, n_angles,
                             C.cast(self._ang, C.POINTER(C.c_double)) if self._ang is not None else None,
                             C.cast(self._gain, C.POINTER(C.c_float)) if self._gain is not None else None)
        traj = _lib.Trajectory(S, P, float(A), float(phi0), int(zigzag), int(Q))
        psf = _lib.Psf(float(fwhm))
        nb = (k_max - k_min + 1) * (2 * half_width + 1)
        dg = None
        if d_gamma is not None:
            d = np.asarray(d_gamma, dtype=np.complex64).reshape(nb)
            dg = (C.c_float * (2 * nb))(*np.stack([d.real, d.imag], -1).reshape(-1).tolist())
        harm = _lib.Harmonics(k_min, k_max, half_width, C.cast(dg, C.POINTER(C.c_float)) if dg is not None else None)
        h = C.c_void_p()
        with torch.cuda.device(torch.cuda.current_device()):
            rc = lib.mpi_ffl_create(C.byref(geom), C.byref(traj), C.byref(psf), C.byref(harm), C.byref(h))
        if rc != _lib.OK:
            raise _lib.MpiFflError(rc, lib.mpi_ffl_last_error(None).decode())
        self._h = h
        self._lib = lib
        self.device = torch.device("cuda", torch.cuda.current_device())
        sz = _lib.Sizes()
        check(lib.mpi_ffl_get_sizes(h, C.byref(sz)), h)
        self.sizes = sz
        self.n_bins = sz.n_bins
        self.L = sz.line_len
        self.fine_len = sz.fine_len
        self.fine_len_z = sz.fine_len_z
        self.S, self.P, self.Q = S, P, Q
        self.k_min, self.k_max, self.half_width = k_min, k_max, half_width
        self.fwhm = fwhm
        self.params = dict(nx=nx, nz=nz, n_angles=n_angles, S=S, P=P, A=A, phi0=phi0, zigzag=zigzag,
                           Q=Q, fwhm=fwhm, k_min=k_min, k_max=k_max, half_width=half_width)
        if precision != _lib.PREC_FP32:
            self.set_precision(precision)
        if path is not None:
            self.set_path(path)

    @classmethod
    def from_config(cls, cfg, **kw):
        keys = ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm", "k_min", "k_max",
                "half_width")
        args = {k: cfg[k] for k in keys if k in cfg}
        args.update(kw)
        return cls(**args)

    # ---------------------------------------------------------------- shapes
    @property
    def vol_shape(self):
        return (self.nz, self.nx, self.nx)

    @property
    def data_shape(self):
        return (self.n_angles, self.nz, self.n_bins, 2)

    def _check(self, t, shape, name, host_ok=False):
        on_dev = isinstance(t, torch.Tensor) and (t.is_cuda or (host_ok and t.device.type == "cpu"))
        if not (on_dev and t.dtype == torch.float32 and t.is_contiguous()):
            where = "CUDA or host" if host_ok else "CUDA"
            raise TypeError(f"{name} must be a contiguous float32 {where} tensor")
        if t.numel() != math.prod(shape):
            raise ValueError(f"{name} has {t.numel()} elements, expected {math.prod(shape)}")

    def new_volume(self):
        return torch.empty(self.vol_shape, device=self.device, dtype=torch.float32)

    def new_data(self):
        return torch.empty(self.data_shape, device=self.device, dtype=torch.float32)

    # ---------------------------------------------------------------- operator
    def forward(self, x, out=None):
        """b = A x. x and out may be CUDA tensors or (pinned) host tensors; host buffers
        are staged by the library. Asynchronous on the current stream."""
        self._check(x, self.vol_shape, "x", host_ok=True)
        out = self.new_data() if out is None else out
        self._check(out, self.data_shape, "out", host_ok=True)
        check(self._lib.mpi_ffl_forward(self._h, _ptr(x), _ptr(out), _stream()), self._h)
        return out

    def adjoint(self, b, out=None):
        """x = A^T b; CUDA or host tensors, as forward."""
        self._check(b, self.data_shape, "b", host_ok=True)
        out = self.new_volume() if out is None else out
        self._check(out, self.vol_shape, "out", host_ok=True)
        check(self._lib.mpi_ffl_adjoint(self._h, _ptr(b), _ptr(out), _stream()), self._h)
        return out

    # ---------------------------------------------------------------- z-drive scan
    def forward_zdrive(self, x, out=None):
        """b_z = A_z x: the z-drive scan of the dual-drive acquisition (same data layout
        as forward). CUDA or host tensors."""
        self._check(x, self.vol_shape, "x", host_ok=True)
        out = self.new_data() if out is None else out
        self._check(out, self.data_shape, "out", host_ok=True)
        check(self._lib.mpi_ffl_forward_zdrive(self._h, _ptr(x), _ptr(out), _stream()), self._h)
        return out

    def adjoint_zdrive(self, b, out=None):
        """x = A_z^T b_z; CUDA or host tensors."""
        self._check(b, self.data_shape, "b", host_ok=True)
        out = self.new_volume() if out is None else out
        self._check(out, self.vol_shape, "out", host_ok=True)
        check(self._lib.mpi_ffl_adjoint_zdrive(self._h, _ptr(b), _ptr(out), _stream()), self._h)
        return out

    def apply_stage_zdrive(self, stage, inp, transpose=False):
        """z-drive stage 1 (H_z: proj [M, N_z, N] <-> fine_z [M, N, N_ez]) or 2
        (E_z V_z B: fine_z <-> sig [M, N_z, L])."""
        M, nz, n = self.n_angles, self.nz, self.nx
        shapes = {1: ((M, nz, n), (M, n, self.fine_len_z)), 2: ((M, n, self.fine_len_z), (M, nz, self.L))}
        if stage not in shapes:
            raise ValueError("z-drive stages are 1 and 2")
        sin, sout = shapes[stage][::-1] if transpose else shapes[stage]
        self._check(inp, sin, "input")
        out = torch.empty(sout, device=self.device, dtype=torch.float32)
        check(self._lib.mpi_ffl_apply_stage_zdrive(self._h, int(stage), int(bool(transpose)), _ptr(inp), _ptr(out),
                                                   _stream()), self._h)
        return out

    def stage_shapes(self):
        M, nz = self.n_angles, self.nz
        return [self.vol_shape, (M, nz, self.nx), (M, nz, self.fine_len), (M, nz, self.L), self.data_shape]

    def apply_stage(self, stage, inp, transpose=False):
        shapes = self.stage_shapes()
        sin, sout = (shapes[stage + 1], shapes[stage]) if transpose else (shapes[stage], shapes[stage + 1])
        self._check(inp, sin, "input")
        out = torch.empty(sout, device=self.device, dtype=torch.float32)
        check(self._lib.mpi_ffl_apply_stage(self._h, int(stage), int(bool(transpose)), _ptr(inp), _ptr(out),
                                            _stream()), self._h)
        return out

    def band_energy(self, x):
        """Compression analysis (Appendix A, Eq. (30)): (per-kept-bin energy summed over
        segments, total signal energy), FP64 numpy, for the time signal of x."""
        self._check(x, self.vol_shape, "x")
        e = torch.empty(self.n_bins, device=self.device, dtype=torch.float64)
        tot = torch.empty((), device=self.device, dtype=torch.float64)
        check(self._lib.mpi_ffl_band_energy(self._h, _ptr(x), _ptr(e), _ptr(tot), _stream()), self._h)
        return e.cpu().numpy(), float(tot.item())

    def information_retained(self, x, harmonics, half_widths):
        """I(s, S) of Eq. (30) for the time signal of x, for every sub-band of the kept
        bins with harmonics k_min..K (K in `harmonics`) and |delta| <= w (w in
        `half_widths`), each bin counted with its conjugate L - omega (computed by the
        library: mpi_ffl_information_retained). Returns a [len(harmonics),
        len(half_widths)] numpy array."""
        self._check(x, self.vol_shape, "x")
        ks = [int(k) for k in harmonics]
        ws = [int(w) for w in half_widths]
        if not all(self.k_min <= k <= self.k_max for k in ks) or not all(0 <= w <= self.half_width for w in ws):
            raise ValueError("sub-band outside the kept bins")
        out = torch.empty((len(ks), len(ws)), device=self.device, dtype=torch.float64)
        ka = (C.c_int32 * len(ks))(*ks)
        wa = (C.c_int32 * len(ws))(*ws)
        check(self._lib.mpi_ffl_information_retained(self._h, _ptr(x), len(ks), ka, len(ws), wa, _ptr(out),
                                                     _stream()), self._h)
        return out.cpu().numpy()

    def apply_ttt(self, x):
        self._check(x, self.vol_shape, "x")
        out = self.new_volume()
        check(self._lib.mpi_ffl_apply_ttt(self._h, _ptr(x), _ptr(out), _stream()), self._h)
        return out

    def dot(self, a, b):
        """FP64 real inner product of two float32 CUDA tensors of equal size (a 0-d float64 tensor)."""
        if a.numel() != b.numel():
            raise ValueError("size mismatch")
        for t, nm in ((a, "a"), (b, "b")):
            self._check(t, (t.numel(),), nm)
        out = torch.empty((), device=self.device, dtype=torch.float64)
        check(self._lib.mpi_ffl_dot_f64(self._h, _ptr(a), _ptr(b), C.c_int64(a.numel()), _ptr(out), _stream()),
              self._h)
        return out

    def param_grad(self, x, grad_b, want_gain=True, want_fwhm=True):
        """(d loss/d gain [M], d loss/d fwhm [1]) for loss gradient grad_b at b = A x."""
        self._check(x, self.vol_shape, "x")
        self._check(grad_b, self.data_shape, "grad_b")
        gg = torch.empty(self.n_angles, device=self.device, dtype=torch.float32) if want_gain else None
        gf = torch.empty(1, device=self.device, dtype=torch.float32) if want_fwhm else None
        check(self._lib.mpi_ffl_param_grad(self._h, _ptr(x), _ptr(grad_b), _ptr(gg) if gg is not None else None,
                                           _ptr(gf) if gf is not None else None, _stream()), self._h)
        return gg, gf

    def project(self, x):
        """P x: projections [M, N_z, N]."""
        return self.apply_stage(0, x)

    def backproject(self, proj):
        """P^T proj: a volume."""
        return self.apply_stage(0, proj, transpose=True)

    def line_forward(self, proj, out=None):
        """blockdiag(A_DC) on projections [M, N_z, N] -> data."""
        self._check(proj, (self.n_angles, self.nz, self.nx), "proj")
        out = self.new_data() if out is None else out
        check(self._lib.mpi_ffl_line_forward(self._h, _ptr(proj), _ptr(out), _stream()), self._h)
        return out

    def line_adjoint(self, b):
        """blockdiag(A_DC)^T: data -> projections."""
        self._check(b, self.data_shape, "b")
        out = torch.empty((self.n_angles, self.nz, self.nx), device=self.device, dtype=torch.float32)
        check(self._lib.mpi_ffl_line_adjoint(self._h, _ptr(b), _ptr(out), _stream()), self._h)
        return out

    def param_grad_proj(self, proj, grad_b, want_gain=True, want_fwhm=True):
        """As param_grad, from the projections P x."""
        self._check(proj, (self.n_angles, self.nz, self.nx), "proj")
        self._check(grad_b, self.data_shape, "grad_b")
        gg = torch.empty(self.n_angles, device=self.device, dtype=torch.float32) if want_gain else None
        gf = torch.empty(1, device=self.device, dtype=torch.float32) if want_fwhm else None
        check(self._lib.mpi_ffl_param_grad_proj(self._h, _ptr(proj), _ptr(grad_b),
                                                _ptr(gg) if gg is not None else None,
                                                _ptr(gf) if gf is not None else None, _stream()), self._h)
        return gg, gf

    def power_norm(self, n_iter=50, seed=1234):
        out = C.c_double()
        check(self._lib.mpi_ffl_power_norm(self._h, int(n_iter), C.c_uint64(seed), C.byref(out), _stream()), self._h)
        return out.value

    def set_scans(self, scans):
        """Scans the solve and power iteration reconstruct from (Sec. 3.1): 'x' (the default,
        A), 'z' (the z-drive scan A_z) or 'xz' (the stacked [A; A_z]); or SCAN_* bits."""
        if isinstance(scans, str):
            scans = _lib.SCANS[scans]
        check(self._lib.mpi_ffl_set_scans(self._h, int(scans)), self._h)

    @property
    def scans(self):
        return int(self._lib.mpi_ffl_get_scans(self._h))

    @property
    def solve_data_shape(self):
        """Shape of the solve's data: the selected scans' data along the angle axis (x first)."""
        n = bin(self.scans).count("1")
        return (n * self.n_angles,) + self.data_shape[1:]

    def solve(self, b, x0=None, iters=50, lam=-1.0, tau=0.0, n_power=50, seed=1234, nonneg=True,
              stop_rel=0.0, ata_norm=0.0, report=True):
        """Run Eq. (26) on the selected scans (set_scans); returns (x, report dict or None).
        b has solve_data_shape: with both scans, torch.cat([b_x, b_z])."""
        self._check(b, self.solve_data_shape, "b")
        x = torch.zeros(self.vol_shape, device=self.device, dtype=torch.float32) if x0 is None else x0.clone()
        self._check(x, self.vol_shape, "x0")
        p = _lib.SolveParams(int(iters), float(lam), float(tau), int(n_power), C.c_uint64(seed), int(bool(nonneg)),
                             float(stop_rel), float(ata_norm))
        rep = _lib.SolveReport()
        check(self._lib.mpi_ffl_solve(self._h, _ptr(b), _ptr(x), C.byref(p), C.byref(rep) if report else None,
                                      _stream()), self._h)
        if not report:
            return x, None
        return x, dict(iters_done=rep.iters_done, tau=rep.tau, lam=rep.lambda_, ata_norm=rep.ata_norm,
                       residual_first=rep.residual_first, residual_last=rep.residual_last, b_norm=rep.b_norm)

    # ---------------------------------------------------------------- measurement
    def profile(self, enable=True):
        check(self._lib.mpi_ffl_profile_enable(self._h, int(bool(enable))), self._h)

    def profile_read(self):
        """{kernel kind: (ms, launches)} since the last read (waits for the GPU)."""
        n = len(_lib.KERNEL_KINDS)
        ms = (C.c_double * n)()
        ln = (C.c_int64 * n)()
        check(self._lib.mpi_ffl_profile_read(self._h, ms, ln), self._h)
        return {k: (ms[i], ln[i]) for i, k in enumerate(_lib.KERNEL_KINDS)}

    def sync_check(self):
        """Wait for the stream; raise if a kernel gave up on a bounded wait or the stream failed."""
        check(self._lib.mpi_ffl_sync_check(self._h, _stream()), self._h)

    def launch_count(self):
        return int(self._lib.mpi_ffl_launch_count(self._h))

    # ---------------------------------------------------------------- settings
    def set_precision(self, precision):
        check(self._lib.mpi_ffl_set_precision(self._h, int(precision)), self._h)

    def set_host_overlap(self, on=True):
        """Copy host inputs of forward/adjoint on the handle's own stream, overlapping
        the work already queued (see mpi_ffl_set_host_overlap)."""
        check(self._lib.mpi_ffl_set_host_overlap(self._h, int(bool(on))), self._h)

    @property
    def precision(self):
        return int(self._lib.mpi_ffl_get_precision(self._h))

    def set_path(self, path):
        """Evaluation path: PATH_* constant or one of 'staged', 'fused', 'line_gemm', 'full_gemm'."""
        if isinstance(path, str):
            path = _lib.PATHS[path]
        check(self._lib.mpi_ffl_set_path(self._h, int(path)), self._h)

    @property
    def path(self):
        return int(self._lib.mpi_ffl_get_path(self._h))

    def set_gain(self, gains):
        arr = (C.c_float * self.n_angles)(*[float(g) for g in gains])
        check(self._lib.mpi_ffl_set_gain(self._h, arr), self._h)
        self.gains = [float(g) for g in gains]

    def set_fwhm(self, fwhm):
        check(self._lib.mpi_ffl_set_psf_fwhm(self._h, float(fwhm)), self._h)
        self.fwhm = float(fwhm)

    def set_psf_model(self, model):
        """PSF model of the x-drive operator: 'collinear' (1D L' along the drive axis, per
        line) or 'tensor' (the in-plane tensor PSF of Appendix B, Eq. (31): every line reads
        every slice). Selecting 'tensor' builds its per-offset operator on the device."""
        if isinstance(model, str):
            model = _lib.PSF_MODELS[model]
        check(self._lib.mpi_ffl_set_psf_model(self._h, int(model)), self._h)

    @property
    def psf_model(self):
        return int(self._lib.mpi_ffl_get_psf_model(self._h))

    def set_coil_map(self, b):
        """Receive-coil sensitivity b[z][u] (N_z x N, scanner coordinates, the same for every
        angle) applied to each projection before the PSF; None restores a uniform coil."""
        if b is None:
            check(self._lib.mpi_ffl_set_coil_map(self._h, None), self._h)
            return
        arr = np.ascontiguousarray(np.asarray(b.cpu() if isinstance(b, torch.Tensor) else b, dtype=np.float32))
        if arr.shape != (self.nz, self.nx):
            raise ValueError(f"coil map must be {(self.nz, self.nx)}, got {arr.shape}")
        check(self._lib.mpi_ffl_set_coil_map(self._h, arr.ctypes.data), self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mpi_ffl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def box_stats(vol, boxes, pooled=False):
    """FP64 (count, mean, mean absolute deviation, max) of each box of a float32 CUDA volume
    [nz][ny][nx] (or of all boxes together when pooled), as an [n][4] numpy array. Boxes
    are (z0, z1, y0, y1, x0, x1), half-open (Sec. 4.2: sample values and background
    noise of a reconstruction)."""
    import numpy as np

    if not (isinstance(vol, torch.Tensor) and vol.is_cuda and vol.dtype == torch.float32 and vol.is_contiguous()
            and vol.dim() == 3):
        raise TypeError("vol must be a contiguous float32 CUDA tensor [nz][ny][nx]")
    b = np.ascontiguousarray(np.asarray(boxes, dtype=np.int32).reshape(-1, 6))
    out = np.empty((1 if pooled else len(b), 4), dtype=np.float64)
    nz, ny, nx = vol.shape
    check(_lib.load().mpi_ffl_box_stats(_ptr(vol), nz, ny, nx, b.ctypes.data, len(b), int(bool(pooled)),
                                        out.ctypes.data, _stream()))
    return out


def detection_limit(amounts, values, noise, k=3.0):
    """Least-squares line values ~ a + s * amounts and the amount at which it reaches
    k * noise (Sec. 4.2, Fig. 5): dict(limit, slope, intercept); limit NaN unless s > 0."""
    import numpy as np

    a = np.ascontiguousarray(np.asarray(amounts, dtype=np.float64))
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
    if a.shape != v.shape:
        raise ValueError("amounts and values differ in length")
    out = np.empty(3, dtype=np.float64)
    check(_lib.load().mpi_ffl_detection_limit(a.ctypes.data, v.ctypes.data, len(a), float(noise), float(k),
                                              out.ctypes.data))
    return dict(limit=float(out[0]), slope=float(out[1]), intercept=float(out[2]))
