"""ctypes binding of libmpiffl.so (include/mpi_ffl.h): structs and prototypes only.

The library is built in-tree by paper_2511_06627_gb300.build. Loading fails
loudly (RuntimeError) when it is missing: there is no CPU fallback.
"""

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpiffl.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_NONFINITE = -4
ERR_TIMEOUT = -5
ERR_UNSUPPORTED = -6

NOALLOC_MAX_PARTIALS = 65536
NOALLOC_MAX_N = NOALLOC_MAX_PARTIALS * 1024

PREC_FP32 = 0
PREC_BF16X3 = 1
PREC_TF32 = 2

STAGE_P, STAGE_H, STAGE_EVB, STAGE_F = 0, 1, 2, 3

PATH_STAGED, PATH_FUSED, PATH_LINE_GEMM, PATH_FULL_GEMM = 0, 1, 2, 3
PATHS = {"staged": PATH_STAGED, "fused": PATH_FUSED, "line_gemm": PATH_LINE_GEMM, "full_gemm": PATH_FULL_GEMM}
PSF_COLLINEAR, PSF_TENSOR = 0, 1
SCAN_X, SCAN_Z = 1, 2
SCANS = {"x": SCAN_X, "z": SCAN_Z, "xz": SCAN_X | SCAN_Z}
PSF_MODELS = {"collinear": PSF_COLLINEAR, "tensor": PSF_TENSOR}


class Geometry(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("n_angles", C.c_int32),
                ("angles_rad", C.POINTER(C.c_double)), ("gain", C.POINTER(C.c_float))]


class Trajectory(C.Structure):
    _fields_ = [("samples_per_period", C.c_int32), ("periods_per_line", C.c_int32),
                ("drive_amp_vox", C.c_double), ("drive_phase", C.c_double),
                ("zigzag", C.c_int32), ("upsample_q", C.c_int32)]


class Psf(C.Structure):
    _fields_ = [("fwhm_vox", C.c_double)]


class Harmonics(C.Structure):
    _fields_ = [("k_min", C.c_int32), ("k_max", C.c_int32), ("half_width", C.c_int32),
                ("d_gamma_ri", C.POINTER(C.c_float))]


class SolveParams(C.Structure):
    _fields_ = [("iters", C.c_int32), ("lambda_", C.c_double), ("tau", C.c_double),
                ("n_power", C.c_int32), ("seed", C.c_uint64), ("nonneg", C.c_int32),
                ("stop_rel", C.c_double), ("ata_norm", C.c_double)]


class SolveReport(C.Structure):
    _fields_ = [("iters_done", C.c_int32), ("tau", C.c_double), ("lambda_", C.c_double),
                ("ata_norm", C.c_double), ("residual_first", C.c_double),
                ("residual_last", C.c_double), ("b_norm", C.c_double)]


class Sizes(C.Structure):
    _fields_ = [("n_vox", C.c_int64), ("n_data", C.c_int64), ("n_proj", C.c_int64),
                ("n_fine", C.c_int64), ("n_sig", C.c_int64), ("n_bins", C.c_int32),
                ("fine_len", C.c_int32), ("line_len", C.c_int32), ("workspace_bytes", C.c_int64),
                ("fine_len_z", C.c_int32)]


class JobStatus(C.Structure):
    _fields_ = [("iters_done", C.c_int32), ("stopped", C.c_int32), ("finished", C.c_int32),
                ("residual_first", C.c_double), ("residual_last", C.c_double), ("tau", C.c_double),
                ("lambda_", C.c_double), ("device_bytes", C.c_int64)]


H = C.c_void_p
FP = C.c_void_p  # device float* (passed as integer addresses)
ST = C.c_void_p  # cudaStream_t

PROTOTYPES = {
    "mpi_ffl_create": (C.c_int, [C.POINTER(Geometry), C.POINTER(Trajectory), C.POINTER(Psf),
                                 C.POINTER(Harmonics), C.POINTER(H)]),
    "mpi_ffl_destroy": (C.c_int, [H]),
    "mpi_ffl_last_error": (C.c_char_p, [H]),
    "mpi_ffl_get_sizes": (C.c_int, [H, C.POINTER(Sizes)]),
    "mpi_ffl_set_precision": (C.c_int, [H, C.c_int32]),
    "mpi_ffl_set_path": (C.c_int, [H, C.c_int32]),
    "mpi_ffl_get_path": (C.c_int, [H]),
    "mpi_ffl_get_precision": (C.c_int, [H]),
    "mpi_ffl_set_host_overlap": (C.c_int, [H, C.c_int32]),
    "mpi_ffl_band_energy": (C.c_int, [H, FP, FP, FP, FP]),
    "mpi_ffl_forward_zdrive": (C.c_int, [H, FP, FP, FP]),
    "mpi_ffl_adjoint_zdrive": (C.c_int, [H, FP, FP, FP]),
    "mpi_ffl_apply_stage_zdrive": (C.c_int, [H, C.c_int32, C.c_int32, FP, FP, FP]),
    "mpi_ffl_set_gain": (C.c_int, [H, C.POINTER(C.c_float)]),
    "mpi_ffl_set_psf_fwhm": (C.c_int, [H, C.c_double]),
    "mpi_ffl_set_psf_model": (C.c_int, [H, C.c_int32]),
    "mpi_ffl_get_psf_model": (C.c_int, [H]),
    "mpi_ffl_set_coil_map": (C.c_int, [H, FP]),
    "mpi_ffl_set_scans": (C.c_int, [H, C.c_int32]),
    "mpi_ffl_get_scans": (C.c_int, [H]),
    "mpi_ffl_box_stats": (C.c_int, [FP, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                    C.c_void_p, ST]),
    "mpi_ffl_detection_limit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_void_p]),
    "mpi_ffl_sync_check": (C.c_int, [H, ST]),
    "mpi_ffl_forward": (C.c_int, [H, FP, FP, ST]),
    "mpi_ffl_adjoint": (C.c_int, [H, FP, FP, ST]),
    "mpi_ffl_apply_stage": (C.c_int, [H, C.c_int32, C.c_int32, FP, FP, ST]),
    "mpi_ffl_param_grad": (C.c_int, [H, FP, FP, FP, FP, ST]),
    "mpi_ffl_param_grad_proj": (C.c_int, [H, FP, FP, FP, FP, ST]),
    "mpi_ffl_line_forward": (C.c_int, [H, FP, FP, ST]),
    "mpi_ffl_line_adjoint": (C.c_int, [H, FP, FP, ST]),
    "mpi_ffl_apply_ttt": (C.c_int, [H, FP, FP, ST]),
    "mpi_ffl_dot_f64": (C.c_int, [H, FP, FP, C.c_int64, FP, ST]),
    "mpi_ffl_dot_f64_noalloc": (C.c_int, [FP, FP, C.c_int64, FP, ST]),
    "mpi_ffl_power_norm": (C.c_int, [H, C.c_int32, C.c_uint64, C.POINTER(C.c_double), ST]),
    "mpi_ffl_solve": (C.c_int, [H, FP, FP, C.POINTER(SolveParams), C.POINTER(SolveReport), ST]),
    "mpi_ffl_profile_enable": (C.c_int, [H, C.c_int32]),
    "mpi_ffl_profile_read": (C.c_int, [H, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "mpi_ffl_launch_count": (C.c_int64, [H]),
    "mpi_ffl_job_create": (C.c_int, [H, FP, FP, C.POINTER(SolveParams), C.POINTER(C.c_void_p), ST]),
    "mpi_ffl_job_step": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, ST]),
    "mpi_ffl_job_status": (C.c_int, [C.c_void_p, C.POINTER(JobStatus), ST]),
    "mpi_ffl_job_flags": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "mpi_ffl_job_poll": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, ST]),
    "mpi_ffl_job_result": (C.c_int, [C.c_void_p, FP, ST]),
    "mpi_ffl_job_destroy": (C.c_int, [C.c_void_p]),
    "mpi_ffl_test_fail_alloc": (C.c_int, [C.c_int32]),
    "mpi_ffl_test_live_allocs": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mpi_ffl_test_inject_timeout": (C.c_int, [H, C.c_uint32]),
    "mpi_ffl_probe_smem_bandwidth": (C.c_int, [C.POINTER(C.c_double), ST]),
    "mpi_ffl_information_retained": (C.c_int, [H, FP, C.c_int32, C.POINTER(C.c_int32), C.c_int32,
                                               C.POINTER(C.c_int32), FP, ST]),
}

KERNEL_KINDS = ["transpose", "project", "backproject", "psf_fwd", "psf_adj", "resample_fwd", "resample_adj",
                "dft_fwd", "dft_adj", "tc_fwd", "tc_adj", "solver", "gemm_fwd", "gemm_adj", "zdrive",
                "tensor", "coil"]

_lib = None


def load():
    """Load libmpiffl.so and declare its prototypes (RuntimeError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2511_06627_gb300.build` "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MpiFflError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mpi_ffl error {code}: {msg}")
        self.code = code


def check(rc, handle=None):
    if rc != OK:
        msg = load().mpi_ffl_last_error(handle)
        raise MpiFflError(rc, msg.decode() if msg else "")
    return rc
