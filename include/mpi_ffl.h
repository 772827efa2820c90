/*
 * mpi_ffl.h -- C ABI of the GB300 library for the compressed 3D field-free-line
 * (FFL) MPI operator and its regularised reconstruction (arXiv 2511.06627).
 *
 * Operator (Sec. 2.2, Eq. (23); Sec. 3.3, Eq. (24)):
 *     b = A x,  A = blockdiag_m(S D_Gamma F V E H B) [P_theta_1; ...; P_theta_M]
 *   P_theta  parallel-beam line integrals about z (Sec. 2.2, Eqs. (16)-(19)),
 *            Joseph interpolation, rays marched along rows when |cos| >= |sin|
 *   B        one scalar gain per angle (uniform receive coil, Sec. 1.3 Table 1)
 *   H        Langevin-derivative PSF along the drive axis, h(u) = 3 L'(u/a) with
 *            full width at half maximum fwhm_vox (Appendix B, Eq. (31)); evaluated
 *            on a grid upsample_q times finer than the detector bins, full support
 *   E, V     the convolved row sampled at the FFL position xi_j by linear
 *            interpolation on that grid, times the FFL velocity v_j (Eq. (7))
 *   F        unitary DFT with the +i sign (Appendix A, Eq. (27))
 *   D_Gamma  receive-chain transfer function on the kept bins (Sec. 2.1, Eq. (13))
 *   S        harmonic-band selection (Sec. 2.1, Eq. (11)): bins k*P + delta,
 *            k = k_min..k_max, delta = -half_width..half_width
 * Reconstruction (Sec. 3.3, Eqs. (25)-(26)): accelerated projected gradient
 * descent on ||A x - b||^2 + lambda ||T x||^2, T = forward differences along
 * x, y, z with no wrap-around.
 *
 * Layouts
 *   volume  float x[z][y][x], nx == ny, contiguous
 *   data    float b[m][z][k][delta][2]: complex (re, im) interleaved, one raster
 *           line per z slice, bins k-major with delta ascending
 *   A^T is taken under the real inner product: x = Re(A^H b).
 *
 * Ownership and streams
 *   Every pointer named d_* is device memory owned by the caller. The handle owns
 *   its tables and workspace and copies every host array it is given at create.
 *   All work is enqueued on the caller's stream (cudaStream_t passed as void*,
 *   NULL = legacy default stream); calls return without waiting for the GPU unless
 *   stated. A handle may be used from one stream at a time.
 *
 * Determinism
 *   No kernel uses atomics; every sum runs in a fixed order. Repeating a call with
 *   the same handle settings on the same input gives the same bits, on every path
 *   and precision, for A, A^T, the stages, the z-drive scan, the power norm and the
 *   solve.
 *
 * Errors
 *   Every call returns 0 on success or a negative MPI_FFL_ERR_* code; nothing
 *   throws or aborts across the ABI. mpi_ffl_last_error() gives a message for the
 *   last failure of a handle (or of create, when passed NULL; thread-local).
 */
#ifndef MPI_FFL_H
#define MPI_FFL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPI_FFL_OK 0
#define MPI_FFL_ERR_INVALID_ARG (-1)
#define MPI_FFL_ERR_OOM (-2)
#define MPI_FFL_ERR_CUDA (-3)
#define MPI_FFL_ERR_NONFINITE (-4)
#define MPI_FFL_ERR_TIMEOUT (-5)
#define MPI_FFL_ERR_UNSUPPORTED (-6)

/* Arithmetic of the harmonic-band DFT and its transpose (the other stages are FP32). */
#define MPI_FFL_PREC_FP32 0   /* plain: FP32 FMA on CUDA cores, stage by stage        */
#define MPI_FFL_PREC_BF16X3 1 /* tensor cores: bf16 hi+lo split, 3 products, FP32 acc  */
#define MPI_FFL_PREC_TF32 2   /* tensor cores: tf32 hi+lo split, 3 products, FP32 acc  */

/* How A and A^T are evaluated (the operator is the same; only the order of evaluation
 * and the arithmetic differ):
 *   STAGED     P, H, E V B and S D_Gamma F as separate FP32 CUDA-core kernels; the
 *              time signal (L floats per line) passes through HBM. Precision FP32.
 *   FUSED      P and H as above; E V B fused with the band DFT on tensor cores
 *              (tcgen05, BF16x3): the time signal stays on chip.
 *   LINE_GEMM  P and H as above; S D_Gamma F V E, identical for every line of one
 *              trajectory, precomputed in double precision as one matrix per
 *              trajectory (the reassociation of Sec. 2.1, Eq. (13)) and applied as a
 *              tensor-core GEMM (BF16x3).
 *   FULL_GEMM  P, then S D_Gamma F V E H as one matrix per trajectory (BF16x3). */
#define MPI_FFL_PATH_STAGED 0
#define MPI_FFL_PATH_FUSED 1
#define MPI_FFL_PATH_LINE_GEMM 2
#define MPI_FFL_PATH_FULL_GEMM 3

typedef struct mpi_ffl_handle mpi_ffl_handle;

/* Volume and FFL angles (Sec. 2.2; Sec. 3.1: angles equally spaced over 180 deg). */
typedef struct {
    int32_t nx, ny, nz;        /* nx == ny; voxel (x, y) of slice z at x[(z*ny+y)*nx+x]      */
    int32_t n_angles;          /* M >= 1                                                  */
    const double *angles_rad;  /* host, n_angles; NULL -> theta_m = m*pi/M                */
    const float *gain;         /* host, n_angles; NULL -> 1 (B of Sec. 1.3, Table 1)      */
} mpi_ffl_geometry;

/* Drive and slow raster (Sec. 1.2, Eqs. (3)-(4); Sec. 3.1). One raster line per z slice:
 * xi_j = c_j + A sin(2 pi j / S + phi0), c_j = (N-1) j / (L-1) (reversed on odd lines
 * when zigzag), j = 0..L-1, L = S*P; v_j = d xi / d j in detector bins per sample. */
typedef struct {
    int32_t samples_per_period; /* S >= 2                                         */
    int32_t periods_per_line;   /* P >= 1                                         */
    double drive_amp_vox;       /* A >= 0, in detector bins (= voxels)            */
    double drive_phase;         /* phi0, radians                                  */
    int32_t zigzag;             /* 1: odd lines run backwards                     */
    int32_t upsample_q;         /* Q in {1,2,4,...,32}, fine-grid factor of H      */
} mpi_ffl_trajectory;

/* Langevin-derivative PSF width (Appendix B, Eq. (31)). */
typedef struct {
    double fwhm_vox; /* > 0 */
} mpi_ffl_psf;

/* Kept harmonic bands (Sec. 2.1, Eqs. (11), (13)). Requires k_min*P - half_width >= 1
 * and k_max*P + half_width < L/2. */
typedef struct {
    int32_t k_min, k_max, half_width;
    const float *d_gamma_ri; /* host, n_bins complex (re, im) or NULL = identity */
} mpi_ffl_harmonics;

/* Solver settings (Sec. 3.3, Eq. (26)). */
typedef struct {
    int32_t iters;     /* K >= 0 iterations                                            */
    double lambda;     /* < 0 -> 1e-3 * ||A^T A|| / ||T^T T||                          */
    double tau;        /* > 0 used as given; <= 0 -> 1 / (||A^T A|| + lambda ||T^T T||) */
    int32_t n_power;   /* power iterations for ||A^T A|| when it is needed (e.g. 50)   */
    uint64_t seed;     /* SplitMix64 seed of the power-iteration start vector          */
    int32_t nonneg;    /* 1: project each update onto x >= 0                           */
    double stop_rel;   /* > 0: stop when |r_k - r_{k-1}| <= stop_rel r_{k-1}          */
    double ata_norm;   /* > 0: use as ||A^T A|| and skip the power iteration           */
} mpi_ffl_solve_params;

typedef struct {
    int32_t iters_done;
    double tau, lambda, ata_norm;
    double residual_first; /* ||A y - b|| at the first iteration (FP64) */
    double residual_last;  /* ||A y - b|| at the last iteration  (FP64) */
    double b_norm;         /* ||b||                                     */
} mpi_ffl_solve_report;

/* Sizes of a problem, in elements. */
typedef struct {
    int64_t n_vox;   /* nz*ny*nx floats of a volume                       */
    int64_t n_data;  /* 2 * M * nz * n_bins floats of the data             */
    int64_t n_proj;  /* M * nz * nx floats of the projections              */
    int64_t n_fine;  /* M * nz * N_e floats of the PSF-convolved rows      */
    int64_t n_sig;   /* M * nz * L floats of the time signal               */
    int32_t n_bins;  /* (k_max - k_min + 1) * (2 half_width + 1)           */
    int32_t fine_len;/* N_e = (nx-1) Q + 2 ceil(A Q) + 1                  */
    int32_t line_len;/* L = S P                                           */
    int64_t workspace_bytes; /* device memory the handle holds            */
    int32_t fine_len_z; /* N_ez = (N_z - 1) Q + 2 D + 1: fine z grid of the z-drive scan */
} mpi_ffl_sizes;

/* Create a handle on the current CUDA device: validates the description, builds the
 * PSF, trajectory and DFT tables in double precision on the host and uploads them,
 * and allocates the workspace. Returns MPI_FFL_ERR_INVALID_ARG for an invalid
 * description (nx != ny, band outside 1 <= omega < L/2, ...), MPI_FFL_ERR_OOM when a
 * device allocation fails (nothing is leaked), MPI_FFL_ERR_CUDA otherwise. */
int mpi_ffl_create(const mpi_ffl_geometry *geom, const mpi_ffl_trajectory *traj,
                   const mpi_ffl_psf *psf, const mpi_ffl_harmonics *harm,
                   mpi_ffl_handle **out);

/* Release the handle and everything it owns. destroy(NULL) returns 0. Waits for the
 * device to finish work that uses the handle's memory. */
int mpi_ffl_destroy(mpi_ffl_handle *h);

/* Message of the last failure of h (NULL: of the last failed create or handle-free
 * call on this thread). */
const char *mpi_ffl_last_error(const mpi_ffl_handle *h);

int mpi_ffl_get_sizes(const mpi_ffl_handle *h, mpi_ffl_sizes *out);

/* Arithmetic of the line stages for forward/adjoint/solve (MPI_FFL_PREC_*). FP32
 * selects the STAGED path; BF16X3 keeps a tensor-core path, or selects FUSED when the
 * path was STAGED. TF32 (22 of 24 mantissa bits per operand, about 8x smaller error
 * than BF16X3) applies to the two GEMM paths and returns MPI_FFL_ERR_UNSUPPORTED on
 * the others. set_path keeps TF32 when moving between the GEMM paths. */
int mpi_ffl_set_precision(mpi_ffl_handle *h, int32_t precision);
/* Current precision (MPI_FFL_PREC_*), or MPI_FFL_ERR_INVALID_ARG for a NULL handle. */
int mpi_ffl_get_precision(const mpi_ffl_handle *h);

/* Evaluation path (MPI_FFL_PATH_*); returns MPI_FFL_ERR_UNSUPPORTED when the shape is
 * outside what the path's kernels accept (the handle keeps its previous path). */
int mpi_ffl_set_path(mpi_ffl_handle *h, int32_t path);
int mpi_ffl_get_path(const mpi_ffl_handle *h);

/* Replace the per-angle gains (host array of n_angles) or the PSF width. Both take
 * effect for work enqueued after the call returns; the call synchronises the device
 * before touching tables that queued work may still read. A new PSF width also
 * rebuilds the collapsed line operator (W H), which takes a moment on the host. */
int mpi_ffl_set_gain(mpi_ffl_handle *h, const float *gain);
int mpi_ffl_set_psf_fwhm(mpi_ffl_handle *h, double fwhm_vox);

/* PSF models of the x-drive operator (forward, adjoint, solve, line stages). */
#define MPI_FFL_PSF_COLLINEAR 0   /* 1D h(u) = 3 L'(u/a) along the drive axis, per line */
#define MPI_FFL_PSF_TENSOR 1      /* in-plane tensor PSF: lines coupled across slices */

/* Select the PSF model. TENSOR uses the (x, x) component of the tensor PSF of
 * Appendix B, Eq. (31) in the FFL plane: h_uu(u, z) = 3 [L'(xi) u^2/rho^2 +
 * (L(xi)/xi) z^2/rho^2], xi = rho / a, rho^2 = u^2 + z^2, a from the FWHM along the drive
 * axis as for COLLINEAR (on z = 0 the two agree). Every line then reads every slice of
 * its projection, c[l][e] = sum_{z', i} p[z'][i] h_uu(u_lo + e/Q - i, l - z'), with full
 * support. It runs as one GEMM per line (forward) or per slice (adjoint) against
 * per-offset folded line operators W H_d, built on the device in FP64 when the model is
 * first selected (2 n_par (2 N_z - 1) 2 n_b N split operands, 4 bytes each, plus
 * n_par N_z 2 n_b N doubles) and again after set_psf_fwhm or a precision change. It
 * needs the collapsed line operator (the GEMM paths' tables) and applies whatever
 * the handle's path; MPI_FFL_ERR_UNSUPPORTED otherwise. Gradients of mpi_ffl_param_grad
 * and the batched jobs API use COLLINEAR only (MPI_FFL_ERR_UNSUPPORTED / the job runs
 * alone). The call synchronises the device. */
int mpi_ffl_set_psf_model(mpi_ffl_handle *h, int32_t model);
int mpi_ffl_get_psf_model(const mpi_ffl_handle *h);

/* Receive-coil sensitivity map (operator B of Eq. (13)): host array b[z][u] of N_z x N
 * floats in scanner coordinates, the same for every angle (the object rotates, the
 * scanner does not, Eq. (19)); NULL restores a uniform coil. The x-drive operator
 * multiplies each projection by b before its PSF (both models) and its transpose
 * multiplies after; the per-angle gains still apply. The z-drive scan is unaffected.
 * The call synchronises the device. */
int mpi_ffl_set_coil_map(mpi_ffl_handle *h, const float *b_zu);

/* Waits for the stream, then reports whether a kernel of the handle gave up on a
 * bounded wait since the last check (MPI_FFL_ERR_TIMEOUT; the flag is cleared) or
 * the stream holds a CUDA error (MPI_FFL_ERR_CUDA). */
int mpi_ffl_sync_check(mpi_ffl_handle *h, void *stream);

/* b = A x (Sec. 2.2, Eq. (23)). x: n_vox floats; b_ri: n_data floats (written).
 * Either buffer may be device memory or host memory (pinned for asynchronous
 * copies): a host input is copied to the handle's device staging before use and a
 * host output is copied back on `stream`, so it is complete when the stream is. The
 * call is asynchronous: a host input must stay unchanged until the stream's work
 * has completed. */
int mpi_ffl_forward(mpi_ffl_handle *h, const float *x, float *b_ri, void *stream);

/* x = A^T b = Re(A^H b) (transpose of Eq. (23) under the real inner product). Host
 * or device buffers, as mpi_ffl_forward. */
int mpi_ffl_adjoint(mpi_ffl_handle *h, const float *b_ri, float *x, void *stream);

/* The z-drive scan of the dual-drive acquisition (Sec. 3.1: at every angle one scan
 * drives the FFL along x, one along z). Same raster, trajectory parameters, kept bins,
 * D_Gamma and gains as the x-drive scan of mpi_ffl_forward; the drive and the 1D
 * Langevin-derivative PSF act along z. Sample j of line l reads the z-convolved
 * projection, evaluated on a grid Q times finer than the slices (N_ez =
 * (N_z - 1) Q + 2 D + 1 points from -D/Q), bilinearly at detector position c_j (the
 * slow raster) and height l + A sin(2 pi j / S + phi0), and is weighted by the drive
 * velocity along z and the gain. b_z has the layout of b (n_data floats). The
 * dual-drive operator is [A; A_z] with transpose A^T y + A_z^T y_z. FP32 kernels
 * that fuse E_z V_z B with S D_Gamma F (and their transposes), so no time signal is
 * stored. The first call builds the z tables and allocates the z workspace (the fine
 * z grid M N N_ez floats, the projections by column M N N_z floats, the transpose's
 * synthesis coefficients M N_z (2w+1) S floats). It returns MPI_FFL_ERR_UNSUPPORTED
 * when (N_z + 1) S floats exceed 200 KB or the fused kernels' shared-memory tiles
 * exceed 227 KB. Host or device buffers, as mpi_ffl_forward. */
int mpi_ffl_forward_zdrive(mpi_ffl_handle *h, const float *x, float *b_z_ri, void *stream);
int mpi_ffl_adjoint_zdrive(mpi_ffl_handle *h, const float *b_z_ri, float *x, void *stream);

/* Scans of mpi_ffl_solve and mpi_ffl_power_norm (Sec. 3.1: an x-drive and a z-drive scan
 * at every angle). MPI_FFL_SCAN_X (the default) is A alone; MPI_FFL_SCAN_Z is A_z alone;
 * both reconstruct from the stacked operator [A; A_z], whose data d_b are the two scans'
 * data one after the other (x first), 2 n_data floats, and whose transpose is
 * A^T r + A_z^T r_z. ||A^T A|| of the power iteration and the default lambda and tau
 * then refer to that operator. mpi_ffl_forward/adjoint stay the x-drive scan;
 * param_grad and jobs refuse other scan sets (MPI_FFL_ERR_UNSUPPORTED). Selecting the
 * z scan builds its tables (as mpi_ffl_forward_zdrive); both scans add 2 n_data +
 * 2 n_vox floats of workspace. The call synchronises the device. */
#define MPI_FFL_SCAN_X 1
#define MPI_FFL_SCAN_Z 2
int mpi_ffl_set_scans(mpi_ffl_handle *h, int32_t scans);
int mpi_ffl_get_scans(const mpi_ffl_handle *h);

/* Stages of the z-drive scan on caller device buffers (transpose = 1 for the
 * transpose): stage 1 = H_z: proj [M][N_z][N] <-> fine_z [M][N][N_ez];
 * stage 2 = E_z V_z B: fine_z <-> sig [M][N_z][L]. P and S D_Gamma F are the x-drive
 * stages 0 and 3 of mpi_ffl_apply_stage. The first transpose of stage 2 allocates its
 * per-phase partials (M N_z N S floats). */
int mpi_ffl_apply_stage_zdrive(mpi_ffl_handle *h, int32_t stage, int32_t transpose, const float *d_in,
                               float *d_out, void *stream);

/* Detection-limit analysis (Sec. 4.2, Fig. 5), handle-free.
 *
 * mpi_ffl_box_stats: FP64 statistics of boxes of a volume d_vol (device, nz x ny x nx
 * floats, x fastest). boxes: host array of n_boxes x 6 int32 (z0, z1, y0, y1, x0, x1),
 * half-open and inside the volume. pooled = 0: out (host, n_boxes x 4 doubles) gets,
 * per box, (voxel count, mean, mean absolute deviation about the mean, max); pooled = 1:
 * one such row for all boxes taken together (the noise of Fig. 5 over void regions).
 * Synchronous: waits for `stream`, which it uses for its two kernels and copies. It
 * allocates a few bytes of device memory per call. The sums are in a fixed order:
 * repeated calls give the same bits. MPI_FFL_ERR_INVALID_ARG for an empty box or one
 * leaving the volume.
 *
 * mpi_ffl_detection_limit (host only): least-squares line values = a + s * amounts over
 * n >= 2 samples; out (3 doubles) = (limit, s, a), limit = (k * noise - a) / s, NaN
 * unless s > 0 (k = 3 in Fig. 5). MPI_FFL_ERR_INVALID_ARG when all amounts are equal. */
int mpi_ffl_box_stats(const float *d_vol, int32_t nz, int32_t ny, int32_t nx, const int32_t *boxes, int32_t n_boxes,
                      int32_t pooled, double *out, void *stream);
int mpi_ffl_detection_limit(const double *amounts, const double *values, int32_t n, double noise, double k,
                            double *out);

/* on != 0: host inputs of forward/adjoint are copied on a stream of the handle that
 * waits only for the previous use of its (double-buffered) staging slot, so the copy
 * for the next call overlaps the work already queued on `stream`. The caller must
 * then not produce a host input with work queued on `stream` (for example a host
 * output of the previous call) without synchronising the stream first. Default 0:
 * copies are ordered on `stream`. */
int mpi_ffl_set_host_overlap(mpi_ffl_handle *h, int32_t on);

/* One stage of A or of A^T on caller buffers, for stage-by-stage checks:
 *   stage 0 = P   (n_vox  <-> n_proj)      stage 1 = H (n_proj <-> n_fine)
 *   stage 2 = EVB (n_fine <-> n_sig)       stage 3 = S D_Gamma F (n_sig <-> n_data)
 * transpose = 0 applies the stage, 1 its transpose. Stage 3 uses the precision set by
 * mpi_ffl_set_precision only when it is FP32; the tensor-core precisions are used
 * by forward/adjoint, where the DFT is fused with E V B. */
int mpi_ffl_apply_stage(mpi_ffl_handle *h, int32_t stage, int32_t transpose,
                        const float *d_in, float *d_out, void *stream);

/* Gradients for calibration (the scan nonidealities of Sec. 1): given x and the
 * gradient g_b of a loss with respect to b = A x (n_data floats), writes
 *   d_g_gain[m] = <g_b[m], A_m x> / gain_m  (= d loss / d gain_m), n_angles floats
 *   d_g_fwhm[0] = <g_b, (d A / d fwhm) x>  (= d loss / d fwhm)
 * with real inner products accumulated in FP64 and stored as FP32. Either output may
 * be NULL. The gradient with respect to x is mpi_ffl_adjoint(g_b). */
int mpi_ffl_param_grad(mpi_ffl_handle *h, const float *d_x, const float *d_gb_ri,
                       float *d_g_gain, float *d_g_fwhm, void *stream);

/* Real inner product <a, b> = sum_i a_i b_i of two float arrays of n elements
 * (volumes, or interleaved complex data, whose real inner product is the one of
 * Sec. 3.3, Eq. (26)), accumulated in FP64 with a fixed summation order and written
 * to d_out (one double, device memory). Uses the handle's reduction scratch, so calls
 * on one handle must not overlap on the GPU. n >= 0. */
int mpi_ffl_dot_f64(mpi_ffl_handle *h, const float *d_a, const float *d_b, int64_t n, double *d_out,
                    void *stream);

/* As mpi_ffl_param_grad, from the projections P x (n_proj floats, e.g. kept from the
 * forward as a checkpoint) instead of x, so P is not applied again. */
int mpi_ffl_param_grad_proj(mpi_ffl_handle *h, const float *d_proj, const float *d_gb_ri, float *d_g_gain,
                            float *d_g_fwhm, void *stream);

/* The per-angle line operators alone (Sec. 2.2, Eq. (23) without P):
 * b = blockdiag_m(A_DC) proj and proj = blockdiag_m(A_DC)^T b, on the current path.
 * d_proj: n_proj floats [m][z][i]; d_b: n_data floats. */
int mpi_ffl_line_forward(mpi_ffl_handle *h, const float *d_proj, float *d_b_ri, void *stream);
int mpi_ffl_line_adjoint(mpi_ffl_handle *h, const float *d_b_ri, float *d_proj, void *stream);

/* Compression analysis (Appendix A, Eq. (30)). With s = E V B H P x the time signal
 * of every segment (staged FP32 kernels), writes on the device, in FP64:
 *   d_bin_energy[q] = sum over segments of |s_hat_w|^2, w = kP + delta the q-th kept
 *                     bin (data order: k ascending, then delta ascending), s_hat the
 *                     unitary DFT of Sec. 2.1 without D_Gamma (n_bins doubles);
 *   d_total[0]      = sum over segments of ||s||^2.
 * For a real signal the bin L - w carries the same energy as w, so the information a
 * sub-band S' of the kept bins retains, counting each bin with its conjugate, is
 * I = sqrt(2 sum_{q in S'} d_bin_energy[q] / d_total[0]). Uses the time-signal
 * workspace (n_sig floats, allocated on first use). */
int mpi_ffl_band_energy(mpi_ffl_handle *h, const float *d_x, double *d_bin_energy, double *d_total, void *stream);

/* The information retained (Appendix A, Eq. (30)) by sub-bands of the kept bins, for the
 * time signal of x (as mpi_ffl_band_energy computes it): for a = 0..n_k-1 and
 * c = 0..n_w-1, d_out[a n_w + c] (device, FP64) = sqrt(2 sum_{q in S'} e_q / total) with
 * S' the kept bins of harmonics k_min..k_max[a] and |delta| <= half_width[c], each bin
 * counted with its conjugate. k_max (host, n_k <= 16 values in k_min..k_max of the
 * handle) and half_width (host, n_w <= 16 values in 0..half_width of the handle); other
 * values are MPI_FFL_ERR_INVALID_ARG. Uses the time-signal workspace. */
int mpi_ffl_information_retained(mpi_ffl_handle *h, const float *d_x, int32_t n_k, const int32_t *k_max,
                                 int32_t n_w, const int32_t *half_width, double *d_out, void *stream);

/* T^T T x (Sec. 3.3, Eq. (25)) on a volume. */
int mpi_ffl_apply_ttt(mpi_ffl_handle *h, const float *d_x, float *d_out, void *stream);

/* ||A^T A||_2 by n_iter power iterations from a SplitMix64(seed) start vector (the
 * Rayleigh quotient of the last iterate, FP64). Synchronises the stream. */
int mpi_ffl_power_norm(mpi_ffl_handle *h, int32_t n_iter, uint64_t seed, double *out, void *stream);

/* Reconstruct: runs Eq. (26) from x0 = d_x_inout, writes the result to d_x_inout.
 * d_b_ri: n_data floats. Residual norms are reduced in FP64 on the device. If report
 * is non-NULL the call synchronises the stream and fills it; otherwise it returns as
 * soon as the work is enqueued (unless the power iteration or stop_rel needs a value
 * on the host). Returns MPI_FFL_ERR_NONFINITE if a residual norm is not finite. */
int mpi_ffl_solve(mpi_ffl_handle *h, const float *d_b_ri, float *d_x_inout,
                  const mpi_ffl_solve_params *params, mpi_ffl_solve_report *report,
                  void *stream);

/* ---- Continuous batching (serving) -------------------------------------------------
 * A job is one reconstruction of Eq. (26) on its own handle (the handle must not be
 * used for anything else while the job lives): it owns a device copy of the data and
 * the solver state (x, x_prev, y, gradient, residual, residual history), so nothing
 * crosses PCIe between iterations. mpi_ffl_job_step advances any set of jobs by one
 * iteration each; jobs whose handles are on the FULL_GEMM path share one launch per
 * kernel kind (momentum, projector, line GEMM, residual, norm and stop test, adjoint
 * line GEMM, backprojector, update), jobs on other paths run their A and A^T alone
 * between those launches. A job that meets its stop test does no further work on the
 * device; a job that has used its iteration budget is skipped by the host. */
typedef struct mpi_ffl_job mpi_ffl_job;

typedef struct {
    int32_t iters_done;      /* iterations completed                               */
    int32_t stopped;         /* 1: stop test met, 2: non-finite residual            */
    int32_t finished;        /* stopped or iteration budget used                    */
    double residual_first;   /* ||A y - b|| of the first iteration (FP64)          */
    double residual_last;    /* ||A y - b|| of the last iteration (FP64)           */
    double tau, lambda;
    int64_t device_bytes;    /* device memory the job owns (besides its handle)    */
} mpi_ffl_job_status_t;

/* Allocates the job's state, copies d_b (n_data floats) and x0 (n_vox floats or NULL
 * for zero), and fixes tau and lambda as mpi_ffl_solve does (running the power
 * iteration on the handle if needed, which synchronises the stream). */
int mpi_ffl_job_create(mpi_ffl_handle *h, const float *d_b, const float *d_x0, const mpi_ffl_solve_params *p,
                       mpi_ffl_job **out, void *stream);
int mpi_ffl_job_step(mpi_ffl_job *const *jobs, int32_t n, void *stream);
/* Synchronises the stream and reads the job's progress. */
int mpi_ffl_job_status(const mpi_ffl_job *j, mpi_ffl_job_status_t *out, void *stream);
/* Device pointer to the job's three int flags: [0] stop verdict, [1] iterations done,
 * [2] frozen. A server can copy them asynchronously to poll many jobs at once. */
int mpi_ffl_job_flags(const mpi_ffl_job *j, const int32_t **d_flags);
/* Enqueues copies of the flags of jobs[0..n) into host_flags (3 per job; pinned host
 * memory for asynchrony); the values are valid once the stream has reached them. */
int mpi_ffl_job_poll(mpi_ffl_job *const *jobs, int32_t n, int32_t *host_flags, void *stream);
/* Copies the current iterate to d_x (n_vox floats). */
int mpi_ffl_job_result(const mpi_ffl_job *j, float *d_x, void *stream);
/* Waits for the device and frees the job's state (not its handle). NULL is a no-op. */
int mpi_ffl_job_destroy(mpi_ffl_job *j);

/* ---- Handle-free entry point that allocates nothing -----------------------------
 * The paper has no counterpart to this call; it serves callers that cannot call
 * cudaMalloc (or mpi_ffl_create, which allocates): for example code running while a
 * framework's caching allocator has reserved the device memory, code that must not
 * risk the implicit device synchronisation of an allocation, or real-time loops
 * that forbid allocation latency.
 *
 * <a, b> = sum_i a_i b_i of two float arrays of n elements (device memory), summed
 * in FP64 in a fixed order and written to d_out (one double, device memory). It is
 * the computation of mpi_ffl_dot_f64 without a handle: its scratch is a file-scope
 * device array of MPI_FFL_NOALLOC_MAX_PARTIALS doubles (512 KiB, held by every GPU
 * that loads the library until the process exits), one partial sum per block of
 * 1024 elements, so n <= MPI_FFL_NOALLOC_MAX_N; larger n returns
 * MPI_FFL_ERR_INVALID_ARG with a message and launches nothing. It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *
 * The first call on a device looks up the array's device address on the current
 * device (cudaGetSymbolAddress) once and keeps it for the life of the process; make
 * that first call before any stream capture. The kept address does not survive a
 * cudaDeviceReset of that device: a process that resets a device must not call this
 * entry point on it afterwards. A launch error is returned as MPI_FFL_ERR_CUDA; an
 * error that an earlier runtime call left pending on the calling thread is left
 * pending, not reported as this call's. Every call on a device shares the array and leaves its partial sums
 * there; each call writes all the partials it reads before reading them, so nothing
 * has to be cleared between calls. Calls whose work overlaps on the GPU (on
 * different streams, unordered) race on the array and give wrong results: order
 * them on one stream or with events. Asynchronous on `stream`. */
#define MPI_FFL_NOALLOC_MAX_PARTIALS 65536
#define MPI_FFL_NOALLOC_MAX_N ((int64_t)MPI_FFL_NOALLOC_MAX_PARTIALS * 1024)
int mpi_ffl_dot_f64_noalloc(const float *d_a, const float *d_b, int64_t n, double *d_out, void *stream);

/* ---- Failure-detection test hooks (not part of the method) ----------------------
 * These let a test drive the library's error paths without faulting or hanging the
 * GPU: the failures are made on the host (an allocation reported as failed) or by a
 * bounded wait on a barrier that nothing arrives at. The paper has no counterpart.
 *
 * Every device allocation of the library goes through one wrapper. With nth > 0 the
 * nth allocation from now (counted across the process and all handles) fails as
 * cudaMalloc fails on a full device, without allocating; the caller sees
 * MPI_FFL_ERR_OOM and must have freed everything it allocated before. 0 disables the
 * countdown (its state after it fired). Negative nth: MPI_FFL_ERR_INVALID_ARG. */
int mpi_ffl_test_fail_alloc(int32_t nth);
/* Device allocations of the library currently live in this process, and their bytes
 * (count and/or bytes may be NULL): a leak check for the tests. */
int mpi_ffl_test_live_allocs(int64_t *count, int64_t *bytes);
/* With polls > 0, the handle's next interleaved-projector (P) and full/line-GEMM
 * launches do no work: before issuing any copy or MMA, every thread of every block
 * waits at most `polls` polls on a barrier that nothing arrives at, then the block
 * records a timeout (freeing its TMEM where it holds some) and returns, exactly as a
 * block whose pipeline stalled past the kernels' own limit of 2^24 polls does. The
 * results of those calls are undefined; mpi_ffl_sync_check then returns
 * MPI_FFL_ERR_TIMEOUT, clears the flag and disarms the hook, and the handle is usable
 * again. polls = 0 disarms it; polls > 2^24 is MPI_FFL_ERR_INVALID_ARG. Launches of
 * other paths and kernels are unaffected. */
int mpi_ffl_test_inject_timeout(mpi_ffl_handle *h, uint32_t polls);

/* ---- Measurement hooks (not part of the method) ----------------------------------
 * Measured shared-memory read bandwidth of the current device in GB/s: several waves
 * of blocks on every SM read 16-byte words from shared memory in a conflict-free
 * pattern; the best of five timed launches (CUDA events on `stream`, after a warm-up
 * launch). It allocates and frees a small output buffer and synchronises the stream.
 * The projector pair's on-chip roofline is held against this number. */
int mpi_ffl_probe_smem_bandwidth(double *gbs, void *stream);

/* Kernel kinds for the per-kernel timers below. */
#define MPI_FFL_K_TRANSPOSE 0     /* volume x/y transpose for column-marched angles */
#define MPI_FFL_K_PROJECT 1       /* P                                              */
#define MPI_FFL_K_BACKPROJECT 2   /* P^T                                            */
#define MPI_FFL_K_PSF_FWD 3       /* H                                              */
#define MPI_FFL_K_PSF_ADJ 4       /* H^T                                            */
#define MPI_FFL_K_RESAMPLE_FWD 5  /* E V B (staged)                                 */
#define MPI_FFL_K_RESAMPLE_ADJ 6  /* (E V B)^T (staged)                             */
#define MPI_FFL_K_DFT_FWD 7       /* S D_Gamma F (staged, FP32)                     */
#define MPI_FFL_K_DFT_ADJ 8       /* its transpose (staged, FP32)                   */
#define MPI_FFL_K_TC_FWD 9        /* E V B fused with S D_Gamma F (tensor cores)    */
#define MPI_FFL_K_TC_ADJ 10       /* its transpose (tensor cores)                   */
#define MPI_FFL_K_SOLVER 11       /* momentum, residual, update and reductions      */
#define MPI_FFL_K_GEMM_FWD 12     /* collapsed line operator, forward GEMM          */
#define MPI_FFL_K_GEMM_ADJ 13     /* collapsed line operator, adjoint GEMM          */
#define MPI_FFL_K_ZDRIVE 14       /* z-drive scan: column transposes, E_z V_z B with S D F and their transposes */
#define MPI_FFL_K_TENSOR 15       /* tensor-PSF line stages: coil weighting, padding, per-line GEMMs */
#define MPI_FFL_K_COIL 16         /* coil weighting of the collinear model */
#define MPI_FFL_N_KERNEL_KINDS 17

/* enable != 0: record a CUDA event pair around every kernel the handle launches (on
 * the launching stream) until disabled; enable == 0 stops recording. */
int mpi_ffl_profile_enable(mpi_ffl_handle *h, int32_t enable);

/* Waits for the recorded events, then writes per kind (MPI_FFL_N_KERNEL_KINDS entries
 * each) the summed kernel time in ms and the number of timed launches, and clears the
 * record. */
int mpi_ffl_profile_read(mpi_ffl_handle *h, double *ms, int64_t *launches);

/* Total kernel launches issued by the handle since create (always counted). */
int64_t mpi_ffl_launch_count(const mpi_ffl_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* MPI_FFL_H */
