// Internal declarations shared by the library's translation units: the handle,
// table layouts and the kernel launchers of each stage.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mpi_ffl.h"

namespace mpiffl {

// Per-angle ray-march parameters of the projector (Sec. 2.2, Eqs. (16)-(19)).
// Along march step s (a row when row_major, else a column) ray i samples the
// voxel line at position f = inv_c * (i - c) + slope * (s - c) + c, c = (N-1)/2,
// and the sum is multiplied by scale. The kernels take f in Q32.32 fixed point,
// f * 2^32 = fx_a + i fx_d + s fx_b with each constant rounded once on the host, so
// every position is exact to a few 1e-10 voxel at any grid size (an FP32 position
// near 200 voxels is only good to 1.5e-5, which on rough data shows as 1e-5
// relative error); its high word is the cell and its low word the fraction. The
// float fields serve the backprojector's nearest-ray estimate only.
// The slice-interleaved volume volI[z block][y][x][kZc] as the projector's TMA source:
// `row` copies one row (fixed y) of box positions, `col` one column (fixed x); both
// land in shared memory with the 32-byte swizzle (the two 16-byte halves of a
// position swapped when bit 2 of its staged index is set). A line of N positions
// takes nbox boxes of `box` positions (box <= 256, a multiple of 4).
struct IlMaps {
    CUtensorMap row, col;
    int nbox = 0, box = 0;
};

struct AngleParam {
    float inv_c;   // 1/cos (rows) or -1/sin (columns)
    float slope;   // tan (rows) or cot (columns)
    float scale;   // 1/|cos| or 1/|sin|
    int row_major; // 1: march rows of x[z][y][:], 0: columns
    float inv_c_rcp;  // 1 / inv_c (cos, or -sin)
    int pad_;
    long long fx_a, fx_d, fx_b;  // Q32.32: f_0(0), per ray, per march step
};

// One time sample of a raster line: fine-grid cell n and the velocity-weighted
// interpolation weights w0 = (1-f) v, w1 = f v (Sec. 1.2, Eq. (7)).
struct TrajEntry {
    int n;
    float w0;
    float w1;
};

// One entry of the transposed resampling (fine cell <- sample j with weight w).
struct CsrEntry {
    int j;
    float w;
};

// Tables of the z-drive scan (k_zdrive.cu).
struct ZTables {
    const float2 *ua;         // [parity][j]: detector column u0 of the slow position c_j (int
                              // bits) and its fraction c_j - u0
    const int *n0;            // [r]: fine z cell offset floor(Q A sin(2 pi r / S + phi0) + D)
    const float *f0;          // [r]: its fraction
    const float *v;           // [r]: drive velocity along z, A (2 pi / S) cos(2 pi r / S + phi0)
    const int *plo, *phi;     // [parity][r][u]: periods p whose sample pS + r reads column u
    const int *tap_ptr;       // [Q + 1]: taps of each residue of e mod Q
    const int4 *taps;         // (r, e_off, weight bits, 0)
    const int *optr;          // [no + 1]: taps of each offset o = e - Q l of a line's cells
    const int2 *otap;         // 2 S taps: (r, weight bits), n0_r with 1 - f0_r, n0_r + 1 with f0_r
    int no;                   // offsets: max n0_r + 2
};

// A group of raster lines of one angle that share a trajectory (same parity).
struct SegGroup {
    int m;       // angle
    int parity;  // trajectory index (line parity when zig-zag, else 0)
    int z0;      // first line
    int zstride; // 2 with zig-zag, else 1
    int count;   // lines in the group
};

struct Dims {
    int N, Nz, M, S, P, L, Q, D, Ne, K, W, nb, kmin, hw;
    int Nez;                       // fine z grid of the z-drive scan: (N_z - 1) Q + 2 D + 1
    int nseg;                      // M * Nz
    int64_t nvox, nproj, nfine, nsig, ndata;
    int htab_off, htab_len;        // htab[d + htab_off] = h(d / Q), |d| <= htab_off + pad
    int n_par;                     // trajectories: 2 with zig-zag, else 1
};

constexpr int kGroup = 8;          // lines per SegGroup in the staged kernels
constexpr int kRaMaxEntries = 80;  // CSR entries per fine cell the tiled E V B transpose holds
constexpr int kRaTileCells = 256;  // fine cells per tile of the tiled E V B transpose
constexpr int kRaMaxWindow = 24576;  // samples of a tile's window it stages (96 KB)
constexpr int kPsfT = 16;          // tap-table padding, in outputs per phase, of the PSF kernels' windows
constexpr int kMaxHw = 8;          // largest supported half-width

}  // namespace mpiffl

struct mpi_ffl_handle {
    mpiffl::Dims d{};
    int device = 0;
    int precision = MPI_FFL_PREC_FP32;
    std::string err;

    // host copies of the description
    std::vector<double> angles;
    std::vector<float> gains;
    double fwhm = 0, amp = 0, phase = 0;
    int zigzag = 1;
    std::vector<float> dgamma;  // nb complex

    // device tables
    mpiffl::AngleParam *t_ang = nullptr;
    float *t_gain = nullptr;       // M
    float *t_unit_gain = nullptr;  // M ones
    float *t_htab = nullptr;       // PSF taps
    float *t_dhtab = nullptr;      // d h / d fwhm taps
    mpiffl::TrajEntry *t_traj = nullptr;  // n_par * L
    int2 *t_tnf = nullptr;                // n_par * L: (cell n, fraction f as float bits)
    std::vector<int> traj_n;              // host copy of the cells n, n_par * L
    float *t_vr = nullptr;                // n_par * S: velocity v_j, which depends on j mod S only
    // tiled E V B transpose (k_resample_adj_tiled): per (parity, tile of kRaTileCells cells)
    // the sample window (j_lo, len, first cell, cells), and the CSR entries [k][cell] with j
    // relative to the window (ra_cap = the zero word for padding); ra_ntile = 0 when the
    // trajectory does not fit, and the plain CSR gather serves instead
    int4 *t_ra_tile = nullptr;
    uint16_t *t_ra_j = nullptr;
    float *t_ra_w = nullptr;
    int ra_ntile = 0, ra_cap = 0;
    bool ra_built = false;                // the tiles are built on the transpose's first use
    std::vector<int> csr_ptr_host;        // host copies of the CSR, n_par * (Ne + 1) and n_par * 2L
    std::vector<mpiffl::CsrEntry> csr_host;
    float2 *t_twp = nullptr;              // [P] e^{2 pi i q / P}: the period twiddles of the band DFT
    double *w_bins = nullptr;             // n_bins + 1: kept-bin energies and the total (information retained)
    int *t_csr_ptr = nullptr;             // n_par * (Ne + 1)
    mpiffl::CsrEntry *t_csr = nullptr;    // n_par * 2L
    float *t_tw1 = nullptr;               // P * W: cos(2 pi d p / P) d=0..hw, sin d=1..hw
    float2 *t_tw2_ro = nullptr;           // [r][q]: exp(+2 pi i w_q r / L)
    float2 *t_tw2_qr = nullptr;           // [q][r]
    float2 *t_dgam = nullptr;             // nb
    float2 *t_dgam_unit = nullptr;        // nb ones (the bare DFT, for the compression analysis)
    mpiffl::SegGroup *t_groups = nullptr;
    int n_groups = 0;
    int *t_agroups = nullptr;  // projector angle groups: kProjAnglesPerBlock indices, -1 = empty
    float *w_volI = nullptr;  // slice-interleaved volume (il_len floats)
    mpiffl::IlMaps il_maps;   // its tensor maps
    int n_agroups = 0;

    // workspace
    float *w_volT = nullptr;   // nvox
    float *w_proj = nullptr;   // nproj
    float *w_fine = nullptr;   // nfine
    float *w_sig = nullptr;    // nsig
    float *w_data = nullptr;   // ndata
    float *w_vol2 = nullptr;   // nvox
    double *w_red = nullptr;   // reduction partials
    double *w_scal = nullptr;  // device scalars
    int w_red_len = 0;
    // solver state
    float *s_xp = nullptr, *s_y = nullptr, *s_g = nullptr, *s_r = nullptr;
    double *s_hist = nullptr;
    int s_hist_len = 0;
    int *s_flags = nullptr;
    int *w_err = nullptr;      // set by kernels that gave up on a bounded wait
    // failure-detection test hook (mpi_ffl_test_inject_timeout): > 0 makes the next
    // interleaved-projector and line-GEMM launches give up after this many polls of a
    // barrier that nothing arrives at; cleared by mpi_ffl_sync_check
    uint32_t inject_polls = 0;
    // measurement hooks
    int prof_on = 0;
    int64_t launches = 0;
    struct ProfRec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof_rec;
    std::vector<cudaEvent_t> ev_pool;
    // tensor-core path state (tc.cu)
    void *tc_twb = nullptr;
    void *tc_state = nullptr;
    void *col_state = nullptr;  // collapsed line operator (collapsed.cu)
    int path = 0;               // MPI_FFL_PATH_*
    int64_t bytes = 0;
    // host buffers given to forward/adjoint: device staging, allocated on first use
    float *hs_in[2] = {nullptr, nullptr};  // copies of host inputs, alternating
    float *hs_out = nullptr;                // result before its copy to a host output
    cudaStream_t hs_copy = nullptr;         // input copies when host_overlap is on
    cudaEvent_t hs_ready[2] = {}, hs_free[2] = {};
    int hs_slot = 0;
    int host_overlap = 0;                   // mpi_ffl_set_host_overlap
    // scans of the solve and power iteration (MPI_FFL_SCAN_* bits): [A; A_z] when both
    int scans = 1;
    float *w_scanvol = nullptr;  // 2 n_vox: A^T r and A_z^T r_z before their sum
    // PSF model (MPI_FFL_PSF_*) and receive-coil map b[z][u] (NULL: uniform coil)
    int psf_model = 0;
    float *t_coil = nullptr;    // N_z N
    float *w_projc = nullptr;   // M N_z N: coil-weighted projections (collinear model)
    // z-drive scan (k_zdrive.cu): tables and workspace, built on first use
    int z_ready = 0;
    int *tz_n0 = nullptr, *tz_plo = nullptr, *tz_phi = nullptr, *tz_tap_ptr = nullptr;
    float *tz_f0 = nullptr, *tz_v = nullptr;
    float2 *tz_ua = nullptr;
    int4 *tz_taps = nullptr;
    int *tz_optr = nullptr;
    int2 *tz_otap = nullptr;
    int tz_no = 0;
    float *w_fine_z = nullptr;  // M N N_ez
    float *w_zcoef = nullptr;   // M N_z W S (synthesis coefficients of the z adjoint)
    float *w_projT = nullptr;   // M N N_z (projections by column)
    float *w_tz = nullptr;      // M N_z N S (per-phase partials of the staged transpose)
};

namespace mpiffl {

// ---------------------------------------------------------------- batched launches
// One problem of a batched launch (continuous batching, batch.cu). `done` (device
// int, may be NULL) turns the problem's blocks into no-ops once it is nonzero.
struct TransposeJob {
    const float *vol;
    float *volT;
    int N, Nz;
    const int *done;
};
struct ProjectJob {
    const float *vol, *volT;
    const AngleParam *ang;
    const int *agroups;
    float *proj;
    int N, Nz, n_agroups;
    const int *done;
};
struct BackprojectJob {
    const float *proj;
    const AngleParam *ang;
    float *vol;
    int N, Nz, M;
    const int *done;
};
struct MomentumJob {   // y = x + beta (x - xp)
    const float *x, *xp;
    float *y;
    float beta;
    int64_t n;
    const int *done;
};
struct ResidualJob {   // r <- r - b; partial sums of r^2 into partials[0..nblk)
    float *r;
    const float *b;
    int64_t n;
    double *partials;
    int nblk;
    const int *done;
};
struct StopJob {       // hist[k] = sqrt(sum partials); stop test; status out
    const double *partials;
    int nblk;
    double *hist;
    int k;
    double stop_rel;
    int *flags;        // [0] stop (1 converged, 2 non-finite), [1] iterations done
    int *done;         // set when the job must not run further
};
struct UpdateJob {     // x_out = P(y - tau (g + lam T^T T y)); a frozen job copies x_cur
    const float *y, *g;
    float *xo;
    const float *xcur;
    float tau, lam;
    int nonneg, N, Nz;
    const int *done;
};

int transpose_blocks(int N, int Nz);
int project_blocks(int n_agroups, int Nz);
bool project_batch_ok(int N);  // problem size the batched projector takes
int backproject_blocks(int N, int Nz);
int update_blocks(int N, int Nz);
void launch_transpose_batch(const TransposeJob *jobs, const int *offs, int n, int total, cudaStream_t st);
void launch_project_batch(const ProjectJob *jobs, const int *offs, int n, int total, int maxN, int *err,
                          cudaStream_t st);
void launch_backproject_batch(const BackprojectJob *jobs, const int *offs, int n, int total, cudaStream_t st);
void launch_momentum_batch(const MomentumJob *jobs, const int *offs, int n, int total, cudaStream_t st);
void launch_residual_batch(const ResidualJob *jobs, const int *offs, int n, int total, cudaStream_t st);
void launch_stop_batch(const StopJob *jobs, int n, cudaStream_t st);
void launch_update_batch(const UpdateJob *jobs, const int *offs, int n, int total, cudaStream_t st);
void launch_freeze_batch(const StopJob *jobs, int n, cudaStream_t st);  // done = stop verdict

// Launch with programmatic stream serialization: the kernel may be scheduled while the
// previous kernel of the stream finishes (its blocks run their prologue, then wait in
// ptx::grid_dep_wait before touching memory that earlier kernels write or read).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                    Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Message returned by mpi_ffl_last_error(NULL) on this thread.
void set_thread_error(const std::string &msg);

// Every device allocation and release of the library (alloc.cu): cudaMalloc and
// cudaFree plus a registry of live allocations, and the failure-injection countdown
// of mpi_ffl_test_fail_alloc.
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t dev_free(void *p);

// ---------------------------------------------------------------- launchers
// Projector (k_projector.cu)
void launch_transpose_xy(const float *vol, float *volT, int N, int Nz, cudaStream_t st);
// slice-interleaved volume copies and the projector that reads them (k_projector.cu)
bool project_il_ok(int N);
double project_il_cost(const AngleParam &a, int N);
size_t il_len(int N, int Nz);
void launch_interleave(const float *vol, float *volI, int N, int Nz, cudaStream_t st);
// encodes the tensor maps of volI (false if the driver refuses them)
bool make_il_maps(const float *volI, int N, int Nz, IlMaps *maps);
// The forward line-GEMM's A operand written by the projector itself (bf16 or tf32 hi + lo, the
// canonical 1 KB blocks [K chunk][hi, lo][group of 8 rows] per trajectory parity), when
// out[0] is not NULL: rows of parity p are the lines (m, z) with z = p mod n_par, in
// angle-major order, G[p] groups of 8 rows each, nrow[p] rows per angle. proj may then
// be NULL (the projections are not stored).
struct ProjPack {
    uint8_t *out[2];
    int G[2];
    int nrow[2];
    int n_par;
    int tf32;  // 1: tf32 hi + lo (4 K values per 16-byte unit), 0: bf16 (8)
};

void launch_project_il(const IlMaps &maps, const AngleParam *ang, const int *agroups,
                       int n_agroups, float *proj, int N, int Nz, cudaStream_t st, int *err, uint32_t inject = 0, ProjPack pack = ProjPack{});
void launch_project(const float *vol, const float *volT, const AngleParam *ang, const int *agroups,
                    int n_agroups, float *proj, int N, int Nz, cudaStream_t st, int *err);
constexpr int kProjAnglesPerBlock = 2;  // angle slots per projector block (k_projector.cu)
void launch_backproject(const float *proj, const AngleParam *ang, float *vol, int N, int Nz,
                        int M, cudaStream_t st);

// Staged line kernels (k_line.cu)
void launch_psf_fwd(const float *proj, const float *htab, float *fine, const Dims &d, cudaStream_t st);
void launch_psf_adj(const float *fine, const float *htab, float *proj, const Dims &d, cudaStream_t st);
void launch_resample_fwd(const float *fine, const TrajEntry *traj, const float *gain,
                         const SegGroup *groups, int n_groups, float *sig, const Dims &d,
                         cudaStream_t st);
void launch_resample_adj_tiled(const float *sig, const int4 *tiles, const uint16_t *tj, const float *tw,
                               const float *gain, float *fine, const Dims &d, int ntile, int cap, int *err,
                               cudaStream_t st);
void launch_resample_adj(const float *sig, const int *csr_ptr, const CsrEntry *csr,
                         const float *gain, const SegGroup *groups, int n_groups, float *fine,
                         const Dims &d, cudaStream_t st);
void launch_dft_fwd(const float *sig, const float *tw1, const float2 *twp, const float2 *tw2_ro, const float2 *dgam,
                    float *data, const Dims &d, int *err, cudaStream_t st);
void launch_dft_adj(const float *data, const float *tw1, const float2 *twp, const float2 *tw2_qr, const float2 *dgam,
                    float *sig, const Dims &d, cudaStream_t st);

// Solver and reductions (k_solver.cu)
int reduce_blocks(int64_t n);
void launch_momentum(const float *x, const float *xp, float *y, double beta_num, int k,
                     int64_t n, const int *done, cudaStream_t st);
void launch_sub_norm(float *r, const float *b, int64_t n, double *partials, int nblk,
                     const int *done, cudaStream_t st);
void launch_dot(const float *a, const float *b, int64_t n, double *partials, int nblk, cudaStream_t st);
void launch_finalize(const double *partials, int nblk, double *out, cudaStream_t st);
void launch_update(const float *y, const float *g, float *xout, float tau, float lam, int nonneg,
                   int N, int Nz, const int *done, cudaStream_t st, const float *xcur = nullptr);
void launch_freeze(const int *stop, int *frozen, cudaStream_t st);
void launch_bin_energy(const float *data, int nseg, int nb, double *out, cudaStream_t st);
void launch_info_retained(const double *bin_energy, const double *total, int kmin, int w_all, int n_k,
                          const int *hk, int n_w, const int *hw, double *out, cudaStream_t st);
void launch_transpose_2d(const float *in, float *out, int batch, int rows, int cols, cudaStream_t st);
void launch_resample_z_fwd(const float *cz, const ZTables &T, const float *gain, float *sig, const Dims &d,
                           int zigzag, cudaStream_t st);
void launch_resample_z_adj(const float *sig, const ZTables &T, const float *gain, float *tz, float *cz,
                           const Dims &d, int zigzag, cudaStream_t st);
void launch_zdft_fwd(const float *cz, const ZTables &T, const float *gain, const float *tw1, const float2 *tw2_ro,
                     const float2 *dgam, float *data, const Dims &d, int zigzag, cudaStream_t st);
void launch_zdft_adj(const float *data, const float *tw1, const float2 *tw2_qr, const float2 *dgam,
                     const ZTables &T, const float *gain, float *coef, float *cz, const Dims &d, int zigzag,
                     cudaStream_t st);
// coil weighting and row padding (k_coil.cu): out[r'][c] = b[r mod Nz][c] sum_p in[p][r][c],
// c < ncols (nparts partial sums part_stride floats apart); zero up to stride. Output row
// r' = (r / Nz) zp + p0 + r mod Nz (zp 0: Nz)
void launch_coil_pad(const float *in, const float *coil, float *out, long long rows, int Nz, int ncols, int stride,
                     cudaStream_t st, int nparts = 1, long long part_stride = 0, int zp = 0, int p0 = 0);
size_t zdft_fwd_smem(const Dims &d);     // shared memory of the fused z forward
int zsyn_ring(const Dims &d, int no);
size_t zsyn_smem(const Dims &d, int no);
void launch_ttt(const float *x, float *out, int N, int Nz, cudaStream_t st);
void launch_splitmix_fill(float *v, int64_t n, uint64_t seed, cudaStream_t st);
void launch_scale_by_rsqrt(const float *in, float *out, int64_t n, const double *n2, cudaStream_t st);
void launch_stop_check(double *hist, int k, double stop_rel, int *done, int *iters_done,
                       cudaStream_t st);
void launch_angle_dots(const float *a, const float *b, int M, int64_t per_angle, double *partials,
                       int nblk_per_angle, cudaStream_t st);
void launch_angle_finalize(const double *partials, int M, int nblk_per_angle, float *out,
                           cudaStream_t st);
void launch_finalize_to_float(const double *partials, int nblk, float *out, cudaStream_t st);

}  // namespace mpiffl
