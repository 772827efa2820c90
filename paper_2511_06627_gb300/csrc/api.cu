// C ABI of the library (include/mpi_ffl.h): handle life cycle, the host-side
// tables (computed in double precision from the paper's formulas), and the
// orchestration of the stage kernels into A, A^T and the solve of Eq. (26).
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"
#include "collapsed.h"
#include "tc.h"

using namespace mpiffl;

// the z-drive scan (defined with its entry points below)
void z_init(mpi_ffl_handle *h);
void forward_z_impl(mpi_ffl_handle *h, const float *x, float *b, cudaStream_t st);
void adjoint_z_impl(mpi_ffl_handle *h, const float *b, float *x, cudaStream_t st);

namespace {

thread_local std::string g_create_error;

constexpr double kPi = 3.14159265358979323846;

struct Fail {
    int code;
};

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            set_err(h, std::string(#call) + ": " + cudaGetErrorString(e_));                 \
            throw Fail{e_ == cudaErrorMemoryAllocation ? MPI_FFL_ERR_OOM : MPI_FFL_ERR_CUDA}; \
        }                                                                                   \
    } while (0)

void set_err(mpi_ffl_handle *h, const std::string &m) {
    if (h) h->err = m;
    else g_create_error = m;
}

void check_launch(mpi_ffl_handle *h, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_err(h, std::string(what) + ": " + cudaGetErrorString(e));
        throw Fail{MPI_FFL_ERR_CUDA};
    }
}

cudaEvent_t pool_event(mpi_ffl_handle *h) {
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// Counts one kernel launch and, when profiling is on, brackets it with events.
struct KTimer {
    mpi_ffl_handle *h;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    KTimer(mpi_ffl_handle *h_, int kind_, cudaStream_t st_) : h(h_), kind(kind_), st(st_) {
        h->launches++;
        if (h->prof_on) {
            a = pool_event(h);
            cudaEventRecord(a, st);
        }
    }
    ~KTimer() {
        if (a) {
            cudaEvent_t b = pool_event(h);
            cudaEventRecord(b, st);
            h->prof_rec.push_back(mpi_ffl_handle::ProfRec{kind, a, b});
        }
    }
};

#define TIMED(kind, call)                        \
    do {                                         \
        KTimer kt_(h, kind, st);                 \
        call;                                    \
    } while (0)

template <class T>
void dev_alloc(mpi_ffl_handle *h, T **p, size_t n) {
    if (n == 0) n = 1;
    cudaError_t e = dev_malloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_err(h, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed: " + cudaGetErrorString(e));
        throw Fail{e == cudaErrorMemoryAllocation ? MPI_FFL_ERR_OOM : MPI_FFL_ERR_CUDA};
    }
    h->bytes += (int64_t)(n * sizeof(T));
}

template <class T>
void upload(mpi_ffl_handle *h, T **p, const std::vector<T> &v) {
    dev_alloc(h, p, v.size());
    CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
}

// ------------------------------------------------------------ Langevin PSF
// L'(x) = 1/x^2 - 1/sinh(x)^2 (Appendix B, Eq. (31) collinear term), with the
// Taylor series 1/3 - x^2/15 + 2x^4/189 - x^6/675 for |x| < 0.05.
double langevin_d1(double x) {
    const double ax = std::fabs(x);
    if (ax < 0.05) {
        const double x2 = x * x;
        return 1.0 / 3.0 - x2 / 15.0 + 2.0 * x2 * x2 / 189.0 - x2 * x2 * x2 / 675.0;
    }
    if (ax > 350.0) return 1.0 / (x * x);
    const double sh = std::sinh(ax);
    return 1.0 / (ax * ax) - 1.0 / (sh * sh);
}

// L''(x) = -2/x^3 + 2 cosh(x)/sinh(x)^3, series -2x/15 + 8x^3/189 - 6x^5/675.
double langevin_d2(double x) {
    const double ax = std::fabs(x);
    if (ax < 0.05) return -2.0 * x / 15.0 + 8.0 * x * x * x / 189.0 - 6.0 * std::pow(x, 5) / 675.0;
    if (ax > 350.0) return -2.0 / (x * x * x);
    const double sh = std::sinh(x);
    return -2.0 / (x * x * x) + 2.0 * std::cosh(x) / (sh * sh * sh);
}

// x_h with L'(x_h) = L'(0)/2 = 1/6, by bisection (L' decreases on x > 0).
double langevin_half_point() {
    double lo = 0.5, hi = 5.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (langevin_d1(mid) > 1.0 / 6.0) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

namespace mpiffl {
double langevin_d1_host(double x) { return langevin_d1(x); }
double langevin_half_point_host() { return langevin_half_point(); }
// FFL sample j of a line with the given trajectory (parity): fine cell n, fraction f, velocity v
void traj_point_host(const mpi_ffl_handle *h, int par, int j, int &n, double &f, double &v) {
    const Dims &d = h->d;
    const double kPi = 3.14159265358979323846;
    const double slope = (double)(d.N - 1) / (double)(d.L - 1);
    const double slow = par ? (d.N - 1) - slope * j : slope * j;
    const double dslow = par ? -slope : slope;
    const double ph = 2.0 * kPi * (double)(j % d.S) / d.S + h->phase;
    const double xi = slow + h->amp * std::sin(ph);
    v = dslow + h->amp * (2.0 * kPi / d.S) * std::cos(ph);
    const double tt = d.Q * xi + d.D;
    n = (int)std::floor(tt);
    if (n > d.Ne - 2) n = d.Ne - 2;
    f = tt - n;
}
}  // namespace mpiffl

namespace {

void psf_tables(const Dims &d, double fwhm, std::vector<float> &h, std::vector<float> &dh) {
    const double a = fwhm / (2.0 * langevin_half_point());
    h.resize(d.htab_len);
    dh.resize(d.htab_len);
    for (int k = 0; k < d.htab_len; ++k) {
        const double u = (double)(k - d.htab_off) / d.Q;
        const double x = u / a;
        h[k] = (float)(3.0 * langevin_d1(x));
        // d/dfwhm of 3 L'(u/a), a = fwhm / (2 x_h): -3 L''(x) x / fwhm
        dh[k] = (float)(-3.0 * langevin_d2(x) * x / fwhm);
    }
}

// ------------------------------------------------------------ validation
int compute_dims(const mpi_ffl_geometry *g, const mpi_ffl_trajectory *t, const mpi_ffl_harmonics *hm,
                 Dims &d, std::string &why) {
    if (!g || !t || !hm) { why = "NULL description"; return MPI_FFL_ERR_INVALID_ARG; }
    if (g->nx != g->ny) { why = "nx must equal ny"; return MPI_FFL_ERR_INVALID_ARG; }
    if (g->nx < 2 || g->nz < 1 || g->n_angles < 1) { why = "bad volume or angle count"; return MPI_FFL_ERR_INVALID_ARG; }
    if (g->nx > 512) { why = "nx > 512 is not supported by the projector kernels"; return MPI_FFL_ERR_UNSUPPORTED; }
    if (t->samples_per_period < 2 || t->periods_per_line < 1 || t->upsample_q < 1 || t->upsample_q > 32 ||
        (t->upsample_q & (t->upsample_q - 1)) != 0 || !(t->drive_amp_vox >= 0.0)) {
        why = "bad trajectory (S >= 2, P >= 1, A >= 0, Q a power of two <= 32)";
        return MPI_FFL_ERR_INVALID_ARG;
    }
    if (hm->half_width < 0 || hm->half_width > kMaxHw || hm->k_min < 0 || hm->k_max < hm->k_min) {
        why = "bad harmonic band (half_width must be 0..8)";
        return MPI_FFL_ERR_INVALID_ARG;
    }
    d.N = g->nx;
    d.Nz = g->nz;
    d.M = g->n_angles;
    d.S = t->samples_per_period;
    d.P = t->periods_per_line;
    const int64_t L = (int64_t)d.S * d.P;
    if (L < 2 || L > (1 << 28)) { why = "line length out of range"; return MPI_FFL_ERR_INVALID_ARG; }
    d.L = (int)L;
    d.Q = t->upsample_q;
    d.D = (int)std::ceil(t->drive_amp_vox * d.Q - 1e-9);
    d.Ne = (d.N - 1) * d.Q + 2 * d.D + 1;
    d.Nez = (d.Nz - 1) * d.Q + 2 * d.D + 1;
    d.K = hm->k_max - hm->k_min + 1;
    d.hw = hm->half_width;
    d.W = 2 * d.hw + 1;
    d.nb = d.K * d.W;
    d.kmin = hm->k_min;
    if ((int64_t)hm->k_min * d.P - d.hw < 1 || (int64_t)hm->k_max * d.P + d.hw >= L / 2) {
        why = "harmonic band must satisfy 1 <= k*P + delta < L/2";
        return MPI_FFL_ERR_INVALID_ARG;
    }
    if (d.S > 1024 * 8) { why = "samples_per_period too large"; return MPI_FFL_ERR_INVALID_ARG; }
    d.nseg = d.M * d.Nz;
    d.nvox = (int64_t)d.Nz * d.N * d.N;
    d.nproj = (int64_t)d.nseg * d.N;
    d.nfine = (int64_t)d.nseg * d.Ne;
    d.nsig = (int64_t)d.nseg * d.L;
    d.ndata = (int64_t)2 * d.nseg * d.nb;
    // taps for the x-drive rows (N bins) and the z-drive columns (N_z slices)
    d.htab_off = (std::max(d.N, d.Nz) - 1) * d.Q + d.D + d.Q * kPsfT;
    d.htab_len = 2 * d.htab_off + 1;
    d.n_par = t->zigzag ? 2 : 1;
    // shared memory of the staged kernels
    if ((size_t)(d.htab_len + 4 * (size_t)d.Ne) * 4 > 220 * 1024 || (size_t)d.P * d.W * 4 + (size_t)d.S * d.W * 8 > 220 * 1024) {
        why = "problem too large for the staged kernels' shared memory";
        return MPI_FFL_ERR_UNSUPPORTED;
    }
    return 0;
}

void angle_table(mpi_ffl_handle *h) {
    const Dims &d = h->d;
    std::vector<AngleParam> a(d.M);
    const double ctr = 0.5 * (d.N - 1);
    auto fx = [](double v) { return (long long)std::llround(std::ldexp(v, 32)); };
    for (int m = 0; m < d.M; ++m) {
        const double th = h->angles[m];
        const double c = std::cos(th), s = std::sin(th);
        const bool rows = std::fabs(c) >= std::fabs(s) - 1e-9;
        const double inv_c = rows ? 1.0 / c : -1.0 / s;
        const double slope = rows ? s / c : c / s;
        const double scale = rows ? 1.0 / std::fabs(c) : 1.0 / std::fabs(s);
        // f_i(s) = ctr + inv_c (i - ctr) + slope (s - ctr) = f_0(0) + inv_c i + slope s
        a[m] = AngleParam{(float)inv_c, (float)slope, (float)scale, rows ? 1 : 0, (float)(rows ? c : -s), 0,
                          fx(ctr - inv_c * ctr - slope * ctr), fx(inv_c), fx(slope)};
    }
    upload(h, &h->t_ang, a);
    // Projector blocks hold kProjAnglesPerBlock (two) angles of one orientation. Angles
    // differ in cost (oblique rays meet more shared-memory bank conflicts and fewer of
    // them leave the grid), and the blocks run as one wave, so each block pairs a costly
    // angle with a cheap one: sorted by the modelled cost, the costliest of an odd count
    // goes alone, then the costliest remaining with the cheapest. Which block sums an
    // angle does not change its sums.
    static_assert(kProjAnglesPerBlock == 2, "the pairing below forms blocks of two angles");
    std::vector<double> cost(d.M);
    for (int m = 0; m < d.M; ++m) cost[m] = project_il_cost(a[m], d.N);
    std::vector<int> groups;
    for (int orient = 1; orient >= 0; --orient) {
        std::vector<int> ms;
        for (int m = 0; m < d.M; ++m)
            if (a[m].row_major == orient) ms.push_back(m);
        std::stable_sort(ms.begin(), ms.end(), [&](int x, int y) { return cost[x] < cost[y]; });
        size_t lo = 0, hi = ms.size();
        if (ms.size() % 2) {
            groups.push_back(ms[--hi]);
            groups.push_back(-1);
        }
        while (lo < hi) {
            groups.push_back(ms[--hi]);
            groups.push_back(ms[lo++]);
        }
    }
    h->n_agroups = (int)(groups.size() / kProjAnglesPerBlock);
    upload(h, &h->t_agroups, groups);
}

void trajectory_tables(mpi_ffl_handle *h) {
    const Dims &d = h->d;
    std::vector<TrajEntry> tr((size_t)d.n_par * d.L);
    std::vector<int2> tnf((size_t)d.n_par * d.L);
    h->traj_n.assign((size_t)d.n_par * d.L, 0);
    std::vector<float> vr((size_t)d.n_par * d.S);
    std::vector<int> ptr((size_t)d.n_par * (d.Ne + 1), 0);
    std::vector<CsrEntry> csr((size_t)d.n_par * 2 * d.L);
    const double slope = (double)(d.N - 1) / (double)(d.L - 1);
    for (int par = 0; par < d.n_par; ++par) {
        TrajEntry *T = tr.data() + (size_t)par * d.L;
        for (int j = 0; j < d.L; ++j) {
            int n;
            double f, v;
            traj_point_host(h, par, j, n, f, v);
            if (n < 0 || f > 1.0 + 1e-9) {
                set_err(h, "trajectory leaves the fine grid");
                throw Fail{MPI_FFL_ERR_INVALID_ARG};
            }
            T[j] = TrajEntry{n, (float)((1.0 - f) * v), (float)(f * v)};
            const float ff = (float)f;
            int fb;
            std::memcpy(&fb, &ff, 4);
            tnf[(size_t)par * d.L + j] = make_int2(n, fb);
            h->traj_n[(size_t)par * d.L + j] = n;
            if (j < d.S) vr[(size_t)par * d.S + j] = (float)v;  // v_j = v_{j mod S}
        }
        // CSR of the transpose: cell n_j <- (j, w0), cell n_j + 1 <- (j, w1), j ascending
        int *P = ptr.data() + (size_t)par * (d.Ne + 1);
        for (int j = 0; j < d.L; ++j) {
            P[T[j].n + 1]++;
            P[T[j].n + 2]++;
        }
        for (int e = 0; e < d.Ne; ++e) P[e + 1] += P[e];
        std::vector<int> fill(P, P + d.Ne);
        CsrEntry *C = csr.data() + (size_t)par * 2 * d.L;
        for (int e = 0; e < d.Ne; ++e) fill[e] = P[e];
        // two passes keep entries of a cell in ascending j
        for (int j = 0; j < d.L; ++j) {
            C[fill[T[j].n]++] = CsrEntry{j, T[j].w0};
            C[fill[T[j].n + 1]++] = CsrEntry{j, T[j].w1};
        }
    }
    upload(h, &h->t_traj, tr);
    upload(h, &h->t_tnf, tnf);
    upload(h, &h->t_vr, vr);
    upload(h, &h->t_csr_ptr, ptr);
    upload(h, &h->t_csr, csr);
    // the staged transpose's tiles are built from these on its first use
    h->csr_ptr_host = std::move(ptr);
    h->csr_host = std::move(csr);
}

void dft_tables(mpi_ffl_handle *h) {
    const Dims &d = h->d;
    std::vector<float> tw1((size_t)d.P * d.W);
    for (int p = 0; p < d.P; ++p) {
        for (int k = 0; k <= d.hw; ++k) {
            const double ang = 2.0 * kPi * (double)(((int64_t)k * p) % d.P) / d.P;
            tw1[(size_t)p * d.W + k] = (float)std::cos(ang);
            if (k > 0) tw1[(size_t)p * d.W + d.hw + k] = (float)std::sin(ang);
        }
    }
    std::vector<float2> ro((size_t)d.S * d.nb), qr((size_t)d.nb * d.S);
    for (int o = 0; o < d.nb; ++o) {
        const int64_t w = (int64_t)(d.kmin + o / d.W) * d.P + (o % d.W - d.hw);
        for (int r = 0; r < d.S; ++r) {
            const double ang = 2.0 * kPi * (double)((w * r) % d.L) / d.L;
            const float2 v = make_float2((float)std::cos(ang), (float)std::sin(ang));
            ro[(size_t)r * d.nb + o] = v;
            qr[(size_t)o * d.S + r] = v;
        }
    }
    upload(h, &h->t_tw1, tw1);
    // the same period twiddles as one table, e^{2 pi i q / P} for q = k p mod P
    std::vector<float2> twp(d.P);
    for (int q = 0; q < d.P; ++q) {
        const double ang = 2.0 * kPi * (double)q / d.P;
        twp[q] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    upload(h, &h->t_twp, twp);
    upload(h, &h->t_tw2_ro, ro);
    upload(h, &h->t_tw2_qr, qr);
    std::vector<float2> dg(d.nb);
    for (int o = 0; o < d.nb; ++o) dg[o] = make_float2(h->dgamma[2 * o], h->dgamma[2 * o + 1]);
    upload(h, &h->t_dgam, dg);
}

void group_table(mpi_ffl_handle *h) {
    const Dims &d = h->d;
    std::vector<SegGroup> g;
    for (int m = 0; m < d.M; ++m) {
        for (int par = 0; par < d.n_par; ++par) {
            const int stride = d.n_par;
            for (int z0 = par; z0 < d.Nz; z0 += stride * kGroup) {
                const int cnt = std::min(kGroup, (d.Nz - z0 + stride - 1) / stride);
                g.push_back(SegGroup{m, par, z0, stride, cnt});
            }
        }
    }
    h->n_groups = (int)g.size();
    upload(h, &h->t_groups, g);
}

void release(mpi_ffl_handle *h) {
    void *ptrs[] = {h->t_ang, h->t_gain, h->t_unit_gain, h->t_htab, h->t_dhtab, h->t_traj, h->t_csr_ptr,
                    h->t_csr, h->t_tw1, h->t_tw2_ro, h->t_tw2_qr, h->t_dgam, h->t_dgam_unit, h->t_groups, h->w_volT,
                    h->w_proj, h->w_fine, h->w_sig, h->w_data, h->w_vol2, h->w_red, h->w_scal,
                    h->s_xp, h->s_y, h->s_g, h->s_r, h->s_hist, h->s_flags, h->tc_twb, h->t_agroups,
                    h->t_tnf, h->t_vr, h->w_err, h->t_coil, h->w_projc, h->w_scanvol, h->w_volI,
                    h->t_ra_tile, h->t_ra_j, h->t_ra_w, h->t_twp, h->w_bins};
    for (void *p : ptrs)
        if (p) dev_free(p);
    for (auto &r : h->prof_rec) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    for (float *p : {h->hs_in[0], h->hs_in[1], h->hs_out})
        if (p) dev_free(p);
    for (void *p : {(void *)h->tz_ua, (void *)h->tz_n0, (void *)h->tz_plo, (void *)h->tz_phi, (void *)h->tz_tap_ptr,
                    (void *)h->tz_f0, (void *)h->tz_v, (void *)h->tz_taps, (void *)h->tz_optr, (void *)h->tz_otap,
                    (void *)h->w_zcoef, (void *)h->w_fine_z,
                    (void *)h->w_projT, (void *)h->w_tz})
        if (p) dev_free(p);
    for (int k = 0; k < 2; ++k) {
        if (h->hs_ready[k]) cudaEventDestroy(h->hs_ready[k]);
        if (h->hs_free[k]) cudaEventDestroy(h->hs_free[k]);
    }
    if (h->hs_copy) cudaStreamDestroy(h->hs_copy);
    tc_release(h);
    col_release(h);
}

// ------------------------------------------------------------ host buffers
// A pointer CUDA does not know as device or managed memory is a host buffer.
bool is_host_ptr(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

void ensure_host_staging(mpi_ffl_handle *h) {
    const int64_t n = std::max(h->d.nvox, h->d.ndata);
    for (float **p : {&h->hs_in[0], &h->hs_in[1], &h->hs_out})
        if (!*p) dev_alloc(h, p, n);
    if (!h->hs_copy) CK(cudaStreamCreateWithFlags(&h->hs_copy, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        if (!h->hs_ready[k]) CK(cudaEventCreateWithFlags(&h->hs_ready[k], cudaEventDisableTiming));
        if (!h->hs_free[k]) CK(cudaEventCreateWithFlags(&h->hs_free[k], cudaEventDisableTiming));
    }
}

// Device copy of a host input of n floats. With host_overlap the copy runs on the
// handle's copy stream (it waits only for the previous use of its staging slot, so it
// overlaps earlier work on `st`); otherwise on `st`. `slot` is released by host_done.
const float *host_in(mpi_ffl_handle *h, const float *src, int64_t n, cudaStream_t st, int &slot) {
    ensure_host_staging(h);
    slot = h->hs_slot;
    h->hs_slot ^= 1;
    float *dst = h->hs_in[slot];
    if (h->host_overlap) {
        CK(cudaStreamWaitEvent(h->hs_copy, h->hs_free[slot], 0));
        CK(cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyHostToDevice, h->hs_copy));
        CK(cudaEventRecord(h->hs_ready[slot], h->hs_copy));
        CK(cudaStreamWaitEvent(st, h->hs_ready[slot], 0));
    } else {
        CK(cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyHostToDevice, st));
    }
    return dst;
}

void host_done(mpi_ffl_handle *h, int slot, cudaStream_t st) {
    if (slot >= 0) CK(cudaEventRecord(h->hs_free[slot], st));
}

// Runs op(in_dev, out_dev) with host inputs and outputs staged through the handle's
// device buffers; a host output is copied back on `st`.
template <class F>
void with_host_buffers(mpi_ffl_handle *h, const float *in, int64_t n_in, float *out, int64_t n_out,
                       cudaStream_t st, F op) {
    int slot = -1;
    const float *din = in;
    float *dout = out;
    if (is_host_ptr(in)) din = host_in(h, in, n_in, st, slot);
    const bool out_host = is_host_ptr(out);
    if (out_host) {
        ensure_host_staging(h);
        dout = h->hs_out;
    }
    op(din, dout);
    host_done(h, slot, st);
    if (out_host) CK(cudaMemcpyAsync(out, dout, sizeof(float) * n_out, cudaMemcpyDeviceToHost, st));
}

cudaStream_t S(void *s) { return (cudaStream_t)s; }

bool any_column_angle(const mpi_ffl_handle *h) {
    for (double th : h->angles)
        if (!(std::fabs(std::cos(th)) >= std::fabs(std::sin(th)) - 1e-9)) return true;
    return false;
}

void ensure_sig(mpi_ffl_handle *h) {
    if (!h->w_sig) dev_alloc(h, &h->w_sig, h->d.nsig);
}

// ------------------------------------------------------------ stages
// With pack.out[0] set, the interleaved projector writes the forward full stage's A
// operand instead of the projections; returns whether it did (the other projector
// always stores the projections).
bool stage_p(mpi_ffl_handle *h, const float *x, float *proj, cudaStream_t st, const ProjPack &pack = ProjPack{}) {
    if (h->w_volI) {  // the interleaved projector: both orientations from one pass over x
        const bool packed = pack.out[0] != nullptr;
        TIMED(MPI_FFL_K_TRANSPOSE, launch_interleave(x, h->w_volI, h->d.N, h->d.Nz, st));
        TIMED(MPI_FFL_K_PROJECT, launch_project_il(h->il_maps, h->t_ang, h->t_agroups, h->n_agroups,
                                                   packed ? nullptr : proj, h->d.N, h->d.Nz, st, h->w_err,
                                                   h->inject_polls, pack));
        check_launch(h, "project");
        return packed;
    }
    if (any_column_angle(h)) TIMED(MPI_FFL_K_TRANSPOSE, launch_transpose_xy(x, h->w_volT, h->d.N, h->d.Nz, st));
    TIMED(MPI_FFL_K_PROJECT, launch_project(x, h->w_volT, h->t_ang, h->t_agroups, h->n_agroups, proj, h->d.N, h->d.Nz, st, h->w_err));
    check_launch(h, "project");
    return false;
}

// Tiles of the staged E V B transpose, built on its first use (only the staged path and
// the stage entry point run it): the window of samples touching each tile's cells
// (start rounded down to 4 samples for 16-byte copies, length a multiple of 4), and each
// cell's entries, padded with (zero word, weight 0). ra_ntile stays 0 (the CSR gather
// serves) when a cell holds more entries, or a window more samples, than the kernel takes.
void ensure_ra_tables(mpi_ffl_handle *h) {
    if (h->ra_built) return;
    h->ra_built = true;
    const Dims &d = h->d;
    const std::vector<int> &ptr = h->csr_ptr_host;
    const std::vector<CsrEntry> &csr = h->csr_host;
    const int ntile = (d.Ne + kRaTileCells - 1) / kRaTileCells;
    std::vector<int4> tiles((size_t)d.n_par * ntile);
    bool fits = d.L % 4 == 0;
    int cap = 0;
    for (int par = 0; par < d.n_par && fits; ++par) {
        const int *P = ptr.data() + (size_t)par * (d.Ne + 1);
        const CsrEntry *C = csr.data() + (size_t)par * 2 * d.L;
        for (int t = 0; t < ntile && fits; ++t) {
            const int e0 = t * kRaTileCells, e1 = std::min(d.Ne, e0 + kRaTileCells);
            int jlo = d.L, jhi = -1;
            for (int e = e0; e < e1; ++e) {
                if (P[e + 1] - P[e] > kRaMaxEntries) fits = false;
                for (int k = P[e]; k < P[e + 1]; ++k) {
                    jlo = std::min(jlo, C[k].j);
                    jhi = std::max(jhi, C[k].j);
                }
            }
            if (jhi < 0) jlo = jhi = 0;
            jlo &= ~3;
            const int len = std::min(d.L - jlo, (jhi - jlo + 1 + 3) & ~3);
            cap = std::max(cap, len);
            tiles[(size_t)par * ntile + t] = make_int4(jlo, len, e0, e1 - e0);
        }
    }
    cap = (cap + 3) & ~3;
    if (fits && cap <= kRaMaxWindow) {
        const size_t per = (size_t)kRaMaxEntries * kRaTileCells;
        std::vector<uint16_t> tj((size_t)d.n_par * ntile * per, (uint16_t)cap);
        std::vector<float> tw((size_t)d.n_par * ntile * per, 0.f);
        // Entry k of a cell goes to half k & 1. Within a half, the 32 cells of a warp read
        // one entry each per step from the shared window, and two of them conflict when
        // their samples sit in the same 4-byte bank (j mod 32) at different addresses. Each
        // step therefore takes the largest set of lanes whose entries lie in distinct banks
        // (a bipartite matching of lanes to banks by augmenting paths, longest remaining
        // lists first); the other lanes take any entry. This only reorders the terms of
        // each cell's two partial sums: a fixed order per trajectory.
        for (int par = 0; par < d.n_par; ++par) {
            const int *P = ptr.data() + (size_t)par * (d.Ne + 1);
            const CsrEntry *C = csr.data() + (size_t)par * 2 * d.L;
            for (int t = 0; t < ntile; ++t) {
                const int4 T = tiles[(size_t)par * ntile + t];
                const size_t base = (size_t)(par * ntile + t) * per;
                for (int c0 = 0; c0 < T.w; c0 += 32)
                    for (int half = 0; half < 2; ++half) {
                        const int nl = std::min(32, T.w - c0);
                        std::vector<std::vector<CsrEntry>> rem(nl);
                        for (int l = 0; l < nl; ++l) {
                            const int e = T.z + c0 + l;
                            for (int k = P[e] + half; k < P[e + 1]; k += 2) rem[l].push_back(C[k]);
                        }
                        auto bank = [&](const CsrEntry &en) { return (en.j - T.x) & 31; };
                        for (int slot = 0;; ++slot) {
                            std::vector<int> lanes;
                            for (int l = 0; l < nl; ++l)
                                if (!rem[l].empty()) lanes.push_back(l);
                            if (lanes.empty()) break;
                            std::stable_sort(lanes.begin(), lanes.end(),
                                             [&](int a, int b) { return rem[a].size() > rem[b].size(); });
                            int owner[32];
                            std::fill(owner, owner + 32, -1);
                            std::vector<int> choice(nl, -1);
                            std::function<bool(int, uint32_t &)> augment = [&](int l, uint32_t &seen) {
                                for (size_t q = 0; q < rem[l].size(); ++q) {
                                    const int bk = bank(rem[l][q]);
                                    if (seen >> bk & 1u) continue;
                                    seen |= 1u << bk;
                                    if (owner[bk] < 0 || augment(owner[bk], seen)) {
                                        owner[bk] = l;
                                        choice[l] = (int)q;
                                        return true;
                                    }
                                }
                                return false;
                            };
                            for (int l : lanes) {
                                uint32_t seen = 0;
                                augment(l, seen);
                            }
                            for (int l : lanes) {
                                const size_t q = choice[l] >= 0 ? (size_t)choice[l] : 0;
                                const CsrEntry en = rem[l][q];
                                rem[l].erase(rem[l].begin() + (long)q);
                                const size_t at = base + (size_t)(2 * slot + half) * kRaTileCells + c0 + l;
                                tj[at] = (uint16_t)(en.j - T.x);
                                tw[at] = en.w;
                            }
                        }
                    }
            }
        }
        upload(h, &h->t_ra_tile, tiles);
        upload(h, &h->t_ra_j, tj);
        upload(h, &h->t_ra_w, tw);
        h->ra_ntile = ntile;
        h->ra_cap = cap;
    }
}

// E V B transpose: the tiled kernel where the trajectory fits it, else the CSR gather
void resample_adj(mpi_ffl_handle *h, const float *sig, float *fine, cudaStream_t st) {
    const Dims &d = h->d;
    ensure_ra_tables(h);
    if (h->ra_ntile > 0)
        launch_resample_adj_tiled(sig, h->t_ra_tile, h->t_ra_j, h->t_ra_w, h->t_gain, fine, d, h->ra_ntile, h->ra_cap,
                                  h->w_err, st);
    else
        launch_resample_adj(sig, h->t_csr_ptr, h->t_csr, h->t_gain, h->t_groups, h->n_groups, fine, d, st);
}

void stage_pt(mpi_ffl_handle *h, const float *proj, float *x, cudaStream_t st) {
    TIMED(MPI_FFL_K_BACKPROJECT, launch_backproject(proj, h->t_ang, x, h->d.N, h->d.Nz, h->d.M, st));
    check_launch(h, "backproject");
}

// blockdiag(A_DC) on projections: proj -> data
// prepacked: the projector wrote the full stage's A operand (proj not stored)
void line_forward_impl(mpi_ffl_handle *h, const float *proj, float *b, const float *htab, const float *gain,
                       cudaStream_t st, bool prepacked = false) {
    const Dims &d = h->d;
    if (h->psf_model == MPI_FFL_PSF_TENSOR) {
        // slices coupled by the tensor PSF; the coil map and the gains are applied inside
        TIMED(MPI_FFL_K_TENSOR, ten_forward(h, proj, h->t_coil, b, st));
        check_launch(h, "tensor forward");
        return;
    }
    if (h->t_coil) {  // B: the coil map before the PSF
        TIMED(MPI_FFL_K_COIL, launch_coil_pad(proj, h->t_coil, h->w_projc, (long long)d.M * d.Nz, d.Nz, d.N, d.N, st));
        proj = h->w_projc;
    }
    int path = h->path;
    if (path == MPI_FFL_PATH_FULL_GEMM && htab != h->t_htab) path = MPI_FFL_PATH_LINE_GEMM;  // other taps
    if (path == MPI_FFL_PATH_FULL_GEMM) {
        TIMED(MPI_FFL_K_GEMM_FWD, col_forward(h, proj, true, gain, b, st, prepacked));
        check_launch(h, "gemm_fwd");
        return;
    }
    TIMED(MPI_FFL_K_PSF_FWD, launch_psf_fwd(proj, htab, h->w_fine, d, st));
    check_launch(h, "psf_fwd");
    if (path == MPI_FFL_PATH_LINE_GEMM) {
        TIMED(MPI_FFL_K_GEMM_FWD, col_forward(h, h->w_fine, false, gain, b, st));
        check_launch(h, "gemm_fwd");
        return;
    }
    if (path == MPI_FFL_PATH_FUSED) {
        TIMED(MPI_FFL_K_TC_FWD, tc_forward_line(h, h->w_fine, gain, b, st));
        check_launch(h, "tc_forward");
        return;
    }
    ensure_sig(h);
    TIMED(MPI_FFL_K_RESAMPLE_FWD, launch_resample_fwd(h->w_fine, h->t_traj, gain, h->t_groups, h->n_groups, h->w_sig, d, st));
    check_launch(h, "resample_fwd");
    TIMED(MPI_FFL_K_DFT_FWD, launch_dft_fwd(h->w_sig, h->t_tw1, h->t_twp, h->t_tw2_ro, h->t_dgam, b, d, h->w_err, st));
    check_launch(h, "dft_fwd");
}

void forward_impl(mpi_ffl_handle *h, const float *x, float *b, const float *htab, const float *gain,
                  cudaStream_t st) {
    // The full-GEMM stage with the collinear PSF's own taps, no coil map: the projector
    // splits its sums into the GEMM's A operand itself (the packing pass and the
    // projections' round trip through HBM drop out; the same hi + lo values).
    ProjPack pack{};
    const bool fold = h->path == MPI_FFL_PATH_FULL_GEMM && h->psf_model != MPI_FFL_PSF_TENSOR && !h->t_coil &&
                      htab == h->t_htab && col_prepack_targets(h, &pack);
    const bool packed = stage_p(h, x, h->w_proj, st, fold ? pack : ProjPack{});
    line_forward_impl(h, h->w_proj, b, htab, gain, st, packed);
}

// blockdiag(A_DC)^T without B's coil map: data -> projections
void line_adjoint_body(mpi_ffl_handle *h, const float *b, float *proj, cudaStream_t st) {
    const Dims &d = h->d;
    if (h->path == MPI_FFL_PATH_FULL_GEMM) {
        TIMED(MPI_FFL_K_GEMM_ADJ, col_adjoint(h, b, true, h->t_gain, proj, st));
        check_launch(h, "gemm_adj");
        return;
    }
    if (h->path == MPI_FFL_PATH_LINE_GEMM) {
        TIMED(MPI_FFL_K_GEMM_ADJ, col_adjoint(h, b, false, h->t_gain, h->w_fine, st));
        check_launch(h, "gemm_adj");
    } else if (h->path == MPI_FFL_PATH_FUSED) {
        TIMED(MPI_FFL_K_TC_ADJ, tc_adjoint_line(h, b, h->t_gain, h->w_fine, st));
        check_launch(h, "tc_adjoint");
    } else {
        ensure_sig(h);
        TIMED(MPI_FFL_K_DFT_ADJ, launch_dft_adj(b, h->t_tw1, h->t_twp, h->t_tw2_qr, h->t_dgam, h->w_sig, d, st));
        check_launch(h, "dft_adj");
        TIMED(MPI_FFL_K_RESAMPLE_ADJ, resample_adj(h, h->w_sig, h->w_fine, st));
        check_launch(h, "resample_adj");
    }
    TIMED(MPI_FFL_K_PSF_ADJ, launch_psf_adj(h->w_fine, h->t_htab, proj, d, st));
    check_launch(h, "psf_adj");
}

// blockdiag(A_DC)^T: data -> projections
void line_adjoint_impl(mpi_ffl_handle *h, const float *b, float *proj, cudaStream_t st) {
    const Dims &d = h->d;
    if (h->psf_model == MPI_FFL_PSF_TENSOR) {
        TIMED(MPI_FFL_K_TENSOR, ten_adjoint(h, b, h->t_coil, proj, st));
        check_launch(h, "tensor adjoint");
        return;
    }
    line_adjoint_body(h, b, proj, st);
    if (h->t_coil) {  // B^T: the coil map after the PSF's transpose (in place)
        TIMED(MPI_FFL_K_COIL, launch_coil_pad(proj, h->t_coil, proj, (long long)d.M * d.Nz, d.Nz, d.N, d.N, st));
        check_launch(h, "coil");
    }
}

void adjoint_impl(mpi_ffl_handle *h, const float *b, float *x, cudaStream_t st) {
    line_adjoint_impl(h, b, h->w_proj, st);
    stage_pt(h, h->w_proj, x, st);
}

// d loss / d gain_m = <g_b[m], A_m x |_{g_m = 1}> and d loss / d fwhm = <g_b, (dA/dfwhm) x>,
// from the projections P x
void param_grad_impl(mpi_ffl_handle *h, const float *proj, const float *d_gb, float *d_g_gain, float *d_g_fwhm,
                     cudaStream_t st) {
    const Dims &d = h->d;
    if (d_g_gain) {
        line_forward_impl(h, proj, h->s_r, h->t_htab, h->t_unit_gain, st);
        const int64_t per = (int64_t)2 * d.Nz * d.nb;
        const int nbk = std::min(1024, std::max(1, (int)((per + 1023) / 1024)));
        TIMED(MPI_FFL_K_SOLVER, launch_angle_dots(h->s_r, d_gb, d.M, per, h->w_red, nbk, st));
        TIMED(MPI_FFL_K_SOLVER, launch_angle_finalize(h->w_red, d.M, nbk, d_g_gain, st));
        check_launch(h, "gain grad");
    }
    if (d_g_fwhm) {
        line_forward_impl(h, proj, h->s_r, h->t_dhtab, h->t_gain, st);
        const int nbk = reduce_blocks(d.ndata);
        TIMED(MPI_FFL_K_SOLVER, launch_dot(h->s_r, d_gb, d.ndata, h->w_red, nbk, st));
        TIMED(MPI_FFL_K_SOLVER, launch_finalize_to_float(h->w_red, nbk, d_g_fwhm, st));
        check_launch(h, "fwhm grad");
    }
}

double dot_sync(mpi_ffl_handle *h, const float *a, const float *b, int64_t n, cudaStream_t st) {
    const int nb = reduce_blocks(n);
    TIMED(MPI_FFL_K_SOLVER, launch_dot(a, b, n, h->w_red, nb, st));
    TIMED(MPI_FFL_K_SOLVER, launch_finalize(h->w_red, nb, h->w_scal + 7, st));
    check_launch(h, "dot");
    double v = 0;
    CK(cudaMemcpyAsync(&v, h->w_scal + 7, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return v;
}

// The operator of the selected scans (Sec. 3.1: an x-drive and a z-drive scan per
// angle): r = [A x; A_z x] in that order, and its transpose A^T r + A_z^T r_z (the
// two volumes summed in a fixed order).
int64_t scan_data_len(const mpi_ffl_handle *h) {
    return (int64_t)(((h->scans & MPI_FFL_SCAN_X) ? 1 : 0) + ((h->scans & MPI_FFL_SCAN_Z) ? 1 : 0)) * h->d.ndata;
}

void scans_forward(mpi_ffl_handle *h, const float *x, float *r, cudaStream_t st) {
    if (h->scans & MPI_FFL_SCAN_X) {
        forward_impl(h, x, r, h->t_htab, h->t_gain, st);
        r += h->d.ndata;
    }
    if (h->scans & MPI_FFL_SCAN_Z) forward_z_impl(h, x, r, st);
}

void scans_adjoint(mpi_ffl_handle *h, const float *r, float *g, cudaStream_t st) {
    const Dims &d = h->d;
    if (h->scans == (MPI_FFL_SCAN_X | MPI_FFL_SCAN_Z)) {
        adjoint_impl(h, r, h->w_scanvol, st);
        adjoint_z_impl(h, r + d.ndata, h->w_scanvol + d.nvox, st);
        TIMED(MPI_FFL_K_SOLVER, launch_coil_pad(h->w_scanvol, nullptr, g, (long long)d.Nz * d.N, d.Nz, d.N, d.N, st, 2,
                                                d.nvox));
        check_launch(h, "scan sum");
    } else if (h->scans & MPI_FFL_SCAN_X) {
        adjoint_impl(h, r, g, st);
    } else {
        adjoint_z_impl(h, r, g, st);
    }
}

double power_norm_impl(mpi_ffl_handle *h, int n_iter, uint64_t seed, cudaStream_t st) {
    const Dims &d = h->d;
    float *v = h->w_vol2, *w = h->s_g;
    const int nbv = reduce_blocks(d.nvox);
    TIMED(MPI_FFL_K_SOLVER, launch_splitmix_fill(v, d.nvox, seed, st));
    TIMED(MPI_FFL_K_SOLVER, launch_dot(v, v, d.nvox, h->w_red, nbv, st));
    TIMED(MPI_FFL_K_SOLVER, launch_finalize(h->w_red, nbv, h->w_scal + 0, st));
    TIMED(MPI_FFL_K_SOLVER, launch_scale_by_rsqrt(v, v, d.nvox, h->w_scal + 0, st));
    check_launch(h, "power init");
    for (int it = 0; it < n_iter; ++it) {
        scans_forward(h, v, h->w_data, st);
        scans_adjoint(h, h->w_data, w, st);
        TIMED(MPI_FFL_K_SOLVER, launch_dot(v, w, d.nvox, h->w_red, nbv, st));
        TIMED(MPI_FFL_K_SOLVER, launch_finalize(h->w_red, nbv, h->w_scal + 1, st));
        TIMED(MPI_FFL_K_SOLVER, launch_dot(w, w, d.nvox, h->w_red, nbv, st));
        TIMED(MPI_FFL_K_SOLVER, launch_finalize(h->w_red, nbv, h->w_scal + 0, st));
        TIMED(MPI_FFL_K_SOLVER, launch_scale_by_rsqrt(w, v, d.nvox, h->w_scal + 0, st));
        check_launch(h, "power step");
    }
    double mu = 0;
    CK(cudaMemcpyAsync(&mu, h->w_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return mu;
}

double ttt_norm(const Dims &d) {
    double s = 0;
    const int ns[3] = {d.Nz, d.N, d.N};
    for (int n : ns) {
        const double v = std::sin(kPi * (n - 1) / (2.0 * n));
        s += 4.0 * v * v;
    }
    return s;
}

template <class F>
int guarded(mpi_ffl_handle *h, F &&f) {
    if (!h) return MPI_FFL_ERR_INVALID_ARG;
    try {
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev != h->device) cudaSetDevice(h->device);
        return f();
    } catch (const Fail &e) {
        return e.code;
    } catch (const std::bad_alloc &) {
        h->err = "host allocation failed";
        return MPI_FFL_ERR_OOM;
    } catch (...) {
        h->err = "unexpected exception";
        return MPI_FFL_ERR_CUDA;
    }
}

}  // namespace

namespace mpiffl {
void set_thread_error(const std::string &msg) { g_create_error = msg; }
double power_norm_for_job(mpi_ffl_handle *h, int n_iter, uint64_t seed, cudaStream_t st) {
    return power_norm_impl(h, n_iter, seed, st);
}
double ttt_norm_for_job(const Dims &d) { return ttt_norm(d); }
bool handle_has_column_angles(const mpi_ffl_handle *h) { return any_column_angle(h); }
void forward_for_job(mpi_ffl_handle *h, const float *x, float *b, cudaStream_t st) {
    forward_impl(h, x, b, h->t_htab, h->t_gain, st);
}
void adjoint_for_job(mpi_ffl_handle *h, const float *b, float *x, cudaStream_t st) { adjoint_impl(h, b, x, st); }
}  // namespace mpiffl

// ============================================================ C ABI

extern "C" int mpi_ffl_create(const mpi_ffl_geometry *geom, const mpi_ffl_trajectory *traj,
                              const mpi_ffl_psf *psf, const mpi_ffl_harmonics *harm,
                              mpi_ffl_handle **out) {
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return MPI_FFL_ERR_INVALID_ARG;
    }
    *out = nullptr;
    Dims d{};
    std::string why;
    int rc = compute_dims(geom, traj, harm, d, why);
    if (rc) {
        g_create_error = why;
        return rc;
    }
    if (!psf || !(psf->fwhm_vox > 0.0)) {
        g_create_error = "fwhm_vox must be > 0";
        return MPI_FFL_ERR_INVALID_ARG;
    }
    mpi_ffl_handle *h = new (std::nothrow) mpi_ffl_handle();
    if (!h) {
        g_create_error = "host allocation failed";
        return MPI_FFL_ERR_OOM;
    }
    h->d = d;
    try {
        CK(cudaGetDevice(&h->device));
        h->angles.resize(d.M);
        h->gains.resize(d.M);
        for (int m = 0; m < d.M; ++m) {
            h->angles[m] = geom->angles_rad ? geom->angles_rad[m] : m * kPi / d.M;
            h->gains[m] = geom->gain ? geom->gain[m] : 1.0f;
            if (!std::isfinite(h->angles[m]) || !std::isfinite(h->gains[m])) {
                set_err(nullptr, "non-finite angle or gain");
                throw Fail{MPI_FFL_ERR_INVALID_ARG};
            }
        }
        h->fwhm = psf->fwhm_vox;
        h->amp = traj->drive_amp_vox;
        h->phase = traj->drive_phase;
        h->zigzag = traj->zigzag ? 1 : 0;
        h->dgamma.assign(2 * d.nb, 0.f);
        for (int o = 0; o < d.nb; ++o) {
            h->dgamma[2 * o] = harm->d_gamma_ri ? harm->d_gamma_ri[2 * o] : 1.f;
            h->dgamma[2 * o + 1] = harm->d_gamma_ri ? harm->d_gamma_ri[2 * o + 1] : 0.f;
        }
        angle_table(h);
        upload(h, &h->t_gain, h->gains);
        upload(h, &h->t_unit_gain, std::vector<float>(d.M, 1.f));
        std::vector<float> ht, dht;
        psf_tables(d, h->fwhm, ht, dht);
        upload(h, &h->t_htab, ht);
        upload(h, &h->t_dhtab, dht);
        trajectory_tables(h);
        dft_tables(h);
        group_table(h);
        dev_alloc(h, &h->w_volT, d.nvox);
        if (project_il_ok(d.N)) {
            dev_alloc(h, &h->w_volI, il_len(d.N, d.Nz));
            if (!make_il_maps(h->w_volI, d.N, d.Nz, &h->il_maps)) {  // the pipelined projector serves
                dev_free(h->w_volI);
                h->w_volI = nullptr;
                h->bytes -= (int64_t)(il_len(d.N, d.Nz) * sizeof(float));
            }
        }
        dev_alloc(h, &h->w_proj, d.nproj);
        dev_alloc(h, &h->w_fine, d.nfine);
        dev_alloc(h, &h->w_data, d.ndata);
        dev_alloc(h, &h->w_vol2, d.nvox);
        h->w_red_len = std::max(reduce_blocks(std::max(d.nvox, d.ndata)) + 16, 1024 * std::max(d.M, 1));
        dev_alloc(h, &h->w_red, (size_t)h->w_red_len);
        dev_alloc(h, &h->w_scal, 16);
        dev_alloc(h, &h->s_xp, d.nvox);
        dev_alloc(h, &h->s_y, d.nvox);
        dev_alloc(h, &h->s_g, d.nvox);
        dev_alloc(h, &h->s_r, d.ndata);
        dev_alloc(h, &h->s_flags, 4);
        dev_alloc(h, &h->w_err, 1);
        CK(cudaMemset(h->w_err, 0, sizeof(int)));
        tc_init(h);
        if (tc_init_oom(h)) {
            set_err(h, "device allocation failed for the tensor-core tables");
            throw Fail{MPI_FFL_ERR_OOM};
        }
        CK(cudaDeviceSynchronize());
    } catch (const Fail &e) {
        if (g_create_error.empty()) g_create_error = h->err.empty() ? "create failed" : h->err;
        release(h);
        delete h;
        return e.code;
    } catch (...) {
        g_create_error = "create failed (host exception)";
        release(h);
        delete h;
        return MPI_FFL_ERR_OOM;
    }
    *out = h;
    return MPI_FFL_OK;
}

extern "C" int mpi_ffl_destroy(mpi_ffl_handle *h) {
    if (!h) return MPI_FFL_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) cudaSetDevice(h->device);
    const int own = h->device;
    cudaDeviceSynchronize();
    release(h);
    delete h;
    if (dev != own) cudaSetDevice(dev);
    return MPI_FFL_OK;
}

extern "C" const char *mpi_ffl_last_error(const mpi_ffl_handle *h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

extern "C" int mpi_ffl_get_sizes(const mpi_ffl_handle *h, mpi_ffl_sizes *o) {
    if (!h || !o) return MPI_FFL_ERR_INVALID_ARG;
    o->n_vox = h->d.nvox;
    o->n_data = h->d.ndata;
    o->n_proj = h->d.nproj;
    o->n_fine = h->d.nfine;
    o->n_sig = h->d.nsig;
    o->n_bins = h->d.nb;
    o->fine_len = h->d.Ne;
    o->line_len = h->d.L;
    o->fine_len_z = h->d.Nez;
    o->workspace_bytes = h->bytes;
    return MPI_FFL_OK;
}

static int set_precision_impl(mpi_ffl_handle *h, int32_t precision) {
    if (!h) return MPI_FFL_ERR_INVALID_ARG;
    if (precision < MPI_FFL_PREC_FP32 || precision > MPI_FFL_PREC_TF32) {
        h->err = "unknown precision";
        return MPI_FFL_ERR_INVALID_ARG;
    }
    if (precision == MPI_FFL_PREC_TF32) {
        if (h->path != MPI_FFL_PATH_LINE_GEMM && h->path != MPI_FFL_PATH_FULL_GEMM) {
            h->err = "TF32 splits are built for the GEMM paths only";
            return MPI_FFL_ERR_UNSUPPORTED;
        }
        h->precision = precision;
        return MPI_FFL_OK;
    }
    if (precision == MPI_FFL_PREC_FP32) {
        h->precision = precision;
        h->path = MPI_FFL_PATH_STAGED;
        return MPI_FFL_OK;
    }
    if (h->path == MPI_FFL_PATH_STAGED) {
        if (!tc_supported(h)) {
            h->err = "tensor-core path does not support this problem shape";
            return MPI_FFL_ERR_UNSUPPORTED;
        }
        h->path = MPI_FFL_PATH_FUSED;
    }
    h->precision = precision;
    return MPI_FFL_OK;
}

static int set_path_impl(mpi_ffl_handle *h, int32_t path) {
    if (!h) return MPI_FFL_ERR_INVALID_ARG;
    if (path < MPI_FFL_PATH_STAGED || path > MPI_FFL_PATH_FULL_GEMM) {
        h->err = "unknown path";
        return MPI_FFL_ERR_INVALID_ARG;
    }
    if (path == MPI_FFL_PATH_FULL_GEMM && col_psf_stale(h)) col_release(h);  // rebuilt below for this PSF
    if ((path == MPI_FFL_PATH_LINE_GEMM || path == MPI_FFL_PATH_FULL_GEMM) && !h->col_state) {
        try {
            col_init(h);  // W and W H are built on first use
        } catch (...) {
            col_release(h);
            h->err = "building the collapsed line operator failed";
            return MPI_FFL_ERR_OOM;
        }
        if (col_init_oom(h)) {  // nothing of a failed build is kept: the next call retries
            col_release(h);
            h->err = "device allocation failed while building the collapsed line operator";
            return MPI_FFL_ERR_OOM;
        }
    }
    if ((path == MPI_FFL_PATH_FUSED && !tc_supported(h)) ||
        ((path == MPI_FFL_PATH_LINE_GEMM || path == MPI_FFL_PATH_FULL_GEMM) && !col_supported(h))) {
        h->err = "this path does not support the problem shape";
        return MPI_FFL_ERR_UNSUPPORTED;
    }
    const bool keep_tf32 = h->precision == MPI_FFL_PREC_TF32 &&
                           (path == MPI_FFL_PATH_LINE_GEMM || path == MPI_FFL_PATH_FULL_GEMM);
    h->path = path;
    h->precision = path == MPI_FFL_PATH_STAGED ? MPI_FFL_PREC_FP32
                   : keep_tf32                 ? MPI_FFL_PREC_TF32
                                               : MPI_FFL_PREC_BF16X3;
    return MPI_FFL_OK;
}

// the tensor-PSF tables hold split operands of the handle's precision
static int refresh_tensor(mpi_ffl_handle *h, int rc) {
    if (rc != MPI_FFL_OK || h->psf_model != MPI_FFL_PSF_TENSOR) return rc;
    return guarded(h, [&]() {
        CK(cudaDeviceSynchronize());
        const int r = ten_refresh(h, false);
        if (r != MPI_FFL_OK) h->err = "rebuilding the tensor-PSF operands failed";
        return r;
    });
}

extern "C" int mpi_ffl_set_precision(mpi_ffl_handle *h, int32_t precision) {
    return refresh_tensor(h, set_precision_impl(h, precision));
}

extern "C" int mpi_ffl_set_path(mpi_ffl_handle *h, int32_t path) { return refresh_tensor(h, set_path_impl(h, path)); }

extern "C" int mpi_ffl_set_psf_model(mpi_ffl_handle *h, int32_t model) {
    return guarded(h, [&]() {
        if (model != MPI_FFL_PSF_COLLINEAR && model != MPI_FFL_PSF_TENSOR) {
            h->err = "unknown PSF model";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        CK(cudaDeviceSynchronize());
        if (model == MPI_FFL_PSF_TENSOR && !ten_ready(h)) {
            if (!h->col_state) col_init(h);
            const int rc = ten_init(h);
            if (rc != MPI_FFL_OK) {
                h->err = rc == MPI_FFL_ERR_UNSUPPORTED
                             ? "the tensor PSF needs the collapsed line operator, which this shape does not support"
                             : "building the tensor-PSF operator failed";
                return rc;
            }
        }
        h->psf_model = model;
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_get_psf_model(const mpi_ffl_handle *h) { return h ? h->psf_model : MPI_FFL_ERR_INVALID_ARG; }

extern "C" int mpi_ffl_set_coil_map(mpi_ffl_handle *h, const float *b_zu) {
    return guarded(h, [&]() {
        const Dims &d = h->d;
        CK(cudaDeviceSynchronize());
        if (!b_zu) {
            if (h->t_coil) CK(dev_free(h->t_coil));
            h->t_coil = nullptr;
            return MPI_FFL_OK;
        }
        for (int64_t k = 0; k < (int64_t)d.Nz * d.N; ++k)
            if (!std::isfinite(b_zu[k])) {
                h->err = "coil map holds a non-finite value";
                return MPI_FFL_ERR_INVALID_ARG;
            }
        if (!h->t_coil) dev_alloc(h, &h->t_coil, (size_t)d.Nz * d.N);
        if (!h->w_projc) dev_alloc(h, &h->w_projc, (size_t)d.M * d.Nz * d.N);
        CK(cudaMemcpy(h->t_coil, b_zu, sizeof(float) * d.Nz * d.N, cudaMemcpyHostToDevice));
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_set_scans(mpi_ffl_handle *h, int32_t scans) {
    return guarded(h, [&]() {
        if (scans < MPI_FFL_SCAN_X || scans > (MPI_FFL_SCAN_X | MPI_FFL_SCAN_Z)) {
            h->err = "scans must be MPI_FFL_SCAN_X, MPI_FFL_SCAN_Z or both";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        const Dims &d = h->d;
        CK(cudaDeviceSynchronize());
        if (scans & MPI_FFL_SCAN_Z) z_init(h);
        const int n = ((scans & MPI_FFL_SCAN_X) ? 1 : 0) + ((scans & MPI_FFL_SCAN_Z) ? 1 : 0);
        if (n == 2 && !h->w_scanvol) {
            // residual and power-iteration data of both scans, and the two transposes
            float *r = nullptr, *w = nullptr;
            dev_alloc(h, &r, (size_t)2 * d.ndata);
            dev_alloc(h, &w, (size_t)2 * d.ndata);
            dev_alloc(h, &h->w_scanvol, (size_t)2 * d.nvox);
            CK(dev_free(h->s_r));
            CK(dev_free(h->w_data));
            h->bytes -= (int64_t)(2 * d.ndata * sizeof(float));
            h->s_r = r;
            h->w_data = w;
        }
        h->scans = scans;
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_get_scans(const mpi_ffl_handle *h) { return h ? h->scans : MPI_FFL_ERR_INVALID_ARG; }

extern "C" int mpi_ffl_get_path(const mpi_ffl_handle *h) { return h ? h->path : MPI_FFL_ERR_INVALID_ARG; }
extern "C" int mpi_ffl_get_precision(const mpi_ffl_handle *h) {
    return h ? h->precision : MPI_FFL_ERR_INVALID_ARG;
}

extern "C" int mpi_ffl_set_gain(mpi_ffl_handle *h, const float *gain) {
    return guarded(h, [&]() {
        if (!gain) {
            h->err = "gain is NULL";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        for (int m = 0; m < h->d.M; ++m) h->gains[m] = gain[m];
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(h->t_gain, h->gains.data(), sizeof(float) * h->d.M, cudaMemcpyHostToDevice));
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_set_psf_fwhm(mpi_ffl_handle *h, double fwhm) {
    return guarded(h, [&]() {
        if (!(fwhm > 0.0)) {
            h->err = "fwhm must be > 0";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        h->fwhm = fwhm;
        std::vector<float> ht, dht;
        psf_tables(h->d, fwhm, ht, dht);
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(h->t_htab, ht.data(), sizeof(float) * ht.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->t_dhtab, dht.data(), sizeof(float) * dht.size(), cudaMemcpyHostToDevice));
        tc_tables_changed(h);
        // W H holds the PSF: rebuild the collapsed operator if it was built and the
        // full-GEMM path is selected; otherwise W (which holds no PSF) stays and W H is
        // rebuilt when the full-GEMM path is next selected
        const bool had = col_supported(h);
        if (h->col_state) {
            if (h->path == MPI_FFL_PATH_FULL_GEMM) {
                col_release(h);
                col_init(h);
            } else {
                col_mark_psf_stale(h);
            }
        }
        if (had && !col_supported(h) && (h->path == MPI_FFL_PATH_LINE_GEMM || h->path == MPI_FFL_PATH_FULL_GEMM)) {
            h->path = MPI_FFL_PATH_STAGED;
            h->precision = MPI_FFL_PREC_FP32;
            h->psf_model = MPI_FFL_PSF_COLLINEAR;
            h->err = "collapsed operator could not be rebuilt; fell back to the staged path";
            return MPI_FFL_ERR_OOM;
        }
        if (h->psf_model == MPI_FFL_PSF_TENSOR && ten_init(h) != MPI_FFL_OK) {
            h->psf_model = MPI_FFL_PSF_COLLINEAR;
            h->err = "tensor-PSF operator could not be rebuilt; fell back to the collinear PSF";
            return MPI_FFL_ERR_OOM;
        }
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_sync_check(mpi_ffl_handle *h, void *stream) {
    return guarded(h, [&]() {
        CK(cudaStreamSynchronize(S(stream)));
        h->inject_polls = 0;
        int werr = 0;
        CK(cudaMemcpy(&werr, h->w_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (werr) CK(cudaMemset(h->w_err, 0, sizeof(int)));
        if (tc_take_error(h) | col_take_error(h) | werr) {
            h->err = "a tensor-core kernel gave up on a bounded wait";
            return MPI_FFL_ERR_TIMEOUT;
        }
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_test_inject_timeout(mpi_ffl_handle *h, uint32_t polls) {
    return guarded(h, [&]() {
        if (polls > (1u << 24)) {
            h->err = "polls above the kernels' own limit of 2^24";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        h->inject_polls = polls;
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_forward(mpi_ffl_handle *h, const float *x, float *b, void *stream) {
    return guarded(h, [&]() {
        if (!x || !b) {
            h->err = "NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        cudaStream_t st = S(stream);
        with_host_buffers(h, x, h->d.nvox, b, h->d.ndata, st, [&](const float *dx, float *db) {
            forward_impl(h, dx, db, h->t_htab, h->t_gain, st);
        });
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_adjoint(mpi_ffl_handle *h, const float *b, float *x, void *stream) {
    return guarded(h, [&]() {
        if (!x || !b) {
            h->err = "NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        cudaStream_t st = S(stream);
        with_host_buffers(h, b, h->d.ndata, x, h->d.nvox, st, [&](const float *db, float *dx) {
            adjoint_impl(h, db, dx, st);
        });
        return MPI_FFL_OK;
    });
}

// ------------------------------------------------------------ z-drive scan
int float_bits(float f) {
    int i;
    std::memcpy(&i, &f, 4);
    return i;
}

// Tables of the z-drive scan, in double precision on the host: the slow raster's
// detector column and fraction per (parity, j), the drive's fine z offset, fraction
// and velocity per phase r = j mod S, the periods reading each column, and the
// transpose's taps grouped by residue of the fine index modulo Q.
void z_init(mpi_ffl_handle *h) {
    if (h->z_ready) return;
    const Dims &d = h->d;
    const int L = d.L, S = d.S, N = d.N, P = d.P, Q = d.Q, npar = d.n_par;
    if ((size_t)(d.Nz + 1) * S * 4 > 200 * 1024) {
        h->err = "the z-drive transpose keeps (N_z + 1) x S floats in shared memory (at most 200 KB)";
        throw Fail{MPI_FFL_ERR_UNSUPPORTED};
    }
    const double slope = (double)(N - 1) / (double)(L - 1);
    std::vector<int> u0((size_t)npar * L);
    std::vector<float2> ua((size_t)npar * L);
    for (int par = 0; par < npar; ++par)
        for (int j = 0; j < L; ++j) {
            const double c = par ? (N - 1) - slope * j : slope * j;
            int k = (int)std::floor(c);
            k = std::min(std::max(k, 0), N - 1);
            u0[(size_t)par * L + j] = k;
            float kb;
            std::memcpy(&kb, &k, 4);
            ua[(size_t)par * L + j] = make_float2(kb, (float)(c - k));
        }
    const double kPi = 3.14159265358979323846;
    std::vector<int> n0(S);
    std::vector<float> f0(S), v(S);
    for (int r = 0; r < S; ++r) {
        const double ph = 2.0 * kPi * r / S + h->phase;
        const double t = Q * h->amp * std::sin(ph) + d.D;
        n0[r] = (int)std::floor(t);
        f0[r] = (float)(t - n0[r]);
        v[r] = (float)(h->amp * (2.0 * kPi / S) * std::cos(ph));
    }
    std::vector<int> plo((size_t)npar * S * N, 0), phi((size_t)npar * S * N, -1);
    for (int par = 0; par < npar; ++par)
        for (int r = 0; r < S; ++r)
            for (int p = 0; p < P; ++p) {
                const int k = u0[(size_t)par * L + (size_t)p * S + r];
                for (int u : {k, k + 1}) {
                    if (u >= N) continue;
                    const size_t i = ((size_t)par * S + r) * N + u;
                    if (phi[i] < 0) plo[i] = p;
                    phi[i] = p;
                }
            }
    std::vector<int> ptr(Q + 1, 0);
    std::vector<int4> taps;
    for (int rho = 0; rho < Q; ++rho) {
        ptr[rho] = (int)taps.size();
        for (int r = 0; r < S; ++r) {
            if (((n0[r] % Q) + Q) % Q == rho) taps.push_back(make_int4(r, n0[r], float_bits(1.f - f0[r]), 0));
            if ((((n0[r] + 1) % Q) + Q) % Q == rho) taps.push_back(make_int4(r, n0[r] + 1, float_bits(f0[r]), 0));
        }
    }
    ptr[Q] = (int)taps.size();
    // the same taps by offset o = e - Q l within a line's cells (the fused transpose)
    int no = 0;
    for (int r = 0; r < S; ++r) no = std::max(no, n0[r] + 2);
    std::vector<int> optr(no + 1, 0);
    std::vector<int2> otap;
    for (int o = 0; o < no; ++o) {
        optr[o] = (int)otap.size();
        for (int r = 0; r < S; ++r) {
            if (n0[r] == o) otap.push_back(make_int2(r, float_bits(1.f - f0[r])));
            if (n0[r] + 1 == o) otap.push_back(make_int2(r, float_bits(f0[r])));
        }
    }
    optr[no] = (int)otap.size();
    h->tz_no = no;
    if (zsyn_smem(d, no) > 227 * 1024 || zdft_fwd_smem(d) > 227 * 1024) {
        h->err = "the fused z-drive kernels keep twiddles and tiles in shared memory (at most 227 KB)";
        throw Fail{MPI_FFL_ERR_UNSUPPORTED};
    }
    upload(h, &h->tz_optr, optr);
    upload(h, &h->tz_otap, otap);
    upload(h, &h->tz_ua, ua);
    upload(h, &h->tz_n0, n0);
    upload(h, &h->tz_f0, f0);
    upload(h, &h->tz_v, v);
    upload(h, &h->tz_plo, plo);
    upload(h, &h->tz_phi, phi);
    upload(h, &h->tz_tap_ptr, ptr);
    upload(h, &h->tz_taps, taps);
    dev_alloc(h, &h->w_fine_z, (size_t)d.M * N * d.Nez);
    dev_alloc(h, &h->w_projT, (size_t)d.M * N * d.Nz);
    dev_alloc(h, &h->w_zcoef, (size_t)d.M * d.Nz * (2 * d.hw + 1) * S);
    h->z_ready = 1;
}

ZTables z_tables(const mpi_ffl_handle *h) {
    return ZTables{h->tz_ua,  h->tz_n0,      h->tz_f0,   h->tz_v,    h->tz_plo, h->tz_phi,
                   h->tz_tap_ptr, h->tz_taps, h->tz_optr, h->tz_otap, h->tz_no};
}

// the PSF kernels along z: lines are the M N detector columns, N_z slices long
Dims z_dims(const Dims &d) {
    Dims dz = d;
    dz.N = d.Nz;
    dz.Nz = d.N;
    dz.nseg = d.M * d.N;
    dz.Ne = d.Nez;
    return dz;
}

void zstage_h(mpi_ffl_handle *h, const float *proj, float *cz, cudaStream_t st) {
    const Dims &d = h->d;
    TIMED(MPI_FFL_K_ZDRIVE, launch_transpose_2d(proj, h->w_projT, d.M, d.Nz, d.N, st));
    TIMED(MPI_FFL_K_PSF_FWD, launch_psf_fwd(h->w_projT, h->t_htab, cz, z_dims(d), st));
}

void zstage_ht(mpi_ffl_handle *h, const float *cz, float *proj, cudaStream_t st) {
    const Dims &d = h->d;
    TIMED(MPI_FFL_K_PSF_ADJ, launch_psf_adj(cz, h->t_htab, h->w_projT, z_dims(d), st));
    TIMED(MPI_FFL_K_ZDRIVE, launch_transpose_2d(h->w_projT, proj, d.M, d.N, d.Nz, st));
}

void zstage_ev(mpi_ffl_handle *h, const float *cz, float *sig, cudaStream_t st) {
    TIMED(MPI_FFL_K_ZDRIVE, launch_resample_z_fwd(cz, z_tables(h), h->t_gain, sig, h->d, h->zigzag, st));
}

void zstage_evt(mpi_ffl_handle *h, const float *sig, float *cz, cudaStream_t st) {
    if (!h->w_tz) dev_alloc(h, &h->w_tz, (size_t)h->d.M * h->d.Nz * h->d.N * h->d.S);
    TIMED(MPI_FFL_K_ZDRIVE, launch_resample_z_adj(sig, z_tables(h), h->t_gain, h->w_tz, cz, h->d, h->zigzag, st));
}

void forward_z_impl(mpi_ffl_handle *h, const float *x, float *b, cudaStream_t st) {
    const Dims &d = h->d;
    z_init(h);
    stage_p(h, x, h->w_proj, st);
    zstage_h(h, h->w_proj, h->w_fine_z, st);
    // E_z V_z B fused with S D_Gamma F: the time signal is not stored
    TIMED(MPI_FFL_K_ZDRIVE, launch_zdft_fwd(h->w_fine_z, z_tables(h), h->t_gain, h->t_tw1, h->t_tw2_ro, h->t_dgam, b,
                                            d, h->zigzag, st));
    check_launch(h, "z-drive forward");
}

void adjoint_z_impl(mpi_ffl_handle *h, const float *b, float *x, cudaStream_t st) {
    const Dims &d = h->d;
    z_init(h);
    TIMED(MPI_FFL_K_ZDRIVE, launch_zdft_adj(b, h->t_tw1, h->t_tw2_qr, h->t_dgam, z_tables(h), h->t_gain,
                                            h->w_zcoef, h->w_fine_z, d, h->zigzag, st));
    zstage_ht(h, h->w_fine_z, h->w_proj, st);
    stage_pt(h, h->w_proj, x, st);
    check_launch(h, "z-drive adjoint");
}

extern "C" int mpi_ffl_forward_zdrive(mpi_ffl_handle *h, const float *x, float *b, void *stream) {
    return guarded(h, [&]() {
        if (!x || !b) {
            h->err = "NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        cudaStream_t st = S(stream);
        with_host_buffers(h, x, h->d.nvox, b, h->d.ndata, st,
                          [&](const float *dx, float *db) { forward_z_impl(h, dx, db, st); });
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_adjoint_zdrive(mpi_ffl_handle *h, const float *b, float *x, void *stream) {
    return guarded(h, [&]() {
        if (!x || !b) {
            h->err = "NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        cudaStream_t st = S(stream);
        with_host_buffers(h, b, h->d.ndata, x, h->d.nvox, st,
                          [&](const float *db, float *dx) { adjoint_z_impl(h, db, dx, st); });
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_apply_stage_zdrive(mpi_ffl_handle *h, int32_t stage, int32_t transpose, const float *in,
                                          float *out, void *stream) {
    return guarded(h, [&]() {
        if (!in || !out || (stage != 1 && stage != 2)) {
            h->err = "bad z-drive stage or NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        z_init(h);
        cudaStream_t st = S(stream);
        if (stage == 1) {
            if (transpose) zstage_ht(h, in, out, st);
            else zstage_h(h, in, out, st);
        } else {
            if (transpose) zstage_evt(h, in, out, st);
            else zstage_ev(h, in, out, st);
        }
        check_launch(h, "z-drive stage");
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_set_host_overlap(mpi_ffl_handle *h, int32_t on) {
    if (!h) return MPI_FFL_ERR_INVALID_ARG;
    h->host_overlap = on ? 1 : 0;
    return MPI_FFL_OK;
}

extern "C" int mpi_ffl_apply_stage(mpi_ffl_handle *h, int32_t stage, int32_t transpose, const float *in,
                                   float *out, void *stream) {
    return guarded(h, [&]() {
        if (!in || !out || stage < 0 || stage > 3) {
            h->err = "bad stage or NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        const Dims &d = h->d;
        cudaStream_t st = S(stream);
        switch (stage * 2 + (transpose ? 1 : 0)) {
            case 0: stage_p(h, in, out, st); break;
            case 1: stage_pt(h, in, out, st); break;
            case 2: TIMED(MPI_FFL_K_PSF_FWD, launch_psf_fwd(in, h->t_htab, out, d, st)); break;
            case 3: TIMED(MPI_FFL_K_PSF_ADJ, launch_psf_adj(in, h->t_htab, out, d, st)); break;
            case 4: TIMED(MPI_FFL_K_RESAMPLE_FWD, launch_resample_fwd(in, h->t_traj, h->t_gain, h->t_groups, h->n_groups, out, d, st)); break;
            case 5: TIMED(MPI_FFL_K_RESAMPLE_ADJ, resample_adj(h, in, out, st)); break;
            case 6: TIMED(MPI_FFL_K_DFT_FWD, launch_dft_fwd(in, h->t_tw1, h->t_twp, h->t_tw2_ro, h->t_dgam, out, d, h->w_err, st)); break;
            case 7: TIMED(MPI_FFL_K_DFT_ADJ, launch_dft_adj(in, h->t_tw1, h->t_twp, h->t_tw2_qr, h->t_dgam, out, d, st)); break;
        }
        check_launch(h, "apply_stage");
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_param_grad(mpi_ffl_handle *h, const float *d_x, const float *d_gb, float *d_g_gain,
                                  float *d_g_fwhm, void *stream) {
    return guarded(h, [&]() {
        if (h->psf_model == MPI_FFL_PSF_TENSOR || h->scans != MPI_FFL_SCAN_X) {
            h->err = "parameter gradients are built for the collinear PSF of the x-drive scan only";
            return MPI_FFL_ERR_UNSUPPORTED;
        }
        if (!d_x || !d_gb) {
            h->err = "NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        cudaStream_t st = S(stream);
        stage_p(h, d_x, h->w_proj, st);
        param_grad_impl(h, h->w_proj, d_gb, d_g_gain, d_g_fwhm, st);
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_param_grad_proj(mpi_ffl_handle *h, const float *d_proj, const float *d_gb, float *d_g_gain,
                                       float *d_g_fwhm, void *stream) {
    return guarded(h, [&]() {
        if (h->psf_model == MPI_FFL_PSF_TENSOR || h->scans != MPI_FFL_SCAN_X) {
            h->err = "parameter gradients are built for the collinear PSF of the x-drive scan only";
            return MPI_FFL_ERR_UNSUPPORTED;
        }
        if (!d_proj || !d_gb) {
            h->err = "NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        param_grad_impl(h, d_proj, d_gb, d_g_gain, d_g_fwhm, S(stream));
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_line_forward(mpi_ffl_handle *h, const float *d_proj, float *d_b, void *stream) {
    return guarded(h, [&]() {
        if (!d_proj || !d_b) {
            h->err = "NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        line_forward_impl(h, d_proj, d_b, h->t_htab, h->t_gain, S(stream));
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_line_adjoint(mpi_ffl_handle *h, const float *d_b, float *d_proj, void *stream) {
    return guarded(h, [&]() {
        if (!d_proj || !d_b) {
            h->err = "NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        line_adjoint_impl(h, d_b, d_proj, S(stream));
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_dot_f64(mpi_ffl_handle *h, const float *d_a, const float *d_b, int64_t n, double *d_out,
                               void *stream) {
    return guarded(h, [&]() {
        if (!d_out || n < 0 || (n > 0 && (!d_a || !d_b))) {
            h->err = "bad dot arguments";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        cudaStream_t st = S(stream);
        const int nb = reduce_blocks(n);
        TIMED(MPI_FFL_K_SOLVER, launch_dot(d_a, d_b, n, h->w_red, nb, st));
        TIMED(MPI_FFL_K_SOLVER, launch_finalize(h->w_red, nb, d_out, st));
        check_launch(h, "dot");
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_band_energy(mpi_ffl_handle *h, const float *d_x, double *d_bin_energy, double *d_total,
                                   void *stream) {
    return guarded(h, [&]() {
        if (!d_x || !d_bin_energy || !d_total) {
            h->err = "NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        const Dims &d = h->d;
        cudaStream_t st = S(stream);
        ensure_sig(h);
        if (!h->t_dgam_unit) upload(h, &h->t_dgam_unit, std::vector<float2>(d.nb, make_float2(1.f, 0.f)));
        // s = E V B H P x on the staged kernels (FP32), then its energy and its kept bins
        stage_p(h, d_x, h->w_proj, st);
        TIMED(MPI_FFL_K_PSF_FWD, launch_psf_fwd(h->w_proj, h->t_htab, h->w_fine, d, st));
        TIMED(MPI_FFL_K_RESAMPLE_FWD, launch_resample_fwd(h->w_fine, h->t_traj, h->t_gain, h->t_groups, h->n_groups,
                                                          h->w_sig, d, st));
        const int nbr = reduce_blocks(d.nsig);
        TIMED(MPI_FFL_K_SOLVER, launch_dot(h->w_sig, h->w_sig, d.nsig, h->w_red, nbr, st));
        TIMED(MPI_FFL_K_SOLVER, launch_finalize(h->w_red, nbr, d_total, st));
        TIMED(MPI_FFL_K_DFT_FWD, launch_dft_fwd(h->w_sig, h->t_tw1, h->t_twp, h->t_tw2_ro, h->t_dgam_unit, h->w_data, d, h->w_err, st));
        TIMED(MPI_FFL_K_SOLVER, launch_bin_energy(h->w_data, d.nseg, d.nb, d_bin_energy, st));
        check_launch(h, "band energy");
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_information_retained(mpi_ffl_handle *h, const float *d_x, int32_t n_k, const int32_t *k_max,
                                            int32_t n_w, const int32_t *half_width, double *d_out, void *stream) {
    return guarded(h, [&]() {
        const Dims &d = h->d;
        if (!d_x || !d_out || !k_max || !half_width || n_k < 1 || n_k > 16 || n_w < 1 || n_w > 16) {
            h->err = "NULL buffer or sub-band count outside 1..16";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        for (int i = 0; i < n_k; ++i)
            if (k_max[i] < d.kmin || k_max[i] > d.kmin + d.K - 1) {
                h->err = "harmonic limit outside the kept harmonics";
                return MPI_FFL_ERR_INVALID_ARG;
            }
        for (int i = 0; i < n_w; ++i)
            if (half_width[i] < 0 || half_width[i] > d.hw) {
                h->err = "half-width outside the kept bins";
                return MPI_FFL_ERR_INVALID_ARG;
            }
        if (!h->w_bins) dev_alloc(h, &h->w_bins, (size_t)d.nb + 1);
        const int rc = mpi_ffl_band_energy(h, d_x, h->w_bins, h->w_bins + d.nb, stream);
        if (rc != MPI_FFL_OK) return rc;
        cudaStream_t st = S(stream);
        TIMED(MPI_FFL_K_SOLVER, launch_info_retained(h->w_bins, h->w_bins + d.nb, d.kmin, d.hw, n_k, k_max, n_w,
                                                     half_width, d_out, st));
        check_launch(h, "information retained");
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_apply_ttt(mpi_ffl_handle *h, const float *d_x, float *d_out, void *stream) {
    return guarded(h, [&]() {
        if (!d_x || !d_out) {
            h->err = "NULL buffer";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        cudaStream_t st = S(stream);
        TIMED(MPI_FFL_K_SOLVER, launch_ttt(d_x, d_out, h->d.N, h->d.Nz, st));
        check_launch(h, "ttt");
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_power_norm(mpi_ffl_handle *h, int32_t n_iter, uint64_t seed, double *out, void *stream) {
    return guarded(h, [&]() {
        if (!out || n_iter < 1) {
            h->err = "bad power-iteration arguments";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        *out = power_norm_impl(h, n_iter, seed, S(stream));
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_solve(mpi_ffl_handle *h, const float *d_b, float *d_x, const mpi_ffl_solve_params *p,
                             mpi_ffl_solve_report *rep, void *stream) {
    return guarded(h, [&]() {
        if (!d_b || !d_x || !p || p->iters < 0) {
            h->err = "bad solve arguments";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        const Dims &d = h->d;
        cudaStream_t st = S(stream);
        const double tn = ttt_norm(d);
        double ata = p->ata_norm;
        if ((p->tau <= 0.0 || p->lambda < 0.0) && !(ata > 0.0)) {
            ata = power_norm_impl(h, p->n_power > 0 ? p->n_power : 50, p->seed, st);
        }
        const double lam = p->lambda >= 0.0 ? p->lambda : 1e-3 * ata / tn;
        const double tau = p->tau > 0.0 ? p->tau : 1.0 / (ata + lam * tn);
        if (h->s_hist_len < p->iters + 1) {
            if (h->s_hist) dev_free(h->s_hist);
            h->s_hist = nullptr;
            dev_alloc(h, &h->s_hist, (size_t)p->iters + 1);
            h->s_hist_len = p->iters + 1;
        }
        int *flags = h->s_flags;  // [0] stop flag, [1] iterations done, [2] frozen
        CK(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
        // With a stop rule the host looks at the flags every kPoll iterations only;
        // iterations after the stop are frozen on the device (momentum, residual and
        // update do nothing, the update keeps the final iterate), so the result does
        // not depend on when the host looks.
        constexpr int kPoll = 4;
        const int *frozen = p->stop_rel > 0.0 ? flags + 2 : nullptr;
        CK(cudaMemcpyAsync(h->s_xp, d_x, sizeof(float) * d.nvox, cudaMemcpyDeviceToDevice, st));
        float *xc = d_x, *xp = h->s_xp;
        const int64_t nd = scan_data_len(h);  // data of the selected scans
        const int nbd = reduce_blocks(nd);
        int done_host = 0, k_run = 0;
        for (int k = 1; k <= p->iters; ++k) {
            const double beta = (k - 1.0) / (k + 2.0);
            TIMED(MPI_FFL_K_SOLVER, launch_momentum(xc, xp, h->s_y, beta, k, d.nvox, frozen, st));
            scans_forward(h, h->s_y, h->s_r, st);
            TIMED(MPI_FFL_K_SOLVER, launch_sub_norm(h->s_r, d_b, nd, h->w_red, nbd, frozen, st));
            TIMED(MPI_FFL_K_SOLVER, launch_finalize(h->w_red, nbd, h->s_hist + (k - 1), st));
            TIMED(MPI_FFL_K_SOLVER, launch_stop_check(h->s_hist, k - 1, p->stop_rel, flags, flags + 1, st));
            scans_adjoint(h, h->s_r, h->s_g, st);
            TIMED(MPI_FFL_K_SOLVER, launch_update(h->s_y, h->s_g, xp, (float)tau, (float)lam, p->nonneg ? 1 : 0,
                                                  d.N, d.Nz, frozen, st, xc));
            if (frozen) TIMED(MPI_FFL_K_SOLVER, launch_freeze(flags, flags + 2, st));
            check_launch(h, "solve iteration");
            std::swap(xc, xp);
            k_run = k;
            if (frozen && (k % kPoll == 0 || k == p->iters)) {
                CK(cudaMemcpyAsync(&done_host, flags + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                if (done_host) break;
            }
        }
        if (xc != d_x) CK(cudaMemcpyAsync(d_x, xc, sizeof(float) * d.nvox, cudaMemcpyDeviceToDevice, st));
        if (rep || p->stop_rel > 0.0) {
            int fl[2] = {0, 0};
            CK(cudaMemcpyAsync(fl, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            k_run = fl[1];  // iterations whose update ran (frozen ones excluded)
            double first = 0, last = 0;
            if (k_run > 0) {
                CK(cudaMemcpyAsync(&first, h->s_hist, sizeof(double), cudaMemcpyDeviceToHost, st));
                CK(cudaMemcpyAsync(&last, h->s_hist + (k_run - 1), sizeof(double), cudaMemcpyDeviceToHost, st));
            }
            const double bn = std::sqrt(dot_sync(h, d_b, d_b, nd, st));
            if (rep) {
                rep->iters_done = k_run;
                rep->tau = tau;
                rep->lambda = lam;
                rep->ata_norm = ata;
                rep->residual_first = first;
                rep->residual_last = last;
                rep->b_norm = bn;
            }
            if (fl[0] == 2) {
                h->err = "non-finite residual";
                return MPI_FFL_ERR_NONFINITE;
            }
        }
        return MPI_FFL_OK;
    });
}

extern "C" int mpi_ffl_profile_enable(mpi_ffl_handle *h, int32_t enable) {
    if (!h) return MPI_FFL_ERR_INVALID_ARG;
    h->prof_on = enable ? 1 : 0;
    return MPI_FFL_OK;
}

extern "C" int mpi_ffl_profile_read(mpi_ffl_handle *h, double *ms, int64_t *launches) {
    return guarded(h, [&]() {
        if (!ms || !launches) {
            h->err = "NULL output";
            return MPI_FFL_ERR_INVALID_ARG;
        }
        for (int k = 0; k < MPI_FFL_N_KERNEL_KINDS; ++k) {
            ms[k] = 0.0;
            launches[k] = 0;
        }
        for (auto &r : h->prof_rec) {
            CK(cudaEventSynchronize(r.b));
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, r.a, r.b));
            if (r.kind >= 0 && r.kind < MPI_FFL_N_KERNEL_KINDS) {
                ms[r.kind] += t;
                launches[r.kind] += 1;
            }
            h->ev_pool.push_back(r.a);
            h->ev_pool.push_back(r.b);
        }
        h->prof_rec.clear();
        return MPI_FFL_OK;
    });
}

extern "C" int64_t mpi_ffl_launch_count(const mpi_ffl_handle *h) { return h ? h->launches : -1; }
