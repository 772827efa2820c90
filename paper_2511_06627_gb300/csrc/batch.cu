// Continuous batching of reconstructions (the serving form of the solve, Eq. (26)).
//
// A job is one reconstruction: its handle (tables and workspace), its compressed
// data and its solver state (x, x_prev, y, gradient, residual, residual history),
// all resident on the device. mpi_ffl_job_step advances a set of jobs by one
// iteration each, as one launch per kernel kind for all of them: momentum, residual,
// residual norm and stop test, update for every job; x/y transpose, projector, line
// GEMM, adjoint line GEMM and backprojector for the jobs on the full-GEMM path (jobs
// on other paths apply their A and A^T alone between those launches). Each launch is
// persistent: a grid of what the GPU holds at once loops over the work items of every
// job (found through an offset table), so the launch count per iteration does not grow
// with the number of jobs. Jobs that have met their stop test do no further work on
// the device (their update only keeps the final iterate).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "collapsed.h"
#include "internal.h"

using namespace mpiffl;

struct mpi_ffl_job {
    mpi_ffl_handle *h = nullptr;
    float *x = nullptr, *xp = nullptr, *y = nullptr, *g = nullptr, *r = nullptr, *b = nullptr;
    double *hist = nullptr, *partials = nullptr;
    int *flags = nullptr;  // [0] stop verdict, [1] iterations done, [2] frozen (no further work)
    int nblk = 1;
    int k = 1;             // next iteration (1-based)
    int iters = 0;
    double tau = 0, lam = 0, stop_rel = 0;
    int nonneg = 1;
    bool col_angles = false;
    int64_t bytes = 0;
};

namespace mpiffl {
// from api.cu
double power_norm_for_job(mpi_ffl_handle *h, int n_iter, uint64_t seed, cudaStream_t st);
double ttt_norm_for_job(const Dims &d);
bool handle_has_column_angles(const mpi_ffl_handle *h);
void forward_for_job(mpi_ffl_handle *h, const float *x, float *b, cudaStream_t st);
void adjoint_for_job(mpi_ffl_handle *h, const float *b, float *x, cudaStream_t st);
}  // namespace mpiffl

namespace {

// per-step staging of the batched launches' arguments
struct Staging {
    size_t cap = 0;
    uint8_t *host[2] = {nullptr, nullptr};
    uint8_t *dev[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int which = 0;
    int dev_id = -1;
};
thread_local Staging g_stage;

bool staging_ready(size_t need) {
    int dev = 0;
    cudaGetDevice(&dev);
    Staging &s = g_stage;
    if (s.cap >= need && s.dev_id == dev) return true;
    for (int i = 0; i < 2; ++i) {
        if (s.ev[i]) cudaEventSynchronize(s.ev[i]);
        if (s.host[i]) cudaFreeHost(s.host[i]);
        if (s.dev[i]) dev_free(s.dev[i]);
        if (s.ev[i]) cudaEventDestroy(s.ev[i]);
        s.host[i] = s.dev[i] = nullptr;
        s.ev[i] = nullptr;
    }
    s.cap = std::max<size_t>(need, 1 << 20);
    for (int i = 0; i < 2; ++i) {
        if (cudaMallocHost((void **)&s.host[i], s.cap) != cudaSuccess) return false;
        if (dev_malloc((void **)&s.dev[i], s.cap) != cudaSuccess) return false;
        if (cudaEventCreateWithFlags(&s.ev[i], cudaEventDisableTiming) != cudaSuccess) return false;
    }
    s.dev_id = dev;
    col_batch_init();
    return true;
}

template <class T>
size_t put(std::vector<uint8_t> &buf, const T *p, size_t n) {
    const size_t off = (buf.size() + 15) / 16 * 16;
    buf.resize(off + n * sizeof(T));
    if (n) std::memcpy(buf.data() + off, p, n * sizeof(T));
    return off;
}

template <class T>
size_t put(std::vector<uint8_t> &buf, const std::vector<T> &v) {
    return put(buf, v.data(), v.size());
}

void free_job(mpi_ffl_job *j) {
    void *ptrs[] = {j->x, j->xp, j->y, j->g, j->r, j->b, j->hist, j->partials, j->flags};
    for (void *p : ptrs)
        if (p) dev_free(p);
}

}  // namespace

extern "C" int mpi_ffl_job_create(mpi_ffl_handle *h, const float *d_b, const float *d_x0,
                                  const mpi_ffl_solve_params *p, mpi_ffl_job **out, void *stream) {
    if (!h || !d_b || !p || !out || p->iters < 1) return MPI_FFL_ERR_INVALID_ARG;
    *out = nullptr;
    if (h->scans != MPI_FFL_SCAN_X) {  // jobs reconstruct from the x-drive scan
        h->err = "jobs use the x-drive scan only (mpi_ffl_set_scans)";
        return MPI_FFL_ERR_UNSUPPORTED;
    }
    mpi_ffl_job *j = new (std::nothrow) mpi_ffl_job();
    if (!j) return MPI_FFL_ERR_OOM;
    const Dims &d = h->d;
    cudaStream_t st = (cudaStream_t)stream;
    j->h = h;
    j->iters = p->iters;
    j->nonneg = p->nonneg ? 1 : 0;
    j->stop_rel = p->stop_rel;
    j->nblk = std::max(1, std::min(1024, (int)((d.ndata + 4095) / 4096)));
    j->col_angles = handle_has_column_angles(h);
    auto alloc = [&](void **ptr, size_t bytes) {
        if (dev_malloc(ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        j->bytes += (int64_t)bytes;
        return true;
    };
    const size_t vb = sizeof(float) * d.nvox, db = sizeof(float) * d.ndata;
    if (!alloc((void **)&j->x, vb) || !alloc((void **)&j->xp, vb) || !alloc((void **)&j->y, vb) ||
        !alloc((void **)&j->g, vb) || !alloc((void **)&j->r, db) || !alloc((void **)&j->b, db) ||
        !alloc((void **)&j->hist, sizeof(double) * (p->iters + 1)) ||
        !alloc((void **)&j->partials, sizeof(double) * j->nblk) || !alloc((void **)&j->flags, 4 * sizeof(int))) {
        free_job(j);
        delete j;
        h->err = "job allocation failed";
        return MPI_FFL_ERR_OOM;
    }
    cudaMemcpyAsync(j->b, d_b, db, cudaMemcpyDeviceToDevice, st);
    if (d_x0) cudaMemcpyAsync(j->x, d_x0, vb, cudaMemcpyDeviceToDevice, st);
    else cudaMemsetAsync(j->x, 0, vb, st);
    cudaMemcpyAsync(j->xp, j->x, vb, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(j->flags, 0, 4 * sizeof(int), st);
    const double tn = ttt_norm_for_job(d);
    double ata = p->ata_norm;
    if ((p->tau <= 0.0 || p->lambda < 0.0) && !(ata > 0.0))
        ata = power_norm_for_job(h, p->n_power > 0 ? p->n_power : 50, p->seed, st);
    j->lam = p->lambda >= 0.0 ? p->lambda : 1e-3 * ata / tn;
    j->tau = p->tau > 0.0 ? p->tau : 1.0 / (ata + j->lam * tn);
    if (cudaGetLastError() != cudaSuccess) {
        free_job(j);
        delete j;
        h->err = "job setup failed";
        return MPI_FFL_ERR_CUDA;
    }
    *out = j;
    return MPI_FFL_OK;
}

extern "C" int mpi_ffl_job_destroy(mpi_ffl_job *j) {
    if (!j) return MPI_FFL_OK;
    cudaDeviceSynchronize();
    free_job(j);
    delete j;
    return MPI_FFL_OK;
}

extern "C" int mpi_ffl_job_step(mpi_ffl_job *const *jobs, int32_t n, void *stream) {
    if (n < 0 || (n > 0 && !jobs)) return MPI_FFL_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<mpi_ffl_job *> all, batch, single;
    for (int i = 0; i < n; ++i) {
        mpi_ffl_job *j = jobs[i];
        if (!j) return MPI_FFL_ERR_INVALID_ARG;
        if (j->k > j->iters) continue;  // iteration budget used up
        all.push_back(j);
        if (j->h->path == MPI_FFL_PATH_FULL_GEMM && col_supported(j->h) && project_batch_ok(j->h->d.N) &&
            j->h->psf_model == MPI_FFL_PSF_COLLINEAR && !j->h->t_coil)
            batch.push_back(j);
        else single.push_back(j);
    }
    const int na = (int)all.size(), nb = (int)batch.size();
    if (na == 0) return MPI_FFL_OK;

    // ---------------------------------------------------------------- staging
    std::vector<uint8_t> buf;
    std::vector<MomentumJob> mom(na);
    std::vector<ResidualJob> rs(na);
    std::vector<StopJob> sp(na);
    std::vector<UpdateJob> up(na);
    std::vector<int> off_m(na + 1, 0), off_r(na + 1, 0), off_u(na + 1, 0);
    for (int i = 0; i < na; ++i) {
        mpi_ffl_job *j = all[i];
        const Dims &d = j->h->d;
        const int *done = j->flags + 2;
        mom[i] = MomentumJob{j->x, j->xp, j->y, (float)((j->k - 1.0) / (j->k + 2.0)), d.nvox, done};
        off_m[i + 1] = off_m[i] + (int)((d.nvox + 2047) / 2048);
        rs[i] = ResidualJob{j->r, j->b, d.ndata, j->partials, j->nblk, done};
        off_r[i + 1] = off_r[i] + j->nblk;
        sp[i] = StopJob{j->partials, j->nblk, j->hist, j->k - 1, j->stop_rel, j->flags, j->flags + 2};
        up[i] = UpdateJob{j->y, j->g, j->xp, j->x, (float)j->tau, (float)j->lam, j->nonneg, d.N, d.Nz, done};
        off_u[i + 1] = off_u[i] + update_blocks(d.N, d.Nz);
    }
    std::vector<TransposeJob> tr;
    std::vector<ProjectJob> pj(nb);
    std::vector<BackprojectJob> bp(nb);
    std::vector<int> off_t(1, 0), off_p(nb + 1, 0), off_b(nb + 1, 0);
    std::vector<mpi_ffl_handle *> hs(nb);
    std::vector<const float *> gin_f(nb), gin_a(nb);
    std::vector<float *> gout_f(nb), gout_a(nb);
    std::vector<const int *> dn(nb);
    int maxN = 0;
    for (int i = 0; i < nb; ++i) {
        mpi_ffl_job *j = batch[i];
        mpi_ffl_handle *h = j->h;
        const Dims &d = h->d;
        const int *done = j->flags + 2;
        dn[i] = done;
        hs[i] = h;
        maxN = std::max(maxN, d.N);
        if (j->col_angles) {
            tr.push_back(TransposeJob{j->y, h->w_volT, d.N, d.Nz, done});
            off_t.push_back(off_t.back() + transpose_blocks(d.N, d.Nz));
        }
        pj[i] = ProjectJob{j->y, h->w_volT, h->t_ang, h->t_agroups, h->w_proj, d.N, d.Nz, h->n_agroups, done};
        off_p[i + 1] = off_p[i] + project_blocks(h->n_agroups, d.Nz);
        gin_f[i] = h->w_proj;
        gout_f[i] = j->r;
        gin_a[i] = j->r;
        gout_a[i] = h->w_proj;
        bp[i] = BackprojectJob{h->w_proj, h->t_ang, j->g, d.N, d.Nz, d.M, done};
        off_b[i + 1] = off_b[i] + backproject_blocks(d.N, d.Nz);
    }
    const int arg_cap = 2 * std::max(nb, 1);
    const int item_cap = 65536;
    std::vector<uint8_t> gf(gemm_args_size() * arg_cap), ga(gemm_args_size() * arg_cap);
    std::vector<int4> itf(item_cap), ita(item_cap);
    int nif = 0, nia = 0, npf = 0, npa = 0;
    size_t smf = 0, sma = 0;
    uint32_t tcf = 32, tca = 32;
    if (nb > 0) {
        npf = col_batch_prepare(hs.data(), gin_f.data(), gout_f.data(), dn.data(), nb, false, gf.data(), itf.data(),
                                arg_cap, item_cap, nif, smf, tcf);
        npa = col_batch_prepare(hs.data(), gin_a.data(), gout_a.data(), dn.data(), nb, true, ga.data(), ita.data(),
                                arg_cap, item_cap, nia, sma, tca);
        if (npf < 0 || npa < 0) return MPI_FFL_ERR_UNSUPPORTED;
    }
    const size_t o_mom = put(buf, mom), o_offm = put(buf, off_m);
    const size_t o_rs = put(buf, rs), o_offr = put(buf, off_r);
    const size_t o_sp = put(buf, sp);
    const size_t o_up = put(buf, up), o_offu = put(buf, off_u);
    const size_t o_tr = put(buf, tr), o_offt = put(buf, off_t);
    const size_t o_pj = put(buf, pj), o_offp = put(buf, off_p);
    const size_t o_gf = put(buf, gf.data(), gemm_args_size() * npf), o_itf = put(buf, itf.data(), nif);
    const size_t o_ga = put(buf, ga.data(), gemm_args_size() * npa), o_ita = put(buf, ita.data(), nia);
    const size_t o_bp = put(buf, bp), o_offb = put(buf, off_b);
    if (!staging_ready(buf.size())) return MPI_FFL_ERR_OOM;
    Staging &S = g_stage;
    const int w = S.which;
    S.which ^= 1;
    cudaEventSynchronize(S.ev[w]);  // the previous use of this staging buffer has been copied
    std::memcpy(S.host[w], buf.data(), buf.size());
    cudaMemcpyAsync(S.dev[w], S.host[w], buf.size(), cudaMemcpyHostToDevice, st);
    cudaEventRecord(S.ev[w], st);
    uint8_t *D = S.dev[w];
    auto at = [&](size_t o) { return (void *)(D + o); };

    // ---------------------------------------------------------------- one iteration, every job
    launch_momentum_batch((const MomentumJob *)at(o_mom), (const int *)at(o_offm), na, off_m[na], st);
    if (nb > 0) {
        if (!tr.empty())
            launch_transpose_batch((const TransposeJob *)at(o_tr), (const int *)at(o_offt), (int)tr.size(),
                                   off_t.back(), st);
        launch_project_batch((const ProjectJob *)at(o_pj), (const int *)at(o_offp), nb, off_p[nb], maxN,
                             batch[0]->h->w_err, st);
        col_batch_launch(at(o_gf), (const int4 *)at(o_itf), nif, smf, tcf, st);
    }
    for (mpi_ffl_job *j : single) forward_for_job(j->h, j->y, j->r, st);
    launch_residual_batch((const ResidualJob *)at(o_rs), (const int *)at(o_offr), na, off_r[na], st);
    launch_stop_batch((const StopJob *)at(o_sp), na, st);
    if (nb > 0) {
        col_batch_launch(at(o_ga), (const int4 *)at(o_ita), nia, sma, tca, st);
        launch_backproject_batch((const BackprojectJob *)at(o_bp), (const int *)at(o_offb), nb, off_b[nb], st);
    }
    for (mpi_ffl_job *j : single) adjoint_for_job(j->h, j->r, j->g, st);
    launch_update_batch((const UpdateJob *)at(o_up), (const int *)at(o_offu), na, off_u[na], st);
    launch_freeze_batch((const StopJob *)at(o_sp), na, st);
    for (mpi_ffl_job *j : all) {
        std::swap(j->x, j->xp);
        ++j->k;
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPI_FFL_OK : MPI_FFL_ERR_CUDA;
}

extern "C" int mpi_ffl_job_status(const mpi_ffl_job *j, mpi_ffl_job_status_t *out, void *stream) {
    if (!j || !out) return MPI_FFL_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int fl[3] = {0, 0, 0};
    cudaMemcpyAsync(fl, j->flags, 3 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return MPI_FFL_ERR_CUDA;
    out->iters_done = fl[1];
    out->stopped = fl[0];
    out->finished = (fl[2] != 0 || fl[1] >= j->iters) ? 1 : 0;
    out->residual_first = out->residual_last = 0.0;
    if (fl[1] > 0) {
        cudaMemcpy(&out->residual_first, j->hist, sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(&out->residual_last, j->hist + (fl[1] - 1), sizeof(double), cudaMemcpyDeviceToHost);
    }
    out->tau = j->tau;
    out->lambda = j->lam;
    out->device_bytes = j->bytes;
    return fl[0] == 2 ? MPI_FFL_ERR_NONFINITE : MPI_FFL_OK;
}

extern "C" int mpi_ffl_job_flags(const mpi_ffl_job *j, const int32_t **d_flags) {
    if (!j || !d_flags) return MPI_FFL_ERR_INVALID_ARG;
    *d_flags = j->flags;
    return MPI_FFL_OK;
}

extern "C" int mpi_ffl_job_poll(mpi_ffl_job *const *jobs, int32_t n, int32_t *host_flags, void *stream) {
    if (n < 0 || (n > 0 && (!jobs || !host_flags))) return MPI_FFL_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!jobs[i]) return MPI_FFL_ERR_INVALID_ARG;
        if (cudaMemcpyAsync(host_flags + 3 * i, jobs[i]->flags, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                            (cudaStream_t)stream) != cudaSuccess)
            return MPI_FFL_ERR_CUDA;
    }
    return MPI_FFL_OK;
}

extern "C" int mpi_ffl_job_result(const mpi_ffl_job *j, float *d_x, void *stream) {
    if (!j || !d_x) return MPI_FFL_ERR_INVALID_ARG;
    const cudaError_t e = cudaMemcpyAsync(d_x, j->x, sizeof(float) * j->h->d.nvox, cudaMemcpyDeviceToDevice,
                                          (cudaStream_t)stream);
    return e == cudaSuccess ? MPI_FFL_OK : MPI_FFL_ERR_CUDA;
}
