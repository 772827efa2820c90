// Detection-limit analysis of a reconstruction (Sec. 4.2, Fig. 5): FP64 statistics of
// boxes of a volume on the GPU, and the least-squares crossing of the sample values
// with three times the background noise on the host.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace mpiffl {

// Information retained by sub-bands of the kept bins (Appendix A, Eq. (30)): thread t =
// (harmonic limit a, half-width c) sums, in a fixed order, the per-bin energies of the
// bins with harmonics k_min..hk[a] and |delta| <= hw[c] (each bin counted with its
// conjugate, which carries the same energy for a real signal) and writes
// sqrt(2 sum / total), 0 for a zero total.
struct InfoBands {
    int n_k, n_w;
    int hk[16], hw[16];
};

__global__ void k_info_retained(const double *__restrict__ bin_energy, const double *__restrict__ total, int kmin,
                                int w_all, InfoBands B, double *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B.n_k * B.n_w) return;
    const int a = t / B.n_w, c = t - a * B.n_w;
    const int W = 2 * w_all + 1;
    double sub = 0.0;
    for (int k = 0; k <= B.hk[a] - kmin; ++k)
        for (int dd = -B.hw[c]; dd <= B.hw[c]; ++dd) sub += bin_energy[k * W + w_all + dd];
    const double tot = *total;
    out[t] = tot > 0.0 ? sqrt(2.0 * sub / tot) : 0.0;
}

void launch_info_retained(const double *bin_energy, const double *total, int kmin, int w_all, int n_k,
                          const int *hk, int n_w, const int *hw, double *out, cudaStream_t st) {
    InfoBands B{};
    B.n_k = n_k;
    B.n_w = n_w;
    for (int i = 0; i < n_k; ++i) B.hk[i] = hk[i];
    for (int i = 0; i < n_w; ++i) B.hw[i] = hw[i];
    k_info_retained<<<(n_k * n_w + 127) / 128, 128, 0, st>>>(bin_energy, total, kmin, w_all, B, out);
}

// Block per box: over the box's voxels, part[b] = (count, sum, max) when pass == 0,
// (count, sum |v - mean[g[b]]|, max) when pass == 1. Each thread visits a fixed set of
// voxels and the block reduces in a fixed order: the sums are reproducible.
__global__ void __launch_bounds__(256) k_box_stats(const float *__restrict__ vol, int ny, int nx,
                                                   const int *__restrict__ boxes, const int *__restrict__ group,
                                                   const double *__restrict__ mean, int pass,
                                                   double *__restrict__ part) {
    const int b = blockIdx.x;
    const int z0 = boxes[6 * b], z1 = boxes[6 * b + 1], y0 = boxes[6 * b + 2], y1 = boxes[6 * b + 3];
    const int x0 = boxes[6 * b + 4], x1 = boxes[6 * b + 5];
    const int wx = x1 - x0, wy = y1 - y0;
    const long long n = (long long)(z1 - z0) * wy * wx;
    const double mu = pass ? mean[group[b]] : 0.0;
    double s = 0.0, mx = -INFINITY;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) {
        const int x = x0 + (int)(t % wx);
        const long long r = t / wx;
        const int y = y0 + (int)(r % wy), z = z0 + (int)(r / wy);
        const double v = vol[((size_t)z * ny + y) * nx + x];
        s += pass ? fabs(v - mu) : v;
        mx = fmax(mx, v);
    }
    __shared__ double ss[8], sm[8];
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        ss[w] = s;
        sm[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, m = -INFINITY;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += ss[k];
            m = fmax(m, sm[k]);
        }
        part[3 * b] = (double)n;
        part[3 * b + 1] = a;
        part[3 * b + 2] = m;
    }
}

}  // namespace mpiffl

namespace {

int set_analysis_error(const char *msg) {
    mpiffl::set_thread_error(msg);
    return MPI_FFL_ERR_INVALID_ARG;
}

}  // namespace

extern "C" int mpi_ffl_box_stats(const float *d_vol, int32_t nz, int32_t ny, int32_t nx, const int32_t *boxes,
                                 int32_t n_boxes, int32_t pooled, double *out, void *stream) {
    using namespace mpiffl;
    if (!d_vol || !boxes || !out || n_boxes <= 0 || nz <= 0 || ny <= 0 || nx <= 0)
        return set_analysis_error("box_stats: NULL buffer or empty volume / box list");
    for (int b = 0; b < n_boxes; ++b) {
        const int32_t *q = boxes + 6 * b;
        if (q[0] < 0 || q[1] > nz || q[2] < 0 || q[3] > ny || q[4] < 0 || q[5] > nx || q[0] >= q[1] || q[2] >= q[3] ||
            q[4] >= q[5])
            return set_analysis_error("box_stats: a box is empty or leaves the volume");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ng = pooled ? 1 : n_boxes;
    std::vector<int> grp(n_boxes);
    for (int b = 0; b < n_boxes; ++b) grp[b] = pooled ? 0 : b;
    int *d_boxes = nullptr, *d_grp = nullptr;
    double *d_mean = nullptr, *d_part = nullptr;
    auto release = [&]() {
        for (void *p : {(void *)d_boxes, (void *)d_grp, (void *)d_mean, (void *)d_part})
            if (p) dev_free(p);
    };
    if (dev_malloc((void **)&d_boxes, sizeof(int) * 6 * n_boxes) != cudaSuccess ||
        dev_malloc((void **)&d_grp, sizeof(int) * n_boxes) != cudaSuccess ||
        dev_malloc((void **)&d_mean, sizeof(double) * ng) != cudaSuccess ||
        dev_malloc((void **)&d_part, sizeof(double) * 3 * n_boxes) != cudaSuccess) {
        release();
        cudaGetLastError();
        mpiffl::set_thread_error("box_stats: device allocation failed");
        return MPI_FFL_ERR_OOM;
    }
    std::vector<double> part(3 * (size_t)n_boxes), cnt(ng, 0.0), sum(ng, 0.0), mx(ng, -INFINITY), dev(ng, 0.0),
        mean(ng, 0.0);
    bool ok = cudaMemcpyAsync(d_boxes, boxes, sizeof(int) * 6 * n_boxes, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(d_grp, grp.data(), sizeof(int) * n_boxes, cudaMemcpyHostToDevice, st) == cudaSuccess;
    for (int pass = 0; ok && pass < 2; ++pass) {
        k_box_stats<<<n_boxes, 256, 0, st>>>(d_vol, ny, nx, d_boxes, d_grp, d_mean, pass, d_part);
        ok = cudaMemcpyAsync(part.data(), d_part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st) ==
                 cudaSuccess &&
             cudaStreamSynchronize(st) == cudaSuccess;
        if (!ok) break;
        for (int b = 0; b < n_boxes; ++b) {  // groups in box order: a fixed order
            const int g = grp[b];
            if (pass == 0) {
                cnt[g] += part[3 * b];
                sum[g] += part[3 * b + 1];
                mx[g] = std::fmax(mx[g], part[3 * b + 2]);
            } else {
                dev[g] += part[3 * b + 1];
            }
        }
        if (pass == 0) {
            for (int g = 0; g < ng; ++g) mean[g] = sum[g] / cnt[g];
            ok = cudaMemcpyAsync(d_mean, mean.data(), sizeof(double) * ng, cudaMemcpyHostToDevice, st) == cudaSuccess;
        }
    }
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    release();
    if (!ok) {
        cudaGetLastError();
        mpiffl::set_thread_error("box_stats: a CUDA call failed");
        return MPI_FFL_ERR_CUDA;
    }
    for (int g = 0; g < ng; ++g) {
        out[4 * g] = cnt[g];
        out[4 * g + 1] = mean[g];
        out[4 * g + 2] = dev[g] / cnt[g];
        out[4 * g + 3] = mx[g];
    }
    return MPI_FFL_OK;
}

extern "C" int mpi_ffl_detection_limit(const double *amounts, const double *values, int32_t n, double noise, double k,
                                       double *out) {
    if (!amounts || !values || !out || n < 2) return set_analysis_error("detection_limit: need two or more samples");
    double xm = 0.0, ym = 0.0;
    for (int i = 0; i < n; ++i) {
        xm += amounts[i];
        ym += values[i];
    }
    xm /= n;
    ym /= n;
    double sxx = 0.0, sxy = 0.0;
    for (int i = 0; i < n; ++i) {
        sxx += (amounts[i] - xm) * (amounts[i] - xm);
        sxy += (amounts[i] - xm) * (values[i] - ym);
    }
    if (!(sxx > 0.0)) return set_analysis_error("detection_limit: the amounts are all equal");
    const double s = sxy / sxx, a = ym - s * xm;
    out[0] = s > 0.0 ? (k * noise - a) / s : NAN;
    out[1] = s;
    out[2] = a;
    return MPI_FFL_OK;
}
