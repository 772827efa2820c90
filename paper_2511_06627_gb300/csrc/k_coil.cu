// Receive-coil weighting (operator B of Eq. (13) with a spatial sensitivity map) and
// row padding for the tensor-PSF GEMMs.
#include "internal.h"

#include <algorithm>

namespace mpiffl {

// out[r'][c] = b[r mod Nz][c] sum_p in[p][r][c] for c < ncols (nparts partial sums
// part_stride floats apart, added in order), 0 for ncols <= c < stride (b NULL: a
// uniform coil). rows = M Nz rows of one projection or data set; output row
// r' = (r / Nz) zp + p0 + r mod Nz places each angle's Nz rows after p0 rows of a
// block of zp (zp = Nz, p0 = 0: the same layout). in and out may be the same buffer
// when nparts == 1, stride == ncols and the layouts agree.
__global__ void __launch_bounds__(256) k_coil_pad(const float *__restrict__ in, int nparts, long long part_stride,
                                                  const float *__restrict__ coil, float *__restrict__ out,
                                                  long long rows, int Nz, int ncols, int stride, int zp, int p0) {
    const long long total = rows * stride;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / stride;
        const int c = (int)(t - r * stride);
        float v = 0.f;
        if (c < ncols) {
            const long long k = r * ncols + c;
            v = in[k];
            for (int p = 1; p < nparts; ++p) v += in[p * part_stride + k];
            if (coil) v *= __ldg(coil + (size_t)(r % Nz) * ncols + c);
        }
        const long long ro = (r / Nz) * zp + p0 + r % Nz;
        out[ro * stride + c] = v;
    }
}

void launch_coil_pad(const float *in, const float *coil, float *out, long long rows, int Nz, int ncols, int stride,
                     cudaStream_t st, int nparts, long long part_stride, int zp, int p0) {
    const long long total = rows * stride;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    k_coil_pad<<<std::max(1, blocks), 256, 0, st>>>(in, nparts, part_stride, coil, out, rows, Nz, ncols, stride,
                                                    zp > 0 ? zp : Nz, p0);
}

}  // namespace mpiffl
