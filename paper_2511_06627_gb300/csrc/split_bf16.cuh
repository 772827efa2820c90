// Split of FP32 values into bf16 hi + lo operands for the three-product tensor-core
// GEMMs: hi = bf16(v) rounded to nearest, lo = bf16(v - hi), eight values into one
// 16-byte unit of each (the canonical K-major core-matrix row). Shared by the GEMM's
// packing and the projector's fused packing, so both write the same bits.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace mpiffl {

__device__ __forceinline__ void split8_bf16(const float (&v)[8], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h2 = __float22bfloat162_rn(make_float2(v[2 * i], v[2 * i + 1]));
        const uint32_t hb = *reinterpret_cast<uint32_t *>(&h2);
        const float h0 = __uint_as_float(hb << 16), h1 = __uint_as_float(hb & 0xFFFF0000u);
        __nv_bfloat162 l2 = __float22bfloat162_rn(make_float2(v[2 * i] - h0, v[2 * i + 1] - h1));
        h[i] = hb;
        l[i] = *reinterpret_cast<uint32_t *>(&l2);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

}  // namespace mpiffl
