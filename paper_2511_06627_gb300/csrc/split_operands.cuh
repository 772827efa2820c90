// Split of FP32 values into hi + lo operands for the three-product tensor-core GEMMs,
// one 16-byte unit of each (the canonical K-major core-matrix row): bf16, eight values,
// hi = bf16(v) rounded to nearest, lo = bf16(v - hi); tf32, four values, hi = tf32(v)
// and lo = tf32(v - hi), rounded to nearest with ties away. Shared by the GEMM's
// producers and packing pass and the projector's fused packing, so all write the same
// bits.
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

__device__ __forceinline__ uint32_t to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ void split4_tf32(const float (&v)[4], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i] = to_tf32(v[i]);
        l[i] = to_tf32(v[i] - __uint_as_float(h[i]));
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

}  // namespace mpiffl
