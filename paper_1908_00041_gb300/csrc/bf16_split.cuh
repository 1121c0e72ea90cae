// Three-piece bf16 split of FP32 values for the tensor-core operands of the split-precision
// path: hi = rn(v), mid = rn(v - hi), lo = rn(v - hi - mid) (round to nearest even), so
// that hi + mid + lo carries the 24-bit FP32 mantissa.
#pragma once

#include <cuda_bf16.h>

namespace favest {

// 8 floats (one core-matrix row) as three bf16 pieces of 16 bytes, two values per conversion
__device__ __forceinline__ void pack_row3(const float (&v)[8], uint4 (&out)[3])
{
    unsigned w[3][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = make_float2(v[2 * i], v[2 * i + 1]);
        const __nv_bfloat162 h = __float22bfloat162_rn(f);
        const float2 hf = __bfloat1622float2(h);
        const float2 r1 = make_float2(f.x - hf.x, f.y - hf.y);
        const __nv_bfloat162 m = __float22bfloat162_rn(r1);
        const float2 mf = __bfloat1622float2(m);
        const __nv_bfloat162 l = __float22bfloat162_rn(make_float2(r1.x - mf.x, r1.y - mf.y));
        w[0][i] = *reinterpret_cast<const unsigned *>(&h);
        w[1][i] = *reinterpret_cast<const unsigned *>(&m);
        w[2][i] = *reinterpret_cast<const unsigned *>(&l);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) out[q] = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

}  // namespace favest
