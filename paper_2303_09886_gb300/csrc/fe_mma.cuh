// Warp-level tensor-core helpers of the reduced-precision forms:
// mma.sync m16n8k16 with FP16 or BF16 operands and FP32 accumulation, and
// the operand packing they use (PREC 1 = FP16, PREC 2 = BF16).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace fe {

template <int PREC>
__device__ __forceinline__ unsigned pack2(float lo, float hi) {
    if constexpr (PREC == 1) {
        const __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const unsigned *>(&h);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const unsigned *>(&h);
    }
}

// x rounded to the operand type (round to nearest even); x - prec_round(x)
// is the remainder that a second, "lo" operand carries.
template <int PREC>
__device__ __forceinline__ float prec_round(float x) {
    if constexpr (PREC == 1) return __half2float(__float2half_rn(x));
    else return __bfloat162float(__float2bfloat16_rn(x));
}

template <int PREC>
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    if constexpr (PREC == 1) {
        asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                     "{%8,%9}, {%0,%1,%2,%3};"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                     "{%8,%9}, {%0,%1,%2,%3};"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

template <int PREC>
__device__ __forceinline__ void mma16816(float (&d)[4], uint4 a, unsigned b0, unsigned b1) {
    const unsigned r[4] = {a.x, a.y, a.z, a.w};
    mma16816<PREC>(d, r, b0, b1);
}

}  // namespace fe
