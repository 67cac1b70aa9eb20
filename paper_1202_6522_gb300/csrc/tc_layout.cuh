// tc_layout.cuh -- the blocked bf16 hi/lo operand layout of the tensor-core
// Legendre contraction (tc.cu).
//
// A block is [rows x kKc] bf16 values, K-major without swizzle: 8-row x
// 16-byte core matrices, kLbo bytes between K-adjacent core matrices, kSbo
// bytes between 8-row groups.  A data chunk is [class][hi|lo] blocks, where
// class is the parity of n - m (synthesis) or the fold s / d (analysis).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace sht {

constexpr int kKc = 16;                     // K per chunk: one MMA K step
constexpr uint32_t kSbo = (kKc / 8) * 128;  // 8-row group stride in a [rows x kKc] block
constexpr uint32_t kLbo = 128;              // K-adjacent core matrices

// byte offset of element (row, k) in a K-major [rows x kKc] bf16 block
__host__ __device__ __forceinline__ uint32_t blk_off(int row, int k)
{
    return (uint32_t)((row >> 3) * kSbo + (k >> 3) * kLbo + (row & 7) * 16 + (k & 7) * 2);
}

// bytes of one data chunk of `rows` rows: [2 classes][hi|lo] blocks
__host__ __device__ inline size_t data_chunk_bytes(int rows) { return 4 * (size_t)rows * kKc * 2; }

// v = hi + lo with hi = bf16(v), lo = bf16(v - hi)
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// v0, v1 -> bf16x2 hi and lo words (v0 in the low half) with v = hi + lo per element
__device__ __forceinline__ void split2(float v0, float v1, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

}  // namespace sht
