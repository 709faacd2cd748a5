// sfft_measure.cu -- a measurement kernel (no part of the transform): the rate at which this device
// serves a given list of sample reads, so that a gather can be compared with the same reads issued
// by a kernel that does nothing else (sfft_gather_rate in include/sfft.h).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sfft.h"
#include "sfft_internal.h"

namespace sfft {

// Row r of d_x holds row_elems complex64 values; CTA (r, chunk) reads d_x[r][idx[r][i]] for the
// kRatePerCta entries i of its chunk, 16 loads in flight per thread, through L2 only (one 32-byte
// sector per read, as the transform's gathers), and folds them into one word so that no load is
// dead code.
constexpr uint32_t kRateInFlight = 16;
constexpr uint32_t kRatePerCta = kThreads * kRateInFlight;
__global__ void __launch_bounds__(kThreads) k_gather_rate(const float2* __restrict__ x, uint64_t row_elems,
                                                         const uint32_t* __restrict__ idx, uint32_t per_row,
                                                         uint32_t chunks, uint32_t* __restrict__ sink) {
    const uint32_t r = blockIdx.x / chunks, c = blockIdx.x % chunks;
    const float2* xr = x + (size_t)r * row_elems;
    const uint32_t* ir = idx + (size_t)r * per_row;
    const uint32_t i0 = c * kRatePerCta, i1 = min(i0 + kRatePerCta, per_row);
    const uint32_t mask = (uint32_t)(row_elems - 1);
    uint32_t acc = 0;
    uint32_t ii[kRateInFlight];
#pragma unroll
    for (uint32_t q = 0; q < kRateInFlight; ++q) {
        const uint32_t i = i0 + threadIdx.x + q * kThreads;
        ii[q] = i < i1 ? __ldg(ir + i) & mask : 0xFFFFFFFFu;
    }
    float2 v[kRateInFlight];
#pragma unroll
    for (uint32_t q = 0; q < kRateInFlight; ++q)
        v[q] = ii[q] != 0xFFFFFFFFu ? __ldcg(xr + ii[q]) : make_float2(0.0f, 0.0f);
#pragma unroll
    for (uint32_t q = 0; q < kRateInFlight; ++q) acc ^= __float_as_uint(v[q].x) ^ __float_as_uint(v[q].y);
    acc = __reduce_xor_sync(0xFFFFFFFFu, acc);
    if ((threadIdx.x & 31u) == 0) atomicXor(sink + (blockIdx.x & 63u), acc);
}

}  // namespace sfft

extern "C" sfft_status sfft_gather_rate(const void* d_x, uint64_t row_elems, uint32_t rows, const uint32_t* d_idx,
                                        uint32_t per_row, uint32_t* d_sink, void* stream) {
    if (!d_x || !d_idx || !d_sink || rows == 0 || per_row == 0) return SFFT_ERR_INVALID_ARG;
    if (row_elems < 2 || (row_elems & (row_elems - 1)) || row_elems > (1ull << 31)) return SFFT_ERR_INVALID_ARG;
    const uint32_t chunks = (per_row + sfft::kRatePerCta - 1) / sfft::kRatePerCta;
    const uint64_t blocks = (uint64_t)rows * chunks;
    if (blocks > 0x7FFFFFFFull) return SFFT_ERR_INVALID_ARG;
    sfft::k_gather_rate<<<(uint32_t)blocks, sfft::kThreads, 0, (cudaStream_t)stream>>>(
        static_cast<const float2*>(d_x), row_elems, d_idx, per_row, chunks, d_sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        sfft::set_last_error(std::string("gather rate: ") + cudaGetErrorString(e));
        return SFFT_ERR_CUDA;
    }
    return SFFT_OK;
}
