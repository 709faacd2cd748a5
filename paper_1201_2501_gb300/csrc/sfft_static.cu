// sfft_static.cu -- sfft_hash_to_bins_static: HashToBins for callers that cannot allocate device
// memory (see include/sfft.h).  It launches the same round kernel as sfft_hash_to_bins in its
// single-hashing mode; only the scratch differs: instead of a plan's workspace, the partial fold
// sums and the arrival counter live in a fixed array compiled into this library.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "sfft_internal.h"

namespace {

// Bytes [0, 256) hold the arrival counter; the partial folds start at byte 256.  Every device that
// loads the library holds this array until the process exits.
__device__ __align__(256) unsigned char g_sfft_static_scratch[SFFT_STATIC_SCRATCH_BYTES];
constexpr size_t kCounterBytes = 256;
constexpr int kMaxDevices = 64;

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device ordinal

bool pow2(uint64_t v) { return v && !(v & (v - 1)); }

// In host code g_sfft_static_scratch names a host-side stand-in, not device memory: the device
// address comes from cudaGetSymbolAddress, looked up once per device with that device current.
sfft_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        sfft::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return SFFT_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return SFFT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sfft_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            sfft::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return SFFT_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SFFT_OK;
}

}  // namespace

extern "C" sfft_status sfft_hash_to_bins_static(uint64_t n, uint32_t B, int64_t T, const float* d_taps,
                                                const double* d_wtab, const void* d_x, uint64_t sigma, uint64_t a,
                                                uint64_t b, const uint32_t* d_zidx, const double* d_zval, uint32_t nz,
                                                double* d_u, void* stream) {
    using namespace sfft;
    if (!d_taps || !d_x || !d_u) return SFFT_ERR_INVALID_ARG;
    if (!pow2(n) || n < 64 || n > (uint64_t(1) << 30)) return SFFT_ERR_N_NOT_POW2;
    if (!pow2(B) || B < 2 || (uint64_t)B > n / 2 || B > kMaxB) return SFFT_ERR_INVALID_ARG;
    if (T < 0 || T > (int64_t(1) << 28)) return SFFT_ERR_INVALID_ARG;
    if (!(sigma & 1) || sigma >= n || a >= n || b >= n) return SFFT_ERR_INVALID_ARG;
    if (nz > 4096 || (nz > 0 && (!d_zidx || !d_zval || !d_wtab))) return SFFT_ERR_INVALID_ARG;
    const uint64_t chunks = (2 * (uint64_t)T + 1 + kChunkTaps - 1) / kChunkTaps;
    const uint64_t need = kCounterBytes + chunks * (uint64_t)B * sizeof(float2);
    if (need > SFFT_STATIC_SCRATCH_BYTES) {
        set_last_error("sfft_hash_to_bins_static: " + std::to_string(need) + " bytes of scratch needed, " +
                       std::to_string(SFFT_STATIC_SCRATCH_BYTES) + " available");
        return SFFT_ERR_CAPACITY;
    }
    void* scratch = nullptr;
    sfft_status st = scratch_address(&scratch);
    if (st != SFFT_OK) return st;

    uint32_t logB = 0;
    while ((1u << logB) < B) ++logB;
    ExactArgs args;
    std::memset(&args, 0, sizeof(args));
    args.x = d_x;
    args.n = n;
    args.nmask = (uint32_t)(n - 1);
    args.B = B;
    args.logB = logB;
    args.T = T;
    args.H = 1;
    args.a_base = (uint32_t)a;
    args.chunks = (uint32_t)chunks;
    args.stage = kChunkTaps;
    args.ctaps = kChunkTaps;
    args.maxshift = 0;
    args.taps32 = d_taps;
    args.wtab = d_wtab;
    args.counter = reinterpret_cast<uint32_t*>(scratch);
    args.part = reinterpret_cast<unsigned char*>(scratch) + kCounterBytes;
    args.part_stride = chunks * B;
    args.zidx = const_cast<uint32_t*>(d_zidx);
    args.zval = reinterpret_cast<double2*>(const_cast<double*>(d_zval));
    args.zcap = nz > 0 ? nz : 1;
    args.e_nz = nz;
    args.bins_only = 1;
    args.e_sigma = (uint32_t)sigma;
    args.e_b = (uint32_t)b;
    args.ubins = reinterpret_cast<double2*>(d_u);
    const size_t gs = exact_gather_smem(kChunkTaps, false) + (size_t)(B > (uint32_t)kThreads ? B : kThreads) * 8;
    const size_t fs = exact_finish_smem(B, 1, args.zcap, false);
    const size_t smem = gs > fs ? gs : fs;
    if (smem > 200 * 1024) return SFFT_ERR_INVALID_ARG;
    cudaError_t e = set_exact_smem_limit(smem, false);
    if (e == cudaSuccess) e = cudaMemsetAsync(args.counter, 0, sizeof(uint32_t), (cudaStream_t)stream);
    if (e == cudaSuccess) e = launch_exact_round(args, 1, smem, (cudaStream_t)stream, false);
    if (e != cudaSuccess) {
        set_last_error(std::string("sfft_hash_to_bins_static: ") + cudaGetErrorString(e));
        return SFFT_ERR_CUDA;
    }
    return SFFT_OK;
}
