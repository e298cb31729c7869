// dna_kl_noalloc: d_KL(V, WH), the value of dna_kl, for callers that cannot allocate
// device memory (the paper has no counterpart of this entry point).
//
// Some callers cannot call cudaMalloc: code whose device memory is all owned by another
// framework's pool allocator, and latency-critical code that cannot afford cudaMalloc's
// cost or the implicit device synchronisation of cudaFree.  This entry point computes the
// same value as dna_kl without a context: its scratch (per-column partial sums and a
// status word) lives in the file-scope array below, which every GPU that loads this
// library holds until the process exits.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "dna.h"
#include "simt_kernels.cuh"

namespace {

// Layout of the static scratch: bytes [0, 256) hold the int status word, then
// DNA_KL_NOALLOC_MAX_PARTIALS float64 partial sums.
constexpr size_t kStatusBytes = 256;
constexpr size_t kScratchBytes = kStatusBytes + sizeof(double) * (size_t)DNA_KL_NOALLOC_MAX_PARTIALS;

static __device__ __align__(256) unsigned char g_kl_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
int g_sms[kMaxDevices] = {};

// Device address of g_kl_scratch in the current context, looked up on every call (a
// lookup, no allocation): an address cached per device would go stale under another
// context or after a device reset.  The host-side name of the array is not a device
// address.  The SM count is cached per device.
int scratch_base(int dev, void** base, int* sms) {
    if (dev < 0 || dev >= kMaxDevices) return DNA_ERR_UNSUPPORTED;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_kl_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return DNA_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_sms[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return DNA_ERR_CUDA;
        }
        g_sms[dev] = n;
    }
    *base = p;
    *sms = g_sms[dev];
    return DNA_OK;
}

// Sum the partials in a fixed order; +inf when a kernel saw z <= 0 where v > 0 (the cost
// is then infinite).
__global__ void k_kl_finish(const double* __restrict__ part, int64_t n,
                            const int* __restrict__ status, double* __restrict__ out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (*status & dna::STATUS_NONFINITE) ? (double)INFINITY : red[0];
}

template <int RB>
int launch(const dna::View& v, double* part, int splits, int64_t s_per, int* status,
           cudaStream_t st) {
    using namespace dna::simt;
    const size_t smem = Pass2Cfg<float, RB, 1>::smem;
    auto k = k_pass2<float, RB, 1, true>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return DNA_ERR_CUDA;
    dim3 grid((unsigned)((v.O + OB - 1) / OB), (unsigned)splits);
    k<<<grid, NT, smem, st>>>(v, static_cast<const float*>(v.X), static_cast<const float*>(v.X),
                              v.xr, v.xo, part, s_per, status);
    return cudaGetLastError() == cudaSuccess ? DNA_OK : DNA_ERR_CUDA;
}

}  // namespace

extern "C" int dna_kl_noalloc(const float* V, int64_t ldv, const float* W, const float* H,
                              int64_t N, int64_t T, int64_t R, double* kl_out, void* stream) {
    if (!V || !W || !H || !kl_out || N < 1 || T < 1 || R < 1 || R > 512 || ldv < T)
        return DNA_ERR_ARG;
    if (T > DNA_KL_NOALLOC_MAX_PARTIALS) return DNA_ERR_LIMIT;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DNA_ERR_CUDA;
    void* base = nullptr;
    int sms = 1;
    if (int e = scratch_base(dev, &base, &sms)) return e;
    int* status = static_cast<int*>(base);
    double* part = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kStatusBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // Split the sum over n so the grid covers the GPU, within the scratch capacity.
    const int ob = dna::simt::OB, sb = dna::simt::SB;
    const int64_t nob = (T + ob - 1) / ob, chunks = (N + sb - 1) / sb;
    int64_t splits = (sms + nob - 1) / nob;
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, chunks / 4));
    splits = std::min<int64_t>(splits, 32);
    splits = std::min<int64_t>(splits, DNA_KL_NOALLOC_MAX_PARTIALS / T);
    splits = std::max<int64_t>(splits, 1);
    const int64_t s_per = (chunks + splits - 1) / splits * sb;
    splits = (N + s_per - 1) / s_per;

    dna::View v{};
    v.S = N; v.O = T; v.R = R;
    v.V = V; v.vs = ldv;
    v.X = const_cast<float*>(H); v.xr = T; v.xo = 1;
    v.Y = W; v.ys = R; v.yr = 1;
    v.vsum = nullptr;

    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return DNA_ERR_CUDA;
    int e;
    const int rb = R <= 32 ? 32 : (R <= 64 ? 64 : 128);
    if (rb == 32) e = launch<32>(v, part, (int)splits, s_per, status, st);
    else if (rb == 64) e = launch<64>(v, part, (int)splits, s_per, status, st);
    else e = launch<128>(v, part, (int)splits, s_per, status, st);
    if (e) return e;
    k_kl_finish<<<1, 1024, 0, st>>>(part, splits * T, status, kl_out);
    return cudaGetLastError() == cudaSuccess ? DNA_OK : DNA_ERR_CUDA;
}
