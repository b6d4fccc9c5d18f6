// Mass and momentum sums of a population buffer without any device
// allocation, for callers that cannot allocate device memory.
//
// Who needs this: a caller whose device memory is fully committed before the
// run starts -- for example a process whose framework caching allocator has
// reserved the whole GPU, or a simulation loop that forbids allocations after
// start-up so that its memory footprint and latency stay fixed -- cannot give
// lb_conservation a context arena or let it allocate temporary space.  This
// entry point takes the populations and an output buffer only; its per-block
// partial sums live in one fixed array compiled into the library.
//
// The array: g_sums_scratch below, 16384 blocks x 4 doubles = 512 KiB, held
// on every GPU that loads the library until the process exits.  Host code
// cannot use the array's name as a device address (in host code it is only a
// stand-in for the symbol), so the first call on each device looks the
// address up with cudaGetSymbolAddress while that device is current, checks
// the result, caches it, and passes it to the kernels.  The cache is keyed on
// the device and on its current CUDA context: after a device reset (or any
// new context on that device) the module, and with it the array, may load at
// another address, so the next call looks the address up again -- the
// first-call rule then applies anew.  The first call on a device (and the
// first after a reset) should come before any stream capture.  Every call
// overwrites the partial sums it later reads, so nothing needs clearing;
// calls that overlap on the GPU (for example on two streams at once) share
// the array and race.
#include <mutex>
#include <string>

#include "lbt_device.cuh"

namespace lbt {

constexpr int kNaThreads = 256;
constexpr int kNaSitesPerThread = 16;
constexpr int64_t kNaChunk = (int64_t)kNaThreads * kNaSitesPerThread;  // sites per block
constexpr int64_t kNaMaxChunks = 16384;                                 // partials the array holds
constexpr int kNaMaxEdge = 400;  // documented limit: 400^3 sites need 15625 of the 16384 partials
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) double g_sums_scratch[kNaMaxChunks * 4];

// Block c sums sites [c * kNaChunk, (c + 1) * kNaChunk): sum_i d_i and
// sum_i c_i d_i in FP64, written to partial[4 c .. 4 c + 3].
template <int ST>
__global__ void __launch_bounds__(kNaThreads) k_na_partial(const typename Stor<ST>::E* A, int64_t n3, double* partial)
{
    const int64_t c0 = (int64_t)blockIdx.x * kNaChunk;
    double acc[4] = {0, 0, 0, 0};
    for (int k = 0; k < kNaSitesPerThread; k++) {
        const int64_t s = c0 + (int64_t)k * kNaThreads + threadIdx.x;
        if (s >= n3) break;
#pragma unroll
        for (int i = 0; i < kQ; i++) {
            const double d = (double)Stor<ST>::in(A[(int64_t)i * n3 + s]);
            acc[0] += d;
            if (cvec(i, 0)) acc[1] += cvec(i, 0) * d;
            if (cvec(i, 1)) acc[2] += cvec(i, 1) * d;
            if (cvec(i, 2)) acc[3] += cvec(i, 2) * d;
        }
    }
    __shared__ double red[kNaThreads / 32][4];
    for (int a = 0; a < 4; a++)
        for (int o = 16; o > 0; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 4; a++) red[threadIdx.x >> 5][a] = acc[a];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0, 0, 0, 0};
        for (int w = 0; w < kNaThreads / 32; w++)
            for (int a = 0; a < 4; a++) t[a] += red[w][a];
        for (int a = 0; a < 4; a++) partial[4 * blockIdx.x + a] = t[a];
    }
}

// One thread adds the partials in block order: out = (n3 + sum d, sum c d).
__global__ void k_na_final(int64_t n3, int64_t nchunks, const double* partial, double* out)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double t[4] = {0, 0, 0, 0};
    for (int64_t c = 0; c < nchunks; c++)
        for (int a = 0; a < 4; a++) t[a] += partial[4 * c + a];
    out[0] = (double)n3 + t[0];
    for (int a = 1; a < 4; a++) out[a] = t[a];
}

namespace {
std::mutex g_na_mu;
double* g_na_addr[kNaMaxDevices] = {};
void* g_na_ctx[kNaMaxDevices] = {};  // CUDA context the cached address belongs to

// Current CUDA context (driver handle) through the runtime's driver entry
// point, so the library needs no link against the driver library.
cudaError_t current_context(void** ctx)
{
    using CtxGetCurrent = int (*)(void**);
    static CtxGetCurrent fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !f) return cudaErrorNotSupported;
        fn = reinterpret_cast<CtxGetCurrent>(f);
    }
    return fn(ctx) == 0 ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of g_sums_scratch on the current device, looked up once per
// device and context (again after a reset has replaced the context).
cudaError_t scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    // no context may be current yet (the runtime starts it lazily): then the
    // look-up below, which starts it, runs and the context is read after it
    void* ctx = nullptr;
    e = current_context(&ctx);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!ctx || !g_na_addr[dev] || g_na_ctx[dev] != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sums_scratch);
        if (e != cudaSuccess) return e;
        e = current_context(&ctx);
        if (e != cudaSuccess) return e;
        g_na_addr[dev] = reinterpret_cast<double*>(p);
        g_na_ctx[dev] = ctx;
    }
    *out = g_na_addr[dev];
    return cudaSuccess;
}
}  // namespace

}  // namespace lbt

using namespace lbt;

extern "C" int32_t lb_population_sums_noalloc(const void* populations, int32_t storage, int32_t E, double* out,
                                              void* stream)
{
    if (!populations || !out || storage < LB_STORE_F64 || storage > LB_STORE_BF16DEV || E < 1) {
        lbt_set_last_error("lb_population_sums_noalloc: null pointer, unknown storage or E < 1");
        return LB_ERR_ARG;
    }
    const int64_t n3 = (int64_t)E * E * E;
    const int64_t nchunks = (n3 + kNaChunk - 1) / kNaChunk;
    if (E > kNaMaxEdge || nchunks > kNaMaxChunks) {
        lbt_set_last_error("lb_population_sums_noalloc: box of E^3 sites exceeds the fixed scratch "
                           "(at most 64 Mi sites, E <= 400)");
        return LB_ERR_SIZE;
    }
    double* partial = nullptr;
    cudaError_t e = scratch_address(&partial);
    if (e != cudaSuccess) {
        lbt_set_last_error((std::string("lb_population_sums_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
        return LB_ERR_CUDA;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (storage) {
        case LB_STORE_F64:
            k_na_partial<kF64><<<(unsigned)nchunks, kNaThreads, 0, s>>>(reinterpret_cast<const double*>(populations), n3, partial);
            break;
        case LB_STORE_F32:
            k_na_partial<kF32><<<(unsigned)nchunks, kNaThreads, 0, s>>>(reinterpret_cast<const float*>(populations), n3, partial);
            break;
        case LB_STORE_F16DEV:
            k_na_partial<kF16><<<(unsigned)nchunks, kNaThreads, 0, s>>>(reinterpret_cast<const uint16_t*>(populations), n3, partial);
            break;
        default:
            k_na_partial<kBF16><<<(unsigned)nchunks, kNaThreads, 0, s>>>(reinterpret_cast<const uint16_t*>(populations), n3, partial);
            break;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_na_final<<<1, 1, 0, s>>>(n3, nchunks, partial, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        lbt_set_last_error((std::string("lb_population_sums_noalloc: launch: ") + cudaGetErrorString(e)).c_str());
        return LB_ERR_CUDA;
    }
    return LB_OK;
}
