// Inference forward of the learned boundary upsampler on the fifth-generation
// tensor cores (tcgen05): 128-row tiles, the three layers as UMMA
// instructions with bf16 operands in shared memory and FP32 accumulators in
// tensor memory (TMEM), bias + ReLU + bf16 epilogues read back with
// tcgen05.ld.  The same network and rounding points as the warp-level
// (mma.sync) forward in lbt_mlp.cu, which stays for training (it also saves
// the hidden activations for the backward pass).
//
// Operand layout: both operands K-major without swizzle, in 8 x 8 "core
// matrices" of 128 bytes (8 rows of 16 bytes); core matrices adjacent along
// K are 128 bytes apart (the descriptor's leading byte offset), those
// adjacent along M / N are K/8 x 128 bytes apart (its stride byte offset).
// One UMMA covers K = 16: its descriptors advance by two core matrices.
#include <cuda_bf16.h>

#include <cstdio>

#include "lbt_device.cuh"
#include "lbt_mlp.h"

namespace lbt {

namespace {

constexpr int kTcRows = 128;     // rows per tile (UMMA M)
constexpr int kTcThreads = 128;  // four warps: warp w reads TMEM lanes 32w .. 32w+31
constexpr int kTcCols = 256;     // TMEM columns: hidden accumulators at 0, output at 128

__host__ __device__ constexpr int pad16(int n) { return (n + 15) / 16 * 16; }

// element (r, k) of an R x K K-major operand in the core-matrix layout
__device__ __forceinline__ int core_off(int r, int k, int K) { return (r >> 3) * (K >> 3) * 64 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7); }

template <int NOUT>
struct TcSmem {
    static constexpr int kNP = pad16(NOUT);
    __nv_bfloat16 w1[kMlpHidden * kMlpIn];
    __nv_bfloat16 w2[kMlpHidden * kMlpHidden];
    __nv_bfloat16 w3[kNP * kMlpHidden];
    __nv_bfloat16 x[kTcRows * kMlpIn];
    __nv_bfloat16 h[kTcRows * kMlpHidden];
    __align__(16) float b1[kMlpHidden];
    __align__(16) float b2[kMlpHidden];
    __align__(16) float b3[kNP];
    uint64_t bar;
    uint32_t tmem;
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, N / 8 at bit 17, M / 16 at bit 24
__device__ __forceinline__ uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, bool acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc ? 1u : 0u)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

// 32 FP32 columns of this thread's TMEM lane, without waiting (tc_ld_wait)
__device__ __forceinline__ void tc_ld32_nowait(uint32_t taddr, uint32_t r[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tc_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_ld16_nowait(uint32_t taddr, uint32_t r[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// wait for a phase of the MMA barrier, giving up after about one second
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok = 0;
    const uint64_t t0 = [] {
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        return t;
    }();
    while (true) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(su32(bar)), "r"(phase), "r"(20000u)
            : "memory");
        if (ok) return true;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 1000000000ull) return false;
    }
}

// accumulator columns [col0, col0 + 128) of this thread's row -> bias, ReLU,
// bf16 -> row m of the next layer's A operand
// (64 columns per round: two 32-column TMEM loads in flight, one wait)
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem_row, const float* bias, __nv_bfloat16* h, int m)
{
#pragma unroll 1
    for (int c0 = 0; c0 < kMlpHidden; c0 += 64) {
        uint32_t r[64];
        tc_ld32_nowait(tmem_row + c0, r);
        tc_ld32_nowait(tmem_row + c0 + 32, r + 32);
        tc_ld_wait();
#pragma unroll
        for (int g = 0; g < 64; g += 16) {
            float bj[16];
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4*>(bj + j) = *reinterpret_cast<const float4*>(bias + c0 + g + j);
            uint32_t pk[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const float a = fmaxf(__uint_as_float(r[g + 2 * j]) + bj[2 * j], 0.f);
                const float b = fmaxf(__uint_as_float(r[g + 2 * j + 1]) + bj[2 * j + 1], 0.f);
                __nv_bfloat162 p2 = __floats2bfloat162_rn(a, b);
                pk[j] = *reinterpret_cast<uint32_t*>(&p2);
            }
            *reinterpret_cast<uint4*>(h + core_off(m, c0 + g, kMlpHidden)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *reinterpret_cast<uint4*>(h + core_off(m, c0 + g + 8, kMlpHidden)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
    }
}

template <int NOUT>
__global__ void __launch_bounds__(kTcThreads) k_mlp_forward_tc(const __nv_bfloat16* __restrict__ X, int64_t rows,
                                                               const unsigned char* __restrict__ params, MlpLayout L,
                                                               float* __restrict__ Y, int64_t col_stride, int32_t* err)
{
    using Sm = TcSmem<NOUT>;
    constexpr int NP = Sm::kNP;
    extern __shared__ __align__(128) unsigned char tc_smem_raw[];
    Sm& sm = *reinterpret_cast<Sm*>(tc_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;

    // weights into the core-matrix layout (W3 padded with zero rows to NP)
    const __nv_bfloat16* w1 = reinterpret_cast<const __nv_bfloat16*>(params + L.w1);
    const __nv_bfloat16* w2 = reinterpret_cast<const __nv_bfloat16*>(params + L.w2);
    const __nv_bfloat16* w3 = reinterpret_cast<const __nv_bfloat16*>(params + L.w3);
    for (int i = tid; i < kMlpHidden * kMlpIn; i += kTcThreads) sm.w1[core_off(i / kMlpIn, i % kMlpIn, kMlpIn)] = w1[i];
    for (int i = tid; i < kMlpHidden * kMlpHidden; i += kTcThreads)
        sm.w2[core_off(i / kMlpHidden, i % kMlpHidden, kMlpHidden)] = w2[i];
    for (int i = tid; i < NP * kMlpHidden; i += kTcThreads)
        sm.w3[core_off(i / kMlpHidden, i % kMlpHidden, kMlpHidden)] =
            i < NOUT * kMlpHidden ? w3[i] : __float2bfloat16(0.f);
    for (int i = tid; i < kMlpHidden; i += kTcThreads) {
        sm.b1[i] = reinterpret_cast<const float*>(params + L.b1)[i];
        sm.b2[i] = reinterpret_cast<const float*>(params + L.b2)[i];
    }
    for (int i = tid; i < NP; i += kTcThreads) sm.b3[i] = i < NOUT ? reinterpret_cast<const float*>(params + L.b3)[i] : 0.f;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sm.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sm.tmem)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;
    const uint32_t tmem_row = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's lanes
    const int m = tid;                                                // row of the tile this thread owns
    const uint32_t id_h = tc_idesc(kTcRows, kMlpHidden), id_o = tc_idesc(kTcRows, NP);
    const uint32_t ax = su32(sm.x), ah = su32(sm.h), a1 = su32(sm.w1), a2 = su32(sm.w2), a3 = su32(sm.w3);
    constexpr uint32_t kLbo = 128, kSbo32 = (kMlpIn / 8) * 128, kSbo128 = (kMlpHidden / 8) * 128;
    uint32_t phase = 0;
    bool ok = true;

    const int64_t ntiles = (rows + kTcRows - 1) / kTcRows;
    // features of a tile, row m = this thread (zeros past the last row); the
    // next tile's are loaded into registers while this one is computed
    uint4 xr[kMlpIn / 8];
    auto load_x = [&](int64_t tile) {
        const int64_t r = tile * kTcRows + m;
        const bool in = tile < ntiles && r < rows;
        const uint4* src = reinterpret_cast<const uint4*>(X + (in ? r : 0) * kMlpIn);
#pragma unroll
        for (int c = 0; c < kMlpIn / 8; c++) xr[c] = in ? __ldg(src + c) : make_uint4(0u, 0u, 0u, 0u);
    };
    load_x(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t r0 = tile * kTcRows;
#pragma unroll
        for (int c = 0; c < kMlpIn / 8; c++) *reinterpret_cast<uint4*>(sm.x + core_off(m, 8 * c, kMlpIn)) = xr[c];
        load_x(tile + gridDim.x);
        // the three layers; each: MMAs by one thread, commit, wait, epilogue
        for (int layer = 0; layer < 3 && ok; layer++) {
            proxy_fence();  // generic-proxy shared-memory writes -> tensor-core reads
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                if (layer == 0) {
                    for (int ks = 0; ks < kMlpIn / 16; ks++)
                        tc_mma(tmem, tc_desc(ax + ks * 256, kLbo, kSbo32), tc_desc(a1 + ks * 256, kLbo, kSbo32), id_h,
                               ks > 0);
                } else {
                    const uint32_t ab = layer == 1 ? a2 : a3;
                    const uint32_t dcol = layer == 1 ? 0u : 128u;
                    const uint32_t id = layer == 1 ? id_h : id_o;
                    for (int ks = 0; ks < kMlpHidden / 16; ks++)
                        tc_mma(tmem + dcol, tc_desc(ah + ks * 256, kLbo, kSbo128), tc_desc(ab + ks * 256, kLbo, kSbo128),
                               id, ks > 0);
                }
                tc_commit(&sm.bar);
            }
            const bool arrived = tc_wait(&sm.bar, phase);
            phase ^= 1u;
            if (!__syncthreads_and(arrived)) {
                ok = false;  // the MMAs did not complete within a second
                break;
            }
            tc_fence_after();
            if (layer == 0) {
                hidden_epilogue(tmem_row, sm.b1, sm.h, m);
            } else if (layer == 1) {
                hidden_epilogue(tmem_row, sm.b2, sm.h, m);
            } else {
                // every lane takes part in the (warp-collective) TMEM loads;
                // rows past the end store nothing
                const bool in = r0 + m < rows;
                static_assert(NP == 32 || NP == 48, "output columns: one 32-column load and at most one 16-column one");
                uint32_t r[NP];  // every output column in flight at once, one wait
                tc_ld32_nowait(tmem_row + 128, r);
                if constexpr (NP == 48) tc_ld16_nowait(tmem_row + 128 + 32, r + 32);
                tc_ld_wait();
#pragma unroll
                for (int c0 = 0; c0 < NP; c0 += 16) {
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[c0 + j]);
                    if (col_stride == 0) {  // row-major [rows][NOUT]: four 16-byte stores per lane
                        float* y = Y + (r0 + m) * NOUT;
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            if (in && c0 + j < NOUT) {
                                const float4 bb = *reinterpret_cast<const float4*>(sm.b3 + c0 + j);
                                *reinterpret_cast<float4*>(y + c0 + j) =
                                    make_float4(v[j] + bb.x, v[j + 1] + bb.y, v[j + 2] + bb.z, v[j + 3] + bb.w);
                            }
                    } else {  // column-major Y[col * col_stride + row]: the warp's 32 rows in one line per column
#pragma unroll
                        for (int j = 0; j < 16; j++)
                            if (in && c0 + j < NOUT) Y[(int64_t)(c0 + j) * col_stride + r0 + m] = v[j] + sm.b3[c0 + j];
                    }
                }
            }
        }
    }
    if (!ok) {
        if (tid == 0 && err) atomicCAS(err, 0, LB_ERR_TIMEOUT);
        tc_wait(&sm.bar, phase ^ 1u);  // let an MMA still in flight finish (bounded)
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

template <int NOUT>
cudaError_t forward_tc(const void* X, int64_t rows, const void* params, const MlpLayout& L, float* Y,
                       int64_t col_stride, int32_t* err, cudaStream_t s)
{
    static int attr_done[kMaxDevices] = {};  // per instantiation and device
    const int smem = (int)sizeof(TcSmem<NOUT>);
    cudaError_t e = smem_attr_per_device(k_mlp_forward_tc<NOUT>, smem, attr_done);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (rows + kTcRows - 1) / kTcRows;
    int64_t blocks = 2LL * sms;  // two blocks per SM: 2 x 256 TMEM columns, 2 x 94 KB shared memory
    if (blocks > tiles) blocks = tiles;
    if (blocks < 1) return cudaSuccess;
    k_mlp_forward_tc<NOUT><<<(unsigned)blocks, kTcThreads, smem, s>>>(
        reinterpret_cast<const __nv_bfloat16*>(X), rows, reinterpret_cast<const unsigned char*>(params), L, Y, col_stride,
        err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t mlp_forward_tc(const void* X, int64_t rows, const void* params, int K, float* Y, int32_t* err,
                           cudaStream_t s, int64_t col_stride)
{
    const MlpLayout L = mlp_layout(K);
    if (K == 16) return forward_tc<48>(X, rows, params, L, Y, col_stride, err, s);
    if (K == 8) return forward_tc<24>(X, rows, params, L, Y, col_stride, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace lbt
