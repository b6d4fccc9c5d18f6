// Forward and backward of the learned boundary upsampler on the fifth-generation
// tensor cores (tcgen05): 128-row tiles, the three layers as UMMA
// instructions with bf16 operands in shared memory and FP32 accumulators in
// tensor memory (TMEM), bias + ReLU + bf16 epilogues read back with
// tcgen05.ld.  Training uses the same forward (saving the bf16 activations)
// and a backward of the same construction: activation gradients per row tile,
// weight gradients as UMMAs that reduce over the rows (below).
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
constexpr int kTcThreads = 128;  // backward kernels: four warps, warp w reads TMEM lanes 32w .. 32w+31
// Forward: four groups of four warps per block (one block per SM), each
// group with its own 128-row tile, activations in shared memory, 128 TMEM
// columns and MMA barrier, so that four tiles are in flight per SM and a
// group's epilogue overlaps the other groups' MMAs.
constexpr int kFwGroups = 4;
constexpr int kFwThreads = kFwGroups * kTcRows;
constexpr int kFwCols = kFwGroups * kMlpHidden;  // 512: the whole TMEM of the SM

__host__ __device__ constexpr int pad16(int n) { return (n + 15) / 16 * 16; }

// element (r, k) of an R x K K-major operand in the core-matrix layout
__device__ __forceinline__ int core_off(int r, int k, int K) { return (r >> 3) * (K >> 3) * 64 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7); }

template <int NOUT>
struct TcSmem {
    static constexpr int kNP = pad16(NOUT);
    __nv_bfloat16 w1[kMlpHidden * kMlpIn];
    __nv_bfloat16 w2[kMlpHidden * kMlpHidden];
    __nv_bfloat16 w3[kNP * kMlpHidden];
    __nv_bfloat16 x[kFwGroups][kTcRows * kMlpIn];
    __nv_bfloat16 h[kFwGroups][kTcRows * kMlpHidden];
    // biases inside the MMAs: an A tile of ones in K columns 0 and 1, and B
    // tiles whose K columns 0 and 1 hold the FP32 bias split into bf16
    // high and low parts (their sum is the bias to 2^-16 relative); layer 1
    // uses feature columns 24 and 25 (zero padding) and rows 24, 25 of W1
    __nv_bfloat16 ones[kTcRows * 16];
    __nv_bfloat16 bb2[kMlpHidden * 16];
    __nv_bfloat16 bb3[kNP * 16];
    uint64_t bar[kFwGroups];
    uint32_t tmem;
};
static_assert(sizeof(TcSmem<48>) <= 227 * 1024, "forward shared memory");

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
// barrier over the 128 threads of one forward group (ids 1 .. 4; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kTcRows) : "memory"); }
__device__ __forceinline__ bool group_all(int g, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbarrier.cta.red.and.pred po, %2, %3, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(g + 1), "r"(kTcRows)
        : "memory");
    return r != 0;
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

// ReLU and bf16 of two accumulators in one instruction, a in the low half
__device__ __forceinline__ uint32_t relu_bf16x2(float a, float b)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}

// accumulator columns [0, 128) of this thread's row (the bias is already in
// them) -> ReLU, bf16 -> row m of the next layer's A operand, and (training)
// the same bf16 row to save (row-major, nullptr: not saved)
// (64 columns per round: two 32-column TMEM loads in flight, one wait)
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem_row, __nv_bfloat16* h, int m, __nv_bfloat16* save_row)
{
#pragma unroll 1
    for (int c0 = 0; c0 < kMlpHidden; c0 += 64) {
        uint32_t r[64];
        tc_ld32_nowait(tmem_row + c0, r);
        tc_ld32_nowait(tmem_row + c0 + 32, r + 32);
        tc_ld_wait();
#pragma unroll
        for (int g = 0; g < 64; g += 16) {
            uint32_t pk[8];
#pragma unroll
            for (int j = 0; j < 8; j++) pk[j] = relu_bf16x2(__uint_as_float(r[g + 2 * j]), __uint_as_float(r[g + 2 * j + 1]));
            *reinterpret_cast<uint4*>(h + core_off(m, c0 + g, kMlpHidden)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *reinterpret_cast<uint4*>(h + core_off(m, c0 + g + 8, kMlpHidden)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            if (save_row) {
                *reinterpret_cast<uint4*>(save_row + c0 + g) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4*>(save_row + c0 + g + 8) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
        }
    }
}

// SAVE (training): the bf16 hidden activations after ReLU -- the values the
// next layer consumed -- are also written row-major to H1s and H2s
// ([rows][128]), for the masks of the backward pass.
template <int NOUT, bool SAVE>
__global__ void __launch_bounds__(kFwThreads, 1) k_mlp_forward_tc(const __nv_bfloat16* __restrict__ X, int64_t rows,
                                                                  const unsigned char* __restrict__ params, MlpLayout L,
                                                                  float* __restrict__ Y, int64_t col_stride,
                                                                  int32_t* err, __nv_bfloat16* __restrict__ H1s,
                                                                  __nv_bfloat16* __restrict__ H2s)
{
    using Sm = TcSmem<NOUT>;
    constexpr int NP = Sm::kNP;
    extern __shared__ __align__(128) unsigned char tc_smem_raw[];
    Sm& sm = *reinterpret_cast<Sm*>(tc_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = warp / 4;          // group: its tile, buffers, TMEM columns and barrier
    const int q = warp % 4;          // TMEM lane quadrant this warp reads
    const int m = 32 * q + (tid & 31);  // row of the group's tile this thread owns
    const int gt = tid % kTcRows;    // thread index within the group

    // weights into the core-matrix layout (W3 padded with zero rows to NP), once per block
    const __nv_bfloat16* w1 = reinterpret_cast<const __nv_bfloat16*>(params + L.w1);
    const __nv_bfloat16* w2 = reinterpret_cast<const __nv_bfloat16*>(params + L.w2);
    const __nv_bfloat16* w3 = reinterpret_cast<const __nv_bfloat16*>(params + L.w3);
    for (int i = tid; i < kMlpHidden * kMlpIn; i += kFwThreads) sm.w1[core_off(i / kMlpIn, i % kMlpIn, kMlpIn)] = w1[i];
    for (int i = tid; i < kMlpHidden * kMlpHidden; i += kFwThreads)
        sm.w2[core_off(i / kMlpHidden, i % kMlpHidden, kMlpHidden)] = w2[i];
    for (int i = tid; i < NP * kMlpHidden; i += kFwThreads)
        sm.w3[core_off(i / kMlpHidden, i % kMlpHidden, kMlpHidden)] =
            i < NOUT * kMlpHidden ? w3[i] : __float2bfloat16(0.f);
    // bias b as two bf16 parts hi + lo: hi = bf16(b), lo = bf16(b - hi)
    auto split = [](float b, __nv_bfloat16& hi, __nv_bfloat16& lo) {
        hi = __float2bfloat16_rn(b);
        lo = __float2bfloat16_rn(b - __bfloat162float(hi));
    };
    const float* b1 = reinterpret_cast<const float*>(params + L.b1);
    const float* b2 = reinterpret_cast<const float*>(params + L.b2);
    const float* b3 = reinterpret_cast<const float*>(params + L.b3);
    __syncthreads();  // W1 rows 24, 25 are overwritten below
    for (int n = tid; n < kMlpHidden; n += kFwThreads) {
        __nv_bfloat16 hi, lo;
        split(b1[n], hi, lo);  // layer 1: feature columns 24, 25 are set to one at staging
        sm.w1[core_off(n, kMlpFeat, kMlpIn)] = hi;
        sm.w1[core_off(n, kMlpFeat + 1, kMlpIn)] = lo;
    }
    for (int i = tid; i < kMlpHidden * 16; i += kFwThreads) {
        const int n = i / 16, k = i % 16;
        __nv_bfloat16 hi, lo;
        split(b2[n], hi, lo);
        sm.bb2[core_off(n, k, 16)] = k == 0 ? hi : (k == 1 ? lo : __float2bfloat16(0.f));
        sm.ones[core_off(n, k, 16)] = k < 2 ? __float2bfloat16(1.f) : __float2bfloat16(0.f);
    }
    for (int i = tid; i < NP * 16; i += kFwThreads) {
        const int n = i / 16, k = i % 16;
        __nv_bfloat16 hi = __float2bfloat16(0.f), lo = __float2bfloat16(0.f);
        if (n < NOUT) split(b3[n], hi, lo);
        sm.bb3[core_off(n, k, 16)] = k == 0 ? hi : (k == 1 ? lo : __float2bfloat16(0.f));
    }
    if (tid < kFwGroups) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sm.bar[tid])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sm.tmem)),
                     "r"(kFwCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // the group's 128 columns hold the hidden accumulators of layers 1 and 2
    // and then the output (each written after the previous epilogue read it)
    const uint32_t tmem_g = sm.tmem + (uint32_t)(kMlpHidden * g);
    const uint32_t tmem_row = tmem_g + ((uint32_t)(32 * q) << 16);
    const uint32_t id_h = tc_idesc(kTcRows, kMlpHidden), id_o = tc_idesc(kTcRows, NP);
    const uint32_t ax = su32(sm.x[g]), ah = su32(sm.h[g]), a1 = su32(sm.w1), a2 = su32(sm.w2), a3 = su32(sm.w3);
    const uint32_t a_one = su32(sm.ones), ab2 = su32(sm.bb2), ab3 = su32(sm.bb3);
    constexpr uint32_t kLbo = 128, kSbo16 = (16 / 8) * 128, kSbo32 = (kMlpIn / 8) * 128,
                       kSbo128 = (kMlpHidden / 8) * 128;
    uint32_t phase = 0;
    bool ok = true;

    const int64_t ntiles = (rows + kTcRows - 1) / kTcRows;
    const int64_t stride = (int64_t)gridDim.x * kFwGroups;
    // features of a tile, row m = this thread (zeros past the last row); the
    // next tile's are loaded into registers while this one is computed
    uint4 xr[kMlpIn / 8];
    auto load_x = [&](int64_t tile) {
        const int64_t r = tile * kTcRows + m;
        const bool in = tile < ntiles && r < rows;
        const uint4* src = reinterpret_cast<const uint4*>(X + (in ? r : 0) * kMlpIn);
#pragma unroll
        for (int c = 0; c < kMlpIn / 8; c++) xr[c] = in ? __ldg(src + c) : make_uint4(0u, 0u, 0u, 0u);
        // feature columns 24 and 25 (zero padding) carry the ones of layer 1's bias
        static_assert(kMlpFeat == 24, "the bias columns follow the 24 features");
        xr[3].x = 0x3F803F80u;  // bf16 1.0 in both halves
    };
    int64_t tile = (int64_t)blockIdx.x * kFwGroups + g;
    load_x(tile);
    for (; tile < ntiles && ok; tile += stride) {
        const int64_t r0 = tile * kTcRows;
#pragma unroll
        for (int c = 0; c < kMlpIn / 8; c++) *reinterpret_cast<uint4*>(sm.x[g] + core_off(m, 8 * c, kMlpIn)) = xr[c];
        load_x(tile + stride);
        // the three layers; each: MMAs by one thread of the group, commit, wait, epilogue
        for (int layer = 0; layer < 3 && ok; layer++) {
            proxy_fence();  // generic-proxy shared-memory writes -> tensor-core reads
            tc_fence_before();
            group_sync(g);
            tc_fence_after();
            if (gt == 0) {
                if (layer == 0) {
                    for (int ks = 0; ks < kMlpIn / 16; ks++)
                        tc_mma(tmem_g, tc_desc(ax + ks * 256, kLbo, kSbo32), tc_desc(a1 + ks * 256, kLbo, kSbo32), id_h,
                               ks > 0);
                } else {
                    const uint32_t ab = layer == 1 ? a2 : a3;
                    const uint32_t id = layer == 1 ? id_h : id_o;
                    for (int ks = 0; ks < kMlpHidden / 16; ks++)
                        tc_mma(tmem_g, tc_desc(ah + ks * 256, kLbo, kSbo128), tc_desc(ab + ks * 256, kLbo, kSbo128), id,
                               ks > 0);
                    // + ones x (bias hi, lo): the layer's bias
                    tc_mma(tmem_g, tc_desc(a_one, kLbo, kSbo16), tc_desc(layer == 1 ? ab2 : ab3, kLbo, kSbo16), id, true);
                }
                tc_commit(&sm.bar[g]);
            }
            const bool arrived = tc_wait(&sm.bar[g], phase);
            phase ^= 1u;
            if (!group_all(g, arrived)) {
                ok = false;  // the MMAs did not complete within a second
                break;
            }
            tc_fence_after();
            if (layer < 2) {
                __nv_bfloat16* save = nullptr;
                if (SAVE && r0 + m < rows) save = (layer == 0 ? H1s : H2s) + (r0 + m) * kMlpHidden;
                hidden_epilogue(tmem_row, sm.h[g], m, save);
            } else {
                // every lane takes part in the (warp-collective) TMEM loads;
                // rows past the end store nothing
                const bool in = r0 + m < rows;
                static_assert(NP == 32 || NP == 48, "output columns: one 32-column load and at most one 16-column one");
                uint32_t r[NP];  // every output column in flight at once, one wait
                tc_ld32_nowait(tmem_row, r);
                if constexpr (NP == 48) tc_ld16_nowait(tmem_row + 32, r + 32);
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
                            if (in && c0 + j < NOUT)
                                *reinterpret_cast<float4*>(y + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    } else {  // column-major Y[col * col_stride + row]: the warp's 32 rows in one line per column
#pragma unroll
                        for (int j = 0; j < 16; j++)
                            if (in && c0 + j < NOUT) Y[(int64_t)(c0 + j) * col_stride + r0 + m] = v[j];
                    }
                }
            }
        }
    }
    if (!ok) {
        if (gt == 0 && err) atomicCAS(err, 0, LB_ERR_TIMEOUT);
        tc_wait(&sm.bar[g], phase ^ 1u);  // let an MMA still in flight finish (bounded)
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem), "r"(kFwCols) : "memory");
}

template <int NOUT, bool SAVE>
cudaError_t forward_tc(const void* X, int64_t rows, const void* params, const MlpLayout& L, float* Y,
                       int64_t col_stride, int32_t* err, cudaStream_t s, __nv_bfloat16* H1s = nullptr,
                       __nv_bfloat16* H2s = nullptr)
{
    static int attr_done[kMaxDevices] = {};  // per instantiation and device
    const int smem = (int)sizeof(TcSmem<NOUT>);
    cudaError_t e = smem_attr_per_device(k_mlp_forward_tc<NOUT, SAVE>, smem, attr_done);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (rows + kTcRows - 1) / kTcRows;
    int64_t blocks = sms;  // one block per SM: all 512 TMEM columns, four groups of 128 rows
    if (blocks > (tiles + kFwGroups - 1) / kFwGroups) blocks = (tiles + kFwGroups - 1) / kFwGroups;
    if (blocks < 1) return cudaSuccess;
    k_mlp_forward_tc<NOUT, SAVE><<<(unsigned)blocks, kFwThreads, smem, s>>>(
        reinterpret_cast<const __nv_bfloat16*>(X), rows, reinterpret_cast<const unsigned char*>(params), L, Y, col_stride,
        err, H1s, H2s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Backward pass on the tensor cores.
//
// Activation gradients, per 128-row tile (the forward's shape):
//     dH[r][i] = (sum_o dZ[r][o] W[i][o]) [H[r][i] > 0],
// A = the dZ tile (bf16, K = the columns of dZ padded to KZ), B = W as
// [N = i][K = o] (the transpose of the out-major inference weights, staged
// once per block), D in TMEM, the mask and the bf16 rounding in the epilogue.
// ---------------------------------------------------------------------------
template <int KZ>
struct DhSmem {
    __nv_bfloat16 w[kMlpHidden * KZ];  // B: W[i][o], K-major
    __nv_bfloat16 a[kTcRows * KZ];     // A: dZ tile, K-major
    uint64_t bar;
    uint32_t tmem;
};

template <int KZ, class ZT>
__global__ void __launch_bounds__(kTcThreads) k_mlp_dh_tc(const ZT* __restrict__ dZ, int nz, int64_t rows,
                                                          const __nv_bfloat16* __restrict__ Wt,
                                                          const __nv_bfloat16* __restrict__ H,
                                                          __nv_bfloat16* __restrict__ dH, int32_t* err)
{
    static_assert(KZ % 16 == 0, "K of the tile in steps of 16");
    using Sm = DhSmem<KZ>;
    extern __shared__ __align__(128) unsigned char dh_smem_raw[];
    Sm& sm = *reinterpret_cast<Sm*>(dh_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int e = tid; e < kMlpHidden * KZ; e += kTcThreads) {  // W[i][o] = Wt[o][i], zero for o >= nz
        const int i = e / KZ, o = e % KZ;
        sm.w[core_off(i, o, KZ)] = o < nz ? Wt[o * kMlpHidden + i] : __float2bfloat16(0.f);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sm.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sm.tmem)),
                     "r"(kMlpHidden)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;
    const uint32_t tmem_row = tmem + ((uint32_t)(32 * warp) << 16);
    const int m = tid;
    const uint32_t idesc = tc_idesc(kTcRows, kMlpHidden);
    const uint32_t aa = su32(sm.a), ab = su32(sm.w);
    constexpr uint32_t kLbo = 128, kSbo = (KZ / 8) * 128;
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (rows + kTcRows - 1) / kTcRows;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t r = tile * kTcRows + m;
        const bool in = r < rows;
        // row m of the A tile: dZ[r][0 .. nz) as bf16, zero past nz and past the last row
#pragma unroll
        for (int o0 = 0; o0 < KZ; o0 += 8) {
            uint32_t pk[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int o = o0 + 2 * j;
                const float a = in && o < nz ? (float)dZ[r * nz + o] : 0.f;
                const float b = in && o + 1 < nz ? (float)dZ[r * nz + o + 1] : 0.f;
                __nv_bfloat162 p2 = __floats2bfloat162_rn(a, b);
                pk[j] = *reinterpret_cast<uint32_t*>(&p2);
            }
            *reinterpret_cast<uint4*>(sm.a + core_off(m, o0, KZ)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            for (int ks = 0; ks < KZ / 16; ks++)
                tc_mma(tmem, tc_desc(aa + ks * 256, kLbo, kSbo), tc_desc(ab + ks * 256, kLbo, kSbo), idesc, ks > 0);
            tc_commit(&sm.bar);
        }
        const bool arrived = tc_wait(&sm.bar, phase);
        phase ^= 1u;
        if (!__syncthreads_and(arrived)) {
            ok = false;
            break;
        }
        tc_fence_after();
        // epilogue: mask by the saved activation, bf16, row-major
#pragma unroll 1
        for (int c0 = 0; c0 < kMlpHidden; c0 += 64) {
            uint32_t v[64];
            tc_ld32_nowait(tmem_row + c0, v);
            tc_ld32_nowait(tmem_row + c0 + 32, v + 32);
            tc_ld_wait();
            if (in) {
                const __nv_bfloat16* hrow = H + r * kMlpHidden + c0;
#pragma unroll
                for (int g = 0; g < 64; g += 8) {
                    const uint4 hv = *reinterpret_cast<const uint4*>(hrow + g);
                    const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&hv);
                    uint32_t pk[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const float a = __bfloat162float(hb[2 * j]) > 0.f ? __uint_as_float(v[g + 2 * j]) : 0.f;
                        const float b = __bfloat162float(hb[2 * j + 1]) > 0.f ? __uint_as_float(v[g + 2 * j + 1]) : 0.f;
                        __nv_bfloat162 p2 = __floats2bfloat162_rn(a, b);
                        pk[j] = *reinterpret_cast<uint32_t*>(&p2);
                    }
                    *reinterpret_cast<uint4*>(dH + r * kMlpHidden + c0 + g) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
            }
        }
        tc_fence_before();
        __syncthreads();  // every TMEM read done before the next tile's MMAs overwrite D
        tc_fence_after();
    }
    if (!ok) {
        if (tid == 0 && err) atomicCAS(err, 0, LB_ERR_TIMEOUT);
        tc_wait(&sm.bar, phase ^ 1u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMlpHidden) : "memory");
}

// ---------------------------------------------------------------------------
// Weight gradients: D[m][n] = sum_r A[r][m] B[r][n] over the rows of a chunk,
// m < 128, n < NB (A row-major [rows][128] bf16, B row-major [rows][nb], bf16
// or FP32).  The reduction over rows is the K dimension of the UMMA: each
// 128-row slice is staged transposed -- A^T [128][128 rows] and B^T [NB][128
// rows], K-major core matrices -- and accumulated in TMEM; at the end every
// block adds its D into the FP32 gradient with atomics, out[m ms + n ns].
// ---------------------------------------------------------------------------
template <int NB>
struct DwSmem {
    __nv_bfloat16 a[kMlpHidden * kTcRows];  // A^T: [m][r]
    __nv_bfloat16 b[NB * kTcRows];          // B^T: [n][r]
    uint64_t bar;
    uint32_t tmem;
};

template <int NB>
__host__ __device__ constexpr int dw_tmem_cols() { return NB <= 32 ? 32 : (NB <= 64 ? 64 : (NB <= 128 ? 128 : 256)); }

template <int NB, class BT>
__global__ void __launch_bounds__(kTcThreads) k_mlp_dw_tc(const __nv_bfloat16* __restrict__ A,
                                                          const BT* __restrict__ B, int nb, int64_t rows,
                                                          int64_t rows_per_block, float* __restrict__ out, int ms,
                                                          int ns, int32_t* err)
{
    static_assert(NB % 16 == 0 && NB >= 16 && NB <= 256, "UMMA N for M = 128");
    using Sm = DwSmem<NB>;
    constexpr int kCols = dw_tmem_cols<NB>();
    extern __shared__ __align__(128) unsigned char dw_smem_raw[];
    Sm& sm = *reinterpret_cast<Sm*>(dw_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sm.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sm.tmem)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;
    const uint32_t idesc = tc_idesc(kTcRows, NB);
    const uint32_t aa = su32(sm.a), ab = su32(sm.b);
    constexpr uint32_t kLbo = 128, kSbo = (kTcRows / 8) * 128;  // K = 128 rows per slice
    uint32_t phase = 0;
    bool ok = true, any = false;
    const int64_t r_beg = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r_end = r_beg + rows_per_block < rows ? r_beg + rows_per_block : rows;
    for (int64_t r0 = r_beg; r0 < r_end && ok; r0 += kTcRows) {
        // A^T: thread t takes rows r0 + (t % 128) ... one row per thread, 128 m values,
        // scattered into the [m][r] core layout (zero past the chunk's end)
        {
            const int rr = tid;
            const bool in = r0 + rr < r_end;
            const __nv_bfloat16* arow = A + (r0 + rr) * kMlpHidden;
#pragma unroll 4
            for (int m0 = 0; m0 < kMlpHidden; m0 += 8) {
                uint4 v = in ? *reinterpret_cast<const uint4*>(arow + m0) : make_uint4(0u, 0u, 0u, 0u);
                const __nv_bfloat16* vb = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
                for (int j = 0; j < 8; j++) sm.a[core_off(m0 + j, rr, kTcRows)] = vb[j];
            }
            for (int n = 0; n < NB; n++) {
                const float x = in && n < nb ? (float)B[(r0 + rr) * nb + n] : 0.f;
                sm.b[core_off(n, rr, kTcRows)] = __float2bfloat16_rn(x);
            }
        }
        proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            for (int ks = 0; ks < kTcRows / 16; ks++)
                tc_mma(tmem, tc_desc(aa + ks * 256, kLbo, kSbo), tc_desc(ab + ks * 256, kLbo, kSbo), idesc,
                       any || ks > 0);
            tc_commit(&sm.bar);
        }
        any = true;
        const bool arrived = tc_wait(&sm.bar, phase);  // the slice's operands are read before they are restaged
        phase ^= 1u;
        if (!__syncthreads_and(arrived)) ok = false;
        tc_fence_after();
    }
    if (ok && any) {
        const uint32_t tmem_row = tmem + ((uint32_t)(32 * warp) << 16);
        const int m = tid;
#pragma unroll
        for (int c0 = 0; c0 < NB; c0 += 16) {
            uint32_t v[16];
            tc_ld16_nowait(tmem_row + c0, v);
            tc_ld_wait();
#pragma unroll
            for (int j = 0; j < 16; j++)
                if (c0 + j < nb) atomicAdd(out + (int64_t)m * ms + (int64_t)(c0 + j) * ns, __uint_as_float(v[j]));
        }
    }
    if (!ok) {
        if (tid == 0 && err) atomicCAS(err, 0, LB_ERR_TIMEOUT);
        tc_wait(&sm.bar, phase ^ 1u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// bias gradients: db[o] += sum over a chunk of rows of Z[r][o]
template <class ZT>
__global__ void k_mlp_col_sum(const ZT* __restrict__ Z, int nz, int64_t rows, int64_t rows_per_block, float* db)
{
    const int o = threadIdx.x;
    if (o >= nz) return;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = r0 + rows_per_block < rows ? r0 + rows_per_block : rows;
    float acc = 0.f;
    for (int64_t r = r0; r < r1; r++) acc += (float)Z[r * nz + o];
    atomicAdd(db + o, acc);
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <int KZ, class ZT>
cudaError_t dh_tc(const ZT* dZ, int nz, int64_t rows, const __nv_bfloat16* Wt, const __nv_bfloat16* H,
                  __nv_bfloat16* dH, cudaStream_t s)
{
    static int attr_done[kMaxDevices] = {};
    const int smem = (int)sizeof(DhSmem<KZ>);
    cudaError_t e = smem_attr_per_device(k_mlp_dh_tc<KZ, ZT>, smem, attr_done);
    if (e != cudaSuccess) return e;
    int64_t blocks = (rows + kTcRows - 1) / kTcRows;
    if (blocks > 2LL * sm_count()) blocks = 2LL * sm_count();
    if (blocks < 1) return cudaSuccess;
    k_mlp_dh_tc<KZ, ZT><<<(unsigned)blocks, kTcThreads, smem, s>>>(dZ, nz, rows, Wt, H, dH, nullptr);
    return cudaGetLastError();
}

template <int NB, class BT>
cudaError_t dw_tc(const __nv_bfloat16* A, const BT* B, int nb, int64_t rows, float* out, int ms, int ns,
                  cudaStream_t s)
{
    static int attr_done[kMaxDevices] = {};
    const int smem = (int)sizeof(DwSmem<NB>);
    cudaError_t e = smem_attr_per_device(k_mlp_dw_tc<NB, BT>, smem, attr_done);
    if (e != cudaSuccess) return e;
    // chunks of whole 128-row slices, at most 32 blocks (each adds its whole
    // D into the gradient with atomics)
    const int64_t slices = (rows + kTcRows - 1) / kTcRows;
    int64_t per = (slices + 31) / 32;
    if (per < 1) per = 1;
    const int64_t rpb = per * kTcRows;
    const int64_t blocks = (rows + rpb - 1) / rpb;
    if (blocks < 1) return cudaSuccess;
    k_mlp_dw_tc<NB, BT><<<(unsigned)blocks, kTcThreads, smem, s>>>(A, B, nb, rows, rpb, out, ms, ns, nullptr);
    return cudaGetLastError();
}

template <class ZT>
cudaError_t col_sum(const ZT* Z, int nz, int64_t rows, float* db, cudaStream_t s)
{
    const int64_t rpb = 256;
    const int64_t blocks = (rows + rpb - 1) / rpb;
    if (blocks < 1) return cudaSuccess;
    k_mlp_col_sum<ZT><<<(unsigned)blocks, 128, 0, s>>>(Z, nz, rows, rpb, db);
    return cudaGetLastError();
}

template <int NOUT>
cudaError_t grad_tc(const void* X, int64_t rows, const unsigned char* params, const MlpLayout& L, float* Y,
                    __nv_bfloat16* H1, __nv_bfloat16* H2, float* dY, __nv_bfloat16* dH2, __nv_bfloat16* dH1,
                    float* grad, cudaStream_t s)
{
    constexpr int NP = pad16(NOUT);
    const __nv_bfloat16* W2t = reinterpret_cast<const __nv_bfloat16*>(params + L.w2);
    const __nv_bfloat16* W3t = reinterpret_cast<const __nv_bfloat16*>(params + L.w3);
    const __nv_bfloat16* Xb = reinterpret_cast<const __nv_bfloat16*>(X);
    cudaError_t e;
    // layer 3: dW3[i][o] = sum_r H2[r][i] dY[r][o]; db3 = sum_r dY[r][o]
    if ((e = dw_tc<NP, float>(H2, dY, NOUT, rows, grad + L.m_w3, NOUT, 1, s)) != cudaSuccess) return e;
    if ((e = col_sum<float>(dY, NOUT, rows, grad + L.m_b3, s)) != cudaSuccess) return e;
    // dH2 = (dY W3^T) [H2 > 0]
    if ((e = dh_tc<NP, float>(dY, NOUT, rows, W3t, H2, dH2, s)) != cudaSuccess) return e;
    // layer 2
    if ((e = dw_tc<kMlpHidden, __nv_bfloat16>(H1, dH2, kMlpHidden, rows, grad + L.m_w2, kMlpHidden, 1, s)) !=
        cudaSuccess)
        return e;
    if ((e = col_sum<__nv_bfloat16>(dH2, kMlpHidden, rows, grad + L.m_b2, s)) != cudaSuccess) return e;
    if ((e = dh_tc<kMlpHidden, __nv_bfloat16>(dH2, kMlpHidden, rows, W2t, H1, dH1, s)) != cudaSuccess) return e;
    // layer 1: dW1[f][o] = sum_r X[r][f] dH1[r][o], formed as D[o][f] (M = 128 hidden units)
    if ((e = dw_tc<kMlpIn, __nv_bfloat16>(dH1, Xb, kMlpIn, rows, grad + L.m_w1, 1, kMlpHidden, s)) != cudaSuccess)
        return e;
    return col_sum<__nv_bfloat16>(dH1, kMlpHidden, rows, grad + L.m_b1, s);
}

}  // namespace

cudaError_t mlp_forward_tc(const void* X, int64_t rows, const void* params, int K, float* Y, int32_t* err,
                           cudaStream_t s, int64_t col_stride)
{
    const MlpLayout L = mlp_layout(K);
    if (K == 16) return forward_tc<48, false>(X, rows, params, L, Y, col_stride, err, s);
    if (K == 8) return forward_tc<24, false>(X, rows, params, L, Y, col_stride, err, s);
    return cudaErrorInvalidValue;
}

cudaError_t mlp_forward_save_tc(const void* X, int64_t rows, const void* params, int K, float* Y, void* H1, void* H2,
                                cudaStream_t s)
{
    const MlpLayout L = mlp_layout(K);
    __nv_bfloat16* h1 = reinterpret_cast<__nv_bfloat16*>(H1);
    __nv_bfloat16* h2 = reinterpret_cast<__nv_bfloat16*>(H2);
    if (K == 16) return forward_tc<48, true>(X, rows, params, L, Y, 0, nullptr, s, h1, h2);
    if (K == 8) return forward_tc<24, true>(X, rows, params, L, Y, 0, nullptr, s, h1, h2);
    return cudaErrorInvalidValue;
}

cudaError_t mlp_backward_tc(const void* X, int64_t rows, const void* params, int K, const void* H1, const void* H2,
                            const float* dY, void* dH2, void* dH1, float* grad, cudaStream_t s)
{
    const MlpLayout L = mlp_layout(K);
    const unsigned char* P = reinterpret_cast<const unsigned char*>(params);
    auto b = [](const void* p) { return reinterpret_cast<__nv_bfloat16*>(const_cast<void*>(p)); };
    if (K == 16)
        return grad_tc<48>(X, rows, P, L, nullptr, b(H1), b(H2), const_cast<float*>(dY), b(dH2), b(dH1), grad, s);
    if (K == 8)
        return grad_tc<24>(X, rows, P, L, nullptr, b(H1), b(H2), const_cast<float*>(dY), b(dH2), b(dH1), grad, s);
    return cudaErrorInvalidValue;
}

}  // namespace lbt
