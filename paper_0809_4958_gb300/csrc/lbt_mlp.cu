// Learned boundary upsampler: a small MLP that predicts, per face site and
// coarse interval, the residual of the boundary velocity over the cubic
// Hermite interpolant at the K substeps (the paper interpolates the DNS
// boundary linearly between samples, Sec. 3; the residual network is an
// added form).  Network: 24 features (padded to 32) -> 128 -> 128 -> 3K,
// ReLU, BF16 weights and activations on the tensor cores with FP32
// accumulation.  Training runs on the GPU with the kernels below: the same
// BF16 forward, an FP32 backward and Adam on FP32 master weights.
//
// Layouts
//   feature matrix X: bf16 [rows][32], row = (f E + q) E + p per box
//   output Y:         f32  [rows][3K], Y[row][3 (s-1) + c] = residual / u_max
//   inference params: bf16 W1t [128][32], W2t [128][128], W3t [3K][128]
//                     (out-major), f32 b1 [128], b2 [128], b3 [3K]
//   master params:    f32 W1 [32][128], b1, W2 [128][128], b2, W3 [128][3K], b3
//                     (in-major, as in the CPU oracle)
#include <cuda_bf16.h>

#include <cstdio>

#include "lbt_device.cuh"
#include "lbt_mlp.h"
#include "lbt_internal.h"

namespace lbt {

// ---------------------------------------------------------------------------
// parameter layouts
// ---------------------------------------------------------------------------
static inline size_t al256(size_t v) { return (v + 255) / 256 * 256; }

MlpLayout mlp_layout(int K)
{
    MlpLayout L{};
    L.nout = 3 * K;
    size_t o = 0;
    L.w1 = o; o = al256(o + 2 * (size_t)kMlpHidden * kMlpIn);
    L.w2 = o; o = al256(o + 2 * (size_t)kMlpHidden * kMlpHidden);
    L.w3 = o; o = al256(o + 2 * (size_t)L.nout * kMlpHidden);
    L.b1 = o; o = al256(o + 4 * (size_t)kMlpHidden);
    L.b2 = o; o = al256(o + 4 * (size_t)kMlpHidden);
    L.b3 = o; o = al256(o + 4 * (size_t)L.nout);
    L.bytes = o;
    // master (float offsets)
    L.m_w1 = 0;
    L.m_b1 = L.m_w1 + kMlpIn * kMlpHidden;
    L.m_w2 = L.m_b1 + kMlpHidden;
    L.m_b2 = L.m_w2 + kMlpHidden * kMlpHidden;
    L.m_w3 = L.m_b2 + kMlpHidden;
    L.m_b3 = L.m_w3 + kMlpHidden * L.nout;
    L.nmaster = L.m_b3 + L.nout;
    return L;
}

// ---------------------------------------------------------------------------
// tensor-core helpers (mma.sync m16n8k16, bf16 inputs, f32 accumulators)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// shared-memory row strides (bf16 elements), padded so that the eight
// groups of a warp hit distinct banks when loading B fragments
constexpr int kLd1 = kMlpIn + 8;
constexpr int kLd2 = kMlpHidden + 8;

template <int NOUT>
struct MlpSmem {
    __nv_bfloat16 w1[kMlpHidden * kLd1];
    __nv_bfloat16 w2[kMlpHidden * kLd2];
    __nv_bfloat16 w3[NOUT * kLd2];
    float b1[kMlpHidden], b2[kMlpHidden], b3[NOUT];
};

// Hidden layer from the accumulators: bias, ReLU, bf16, packed as the A
// fragments of the next layer (the C fragment of n-tiles 2k and 2k+1 is the A
// fragment of k-step k).  Optionally stores the activations (as floats).
__device__ __forceinline__ void hidden_to_a(const float acc[16][4], const float* bias, uint32_t a[8][4], float* save,
                                            int64_t r0, int64_t rows, int g, int t)
{
#pragma unroll
    for (int ks = 0; ks < 8; ks++) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int nt = 2 * ks + h;
            const int col = 8 * nt + 2 * t;
            const float v0 = bf16_round(fmaxf(acc[nt][0] + bias[col], 0.f));
            const float v1 = bf16_round(fmaxf(acc[nt][1] + bias[col + 1], 0.f));
            const float v2 = bf16_round(fmaxf(acc[nt][2] + bias[col], 0.f));
            const float v3 = bf16_round(fmaxf(acc[nt][3] + bias[col + 1], 0.f));
            a[ks][2 * h + 0] = pack_bf16(v0, v1);
            a[ks][2 * h + 1] = pack_bf16(v2, v3);
            if (save) {
                if (r0 + g < rows) *reinterpret_cast<float2*>(save + (r0 + g) * kMlpHidden + col) = make_float2(v0, v1);
                if (r0 + g + 8 < rows)
                    *reinterpret_cast<float2*>(save + (r0 + g + 8) * kMlpHidden + col) = make_float2(v2, v3);
            }
        }
    }
}

// Fused forward of the three layers: one warp per 16 rows, weights staged
// once per block in shared memory, blocks stride over the row tiles.
template <int NOUT, bool SAVE>
__global__ void __launch_bounds__(256) k_mlp_forward(const __nv_bfloat16* __restrict__ X, int64_t rows,
                                                     const unsigned char* __restrict__ params, MlpLayout L,
                                                     float* __restrict__ Y, float* H1, float* H2)
{
    extern __shared__ __align__(16) unsigned char mlp_smem_raw[];
    MlpSmem<NOUT>& sm = *reinterpret_cast<MlpSmem<NOUT>*>(mlp_smem_raw);
    const __nv_bfloat16* w1 = reinterpret_cast<const __nv_bfloat16*>(params + L.w1);
    const __nv_bfloat16* w2 = reinterpret_cast<const __nv_bfloat16*>(params + L.w2);
    const __nv_bfloat16* w3 = reinterpret_cast<const __nv_bfloat16*>(params + L.w3);
    for (int i = threadIdx.x; i < kMlpHidden * kMlpIn; i += blockDim.x)
        sm.w1[(i / kMlpIn) * kLd1 + i % kMlpIn] = w1[i];
    for (int i = threadIdx.x; i < kMlpHidden * kMlpHidden; i += blockDim.x)
        sm.w2[(i / kMlpHidden) * kLd2 + i % kMlpHidden] = w2[i];
    for (int i = threadIdx.x; i < NOUT * kMlpHidden; i += blockDim.x)
        sm.w3[(i / kMlpHidden) * kLd2 + i % kMlpHidden] = w3[i];
    for (int i = threadIdx.x; i < kMlpHidden; i += blockDim.x) {
        sm.b1[i] = reinterpret_cast<const float*>(params + L.b1)[i];
        sm.b2[i] = reinterpret_cast<const float*>(params + L.b2)[i];
    }
    for (int i = threadIdx.x; i < NOUT; i += blockDim.x) sm.b3[i] = reinterpret_cast<const float*>(params + L.b3)[i];
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t ntiles = (rows + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * 8 + warp; tile < ntiles; tile += (int64_t)gridDim.x * 8) {
        const int64_t r0 = tile * 16;
        // layer 1: A fragments straight from the feature matrix
        uint32_t a1[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            const int c = 16 * ks + 2 * t;
            const uint32_t* x0 = reinterpret_cast<const uint32_t*>(X + (r0 + g) * kMlpIn + c);
            const uint32_t* x8 = reinterpret_cast<const uint32_t*>(X + (r0 + g + 8) * kMlpIn + c);
            const bool v0 = r0 + g < rows, v8 = r0 + g + 8 < rows;
            a1[ks][0] = v0 ? x0[0] : 0u;
            a1[ks][1] = v8 ? x8[0] : 0u;
            a1[ks][2] = v0 ? x0[4] : 0u;  // columns c + 8
            a1[ks][3] = v8 ? x8[4] : 0u;
        }
        float acc[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; nt++) {
            acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
            for (int ks = 0; ks < 2; ks++) {
                const uint32_t* wb = reinterpret_cast<const uint32_t*>(sm.w1 + (8 * nt + g) * kLd1 + 16 * ks + 2 * t);
                mma_16816(acc[nt], a1[ks], wb[0], wb[4]);
            }
        }
        uint32_t a2[8][4];
        hidden_to_a(acc, sm.b1, a2, SAVE ? H1 : nullptr, r0, rows, g, t);
        // layer 2
#pragma unroll
        for (int nt = 0; nt < 16; nt++) {
            acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
            for (int ks = 0; ks < 8; ks++) {
                const uint32_t* wb = reinterpret_cast<const uint32_t*>(sm.w2 + (8 * nt + g) * kLd2 + 16 * ks + 2 * t);
                mma_16816(acc[nt], a2[ks], wb[0], wb[4]);
            }
        }
        uint32_t a3[8][4];
        hidden_to_a(acc, sm.b2, a3, SAVE ? H2 : nullptr, r0, rows, g, t);
        // layer 3 and the output
#pragma unroll
        for (int nt = 0; nt < NOUT / 8; nt++) {
            float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 8; ks++) {
                const uint32_t* wb = reinterpret_cast<const uint32_t*>(sm.w3 + (8 * nt + g) * kLd2 + 16 * ks + 2 * t);
                mma_16816(o, a3[ks], wb[0], wb[4]);
            }
            const int col = 8 * nt + 2 * t;
            if (r0 + g < rows)
                *reinterpret_cast<float2*>(Y + (r0 + g) * NOUT + col) = make_float2(o[0] + sm.b3[col], o[1] + sm.b3[col + 1]);
            if (r0 + g + 8 < rows)
                *reinterpret_cast<float2*>(Y + (r0 + g + 8) * NOUT + col) =
                    make_float2(o[2] + sm.b3[col], o[3] + sm.b3[col + 1]);
        }
    }
}

// ---------------------------------------------------------------------------
// features of interval j of one face set: samples j-1 (clamped), j, j+1, j+2
// and in-face differences at j and j+1, all divided by u_max, as bf16
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ float face_val(const R* s, int E, int f, int c, int q, int p)
{
    return (float)s[(((int64_t)f * 3 + c) * E + q) * E + p];
}

template <class R>
__device__ void features_row(const R* const smp[4], int E, float inv_umax, int64_t row, __nv_bfloat16* out)
{
    const int p = (int)(row % E), q = (int)((row / E) % E), f = (int)(row / ((int64_t)E * E));
    float v[kMlpIn];
    int k = 0;
    for (int a = 0; a < 4; a++)
        for (int c = 0; c < 3; c++) v[k++] = face_val(smp[a], E, f, c, q, p) * inv_umax;
    const int pm = p > 0 ? p - 1 : p, pp = p < E - 1 ? p + 1 : p;
    const int qm = q > 0 ? q - 1 : q, qp = q < E - 1 ? q + 1 : q;
    const float sp = (pp - pm) == 2 ? 0.5f : 1.0f, sq = (qp - qm) == 2 ? 0.5f : 1.0f;
    for (int a = 1; a <= 2; a++) {
        for (int c = 0; c < 3; c++) v[k++] = (face_val(smp[a], E, f, c, q, pp) - face_val(smp[a], E, f, c, q, pm)) * sp * inv_umax;
        for (int c = 0; c < 3; c++) v[k++] = (face_val(smp[a], E, f, c, qp, p) - face_val(smp[a], E, f, c, qm, p)) * sq * inv_umax;
    }
    for (; k < kMlpIn; k++) v[k] = 0.f;
    // the row's 64 bytes as four 16-byte stores (rows are 64-byte aligned)
    uint4* o = reinterpret_cast<uint4*>(out);
#pragma unroll
    for (int q4 = 0; q4 < kMlpIn / 8; q4++) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * q4 + 2 * h], v[8 * q4 + 2 * h + 1]);
            w[h] = *reinterpret_cast<const uint32_t*>(&b2);
        }
        o[q4] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// One launch for several face sets: set b has rows [row_off[b], row_off[b] +
// 6 E_b^2) and its four samples at smp[4 b .. 4 b + 3].
template <class R>
__global__ void k_mlp_features(const MlpFeatureSet* sets, int nsets, int64_t total_rows, float inv_umax,
                               __nv_bfloat16* X)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < total_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nsets - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sets[mid].row_off <= r) lo = mid;
            else hi = mid - 1;
        }
        const MlpFeatureSet& s = sets[lo];
        const R* smp[4] = {reinterpret_cast<const R*>(s.smp[0]), reinterpret_cast<const R*>(s.smp[1]),
                           reinterpret_cast<const R*>(s.smp[2]), reinterpret_cast<const R*>(s.smp[3])};
        features_row<R>(smp, s.E, inv_umax, r - s.row_off, X + r * kMlpIn);
    }
}

template <class R>
__global__ void k_mlp_features_one(MlpFeatureSet set, float inv_umax, __nv_bfloat16* X)
{
    const int64_t rows = 6LL * set.E * set.E;
    const R* smp[4] = {reinterpret_cast<const R*>(set.smp[0]), reinterpret_cast<const R*>(set.smp[1]),
                       reinterpret_cast<const R*>(set.smp[2]), reinterpret_cast<const R*>(set.smp[3])};
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
        features_row<R>(smp, set.E, inv_umax, r, X + r * kMlpIn);
}

// Targets of interval j: (fine velocity at jK + s - Hermite) / u_max.
// fine: [K + 1][6][3][E][E] at t = jK .. jK + K (only 1..K are used).
template <class R>
__global__ void k_mlp_targets(const R* s_prev, const R* s0, const R* s1, const R* s2, const R* fine, int E, int K,
                              int first_interval, float inv_umax, float* T)
{
    const int64_t rows = 6LL * E * E;
    const int64_t fe = 3LL * E * E;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(r % E), q = (int)((r / E) % E), f = (int)(r / ((int64_t)E * E));
        for (int s = 1; s <= K; s++) {
            const float th = (float)s / (float)K;
            const float h00 = 2 * th * th * th - 3 * th * th + 1, h10 = th * th * th - 2 * th * th + th;
            const float h01 = -2 * th * th * th + 3 * th * th, h11 = th * th * th - th * th;
            for (int c = 0; c < 3; c++) {
                const int64_t o = ((int64_t)f * 3 + c) * E * E + (int64_t)q * E + p;
                const float u0 = (float)s0[o], u1 = (float)s1[o], u2 = (float)s2[o];
                const float m0 = first_interval ? (u1 - u0) : 0.5f * (u1 - (float)s_prev[o]);
                const float m1 = 0.5f * (u2 - u0);
                const float herm = h00 * u0 + h10 * m0 + h01 * u1 + h11 * m1;
                T[r * 3 * K + 3 * (s - 1) + c] = ((float)fine[(int64_t)s * 6 * fe + o] - herm) * inv_umax;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// training: FP32 backward and Adam
// ---------------------------------------------------------------------------
// dY = 2 (Y - T) / (rows nout); loss += sum (Y - T)^2 / (rows nout)
__global__ void k_mse(const float* Y, const float* T, int64_t n, float scale, float* dY, double* loss)
{
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        dY[i] = 2.f * d * scale;
        acc += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc * scale);
}

// dW[i][o] += sum_r Hin[r][i] dZ[r][o] and db[o] += sum_r dZ[r][o] over a
// chunk of rows; 32 x 32 output tile per block, 256 threads x 4 outputs.
template <class TIN>
__global__ void __launch_bounds__(256) k_grad_w(const TIN* Hin, int nin, const float* dZ, int nout, int64_t rows,
                                                int64_t rows_per_block, float* dW, float* db)
{
    __shared__ float sH[64][33];
    __shared__ float sZ[64][33];
    const int i0 = blockIdx.x * 32, o0 = blockIdx.y * 32;
    const int64_t rbeg = blockIdx.z * rows_per_block;
    const int64_t rend = min(rows, rbeg + rows_per_block);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty 0..7: outputs i = i0 + ty + 8 k
    float acc[4] = {0, 0, 0, 0};
    float bacc = 0.f;
    for (int64_t r = rbeg; r < rend; r += 64) {
        for (int e = threadIdx.x; e < 64 * 32; e += 256) {
            const int rr = e >> 5, cc = e & 31;
            const int64_t row = r + rr;
            sH[rr][cc] = (row < rend && i0 + cc < nin) ? (float)Hin[row * nin + i0 + cc] : 0.f;
            sZ[rr][cc] = (row < rend && o0 + cc < nout) ? dZ[row * nout + o0 + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < 64; rr++) {
            const float z = sZ[rr][tx];
#pragma unroll
            for (int k = 0; k < 4; k++) acc[k] += sH[rr][ty + 8 * k] * z;
            if (ty == 0 && blockIdx.x == 0) bacc += z;
        }
        __syncthreads();
    }
    if (o0 + tx < nout) {
        for (int k = 0; k < 4; k++)
            if (i0 + ty + 8 * k < nin) atomicAdd(&dW[(i0 + ty + 8 * k) * nout + o0 + tx], acc[k]);
        if (ty == 0 && blockIdx.x == 0 && db) atomicAdd(&db[o0 + tx], bacc);
    }
}

// dHin[r][i] = (sum_o dZ[r][o] W[i][o]) * (Hin[r][i] > 0), W taken from the
// bf16 out-major inference weights (the ones the forward used).
__global__ void k_grad_h(const float* dZ, int nout, const __nv_bfloat16* Wt, int nin, const float* Hin, int64_t rows,
                         float* dH)
{
    const int64_t n = rows * nin;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / nin;
        const int i = (int)(e - r * nin);
        float s = 0.f;
        if (Hin[e] > 0.f)
            for (int o = 0; o < nout; o++) s += dZ[r * nout + o] * __bfloat162float(Wt[o * nin + i]);
        dH[e] = s;
    }
}

// Adam on the master weights, then the bf16 / f32 inference copy.
__global__ void k_adam(float* master, float* m, float* v, const float* grad, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        master[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_export(const float* master, MlpLayout L, unsigned char* params)
{
    __nv_bfloat16* w1 = reinterpret_cast<__nv_bfloat16*>(params + L.w1);
    __nv_bfloat16* w2 = reinterpret_cast<__nv_bfloat16*>(params + L.w2);
    __nv_bfloat16* w3 = reinterpret_cast<__nv_bfloat16*>(params + L.w3);
    float* b1 = reinterpret_cast<float*>(params + L.b1);
    float* b2 = reinterpret_cast<float*>(params + L.b2);
    float* b3 = reinterpret_cast<float*>(params + L.b3);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int e = tid; e < kMlpHidden * kMlpIn; e += nt) {  // W1t[o][i] = W1[i][o]
        const int o = e / kMlpIn, i = e % kMlpIn;
        w1[e] = __float2bfloat16_rn(master[L.m_w1 + i * kMlpHidden + o]);
    }
    for (int e = tid; e < kMlpHidden * kMlpHidden; e += nt) {
        const int o = e / kMlpHidden, i = e % kMlpHidden;
        w2[e] = __float2bfloat16_rn(master[L.m_w2 + i * kMlpHidden + o]);
    }
    for (int e = tid; e < L.nout * kMlpHidden; e += nt) {
        const int o = e / kMlpHidden, i = e % kMlpHidden;
        w3[e] = __float2bfloat16_rn(master[L.m_w3 + i * L.nout + o]);
    }
    for (int e = tid; e < kMlpHidden; e += nt) {
        b1[e] = master[L.m_b1 + e];
        b2[e] = master[L.m_b2 + e];
    }
    for (int e = tid; e < L.nout; e += nt) b3[e] = master[L.m_b3 + e];
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int grid_cap(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

template <int NOUT, bool SAVE>
static cudaError_t forward_t(const void* X, int64_t rows, const void* params, const MlpLayout& L, float* Y, float* H1,
                             float* H2, cudaStream_t s)
{
    static int attr_done[kMaxDevices] = {};  // per instantiation and device
    const int smem = (int)sizeof(MlpSmem<NOUT>);
    cudaError_t e = smem_attr_per_device(k_mlp_forward<NOUT, SAVE>, smem, attr_done);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (rows + 15) / 16;
    int64_t blocks = (tiles + 7) / 8;
    if (blocks > 152 * 2) blocks = 152 * 2;
    if (blocks < 1) blocks = 1;
    k_mlp_forward<NOUT, SAVE><<<(unsigned)blocks, 256, smem, s>>>(reinterpret_cast<const __nv_bfloat16*>(X), rows,
                                                                  reinterpret_cast<const unsigned char*>(params), L, Y,
                                                                  H1, H2);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const void* X, int64_t rows, const void* params, int K, float* Y, float* H1, float* H2,
                        cudaStream_t s)
{
    const MlpLayout L = mlp_layout(K);
    const bool save = H1 != nullptr;
    if (!save) return mlp_forward_tc(X, rows, params, K, Y, nullptr, s);  // inference: tcgen05
    if (K == 16) return save ? forward_t<48, true>(X, rows, params, L, Y, H1, H2, s) : forward_t<48, false>(X, rows, params, L, Y, H1, H2, s);
    if (K == 8) return save ? forward_t<24, true>(X, rows, params, L, Y, H1, H2, s) : forward_t<24, false>(X, rows, params, L, Y, H1, H2, s);
    return cudaErrorInvalidValue;
}

cudaError_t mlp_features(const MlpFeatureSet* sets_dev, int nsets, int64_t total_rows, double u_max, int real_f64,
                         void* X, cudaStream_t s)
{
    const float inv = (float)(1.0 / u_max);
    if (real_f64)
        k_mlp_features<double><<<grid_cap(total_rows, 256), 256, 0, s>>>(sets_dev, nsets, total_rows, inv,
                                                                         reinterpret_cast<__nv_bfloat16*>(X));
    else
        k_mlp_features<float><<<grid_cap(total_rows, 256), 256, 0, s>>>(sets_dev, nsets, total_rows, inv,
                                                                        reinterpret_cast<__nv_bfloat16*>(X));
    return cudaGetLastError();
}

cudaError_t mlp_features_one(const MlpFeatureSet& set, double u_max, int real_f64, void* X, cudaStream_t s)
{
    const float inv = (float)(1.0 / u_max);
    const int64_t rows = 6LL * set.E * set.E;
    if (real_f64)
        k_mlp_features_one<double><<<grid_cap(rows, 256), 256, 0, s>>>(set, inv, reinterpret_cast<__nv_bfloat16*>(X));
    else
        k_mlp_features_one<float><<<grid_cap(rows, 256), 256, 0, s>>>(set, inv, reinterpret_cast<__nv_bfloat16*>(X));
    return cudaGetLastError();
}

cudaError_t mlp_targets(const void* const smp[4], const void* fine, int E, int K, int first_interval, double u_max,
                        int real_f64, float* T, cudaStream_t s)
{
    const float inv = (float)(kMlpOutDiv / u_max);  // targets in the output unit
    const int64_t rows = 6LL * E * E;
    if (real_f64)
        k_mlp_targets<double><<<grid_cap(rows, 256), 256, 0, s>>>(
            (const double*)smp[0], (const double*)smp[1], (const double*)smp[2], (const double*)smp[3],
            (const double*)fine, E, K, first_interval, inv, T);
    else
        k_mlp_targets<float><<<grid_cap(rows, 256), 256, 0, s>>>(
            (const float*)smp[0], (const float*)smp[1], (const float*)smp[2], (const float*)smp[3], (const float*)fine,
            E, K, first_interval, inv, T);
    return cudaGetLastError();
}

// Training workspace layout (float offsets), batch rows B.
MlpTrain mlp_train_layout(int K, int64_t B)
{
    MlpTrain W{};
    W.L = mlp_layout(K);
    W.K = K;
    W.batch = B;
    const int64_t P = W.L.nmaster;
    size_t o = 0;
    auto take = [&](size_t floats) {
        const size_t at = o;
        o = al256((o + floats) * 4) / 4;
        return at;
    };
    W.master = take(P);
    W.m = take(P);
    W.v = take(P);
    W.grad = take(P);
    W.h1 = take(B * kMlpHidden);
    W.h2 = take(B * kMlpHidden);
    W.y = take(B * W.L.nout);
    W.dy = take(B * W.L.nout);
    W.dh2 = take(B * kMlpHidden);
    W.dh1 = take(B * kMlpHidden);
    W.loss = take(2);  // one double
    W.params_byte = o * 4;
    W.bytes = al256(W.params_byte + W.L.bytes);
    return W;
}

cudaError_t mlp_grad(unsigned char* ws, const MlpTrain& W, const void* X, const float* T, int64_t rows, cudaStream_t s)
{
    float* f = reinterpret_cast<float*>(ws);
    const MlpLayout& L = W.L;
    const unsigned char* params = ws + W.params_byte;
    cudaError_t e = mlp_forward(X, rows, params, W.K, f + W.y, f + W.h1, f + W.h2, s);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(f + W.grad, 0, sizeof(float) * L.nmaster, s);
    cudaMemsetAsync(f + W.loss, 0, sizeof(double), s);
    const int64_t ny = rows * L.nout;
    k_mse<<<grid_cap(ny, 256), 256, 0, s>>>(f + W.y, T, ny, 1.0f / (float)ny, f + W.dy,
                                            reinterpret_cast<double*>(f + W.loss));
    const int64_t rpb = 1024;
    const unsigned zsplit = (unsigned)((rows + rpb - 1) / rpb);
    // layer 3
    k_grad_w<float><<<dim3(kMlpHidden / 32, (L.nout + 31) / 32, zsplit), 256, 0, s>>>(
        f + W.h2, kMlpHidden, f + W.dy, L.nout, rows, rpb, f + W.grad + L.m_w3, f + W.grad + L.m_b3);
    k_grad_h<<<grid_cap(rows * kMlpHidden, 256), 256, 0, s>>>(
        f + W.dy, L.nout, reinterpret_cast<const __nv_bfloat16*>(params + L.w3), kMlpHidden, f + W.h2, rows, f + W.dh2);
    // layer 2
    k_grad_w<float><<<dim3(kMlpHidden / 32, kMlpHidden / 32, zsplit), 256, 0, s>>>(
        f + W.h1, kMlpHidden, f + W.dh2, kMlpHidden, rows, rpb, f + W.grad + L.m_w2, f + W.grad + L.m_b2);
    k_grad_h<<<grid_cap(rows * kMlpHidden, 256), 256, 0, s>>>(
        f + W.dh2, kMlpHidden, reinterpret_cast<const __nv_bfloat16*>(params + L.w2), kMlpHidden, f + W.h1, rows,
        f + W.dh1);
    // layer 1 (input: the bf16 features)
    k_grad_w<__nv_bfloat16><<<dim3(kMlpIn / 32, kMlpHidden / 32, zsplit), 256, 0, s>>>(
        reinterpret_cast<const __nv_bfloat16*>(X), kMlpIn, f + W.dh1, kMlpHidden, rows, rpb, f + W.grad + L.m_w1,
        f + W.grad + L.m_b1);
    return cudaGetLastError();
}

cudaError_t mlp_adam(unsigned char* ws, const MlpTrain& W, float lr, int64_t t, cudaStream_t s)
{
    float* f = reinterpret_cast<float*>(ws);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<grid_cap(W.L.nmaster, 256), 256, 0, s>>>(f + W.master, f + W.m, f + W.v, f + W.grad, W.L.nmaster, lr, b1,
                                                       b2, eps, c1, c2);
    return mlp_export(f + W.master, W.K, ws + W.params_byte, s);
}

cudaError_t mlp_export(const float* master, int K, void* params, cudaStream_t s)
{
    k_export<<<64, 256, 0, s>>>(master, mlp_layout(K), reinterpret_cast<unsigned char*>(params));
    return cudaGetLastError();
}

__global__ void k_mlp_sets_from_ring(MlpFeatureSet* sets, int nsets, const BoxDev* boxes, const unsigned char* ring,
                                     int64_t slot_bytes, int ring_slots, int real_bytes, const int64_t* step)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsets) return;
    const BoxDev& bd = boxes[sets[i].box];
    const int64_t j = *step / bd.K;
    for (int a = 0; a < 4; a++) {
        int64_t jj = j - 1 + a;
        if (jj < 0) jj = 0;
        sets[i].smp[a] = ring + (jj % ring_slots) * slot_bytes + bd.ring_off * real_bytes;
    }
}

cudaError_t mlp_sets_from_ring(MlpFeatureSet* sets, int nsets, const BoxDev* boxes, const void* ring,
                               int64_t slot_bytes, int ring_slots, int real_bytes, const int64_t* step, cudaStream_t s)
{
    k_mlp_sets_from_ring<<<(nsets + 127) / 128, 128, 0, s>>>(sets, nsets, boxes, reinterpret_cast<const unsigned char*>(ring),
                                                             slot_bytes, ring_slots, real_bytes, step);
    return cudaGetLastError();
}

}  // namespace lbt
