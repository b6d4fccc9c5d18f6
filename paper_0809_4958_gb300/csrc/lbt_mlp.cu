// Learned boundary upsampler: a small MLP that predicts, per face site and
// coarse interval, the residual of the boundary velocity over the cubic
// Hermite interpolant at the K substeps (the paper interpolates the DNS
// boundary linearly between samples, Sec. 3; the residual network is an
// added form).  Network: 24 features (padded to 32) -> 128 -> 128 -> 3K,
// ReLU, BF16 weights and activations on the tensor cores with FP32
// accumulation.  Training runs on the GPU: the forward and the backward on the
// tcgen05 tensor cores (lbt_mlp_tc.cu), the loss and Adam on FP32 master
// weights below.
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

cudaError_t mlp_forward(const void* X, int64_t rows, const void* params, int K, float* Y, cudaStream_t s)
{
    return mlp_forward_tc(X, rows, params, K, Y, nullptr, s);  // row-major output
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
    // forward on tcgen05, saving the bf16 activations (h1, h2 hold bf16 rows)
    cudaError_t e = mlp_forward_save_tc(X, rows, params, W.K, f + W.y, f + W.h1, f + W.h2, s);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(f + W.grad, 0, sizeof(float) * L.nmaster, s);
    cudaMemsetAsync(f + W.loss, 0, sizeof(double), s);
    const int64_t ny = rows * L.nout;
    k_mse<<<grid_cap(ny, 256), 256, 0, s>>>(f + W.y, T, ny, 1.0f / (float)ny, f + W.dy,
                                            reinterpret_cast<double*>(f + W.loss));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // backward on tcgen05 (dh2, dh1 hold bf16 rows)
    return mlp_backward_tc(X, rows, params, W.K, f + W.h1, f + W.h2, f + W.dy, f + W.dh2, f + W.dh1, f + W.grad, s);
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
