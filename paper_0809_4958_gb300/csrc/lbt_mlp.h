// Internal interface of the learned boundary upsampler (lbt_mlp.cu).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace lbt {

constexpr int kMlpIn = 32;       // 24 features, zero padded
constexpr int kMlpFeat = 24;
constexpr int kMlpHidden = 128;
constexpr float kMlpOutDiv = 64.0f;  // network output unit: u_max / kMlpOutDiv

// Byte offsets of the inference parameters and float offsets of the master copy.
struct MlpLayout {
    int nout;
    size_t w1, w2, w3, b1, b2, b3, bytes;
    int64_t m_w1, m_b1, m_w2, m_b2, m_w3, m_b3, nmaster;
};

// Float offsets of the training workspace (batch rows B), then the inference
// parameters at params_byte.
struct MlpTrain {
    MlpLayout L;
    int K;
    int64_t batch;
    size_t master, m, v, grad, h1, h2, y, dy, dh2, dh1, loss;
    size_t params_byte, bytes;
};

// One set of face rows for the feature kernel: rows [row_off, row_off + 6 E^2),
// samples j-1 (clamped), j, j+1, j+2 of the set's faces ([6][3][E][E] each).
struct MlpFeatureSet {
    int64_t row_off;
    const void* smp[4];
    int32_t E;
    int32_t box;  // box of a context (ring sets), unused otherwise
};

MlpLayout mlp_layout(int K);
MlpTrain mlp_train_layout(int K, int64_t batch_rows);

// Inference forward, Y row-major [rows][3K] (tcgen05).
cudaError_t mlp_forward(const void* X, int64_t rows, const void* params, int K, float* Y, cudaStream_t s);
// Inference forward on the tcgen05 tensor cores (lbt_mlp_tc.cu); err (device,
// may be null) receives LB_ERR_TIMEOUT if an MMA does not complete.  Y is
// row-major [rows][3K] when col_stride is 0, else column-major: output c of
// row r at Y[c * col_stride + r] (the step's layout: a boundary site's
// residual at one substep is then read from consecutive rows).
cudaError_t mlp_forward_tc(const void* X, int64_t rows, const void* params, int K, float* Y, int32_t* err,
                           cudaStream_t s, int64_t col_stride = 0);
// Training forward on tcgen05: Y row-major [rows][3K] FP32 and the bf16
// hidden activations after ReLU, H1 and H2 row-major [rows][128].
cudaError_t mlp_forward_save_tc(const void* X, int64_t rows, const void* params, int K, float* Y, void* H1, void* H2,
                                cudaStream_t s);
// Backward on tcgen05 from dY (FP32 [rows][3K]): the FP32 gradient (master
// layout, added to `grad`), with dH2 and dH1 (bf16 [rows][128]) as scratch.
cudaError_t mlp_backward_tc(const void* X, int64_t rows, const void* params, int K, const void* H1, const void* H2,
                            const float* dY, void* dH2, void* dH1, float* grad, cudaStream_t s);
cudaError_t mlp_features(const MlpFeatureSet* sets_dev, int nsets, int64_t total_rows, double u_max, int real_f64,
                         void* X, cudaStream_t s);
// Features of one face set passed by value (6 E^2 rows from row 0).
cudaError_t mlp_features_one(const MlpFeatureSet& set, double u_max, int real_f64, void* X, cudaStream_t s);
cudaError_t mlp_targets(const void* const smp[4], const void* fine, int E, int K, int first_interval, double u_max,
                        int real_f64, float* T, cudaStream_t s);
cudaError_t mlp_grad(unsigned char* ws, const MlpTrain& W, const void* X, const float* T, int64_t rows, cudaStream_t s);
cudaError_t mlp_adam(unsigned char* ws, const MlpTrain& W, float lr, int64_t t, cudaStream_t s);
cudaError_t mlp_export(const float* master, int K, void* params, cudaStream_t s);

struct BoxDev;
// Fill the sample pointers of the ring sets for the interval of the current
// device step (samples j-1 clamped, j, j+1, j+2 of every upsampler box).
cudaError_t mlp_sets_from_ring(MlpFeatureSet* sets, int nsets, const BoxDev* boxes, const void* ring,
                               int64_t slot_bytes, int ring_slots, int real_bytes, const int64_t* step, cudaStream_t s);

}  // namespace lbt
