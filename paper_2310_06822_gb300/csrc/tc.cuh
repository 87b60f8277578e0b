// Tensor-core (tcgen05 / TMEM) paths: BF16 and FP8 forward, BF16 training step.
#pragma once

#include "common.cuh"

// Low-precision weight images and their launch state, owned by a model.
struct TcModel {
    int infer_prec = 0, train_prec = 0;
    void *img = nullptr;     // device: packed operand images of every layer
    size_t img_bytes = 0;
    float *scales = nullptr; // device (FP8): 1 / s_n of every E4M3 weight row, folded biases, head
    void *train_img = nullptr;   // device: BF16 weights for the tensor-core training step
    size_t train_img_bytes = 0;
    int *err = nullptr;      // device: status of the last bounded wait that gave up (0 = none)
    int train_tc = 0;        // BF16 training runs the tcgen05 step (train_tc.cu) on a training image in its layout
    // Hidden widths below the kernels' 64 / 128 (the paper's 25-, 50- and 75-wide networks):
    // the forward runs on a copy of the parameters zero-padded to that width.  Padded
    // neurons have zero weights and bias, so they stay 0 through the ReLU and add exact
    // zeros downstream: the padded network computes the same logits.
    float *pad_p = nullptr;  // device: padded FP32 parameters (refreshed with the master copy)
    MlpDesc pad{};           // their layout (pad.p = pad_p)
};

// split-FP16 forward (tc_split.cu)
size_t nb_split_img_bytes(int H, int NH);
size_t nb_split_smem_bytes(int H, int NH);
nb_status nb_split_refresh(TcModel *tc, const MlpDesc &d, cudaStream_t s);
nb_status nb_split_query(TcModel *tc, const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin,
                         uint32_t *bits, float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s);

// FP8 (E4M3) forward (tc_fp8.cu)
size_t nb_fp8_img_bytes(int H, int NHH);
size_t nb_fp8_smem_bytes(int H, int NHH);
nb_status nb_fp8_refresh(TcModel *tc, const MlpDesc &d, cudaStream_t s);
nb_status nb_fp8_query(TcModel *tc, const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin,
                       uint32_t *bits, float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s);

// NB_OK, or the status a tensor-core kernel recorded since the last check (synchronous).
nb_status nb_tc_check(TcModel *tc);

nb_status nb_tc_init(TcModel *tc, const MlpDesc &d, int infer_prec, int train_prec);
void nb_tc_free(TcModel *tc);
nb_status nb_tc_refresh(TcModel *tc, const MlpDesc &d, cudaStream_t s);
// the inference images only (the training image left as it is)
nb_status nb_tc_refresh_query(TcModel *tc, const MlpDesc &d, cudaStream_t s);
nb_status nb_tc_query(TcModel *tc, const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin,
                      uint32_t *bits, float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s);
// BF16 tensor-core training step (train_bf16.cu)
nb_status nb_train_bf16_check(const MlpDesc &d);
size_t nb_train_bf16_img_bytes(const MlpDesc &d);
size_t nb_train_bf16_smem(int H, int NH, long long P);
nb_status nb_train_bf16_refresh(TcModel *tc, const MlpDesc &d, cudaStream_t s);
int nb_train_bf16_ctas(int64_t n);
nb_status nb_launch_train_bf16(TcModel *tc, const MlpDesc &d, const float *q, const uint32_t *labels, int64_t n,
                               float alpha, float beta, TauF tau, TrainWs ws, nb_step_stats *st, cudaStream_t s);
// tcgen05 BF16 training step of 128-wide networks with 2..4 hidden layers (train_tc.cu)
bool nb_train_tc_supported(const MlpDesc &d);
int nb_train_tc_ctas(int64_t n);
nb_status nb_train_tc_refresh(TcModel *tc, const MlpDesc &d, cudaStream_t s);
nb_status nb_launch_train_tc(TcModel *tc, const MlpDesc &d, const float *q, const uint32_t *labels, int64_t n,
                             float alpha, float beta, TauF tau, TrainWs ws, nb_step_stats *st, cudaStream_t s);
