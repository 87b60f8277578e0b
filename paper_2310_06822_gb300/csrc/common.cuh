// Internal definitions shared by the libnb translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "nb.h"

#define NB_MAXL 8          // maximum number of layers (weight matrices)
#define NB_MAXW 256        // maximum hidden width

// ---------------------------------------------------------------- errors
void nb_set_error(const std::string &msg);
nb_status nb_fail(nb_status s, const std::string &msg);
nb_status nb_cuda_check(cudaError_t e, const char *what);

#define NB_CUDA(call)                                              \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return nb_cuda_check(_e, #call);    \
    } while (0)

// ---------------------------------------------------------------- network description
// Plain-old-data view of an MLP passed by value to kernels.
struct MlpDesc {
    int L;                   // number of weight layers; widths w[0..L], w[L] == 1
    int w[NB_MAXL + 1];
    int off[NB_MAXL];        // offset of W_l in the flat parameter array; b_l follows W_l
    int maxw;                // max(w[0..L-1])
    int act;                 // hidden activation: NB_ACT_RELU or NB_ACT_SINE
    const float *p;          // device FP32 master parameters
    const float *pT;         // the same with every W_l stored transposed ([K][N]), biases as in p
};

// Rounding-error constants of the rigorous bounds, rounded up, one per layer:
//   g[l]   = gamma_{K+8} = k u / (1 - k u), u = 2^-24, k = fan-in K + 8 (FP32 stage)
//   gd2[l] = gamma_{3K+4} (compensated stage)
//   gff[l] = gamma_{4K+4} (three-word stage)
struct GammaTab {
    float g[NB_MAXL];
    float gd2[NB_MAXL];
    float gff[NB_MAXL];
};

// tau bracketed by two floats: tau_dn <= tau <= tau_up, equal when tau is a float;
// and split as tau = hi + lo + r with |r| <= err (float-float comparisons).
struct TauF {
    float dn, up;
    float hi, lo, err;
};
TauF nb_tau_bracket(double tau);
void nb_fill_gamma(const int *widths, int L, GammaTab *gt);
// tau = (minimum positive FP64 logit, given as order-preserving bits) - eps, rounded
// toward -infinity; +inf without positives, -inf if a positive had a NaN logit
double nb_tau_from_min_bits(unsigned long long zmin_bits, unsigned npos, double eps);

// ---------------------------------------------------------------- launchers (per .cu)
nb_status nb_launch_label(const nb_shape *shape, int kind, const float *q, int64_t n, uint32_t *bits,
                          nb_label_stats *st, cudaStream_t s);

struct QueryWs {
    unsigned int *flag_count;   // [1] queries within the margin of tau
    unsigned int *flag_idx;     // [n]
    unsigned int *ff_count;     // [1] queries left ambiguous by the FP32 bound
    unsigned int *ff_idx;       // [n]
};

nb_status nb_launch_fwd_f32(const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin,
                            uint32_t *bits, float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s);
// thread-per-query FP32 forward of networks with input width <= 8 and stored hidden
// layers <= 128 wide (narrow.cu)
bool nb_narrow_eligible(const MlpDesc &d);
nb_status nb_launch_fwd_narrow(const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin,
                               uint32_t *bits, float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s);
// first stage of the early-out for a one-hidden-layer ReLU early network: settled rows get
// bit 1, the others bit 0 and are gathered (qc, [count][w0]), pos_w[w] the first gathered
// row of word w; then the late bits of the gathered rows merged into the words (narrow.cu)
bool nb_early_settle_eligible(const MlpDesc &d);
nb_status nb_launch_early_settle(const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin,
                                 uint32_t *out_bits, unsigned *count, unsigned *pos_w, float *qc, cudaStream_t s);
nb_status nb_launch_early_merge(const uint32_t *bits_c, const unsigned *pos_w, int64_t n, uint32_t *out_bits,
                                cudaStream_t s);
// neural early-out (early.cu)
nb_status nb_launch_early_compact(const uint32_t *bits_e, int64_t n, unsigned *count, unsigned *idx, uint32_t *out_bits,
                                  cudaStream_t s);
nb_status nb_launch_early_gather(const float *q, int w, const unsigned *idx, int64_t m, float *qc, cudaStream_t s);
nb_status nb_launch_early_scatter(const uint32_t *bits_c, const unsigned *idx, int64_t m, uint32_t *out_bits,
                                  cudaStream_t s);
nb_status nb_launch_bits_not(const uint32_t *in, int64_t n, uint32_t *out, cudaStream_t s);
nb_status nb_launch_three_way(const uint32_t *bits_outer, const uint32_t *bits_inner, int64_t n, uint8_t *codes,
                              nb_three_way_stats *st, cudaStream_t s);

// pT <- p with every weight matrix transposed, for n_objects parameter sets P apart
nb_status nb_launch_transpose(const MlpDesc &d, float *pT, int n_objects, long long P, cudaStream_t s);
nb_status nb_launch_recheck(const MlpDesc &d, const GammaTab &gt, const float *q, TauF tau, uint32_t *bits,
                            nb_query_stats *st, QueryWs ws, int64_t n, cudaStream_t s);

struct CalibWs {
    unsigned int *umin_bits;          // [1] order-preserving bits of min upper bound
    unsigned long long *zmin_bits;    // [1] order-preserving bits of min FP64 logit
    unsigned int *npos;               // [1] number of positives
    unsigned int *pos_idx;            // [n] indices of the positives
    float *lo;                        // [n] lower bound of each listed positive
};
nb_status nb_launch_calibrate(const MlpDesc &d, const GammaTab &gt, const float *q, const uint32_t *labels,
                              int64_t row0, int64_t row1, CalibWs ws, cudaStream_t s);
nb_status nb_launch_recheck_grouped(const MlpDesc &d, const GammaTab &gt, const float *q, const long long *offsets,
                                    int n_objects, long long P, const TauF *taus, uint32_t *bits, nb_query_stats *st,
                                    QueryWs ws, int64_t n, cudaStream_t s);

struct TrainWs {
    float *partial;          // [G][stride] per-CTA gradient partials
    float *loss_partial;     // [G]
    int G;                   // CTAs used
    long long stride;        // floats between two CTAs' partials (0: P)
};
int nb_train_f32_ctas(const MlpDesc &d, int64_t n, int num_sms);
nb_status nb_launch_train_f32(const MlpDesc &d, const float *q, const uint32_t *labels, int64_t n, float alpha,
                              float beta, TauF tau, TrainWs ws, nb_step_stats *st, cudaStream_t s);
// The BF16 copy of the hidden layers' weights that the tcgen05 training step reads (its
// "training image"), written by the Adam step as it updates each weight; img null: none.
// Layer 0 (128 x 16) is 8 x 16-byte core matrices; layers 1 .. NH-1 are two 64-column
// blocks of 128 rows each, 128-byte swizzled, after the first layer's 4 KB.
struct TrainImgMap {
    uint8_t *img = nullptr;
    int NH = 0;                 // hidden layers (image layers 0 .. NH - 1)
    int w[NB_MAXL + 1] = {0};
    int off[NB_MAXL] = {0};
};
__host__ __device__ __forceinline__ uint32_t nb_train_img_offset(int l, int n, int k) {
    if (l == 0)
        return (uint32_t)(n >> 3) * 256u + (uint32_t)(k >> 3) * 128u + (uint32_t)(n & 7) * 16u + (uint32_t)(k & 7) * 2u;
    return 4096u + (uint32_t)(l - 1) * 32768u + (uint32_t)(k >> 6) * 16384u + (uint32_t)n * 128u +
           ((uint32_t)(((k & 63) >> 3) ^ (n & 7)) << 4) + (uint32_t)(k & 7) * 2u;
}
nb_status nb_launch_adam(int64_t P, float inv_n, float *params, float *m, float *v, float *grad,
                         TrainWs ws, float lr, float b1, float b2, float eps, float c1, float sqrt_c2,
                         nb_step_stats *st, cudaStream_t s, const TrainImgMap &img = TrainImgMap{});
