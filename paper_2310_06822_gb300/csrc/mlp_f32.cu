// FP32 kernels of the bounding network h (Sec. 3.4 "Architecture": MLP, sigmoid
// output rounded to {0,1}; hidden activation ReLU as the configurations state):
//   fwd_f32_kernel     plain FP32 forward over query tiles -> decision bits, margin flags
//   train_f32_kernel   forward + asymmetric BCE of Eq. (loss) + backward, per-CTA partials
//   adam_kernel        deterministic reduction of the partials + Adam (Sec. 3.4 "Training")
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "mlp_tile.cuh"

namespace {

using namespace nbf32;


// ------------------------------------------------------------------ fast FP32 forward
template <int NJ>
__global__ void __launch_bounds__(256, NJ >= 16 ? 1 : 2) fwd_f32_kernel(const __grid_constant__ MlpDesc d,
                                                                        const float *__restrict__ q, long long n, TauF tau,
                                                      float margin, uint32_t *__restrict__ bits,
                                                      float *__restrict__ logits, nb_query_stats *st,
                                                      unsigned *flag_count, unsigned *flag_idx) {
    extern __shared__ float smem[];
    __shared__ float zs[TMF];
    const int t = threadIdx.x, lane = t & 31;
    const long long ntiles = (n + TMF - 1) / TMF;
    unsigned long long c_in = 0, c_flag = 0, c_nf = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long base = tile * TMF;
        const int rows = (int)min((long long)TMF, n - base);
        // from width 49 on, the weights come from the transposed copy with float4 loads
        fwd_tile<NJ, (NJ >= 4)>(d, q, base, rows, tau, margin, bits, logits, flag_count, flag_idx, smem, zs, c_in,
                                c_flag, c_nf);
    }
    if (st && lane == 0 && t < TMF) {
        if (c_in) atomicAdd(&st->n_inside, c_in);
        if (c_flag) atomicAdd(&st->n_flagged, c_flag);
        if (c_nf) atomicAdd(&st->n_nonfinite, c_nf);
    }
}

// One CTA walks tiles of TM samples; it keeps every layer's activations of the tile
// in shared memory, evaluates the loss, back-propagates and accumulates its own
// gradient partial (partial[blockIdx.x][*]), which adam_kernel sums in CTA order.
template <int NJ, int TM>
__global__ void __launch_bounds__(256) train_f32_kernel(MlpDesc d, const float *__restrict__ q,
                                                        const uint32_t *__restrict__ labels, long long n,
                                                        float alpha, float beta, float inv_n, TauF tau,
                                                        float *__restrict__ partial, float *loss_partial,
                                                        long long P, nb_step_stats *st) {
    extern __shared__ float smem[];
    __shared__ float zs[TM], dz[TM], ls[TM];
    const int t = threadIdx.x;
    float *slot = partial + (size_t)blockIdx.x * P;
    const long long ntiles = (n + TM - 1) / TM;
    float lossacc = 0.f;
    unsigned long long c_fn = 0, c_fp = 0, c_nf = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long base = tile * TM;
        const int rows = (int)min((long long)TM, n - base);
        train_tile<NJ, TM>(d, q, labels, base, rows, alpha, beta, inv_n, tau, slot, smem, zs, dz, ls, lossacc, c_fn,
                           c_fp, c_nf);
    }
    if (t == 0) loss_partial[blockIdx.x] = lossacc;
    if (st && t < TM) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            c_fn += __shfl_xor_sync(FULL, c_fn, o);
            c_fp += __shfl_xor_sync(FULL, c_fp, o);
            c_nf += __shfl_xor_sync(FULL, c_nf, o);
        }
        if ((t & 31) == 0) {
            if (c_fn) atomicAdd(&st->fn, c_fn);
            if (c_fp) atomicAdd(&st->fp, c_fp);
            if (c_nf) atomicAdd(&st->n_nonfinite, c_nf);
        }
    }
}

// Sum the per-CTA partials (deterministic: every parameter's G partials are summed as eight
// strided slices, c = s, s + 8, ..., added in a fixed tree), keep the gradient, take one
// Adam step (Kingma & Ba, in PyTorch's arithmetic order: denom = sqrt(v)/sqrt(c2) + eps,
// theta -= (lr / c1) m / denom).  A block serves 32 parameters with 8 slices each, so every
// thread has several independent loads in flight.
constexpr int ADAM_P = 32, ADAM_S = 8;
__global__ void __launch_bounds__(ADAM_P * ADAM_S) adam_kernel(long long P, int G, long long stride,
                                                               const float *__restrict__ partial,
                                                               const float *__restrict__ loss_partial, float inv_n,
                                                               float *__restrict__ params, float *__restrict__ m,
                                                               float *__restrict__ v, float *__restrict__ grad,
                                                               float lr, float b1, float b2, float eps, float c1,
                                                               float sqrt_c2, nb_step_stats *st, TrainImgMap img) {
    __shared__ float part[ADAM_S][ADAM_P + 1];
    const int pc = threadIdx.x % ADAM_P, sl = threadIdx.x / ADAM_P;
    if (blockIdx.x == 0 && st) {  // the loss: same slicing over the CTAs' loss partials
        float s = 0.f;
        for (int c = threadIdx.x; c < G; c += ADAM_P * ADAM_S) s += loss_partial[c];
        __shared__ float ls[ADAM_P * ADAM_S];
        ls[threadIdx.x] = s;
        __syncthreads();
        for (int w = ADAM_P * ADAM_S / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) ls[threadIdx.x] += ls[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) st->loss = ls[0] * inv_n;
    }
    const long long p = (long long)blockIdx.x * ADAM_P + pc;
    float g = 0.f;
    if (p < P)
        for (int c = sl; c < G; c += ADAM_S) g += partial[(size_t)c * stride + p];
    part[sl][pc] = g;
    __syncthreads();
    if (sl != 0 || p >= P) return;
    g = ((part[0][pc] + part[1][pc]) + (part[2][pc] + part[3][pc])) +
        ((part[4][pc] + part[5][pc]) + (part[6][pc] + part[7][pc]));
    grad[p] = g;
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float denom = sqrtf(vv) / sqrt_c2 + eps;
    const float np_ = params[p] - (lr / c1) * (mm / denom);
    params[p] = np_;
    if (img.img) {
        // the weight's BF16 copy in the training image (biases and the head are read in
        // FP32 from the master copy)
        for (int l = 0; l < img.NH; l++) {
            const long long r = p - img.off[l];
            const int K = img.w[l], N = img.w[l + 1];
            if (r >= 0 && r < (long long)N * K) {
                const int n = (int)(r / K), k = (int)(r - (long long)n * K);
                *reinterpret_cast<__nv_bfloat16 *>(img.img + nb_train_img_offset(l, n, k)) = __float2bfloat16_rn(np_);
                break;
            }
        }
    }
}

int nj_for(int maxw) {
    int nj = (maxw + 15) / 16;
    if (nj <= 1) return 1;
    if (nj <= 2) return 2;
    if (nj <= 4) return 4;
    if (nj <= 8) return 8;
    return 16;
}

int num_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

template <int NJ>
nb_status fwd_launch(const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin, uint32_t *bits,
                     float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s) {
    const size_t smem = (size_t)fwd_tile_floats<NJ>(NJ >= 4) * sizeof(float);
    auto k = fwd_f32_kernel<NJ>;
    NB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 1;
    NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem));
    if (per_sm < 1) return nb_fail(NB_EUNSUPPORTED, "fwd_f32: kernel does not fit on an SM");
    const int64_t tiles = (n + TMF - 1) / TMF;
    int64_t grid = (int64_t)num_sms() * per_sm;
    if (grid > tiles) grid = tiles;
    k<<<(unsigned)grid, 256, smem, s>>>(d, q, (long long)n, tau, margin, bits, logits, st, ws.flag_count,
                                       ws.flag_idx);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

template <int NJ, int TM>
nb_status train_launch(const MlpDesc &d, const float *q, const uint32_t *labels, int64_t n, float alpha,
                       float beta, TauF tau, TrainWs ws, nb_step_stats *st, cudaStream_t s, long long P) {
    constexpr int KP = 16 * NJ + 1;
    const size_t smem = (size_t)((d.L + 2) * TM * KP + KC * (16 * NJ + 1) +
                                 (d.act == NB_ACT_SINE ? d.L * TM * KP : 0)) *
                        sizeof(float);
    auto k = train_f32_kernel<NJ, TM>;
    NB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<ws.G, 256, smem, s>>>(d, q, labels, (long long)n, alpha, beta, 1.0f / (float)n, tau, ws.partial,
                              ws.loss_partial, P, st);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

}  // namespace

nb_status nb_launch_fwd_f32(const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin, uint32_t *bits,
                            float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s) {
    switch (nj_for(d.maxw)) {
    case 1: return fwd_launch<1>(d, q, n, tau, margin, bits, logits, st, ws, s);
    case 2: return fwd_launch<2>(d, q, n, tau, margin, bits, logits, st, ws, s);
    case 4: return fwd_launch<4>(d, q, n, tau, margin, bits, logits, st, ws, s);
    case 8: return fwd_launch<8>(d, q, n, tau, margin, bits, logits, st, ws, s);
    default: return fwd_launch<16>(d, q, n, tau, margin, bits, logits, st, ws, s);
    }
}

int nb_train_f32_ctas(const MlpDesc &d, int64_t n, int sms) {
    const int TM = nj_for(d.maxw) >= 16 ? 16 : 32;
    const int64_t tiles = (n + TM - 1) / TM;
    int64_t g = sms;
    if (g > tiles) g = tiles;
    return (int)(g < 1 ? 1 : g);
}

nb_status nb_launch_train_f32(const MlpDesc &d, const float *q, const uint32_t *labels, int64_t n, float alpha,
                              float beta, TauF tau, TrainWs ws, nb_step_stats *st, cudaStream_t s) {
    long long P = 0;
    for (int l = 0; l < d.L; l++) P += (long long)d.w[l + 1] * (d.w[l] + 1);
    NB_CUDA(cudaMemsetAsync(ws.partial, 0, (size_t)ws.G * P * sizeof(float), s));
    if (st) NB_CUDA(cudaMemsetAsync(st, 0, sizeof(nb_step_stats), s));
    switch (nj_for(d.maxw)) {
    case 1: return train_launch<1, 32>(d, q, labels, n, alpha, beta, tau, ws, st, s, P);
    case 2: return train_launch<2, 32>(d, q, labels, n, alpha, beta, tau, ws, st, s, P);
    case 4: return train_launch<4, 32>(d, q, labels, n, alpha, beta, tau, ws, st, s, P);
    case 8: return train_launch<8, 32>(d, q, labels, n, alpha, beta, tau, ws, st, s, P);
    default: return train_launch<16, 16>(d, q, labels, n, alpha, beta, tau, ws, st, s, P);
    }
}

nb_status nb_launch_adam(int64_t P, float inv_n, float *params, float *m, float *v, float *grad, TrainWs ws,
                         float lr, float b1, float b2, float eps, float c1, float sqrt_c2, nb_step_stats *st,
                         cudaStream_t s, const TrainImgMap &img) {
    const int64_t blocks = (P + ADAM_P - 1) / ADAM_P;
    adam_kernel<<<(unsigned)blocks, ADAM_P * ADAM_S, 0, s>>>((long long)P, ws.G, ws.stride > 0 ? ws.stride : (long long)P,
                                                 ws.partial, ws.loss_partial, inv_n, params, m, v, grad, lr, b1, b2,
                                                 eps, c1, sqrt_c2, st, img);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}
