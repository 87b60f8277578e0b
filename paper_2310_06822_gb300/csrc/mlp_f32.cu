// FP32 kernels of the bounding network h (Sec. 3.4 "Architecture": MLP, sigmoid
// output rounded to {0,1}; hidden activation ReLU as the configurations state):
//   fwd_f32_kernel     plain FP32 forward over query tiles -> decision bits, margin flags
//   train_f32_kernel   forward + asymmetric BCE of Eq. (loss) + backward, per-CTA partials
//   adam_kernel        deterministic reduction of the partials + Adam (Sec. 3.4 "Training")
#include <math.h>

#include "common.cuh"

namespace {

constexpr int TMF = 64;  // queries per forward tile
constexpr int KC = 32;   // k-chunk of weights staged in shared memory
constexpr unsigned FULL = 0xffffffffu;

// hidden layer l of a tile: aout[m][n] = relu(b_n + sum_k W[n][k] ain[m][k]) for MI*16 rows.
// Thread (tm, tn) owns rows tm + 16 i and neurons tn + 16 j.
template <int NJ, int MI>
__device__ __forceinline__ void hidden_layer_tile(const float *__restrict__ W, const float *__restrict__ b, int K,
                                                  int N, const float *ain, float *aout, float *wt, int KP) {
    constexpr int WS = 16 * NJ + 1;
    const int t = threadIdx.x, tn = t & 15, tm = t >> 4;
    float acc[MI][NJ];
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        const int nn = tn + 16 * j;
        const float bv = nn < N ? __ldg(b + nn) : 0.f;
#pragma unroll
        for (int i = 0; i < MI; i++) acc[i][j] = bv;
    }
    for (int kc = 0; kc < K; kc += KC) {
        const int kw = min(KC, K - kc);
        __syncthreads();
        for (int e = t; e < N * KC; e += blockDim.x) {
            const int nn = e / KC, kk = e % KC;
            wt[kk * WS + nn] = kk < kw ? __ldg(W + (size_t)nn * K + kc + kk) : 0.f;
        }
        __syncthreads();
        for (int kk = 0; kk < kw; kk++) {
            float a[MI], w[NJ];
#pragma unroll
            for (int i = 0; i < MI; i++) a[i] = ain[(tm + 16 * i) * KP + kc + kk];
#pragma unroll
            for (int j = 0; j < NJ; j++) w[j] = wt[kk * WS + tn + 16 * j];
#pragma unroll
            for (int i = 0; i < MI; i++)
#pragma unroll
                for (int j = 0; j < NJ; j++) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        const int nn = tn + 16 * j;
        if (nn < N)
#pragma unroll
            for (int i = 0; i < MI; i++) aout[(tm + 16 * i) * KP + nn] = fmaxf(acc[i][j], 0.f);
    }
}

// ------------------------------------------------------------------ fast FP32 forward
template <int NJ>
__global__ void __launch_bounds__(256) fwd_f32_kernel(MlpDesc d, const float *__restrict__ q, long long n, TauF tau,
                                                      float margin, uint32_t *__restrict__ bits,
                                                      float *__restrict__ logits, nb_query_stats *st,
                                                      unsigned *flag_count, unsigned *flag_idx) {
    constexpr int KP = 16 * NJ + 1;
    extern __shared__ float smem[];
    float *act0 = smem;
    float *act1 = act0 + TMF * KP;
    float *wt = act1 + TMF * KP;
    __shared__ float zs[TMF];
    const int t = threadIdx.x, lane = t & 31;
    const int w0 = d.w[0];
    const long long ntiles = (n + TMF - 1) / TMF;
    unsigned long long c_in = 0, c_flag = 0, c_nf = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long base = tile * TMF;
        const int rows = (int)min((long long)TMF, n - base);
        __syncthreads();
        for (int e = t; e < TMF * w0; e += blockDim.x) {
            const int m = e / w0, k = e % w0;
            act0[m * KP + k] = m < rows ? q[(base + m) * w0 + k] : 0.f;
        }
        float *ain = act0, *aout = act1;
        for (int l = 0; l < d.L - 1; l++) {
            const int K = d.w[l], N = d.w[l + 1];
            const float *W = d.p + d.off[l];
            hidden_layer_tile<NJ, TMF / 16>(W, W + (size_t)N * K, K, N, ain, aout, wt, KP);
            float *tmp = ain;
            ain = aout;
            aout = tmp;
        }
        __syncthreads();
        {
            const int K = d.w[d.L - 1];
            const float *W = d.p + d.off[d.L - 1];
            const int m = t >> 2, part = t & 3;
            float s = 0.f;
            for (int k = part; k < K; k += 4) s = fmaf(__ldg(W + k), ain[m * KP + k], s);
            s += __shfl_xor_sync(FULL, s, 1);
            s += __shfl_xor_sync(FULL, s, 2);
            if (part == 0) zs[m] = s + __ldg(W + K);
        }
        __syncthreads();
        if (t < TMF) {
            const int m = t;
            const long long i = base + m;
            const bool valid = m < rows;
            const float z = zs[m];
            const bool fin = isfinite(z);
            const bool inside = valid && (!fin || z >= tau.up);
            const bool flag = valid && fin && (fabsf(z - tau.up) < margin || (z >= tau.dn && z < tau.up));
            const unsigned bi = __ballot_sync(FULL, inside);
            const unsigned bf = __ballot_sync(FULL, flag);
            const unsigned bn = __ballot_sync(FULL, valid && !fin);
            if (lane == 0 && base + 32 * (t >> 5) < n) bits[(base >> 5) + (t >> 5)] = bi;
            if (valid && logits) logits[i] = z;
            if (bf) {
                unsigned pos = 0;
                if (lane == 0) pos = atomicAdd(flag_count, (unsigned)__popc(bf));
                pos = __shfl_sync(FULL, pos, 0);
                if (flag) flag_idx[pos + __popc(bf & ((1u << lane) - 1u))] = (unsigned)i;
            }
            if (lane == 0) {
                c_in += __popc(bi);
                c_flag += __popc(bf);
                c_nf += __popc(bn);
            }
        }
    }
    if (st && lane == 0 && t < TMF) {
        if (c_in) atomicAdd(&st->n_inside, c_in);
        if (c_flag) atomicAdd(&st->n_flagged, c_flag);
        if (c_nf) atomicAdd(&st->n_nonfinite, c_nf);
    }
}

// ------------------------------------------------------------------ training step
__device__ __forceinline__ float softplusf(float u) { return u > 0.f ? u + log1pf(expf(-u)) : log1pf(expf(u)); }
__device__ __forceinline__ float sigmoidf(float u) {
    return u >= 0.f ? 1.f / (1.f + expf(-u)) : expf(u) / (1.f + expf(u));
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
    constexpr int NP = 16 * NJ, KP = NP + 1, MI = TM / 16, WS = NP + 1;
    constexpr int TPQ = 256 / TM;  // threads per sample in the output layer
    extern __shared__ float smem[];
    const int L = d.L;
    float *acts = smem;                        // [L][TM][KP]: a_0 .. a_{L-1}
    float *dcur = acts + (size_t)L * TM * KP;  // [TM][KP]
    float *dnext = dcur + TM * KP;             // [TM][KP]
    float *wt = dnext + TM * KP;               // [KC][WS]
    __shared__ float zs[TM], dz[TM], ls[TM];
    const int t = threadIdx.x, tn = t & 15, tm = t >> 4;
    const int w0 = d.w[0];
    float *slot = partial + (size_t)blockIdx.x * P;
    const long long ntiles = (n + TM - 1) / TM;
    float lossacc = 0.f;
    unsigned long long c_fn = 0, c_fp = 0, c_nf = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long base = tile * TM;
        const int rows = (int)min((long long)TM, n - base);
        __syncthreads();
        for (int e = t; e < TM * w0; e += blockDim.x) {
            const int m = e / w0, k = e % w0;
            acts[m * KP + k] = m < rows ? q[(base + m) * w0 + k] : 0.f;
        }
        for (int l = 0; l < L - 1; l++) {
            const int K = d.w[l], N = d.w[l + 1];
            const float *W = d.p + d.off[l];
            hidden_layer_tile<NJ, MI>(W, W + (size_t)N * K, K, N, acts + (size_t)l * TM * KP,
                                      acts + (size_t)(l + 1) * TM * KP, wt, KP);
        }
        __syncthreads();
        const float *aL = acts + (size_t)(L - 1) * TM * KP;
        const int KL = d.w[L - 1];
        const float *WL = d.p + d.off[L - 1];
        {
            const int m = t / TPQ, part = t % TPQ;
            float s = 0.f;
            for (int k = part; k < KL; k += TPQ) s = fmaf(__ldg(WL + k), aL[m * KP + k], s);
#pragma unroll
            for (int o = 1; o < TPQ; o <<= 1) s += __shfl_xor_sync(FULL, s, o);
            if (part == 0) zs[m] = s + __ldg(WL + KL);
        }
        __syncthreads();
        if (t < TM) {
            const int m = t;
            float g = 0.f, lv = 0.f;
            if (m < rows) {
                const long long i = base + m;
                const float y = (float)((labels[i >> 5] >> (i & 31)) & 1u);
                const float z = zs[m];
                if (isfinite(z)) {
                    // Eq. (loss): -alpha y log(s) - beta (1-y) log(1-s), s = sigmoid(z)
                    lv = alpha * y * softplusf(-z) + beta * (1.f - y) * softplusf(z);
                    const float sg = sigmoidf(z);
                    g = (alpha * y * (sg - 1.f) + beta * (1.f - y) * sg) * inv_n;
                    const bool dec = z >= tau.up;
                    c_fn += (y != 0.f && !dec);
                    c_fp += (y == 0.f && dec);
                } else {
                    c_nf++;
                }
            }
            dz[m] = g;
            ls[m] = lv;
        }
        __syncthreads();
        if (t == 0)
            for (int m = 0; m < rows; m++) lossacc += ls[m];
        // output layer gradient: dW_L[k] += sum_m dz_m a_L[m][k], db_L += sum_m dz_m,
        // and delta_{L-1}[m][k] = dz_m W_L[k] 1[a_L[m][k] > 0]
        {
            float *gW = slot + d.off[L - 1];
            for (int k = t; k <= KL; k += blockDim.x) {
                float s = 0.f;
                if (k < KL)
                    for (int m = 0; m < TM; m++) s = fmaf(dz[m], aL[m * KP + k], s);
                else
                    for (int m = 0; m < TM; m++) s += dz[m];
                gW[k] += s;
            }
            if (L > 1)
                for (int e = t; e < TM * KL; e += blockDim.x) {
                    const int m = e / KL, k = e % KL;
                    const float a = aL[m * KP + k];
                    dcur[m * KP + k] = a > 0.f ? dz[m] * __ldg(WL + k) : 0.f;
                }
        }
        for (int l = L - 2; l >= 0; l--) {
            __syncthreads();
            const int K = d.w[l], N = d.w[l + 1];
            const float *W = d.p + d.off[l];
            const float *al = acts + (size_t)l * TM * KP;
            float *gW = slot + d.off[l];
            for (int e = t; e < N * K; e += blockDim.x) {
                const int nn = e / K, k = e % K;
                float s = 0.f;
                for (int m = 0; m < TM; m++) s = fmaf(dcur[m * KP + nn], al[m * KP + k], s);
                gW[e] += s;
            }
            for (int nn = t; nn < N; nn += blockDim.x) {
                float s = 0.f;
                for (int m = 0; m < TM; m++) s += dcur[m * KP + nn];
                gW[(size_t)N * K + nn] += s;
            }
            if (l > 0) {
                // delta_l[m][k] = (sum_n delta_{l+1}[m][n] W[n][k]) 1[a_l[m][k] > 0]
                float acc[MI][NJ];
#pragma unroll
                for (int i = 0; i < MI; i++)
#pragma unroll
                    for (int j = 0; j < NJ; j++) acc[i][j] = 0.f;
                for (int nc = 0; nc < N; nc += KC) {
                    const int nw = min(KC, N - nc);
                    __syncthreads();
                    for (int e = t; e < KC * K; e += blockDim.x) {
                        const int nn = e / K, k = e % K;
                        wt[nn * WS + k] = nn < nw ? __ldg(W + (size_t)(nc + nn) * K + k) : 0.f;
                    }
                    __syncthreads();
                    for (int nn = 0; nn < nw; nn++) {
                        float dv[MI], w[NJ];
#pragma unroll
                        for (int i = 0; i < MI; i++) dv[i] = dcur[(tm + 16 * i) * KP + nc + nn];
#pragma unroll
                        for (int j = 0; j < NJ; j++) w[j] = wt[nn * WS + tn + 16 * j];
#pragma unroll
                        for (int i = 0; i < MI; i++)
#pragma unroll
                            for (int j = 0; j < NJ; j++) acc[i][j] = fmaf(dv[i], w[j], acc[i][j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < NJ; j++) {
                    const int k = tn + 16 * j;
                    if (k < K)
#pragma unroll
                        for (int i = 0; i < MI; i++) {
                            const int m = tm + 16 * i;
                            dnext[m * KP + k] = al[m * KP + k] > 0.f ? acc[i][j] : 0.f;
                        }
                }
                __syncthreads();
                float *tp = dcur;
                dcur = dnext;
                dnext = tp;
            }
        }
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

// Sum the per-CTA partials in CTA order (deterministic), keep the gradient, take one
// Adam step (Kingma & Ba, in PyTorch's arithmetic order: denom = sqrt(v)/sqrt(c2) + eps,
// theta -= (lr / c1) m / denom).
__global__ void __launch_bounds__(256) adam_kernel(long long P, int G, const float *__restrict__ partial,
                                                   const float *__restrict__ loss_partial, float inv_n,
                                                   float *__restrict__ params, float *__restrict__ m,
                                                   float *__restrict__ v, float *__restrict__ grad, float lr,
                                                   float b1, float b2, float eps, float c1, float sqrt_c2,
                                                   nb_step_stats *st) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && st) {
        float s = 0.f;
        for (int c = 0; c < G; c++) s += loss_partial[c];
        st->loss = s * inv_n;
    }
    if (p >= P) return;
    float g = 0.f;
    for (int c = 0; c < G; c++) g += partial[(size_t)c * P + p];
    grad[p] = g;
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float denom = sqrtf(vv) / sqrt_c2 + eps;
    params[p] = params[p] - (lr / c1) * (mm / denom);
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
    constexpr int KP = 16 * NJ + 1;
    const size_t smem = (size_t)(2 * TMF * KP + KC * (16 * NJ + 1)) * sizeof(float);
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
    const size_t smem = (size_t)((d.L + 2) * TM * KP + KC * (16 * NJ + 1)) * sizeof(float);
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
                         cudaStream_t s) {
    const int64_t blocks = (P + 255) / 256;
    adam_kernel<<<(unsigned)blocks, 256, 0, s>>>((long long)P, ws.G, ws.partial, ws.loss_partial, inv_n, params, m, v,
                                                 grad, lr, b1, b2, eps, c1, sqrt_c2, st);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}
