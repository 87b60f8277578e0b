// FP32 tile building blocks shared by the single-object and the grouped kernels.
#pragma once

#include <math.h>

#include "common.cuh"

namespace nbf32 {

constexpr int KC = 32;   // k-chunk of weights staged in shared memory
constexpr int TMF = 64;  // queries per forward tile
constexpr unsigned FULL = 0xffffffffu;

template <int NJ, int MI>
__device__ __forceinline__ void hidden_layer_tile(const float *__restrict__ W, const float *__restrict__ b, int K,
                                                  int N, const float *ain, float *aout, float *wt, int KP, int act,
                                                  float *cout);
template <int NJ, int MI>
__device__ __forceinline__ void hidden_layer_tile_t(const float *__restrict__ Wt, const float *__restrict__ b, int K,
                                                    int N, const float *ain, float *aout, float *wt, int KP, int act);

// Layout of the forward tile from the transposed weights (TR, widths above 48): rows of
// KP_T floats (a multiple of four, for float4 loads), weights staged in two chunks of CK_T
// input rows.
template <int NJ>
__host__ __device__ constexpr int kp_fwd(bool tr) {
    return tr ? 16 * NJ + 4 : 16 * NJ + 1;
}
constexpr int CK_T = 16;
template <int NJ>
__host__ __device__ constexpr int fwd_tile_floats(bool tr) {
    return tr ? 2 * TMF * kp_fwd<NJ>(true) + 2 * CK_T * kp_fwd<NJ>(true)
              : 2 * TMF * kp_fwd<NJ>(false) + KC * (16 * NJ + 1);
}

// Forward of one tile of TMF queries starting at row `base` (rows valid) with the
// decision z >= tau: bits of the tile's 32-row words (base is a multiple of 32),
// optional logits, and the margin band appended to flag_idx.  A non-finite logit is
// always flagged.  smem: 2 x [TMF][KP] activations + [KC][16 NJ + 1] weight chunk, or
// with TR (the weights read from the transposed copy d.pT, NJ >= 4) fwd_tile_floats<NJ>(true).
template <int NJ, bool TR = false>
__device__ __forceinline__ void fwd_tile(const MlpDesc &d, const float *__restrict__ q, long long base, int rows,
                                         TauF tau, float margin, uint32_t *__restrict__ bits,
                                         float *__restrict__ logits, unsigned *flag_count, unsigned *flag_idx,
                                         float *smem, float *zs, unsigned long long &c_in,
                                         unsigned long long &c_flag, unsigned long long &c_nf) {
    constexpr int KP = kp_fwd<NJ>(TR);
    float *act0 = smem;
    float *act1 = act0 + TMF * KP;
    float *wt = act1 + TMF * KP;
    const int t = threadIdx.x, lane = t & 31;
    const int w0 = d.w[0];
    __syncthreads();
    for (int e = t; e < TMF * w0; e += blockDim.x) {
        const int m = e / w0, k = e % w0;
        act0[m * KP + k] = m < rows ? q[(base + m) * w0 + k] : 0.f;
    }
    float *ain = act0, *aout = act1;
    for (int l = 0; l < d.L - 1; l++) {
        const int K = d.w[l], N = d.w[l + 1];
        if constexpr (TR) {
            const float *Wt = d.pT + d.off[l];
            hidden_layer_tile_t<NJ, TMF / 16>(Wt, Wt + (size_t)N * K, K, N, ain, aout, wt, KP, d.act);
        } else {
            const float *W = d.p + d.off[l];
            hidden_layer_tile<NJ, TMF / 16>(W, W + (size_t)N * K, K, N, ain, aout, wt, KP, d.act, nullptr);
        }
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
        bool xfin = true;  // a non-finite input coordinate: the logit is made NaN
        for (int k = 0; valid && k < w0; k++) xfin = xfin && isfinite(__ldg(q + i * w0 + k));
        const float z = xfin ? zs[m] : __int_as_float(0x7fc00000);
        const bool fin = isfinite(z);
        const bool inside = valid && fin && z >= tau.up;
        const bool flag = valid && (!fin || fabsf(z - tau.up) < margin || (z >= tau.dn && z < tau.up));
        const unsigned bi = __ballot_sync(FULL, inside);
        const unsigned bf = __ballot_sync(FULL, flag);
        const unsigned bn = __ballot_sync(FULL, valid && !fin);
        if (lane == 0 && 32 * (t >> 5) < rows) bits[(base >> 5) + (t >> 5)] = bi;
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

// hidden layer l of a tile: aout[m][n] = act(b_n + sum_k W[n][k] ain[m][k]) for MI*16 rows,
// act = ReLU or sin (NB_ACT_SINE), and, when cout is given, cout[m][n] = act'(the same sum)
// -- cos for sine, the backward pass's factor.  Thread (tm, tn) owns rows tm + 16 i and
// neurons tn + 16 j.
template <int NJ, int MI>
__device__ __forceinline__ void hidden_layer_tile(const float *__restrict__ W, const float *__restrict__ b, int K,
                                                  int N, const float *ain, float *aout, float *wt, int KP, int act,
                                                  float *cout) {
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
            for (int i = 0; i < MI; i++) {
                const int o = (tm + 16 * i) * KP + nn;
                if (act == NB_ACT_SINE) {
                    float sv, cv;
                    sincosf(acc[i][j], &sv, &cv);
                    aout[o] = sv;
                    if (cout) cout[o] = cv;
                } else {
                    aout[o] = fmaxf(acc[i][j], 0.f);
                }
            }
    }
}

// Hidden layer from the transposed weights Wt = W^T [K][N] (contiguous rows, 16-byte
// aligned when N is a multiple of four), NJ >= 4: thread (tm, tn) owns rows tm + 16 i and
// groups of four consecutive neurons 64 g + 4 tn + e; activations are read as float4s along
// k and weights as float4s along n (16 threads read 256 consecutive bytes), so a shared-
// memory load feeds 4 MI (activations) or 4 MI (weights) FMAs instead of MI or 1.  The
// weights are staged in two CK_T-row buffers: the next chunk is loaded into registers while
// the current one's products run, then stored into the other buffer; one barrier per chunk.
// aout[m][n] = act(b_n + sum_k W[n][k] ain[m][k]); KP a multiple of four.
template <int NJ, int MI>
__device__ __forceinline__ void hidden_layer_tile_t(const float *__restrict__ Wt, const float *__restrict__ b, int K,
                                                    int N, const float *ain, float *aout, float *wt, int KP, int act) {
    constexpr int CK = CK_T;
    const int WS = KP;
    const int t = threadIdx.x, tn = t & 15, tm = t >> 4;
    auto neuron = [&](int j) { return 64 * (j >> 2) + 4 * tn + (j & 3); };
    float acc[MI][NJ];
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        const int nn = neuron(j);
        const float bv = nn < N ? __ldg(b + nn) : 0.f;
#pragma unroll
        for (int i = 0; i < MI; i++) acc[i][j] = bv;
    }
    auto stage = [&](float *dst, int kc, int kw) {
        for (int e = t; e < N * CK; e += blockDim.x) {
            const int kk = e / N, nn = e % N;
            dst[kk * WS + nn] = kk < kw ? __ldg(Wt + (size_t)(kc + kk) * N + nn) : 0.f;
        }
    };
    auto chunk = [&](const float *w_s, int kc, int kw) {
        int kk = 0;
        for (; kk + 4 <= kw; kk += 4) {
            float a[MI][4];
#pragma unroll
            for (int i = 0; i < MI; i++) {
                const float4 a4 = *reinterpret_cast<const float4 *>(ain + (tm + 16 * i) * KP + kc + kk);
                a[i][0] = a4.x;
                a[i][1] = a4.y;
                a[i][2] = a4.z;
                a[i][3] = a4.w;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                float w[NJ];
#pragma unroll
                for (int q4 = 0; q4 < NJ / 4; q4++) {
                    const float4 w4 = *reinterpret_cast<const float4 *>(w_s + (kk + u) * WS + 64 * q4 + 4 * tn);
                    w[4 * q4] = w4.x;
                    w[4 * q4 + 1] = w4.y;
                    w[4 * q4 + 2] = w4.z;
                    w[4 * q4 + 3] = w4.w;
                }
#pragma unroll
                for (int i = 0; i < MI; i++)
#pragma unroll
                    for (int j = 0; j < NJ; j++) acc[i][j] = fmaf(a[i][u], w[j], acc[i][j]);
            }
        }
        for (; kk < kw; kk++) {
            float a[MI];
#pragma unroll
            for (int i = 0; i < MI; i++) a[i] = ain[(tm + 16 * i) * KP + kc + kk];
#pragma unroll
            for (int j = 0; j < NJ; j++) {
                const float w = w_s[kk * WS + neuron(j)];
#pragma unroll
                for (int i = 0; i < MI; i++) acc[i][j] = fmaf(a[i], w, acc[i][j]);
            }
        }
    };
    constexpr int PRE = (CK * 16 * NJ / 4 + 255) / 256;
    const bool vload = (N % 4 == 0) && ((reinterpret_cast<uintptr_t>(Wt) & 15u) == 0);
    const int nch = (K + CK - 1) / CK;
    __syncthreads();  // inputs written, the previous layer's chunks consumed
    stage(wt, 0, min(CK, K));
    __syncthreads();
    for (int c = 0; c < nch; c++) {
        const int kc = c * CK, kw = min(CK, K - kc);
        const bool next = c + 1 < nch;
        const int kn = kc + CK, kwn = next ? min(CK, K - kn) : 0;
        float4 pre[PRE];
        if (next && vload) {
            const float4 *src = reinterpret_cast<const float4 *>(Wt + (size_t)kn * N);
            const int n4 = kwn * N / 4;
#pragma unroll
            for (int r = 0; r < PRE; r++) {
                const int e4 = t + 256 * r;
                pre[r] = e4 < n4 ? __ldg(src + e4) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        chunk(wt + (c & 1) * CK * WS, kc, kw);
        if (next) {
            float *dst = wt + ((c + 1) & 1) * CK * WS;
            if (vload) {
                const int n4 = kwn * N / 4;
#pragma unroll
                for (int r = 0; r < PRE; r++) {
                    const int e4 = t + 256 * r;
                    if (e4 < n4) {
                        const int e = 4 * e4, kk = e / N, nn = e % N;
                        *reinterpret_cast<float4 *>(dst + kk * WS + nn) = pre[r];
                    }
                }
            } else {
                stage(dst, kn, kwn);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        const int nn = neuron(j);
        if (nn < N)
#pragma unroll
            for (int i = 0; i < MI; i++)
                aout[(tm + 16 * i) * KP + nn] = act == NB_ACT_SINE ? sinf(acc[i][j]) : fmaxf(acc[i][j], 0.f);
    }
}

__device__ __forceinline__ float softplusf(float u) { return u > 0.f ? u + log1pf(expf(-u)) : log1pf(expf(u)); }
__device__ __forceinline__ float sigmoidf(float u) {
    return u >= 0.f ? 1.f / (1.f + expf(-u)) : expf(u) / (1.f + expf(u));
}

// One tile of TM training samples starting at global row `base` (rows valid): forward
// keeping every layer's activations in shared memory, the asymmetric BCE of Eq. (loss)
// with its derivative scaled by inv_n (batch mean), and the backward pass accumulating
// dW and db into `slot` (a gradient partial owned by the calling CTA).
// smem: [L][TM][KP] activations, 2 x [TM][KP] deltas, [KC][16 NJ + 1] weight chunk, and for
// sine networks [L][TM][KP] activation derivatives cos(z) (layer l's at l).
template <int NJ, int TM>
__device__ __forceinline__ void train_tile(const MlpDesc &d, const float *__restrict__ q,
                                           const uint32_t *__restrict__ labels, long long base, int rows,
                                           float alpha, float beta, float inv_n, TauF tau, float *__restrict__ slot,
                                           float *smem, float *zs, float *dz, float *ls, float &lossacc,
                                           unsigned long long &c_fn, unsigned long long &c_fp,
                                           unsigned long long &c_nf) {
    constexpr int NP = 16 * NJ, KP = NP + 1, MI = TM / 16, WS = NP + 1;
    constexpr int TPQ = 256 / TM;  // threads per sample in the output layer
    const int L = d.L;
    float *acts = smem;
    float *dcur = acts + (size_t)L * TM * KP;
    float *dnext = dcur + TM * KP;
    float *wt = dnext + TM * KP;
    float *cs = wt + KC * WS;  // sine networks only
    const bool sine = d.act == NB_ACT_SINE;
    const int t = threadIdx.x, tn = t & 15, tm = t >> 4;
    const int w0 = d.w[0];
    __syncthreads();
    for (int e = t; e < TM * w0; e += blockDim.x) {
        const int m = e / w0, k = e % w0;
        acts[m * KP + k] = m < rows ? q[(base + m) * w0 + k] : 0.f;
    }
    for (int l = 0; l < L - 1; l++) {
        const int K = d.w[l], N = d.w[l + 1];
        const float *W = d.p + d.off[l];
        hidden_layer_tile<NJ, MI>(W, W + (size_t)N * K, K, N, acts + (size_t)l * TM * KP,
                                  acts + (size_t)(l + 1) * TM * KP, wt, KP, d.act,
                                  sine ? cs + (size_t)(l + 1) * TM * KP : nullptr);
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
            bool xfin = true;  // a non-finite input coordinate counts as a non-finite logit
            for (int k = 0; k < w0; k++) xfin = xfin && isfinite(acts[m * KP + k]);
            if (isfinite(z) && xfin) {
                // Eq. (loss): -alpha y log(s) - beta (1-y) log(1-s), s = sigmoid(z)
                lv = alpha * y * softplusf(-z) + beta * (1.f - y) * softplusf(z);
                const float sg = sigmoidf(z);
                g = (alpha * y * (sg - 1.f) + beta * (1.f - y) * sg) * inv_n;
                const bool dec = z >= tau.up;
                c_fn += (y != 0.f && !dec);
                c_fp += (y == 0.f && dec);
            } else {
                c_nf++;
                // the skipped sample must not meet its zero gradient with an inf or NaN
                // activation in the weight products
                for (int l = 0; l < L; l++)
                    for (int k = 0; k < KP; k++) {
                        acts[(size_t)l * TM * KP + m * KP + k] = 0.f;
                        if (sine) cs[(size_t)l * TM * KP + m * KP + k] = 0.f;
                    }
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
                const float dv = dz[m] * __ldg(WL + k);
                dcur[m * KP + k] = sine ? dv * cs[(size_t)(L - 1) * TM * KP + m * KP + k] : (a > 0.f ? dv : 0.f);
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
            // delta_l[m][k] = (sum_n delta_{l+1}[m][n] W[n][k]) act'(z_l[m][k]): 1[a_l > 0] or cos
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
                        dnext[m * KP + k] = sine ? acc[i][j] * cs[(size_t)l * TM * KP + m * KP + k]
                                                 : (al[m * KP + k] > 0.f ? acc[i][j] : 0.f);
                    }
            }
            __syncthreads();
            float *tp = dcur;
            dcur = dnext;
            dnext = tp;
        }
    }

}

}  // namespace nbf32
