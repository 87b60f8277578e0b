// Rigorous evaluation of the decision z >= tau for the queries the fast path could not
// settle (fast logit within the margin of tau), and the bound pass of the threshold
// calibration (Suppl. "Numerics": output epsilon; the calibrated threshold keeps the
// calibration set free of false negatives).
//
// Stage 1 (bound_tile_kernel): FP32 forward over tiles of listed queries carrying,
// for every neuron, a bound B >= |computed - exact| on the distance of the computed
// value to the exact real-valued network output on the same input:
//     B_n = gamma_l |b_n| + sum_k |W_nk| (gamma_l |a^_k| + e_k),
// gamma_l = gamma_{fan-in + 8} covering the rounding of this layer's dot product
// (at most fan-in + 8 roundings per term, any order), e_k the propagated bound of the
// inputs; ReLU is 1-Lipschitz so e_n = B_n after it -- and e_n = 0 where the computed value
// is certainly negative (computed + B_n < 0, evaluated rounding up): the exact value is then
// negative too, and both activations are exactly 0.  On trained networks most of the error
// flows through inactive neurons otherwise: on a 256-wide box network this cut the bound
// of the last layer about 180-fold and let stage 1 settle 99 % of the margin band instead
// of 1 %.  The sinusoidal activation
// (NB_ACT_SINE) is 1-Lipschitz too: e_n = B_n + 2^-22, the second term covering CUDA's
// sinf (documented maximum error 2 ulp; |sin| <= 1, so 2 ulp <= 2^-22).  Every bound is
// accumulated with upward rounding, so it only over-estimates.  One extra FMA per MAC.
// Stage 2 (ff_kernel): the queries stage 1 leaves ambiguous are evaluated with
// error-free transformations (TwoProd / TwoSum, Ogita, Rump & Oishi 2005) on activations
// carried as float pairs, first as compensated dot products (2a, bound about
// gamma_{3K} u |terms|), then, for the few still ambiguous, in three-word accumulation
// (2b, bound about gamma_{4K} u^2 |terms|), each with its bound evaluated at run time.
// Sine activations of a float pair are evaluated in FP64 (CUDA's sin, documented maximum
// error 2 ulp) and split back into a pair; their bound adds that error, the rounding of
// the pair to a double and of the low word (see sine_pair).
#include <math.h>

#include "common.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr float U = 5.9604644775390625e-08f;  // unit roundoff 2^-24
constexpr int FF_WARPS_PER_SM = 32;              // stage-2 launch: 8 blocks of 4 warps per SM
constexpr float E_SINF = 2.384185791015625e-07f;  // 2^-22: |sinf(x) - sin(x)| (2 ulp at |sin| <= 1)

__device__ __forceinline__ unsigned ord_f32(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_f32(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ unsigned long long ord_f64(double f) {
    unsigned long long u = (unsigned long long)__double_as_longlong(f);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// One hidden layer over a tile, in place: a <- relu(b + W a) and e <- its bound.  Each
// thread owns MI rows x NJ neurons.  The weights are staged through shared memory KC input
// rows at a time from the transposed copy (row k of W^T is contiguous: coalesced), and the
// outputs overwrite the inputs after a barrier, so a CTA needs two activation buffers and
// one weight chunk -- a third of the shared memory of separate in/out buffers -- and two
// or more CTAs share an SM to hide the staging latency.
//
// Shared-memory loads, not the FMA pipe, bound the scalar form (2 MI + NJ loads per
// 2 MI NJ FMAs).  From NJ = 4 on, a thread owns groups of four consecutive neurons
// (64 g + 4 tn + e) and the inner loop takes four inputs at a time: the activations and
// their bounds as float4s along k, the weights as float4s along n, conflict-free (16
// threads read 256 consecutive bytes).  The row stride is then a multiple of four.
constexpr int KC = 32;
template <int NJ>
__host__ __device__ constexpr int kp_of() {
    return NJ >= 4 ? 16 * NJ + 4 : 16 * NJ + 1;
}

// the weight chunks of the vector form: CK input rows, double-buffered (2 CK WS floats)
template <int NJ>
__host__ __device__ constexpr int chunk_of() {
    return NJ >= 4 ? 16 : KC;
}
template <int NJ>
__host__ __device__ constexpr int wt_floats() {
    return NJ >= 4 ? 2 * chunk_of<NJ>() * kp_of<NJ>() : KC * kp_of<NJ>();
}

template <int NJ, int MI>
__device__ __forceinline__ void bound_layer_tile(const float *__restrict__ Wt, const float *__restrict__ b, int K,
                                                 int N, float g, float *a_s, float *e_s, float *wt, int KP, int act) {
    constexpr int WS = kp_of<NJ>();
    constexpr bool VEC = NJ >= 4;
    constexpr int CK = chunk_of<NJ>();
    const int t = threadIdx.x, tn = t & 15, tm = t >> 4;
    // neuron j of this thread
    auto neuron = [&](int j) { return VEC ? 64 * (j >> 2) + 4 * tn + (j & 3) : tn + 16 * j; };
    float acc[MI][NJ], bnd[MI][NJ];
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        const int nn = neuron(j);
        const float bv = nn < N ? __ldg(b + nn) : 0.f;
        const float bb = __fmul_ru(g, fabsf(bv));
#pragma unroll
        for (int i = 0; i < MI; i++) {
            acc[i][j] = bv;
            bnd[i][j] = bb;
        }
    }
    // rows kc .. kc + kw of W^T (contiguous: kw N floats) into buffer dst, scalar loads
    auto stage = [&](float *dst, int kc, int kw) {
        for (int e = t; e < N * CK; e += blockDim.x) {
            const int kk = e / N, nn = e % N;
            dst[kk * WS + nn] = kk < kw ? __ldg(Wt + (size_t)(kc + kk) * N + nn) : 0.f;
        }
    };
    // one chunk's products: inputs kc .. kc + kw against the staged rows in w_s
    auto chunk = [&](const float *w_s, int kc, int kw) {
        int kk = 0;
        if constexpr (VEC) {
            for (; kk + 4 <= kw; kk += 4) {
                float a[MI][4], v[MI][4];
#pragma unroll
                for (int i = 0; i < MI; i++) {
                    const int idx = (tm + 16 * i) * KP + kc + kk;
                    const float4 a4 = *reinterpret_cast<const float4 *>(a_s + idx);
                    const float4 e4 = *reinterpret_cast<const float4 *>(e_s + idx);
                    a[i][0] = a4.x;
                    a[i][1] = a4.y;
                    a[i][2] = a4.z;
                    a[i][3] = a4.w;
                    v[i][0] = __fmaf_ru(g, fabsf(a4.x), e4.x);
                    v[i][1] = __fmaf_ru(g, fabsf(a4.y), e4.y);
                    v[i][2] = __fmaf_ru(g, fabsf(a4.z), e4.z);
                    v[i][3] = __fmaf_ru(g, fabsf(a4.w), e4.w);
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
                        for (int j = 0; j < NJ; j++) {
                            acc[i][j] = fmaf(a[i][u], w[j], acc[i][j]);
                            bnd[i][j] = __fmaf_ru(v[i][u], fabsf(w[j]), bnd[i][j]);
                        }
                }
            }
        }
        for (; kk < kw; kk++) {
            float a[MI], v[MI], w[NJ];
#pragma unroll
            for (int i = 0; i < MI; i++) {
                const int idx = (tm + 16 * i) * KP + kc + kk;
                a[i] = a_s[idx];
                v[i] = __fmaf_ru(g, fabsf(a[i]), e_s[idx]);
            }
#pragma unroll
            for (int j = 0; j < NJ; j++) w[j] = w_s[kk * WS + neuron(j)];
#pragma unroll
            for (int i = 0; i < MI; i++)
#pragma unroll
                for (int j = 0; j < NJ; j++) {
                    acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
                    bnd[i][j] = __fmaf_ru(v[i], fabsf(w[j]), bnd[i][j]);
                }
        }
    };
    if constexpr (!VEC) {
        for (int kc = 0; kc < K; kc += CK) {
            const int kw = min(CK, K - kc);
            __syncthreads();  // inputs in place, previous chunk consumed
            stage(wt, kc, kw);
            __syncthreads();
            chunk(wt, kc, kw);
        }
    } else {
        // Double-buffered chunks: the next chunk's rows are loaded into registers (float4s,
        // when the rows are 16-byte aligned) while this chunk's products run, then stored
        // into the other buffer; one barrier per chunk.  A buffer is rewritten only after the
        // barrier that ends the products reading it.
        constexpr int PRE = (CK * 16 * NJ / 4 + 255) / 256;  // float4s per thread and chunk
        const bool vload = (N % 4 == 0) && ((reinterpret_cast<uintptr_t>(Wt) & 15u) == 0);
        const int nch = (K + CK - 1) / CK;
        __syncthreads();  // inputs in place, the previous layer's last chunk consumed
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
    }
    __syncthreads();  // every thread has read the inputs: overwrite them
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        const int nn = neuron(j);
        if (nn < N)
#pragma unroll
            for (int i = 0; i < MI; i++) {
                if (act == NB_ACT_SINE) {
                    a_s[(tm + 16 * i) * KP + nn] = sinf(acc[i][j]);
                    e_s[(tm + 16 * i) * KP + nn] = __fadd_ru(bnd[i][j], E_SINF);
                } else {
                    a_s[(tm + 16 * i) * KP + nn] = fmaxf(acc[i][j], 0.f);
                    // certainly inactive: both activations are exactly 0
                    e_s[(tm + 16 * i) * KP + nn] = __fadd_ru(acc[i][j], bnd[i][j]) < 0.f ? 0.f : bnd[i][j];
                }
            }
    }
}

// decision of z in [lo, hi] against tau: 1 inside, 0 outside, -1 undecided
__device__ __forceinline__ int decide_interval(float lo, float hi, TauF tau) {
    if (lo >= tau.up) return 1;
    if (hi < tau.dn || (tau.dn == tau.up && hi < tau.up)) return 0;
    return -1;
}

// MODE 0: re-check listed queries, settle their bits, forward the rest to stage 2.
// MODE 1: calibration: lower bound of every listed (positive) query -> lo_out,
//         minimum upper bound -> umin_bits.
template <int NJ, int MI, int MODE>
__global__ void __launch_bounds__(256, (NJ >= 16 && MI >= 4) ? 1 : 2) bound_tile_kernel(const __grid_constant__ MlpDesc d, const __grid_constant__ GammaTab gt,
                                                         const float *__restrict__ q, TauF tau,
                                                         const unsigned *count, const unsigned *idx, uint32_t *bits,
                                                         nb_query_stats *st, unsigned *ff_count, unsigned *ff_idx,
                                                         float *lo_out, unsigned *umin_bits, unsigned direct_max) {
    constexpr int TM = 16 * MI, KP = kp_of<NJ>(), TPQ = 256 / TM;
    extern __shared__ float smem[];
    float *a0 = smem, *e0 = a0 + TM * KP, *wt = e0 + TM * KP;
    __shared__ unsigned rowidx[TM];
    __shared__ float zs[TM], bs[TM];
    const int t = threadIdx.x, w0 = d.w[0];
    const unsigned cnt = *count;
    if (MODE == 0 && cnt <= direct_max) {
        // a band this small is settled sooner by stage 2 alone: hand it over whole
        for (unsigned f = blockIdx.x * blockDim.x + t; f < cnt; f += gridDim.x * blockDim.x) ff_idx[f] = idx[f];
        if (blockIdx.x == 0 && t == 0) *ff_count = cnt;
        return;
    }
    const unsigned ntiles = (cnt + TM - 1) / TM;
    unsigned long long r32 = 0;
    long long dinside = 0;
    unsigned umin = 0xffffffffu;
    for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int rows = (int)min((unsigned)TM, cnt - tile * TM);
        __syncthreads();
        if (t < TM) rowidx[t] = t < rows ? idx[tile * TM + t] : 0u;
        __syncthreads();
        for (int e = t; e < TM * w0; e += blockDim.x) {
            const int m = e / w0, k = e % w0;
            a0[m * KP + k] = m < rows ? q[(size_t)rowidx[m] * w0 + k] : 0.f;
            e0[m * KP + k] = 0.f;
        }
        const float *ain = a0, *ein = e0;
        for (int l = 0; l < d.L - 1; l++) {
            const int K = d.w[l], N = d.w[l + 1];
            const float *Wt = d.pT + d.off[l];
            bound_layer_tile<NJ, MI>(Wt, Wt + (size_t)N * K, K, N, gt.g[l], a0, e0, wt, KP, d.act);
        }
        __syncthreads();
        {
            const int K = d.w[d.L - 1];
            const float *W = d.p + d.off[d.L - 1];
            const float g = gt.g[d.L - 1];
            const int m = t / TPQ, part = t % TPQ;
            float s = 0.f, bb = 0.f;
            for (int k = part; k < K; k += TPQ) {
                const float w = __ldg(W + k), a = ain[m * KP + k];
                s = fmaf(w, a, s);
                bb = __fmaf_ru(fabsf(w), __fmaf_ru(g, fabsf(a), ein[m * KP + k]), bb);
            }
#pragma unroll
            for (int o = 1; o < TPQ; o <<= 1) {
                s += __shfl_xor_sync(FULL, s, o);
                bb = __fadd_ru(bb, __shfl_xor_sync(FULL, bb, o));
            }
            if (part == 0) {
                const float bL = __ldg(W + K);
                zs[m] = s + bL;
                bs[m] = __fmaf_ru(g, fabsf(bL), bb);
            }
        }
        __syncthreads();
        if (t < rows) {
            const unsigned i = rowidx[t];
            const float z = zs[t], B = bs[t];
            const float lo = __fsub_rd(z, B), hi = __fadd_ru(z, B);
            if (MODE == 0) {
                int dec = decide_interval(lo, hi, tau);
                if (dec < 0) {
                    ff_idx[atomicAdd(ff_count, 1u)] = i;  // stage 2 settles this bit
                } else {
                    r32++;
                    const unsigned bit = 1u << (i & 31);
                    const unsigned old = dec ? atomicOr(bits + (i >> 5), bit) : atomicAnd(bits + (i >> 5), ~bit);
                    dinside += dec - (int)((old & bit) != 0);
                }
            } else {
                float l2 = lo, h2 = hi;
                if (!(l2 == l2) || !(h2 == h2)) {  // NaN: always a candidate
                    l2 = -INFINITY;
                    h2 = -INFINITY;
                }
                lo_out[tile * TM + t] = l2;
                umin = min(umin, ord_f32(h2));
            }
        }
    }
    if (MODE == 0) {
        if (st && t < TM) {
            unsigned long long rr = r32;
            long long di = dinside;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                rr += __shfl_xor_sync(FULL, rr, o);
                di += __shfl_xor_sync(FULL, di, o);
            }
            if ((t & 31) == 0) {
                if (rr) atomicAdd(&st->n_resolved_f32, rr);
                if (di) atomicAdd(&st->n_inside, (unsigned long long)di);
            }
        }
    } else if (t < TM) {
#pragma unroll
        for (int o = 16; o; o >>= 1) umin = min(umin, __shfl_xor_sync(FULL, umin, o));
        if ((t & 31) == 0 && umin != 0xffffffffu) atomicMin(umin_bits, umin);
    }
}

// ---------------------------------------------------------------- float-float stage
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Extended-precision dot product of one neuron: z = b + sum_k W_k (h_k + l_k) on
// inputs given as float pairs (h, l) carrying bounds e_k.  Every product is split
// exactly (TwoProd) and accumulated in three words s1 + s2 + s3: s1 and s2 by
// error-free TwoSum chains, s3 (terms of size O(K u^2)) by plain additions.  The
// result is renormalised to a pair (hi, lo).  s1 + s2 + (exact sum of the s3 terms)
// equals the exact dot product, so the only roundings are the 4K additions into s3
// and the last addition lo = t4 + t3.  Bound on |hi + lo - exact|, all evaluated with
// upward rounding at run time:
//     gamma_{4K+4} A3 + 2u (|t4| + |t3|) + sum_k |W_k| e_k,
// A3 = sum of the magnitudes of the terms added into s3, g4 = gamma_{4K+4}.
__device__ __forceinline__ void ff_neuron(const float *__restrict__ Wr, int stride, float bv, int K, float g4,
                                          const float *h, const float *l, const float *e, float &hi, float &lo,
                                          float &bound) {
    float s1 = bv, s2 = 0.f, s3 = 0.f, A3 = 0.f, P = 0.f;
    for (int k = 0; k < K; k++) {
        const float w = __ldg(Wr + (size_t)k * stride), hk = h[k], lk = l[k];
        const float p = __fmul_rn(w, hk);
        const float pq = fmaf(w, hk, -p);  // w hk = p + pq exactly
        const float r = __fmul_rn(w, lk);
        const float rq = fmaf(w, lk, -r);  // w lk = r + rq exactly
        float t, e1, e2, e3, e4;
        two_sum(s1, p, t, e1);
        s1 = t;
        two_sum(s2, e1, t, e2);
        s2 = t;
        two_sum(s2, pq, t, e3);
        s2 = t;
        two_sum(s2, r, t, e4);
        s2 = t;
        s3 = __fadd_rn(s3, e2);
        s3 = __fadd_rn(s3, e3);
        s3 = __fadd_rn(s3, e4);
        s3 = __fadd_rn(s3, rq);
        A3 = __fadd_ru(A3, __fadd_ru(__fadd_ru(fabsf(e2), fabsf(e3)), __fadd_ru(fabsf(e4), fabsf(rq))));
        P = __fmaf_ru(fabsf(w), e[k], P);
    }
    float t2, t3, t4;
    two_sum(s2, s3, t2, t3);
    two_sum(s1, t2, hi, t4);
    lo = __fadd_rn(t4, t3);
    bound = __fmaf_ru(g4, A3, __fmaf_ru(2.f * U, __fadd_ru(fabsf(t4), fabsf(t3)), P));
}

// Compensated dot products (Dot2, Ogita, Rump & Oishi 2005) of the neurons nn0, nn0 + 32,
// ..., nn0 + 32 (NB - 1) of one layer (those below N), on inputs given as float pairs
// (h, l) carrying bounds e.  Per input: the product w h is split exactly (p + pq), p is
// added to the running sum s by an error-free TwoSum (error er), and er, pq and w l are
// accumulated in a second word c.  s plus the exact sum of the c terms equals
// b + sum_k w (h_k + l_k), so the only roundings are the 3K additions into c:
//     |hi + lo - exact| <= gamma_{3K} A + sum_k |w_k| e_k,
// A = sum of the magnitudes of the c terms, both evaluated with upward rounding, and
// (hi, lo) = TwoSum(s, c) holding s + c exactly.  About 15 operations per product, where
// the three-word evaluation below takes about 40 and a bound near u^2 instead of u.
template <int NB>
__device__ __forceinline__ void dot2_core(const float *__restrict__ Wt, const float *__restrict__ bias, int K, int N,
                                          int nn0, float g3, const float *h, const float *l, const float *e,
                                          float (&hi)[NB], float (&lo)[NB], float (&bd)[NB]) {
    float s[NB], c[NB], A[NB], P[NB];
    const float *Wr[NB];
#pragma unroll
    for (int j = 0; j < NB; j++) {
        const int nn = nn0 + 32 * j;
        const bool ok = nn < N;
        Wr[j] = Wt + (ok ? nn : 0);
        s[j] = ok ? __ldg(bias + nn) : 0.f;
        c[j] = 0.f;
        A[j] = 0.f;
        P[j] = 0.f;
    }
    // The weights of the next KB inputs are loaded while the current KB are accumulated:
    // one warp walks one query through the network, so without this every input would
    // wait for its weights' round trip to L2.  The arithmetic and its order are unchanged.
    constexpr int KB = 8;
    float wn[KB][NB];
#pragma unroll
    for (int kk = 0; kk < KB; kk++)
#pragma unroll
        for (int j = 0; j < NB; j++) wn[kk][j] = kk < K ? __ldg(Wr[j] + (size_t)kk * N) : 0.f;
    for (int k0 = 0; k0 < K; k0 += KB) {
        float wc[KB][NB];
#pragma unroll
        for (int kk = 0; kk < KB; kk++)
#pragma unroll
            for (int j = 0; j < NB; j++) wc[kk][j] = wn[kk][j];
#pragma unroll
        for (int kk = 0; kk < KB; kk++)
#pragma unroll
            for (int j = 0; j < NB; j++)
                wn[kk][j] = k0 + KB + kk < K ? __ldg(Wr[j] + (size_t)(k0 + KB + kk) * N) : 0.f;
#pragma unroll
        for (int kk = 0; kk < KB; kk++) {
            const int k = k0 + kk;
            if (k >= K) break;
            const float hk = h[k], lk = l[k], ek = e[k];
#pragma unroll
            for (int j = 0; j < NB; j++) {
                const float w = wc[kk][j];
                const float p = __fmul_rn(w, hk);
                const float pq = fmaf(w, hk, -p);  // w hk = p + pq exactly
                float t, er;
                two_sum(s[j], p, t, er);
                s[j] = t;
                c[j] = __fadd_rn(__fadd_rn(c[j], er), pq);
                c[j] = fmaf(w, lk, c[j]);
                A[j] = __fmaf_ru(fabsf(w), fabsf(lk), __fadd_ru(A[j], __fadd_ru(fabsf(er), fabsf(pq))));
                P[j] = __fmaf_ru(fabsf(w), ek, P[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NB; j++) {
        two_sum(s[j], c[j], hi[j], lo[j]);
        bd[j] = __fmaf_ru(g3, A[j], P[j]);
    }
}

// relu(hi + lo) as a pair: |lo| is far below |hi| unless hi = 0, so the sign is hi's
__device__ __forceinline__ void relu_pair(float hi, float lo, float &h2, float &l2) {
    if (hi > 0.f) {
        h2 = hi;
        l2 = lo;
    } else {
        h2 = hi == 0.f ? fmaxf(lo, 0.f) : 0.f;
        l2 = 0.f;
    }
}

// sin(hi + lo) as a pair (h2, l2) and what it adds to the propagated bound bd (sin is
// 1-Lipschitz, so bd carries over): hi + lo rounded to a double (<= 2^-53 |hi + lo|),
// CUDA's sin (2 ulp, <= 2^-52 at |sin| <= 1), and the float low word (<= 2^-48, since
// |s - h2| <= 2^-24 |s| and the low word rounds that to 24 bits); 2^-47 + 2^-53 |x|
// covers the sum.
__device__ __forceinline__ void sine_pair(float hi, float lo, float bd, float &h2, float &l2, float &e2) {
    const double sv = sin((double)hi + (double)lo);
    h2 = (float)sv;
    l2 = (float)(sv - (double)h2);
    const float ax = __fadd_ru(fabsf(hi), fabsf(lo));
    e2 = __fadd_ru(bd, __fmaf_ru(1.1102230246251565e-16f, ax, 7.105427357601002e-15f));
}

// the activation of a pair with its bound; a ReLU neuron whose computed value is certainly
// negative (hi + lo + bd < 0, rounding up) is exactly 0 in both networks: no error
__device__ __forceinline__ void act_pair(int act, float hi, float lo, float bd, float &h2, float &l2, float &e2) {
    if (act == NB_ACT_SINE) {
        sine_pair(hi, lo, bd, h2, l2, e2);
    } else {
        relu_pair(hi, lo, h2, l2);
        e2 = __fadd_ru(__fadd_ru(hi, lo), bd) < 0.f ? 0.f : bd;
    }
}

template <int NB>
__device__ __forceinline__ void dot2_neurons_relu(const float *__restrict__ Wt, const float *__restrict__ bias, int K,
                                                  int N, int nn0, float g3, const float *h, const float *l,
                                                  const float *e, float *h2, float *l2, float *e2, int act) {
    float hi[NB], lo[NB], bd[NB];
    dot2_core<NB>(Wt, bias, K, N, nn0, g3, h, l, e, hi, lo, bd);
#pragma unroll
    for (int j = 0; j < NB; j++) {
        const int nn = nn0 + 32 * j;
        if (nn < N) act_pair(act, hi[j], lo[j], bd[j], h2[nn], l2[nn], e2[nn]);
    }
}

// ff_neuron for the neurons nn0, nn0 + 32, ..., nn0 + 32 (NB - 1) of one layer (those
// below N), their chains interleaved so that the dependent TwoSum sequences of different
// neurons overlap; every neuron's arithmetic is exactly that of ff_neuron.  Writes
// relu(hi + lo) as a pair and the propagated bound.
template <int NB>
__device__ __forceinline__ void ff_neurons_relu(const float *__restrict__ Wt, const float *__restrict__ bias, int K,
                                                int N, int nn0, float g4, const float *h, const float *l,
                                                const float *e, float *h2, float *l2, float *e2, int act) {
    float s1[NB], s2[NB], s3[NB], A3[NB], P[NB];
    const float *Wr[NB];
#pragma unroll
    for (int j = 0; j < NB; j++) {
        const int nn = nn0 + 32 * j;
        const bool ok = nn < N;
        Wr[j] = Wt + (ok ? nn : 0);
        s1[j] = ok ? __ldg(bias + nn) : 0.f;
        s2[j] = 0.f;
        s3[j] = 0.f;
        A3[j] = 0.f;
        P[j] = 0.f;
    }
    for (int k = 0; k < K; k++) {
        const float hk = h[k], lk = l[k], ek = e[k];
#pragma unroll
        for (int j = 0; j < NB; j++) {
            const float w = __ldg(Wr[j] + (size_t)k * N);
            const float p = __fmul_rn(w, hk);
            const float pq = fmaf(w, hk, -p);
            const float r = __fmul_rn(w, lk);
            const float rq = fmaf(w, lk, -r);
            float t, e1, ea, eb, ec;
            two_sum(s1[j], p, t, e1);
            s1[j] = t;
            two_sum(s2[j], e1, t, ea);
            s2[j] = t;
            two_sum(s2[j], pq, t, eb);
            s2[j] = t;
            two_sum(s2[j], r, t, ec);
            s2[j] = t;
            s3[j] = __fadd_rn(s3[j], ea);
            s3[j] = __fadd_rn(s3[j], eb);
            s3[j] = __fadd_rn(s3[j], ec);
            s3[j] = __fadd_rn(s3[j], rq);
            A3[j] = __fadd_ru(A3[j], __fadd_ru(__fadd_ru(fabsf(ea), fabsf(eb)), __fadd_ru(fabsf(ec), fabsf(rq))));
            P[j] = __fmaf_ru(fabsf(w), ek, P[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < NB; j++) {
        const int nn = nn0 + 32 * j;
        if (nn < N) {
            float t2, t3, t4, hi;
            two_sum(s2[j], s3[j], t2, t3);
            two_sum(s1[j], t2, hi, t4);
            const float lo = __fadd_rn(t4, t3);
            const float bd = __fmaf_ru(g4, A3[j], __fmaf_ru(2.f * U, __fadd_ru(fabsf(t4), fabsf(t3)), P[j]));
            act_pair(act, hi, lo, bd, h2[nn], l2[nn], e2[nn]);
        }
    }
}

// One warp per query still ambiguous after stage 1.  STAGE 0: compensated (Dot2)
// evaluation; queries it cannot decide are appended to (out_count, out_idx).  STAGE 1:
// three-word evaluation; queries it cannot decide are decided inside (conservative) and
// counted as unresolved.
// Grouped form: when `offsets` is given, query i belongs to the object o with
// offsets[o] <= i < offsets[o+1], whose parameters start at d.pT + o * P and whose
// threshold is taus[o].
template <int STAGE>
__global__ void __launch_bounds__(128) ff_kernel(MlpDesc d, GammaTab gt, const float *__restrict__ q, TauF tau0,
                                                 const unsigned *ff_count, const unsigned *ff_idx, uint32_t *bits,
                                                 nb_query_stats *st, const long long *offsets, int n_objects,
                                                 long long P, const TauF *taus, unsigned *out_count,
                                                 unsigned *out_idx) {
    __shared__ float sh_[4][3][2][NB_MAXW];  // [warp][h,l,e][buffer][k]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned cnt = *ff_count;
    unsigned long long rff = 0, unres = 0;
    long long dinside = 0;
    for (unsigned f = blockIdx.x * 4 + warp; f < cnt; f += gridDim.x * 4) {
        const unsigned i = ff_idx[f];
        MlpDesc dd = d;
        TauF tau = tau0;
        if (offsets) {
            int lo_o = 0, hi_o = n_objects - 1;  // last object whose first row is <= i
            while (lo_o < hi_o) {
                const int mid = (lo_o + hi_o + 1) >> 1;
                if (offsets[mid] <= (long long)i) lo_o = mid; else hi_o = mid - 1;
            }
            dd.pT = d.pT + (size_t)lo_o * P;
            tau = taus[lo_o];
        }
        float *h = sh_[warp][0][0], *l = sh_[warp][1][0], *e = sh_[warp][2][0];
        float *h2 = sh_[warp][0][1], *l2 = sh_[warp][1][1], *e2 = sh_[warp][2][1];
        const float *x = q + (size_t)i * d.w[0];
        for (int k = lane; k < d.w[0]; k += 32) {
            h[k] = x[k];
            l[k] = 0.f;
            e[k] = 0.f;
        }
        __syncwarp();
        for (int ly = 0; ly < d.L - 1; ly++) {
            const int K = d.w[ly], N = d.w[ly + 1];
            const float *W = dd.pT + dd.off[ly];  // W_l transposed: [K][N]
            for (int nn0 = lane; nn0 < N; nn0 += 32 * 4) {
                if (STAGE == 0)
                    dot2_neurons_relu<4>(W, W + (size_t)N * K, K, N, nn0, gt.gd2[ly], h, l, e, h2, l2, e2, d.act);
                else
                    ff_neurons_relu<4>(W, W + (size_t)N * K, K, N, nn0, gt.gff[ly], h, l, e, h2, l2, e2, d.act);
            }
            __syncwarp();
            float *tp = h;
            h = h2;
            h2 = tp;
            tp = l;
            l = l2;
            l2 = tp;
            tp = e;
            e = e2;
            e2 = tp;
        }
        if (lane == 0) {
            const int K = d.w[d.L - 1];
            const float *W = dd.pT + dd.off[d.L - 1];
            float zh, zl, B;
            if (STAGE == 0) {
                float hh[1], ll[1], bb[1];
                dot2_core<1>(W, W + K, K, 1, 0, gt.gd2[d.L - 1], h, l, e, hh, ll, bb);
                zh = hh[0];
                zl = ll[0];
                B = bb[0];
            } else {
                ff_neuron(W, 1, __ldg(W + K), K, gt.gff[d.L - 1], h, l, e, zh, zl, B);
            }
            // D = z - tau in float-float: (s, ee) = zh - tau_hi exactly, t = (zl - tau_lo) + ee
            float s, ee;
            two_sum(zh, -tau.hi, s, ee);
            const float tt = __fadd_rn(__fsub_rn(zl, tau.lo), ee);
            const float Et = __fmul_ru(3.f * U, __fadd_ru(__fadd_ru(fabsf(zl), fabsf(tau.lo)), fabsf(ee)));
            const float v = __fadd_rn(s, tt);
            const float M = __fadd_ru(__fadd_ru(__fadd_ru(B, Et), tau.err), __fmul_ru(2.f * U, fabsf(v)));
            int dec;
            if (__fsub_rd(v, M) >= 0.f) {
                dec = 1;
                rff++;
            } else if (__fadd_ru(v, M) < 0.f) {
                dec = 0;
                rff++;
            } else if (STAGE == 0) {
                out_idx[atomicAdd(out_count, 1u)] = i;  // the three-word stage settles this bit
                dec = -1;
            } else {
                dec = 1;  // unresolved: conservative
                unres++;
            }
            if (dec >= 0) {
                const unsigned bit = 1u << (i & 31);
                const unsigned old = dec ? atomicOr(bits + (i >> 5), bit) : atomicAnd(bits + (i >> 5), ~bit);
                dinside += dec - (int)((old & bit) != 0);
            }
        }
        __syncwarp();
    }
    if (st && lane == 0) {
        if (rff) atomicAdd(&st->n_resolved_ff, rff);
        if (unres) atomicAdd(&st->n_unresolved, unres);
        if (dinside) atomicAdd(&st->n_inside, (unsigned long long)dinside);
    }
}

// ---------------------------------------------------------------- calibration helpers
// list of the indices whose label bit is 1
__global__ void compact_positive_kernel(const uint32_t *__restrict__ labels, long long row0, long long row1,
                                        unsigned *count, unsigned *idx) {
    const int lane = threadIdx.x & 31;
    const long long nw = (row1 - row0 + 31) / 32;
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw;
         w += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long i = row0 + w * 32 + lane;
        const bool pos = i < row1 && ((labels[i >> 5] >> (i & 31)) & 1u);
        const unsigned b = __ballot_sync(FULL, pos);
        if (!b) continue;
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(count, (unsigned)__popc(b));
        base = __shfl_sync(FULL, base, 0);
        if (pos) idx[base + __popc(b & ((1u << lane) - 1u))] = (unsigned)i;
    }
}

// FP64 forward of the candidates for the minimum (lower bound <= minimum upper bound)
__global__ void __launch_bounds__(256) calib_f64_kernel(MlpDesc d, const float *__restrict__ q, const unsigned *count,
                                                        const unsigned *idx, const float *__restrict__ lo,
                                                        const unsigned *umin_bits, unsigned long long *zmin_bits) {
    __shared__ double sa[8][2 * NB_MAXW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned cnt = *count;
    const float umin = unord_f32(*umin_bits);
    unsigned long long best = ~0ull;
    for (unsigned j = blockIdx.x * 8 + warp; j < cnt; j += gridDim.x * 8) {
        if (!(lo[j] <= umin)) continue;
        double *a = sa[warp], *a2 = sa[warp] + NB_MAXW;
        const float *x = q + (size_t)idx[j] * d.w[0];
        for (int k = lane; k < d.w[0]; k += 32) a[k] = (double)x[k];
        __syncwarp();
        for (int l = 0; l < d.L - 1; l++) {
            const int K = d.w[l], N = d.w[l + 1];
            const float *Wt = d.pT + d.off[l];
            for (int nn = lane; nn < N; nn += 32) {
                double s = (double)__ldg(Wt + (size_t)N * K + nn);
                for (int k = 0; k < K; k++) s = fma((double)__ldg(Wt + (size_t)k * N + nn), a[k], s);
                a2[nn] = d.act == NB_ACT_SINE ? sin(s) : (s > 0.0 ? s : 0.0);
            }
            __syncwarp();
            double *tp = a;
            a = a2;
            a2 = tp;
        }
        const int K = d.w[d.L - 1];
        const float *W = d.p + d.off[d.L - 1];
        double s = 0.0;
        for (int k = lane; k < K; k += 32) s = fma((double)__ldg(W + k), a[k], s);
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        s += (double)__ldg(W + K);
        __syncwarp();
        if (lane == 0) best = min(best, (s == s) ? ord_f64(s) : 0ull);  // NaN sorts lowest
    }
    if (lane == 0 && best != ~0ull) atomicMin(zmin_bits, best);
}

// pT[o][.] <- p[o][.] with W_l[n][k] moved to [k][n]; biases copied in place
__global__ void transpose_params_kernel(MlpDesc d, float *__restrict__ pT, long long P) {
    const float *p = d.p + (size_t)blockIdx.y * P;
    float *o = pT + (size_t)blockIdx.y * P;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (long long)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < d.L && e >= d.off[l + 1]) l++;
        const long long local = e - d.off[l];
        const int K = d.w[l], N = d.w[l + 1];
        if (local < (long long)N * K) {
            const long long nn = local / K, k = local % K;
            o[d.off[l] + k * N + nn] = p[e];
        } else {
            o[e] = p[e];
        }
    }
}

int num_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

template <int NJ, int MI, int MODE>
nb_status tile_launch(const MlpDesc &d, const GammaTab &gt, const float *q, TauF tau, const unsigned *count,
                      const unsigned *idx, int64_t max_count, uint32_t *bits, nb_query_stats *st, unsigned *ff_count,
                      unsigned *ff_idx, float *lo_out, unsigned *umin_bits, cudaStream_t s) {
    constexpr int TM = 16 * MI, KP = kp_of<NJ>();
    const size_t smem = (size_t)(2 * TM * KP + wt_floats<NJ>()) * sizeof(float);
    auto k = bound_tile_kernel<NJ, MI, MODE>;
    NB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 1;
    NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)num_sms() * per_sm;
    const int64_t need = (max_count + TM - 1) / TM;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    // bands of at most a few queries per stage-2 warp skip stage 1 (MODE 0 only)
    const unsigned direct_max = MODE == 0 ? (unsigned)(FF_WARPS_PER_SM * 2) * (unsigned)num_sms() : 0u;
    k<<<(unsigned)grid, 256, smem, s>>>(d, gt, q, tau, count, idx, bits, st, ff_count, ff_idx, lo_out, umin_bits,
                                        direct_max);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

template <int MODE>
nb_status tile_dispatch(const MlpDesc &d, const GammaTab &gt, const float *q, TauF tau, const unsigned *count,
                        const unsigned *idx, int64_t max_count, uint32_t *bits, nb_query_stats *st,
                        unsigned *ff_count, unsigned *ff_idx, float *lo_out, unsigned *umin_bits, cudaStream_t s) {
    const int nj = (d.maxw + 15) / 16;
    if (nj <= 2)
        return tile_launch<2, 4, MODE>(d, gt, q, tau, count, idx, max_count, bits, st, ff_count, ff_idx, lo_out,
                                       umin_bits, s);
    if (nj <= 4)
        return tile_launch<4, 4, MODE>(d, gt, q, tau, count, idx, max_count, bits, st, ff_count, ff_idx, lo_out,
                                       umin_bits, s);
    if (nj <= 8)
        return tile_launch<8, 4, MODE>(d, gt, q, tau, count, idx, max_count, bits, st, ff_count, ff_idx, lo_out,
                                       umin_bits, s);
    return tile_launch<16, 4, MODE>(d, gt, q, tau, count, idx, max_count, bits, st, ff_count, ff_idx, lo_out,
                                    umin_bits, s);
}

}  // namespace

nb_status nb_launch_transpose(const MlpDesc &d, float *pT, int n_objects, long long P, cudaStream_t s) {
    const long long blocks = (P + 255) / 256;
    transpose_params_kernel<<<dim3((unsigned)(blocks < 1024 ? blocks : 1024), (unsigned)n_objects), 256, 0, s>>>(
        d, pT, P);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_launch_recheck(const MlpDesc &d, const GammaTab &gt, const float *q, TauF tau, uint32_t *bits,
                            nb_query_stats *st, QueryWs ws, int64_t n, cudaStream_t s) {
    NB_CUDA(cudaMemsetAsync(ws.ff_count, 0, sizeof(unsigned), s));
    nb_status r = tile_dispatch<0>(d, gt, q, tau, ws.flag_count, ws.flag_idx, n, bits, st, ws.ff_count, ws.ff_idx,
                                   nullptr, nullptr, s);
    if (r != NB_OK) return r;
    int64_t grid = num_sms() * (FF_WARPS_PER_SM / 4);
    if (grid > (n + 3) / 4) grid = (n + 3) / 4;
    if (grid < 1) grid = 1;
    // stage 2a (Dot2) on the stage-1 leftovers; its own leftovers go to the flag list,
    // free again once stage 1 has read it, and from there to stage 2b (three words)
    NB_CUDA(cudaMemsetAsync(ws.flag_count, 0, sizeof(unsigned), s));
    ff_kernel<0><<<(unsigned)grid, 128, 0, s>>>(d, gt, q, tau, ws.ff_count, ws.ff_idx, bits, st, nullptr, 0, 0,
                                                nullptr, ws.flag_count, ws.flag_idx);
    NB_CUDA(cudaGetLastError());
    // stage 2b sees the few queries stage 2a left (usually none): two CTAs per SM, so that
    // an empty launch costs one short wave
    const int64_t grid_b = grid < 2 * (int64_t)num_sms() ? grid : 2 * (int64_t)num_sms();
    ff_kernel<1><<<(unsigned)grid_b, 128, 0, s>>>(d, gt, q, tau, ws.flag_count, ws.flag_idx, bits, st, nullptr, 0, 0,
                                                  nullptr, nullptr, nullptr);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_launch_recheck_grouped(const MlpDesc &d, const GammaTab &gt, const float *q, const long long *offsets,
                                    int n_objects, long long P, const TauF *taus, uint32_t *bits, nb_query_stats *st,
                                    QueryWs ws, int64_t n, cudaStream_t s) {
    // the flagged queries of several objects go straight to the extended-precision stage
    int64_t grid = num_sms() * (FF_WARPS_PER_SM / 4);
    if (grid > (n + 3) / 4) grid = (n + 3) / 4;
    if (grid < 1) grid = 1;
    TauF none{};
    NB_CUDA(cudaMemsetAsync(ws.ff_count, 0, sizeof(unsigned), s));
    ff_kernel<0><<<(unsigned)grid, 128, 0, s>>>(d, gt, q, none, ws.flag_count, ws.flag_idx, bits, st, offsets,
                                                n_objects, P, taus, ws.ff_count, ws.ff_idx);
    NB_CUDA(cudaGetLastError());
    ff_kernel<1><<<(unsigned)grid, 128, 0, s>>>(d, gt, q, none, ws.ff_count, ws.ff_idx, bits, st, offsets, n_objects,
                                                P, taus, nullptr, nullptr);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_launch_calibrate(const MlpDesc &d, const GammaTab &gt, const float *q, const uint32_t *labels,
                              int64_t row0, int64_t row1, CalibWs ws, cudaStream_t s) {
    const int64_t n = row1 - row0;
    NB_CUDA(cudaMemsetAsync(ws.umin_bits, 0xff, sizeof(unsigned), s));
    NB_CUDA(cudaMemsetAsync(ws.zmin_bits, 0xff, sizeof(unsigned long long), s));
    NB_CUDA(cudaMemsetAsync(ws.npos, 0, sizeof(unsigned), s));
    int64_t grid = num_sms() * 8;
    const int64_t need = (n + 255) / 256;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    compact_positive_kernel<<<(unsigned)grid, 256, 0, s>>>(labels, (long long)row0, (long long)row1, ws.npos,
                                                             ws.pos_idx);
    NB_CUDA(cudaGetLastError());
    TauF none{};
    nb_status r = tile_dispatch<1>(d, gt, q, none, ws.npos, ws.pos_idx, n, nullptr, nullptr, nullptr, nullptr, ws.lo,
                                   ws.umin_bits, s);
    if (r != NB_OK) return r;
    grid = num_sms() * 8;
    if (grid > (n + 7) / 8) grid = (n + 7) / 8;
    if (grid < 1) grid = 1;
    calib_f64_kernel<<<(unsigned)grid, 256, 0, s>>>(d, q, ws.npos, ws.pos_idx, ws.lo, ws.umin_bits, ws.zmin_bits);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}
