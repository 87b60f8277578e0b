// FP32 forward of bounding networks a thread at a time (Sec. 3.4 "Architecture": MLP with
// ReLU or sine hidden layers; the paper's own networks are 25 to 75 neurons wide).
//
// The weights, transposed to [k][n] and zero-padded to a multiple of four outputs, sit in
// shared memory and are read as broadcast float4s: a group of four output neurons is four
// independent FMA chains over the layer's inputs, which the thread holds in registers.
// Broadcast loads from shared memory, not the FMA pipe, bound this form, so every loaded
// weight is used as often as registers allow:
//   - one hidden layer (fwd_one_hidden_kernel, early_settle_kernel): a thread carries
//     four queries, so each loaded group of four weights feeds sixteen FMAs;
//   - more layers (fwd_narrow_kernel): two queries per thread while the stored layers are
//     at most 64 wide, else one; the first hidden layer is computed straight into
//     registers, a later stored layer writes its outputs to the thread's own columns of a
//     shared-memory buffer ([n / 4][R thread columns] float4s, free of bank conflicts),
//     read back into registers by the next layer.
// The last hidden layer is never stored: each group of four neurons is folded into the
// head's sum as soon as it is computed.
//
//   fwd_narrow_kernel, fwd_one_hidden_kernel
//                        decisions, margin flags and optional logits, with the contract
//                        of the tile kernel (the certified re-check follows unchanged)
//   early_settle_kernel  first stage of the neural early-out (Sec. 3.3) for an early
//                        network with one hidden layer: rows whose logit is certainly
//                        below the early threshold (the FP32 value plus a rigorous bound
//                        of its rounding error) are settled inside; the others are
//                        gathered for the late network, each 32-row word recording where
//                        its gathered rows start
//   early_merge_kernel   the late network's bits of the gathered rows into the words
#include <math.h>

#include <string>

#include "common.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NT = 128;  // threads per block
constexpr int MAXIN = 8;
constexpr int R1 = 4;    // queries per thread in the one-hidden-layer kernels

// Shared-memory plan of one network (floats, every block 16-byte aligned).
//   layer l < L - 1: Wt [kp[l]][np[l]] at wo[l], then the bias [np[l]]
//   head (l = L - 1): v [np[L - 2]] at wo[L - 1], then c
//   activation buffer: [hp / 4][NT R] float4 at abuf (when L > 3), R queries per thread
// hp: padded width of the stored hidden layers (0 for one hidden layer).
struct NarrowDesc {
    int L, w0, act, hp;
    int np[NB_MAXL];
    int kp[NB_MAXL];
    int wo[NB_MAXL];
    int abuf;
    int floats;
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

__device__ __forceinline__ void fma4(float4 &acc, const float4 w, const float a) {
    acc.x = fmaf(w.x, a, acc.x);
    acc.y = fmaf(w.y, a, acc.y);
    acc.z = fmaf(w.z, a, acc.z);
    acc.w = fmaf(w.w, a, acc.w);
}

__device__ __forceinline__ float4 act4(float4 v, int act) {
    if (act == NB_ACT_SINE) return make_float4(sinf(v.x), sinf(v.y), sinf(v.z), sinf(v.w));
    return make_float4(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f), fmaxf(v.z, 0.f), fmaxf(v.w, 0.f));
}

// Every block copies the network into its shared memory from the transposed copy of the
// weights (W_l^T [K][N], then b_l, refreshed with every change of the master weights), so
// consecutive threads read consecutive words; rows and columns beyond the layer's widths
// are zero.  Padded neurons have zero weights and bias, so they output act(0) = 0 and add
// exact zeros downstream.
__device__ void load_image(const MlpDesc &d, const NarrowDesc &nd, float *sm) {
    for (int l = 0; l < d.L; l++) {
        const int K = d.w[l], N = d.w[l + 1];
        const float *Wt = d.pT + d.off[l], *b = Wt + (size_t)N * K;
        if (l == d.L - 1) {  // head: v, c
            const int np = nd.np[l - 1];
            for (int e = threadIdx.x; e <= np; e += NT)
                sm[nd.wo[l] + e] = e < K ? __ldg(Wt + e) : e == np ? __ldg(b) : 0.f;
            continue;
        }
        const int kp = nd.kp[l], np = nd.np[l];
#pragma unroll 4
        for (int e = threadIdx.x; e < kp * np; e += NT) {
            const int k = e / np, j = e - k * np;
            sm[nd.wo[l] + e] = (k < K && j < N) ? __ldg(Wt + (size_t)k * N + j) : 0.f;
        }
        for (int e = threadIdx.x; e < np; e += NT) sm[nd.wo[l] + kp * np + e] = e < N ? __ldg(b + e) : 0.f;
    }
}

// The last hidden layer from the stored inputs in[r][0..HP) of R queries, folded into the
// head: z[r] = c + sum_j v_j h_j, kept as four partial sums (neurons j = 4i + e in sum e,
// so the dependent chains are a quarter as long) that are added pairwise at the end.
template <int HP, int R>
__device__ __forceinline__ void last_layer(const NarrowDesc &nd, const float *sm, const float (&in)[R][HP], int act,
                                           float (&z)[R]) {
    const int l = nd.L - 2, np = nd.np[l];
    const float *Wt = sm + nd.wo[l], *b = Wt + HP * np, *v = sm + nd.wo[l + 1];
    float4 zz[R];
#pragma unroll
    for (int r = 0; r < R; r++) zz[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j0 = 0; j0 < np; j0 += 4) {
        const float4 bb = ld4(b + j0);
        float4 acc[R];
#pragma unroll
        for (int r = 0; r < R; r++) acc[r] = bb;
#pragma unroll
        for (int k = 0; k < HP; k++) {
            const float4 w = ld4(Wt + k * np + j0);
#pragma unroll
            for (int r = 0; r < R; r++) fma4(acc[r], w, in[r][k]);
        }
        const float4 vv = ld4(v + j0);
#pragma unroll
        for (int r = 0; r < R; r++) {
            const float4 h = act4(acc[r], act);
            zz[r].x = fmaf(vv.x, h.x, zz[r].x);
            zz[r].y = fmaf(vv.y, h.y, zz[r].y);
            zz[r].z = fmaf(vv.z, h.z, zz[r].z);
            zz[r].w = fmaf(vv.w, h.w, zz[r].w);
        }
    }
#pragma unroll
    for (int r = 0; r < R; r++) z[r] = v[np] + ((zz[r].x + zz[r].y) + (zz[r].z + zz[r].w));
}

// One hidden layer from R queries x[r][0..W0) straight into the head (the early exit of
// the paper has this shape): z[r] = c + sum_j v_j act(b_j + sum_k W_jk x[r][k]), the head
// sum as four partial sums added pairwise.  With SUMABS, sa[r] = sum_j |v_j| h_j in the
// same order (the rigorous bound of the early-out).
template <int W0, int R, bool SUMABS>
__device__ __forceinline__ void one_hidden(const NarrowDesc &nd, const float *sm, const float (&x)[R][MAXIN],
                                           int act, float (&z)[R], float (&sa)[R]) {
    const int np = nd.np[0];
    const float *Wt = sm + nd.wo[0], *b = Wt + W0 * np, *v = sm + nd.wo[1];
    float4 zz[R], za[R];
#pragma unroll
    for (int r = 0; r < R; r++) zz[r] = za[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j0 = 0; j0 < np; j0 += 4) {
        const float4 bb = ld4(b + j0), vv = ld4(v + j0);
        float4 w[W0];
#pragma unroll
        for (int k = 0; k < W0; k++) w[k] = ld4(Wt + k * np + j0);
#pragma unroll
        for (int r = 0; r < R; r++) {
            float4 acc = bb;
#pragma unroll
            for (int k = 0; k < W0; k++) fma4(acc, w[k], x[r][k]);
            const float4 h = act4(acc, act);
            zz[r].x = fmaf(vv.x, h.x, zz[r].x);
            zz[r].y = fmaf(vv.y, h.y, zz[r].y);
            zz[r].z = fmaf(vv.z, h.z, zz[r].z);
            zz[r].w = fmaf(vv.w, h.w, zz[r].w);
            if (SUMABS) {
                za[r].x = fmaf(fabsf(vv.x), h.x, za[r].x);
                za[r].y = fmaf(fabsf(vv.y), h.y, za[r].y);
                za[r].z = fmaf(fabsf(vv.z), h.z, za[r].z);
                za[r].w = fmaf(fabsf(vv.w), h.w, za[r].w);
            }
        }
    }
    const float c = v[np];
#pragma unroll
    for (int r = 0; r < R; r++) {
        z[r] = c + ((zz[r].x + zz[r].y) + (zz[r].z + zz[r].w));
        if (SUMABS) sa[r] = (za[r].x + za[r].y) + (za[r].z + za[r].w);
    }
}

// The logits of R queries x[r][0..w0) through a network with two or more hidden layers
// (thread t's R columns of the buffer).  The first hidden layer goes straight into
// registers; a stored layer after it writes its outputs to the buffer, from which the next
// layer reloads its registers.  Every loaded weight serves R queries.
template <int HP, int R>
__device__ __forceinline__ void narrow_forward(const NarrowDesc &nd, const float *sm, float4 *abuf,
                                               const float (&x)[R][MAXIN], int t, float (&z)[R]) {
    float a[R][HP];
    {  // layer 0: the queries -> registers
        const float *Wt = sm + nd.wo[0], *b = Wt + nd.kp[0] * HP;
#pragma unroll
        for (int j0 = 0; j0 < HP; j0 += 4) {
            const float4 bb = ld4(b + j0);
            float4 acc[R];
#pragma unroll
            for (int r = 0; r < R; r++) acc[r] = bb;
#pragma unroll
            for (int k = 0; k < MAXIN; k++)
                if (k < nd.w0) {
                    const float4 w = ld4(Wt + k * HP + j0);
#pragma unroll
                    for (int r = 0; r < R; r++) fma4(acc[r], w, x[r][k]);
                }
#pragma unroll
            for (int r = 0; r < R; r++) {
                const float4 h = act4(acc[r], nd.act);
                a[r][j0] = h.x;
                a[r][j0 + 1] = h.y;
                a[r][j0 + 2] = h.z;
                a[r][j0 + 3] = h.w;
            }
        }
    }
    for (int l = 1; l <= nd.L - 3; l++) {  // stored layers: registers -> the buffer -> registers
        const float *Wt = sm + nd.wo[l], *b = Wt + HP * HP;
        for (int j0 = 0; j0 < HP; j0 += 4) {
            const float4 bb = ld4(b + j0);
            float4 acc[R];
#pragma unroll
            for (int r = 0; r < R; r++) acc[r] = bb;
#pragma unroll
            for (int k = 0; k < HP; k++) {
                const float4 w = ld4(Wt + k * HP + j0);
#pragma unroll
                for (int r = 0; r < R; r++) fma4(acc[r], w, a[r][k]);
            }
#pragma unroll
            for (int r = 0; r < R; r++) abuf[(j0 >> 2) * (NT * R) + r * NT + t] = act4(acc[r], nd.act);
        }
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int k4 = 0; k4 < HP / 4; k4++) {
                const float4 v = abuf[k4 * (NT * R) + r * NT + t];
                a[r][4 * k4] = v.x;
                a[r][4 * k4 + 1] = v.y;
                a[r][4 * k4 + 2] = v.z;
                a[r][4 * k4 + 3] = v.w;
            }
    }
    last_layer<HP, R>(nd, sm, a, nd.act, z);
}

// Queries per thread of the multi-layer kernel: two while their registers allow (stored
// layers up to 64 wide), else one.
template <int HP>
struct RowsPerThread {
    static constexpr int value = HP <= 64 ? 2 : 1;
};

// Decisions z >= tau for 32 R consecutive rows per warp and iteration (row base + 32 r +
// lane in slot r): bits, optional logits, the margin band appended to flag_idx; a
// non-finite logit or input coordinate is flagged (the re-check decides it inside).  Same
// contract as the tile kernel.
template <int HP>
__global__ void __launch_bounds__(NT, HP >= 64 ? 2 : 3)
    fwd_narrow_kernel(const __grid_constant__ MlpDesc d, const __grid_constant__ NarrowDesc nd,
                      const float *__restrict__ q, long long n, TauF tau, float margin, uint32_t *__restrict__ bits,
                      float *__restrict__ logits, nb_query_stats *st, unsigned *flag_count, unsigned *flag_idx) {
    constexpr int R = RowsPerThread<HP>::value;
    extern __shared__ __align__(16) float sm[];
    load_image(d, nd, sm);
    __syncthreads();
    float4 *abuf = reinterpret_cast<float4 *>(sm + nd.abuf);
    const int t = threadIdx.x, lane = t & 31;
    const int w0 = nd.w0;
    unsigned long long c_in = 0, c_flag = 0, c_nf = 0;
    const long long stride = (long long)gridDim.x * NT * R;
    for (long long base = ((long long)blockIdx.x * NT + (t & ~31)) * R; base < n; base += stride) {
        float x[R][MAXIN];
        bool xfin[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const long long i = base + 32 * r + lane;
            xfin[r] = true;
#pragma unroll
            for (int k = 0; k < MAXIN; k++) {
                x[r][k] = (i < n && k < w0) ? __ldg(q + i * w0 + k) : 0.f;
                xfin[r] = xfin[r] && isfinite(x[r][k]);
            }
        }
        float z[R];
        narrow_forward<HP, R>(nd, sm, abuf, x, t, z);
#pragma unroll
        for (int r = 0; r < R; r++) {
            const long long i = base + 32 * r + lane;
            const bool valid = i < n;
            const float zr = xfin[r] ? z[r] : __int_as_float(0x7fc00000);
            const bool fin = isfinite(zr);
            const bool inside = valid && fin && zr >= tau.up;
            const bool flag = valid && (!fin || fabsf(zr - tau.up) < margin || (zr >= tau.dn && zr < tau.up));
            const unsigned bi = __ballot_sync(FULL, inside);
            const unsigned bf = __ballot_sync(FULL, flag);
            const unsigned bn = __ballot_sync(FULL, valid && !fin);
            if (lane == 0 && base + 32 * r < n) bits[(base >> 5) + r] = bi;
            if (valid && logits) logits[i] = zr;
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
    if (st && lane == 0) {
        if (c_in) atomicAdd(&st->n_inside, c_in);
        if (c_flag) atomicAdd(&st->n_flagged, c_flag);
        if (c_nf) atomicAdd(&st->n_nonfinite, c_nf);
    }
}

// fwd_narrow_kernel's contract for a network with one hidden layer, R1 queries per thread:
// a warp takes 32 R1 consecutive rows, row base + 32 r + lane in slot r.  The input width
// w0 is at most W0; the weight rows past it are zero.
template <int W0>
__global__ void __launch_bounds__(NT, 4)
    fwd_one_hidden_kernel(const __grid_constant__ MlpDesc d, const __grid_constant__ NarrowDesc nd,
                          const float *__restrict__ q, long long n, TauF tau, float margin,
                          uint32_t *__restrict__ bits, float *__restrict__ logits, nb_query_stats *st,
                          unsigned *flag_count, unsigned *flag_idx) {
    extern __shared__ __align__(16) float sm[];
    load_image(d, nd, sm);
    __syncthreads();
    const int t = threadIdx.x, lane = t & 31;
    const int w0 = nd.w0;
    unsigned long long c_in = 0, c_flag = 0, c_nf = 0;
    const long long stride = (long long)gridDim.x * NT * R1;
    for (long long base = ((long long)blockIdx.x * NT + (t & ~31)) * R1; base < n; base += stride) {
        float x[R1][MAXIN];
        bool xfin[R1];
#pragma unroll
        for (int r = 0; r < R1; r++) {
            const long long i = base + 32 * r + lane;
            xfin[r] = true;
#pragma unroll
            for (int k = 0; k < W0; k++) {
                x[r][k] = (i < n && k < w0) ? __ldg(q + i * w0 + k) : 0.f;
                xfin[r] = xfin[r] && isfinite(x[r][k]);
            }
        }
        float z[R1], sa[R1];
        one_hidden<W0, R1, false>(nd, sm, x, nd.act, z, sa);
#pragma unroll
        for (int r = 0; r < R1; r++) {
            const long long i = base + 32 * r + lane;
            const bool valid = i < n;
            const float zr = xfin[r] ? z[r] : __int_as_float(0x7fc00000);
            const bool fin = isfinite(zr);
            const bool inside = valid && fin && zr >= tau.up;
            const bool flag = valid && (!fin || fabsf(zr - tau.up) < margin || (zr >= tau.dn && zr < tau.up));
            const unsigned bi = __ballot_sync(FULL, inside);
            const unsigned bf = __ballot_sync(FULL, flag);
            const unsigned bn = __ballot_sync(FULL, valid && !fin);
            if (lane == 0 && base + 32 * r < n) bits[(base >> 5) + r] = bi;
            if (valid && logits) logits[i] = zr;
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
    if (st && lane == 0) {
        if (c_in) atomicAdd(&st->n_inside, c_in);
        if (c_flag) atomicAdd(&st->n_flagged, c_flag);
        if (c_nf) atomicAdd(&st->n_nonfinite, c_nf);
    }
}

// Neural early-out, first stage, for an early network x -> ReLU(W x + b) -> v . h + c.
// Rounding errors of the FP32 evaluation (u = 2^-24, gamma_k = k u / (1 - k u)):
//   s_j = b_j + sum_k W_jk x_k by W0 FMAs: |s_j - s*_j| <= gamma_W0 (|b_j| + sum_k |W_jk| |x_k|)
//         <= gamma_W0 (|b_j| + A_j xmax), A_j = sum_k |W_jk|, xmax = max_k |x_k|;
//   ReLU is 1-Lipschitz, so |h_j - h*_j| is bounded by the same;
//   z = c + sum_j v_j h_j as four FMA chains of m = H_p / 4 terms (H_p: H rounded up to a
//         multiple of 4) added pairwise, then c: |z - (c + sum_j v_j h_j)| <=
//         gamma_{m+3} (|c| + sum_j |v_j| h_j), and the h errors add sum_j |v_j| |h_j - h*_j|
//         <= gamma_W0 (C_b + xmax C_a), C_b = sum_j |v_j| |b_j|, C_a = sum_j |v_j| A_j.
// g_out = gamma_{2m + 8} also covers the rounding of the computed sum of |v_j| h_j (same
// order, relative error gamma_{m+3}); C_a and C_b are summed in FP64 and rounded up, every
// bound operation rounds up.  A row is settled (inside) when z + bound + margin < tau_dn
// <= tau: its exact logit is below the early network's threshold, and the early network
// bounds the complement 1 - g.  A word's late rows are gathered, in lane order, from
// pos_w[word] on; a block claims its range of the gathered list with one atomic per
// iteration (a counter shared by every block would otherwise serialise the warps).
template <int W0>
__global__ void __launch_bounds__(NT, 4)
    early_settle_kernel(const __grid_constant__ MlpDesc d, const __grid_constant__ NarrowDesc nd,
                        const float *__restrict__ q, long long n, TauF tau, float margin, float g_in, float g_out,
                        uint32_t *__restrict__ out_bits, unsigned *count, unsigned *__restrict__ pos_w,
                        float *__restrict__ qc) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double red[2][NT / 32];
    __shared__ float cab[2];
    __shared__ unsigned wcnt[NT / 32], wbase;
    load_image(d, nd, sm);
    __syncthreads();
    const int t = threadIdx.x, lane = t & 31;
    {
        const int np = nd.np[0];
        const float *Wt = sm + nd.wo[0], *b = Wt + nd.kp[0] * np, *v = sm + nd.wo[1];
        double ca = 0.0, cb = 0.0;
        for (int j = t; j < np; j += NT) {
            double a = 0.0;
            for (int k = 0; k < W0; k++) a += fabs((double)Wt[k * np + j]);
            ca += fabs((double)v[j]) * a;
            cb += fabs((double)v[j]) * fabs((double)b[j]);
        }
        for (int o = 16; o; o >>= 1) {
            ca += __shfl_xor_sync(FULL, ca, o);
            cb += __shfl_xor_sync(FULL, cb, o);
        }
        if (lane == 0) {
            red[0][t >> 5] = ca;
            red[1][t >> 5] = cb;
        }
        __syncthreads();
        if (t == 0) {
            double sa = 0.0, sb = 0.0;
            for (int w = 0; w < NT / 32; w++) {
                sa += red[0][w];
                sb += red[1][w];
            }
            // FP64 sums of at most 2^12 non-negative products are within a relative 2^-40 of
            // the exact ones; the factor covers that before rounding up
            cab[0] = __double2float_ru(sa * (1.0 + 0x1p-39));
            cab[1] = __double2float_ru(sb * (1.0 + 0x1p-39));
        }
        __syncthreads();
    }
    const float C_a = cab[0], C_b = cab[1];
    const float c_abs = fabsf(sm[nd.wo[1] + nd.np[0]]);
    const long long stride = (long long)gridDim.x * NT * R1;
    const int warp = t >> 5;
    // a block takes NT R1 rows per iteration (every warp iterates alike, so the block can
    // synchronise) and claims one range of the gathered list for all its late rows
    for (long long bb = (long long)blockIdx.x * NT * R1; bb < n; bb += stride) {
        const long long base = bb + (long long)warp * 32 * R1;
        float x[R1][MAXIN];
#pragma unroll
        for (int r = 0; r < R1; r++) {
            const long long i = base + 32 * r + lane;
#pragma unroll
            for (int k = 0; k < W0; k++) x[r][k] = i < n ? __ldg(q + i * W0 + k) : 0.f;
        }
        float z[R1], sa[R1];
        one_hidden<W0, R1, true>(nd, sm, x, NB_ACT_RELU, z, sa);
        unsigned bs[R1], bl[R1];
#pragma unroll
        for (int r = 0; r < R1; r++) {
            const long long i = base + 32 * r + lane;
            const bool valid = i < n;
            bool xfin = true;
            float xmax = 0.f;
#pragma unroll
            for (int k = 0; k < W0; k++) {
                xfin = xfin && isfinite(x[r][k]);
                xmax = fmaxf(xmax, fabsf(x[r][k]));
            }
            const float bound = __fadd_ru(__fmul_ru(g_out, __fadd_ru(sa[r], c_abs)),
                                          __fmul_ru(g_in, __fmaf_ru(xmax, C_a, C_b)));
            const float top = __fadd_ru(__fadd_ru(z[r], bound), margin);
            const bool settled = valid && xfin && isfinite(z[r]) && isfinite(top) && top < tau.dn;
            bs[r] = __ballot_sync(FULL, settled);
            bl[r] = __ballot_sync(FULL, valid && !settled);
        }
        unsigned mine = 0;  // this warp's late rows
#pragma unroll
        for (int r = 0; r < R1; r++) mine += __popc(bl[r]);
        if (lane == 0) wcnt[warp] = mine;
        __syncthreads();
        if (t == 0) {
            unsigned tot = 0;
            for (int w = 0; w < NT / 32; w++) tot += wcnt[w];
            wbase = tot ? atomicAdd(count, tot) : 0u;
        }
        __syncthreads();
        unsigned pos = wbase;
        for (int w = 0; w < warp; w++) pos += wcnt[w];
#pragma unroll
        for (int r = 0; r < R1; r++) {
            if ((bl[r] >> lane) & 1u) {
                const unsigned p = pos + __popc(bl[r] & ((1u << lane) - 1u));
#pragma unroll
                for (int k = 0; k < W0; k++) qc[(size_t)p * W0 + k] = x[r][k];
            }
            if (lane == 0 && base + 32 * r < n) {
                out_bits[(base >> 5) + r] = bs[r];
                pos_w[(base >> 5) + r] = pos;
            }
            pos += __popc(bl[r]);
        }
        __syncthreads();  // wcnt and wbase are reused by the next iteration
    }
}

// Word w of the answer: settled rows are already 1; its other valid rows are gathered
// rows pos_w[w], pos_w[w] + 1, ... in lane order, whose late bits (bits_c) are merged in.
__global__ void early_merge_kernel(const uint32_t *__restrict__ bits_c, const unsigned *__restrict__ pos_w,
                                   long long n, uint32_t *__restrict__ out_bits) {
    const int lane = threadIdx.x & 31;
    const long long nw = (n + 31) / 32;
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw;
         w += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long rows = n - w * 32;
        const unsigned valid = rows >= 32 ? FULL : (1u << rows) - 1u;
        const unsigned settled = out_bits[w];
        const unsigned late = valid & ~settled;
        if (!late) continue;
        bool bit = false;
        if ((late >> lane) & 1u) {
            const unsigned j = pos_w[w] + __popc(late & ((1u << lane) - 1u));
            bit = (bits_c[j >> 5] >> (j & 31)) & 1u;
        }
        const unsigned b = __ballot_sync(FULL, bit);
        if (lane == 0) out_bits[w] = settled | b;
    }
}

int num_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

constexpr int MAX_SMEM_FLOATS = 200 * 1024 / 4;

// The shared-memory plan of d, or false when the thread-per-query form does not apply:
// input width above 8, a stored hidden layer wider than 128, or a plan above 200 KB.
bool plan(const MlpDesc &d, NarrowDesc &nd) {
    if (d.L < 2 || d.L > NB_MAXL || d.w[0] < 1 || d.w[0] > MAXIN) return false;
    nd = NarrowDesc{};
    nd.L = d.L;
    nd.w0 = d.w[0];
    nd.act = d.act;
    int widest = 0;  // outputs of the stored layers 0 .. L - 3
    for (int l = 0; l <= d.L - 3; l++) widest = d.w[l + 1] > widest ? d.w[l + 1] : widest;
    nd.hp = d.L == 2 ? 0
            : widest <= 32 ? 32
            : widest <= 64 ? 64
            : widest <= 80 ? 80  // the paper's 75-wide networks
            : widest <= 128 ? 128
                            : -1;
    if (nd.hp < 0) return false;
    auto r4 = [](int v) { return (v + 3) / 4 * 4; };
    // a one-hidden-layer network runs with its input width padded to 2, 3, 4, 6 or 8
    const int w0k = d.w[0] <= 4 ? (d.w[0] < 2 ? 2 : d.w[0]) : d.w[0] <= 6 ? 6 : 8;
    int off = 0;
    for (int l = 0; l < d.L - 1; l++) {
        nd.kp[l] = l == 0 ? (d.L == 2 ? w0k : d.w[0]) : nd.hp;
        nd.np[l] = l == d.L - 2 ? r4(d.w[l + 1]) : nd.hp;
        nd.wo[l] = off;
        off += r4(nd.kp[l] * nd.np[l] + nd.np[l]);
    }
    nd.kp[d.L - 1] = nd.np[d.L - 2];
    nd.np[d.L - 1] = 1;
    nd.wo[d.L - 1] = off;
    off += r4(nd.np[d.L - 2] + 1);
    nd.abuf = off;
    if (d.L > 3) off += nd.hp * NT * (nd.hp <= 64 ? 2 : 1);  // [hp / 4][NT * R] float4
    nd.floats = off;
    return off <= MAX_SMEM_FLOATS;
}

// Launch of one of the kernels above: a persistent grid of the blocks that fit on the SMs,
// at most one block per NT * rows_per_thread rows.
template <typename K, typename... A>
nb_status launch(K kernel, const char *name, const NarrowDesc &nd, int64_t n, int rows_per_thread, cudaStream_t s,
                 A... args) {
    const size_t smem = (size_t)nd.floats * sizeof(float);
    NB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 1;
    NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem));
    if (per_sm < 1) return nb_fail(NB_EUNSUPPORTED, std::string(name) + ": kernel does not fit on an SM");
    const int64_t rows_per_block = (int64_t)NT * rows_per_thread;
    const int64_t blocks = (n + rows_per_block - 1) / rows_per_block;
    int64_t grid = (int64_t)num_sms() * per_sm;
    if (grid > blocks) grid = blocks;
    kernel<<<(unsigned)grid, NT, smem, s>>>(args...);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// gamma_k rounded up to a float
float gamma_up(int k) {
    const double u = 0x1p-24;
    const double g = k * u / (1.0 - k * u);
    float f = (float)g;
    if ((double)f < g) f = nextafterf(f, INFINITY);
    return nextafterf(f, INFINITY);
}

template <int HP>
nb_status fwd_launch(const MlpDesc &d, const NarrowDesc &nd, const float *q, int64_t n, TauF tau, float margin,
                     uint32_t *bits, float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s) {
    return launch(fwd_narrow_kernel<HP>, "fwd_narrow", nd, n, RowsPerThread<HP>::value, s, d, nd, q, (long long)n,
                  tau, margin, bits,
                  logits, st, ws.flag_count, ws.flag_idx);
}

template <int W0>
nb_status one_hidden_launch(const MlpDesc &d, const NarrowDesc &nd, const float *q, int64_t n, TauF tau,
                            float margin, uint32_t *bits, float *logits, nb_query_stats *st, QueryWs ws,
                            cudaStream_t s) {
    return launch(fwd_one_hidden_kernel<W0>, "fwd_one_hidden", nd, n, R1, s, d, nd, q, (long long)n, tau, margin,
                  bits, logits, st, ws.flag_count, ws.flag_idx);
}

template <int W0>
nb_status early_launch(const MlpDesc &d, const NarrowDesc &nd, const float *q, int64_t n, TauF tau, float margin,
                       uint32_t *out_bits, unsigned *count, unsigned *pos_w, float *qc, cudaStream_t s) {
    const float g_in = gamma_up(W0), g_out = gamma_up(2 * (nd.np[0] / 4) + 8);
    return launch(early_settle_kernel<W0>, "early_settle", nd, n, R1, s, d, nd, q, (long long)n, tau, margin, g_in,
                  g_out, out_bits, count, pos_w, qc);
}

}  // namespace

bool nb_narrow_eligible(const MlpDesc &d) {
    NarrowDesc nd;
    return plan(d, nd);
}

nb_status nb_launch_fwd_narrow(const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin, uint32_t *bits,
                               float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s) {
    NarrowDesc nd;
    if (!plan(d, nd)) return nb_fail(NB_EUNSUPPORTED, "fwd_narrow: network outside the thread-per-query form");
    if (nd.hp == 0) switch (nd.kp[0]) {
        case 2: return one_hidden_launch<2>(d, nd, q, n, tau, margin, bits, logits, st, ws, s);
        case 3: return one_hidden_launch<3>(d, nd, q, n, tau, margin, bits, logits, st, ws, s);
        case 4: return one_hidden_launch<4>(d, nd, q, n, tau, margin, bits, logits, st, ws, s);
        case 6: return one_hidden_launch<6>(d, nd, q, n, tau, margin, bits, logits, st, ws, s);
        default: return one_hidden_launch<8>(d, nd, q, n, tau, margin, bits, logits, st, ws, s);
        }
    switch (nd.hp) {
    case 32: return fwd_launch<32>(d, nd, q, n, tau, margin, bits, logits, st, ws, s);
    case 64: return fwd_launch<64>(d, nd, q, n, tau, margin, bits, logits, st, ws, s);
    case 80: return fwd_launch<80>(d, nd, q, n, tau, margin, bits, logits, st, ws, s);
    default: return fwd_launch<128>(d, nd, q, n, tau, margin, bits, logits, st, ws, s);
    }
}

bool nb_early_settle_eligible(const MlpDesc &d) {
    NarrowDesc nd;
    const int w0 = d.w[0];
    return d.L == 2 && d.act == NB_ACT_RELU && (w0 == 2 || w0 == 3 || w0 == 4 || w0 == 6 || w0 == 8) && plan(d, nd);
}

nb_status nb_launch_early_settle(const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin,
                                 uint32_t *out_bits, unsigned *count, unsigned *pos_w, float *qc, cudaStream_t s) {
    NarrowDesc nd;
    if (!nb_early_settle_eligible(d) || !plan(d, nd))
        return nb_fail(NB_EUNSUPPORTED, "early_settle: the early network is not a one-hidden-layer ReLU network");
    switch (d.w[0]) {
    case 2: return early_launch<2>(d, nd, q, n, tau, margin, out_bits, count, pos_w, qc, s);
    case 3: return early_launch<3>(d, nd, q, n, tau, margin, out_bits, count, pos_w, qc, s);
    case 4: return early_launch<4>(d, nd, q, n, tau, margin, out_bits, count, pos_w, qc, s);
    case 6: return early_launch<6>(d, nd, q, n, tau, margin, out_bits, count, pos_w, qc, s);
    default: return early_launch<8>(d, nd, q, n, tau, margin, out_bits, count, pos_w, qc, s);
    }
}

nb_status nb_launch_early_merge(const uint32_t *bits_c, const unsigned *pos_w, int64_t n, uint32_t *out_bits,
                                cudaStream_t s) {
    const int64_t words = (n + 31) / 32;
    int64_t grid = (words * 32 + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    early_merge_kernel<<<(unsigned)grid, 256, 0, s>>>(bits_c, pos_w, (long long)n, out_bits);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}
