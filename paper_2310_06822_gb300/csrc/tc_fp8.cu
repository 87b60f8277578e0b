// FP8 (E4M3) tensor-core forward of the bounding network h (Sec. 3.4 "Architecture").
//
// The hidden-to-hidden layers run on the tensor cores with E4M3 operands and FP32
// accumulation (tcgen05.mma kind::f8f6f4), each operand split into two E4M3 terms,
// x = x_hi + x_lo with x_lo = E4M3(x - x_hi), and three products per k-step,
// a_hi w_hi + a_hi w_lo + a_lo w_hi (the dropped a_lo w_lo is ~2^-8 relative): about 8
// significant bits per operand instead of 4.  On trained networks one E4M3 term was off
// by up to ~20 in the logit (3 mantissa bits against logits in the hundreds, with
// cancellation); two terms bring that below 1 for 1.5x the BF16 tensor work of one
// product (E4M3 runs at twice the BF16 rate).  Scales are powers of two, so applying and
// removing them is exact.  Every query row has its own activation scale r (max_k a_k r in
// [128, 256), E4M3's largest finite value being 448).  Every weight row n of layer l has its
// own s_n, and the layer's outputs are kept scaled by it: the epilogue computes
// a'_n = relu(D_n / r + b_n s_n) = s_n a_n, the next layer's columns carry 1 / s_k
// (W'_nk = W_nk s_n / s_k, s_n chosen so that max_k |W_nk / s_k| s_n is in [128, 256)) and
// the head's weights carry 1 / s_n, so one folded bias per neuron is all the epilogue
// reads.  The first layer (fan-in = the query encoding) runs in
// split FP16 (three products, as in the split-FP16 kernel): quantising the query itself
// to three mantissa bits would move it by several per cent.  The output head runs in FP32
// on the CUDA cores.
//
// Placement (one persistent CTA per SM): shared memory holds the first layer's split image
// (loaded once) and two stages of the streamed hidden-layer weights: the two-term E4M3
// images (2 H^2 bytes per layer, 384 KB for three 256-wide layers -- more than shared
// memory) pass through in chunks of one 128-column K-block of both terms, 2 x H x 128
// bytes, brought in by the bulk-copy engine one chunk ahead of the products that read it.
// Tensor memory holds the FP32 accumulator (H columns) and the next layer's activations
// (H/4 columns per E4M3 term, or the split-FP16 query for the first layer), read by the
// MMA as its A operand.  Warps 0-7 are the epilogue: warps w and w + 4 share the TMEM lanes
// of quarter w mod 4 (one query row per lane) and take one half of the columns each,
// exchanging their partial row maxima and head sums through shared memory; warp 8
// allocates TMEM and issues the MMAs; warp 9 streams the weight chunks.  One tile is in
// flight: its layers alternate between the tensor pipe and the epilogue.  All waits are
// bounded; on expiry the kernel records NB_ETIMEOUT, waits (bounded) for its copies in
// flight, drains the tensor pipe and frees TMEM before returning.
#include <cuda_fp16.h>

#include "tc.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace nbtc;

constexpr int TILE_M = 128;
constexpr int NEPI = 8;
constexpr int THREADS = (NEPI + 2) * 32;  // epilogue warps, the MMA warp, the weight-stream warp
constexpr unsigned SPIN_LIMIT = 1u << 22;
constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t CTL_BYTES = 2048;  // control block and the row-exchange buffer

struct Fp8Desc {
    int in, H, NHH;        // input width, hidden width, hidden-to-hidden layers
    const uint8_t *img;    // layer 0 split image, then NHH two-term E4M3 images in chunk order
    uint32_t img_bytes;
    const float *inv_sw;   // [NHH][H] 1 / s_n of every E4M3 weight row
    const float *bs;       // [NHH][H] b_n s_n: the folded biases
    const float *hw;       // [H + 1] head weights w_n / s_n of the last E4M3 layer, then its bias
    const float *p;        // FP32 master parameters
    int off[NB_MAXL];
};

// Image: layer 0 as H rows x 128 B (split FP16, K = 64); then, for each E4M3 layer, H / 128
// chunks, chunk kb holding K-block kb (columns 128 kb ..) of the hi term then of the lo term,
// H rows x 128 B each, 128-byte swizzled -- so the chunks of all layers follow each other
// in the order the products read them.  fp8_chunk is the bytes of one chunk.
__host__ __device__ inline uint32_t fp8_chunk(int H) { return (uint32_t)(2 * H * 128); }

struct Ctl {
    uint64_t wbar, aready, accfull, drain, full[2], empty[2];
    uint64_t pair[4];  // row-exchange handshake of the two warps of each lane quarter
    uint32_t tmem;
    int abort;
};

__device__ bool wait_bounded(uint32_t bar, uint32_t parity, Ctl *ctl, int *err) {
    for (unsigned i = 0; i < SPIN_LIMIT; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*(volatile int *)&ctl->abort) return false;
    }
    *(volatile int *)&ctl->abort = 1;
    atomicExch(err, NB_ETIMEOUT);
    return false;
}
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, Ctl *ctl, int *err) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = wait_bounded(bar, parity, ctl, err) ? 1 : 0;
    return __shfl_sync(FULL, ok, 0) != 0;
}

// power-of-two r with m r in [128, 256) (m > 0 finite), and 1 / r; 1 otherwise
__device__ __forceinline__ float pow2_scale(float m, float &inv) {
    if (!(m > 0.f) || !(m < INFINITY)) {
        inv = 1.f;
        return 1.f;
    }
    int e;
    frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
    e = max(e, -110);
    inv = ldexpf(1.f, e - 8);
    return ldexpf(1.f, 8 - e);
}

// The two warps sharing a TMEM lane quarter exchange per-row values through xbuf: every
// lane writes its value, arrives on the quarter's barrier (64 arrivals complete a phase)
// and waits, itself and bounded, for the phase before reading the partner's value.
__device__ __forceinline__ bool pair_exchange(float *xbuf, int warp, int wq, float v, float &other, Ctl *ctl,
                                              uint32_t &parity, int *err) {
    const int lane = threadIdx.x & 31;
    xbuf[warp * 32 + lane] = v;
    const uint32_t bar = smem_u32(&ctl->pair[wq]);
    mbar_arrive(bar);
    const bool ok = wait_bounded(bar, parity, ctl, err);
    parity ^= 1;
    other = xbuf[(warp ^ 4) * 32 + lane];
    return __all_sync(FULL, ok);
}

template <int H>
__global__ void __launch_bounds__(THREADS, 1)
    fwd_fp8_kernel(Fp8Desc d, const float *__restrict__ q, long long n, TauF tau, float margin,
                   uint32_t *__restrict__ bits, float *__restrict__ logits, nb_query_stats *st,
                   unsigned *flag_count, unsigned *flag_idx, int *err) {
    constexpr uint32_t TCOLS = H == 256 ? 512 : 256;   // D: H columns; A: from column H
    constexpr int HALF = H / 2;                        // columns per epilogue warp
    extern __shared__ uint8_t smem_raw[];
    Ctl *ctl = reinterpret_cast<Ctl *>(smem_raw);
    float *xbuf = reinterpret_cast<float *>(smem_raw + 128);  // [8 warps][32 lanes]
    uint8_t *Wimg = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023) + CTL_BYTES;
    const uint32_t L0_BYTES = (uint32_t)H * 128, CHUNK = fp8_chunk(H), TERM = (uint32_t)H * 128;
    const uint32_t stage0 = smem_u32(Wimg) + L0_BYTES;  // two stages of CHUNK bytes

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long ntiles = (n + TILE_M - 1) / TILE_M;
    const uint32_t bar_w = smem_u32(&ctl->wbar), bar_ar = smem_u32(&ctl->aready);
    const uint32_t bar_af = smem_u32(&ctl->accfull), bar_drain = smem_u32(&ctl->drain);

    if (threadIdx.x == 0) {
        mbar_init(bar_w, 1);
        mbar_init(bar_ar, NEPI);
        mbar_init(bar_af, 1);
        mbar_init(bar_drain, 1);
        for (int i = 0; i < 2; i++) {
            mbar_init(smem_u32(&ctl->full[i]), 1);
            mbar_init(smem_u32(&ctl->empty[i]), 1);
        }
        for (int i = 0; i < 4; i++) mbar_init(smem_u32(&ctl->pair[i]), 64);
        ctl->abort = 0;
        fence_mbar_init();
    }
    if (warp == NEPI) {
        tmem_alloc(smem_u32(&ctl->tmem), TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem;
    const int NL = d.NHH + 1;  // tensor-core layers: the first layer and the E4M3 layers

    const int CPT = d.NHH * (H / 128);  // weight chunks per tile
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    if (warp == NEPI + 1) {
        // ------------------------------------------------ weight stream: chunk c -> stage c & 1
        if (lane == 0) {
            const long long total = my_tiles * CPT;
            bool ok = true;
            long long issued = 0;
            for (long long c = 0; c < total && ok; c++) {
                const int sidx = (int)(c & 1);
                if (c >= 2) ok = wait_bounded(smem_u32(&ctl->empty[sidx]), (uint32_t)(((c >> 1) - 1) & 1), ctl, err);
                if (!ok) break;
                const uint32_t bar = smem_u32(&ctl->full[sidx]);
                mbar_expect_tx(bar, CHUNK);
                const uint8_t *src = d.img + L0_BYTES + (size_t)(c % CPT) * CHUNK;
                for (uint32_t o = 0; o < CHUNK; o += 16384)
                    bulk_g2s(stage0 + sidx * CHUNK + o, src + o, min(16384u, CHUNK - o), bar);
                issued = c + 1;
            }
            // the copies of the last two chunks (every earlier one has been consumed) have
            // landed before the CTA may exit
            for (long long c = issued - 2; c < issued; c++)
                if (c >= 0) wait_bounded(smem_u32(&ctl->full[c & 1]), (uint32_t)((c >> 1) & 1), ctl, err);
        }
        __syncwarp();
    } else if (warp == NEPI) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            mbar_expect_tx(bar_w, L0_BYTES);
            for (uint32_t o = 0; o < L0_BYTES; o += 16384)
                bulk_g2s(smem_u32(Wimg) + o, d.img + o, min(16384u, L0_BYTES - o), bar_w);
            bool ok = wait_bounded(bar_w, 0, ctl, err);
            uint32_t pa = 0;
            constexpr uint32_t id16 = idesc_f16(TILE_M, H);
            constexpr uint32_t id8 = idesc_e4m3(TILE_M, H);
            const uint32_t wbase = smem_u32(Wimg);
            const uint32_t tD = tmem, tA = tmem + H, tA1 = tmem + H + H / 4;
            long long c = 0;
            for (long long tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                for (int l = 0; l < NL && ok; l++) {
                    ok = wait_bounded(bar_ar, pa, ctl, err);
                    pa ^= 1;
                    if (!ok) break;
                    tc_fence_after();
                    if (l == 0) {  // K = 48: the fourth 16-wide block of A0 and B0 is zero
                        for (int j = 0; j < 3; j++)
                            mma_f16_ts(tD, tA + 8 * j, sdesc_sw128(wbase + 32 * j), id16, j > 0 ? 1u : 0u);
                    } else {
                        for (int kb = 0; kb < H / 128 && ok; kb++, c++) {
                            const int sidx = (int)(c & 1);
                            ok = wait_bounded(smem_u32(&ctl->full[sidx]), (uint32_t)((c >> 1) & 1), ctl, err);
                            if (!ok) break;
                            tc_fence_after();
                            const uint32_t whi = stage0 + sidx * CHUNK, wlo = whi + TERM;
                            for (int j = 0; j < 4; j++) {  // k-steps of 32 within the K-block
                                const uint32_t ks = (uint32_t)(kb * 4 + j), within = (uint32_t)j * 32;
                                mma_f8_ts(tD, tA + 8 * ks, sdesc_sw128(whi + within), id8, (kb | j) ? 1u : 0u);
                                mma_f8_ts(tD, tA + 8 * ks, sdesc_sw128(wlo + within), id8, 1u);
                                mma_f8_ts(tD, tA1 + 8 * ks, sdesc_sw128(whi + within), id8, 1u);
                            }
                            mma_commit(smem_u32(&ctl->empty[sidx]));  // the stage may be refilled
                        }
                    }
                    mma_commit(bar_af);
                }
            }
            mma_commit(bar_drain);
            wait_bounded(bar_drain, 0, ctl, err);
            if (!ok) *(volatile int *)&ctl->abort = 1;
        }
        __syncwarp();
    } else {
        const int wq = warp & 3, half = warp >> 2;
        const int r = wq * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(wq * 32) << 16);
        const uint32_t tD = trow + half * HALF, tA = trow + H, tA1 = trow + H + H / 4;
        const int c0 = half * HALF;  // first column (neuron) of this warp
        uint32_t ph = 0, pp = 0;
        unsigned long long c_in = 0, c_flag = 0, c_nf = 0;
        const int in = d.in;
        float x[16];
        if (half == 0) {
            const long long row0 = (long long)blockIdx.x * TILE_M + r;
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = (row0 < n && k < in) ? __ldg(q + row0 * in + k) : 0.f;
        }
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const long long row = tile * TILE_M + r;
            const bool valid = row < n;
            bool xbad = false;  // a non-finite input coordinate: the logit is made NaN
            if (half == 0) {
#pragma unroll
                for (int k = 0; k < 16; k++) xbad = xbad || !isfinite(x[k]);
                // A0 = [x_hi | x_lo | x_hi | 0], 16 FP16 each, two per 32-bit column
                uint32_t w0[16], w1[16];
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    uint32_t hi, lo;
                    split_f16x2(x[2 * k], x[2 * k + 1], hi, lo);
                    w0[k] = hi;
                    w0[8 + k] = lo;
                    w1[k] = hi;
                    w1[8 + k] = 0u;
                }
                tmem_st16(tA, w0);
                tmem_st16(tA + 16, w1);
                tmem_st_wait();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_ar);
            if (half == 0) {
                const long long nrow = (tile + gridDim.x) * TILE_M + r;
#pragma unroll
                for (int k = 0; k < 16; k++) x[k] = (nrow < n && k < in) ? __ldg(q + nrow * in + k) : 0.f;
            }
            bool ok = true, bad = false;
            float inv_r = 1.f, z = 0.f;
            for (int l = 0; l < NL; l++) {
                ok = warp_wait(bar_af, ph, ctl, err);
                ph ^= 1;
                if (!ok) break;
                tc_fence_after();
                // this layer's output neuron c, kept scaled: relu(D_c inv_r + b_c s_c) = s_c a_c
                // (the first layer: relu(D_c + b_c))
                const float *b = l == 0 ? d.p + d.off[0] + (size_t)H * in : d.bs + (size_t)(l - 1) * H;
                if (l < NL - 1) {
                    float m = 0.f;
#pragma unroll
                    for (int c = 0; c < HALF / 32; c++) {
                        float v[32];
                        tmem_ld32(tD + c * 32, v);
                        tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 32; e++) {
                            const int nn = c0 + c * 32 + e;
                            const float t = fmaf(v[e], inv_r, __ldg(b + nn));
                            bad |= !(fabsf(t) < INFINITY);
                            m = fmaxf(m, t);
                        }
                    }
                    float mo;
                    ok = pair_exchange(xbuf, warp, wq, m, mo, ctl, pp, err);
                    if (!ok) break;
                    m = fmaxf(m, mo);
                    float inv_next;
                    const float rs = pow2_scale(m, inv_next);
                    // 64 activations -> 16 columns of each E4M3 term at column (first neuron) / 4
#pragma unroll
                    for (int cp = 0; cp < HALF / 64; cp++) {
                        uint32_t whi[16], wlo[16];
#pragma unroll
                        for (int hh = 0; hh < 2; hh++) {
                            float v[32];
                            tmem_ld32(tD + cp * 64 + hh * 32, v);
                            tmem_ld_wait();
#pragma unroll
                            for (int e = 0; e < 8; e++) {
                                float a[4];
#pragma unroll
                                for (int u = 0; u < 4; u++) {
                                    const int nn = c0 + cp * 64 + hh * 32 + 4 * e + u;
                                    const float t = fmaf(v[4 * e + u], inv_r, __ldg(b + nn));
                                    a[u] = fmaxf(t, 0.f) * rs;
                                }
                                split_e4m3x4(a, whi[hh * 8 + e], wlo[hh * 8 + e]);
                            }
                        }
                        tmem_st16(tA + (uint32_t)(c0 + cp * 64) / 4, whi);
                        tmem_st16(tA1 + (uint32_t)(c0 + cp * 64) / 4, wlo);
                    }
                    tmem_st_wait();
                    inv_r = inv_next;
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar_ar);
                } else {
                    const float *head = d.hw;
                    float zp = 0.f;
#pragma unroll
                    for (int c = 0; c < HALF / 32; c++) {
                        float v[32];
                        tmem_ld32(tD + c * 32, v);
                        tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 32; e++) {
                            const int nn = c0 + c * 32 + e;
                            const float t = fmaf(v[e], inv_r, __ldg(b + nn));
                            bad |= !(fabsf(t) < INFINITY);
                            zp = fmaf(__ldg(head + nn), fmaxf(t, 0.f), zp);
                        }
                    }
                    tc_fence_before();
                    float zo;
                    ok = pair_exchange(xbuf, warp, wq, bad ? __int_as_float(0x7fc00000) : zp, zo, ctl, pp, err);
                    if (!ok) break;
                    // the same sum on both warps: half 0's partial first
                    z = (half == 0 ? zp + zo : zo + zp) + __ldg(head + H);
                    if (bad) z = __int_as_float(0x7fc00000);
                }
            }
            if (!ok) break;
            if (half == 0) {
                if (xbad) z = __int_as_float(0x7fc00000);
                const bool fin = isfinite(z);
                const bool inside = valid && fin && z >= tau.up;
                // a non-finite fast logit goes to the FP32 re-check
                const bool flag = valid && (!fin || fabsf(z - tau.up) < margin || (z >= tau.dn && z < tau.up));
                const unsigned bi = __ballot_sync(FULL, inside);
                const unsigned bf = __ballot_sync(FULL, flag);
                const unsigned bn = __ballot_sync(FULL, valid && !fin);
                const long long wrow = tile * TILE_M + wq * 32;
                if (lane == 0 && wrow < n) bits[wrow >> 5] = bi;
                if (valid && logits) logits[row] = z;
                if (bf) {
                    unsigned pos = 0;
                    if (lane == 0) pos = atomicAdd(flag_count, (unsigned)__popc(bf));
                    pos = __shfl_sync(FULL, pos, 0);
                    if (flag) flag_idx[pos + __popc(bf & ((1u << lane) - 1u))] = (unsigned)row;
                }
                if (lane == 0) {
                    c_in += __popc(bi);
                    c_flag += __popc(bf);
                    c_nf += __popc(bn);
                }
            }
        }
        if (st && lane == 0 && half == 0) {
            if (c_in) atomicAdd(&st->n_inside, c_in);
            if (c_flag) atomicAdd(&st->n_flagged, c_flag);
            if (c_nf) atomicAdd(&st->n_nonfinite, c_nf);
        }
    }
    __syncthreads();
    if (warp == NEPI) {
        tc_fence_after();
        tmem_dealloc(tmem, TCOLS);
    }
}

// Scales of the E4M3 layer l (one warp per weight row n): s_n = 2^(8 - e) with
// max_k |W_nk / s'_k| = f 2^e, f in [0.5, 1), s'_k the previous E4M3 layer's row scales (1
// for the first); rows of zeros get 1.  Writes 1 / s_n and the folded bias b_n s_n.
__global__ void fp8_scale_kernel(Fp8Desc d, int l, float *inv_sw, float *bs) {
    const int H = d.H;
    const int nrow = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (nrow >= H) return;
    const float *W = d.p + d.off[l] + (size_t)nrow * H;
    const float *prev = l > 1 ? inv_sw + (size_t)(l - 2) * H : nullptr;
    float m = 0.f;
    for (int k = lane; k < H; k += 32) m = fmaxf(m, fabsf(prev ? W[k] * prev[k] : W[k]));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
    if (lane == 0) {
        float inv;
        const float sn = pow2_scale(m, inv);
        inv_sw[(size_t)(l - 1) * H + nrow] = inv;
        bs[(size_t)(l - 1) * H + nrow] = d.p[d.off[l] + H * H + nrow] * sn;
    }
}

// head weights of the folded form: w_n / s_n of the last E4M3 layer, then the bias
__global__ void fp8_head_kernel(Fp8Desc d, float *hw) {
    const int H = d.H;
    const float *inv = d.inv_sw + (size_t)(d.NHH - 1) * H;
    const float *w = d.p + d.off[d.NHH + 1];
    for (int n = threadIdx.x; n <= H; n += blockDim.x) hw[n] = n < H ? w[n] * inv[n] : w[H];
}

// FP32 master weights -> operand images (one thread per 16-byte chunk): the first layer as
// [W_hi | W_hi | W_lo | 0] in FP16 (K = 64), the others as the two E4M3 terms of
// W_nk s_n / s'_k (hi = E4M3 of it, lo = E4M3 of the remainder)
__global__ void pack_fp8_kernel(Fp8Desc d, uint8_t *img) {
    const int H = d.H;
    const uint32_t nchunks = d.img_bytes / 16;
    for (uint32_t ch = blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks; ch += gridDim.x * blockDim.x) {
        const uint32_t byte = ch * 16;
        uint4 o;
        if (byte < (uint32_t)(H * 128)) {
            const uint32_t nrow = byte / 128, pc = (byte % 128) / 16, c = pc ^ (nrow & 7);
            const float *W = d.p + d.off[0] + (size_t)nrow * d.in;
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const int k = (int)(c * 8) + e;
                const int kk = k & 15, sel = k < 32 ? 0 : (k < 48 ? 1 : 2);
                float w = 0.f;
                if (sel < 2 && kk < d.in) {
                    const float wf = W[kk];
                    const float wh = __half2float(__float2half_rn(wf));
                    w = sel == 0 ? wh : __half2float(__float2half_rn(wf - wh));
                }
                v[e] = w;
            }
            o.x = pack_f16(v[0], v[1]);
            o.y = pack_f16(v[2], v[3]);
            o.z = pack_f16(v[4], v[5]);
            o.w = pack_f16(v[6], v[7]);
        } else {
            const uint32_t rel = byte - H * 128;
            const int l = 1 + (int)(rel / (uint32_t)(2 * H * H));
            const uint32_t local = rel % (uint32_t)(2 * H * H);
            const uint32_t kb = local / fp8_chunk(H), in_chunk = local % fp8_chunk(H);
            const uint32_t term = in_chunk / (uint32_t)(H * 128), rem = in_chunk % (uint32_t)(H * 128);
            const uint32_t nrow = rem / 128, pc = (rem % 128) / 16, c = pc ^ (nrow & 7);
            const int k0 = (int)(kb * 128 + c * 16);
            const float *W = d.p + d.off[l] + (size_t)nrow * H + k0;
            const float s = 1.f / d.inv_sw[(size_t)(l - 1) * H + nrow];  // exact: a power of two
            const float *prev = l > 1 ? d.inv_sw + (size_t)(l - 2) * H + k0 : nullptr;
            float v[16];
#pragma unroll
            for (int e = 0; e < 16; e++) v[e] = (prev ? W[e] * prev[e] : W[e]) * s;  // W_nk s_n / s'_k
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const float v4[4] = {v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]};
                uint32_t hi, lo;
                split_e4m3x4(v4, hi, lo);
                w[e] = term == 0 ? hi : lo;
            }
            o = make_uint4(w[0], w[1], w[2], w[3]);
        }
        *reinterpret_cast<uint4 *>(img + byte) = o;
    }
}

Fp8Desc make_desc(const TcModel *tc, const MlpDesc &d) {
    Fp8Desc t{};
    t.in = d.w[0];
    t.H = d.w[1];
    t.NHH = d.L - 2;
    t.img = (const uint8_t *)tc->img;
    t.img_bytes = (uint32_t)tc->img_bytes;
    t.inv_sw = tc->scales;
    t.bs = tc->scales + (size_t)t.NHH * t.H;
    t.hw = tc->scales + (size_t)2 * t.NHH * t.H;
    t.p = d.p;
    for (int l = 0; l < d.L; l++) t.off[l] = d.off[l];
    return t;
}

int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

size_t nb_fp8_img_bytes(int H, int NHH) { return (size_t)H * 128 + (size_t)NHH * 2 * H * H; }
size_t nb_fp8_smem_bytes(int H, int NHH) {
    (void)NHH;
    return 1024 + CTL_BYTES + (size_t)H * 128 + 2 * (size_t)fp8_chunk(H);
}

nb_status nb_fp8_refresh(TcModel *tc, const MlpDesc &d, cudaStream_t s) {
    const Fp8Desc t = make_desc(tc, d);
    for (int l = 1; l <= t.NHH; l++) {  // each layer's scales need the previous layer's
        fp8_scale_kernel<<<(t.H * 32 + 255) / 256, 256, 0, s>>>(t, l, tc->scales, (float *)t.bs);
        NB_CUDA(cudaGetLastError());
    }
    fp8_head_kernel<<<1, 256, 0, s>>>(t, (float *)t.hw);
    NB_CUDA(cudaGetLastError());
    const uint32_t nchunks = t.img_bytes / 16;
    pack_fp8_kernel<<<(nchunks + 255) / 256, 256, 0, s>>>(t, (uint8_t *)tc->img);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_fp8_query(TcModel *tc, const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin,
                       uint32_t *bits, float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s) {
    const Fp8Desc t = make_desc(tc, d);
    const size_t smem = nb_fp8_smem_bytes(t.H, t.NHH);
    const int64_t tiles = (n + TILE_M - 1) / TILE_M;
    int64_t grid = sm_count();
    if (grid > tiles) grid = tiles;
    if (grid < 1) return NB_OK;
    if (t.H == 256) {
        NB_CUDA(cudaFuncSetAttribute(fwd_fp8_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        fwd_fp8_kernel<256><<<(unsigned)grid, THREADS, smem, s>>>(t, q, (long long)n, tau, margin, bits, logits, st,
                                                                  ws.flag_count, ws.flag_idx, tc->err);
    } else {
        NB_CUDA(cudaFuncSetAttribute(fwd_fp8_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        fwd_fp8_kernel<128><<<(unsigned)grid, THREADS, smem, s>>>(t, q, (long long)n, tau, margin, bits, logits, st,
                                                                  ws.flag_count, ws.flag_idx, tc->err);
    }
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}
