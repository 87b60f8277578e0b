// Split-FP16 tensor-core forward of the bounding network h (Sec. 3.4 "Architecture").
//
// Every weight and every activation is carried as an FP16 pair hi + lo (about 22
// significant bits), and each layer is evaluated with three tcgen05 products per
// k-step, W_hi a_hi + W_hi a_lo + W_lo a_hi, accumulated in FP32 in tensor memory.
// The dropped W_lo a_lo term is ~2^-22 relative, so the logits track the FP32 network
// to a few FP32 roundings, where a single BF16 product loses ~2^-9 per operand.
//
// Data placement (one persistent CTA per SM):
//   shared memory  the split weight images of every layer, loaded once by the bulk-copy
//                  (TMA) engine, 128-byte-swizzled K-major (B operands);
//   tensor memory  per tile slot: the FP32 accumulator (H columns) and the next layer's
//                  activations as FP16 hi and lo halves (H/2 + H/2 columns), which the
//                  MMA reads directly as its A operand -- activations never leave the SM.
// Warp roles: two tile slots, each with its epilogue warps (one thread per query row =
// TMEM lane; the grouped kernel splits every row's columns between two warps), and one
// warp that allocates TMEM, loads the weights and issues the MMAs.  Layer 0 takes the
// input split the same way, A0 = [x_hi | x_lo | x_hi | 0] against
// B0 = [W_hi | W_hi | W_lo | 0] (stored K = 64; the products stop at K = 48, the zero
// block adds nothing).
// All waits are bounded; on expiry the kernel records NB_ETIMEOUT, drains the tensor
// pipe and frees TMEM before returning.
#include <cuda_fp16.h>

#include "tc.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace nbtc;

constexpr int TILE_M = 128;
// single-model kernel: 4 epilogue warps per tile slot, as many slots as tensor memory
// holds (2 at width 128, 4 at width 64), and the MMA warp after them
template <int H>
struct Single {
    static constexpr int NS = 512 / (2 * H);
    static constexpr int NEPI = 4 * NS;
    static constexpr int THREADS = (NEPI + 1) * 32;
};
constexpr unsigned SPIN_LIMIT = 1u << 22;
constexpr unsigned FULL = 0xffffffffu;

struct SplitDesc {
    int in, H, NH;
    int act;  // hidden activation (NB_ACT_RELU or NB_ACT_SINE)
    const uint8_t *img;
    uint32_t img_bytes;
    const float *p;
    int off[NB_MAXL];
};

// layer 0: H rows x 128 B; layer l >= 1: hi image then lo image, each H/64 blocks of
// H rows x 128 B
__host__ __device__ inline uint32_t split_off(int H, int l) {
    return l == 0 ? 0u : (uint32_t)(H * 128 + (l - 1) * 4 * H * H);
}

struct Ctl {
    uint64_t wbar, aready[4], accfull[4], drain;
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

// Grouped kernel: 16 epilogue warps, 8 per tile slot; warps w and w + 4 of a slot share
// the TMEM lanes of quarter w mod 4 and take one half of the columns each, so a layer's
// epilogue (TMEM load, bias, ReLU, hi/lo split, TMEM store) has twice the warps; the two
// halves of a row exchange their partial head sums through shared memory under a bounded
// mbarrier handshake.  (At width 64 this is 10 % faster than 4 warps per slot; at width
// 128 the single-model kernel keeps 4 warps per slot, 2 % faster there.)
constexpr int SEPI = 16;
constexpr int STHREADS = (SEPI + 1) * 32;

// hidden activation of the epilogue: ReLU, or sin for NB_ACT_SINE networks
template <bool SINE>
__device__ __forceinline__ float act_f(float x) {
    return SINE ? sinf(x) : fmaxf(x, 0.f);
}

template <int H, bool SINE>
__global__ void __launch_bounds__(Single<H>::THREADS, 1)
    fwd_split_kernel(SplitDesc d, const float *__restrict__ q, long long n, TauF tau, float margin,
                     uint32_t *__restrict__ bits, float *__restrict__ logits, nb_query_stats *st,
                     unsigned *flag_count, unsigned *flag_idx, int *err) {
    constexpr uint32_t SLOT_COLS = 2 * H;  // accumulator H + activations H/2 hi + H/2 lo
    constexpr int NS = Single<H>::NS, NEPI = Single<H>::NEPI, THREADS = Single<H>::THREADS;
    extern __shared__ uint8_t smem_raw[];
    Ctl *ctl = reinterpret_cast<Ctl *>(smem_raw);
    uint8_t *Wimg = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023) + 1024;
    float *bias = reinterpret_cast<float *>(Wimg + d.img_bytes);
    float *head = bias + d.NH * H;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long ntiles = (n + TILE_M - 1) / TILE_M;
    const uint32_t bar_w = smem_u32(&ctl->wbar), bar_drain = smem_u32(&ctl->drain);
    uint32_t bar_ar[NS], bar_af[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) {
        bar_ar[i] = smem_u32(&ctl->aready[i]);
        bar_af[i] = smem_u32(&ctl->accfull[i]);
    }

    if (threadIdx.x == 0) {
        mbar_init(bar_w, 1);
        for (int i = 0; i < NS; i++) {
            mbar_init(bar_ar[i], 4);
            mbar_init(bar_af[i], 1);
        }
        mbar_init(bar_drain, 1);
        ctl->abort = 0;
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < d.NH * H; i += THREADS) {
        const int l = i / H, j = i % H;
        const int K = l == 0 ? d.in : H;
        bias[i] = d.p[d.off[l] + H * K + j];
    }
    for (int i = threadIdx.x; i <= H; i += THREADS) head[i] = d.p[d.off[d.NH] + i];
    if (warp == NEPI) {
        tmem_alloc(smem_u32(&ctl->tmem), NS * SLOT_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem;

    if (warp == NEPI) {
        if (lane == 0) {
            mbar_expect_tx(bar_w, d.img_bytes);
            for (uint32_t o = 0; o < d.img_bytes; o += 16384)
                bulk_g2s(smem_u32(Wimg) + o, d.img + o, min(16384u, d.img_bytes - o), bar_w);
            bool ok = wait_bounded(bar_w, 0, ctl, err);
            uint32_t ph[NS] = {};
            constexpr uint32_t idesc = idesc_f16(TILE_M, H);
            const uint32_t wbase = smem_u32(Wimg);
            for (long long it = 0; ok; it++) {
                if (blockIdx.x + (NS * it) * gridDim.x >= ntiles) break;
                for (int l = 0; l < d.NH && ok; l++)
                    for (int s = 0; s < NS && ok; s++) {
                        if (blockIdx.x + (NS * it + s) * gridDim.x >= ntiles) continue;
                        ok = wait_bounded(bar_ar[s], ph[s], ctl, err);
                        ph[s] ^= 1;
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t dt = tmem + s * SLOT_COLS;
                        const uint32_t ahi = dt + H, alo = dt + H + H / 2;
                        if (l == 0) {  // K = 48: the fourth 16-wide block of A0 and B0 is zero
                            for (int j = 0; j < 3; j++)
                                mma_f16_ts(dt, ahi + 8 * j, sdesc_sw128(wbase + 32 * j), idesc, j > 0 ? 1u : 0u);
                        } else {
                            const uint32_t whi = wbase + split_off(H, l), wlo = whi + 2 * H * H;
                            for (int j = 0; j < H / 16; j++) {
                                const uint32_t kb = j >> 2, within = (j & 3) * 32;
                                const uint64_t bhi = sdesc_sw128(whi + kb * (H * 128) + within);
                                const uint64_t blo = sdesc_sw128(wlo + kb * (H * 128) + within);
                                mma_f16_ts(dt, ahi + 8 * j, bhi, idesc, j > 0 ? 1u : 0u);
                                mma_f16_ts(dt, alo + 8 * j, bhi, idesc, 1u);
                                mma_f16_ts(dt, ahi + 8 * j, blo, idesc, 1u);
                            }
                        }
                        mma_commit(bar_af[s]);
                    }
            }
            mma_commit(bar_drain);
            wait_bounded(bar_drain, 0, ctl, err);
            if (!ok) *(volatile int *)&ctl->abort = 1;
        }
        __syncwarp();
    } else {
        const int s = warp >> 2, wq = warp & 3;
        const int r = wq * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(wq * 32) << 16) + s * SLOT_COLS;
        const uint32_t tD = trow, tAhi = trow + H, tAlo = trow + H + H / 2;
        uint32_t ph = 0;
        unsigned long long c_in = 0, c_flag = 0, c_nf = 0;
        const int in = d.in;
        float x[16];
        {
            const long long tile0 = blockIdx.x + (long long)s * gridDim.x;
            const long long row0 = tile0 * TILE_M + r;
#pragma unroll
            for (int k = 0; k < 16; k++) x[k] = (row0 < n && k < in) ? __ldg(q + row0 * in + k) : 0.f;
        }
        for (long long it = 0;; it++) {
            const long long tile = blockIdx.x + (NS * it + s) * gridDim.x;
            if (tile >= ntiles) break;
            const long long row = tile * TILE_M + r;
            const bool valid = row < n;
            bool xbad = false;  // a non-finite input coordinate: the logit is made NaN
#pragma unroll
            for (int k = 0; k < 16; k++) xbad = xbad || !isfinite(x[k]);
            {
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
                tmem_st16(tAhi, w0);
                tmem_st16(tAhi + 16, w1);
                tmem_st_wait();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_ar[s]);
            {
                // prefetch the next tile's rows while this tile runs through the layers
                const long long nrow = (tile + NS * (long long)gridDim.x) * TILE_M + r;
#pragma unroll
                for (int k = 0; k < 16; k++) x[k] = (nrow < n && k < in) ? __ldg(q + nrow * in + k) : 0.f;
            }
            bool ok = true;
            float z = 0.f;
            for (int l = 0; l < d.NH; l++) {
                ok = warp_wait(bar_af[s], ph, ctl, err);
                ph ^= 1;
                if (!ok) break;
                tc_fence_after();
                const float *b = bias + l * H;
                // hidden layer: relu(acc + b) split into FP16 hi / lo for the next layer's A
                // operand; head: z += head . relu(acc + b)
                auto hidden_chunk = [&](const float(&v)[32], int c) {
                    const float4 *b4 = reinterpret_cast<const float4 *>(b + c * 32);
                    uint32_t hi[16], lo[16];
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const float4 bb = b4[e];
                        split_f16x2(act_f<SINE>(v[4 * e] + bb.x), act_f<SINE>(v[4 * e + 1] + bb.y), hi[2 * e],
                                    lo[2 * e]);
                        split_f16x2(act_f<SINE>(v[4 * e + 2] + bb.z), act_f<SINE>(v[4 * e + 3] + bb.w), hi[2 * e + 1],
                                    lo[2 * e + 1]);
                    }
                    tmem_st16(tAhi + c * 16, hi);
                    tmem_st16(tAlo + c * 16, lo);
                };
                auto head_chunk = [&](const float(&v)[32], int c) {
                    const float4 *b4 = reinterpret_cast<const float4 *>(b + c * 32);
                    const float4 *h4 = reinterpret_cast<const float4 *>(head + c * 32);
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const float4 bb = b4[e], hh = h4[e];
                        z = fmaf(hh.x, act_f<SINE>(v[4 * e] + bb.x), z);
                        z = fmaf(hh.y, act_f<SINE>(v[4 * e + 1] + bb.y), z);
                        z = fmaf(hh.z, act_f<SINE>(v[4 * e + 2] + bb.z), z);
                        z = fmaf(hh.w, act_f<SINE>(v[4 * e + 3] + bb.w), z);
                    }
                };
                const bool last = l == d.NH - 1;
                auto chunk = [&](const float(&v)[32], int c) {
                    if (last) head_chunk(v, c);
                    else hidden_chunk(v, c);
                };
                if constexpr (H == 128) {
                    // the accumulator's four 32-column chunks are read one ahead: chunk c + 1's
                    // TMEM load is in flight while chunk c is converted
                    float va[32], vb[32];
                    tmem_ld32(tD, va);
                    tmem_ld_wait();
                    tmem_reg_fence(va);
                    tmem_ld32(tD + 32, vb);
                    chunk(va, 0);
                    tmem_ld_wait();
                    tmem_reg_fence(vb);
                    tmem_ld32(tD + 64, va);
                    chunk(vb, 1);
                    tmem_ld_wait();
                    tmem_reg_fence(va);
                    tmem_ld32(tD + 96, vb);
                    chunk(va, 2);
                    tmem_ld_wait();
                    tmem_reg_fence(vb);
                    chunk(vb, 3);
                } else {
#pragma unroll
                    for (int c = 0; c < H / 32; c++) {
                        float v[32];
                        tmem_ld32(tD + c * 32, v);
                        tmem_ld_wait();
                        tmem_reg_fence(v);
                        chunk(v, c);
                    }
                }
                if (!last) {
                    tmem_st_wait();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar_ar[s]);
                } else {
                    tc_fence_before();
                    z += head[H];
                }
            }
            if (!ok) break;
            if (xbad) z = __int_as_float(0x7fc00000);
            const bool fin = isfinite(z);
            const bool inside = valid && fin && z >= tau.up;
            // a non-finite fast logit (e.g. an FP16 overflow) goes to the FP32 re-check
            const bool flag =
                valid && (!fin || fabsf(z - tau.up) < margin || (z >= tau.dn && z < tau.up));
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
        if (st && lane == 0) {
            if (c_in) atomicAdd(&st->n_inside, c_in);
            if (c_flag) atomicAdd(&st->n_flagged, c_flag);
            if (c_nf) atomicAdd(&st->n_nonfinite, c_nf);
        }
    }
    __syncthreads();
    if (warp == NEPI) {
        tc_fence_after();
        tmem_dealloc(tmem, NS * SLOT_COLS);
    }
}

// FP32 master weights -> split FP16 operand images (one thread per 16-byte chunk);
// blockIdx.y selects the object of a group (parameters at o * P, image at o * img_bytes)
__global__ void pack_split_kernel(SplitDesc d, uint8_t *img, long long P) {
    d.p += (size_t)blockIdx.y * P;
    img += (size_t)blockIdx.y * d.img_bytes;
    const int H = d.H;
    const uint32_t nchunks = d.img_bytes / 16;
    for (uint32_t ch = blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks; ch += gridDim.x * blockDim.x) {
        const uint32_t byte = ch * 16;
        int l, part = 0;  // part 0: hi image, 1: lo image
        uint32_t local;
        if (byte < (uint32_t)(H * 128)) {
            l = 0;
            local = byte;
        } else {
            const uint32_t rel = byte - H * 128;
            l = 1 + (int)(rel / (uint32_t)(4 * H * H));
            const uint32_t in_layer = rel % (uint32_t)(4 * H * H);
            part = in_layer >= (uint32_t)(2 * H * H);
            local = in_layer % (uint32_t)(2 * H * H);
        }
        const int K = l == 0 ? d.in : H;
        const uint32_t kb = local / (uint32_t)(H * 128), rem = local % (uint32_t)(H * 128);
        const uint32_t nrow = rem / 128, pc = (rem % 128) / 16, c = pc ^ (nrow & 7);
        const float *W = d.p + d.off[l] + (size_t)nrow * K;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int k = (int)(kb * 64 + c * 8) + e;
            float w = 0.f;
            int sel = part;  // 0: hi, 1: lo
            int kk = k;
            if (l == 0) {  // [W_hi | W_hi | W_lo | 0], 16 columns each
                kk = k & 15;
                sel = k < 32 ? 0 : (k < 48 ? 1 : 2);
            }
            if (sel < 2 && kk < K) {
                const float wf = W[kk];
                const float wh = __half2float(__float2half_rn(wf));
                w = sel == 0 ? wh : __half2float(__float2half_rn(wf - wh));
            }
            v[e] = w;
        }
        uint4 o;
        o.x = pack_f16(v[0], v[1]);
        o.y = pack_f16(v[2], v[3]);
        o.z = pack_f16(v[4], v[5]);
        o.w = pack_f16(v[6], v[7]);
        *reinterpret_cast<uint4 *>(img + byte) = o;
    }
}

SplitDesc make_desc(const TcModel *tc, const MlpDesc &d) {
    SplitDesc t{};
    t.in = d.w[0];
    t.H = d.w[1];
    t.NH = d.L - 1;
    t.act = d.act;
    t.img = (const uint8_t *)tc->img;
    t.img_bytes = (uint32_t)tc->img_bytes;
    t.p = d.p;
    for (int l = 0; l < d.L; l++) t.off[l] = d.off[l];
    return t;
}

int num_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

size_t nb_split_img_bytes(int H, int NH) { return split_off(H, NH); }

size_t nb_split_smem_bytes(int H, int NH) {
    return 2048 + nb_split_img_bytes(H, NH) + (size_t)(NH * H + H + 4 + SEPI * 32) * sizeof(float);
}

nb_status nb_split_refresh(TcModel *tc, const MlpDesc &d, cudaStream_t s) {
    const SplitDesc t = make_desc(tc, d);
    const uint32_t nchunks = t.img_bytes / 16;
    pack_split_kernel<<<(nchunks + 255) / 256, 256, 0, s>>>(t, (uint8_t *)tc->img, 0);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_split_query(TcModel *tc, const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin,
                         uint32_t *bits, float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s) {
    const SplitDesc t = make_desc(tc, d);
    const size_t smem = nb_split_smem_bytes(t.H, t.NH);
    const int64_t tiles = (n + TILE_M - 1) / TILE_M;
    int64_t grid = num_sms();
    const int ns = t.H == 64 ? Single<64>::NS : Single<128>::NS;
    if (grid > (tiles + ns - 1) / ns) grid = (tiles + ns - 1) / ns;
    if (grid < 1) grid = 1;
#define NB_SPLIT(HV, SV)                                                                                           \
    do {                                                                                                          \
        NB_CUDA(cudaFuncSetAttribute(fwd_split_kernel<HV, SV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        fwd_split_kernel<HV, SV><<<(unsigned)grid, Single<HV>::THREADS, smem, s>>>(                                 \
            t, q, (long long)n, tau, margin, bits, logits, st, ws.flag_count, ws.flag_idx, tc->err);              \
    } while (0)
    const bool sine = t.act == NB_ACT_SINE;
    if (t.H == 128) {
        if (sine) NB_SPLIT(128, true);
        else NB_SPLIT(128, false);
    } else {
        if (sine) NB_SPLIT(64, true);
        else NB_SPLIT(64, false);
    }
#undef NB_SPLIT
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// ------------------------------------------------------------------ grouped queries
// One persistent launch over the work items of a plan (rows of one object each).  A CTA
// keeps one object's split weights, biases and head in shared memory and reloads them
// only when its next item belongs to another object.  Item hand-off between the MMA warp
// and the epilogue warps uses two more mbarriers (item ready / item done); every wait
// is bounded like the per-layer ones.
#include "group.cuh"

namespace {

struct GCtl {
    uint64_t wbar, aready[4], accfull[4], drain, item_ready, item_done;
    uint64_t pair[8];  // head-sum handshake of the two warps of each (slot, lane quarter)
    uint32_t tmem;
    int abort;
};

__device__ bool gwait(uint32_t bar, uint32_t parity, GCtl *ctl, int *err) {
    for (unsigned i = 0; i < SPIN_LIMIT; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*(volatile int *)&ctl->abort) return false;
    }
    *(volatile int *)&ctl->abort = 1;
    atomicExch(err, NB_ETIMEOUT);
    return false;
}
__device__ __forceinline__ bool gwarp_wait(uint32_t bar, uint32_t parity, GCtl *ctl, int *err) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = gwait(bar, parity, ctl, err) ? 1 : 0;
    return __shfl_sync(FULL, ok, 0) != 0;
}

template <int H>
__global__ void __launch_bounds__(STHREADS, 1)
    fwd_split_group_kernel(SplitDesc d, long long P, const PlanItem *__restrict__ items, int n_items,
                           const TauF *__restrict__ taus, const float *__restrict__ q, float margin,
                           uint32_t *__restrict__ bits, float *__restrict__ logits, nb_query_stats *st,
                           unsigned *flag_count, unsigned *flag_idx, int *err) {
    constexpr uint32_t SLOT_COLS = 2 * H;
    // tile slots: as many as tensor memory holds (4 at width 64, 2 at width 128); the 16
    // epilogue warps are shared out among them, and where a slot has 8 the two warps of a
    // lane quarter split the columns (and exchange partial head sums)
    constexpr int NS = 512 / (int)SLOT_COLS;
    constexpr int WPS = SEPI / NS;
    constexpr bool SPLIT = WPS == 8;
    constexpr int HALF = SPLIT ? H / 2 : H;  // columns per epilogue warp
    extern __shared__ uint8_t smem_raw[];
    GCtl *ctl = reinterpret_cast<GCtl *>(smem_raw);
    uint8_t *Wimg = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023) + 1024;
    float *bias = reinterpret_cast<float *>(Wimg + d.img_bytes);
    float *head = bias + d.NH * H;
    float *xbuf = head + H + 4;  // [16 warps][32 lanes] partial head sums

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar_w = smem_u32(&ctl->wbar), bar_drain = smem_u32(&ctl->drain);
    const uint32_t bar_ready = smem_u32(&ctl->item_ready), bar_done = smem_u32(&ctl->item_done);
    uint32_t bar_ar[NS], bar_af[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) {
        bar_ar[i] = smem_u32(&ctl->aready[i]);
        bar_af[i] = smem_u32(&ctl->accfull[i]);
    }
    if (threadIdx.x == 0) {
        mbar_init(bar_w, 1);
        for (int i = 0; i < NS; i++) {
            mbar_init(bar_ar[i], WPS);
            mbar_init(bar_af[i], 1);
        }
        mbar_init(bar_drain, 1);
        mbar_init(bar_ready, 1);
        mbar_init(bar_done, SEPI);
        for (int i = 0; i < 8; i++) mbar_init(smem_u32(&ctl->pair[i]), 64);
        ctl->abort = 0;
        fence_mbar_init();
    }
    if (warp == SEPI) {
        tmem_alloc(smem_u32(&ctl->tmem), NS * SLOT_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem;

    if (warp == SEPI) {
        uint32_t ph_ar[NS] = {}, ph_w = 0, ph_done = 0, ph_drain = 0;
        int cur_obj = -1;
        bool ok = true;
        constexpr uint32_t idesc = idesc_f16(TILE_M, H);
        const uint32_t wbase = smem_u32(Wimg);
        int k0, k1;
        item_range(n_items, k0, k1);
        for (int k = k0; ok && k < k1; k++) {
            const PlanItem it = items[k];
            if (k != k0) {
                ok = gwarp_wait(bar_done, ph_done, ctl, err);
                ph_done ^= 1;
                if (!ok) break;
            }
            if (it.obj != cur_obj) {
                if (cur_obj >= 0) {  // the previous object's MMAs are done with its weights
                    if (lane == 0) mma_commit(bar_drain);
                    ok = gwarp_wait(bar_drain, ph_drain, ctl, err);
                    ph_drain ^= 1;
                    if (!ok) break;
                }
                const float *pp = d.p + (size_t)it.obj * P;
                for (int i = lane; i < d.NH * H; i += 32) {
                    const int l = i / H, j = i % H;
                    bias[i] = pp[d.off[l] + H * (l == 0 ? d.in : H) + j];
                }
                for (int i = lane; i <= H; i += 32) head[i] = pp[d.off[d.NH] + i];
                if (lane == 0) {
                    const uint8_t *src = d.img + (size_t)it.obj * d.img_bytes;
                    mbar_expect_tx(bar_w, d.img_bytes);
                    for (uint32_t o = 0; o < d.img_bytes; o += 16384)
                        bulk_g2s(wbase + o, src + o, min(16384u, d.img_bytes - o), bar_w);
                }
                ok = gwarp_wait(bar_w, ph_w, ctl, err);
                ph_w ^= 1;
                if (!ok) break;
                cur_obj = it.obj;
            }
            __threadfence_block();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_ready);
            const long long nt = (it.row1 - it.row0 + TILE_M - 1) / TILE_M;
            int okl = 1;
            if (lane == 0) {
                for (long long tp = 0; okl && NS * tp < nt; tp++) {
                    for (int l = 0; l < d.NH && okl; l++)
                        for (int s = 0; s < NS && okl; s++) {
                            if (NS * tp + s >= nt) continue;
                            okl = gwait(bar_ar[s], ph_ar[s], ctl, err);
                            ph_ar[s] ^= 1;
                            if (!okl) break;
                            tc_fence_after();
                            const uint32_t dt = tmem + s * SLOT_COLS;
                            const uint32_t ahi = dt + H, alo = dt + H + H / 2;
                            if (l == 0) {  // K = 48: the fourth 16-wide block of A0 and B0 is zero
                                for (int j = 0; j < 3; j++)
                                    mma_f16_ts(dt, ahi + 8 * j, sdesc_sw128(wbase + 32 * j), idesc, j > 0 ? 1u : 0u);
                            } else {
                                const uint32_t whi = wbase + split_off(H, l), wlo = whi + 2 * H * H;
                                for (int j = 0; j < H / 16; j++) {
                                    const uint32_t kb = j >> 2, within = (j & 3) * 32;
                                    const uint64_t bhi = sdesc_sw128(whi + kb * (H * 128) + within);
                                    const uint64_t blo = sdesc_sw128(wlo + kb * (H * 128) + within);
                                    mma_f16_ts(dt, ahi + 8 * j, bhi, idesc, j > 0 ? 1u : 0u);
                                    mma_f16_ts(dt, alo + 8 * j, bhi, idesc, 1u);
                                    mma_f16_ts(dt, ahi + 8 * j, blo, idesc, 1u);
                                }
                            }
                            mma_commit(bar_af[s]);
                        }
                }
            }
            ok = __shfl_sync(FULL, okl, 0) != 0;
        }
        if (lane == 0) {
            mma_commit(bar_drain);
            gwait(bar_drain, ph_drain, ctl, err);
            if (!ok) *(volatile int *)&ctl->abort = 1;
        }
        __syncwarp();
    } else {
        const int s = warp / WPS, ws = warp % WPS, wq = ws & 3, hf = ws >> 2;
        const int r = wq * 32 + lane;
        const int c0 = hf * HALF;  // first neuron of this warp
        const uint32_t trow = tmem + ((uint32_t)(wq * 32) << 16) + s * SLOT_COLS;
        const uint32_t tD = trow + c0, tAhi = trow + H, tAlo = trow + H + H / 2;
        const uint32_t bar_pair = SPLIT ? smem_u32(&ctl->pair[(s * 4 + wq) & 7]) : 0u;
        const int in = d.in;
        uint32_t ph_acc = 0, ph_ready = 0, pp = 0;
        unsigned long long c_in = 0, c_flag = 0, c_nf = 0;
        bool ok = true;
        int k0, k1;
        item_range(n_items, k0, k1);
        for (int k = k0; ok && k < k1; k++) {
            const PlanItem it = items[k];
            ok = gwarp_wait(bar_ready, ph_ready, ctl, err);
            ph_ready ^= 1;
            if (!ok) break;
            const TauF tau = taus[it.obj];
            const long long nt = (it.row1 - it.row0 + TILE_M - 1) / TILE_M;
            float x[16];
            if (hf == 0) {
                const long long row0 = it.row0 + (long long)s * TILE_M + r;  // the slot's first tile
#pragma unroll
                for (int kk = 0; kk < 16; kk++) x[kk] = (row0 < it.row1 && kk < in) ? __ldg(q + row0 * in + kk) : 0.f;
            }
            for (long long tp = 0; ok && NS * tp + s < nt; tp++) {
                const long long trow0 = it.row0 + (NS * tp + s) * TILE_M;
                const long long row = trow0 + r;
                const bool valid = row < it.row1;
                bool xbad = false;  // a non-finite input coordinate: the logit is made NaN
                if (hf == 0) {
#pragma unroll
                    for (int kk = 0; kk < 16; kk++) xbad = xbad || !isfinite(x[kk]);
                    uint32_t w0[16], w1[16];
#pragma unroll
                    for (int kk = 0; kk < 8; kk++) {
                        uint32_t hi, lo;
                        split_f16x2(x[2 * kk], x[2 * kk + 1], hi, lo);
                        w0[kk] = hi;
                        w0[8 + kk] = lo;
                        w1[kk] = hi;
                        w1[8 + kk] = 0u;
                    }
                    tmem_st16(tAhi, w0);
                    tmem_st16(tAhi + 16, w1);
                    tmem_st_wait();
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_ar[s]);
                if (hf == 0) {
                    const long long nrow = trow0 + NS * TILE_M + r;
#pragma unroll
                    for (int kk = 0; kk < 16; kk++)
                        x[kk] = (nrow < it.row1 && kk < in) ? __ldg(q + nrow * in + kk) : 0.f;
                }
                float z = 0.f;
                for (int l = 0; l < d.NH; l++) {
                    ok = gwarp_wait(bar_af[s], ph_acc, ctl, err);
                    ph_acc ^= 1;
                    if (!ok) break;
                    tc_fence_after();
                    const float *b = bias + l * H + c0;
                    if (l < d.NH - 1) {
#pragma unroll
                        for (int c = 0; c < HALF / 32; c++) {
                            float v[32];
                            tmem_ld32(tD + c * 32, v);
                            tmem_ld_wait();
                            uint32_t hi[16], lo[16];
#pragma unroll
                            for (int e = 0; e < 16; e++) {
                                const float a0 = fmaxf(v[2 * e] + b[c * 32 + 2 * e], 0.f);
                                const float a1 = fmaxf(v[2 * e + 1] + b[c * 32 + 2 * e + 1], 0.f);
                                split_f16x2(a0, a1, hi[e], lo[e]);
                            }
                            tmem_st16(tAhi + c0 / 2 + c * 16, hi);
                            tmem_st16(tAlo + c0 / 2 + c * 16, lo);
                        }
                        tmem_st_wait();
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(bar_ar[s]);
                    } else {
                        float zp = 0.f;
#pragma unroll
                        for (int c = 0; c < HALF / 32; c++) {
                            float v[32];
                            tmem_ld32(tD + c * 32, v);
                            tmem_ld_wait();
#pragma unroll
                            for (int e = 0; e < 32; e++)
                                zp = fmaf(head[c0 + c * 32 + e], fmaxf(v[e] + b[c * 32 + e], 0.f), zp);
                        }
                        tc_fence_before();
                        if (SPLIT) {
                            // exchange the partial sums with the other half of the row
                            xbuf[warp * 32 + lane] = zp;
                            mbar_arrive(bar_pair);
                            ok = gwait(bar_pair, pp, ctl, err);
                            pp ^= 1;
                            const float zo = xbuf[(warp ^ 4) * 32 + lane];
                            ok = __all_sync(FULL, ok);
                            if (!ok) break;
                            z = (hf == 0 ? zp + zo : zo + zp) + head[H];
                        } else {
                            z = zp + head[H];
                        }
                    }
                }
                if (!ok) break;
                if (hf != 0) continue;
                if (xbad) z = __int_as_float(0x7fc00000);
                const bool fin = isfinite(z);
                const bool inside = valid && fin && z >= tau.up;
                const bool flag = valid && (!fin || fabsf(z - tau.up) < margin || (z >= tau.dn && z < tau.up));
                const unsigned bi = __ballot_sync(FULL, inside);
                const unsigned bf = __ballot_sync(FULL, flag);
                const unsigned bn = __ballot_sync(FULL, valid && !fin);
                const long long wrow = trow0 + wq * 32;
                if (lane == 0 && wrow < it.row1) bits[wrow >> 5] = bi;
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
            if (!ok) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_done);
        }
        if (st && lane == 0 && hf == 0) {
            if (c_in) atomicAdd(&st->n_inside, c_in);
            if (c_flag) atomicAdd(&st->n_flagged, c_flag);
            if (c_nf) atomicAdd(&st->n_nonfinite, c_nf);
        }
    }
    __syncthreads();
    if (warp == SEPI) {
        tc_fence_after();
        tmem_dealloc(tmem, NS * SLOT_COLS);
    }
}

}  // namespace

nb_status nb_tc_group_init(TcModel *tc, const MlpDesc &d, int n_objects) {
    tc->infer_prec = NB_F16X3;
    tc->train_prec = NB_F32;
    const int H = d.w[1], NH = d.L - 1;
    if (NH < 1) return nb_fail(NB_EUNSUPPORTED, "tensor-core forward needs at least one hidden layer");
    if (d.w[0] > 16) return nb_fail(NB_EUNSUPPORTED, "tensor-core forward: input width must be <= 16");
    if (H != 64 && H != 128) return nb_fail(NB_EUNSUPPORTED, "tensor-core forward: hidden width must be 64 or 128");
    for (int l = 1; l < d.L; l++)
        if (d.w[l] != H) return nb_fail(NB_EUNSUPPORTED, "tensor-core forward: hidden widths must be equal");
    int dev = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (nb_split_smem_bytes(H, NH) > (size_t)maxsm)
        return nb_fail(NB_EUNSUPPORTED, "tensor-core forward: the network's weights do not fit in shared memory");
    tc->img_bytes = nb_split_img_bytes(H, NH);
    if (cudaMalloc(&tc->img, tc->img_bytes * (size_t)n_objects) != cudaSuccess ||
        cudaMalloc(&tc->err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return nb_fail(NB_ENOMEM, "tensor-core image allocation failed");
    }
    cudaMemset(tc->err, 0, sizeof(int));
    return NB_OK;
}

nb_status nb_tc_group_refresh(TcModel *tc, const MlpDesc &d, int n_objects, cudaStream_t s) {
    const SplitDesc t = make_desc(tc, d);
    long long P = 0;
    for (int l = 0; l < d.L; l++) P += (long long)d.w[l + 1] * (d.w[l] + 1);
    const uint32_t nchunks = t.img_bytes / 16;
    pack_split_kernel<<<dim3((nchunks + 255) / 256, n_objects), 256, 0, s>>>(t, (uint8_t *)tc->img, P);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_tc_group_query(TcModel *tc, const MlpDesc &d, int64_t P, const nb_plan *pl, const float *q,
                            const TauF *taus, float margin, uint32_t *bits, float *logits, nb_query_stats *st,
                            QueryWs ws, cudaStream_t s) {
    const SplitDesc t = make_desc(tc, d);
    const size_t smem = nb_split_smem_bytes(t.H, t.NH);
    int grid = num_sms();
    if (grid > pl->n_items) grid = pl->n_items;
    if (grid < 1) return NB_OK;
    if (t.H == 128) {
        NB_CUDA(cudaFuncSetAttribute(fwd_split_group_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        fwd_split_group_kernel<128><<<grid, STHREADS, smem, s>>>(t, (long long)P, pl->items, pl->n_items, taus, q,
                                                                margin, bits, logits, st, ws.flag_count, ws.flag_idx,
                                                                tc->err);
    } else {
        NB_CUDA(cudaFuncSetAttribute(fwd_split_group_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        fwd_split_group_kernel<64><<<grid, STHREADS, smem, s>>>(t, (long long)P, pl->items, pl->n_items, taus, q,
                                                               margin, bits, logits, st, ws.flag_count, ws.flag_idx,
                                                               tc->err);
    }
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}
