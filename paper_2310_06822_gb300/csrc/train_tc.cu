// tcgen05 training step of a 128-wide bounding network (Sec. 3.4 "Training"): forward,
// asymmetric BCE of Eq. (loss), backward and the CTA's gradient partial in one persistent
// kernel on the tensor cores, accumulators in tensor memory.  adam_kernel then sums the
// partials in CTA order and takes the Adam step on the FP32 master weights.
//
// Per tile of 128 samples (one sample per TMEM lane), every GEMM of the step is one chain
// of tcgen05.mma (BF16 operands in shared memory, FP32 accumulation in TMEM):
//   forward      Z_l  = A_l W_l^T            (A_l K-major, W_l K-major)
//   input grad   dA_l = dZ_l W_l             (dZ_l K-major, W_l read MN-major: the same image)
//   weight grad  dW_l += dZ_l^T A_l          (both read MN-major: the batch is the K dimension)
// so each activation and gradient tile is stored once, row-major and 128-byte swizzled,
// and read in whichever orientation a product needs.  dW_l of the hidden-to-hidden layers
// accumulates in tensor memory over all of the CTA's tiles (128 columns each) and is read
// out once at the end; the 128 remaining columns hold the current tile's forward sums or
// input gradient.  The first layer (input width <= 15) uses 8-row x 16-byte core matrices
// without swizzle; its weight gradient (N = 16) goes to the scratch columns every tile and
// is added up in registers, and a constant-1 input column 15 (zero weights) makes that
// product deliver the first layer's bias gradient too.  The head (width 1), the loss, dL/dz
// and the other bias gradients are
// FP32 in the epilogue warps; the bias and head gradients are summed over a warp's 32 rows
// by a shuffle transpose-reduction and over tiles in shared memory (one owner per sum).
//
// Shared memory holds every layer's BF16 weights (loaded once by the bulk-copy engine),
// the input tile and the hidden activations A_1 .. A_{NH-1}.  The backward pass overwrites
// each A_l in place with dZ_{l-1} once dW_l has consumed it (the tensor pipe completes in
// issue order).  dZ_{NH-1} needs one more buffer; where shared memory has no room for it
// (four hidden layers) it takes A_1's, and A_1 is recomputed from the input (a K = 16
// product) before dW_1.
//
// Warps: 16 epilogue warps (warp w serves TMEM lanes 32 (w mod 4) .. +31, i.e. those rows,
// and columns 32 (w / 4) .. +31 of each layer) and one warp that allocates TMEM, loads the
// weights and issues the MMAs from one lane.  The two sides alternate through two
// mbarriers; every wait is bounded (on expiry the kernel records NB_ETIMEOUT, drains the
// tensor pipe and frees TMEM before returning).
#include <cuda_bf16.h>
#include <math.h>

#include "tc.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace nbtc;

constexpr int TM = 128;         // samples per tile = TMEM lanes
constexpr int H = 128;          // hidden width
constexpr int NEPI = 16;        // epilogue warps
constexpr int THREADS = (NEPI + 1) * 32;
constexpr uint32_t W0_BYTES = 4096;     // 128 x 16 BF16, core matrices
constexpr uint32_t WL_BYTES = 32768;    // 128 x 128 BF16, two 64-column swizzled blocks
constexpr uint32_t BLK = 16384;         // one 64-column block of 128 rows
constexpr unsigned SPIN_LIMIT = 1u << 22;
constexpr unsigned FULL = 0xffffffffu;

struct TTDesc {
    int in, NH;              // input width (<= 16), hidden layers (2..4)
    const uint8_t *img;      // W_0 (core matrices), then W_1 .. W_{NH-1} (swizzled)
    uint32_t img_bytes;
    const float *p;          // FP32 master parameters (biases, head)
    int off[NB_MAXL];
};

struct Ctl {
    uint64_t wbar, mma, epi, drain, pair[4];
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

// lane l returns the sum over the warp's 32 lanes of v[l] (v is clobbered): five halving
// steps, each lane keeping the half of the columns its bit selects
__device__ __forceinline__ float xsum32(float (&v)[32], int lane) {
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool up = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; i++) {
            const float send = up ? v[i] : v[i + w];
            const float keep = up ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, w);
        }
    }
    return v[0];
}

__device__ __forceinline__ float softplusf(float u) { return u > 0.f ? u + log1pf(expf(-u)) : log1pf(expf(u)); }
__device__ __forceinline__ float sigmoidf(float u) {
    return u >= 0.f ? 1.f / (1.f + expf(-u)) : expf(u) / (1.f + expf(u));
}

// byte offset of chunk c (8 columns, 0..7) of row m in the 64-column block of a swizzled buffer
__device__ __forceinline__ uint32_t sw_off(int m, int c) { return (uint32_t)m * 128u + (uint32_t)((c ^ (m & 7)) << 4); }
// byte offset of the 8 columns 8 h .. 8 h + 7 of row m in the core-matrix buffer (128 x 16)
__device__ __forceinline__ uint32_t cm_off(int m, int h) {
    return (uint32_t)(m >> 3) * 256u + (uint32_t)h * 128u + (uint32_t)(m & 7) * 16u;
}

// with four hidden layers dZ_{NH-1} takes A_1's buffer and A_1 is recomputed before dW_1
template <int NH>
__global__ void __launch_bounds__(THREADS, 1)
    train_tc_kernel(TTDesc d, const float *__restrict__ q, const uint32_t *__restrict__ labels, long long n,
                    float alpha, float beta, float inv_n, TauF tau, float *__restrict__ partial,
                    float *__restrict__ loss_partial, long long stride, nb_step_stats *st, int *err) {
    extern __shared__ uint8_t smem_raw[];
    Ctl *ctl = reinterpret_cast<Ctl *>(smem_raw);
    uint8_t *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023) + 1024;
    constexpr bool RECOMP = NH == 4;
    uint8_t *sW = base;                                  // W_0, W_1 .. W_{NH-1}
    uint8_t *sX = sW + d.img_bytes;                      // input tile (core matrices)
    uint8_t *sA = sX + W0_BYTES;                         // A_1 .. A_{NH-1}, then F
    float *bias = reinterpret_cast<float *>(sA + (size_t)(NH - 1 + (RECOMP ? 0 : 1)) * WL_BYTES);
    float *head = bias + NH * H;                         // [H + 1], padded to 132
    float *zpart = head + 132;                           // [4 lane quarters][4 column quarters][32]
    float *dbs = zpart + 512;                            // [4][NH + 1][H] bias and head-weight sums
    float *red2 = dbs + 4 * (NH + 1) * H;                // [4][2] loss and head-bias sums
    const uint32_t sWu = smem_u32(sW), sXu = smem_u32(sX), sAu = smem_u32(sA);
    auto bufA = [&](int l) { return sAu + (uint32_t)(l - 1) * WL_BYTES; };      // A_l, l >= 1
    const uint32_t ZB = RECOMP ? bufA(1) : bufA(NH);                      // dZ_{NH-1}
    auto wimg = [&](int l) { return sWu + (l == 0 ? 0u : W0_BYTES + (uint32_t)(l - 1) * WL_BYTES); };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long ntiles = (n + TM - 1) / TM;
    const uint32_t bar_w = smem_u32(&ctl->wbar), bar_mma = smem_u32(&ctl->mma), bar_epi = smem_u32(&ctl->epi),
                   bar_drain = smem_u32(&ctl->drain);

    if (threadIdx.x == 0) {
        mbar_init(bar_w, 1);
        mbar_init(bar_mma, 1);
        mbar_init(bar_epi, NEPI);
        mbar_init(bar_drain, 1);
        for (int i = 0; i < 4; i++) mbar_init(smem_u32(&ctl->pair[i]), 4);
        ctl->abort = 0;
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < NH * H; i += THREADS) {
        const int l = i / H, j = i % H;
        bias[i] = d.p[d.off[l] + H * (l == 0 ? d.in : H) + j];
    }
    for (int i = threadIdx.x; i <= H; i += THREADS) head[i] = d.p[d.off[NH] + i];
    for (int i = threadIdx.x; i < 4 * (NH + 1) * H; i += THREADS) dbs[i] = 0.f;
    if (warp == NEPI) {
        tmem_alloc(smem_u32(&ctl->tmem), 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem;

    if (warp == NEPI) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            mbar_expect_tx(bar_w, d.img_bytes);
            for (uint32_t o = 0; o < d.img_bytes; o += 16384)
                bulk_g2s(sWu + o, d.img + o, min(16384u, d.img_bytes - o), bar_w);
            bool ok = wait_bounded(bar_w, 0, ctl, err);
            uint32_t pe = 0;
            constexpr uint32_t id_fwd = idesc_bf16_mn(TM, H, 0, 0);   // A K-major, B K-major
            constexpr uint32_t id_da = idesc_bf16_mn(TM, H, 0, 1);    // B MN-major
            constexpr uint32_t id_dw = idesc_bf16_mn(H, H, 1, 1);     // both MN-major
            constexpr uint32_t id_dw0 = idesc_bf16_mn(H, 16, 1, 1);
            auto epi_wait = [&]() {
                if (!ok) return false;
                ok = wait_bounded(bar_epi, pe, ctl, err);
                pe ^= 1;
                if (ok) tc_fence_after();
                return ok;
            };
            // layer 0 forward: X (core matrices: LBO 128 along K, SBO 256 along M) x W_0^T
            auto mma_l0 = [&]() {
                mma_f16(tmem, sdesc_gen(sXu, 128, 256, 0), sdesc_gen(wimg(0), 128, 256, 0), id_fwd, 0u);
            };
            bool first = true;
#pragma unroll 1
            for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                if (!epi_wait()) break;  // input tile written
                mma_l0();
                mma_commit(bar_mma);
#pragma unroll 1
                for (int l = 1; l < NH; l++) {
                    if (!epi_wait()) break;  // A_l written
                    const uint32_t a = bufA(l), w = wimg(l);
                    for (int j = 0; j < H / 16; j++) {
                        const uint32_t o = (uint32_t)(j >> 2) * BLK + (uint32_t)(j & 3) * 32;
                        mma_f16(tmem, sdesc_gen(a + o, 16, 1024, 2), sdesc_gen(w + o, 16, 1024, 2), id_fwd,
                                j > 0 ? 1u : 0u);
                    }
                    mma_commit(bar_mma);
                }
                if (!epi_wait()) break;  // head pass: dZ_{NH-1} written
#pragma unroll 1
                for (int l = NH - 1; l >= 1; l--) {
                    if (l < NH - 1 && !epi_wait()) break;  // dZ_l written (in place of A_{l+1})
                    if (RECOMP && l == 1) {
                        mma_l0();
                        mma_commit(bar_mma);
                        if (!epi_wait()) break;  // A_1 rewritten
                    }
                    const uint32_t dz = l == NH - 1 ? ZB : bufA(l + 1), a = bufA(l), w = wimg(l);
                    const uint32_t dwcol = tmem + (uint32_t)(128 * l);
                    for (int j = 0; j < TM / 16; j++)  // dW_l += dZ_l^T A_l: K = batch rows 16 j ..
                        mma_f16(dwcol, sdesc_gen(dz + 2048u * j, BLK, 1024, 2), sdesc_gen(a + 2048u * j, BLK, 1024, 2),
                                id_dw, (first && j == 0) ? 0u : 1u);
                    for (int j = 0; j < H / 16; j++) {  // dA_l = dZ_l W_l: K = neurons 16 j ..
                        const uint32_t o = (uint32_t)(j >> 2) * BLK + (uint32_t)(j & 3) * 32;
                        mma_f16(tmem, sdesc_gen(dz + o, 16, 1024, 2), sdesc_gen(w + 2048u * j, BLK, 1024, 2), id_da,
                                j > 0 ? 1u : 0u);
                    }
                    mma_commit(bar_mma);
                }
                if (!epi_wait()) break;  // dZ_0 written (in place of A_1)
                // dW_0 (this tile only) = dZ_0^T X -> scratch columns 0 .. 15
                for (int j = 0; j < TM / 16; j++)
                    mma_f16(tmem, sdesc_gen(bufA(1) + 2048u * j, BLK, 1024, 2), sdesc_gen(sXu + 512u * j, 256, 128, 0),
                            id_dw0, j > 0 ? 1u : 0u);
                mma_commit(bar_mma);
                first = false;
            }
            // every issued product has completed before the epilogue's last read and the
            // release of tensor memory
            mma_commit(bar_drain);
            wait_bounded(bar_drain, 0, ctl, err);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue warps
        const int qd = warp & 3, cq = warp >> 2;            // lane quarter, column quarter
        const int m = qd * 32 + lane;                        // row of the tile = TMEM lane
        const uint32_t trow = tmem + ((uint32_t)(qd * 32) << 16);
        const uint32_t tcol = trow + 32 * cq;                // this thread's 32 scratch columns
        const uint32_t blk = (uint32_t)(cq >> 1) * BLK;      // its 64-column block in a swizzled buffer
        const int c0 = (cq & 1) * 4;                         // and its first 16-byte chunk there
        const uint32_t bar_quad = smem_u32(&ctl->pair[qd]);
        float *dbl = dbs + qd * (NH + 1) * H + 32 * cq + lane;  // + l H: this lane's column sums
        uint32_t pm = 0, pq = 0;
        float dw0acc[8];
#pragma unroll
        for (int i = 0; i < 8; i++) dw0acc[i] = 0.f;
        float gsum = 0.f, lossacc = 0.f;
        unsigned long long c_fn = 0, c_fp = 0, c_nf = 0;
        bool ok = true;
        auto mma_wait = [&]() {
            ok = ok && warp_wait(bar_mma, pm, ctl, err);
            pm ^= 1;
            if (ok) tc_fence_after();
            return ok;
        };
        auto arrive = [&]() {
            fence_proxy_async();  // generic-proxy shared-memory writes -> tensor pipe
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_epi);
        };
        // forward epilogue of layer l: A_{l+1} = relu(Z_l + b_l) -> BF16 -> dst (swizzled)
        auto fwd_pass = [&](int l, uint32_t dst) {
            const float4 *b4 = reinterpret_cast<const float4 *>(bias + l * H + 32 * cq);
            float v[32];
            tmem_ld32(tcol, v);
            tmem_ld_wait();
#pragma unroll
            for (int c4 = 0; c4 < 4; c4++) {
                const float4 lo = b4[2 * c4], hi = b4[2 * c4 + 1];
                const float bb[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
                const float *vv = v + 8 * c4;
                st_shared_v4(dst + blk + sw_off(m, c0 + c4), pack_bf16(fmaxf(vv[0] + bb[0], 0.f), fmaxf(vv[1] + bb[1], 0.f)),
                             pack_bf16(fmaxf(vv[2] + bb[2], 0.f), fmaxf(vv[3] + bb[3], 0.f)),
                             pack_bf16(fmaxf(vv[4] + bb[4], 0.f), fmaxf(vv[5] + bb[5], 0.f)),
                             pack_bf16(fmaxf(vv[6] + bb[6], 0.f), fmaxf(vv[7] + bb[7], 0.f)));
            }
        };
        // input rows of a tile: column quarters 0 and 1 hold columns 8 cq .. 8 cq + 7
        float xr[8];
        bool xbad = false;  // a non-finite input coordinate in this thread's part of the row
        auto x_load = [&](long long tile) {
            const long long row = tile * TM + m;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int kk = 8 * cq + k;
                xr[k] = (cq < 2 && tile < ntiles && row < n && kk < d.in) ? __ldg(q + row * d.in + kk) : 0.f;
            }
            // input column 15 is constant 1 (its weights are 0): the dW_0 product's column 15
            // is then the sum of dZ_0 over the tile's rows, the first layer's bias gradient
            if (cq == 1) xr[7] = 1.f;
        };
        x_load(blockIdx.x);
        bool first = true;
#pragma unroll 1
        for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const long long row = tile * TM + m;
            const bool valid = row < n;
            // (the previous tile's dW_0 product, the last reader of X, has completed)
            if (cq < 2)
                st_shared_v4(sXu + cm_off(m, cq), pack_bf16(xr[0], xr[1]), pack_bf16(xr[2], xr[3]),
                             pack_bf16(xr[4], xr[5]), pack_bf16(xr[6], xr[7]));
            xbad = false;
#pragma unroll
            for (int k = 0; k < 8; k++) xbad = xbad || !isfinite(xr[k]);
            arrive();
            x_load(tile + gridDim.x);  // prefetch the next tile's input
#pragma unroll 1
            for (int l = 0; l < NH - 1; l++) {
                if (!mma_wait()) break;
                fwd_pass(l, bufA(l + 1));
                arrive();
            }
            if (!ok || !mma_wait()) break;
            // ---- head (FP32), loss, dL/dz, dZ_{NH-1}, head and bias gradients
            {
                const float *b = bias + (NH - 1) * H + 32 * cq;
                const float *hw = head + 32 * cq;
                float zp = 0.f;
                {
                    float v[32];
                    tmem_ld32(tcol, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int e = 0; e < 32; e++) zp = fmaf(hw[e], fmaxf(v[e] + b[e], 0.f), zp);
                }
                // a non-finite input coordinate makes the logit non-finite (as in the exact
                // network), whatever the ReLUs made of it
                if (xbad) zp = __int_as_float(0x7fc00000);
                // the four warps of a lane quarter add their parts of the head sum, all in
                // the same order
                zpart[(qd * 4 + cq) * 32 + lane] = zp;
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_quad);
                ok = warp_wait(bar_quad, pq, ctl, err);
                pq ^= 1;
                if (!ok) break;
                const float *zq = zpart + qd * 128 + lane;
                const float z = ((zq[0] + zq[32]) + (zq[64] + zq[96])) + head[H];
                float g = 0.f;
                const bool fin = isfinite(z);
                if (valid) {
                    const float y = (float)((labels[row >> 5] >> (row & 31)) & 1u);
                    if (fin) {
                        const float sg = sigmoidf(z);
                        g = (alpha * y * (sg - 1.f) + beta * (1.f - y) * sg) * inv_n;
                        if (cq == 0) {
                            lossacc += alpha * y * softplusf(-z) + beta * (1.f - y) * softplusf(z);
                            const bool dec = z >= tau.up;
                            c_fn += (y != 0.f && !dec);
                            c_fp += (y == 0.f && dec);
                        }
                    } else if (cq == 0) {
                        c_nf++;
                    }
                }
                if (cq == 0) gsum += g;
                if (!fin) {
                    // a sample with a non-finite logit adds nothing: clear its rows so that no
                    // inf or NaN meets a zero gradient in the weight products
                    if (cq < 2) st_shared_v4(sXu + cm_off(m, cq), 0u, 0u, 0u, 0u);
                    for (int l = 1; l < NH; l++)
                        for (int c4 = 0; c4 < 4; c4++) st_shared_v4(bufA(l) + blk + sw_off(m, c0 + c4), 0u, 0u, 0u, 0u);
                }
                // dZ_{NH-1} (and its bias-gradient sums), then the head-weight gradient terms,
                // each from a fresh read of the accumulator (fewer live registers)
                {
                    float v[32];
                    tmem_ld32(tcol, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int e = 0; e < 32; e++) v[e] = (v[e] + b[e]) > 0.f ? g * hw[e] : 0.f;
#pragma unroll
                    for (int c4 = 0; c4 < 4; c4++) {
                        const float *zz = v + 8 * c4;
                        st_shared_v4(ZB + blk + sw_off(m, c0 + c4), pack_bf16(zz[0], zz[1]), pack_bf16(zz[2], zz[3]),
                                     pack_bf16(zz[4], zz[5]), pack_bf16(zz[6], zz[7]));
                    }
                    dbl[(NH - 1) * H] += xsum32(v, lane);
                }
                {
                    float v[32];
                    tmem_ld32(tcol, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int e = 0; e < 32; e++) v[e] = fin ? g * fmaxf(v[e] + b[e], 0.f) : 0.f;
                    dbl[NH * H] += xsum32(v, lane);
                }
                arrive();
            }
            // ---- backward through the hidden layers
#pragma unroll 1
            for (int l = NH - 1; l >= 1; l--) {
                if (RECOMP && l == 1) {
                    if (!mma_wait()) break;
                    fwd_pass(0, bufA(1));
                    arrive();
                }
                if (!ok || !mma_wait()) break;
                // dZ_{l-1} = dA_l masked by A_l > 0, written over A_l
                const uint32_t buf = bufA(l) + blk;
                float v[32];
                tmem_ld32(tcol, v);
                tmem_ld_wait();
#pragma unroll
                for (int c4 = 0; c4 < 4; c4++) {
                    const uint32_t addr = buf + sw_off(m, c0 + c4);
                    const uint4 mk = ld_shared_v4(addr);
                    float *vv = v + 8 * c4;
                    // A_l = +-0: inactive
                    if ((mk.x & 0x7fffu) == 0u) vv[0] = 0.f;
                    if ((mk.x & 0x7fff0000u) == 0u) vv[1] = 0.f;
                    if ((mk.y & 0x7fffu) == 0u) vv[2] = 0.f;
                    if ((mk.y & 0x7fff0000u) == 0u) vv[3] = 0.f;
                    if ((mk.z & 0x7fffu) == 0u) vv[4] = 0.f;
                    if ((mk.z & 0x7fff0000u) == 0u) vv[5] = 0.f;
                    if ((mk.w & 0x7fffu) == 0u) vv[6] = 0.f;
                    if ((mk.w & 0x7fff0000u) == 0u) vv[7] = 0.f;
                    st_shared_v4(addr, pack_bf16(vv[0], vv[1]), pack_bf16(vv[2], vv[3]), pack_bf16(vv[4], vv[5]),
                                 pack_bf16(vv[6], vv[7]));
                }
                if (l > 1) dbl[(l - 1) * H] += xsum32(v, lane);  // b_0's sums come from dW_0
                arrive();
            }
            if (!ok || !mma_wait()) break;
            // ---- dW_0 of this tile (scratch columns 8 cq .. 8 cq + 7 of lane = neuron m)
            if (cq < 2) {
                float v[8];
                tmem_ld8(trow + 8 * cq, v);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 8; i++) dw0acc[i] += v[i];
            }
            tc_fence_before();
            first = false;
        }
        // ---- the CTA's gradient partial (every element written once)
        float *slot = partial + (size_t)blockIdx.x * stride;
        if (ok) {
            // hidden-to-hidden weight gradients from tensor memory: row m, columns 32 cq ..
#pragma unroll 1
            for (int l = 1; l < NH; l++) {
                float *dst = slot + d.off[l] + (size_t)m * H + 32 * cq;
                float v[32];
                tmem_ld32(trow + (uint32_t)(128 * l) + 32 * cq, v);
                tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 32; e += 4)
                    *reinterpret_cast<float4 *>(dst + e) =
                        first ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
            }
            // first layer: row m, columns 8 cq .. (the real input columns), and its bias
            // gradient from the constant column 15
            if (cq < 2)
                for (int i = 0; i < 8; i++) {
                    const int k = 8 * cq + i;
                    if (k < d.in) slot[d.off[0] + (size_t)m * d.in + k] = dw0acc[i];
                }
            if (cq == 1) slot[d.off[0] + (size_t)H * d.in + m] = dw0acc[7];
        }
        tc_fence_before();
        // bias, head and loss sums: each lane quarter's sums, combined in a fixed order
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            lossacc += __shfl_xor_sync(FULL, lossacc, o);
            gsum += __shfl_xor_sync(FULL, gsum, o);
        }
        if (cq == 0 && lane == 0) {
            red2[qd * 2] = lossacc;
            red2[qd * 2 + 1] = gsum;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(NEPI * 32) : "memory");
        if (ok) {
            for (int i = H + threadIdx.x; i < (NH + 1) * H; i += NEPI * 32) {  // b_1 .. b_{NH-1}, head
                const int l = i / H;
                const float *dq = dbs + i;
                const float s = ((dq[0] + dq[(NH + 1) * H]) + dq[2 * (NH + 1) * H]) + dq[3 * (NH + 1) * H];
                if (l < NH)
                    slot[d.off[l] + (size_t)H * H + (i % H)] = s;  // b_l
                else
                    slot[d.off[NH] + (i % H)] = s;  // head weights
            }
            if (threadIdx.x == 0) {
                slot[d.off[NH] + H] = ((red2[1] + red2[3]) + red2[5]) + red2[7];  // head bias
                loss_partial[blockIdx.x] = ((red2[0] + red2[2]) + red2[4]) + red2[6];
            }
        }
        if (st && cq == 0) {
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                c_fn += __shfl_xor_sync(FULL, c_fn, o);
                c_fp += __shfl_xor_sync(FULL, c_fp, o);
                c_nf += __shfl_xor_sync(FULL, c_nf, o);
            }
            if (lane == 0) {
                if (c_fn) atomicAdd(&st->fn, c_fn);
                if (c_fp) atomicAdd(&st->fp, c_fp);
                if (c_nf) atomicAdd(&st->n_nonfinite, c_nf);
            }
        }
    }
    __syncthreads();
    if (warp == NEPI) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// FP32 master weights -> the training image: W_0 as 8 x 16-byte core matrices (core
// (n / 8, k / 8) at (n / 8) 256 + (k / 8) 128, row n mod 8 at 16 B), then each hidden
// layer as two 64-column blocks of 128 rows, 128-byte swizzled.  One thread per 16 bytes.
__global__ void pack_train_tc_kernel(TTDesc d, uint8_t *img) {
    const uint32_t nchunks = d.img_bytes / 16;
    for (uint32_t ch = blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks; ch += gridDim.x * blockDim.x) {
        const uint32_t byte = ch * 16;
        int l, n, k0;
        if (byte < W0_BYTES) {
            l = 0;
            n = (int)(byte / 256) * 8 + (int)((byte % 128) / 16);
            k0 = (int)((byte % 256) / 128) * 8;
        } else {
            const uint32_t rel = byte - W0_BYTES;
            l = 1 + (int)(rel / WL_BYTES);
            const uint32_t in_l = rel % WL_BYTES, blk = in_l / BLK, rem = in_l % BLK;
            n = (int)(rem / 128);
            const int c = (int)((rem % 128) / 16) ^ (n & 7);
            k0 = (int)blk * 64 + c * 8;
        }
        const int K = l == 0 ? d.in : H;
        const float *W = d.p + d.off[l] + (size_t)n * K;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; e++) v[e] = (k0 + e < K) ? W[k0 + e] : 0.f;
        *reinterpret_cast<uint4 *>(img + byte) =
            make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    }
}

TTDesc make_desc(const TcModel *tc, const MlpDesc &d) {
    TTDesc t{};
    t.in = d.w[0];
    t.NH = d.L - 1;
    t.img = (const uint8_t *)tc->train_img;
    t.img_bytes = W0_BYTES + (uint32_t)(t.NH - 1) * WL_BYTES;
    t.p = d.p;
    for (int l = 0; l < d.L; l++) t.off[l] = d.off[l];
    return t;
}

size_t smem_bytes(int NH, bool recompute) {
    const size_t img = W0_BYTES + (size_t)(NH - 1) * WL_BYTES;
    const size_t acts = W0_BYTES + (size_t)(NH - 1 + (recompute ? 0 : 1)) * WL_BYTES;
    return 2048 + img + acts + (size_t)(NH * H + 132 + 512 + 4 * (NH + 1) * H + 8) * sizeof(float);
}

int num_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

bool nb_train_tc_supported(const MlpDesc &d) {
    const int NH = d.L - 1;
    if (NH < 2 || NH > 4 || d.w[0] > 15 || d.w[0] < 1) return false;  // column 15 is the constant 1
    for (int l = 1; l < d.L; l++)
        if (d.w[l] != H) return false;
    int dev = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return smem_bytes(NH, NH == 4) <= (size_t)maxsm;
}

// tiles balanced over the CTAs: every CTA gets ceil(tiles / SMs) or one fewer
int nb_train_tc_ctas(int64_t n) {
    const int64_t tiles = (n + TM - 1) / TM;
    const int64_t sms = num_sms();
    const int64_t per = (tiles + sms - 1) / sms;
    int64_t g = (tiles + per - 1) / per;
    return (int)(g < 1 ? 1 : g);
}

nb_status nb_train_tc_refresh(TcModel *tc, const MlpDesc &d, cudaStream_t s) {
    const TTDesc t = make_desc(tc, d);
    const uint32_t nchunks = t.img_bytes / 16;
    pack_train_tc_kernel<<<(nchunks + 255) / 256, 256, 0, s>>>(t, (uint8_t *)tc->train_img);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_launch_train_tc(TcModel *tc, const MlpDesc &d, const float *q, const uint32_t *labels, int64_t n,
                             float alpha, float beta, TauF tau, TrainWs ws, nb_step_stats *st, cudaStream_t s) {
    const TTDesc t = make_desc(tc, d);
    long long P = 0;
    for (int l = 0; l < d.L; l++) P += (long long)d.w[l + 1] * (d.w[l] + 1);
    const long long stride = ws.stride > 0 ? ws.stride : P;
    if (st) NB_CUDA(cudaMemsetAsync(st, 0, sizeof(nb_step_stats), s));
    const size_t smem = smem_bytes(t.NH, t.NH == 4);
#define NB_TT(NHV)                                                                                                 \
    do {                                                                                                           \
        NB_CUDA(cudaFuncSetAttribute(train_tc_kernel<NHV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        train_tc_kernel<NHV><<<ws.G, THREADS, smem, s>>>(t, q, labels, (long long)n, alpha, beta, 1.0f / (float)n,   \
                                                         tau, ws.partial, ws.loss_partial, stride, st, tc->err);   \
    } while (0)
    if (t.NH == 2) NB_TT(2);
    else if (t.NH == 3) NB_TT(3);
    else NB_TT(4);
#undef NB_TT
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}
