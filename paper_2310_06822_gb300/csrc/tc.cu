// Tensor-core forward of the bounding network h (Sec. 3.4 "Architecture") on sm_103a:
// tcgen05.mma (BF16 x BF16 -> FP32 accumulators in TMEM), weights staged once per CTA
// into shared memory by the bulk-copy (TMA) engine, activations kept on chip.
//
// Persistent CTA of 9 warps:
//   warps 0-3  epilogue group for tile slot 0, warps 4-7 for slot 1: one thread per
//              query row (= TMEM lane).  Each group loads its tile's queries, and after
//              every layer reads the accumulator from TMEM, adds the bias, applies ReLU,
//              rounds to BF16 and writes the next layer's A operand to shared memory;
//              after the last hidden layer it evaluates the 1-wide head in FP32 and
//              writes the decision bit, the logit and the margin flag.
//   warp 8     allocates TMEM, loads the weights, and (one lane) issues the MMAs.
// The two slots ping-pong: while one slot's epilogue runs, the other slot's MMAs run.
// All waits are bounded; a wait that gives up sets an error word and every warp exits
// through the common tail, which drains the tensor pipe and frees TMEM.
#include <cuda_bf16.h>

#include "tc.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace nbtc;

constexpr int TILE_M = 128;
constexpr int NEPI = 8;                    // epilogue warps
constexpr int THREADS = (NEPI + 1) * 32;   // + the MMA / TMEM warp
constexpr unsigned SPIN_LIMIT = 1u << 22;
constexpr unsigned FULL = 0xffffffffu;
constexpr int A_BLOCK = TILE_M * 128;      // one 64-column block of a 128-row operand

struct TcDesc {
    int in, H, NH;          // input width (<= 16), hidden width, hidden layers
    const uint8_t *img;     // packed BF16 operand images, see img_layer_offset
    uint32_t img_bytes;
    const float *p;         // FP32 master parameters (biases and head read from here)
    int off[NB_MAXL];
};

// image of layer l: layer 0 is H rows x 128 B (K padded to 16 within one 64-column
// block); layer l >= 1 is H/64 blocks of H rows x 128 B.
__host__ __device__ inline uint32_t img_layer_offset(int H, int l) {
    return l == 0 ? 0u : (uint32_t)(H * 128 + (l - 1) * H * H * 2);
}
__host__ __device__ inline uint32_t img_total(int H, int NH) { return img_layer_offset(H, NH); }

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

struct Ctl {
    uint64_t wbar, aready[2], accfull[2], drain;
    uint32_t tmem;
    int abort;
};

__device__ bool wait_bounded(uint32_t bar, uint32_t parity, Ctl *ctl, int *err, unsigned limit = SPIN_LIMIT) {
    for (unsigned i = 0; i < limit; i++) {
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

template <int H>
__global__ void __launch_bounds__(THREADS, 1)
    fwd_bf16_kernel(TcDesc d, const float *__restrict__ q, long long n, TauF tau, float margin,
                    uint32_t *__restrict__ bits, float *__restrict__ logits, nb_query_stats *st,
                    unsigned *flag_count, unsigned *flag_idx, int *err) {
    extern __shared__ uint8_t smem_raw[];
    Ctl *ctl = reinterpret_cast<Ctl *>(smem_raw);
    uint8_t *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023) + 1024;
    uint8_t *Wimg = base;
    uint8_t *Abuf = Wimg + d.img_bytes;
    float *bias = reinterpret_cast<float *>(Abuf + 2 * (H / 64) * A_BLOCK);
    float *head = bias + d.NH * H;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long ntiles = (n + TILE_M - 1) / TILE_M;
    const uint32_t bar_w = smem_u32(&ctl->wbar), bar_drain = smem_u32(&ctl->drain);
    const uint32_t bar_ar[2] = {smem_u32(&ctl->aready[0]), smem_u32(&ctl->aready[1])};
    const uint32_t bar_af[2] = {smem_u32(&ctl->accfull[0]), smem_u32(&ctl->accfull[1])};

    if (threadIdx.x == 0) {
        mbar_init(bar_w, 1);
        mbar_init(bar_ar[0], 4);
        mbar_init(bar_ar[1], 4);
        mbar_init(bar_af[0], 1);
        mbar_init(bar_af[1], 1);
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
        tmem_alloc(smem_u32(&ctl->tmem), 2 * H);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem;

    if (warp == NEPI) {
        if (lane == 0) {
            bool ok = true;
            mbar_expect_tx(bar_w, d.img_bytes);
            for (uint32_t o = 0; o < d.img_bytes; o += 16384)
                bulk_g2s(smem_u32(Wimg) + o, d.img + o, min(16384u, d.img_bytes - o), bar_w);
            ok = wait_bounded(bar_w, 0, ctl, err);
            uint32_t ph[2] = {0, 0};
            constexpr uint32_t idesc = idesc_bf16(TILE_M, H);
            for (long long it = 0; ok; it++) {
                const bool has[2] = {blockIdx.x + (2 * it) * gridDim.x < ntiles,
                                     blockIdx.x + (2 * it + 1) * gridDim.x < ntiles};
                if (!has[0] && !has[1]) break;
                for (int l = 0; l < d.NH && ok; l++)
                    for (int s = 0; s < 2 && ok; s++) {
                        if (!has[s]) continue;
                        ok = wait_bounded(bar_ar[s], ph[s], ctl, err);
                        ph[s] ^= 1;
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(Abuf + s * (H / 64) * A_BLOCK);
                        const uint32_t w0 = smem_u32(Wimg) + img_layer_offset(H, l);
                        const int ksteps = l == 0 ? 1 : H / 16;
                        for (int j = 0; j < ksteps; j++) {
                            const uint32_t kb = j >> 2, within = (j & 3) * 32;
                            mma_f16(tmem + s * H, sdesc_sw128(a0 + kb * A_BLOCK + within),
                                    sdesc_sw128(w0 + kb * (H * 128) + within), idesc, j > 0 ? 1u : 0u);
                        }
                        mma_commit(bar_af[s]);
                    }
            }
            // every issued MMA has completed before TMEM is released
            mma_commit(bar_drain);
            wait_bounded(bar_drain, 0, ctl, err);
            if (!ok) {
                *(volatile int *)&ctl->abort = 1;
            }
        }
        __syncwarp();
    } else {
        const int s = warp >> 2, wq = warp & 3;
        const int r = wq * 32 + lane;  // row of the tile = TMEM lane
        const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(s * H);
        const uint32_t A = smem_u32(Abuf + s * (H / 64) * A_BLOCK);
        const uint32_t row_off = (uint32_t)r * 128, sw = (uint32_t)(r & 7);
        uint32_t ph = 0;
        unsigned long long c_in = 0, c_flag = 0, c_nf = 0;
        for (long long it = 0;; it++) {
            const long long tile = blockIdx.x + (2 * it + s) * gridDim.x;
            if (tile >= ntiles) break;
            const long long row = tile * TILE_M + r;
            const bool valid = row < n;
            bool xbad = false;  // a non-finite input coordinate: the logit is made NaN
            {
                float x[16];
#pragma unroll
                for (int k = 0; k < 16; k++) {
                    x[k] = (valid && k < d.in) ? __ldg(q + row * d.in + k) : 0.f;
                    xbad = xbad || !isfinite(x[k]);
                }
                st_shared_v4(A + row_off + ((0u ^ sw) << 4), pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]),
                             pack_bf16(x[4], x[5]), pack_bf16(x[6], x[7]));
                st_shared_v4(A + row_off + ((1u ^ sw) << 4), pack_bf16(x[8], x[9]), pack_bf16(x[10], x[11]),
                             pack_bf16(x[12], x[13]), pack_bf16(x[14], x[15]));
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_ar[s]);
            bool ok = true;
            float z = 0.f;
            for (int l = 0; l < d.NH; l++) {
                ok = warp_wait(bar_af[s], ph, ctl, err);
                ph ^= 1;
                if (!ok) break;
                tc_fence_after();
                const float *b = bias + l * H;
                if (l < d.NH - 1) {
#pragma unroll
                    for (int qc = 0; qc < H / 32; qc++) {
                        float v[32];
                        tmem_ld32(taddr + qc * 32, v);
                        tmem_ld_wait();
#pragma unroll
                        for (int c4 = 0; c4 < 4; c4++) {
                            const int col = qc * 32 + c4 * 8;
                            const uint32_t kb = col >> 6, c = (col & 63) >> 3;
                            const float *bb = b + col;
                            const float *vv = v + c4 * 8;
                            st_shared_v4(A + kb * A_BLOCK + row_off + ((c ^ sw) << 4),
                                         pack_bf16_relu(vv[0] + bb[0], vv[1] + bb[1]),
                                         pack_bf16_relu(vv[2] + bb[2], vv[3] + bb[3]),
                                         pack_bf16_relu(vv[4] + bb[4], vv[5] + bb[5]),
                                         pack_bf16_relu(vv[6] + bb[6], vv[7] + bb[7]));
                        }
                    }
                    tc_fence_before();
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar_ar[s]);
                } else {
                    // 1-wide head in FP32: z = b_L + sum_n w_n relu(acc_n + b_n)
#pragma unroll
                    for (int qc = 0; qc < H / 32; qc++) {
                        float v[32];
                        tmem_ld32(taddr + qc * 32, v);
                        tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 32; e++)
                            z = fmaf(head[qc * 32 + e], fmaxf(v[e] + b[qc * 32 + e], 0.f), z);
                    }
                    tc_fence_before();
                    z += head[H];
                }
            }
            if (!ok) break;
            if (xbad) z = __int_as_float(0x7fc00000);
            const bool fin = isfinite(z);
            const bool inside = valid && (!fin || z >= tau.up);
            const bool flag = valid && fin && (fabsf(z - tau.up) < margin || (z >= tau.dn && z < tau.up));
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
        tmem_dealloc(tmem, 2 * H);
    }
}

// FP32 master weights -> BF16 operand images (one thread per 16-byte chunk)
__global__ void pack_bf16_kernel(TcDesc d, uint8_t *img) {
    const int H = d.H;
    const uint32_t nchunks = d.img_bytes / 16;
    for (uint32_t ch = blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks; ch += gridDim.x * blockDim.x) {
        const uint32_t byte = ch * 16;
        int l;
        uint32_t local;
        if (byte < (uint32_t)(H * 128)) {
            l = 0;
            local = byte;
        } else {
            l = 1 + (int)((byte - H * 128) / (uint32_t)(H * H * 2));
            local = (byte - H * 128) % (uint32_t)(H * H * 2);
        }
        const int K = l == 0 ? d.in : H;
        const uint32_t kb = local / (uint32_t)(H * 128), rem = local % (uint32_t)(H * 128);
        const uint32_t nrow = rem / 128, pc = (rem % 128) / 16, c = pc ^ (nrow & 7);
        const int k0 = (int)(kb * 64 + c * 8);
        const float *W = d.p + d.off[l] + (size_t)nrow * K;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; e++) v[e] = (k0 + e < K) ? W[k0 + e] : 0.f;
        uint4 o;
        o.x = pack_bf16(v[0], v[1]);
        o.y = pack_bf16(v[2], v[3]);
        o.z = pack_bf16(v[4], v[5]);
        o.w = pack_bf16(v[6], v[7]);
        *reinterpret_cast<uint4 *>(img + byte) = o;
    }
}

TcDesc make_desc(const TcModel *tc, const MlpDesc &d) {
    TcDesc t{};
    t.in = d.w[0];
    t.H = d.w[1];
    t.NH = d.L - 1;
    t.img = (const uint8_t *)tc->img;
    t.img_bytes = (uint32_t)tc->img_bytes;
    t.p = d.p;
    for (int l = 0; l < d.L; l++) t.off[l] = d.off[l];
    return t;
}

size_t fwd_smem_bytes(int H, int NH) {
    return 2048 + img_total(H, NH) + 2 * (size_t)(H / 64) * A_BLOCK + (size_t)(NH * H + H + 4) * sizeof(float);
}

int num_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

namespace {
// real parameters -> zero-padded layout (blockIdx.y = layer); positions past the real
// widths are never written and keep the zeros of the allocation
__global__ void pad_params_kernel(MlpDesc real, MlpDesc pad, float *out) {
    const int l = blockIdx.y;
    const int N = real.w[l + 1], K = real.w[l], Kp = pad.w[l];
    const long long total = (long long)N * K + N;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const float v = real.p[real.off[l] + e];
        if (e < (long long)N * K) {
            const long long n = e / K, k = e % K;
            out[pad.off[l] + n * Kp + k] = v;
        } else {
            out[pad.off[l] + (long long)pad.w[l + 1] * Kp + (e - (long long)N * K)] = v;
        }
    }
}
}  // namespace

// the parameter layout the tensor-core forward reads: the model's own, or its padded copy
static const MlpDesc &fwd_desc(const TcModel *tc, const MlpDesc &d) { return tc->pad_p ? tc->pad : d; }

nb_status nb_tc_init(TcModel *tc, const MlpDesc &d, int infer_prec, int train_prec) {
    tc->infer_prec = infer_prec;
    tc->train_prec = train_prec;
    int H = d.w[1];
    const int NH = d.L - 1;
    if (cudaMalloc(&tc->err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return nb_fail(NB_ENOMEM, "tensor-core state allocation failed");
    }
    cudaMemset(tc->err, 0, sizeof(int));
    if (infer_prec == NB_FP8) {
        const int NHH = d.L - 2;
        if (NHH < 1) return nb_fail(NB_EUNSUPPORTED, "FP8 forward needs at least two hidden layers");
        if (d.w[0] > 16) return nb_fail(NB_EUNSUPPORTED, "FP8 forward: input width must be <= 16");
        if (H != 128 && H != 256) return nb_fail(NB_EUNSUPPORTED, "FP8 forward: hidden width must be 128 or 256");
        for (int l = 1; l < d.L; l++)
            if (d.w[l] != H) return nb_fail(NB_EUNSUPPORTED, "FP8 forward: hidden widths must be equal");
        int dev = 0, maxsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (nb_fp8_smem_bytes(H, NHH) > (size_t)maxsm)
            return nb_fail(NB_EUNSUPPORTED, "FP8 forward: the network's weights do not fit in shared memory");
        tc->img_bytes = nb_fp8_img_bytes(H, NHH);
        if (cudaMalloc(&tc->img, tc->img_bytes) != cudaSuccess ||
            cudaMalloc(&tc->scales, sizeof(float) * (2 * NHH * H + H + 1)) != cudaSuccess) {
            cudaGetLastError();
            return nb_fail(NB_ENOMEM, "tensor-core image allocation failed");
        }
        cudaMemset(tc->img, 0, tc->img_bytes);
        cudaMemset(tc->scales, 0, sizeof(float) * (2 * NHH * H + H + 1));
    }
    if (infer_prec == NB_BF16 || infer_prec == NB_F16X3) {
        if (NH < 1) return nb_fail(NB_EUNSUPPORTED, "tensor-core forward needs at least one hidden layer");
        if (d.w[0] > 16) return nb_fail(NB_EUNSUPPORTED, "tensor-core forward: input width must be <= 16");
        for (int l = 1; l < d.L; l++)
            if (d.w[l] != H) return nb_fail(NB_EUNSUPPORTED, "tensor-core forward: hidden widths must be equal");
        if (H > 128) return nb_fail(NB_EUNSUPPORTED, "tensor-core forward: hidden width must be at most 128");
        if (H != 64 && H != 128) {  // run on a zero-padded copy
            MlpDesc pd = d;
            H = H < 64 ? 64 : 128;
            int off = 0;
            for (int l = 0; l < d.L; l++) {
                pd.w[l + 1] = l + 1 < d.L ? H : 1;
                pd.off[l] = off;
                off += pd.w[l + 1] * pd.w[l] + pd.w[l + 1];
            }
            pd.maxw = std::max(d.w[0], H);
            pd.pT = nullptr;
            if (cudaMalloc(&tc->pad_p, sizeof(float) * (size_t)off) != cudaSuccess) {
                cudaGetLastError();
                return nb_fail(NB_ENOMEM, "padded parameter allocation failed");
            }
            cudaMemset(tc->pad_p, 0, sizeof(float) * (size_t)off);
            pd.p = tc->pad_p;
            tc->pad = pd;
        }
        int dev = 0, maxsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t need = infer_prec == NB_BF16 ? fwd_smem_bytes(H, NH) : nb_split_smem_bytes(H, NH);
        if (need > (size_t)maxsm)
            return nb_fail(NB_EUNSUPPORTED, "tensor-core forward: the network's weights do not fit in shared memory");
        tc->img_bytes = infer_prec == NB_BF16 ? img_total(H, NH) : nb_split_img_bytes(H, NH);
        if (cudaMalloc(&tc->img, tc->img_bytes) != cudaSuccess) {
            cudaGetLastError();
            return nb_fail(NB_ENOMEM, "tensor-core image allocation failed");
        }
        cudaMemset(tc->img, 0, tc->img_bytes);
    }
    if (train_prec == NB_BF16) {
        const nb_status st = nb_train_bf16_check(d);
        if (st != NB_OK) return st;
        tc->train_tc = nb_train_tc_supported(d) ? 1 : 0;  // same image size in either layout
        tc->train_img_bytes = nb_train_bf16_img_bytes(d);
        if (cudaMalloc(&tc->train_img, tc->train_img_bytes) != cudaSuccess) {
            cudaGetLastError();
            return nb_fail(NB_ENOMEM, "training image allocation failed");
        }
        cudaMemset(tc->train_img, 0, tc->train_img_bytes);
    }
    return NB_OK;
}

void nb_tc_free(TcModel *tc) {
    cudaFree(tc->pad_p);
    tc->pad_p = nullptr;
    cudaFree(tc->img);
    cudaFree(tc->err);
    cudaFree(tc->train_img);
    cudaFree(tc->scales);
    tc->scales = nullptr;
    tc->img = nullptr;
    tc->err = nullptr;
    tc->train_img = nullptr;
}

nb_status nb_tc_refresh(TcModel *tc, const MlpDesc &d, cudaStream_t s) {
    if (tc->train_img) {
        const nb_status st = tc->train_tc ? nb_train_tc_refresh(tc, d, s) : nb_train_bf16_refresh(tc, d, s);
        if (st != NB_OK) return st;
    }
    return nb_tc_refresh_query(tc, d, s);
}

nb_status nb_tc_refresh_query(TcModel *tc, const MlpDesc &d, cudaStream_t s) {
    if (!tc->img) return NB_OK;
    if (tc->pad_p) {
        pad_params_kernel<<<dim3(32, d.L), 256, 0, s>>>(d, tc->pad, tc->pad_p);
        NB_CUDA(cudaGetLastError());
    }
    const MlpDesc &e = fwd_desc(tc, d);
    if (tc->infer_prec == NB_F16X3) return nb_split_refresh(tc, e, s);
    if (tc->infer_prec == NB_FP8) return nb_fp8_refresh(tc, e, s);
    const TcDesc t = make_desc(tc, e);
    const uint32_t nchunks = t.img_bytes / 16;
    pack_bf16_kernel<<<(nchunks + 255) / 256, 256, 0, s>>>(t, (uint8_t *)tc->img);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_tc_query(TcModel *tc, const MlpDesc &d, const float *q, int64_t n, TauF tau, float margin,
                      uint32_t *bits, float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s) {
    const MlpDesc &e = fwd_desc(tc, d);
    if (tc->infer_prec == NB_F16X3) return nb_split_query(tc, e, q, n, tau, margin, bits, logits, st, ws, s);
    if (tc->infer_prec == NB_FP8) return nb_fp8_query(tc, e, q, n, tau, margin, bits, logits, st, ws, s);
    const TcDesc t = make_desc(tc, e);
    const size_t smem = fwd_smem_bytes(t.H, t.NH);
    const int64_t tiles = (n + TILE_M - 1) / TILE_M;
    int64_t grid = num_sms();
    if (grid > (tiles + 1) / 2) grid = (tiles + 1) / 2;
    if (grid < 1) grid = 1;
    if (t.H == 128) {
        NB_CUDA(cudaFuncSetAttribute(fwd_bf16_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        fwd_bf16_kernel<128><<<(unsigned)grid, THREADS, smem, s>>>(t, q, (long long)n, tau, margin, bits, logits, st,
                                                                   ws.flag_count, ws.flag_idx, tc->err);
    } else {
        NB_CUDA(cudaFuncSetAttribute(fwd_bf16_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        fwd_bf16_kernel<64><<<(unsigned)grid, THREADS, smem, s>>>(t, q, (long long)n, tau, margin, bits, logits, st,
                                                                  ws.flag_count, ws.flag_idx, tc->err);
    }
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

namespace {
// A wait that nothing completes: one thread waits on an mbarrier no one arrives at, with
// the bounded wait of the forward kernels, gives up after `polls` polls and records
// NB_ETIMEOUT, and the kernel returns.
__global__ void selftest_wait_kernel(unsigned polls, int *err) {
    __shared__ Ctl ctl;
    const uint32_t bar = smem_u32(&ctl.wbar);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        ctl.abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) wait_bounded(bar, 0, &ctl, err, polls);
}
}  // namespace

extern "C" nb_status nb_selftest_bounded_wait(int32_t polls, void *stream) {
    if (polls < 1 || polls > (1 << 20)) return nb_fail(NB_EINVAL, "nb_selftest_bounded_wait: polls must be 1..2^20");
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return nb_fail(NB_ENOMEM, "nb_selftest_bounded_wait: allocation failed");
    }
    cudaStream_t s = (cudaStream_t)stream;
    int e = 0;
    cudaError_t ce = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (ce == cudaSuccess) {
        selftest_wait_kernel<<<1, 32, 0, s>>>((unsigned)polls, err);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFree(err);
    if (ce != cudaSuccess) return nb_fail(NB_ECUDA, cudaGetErrorString(ce));
    if (e) return nb_fail((nb_status)e, "bounded device wait gave up (expected)");
    return NB_OK;
}

nb_status nb_tc_check(TcModel *tc) {
    if (!tc->err) return NB_OK;
    int e = 0;
    NB_CUDA(cudaMemcpy(&e, tc->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        cudaMemset(tc->err, 0, sizeof(int));
        return nb_fail((nb_status)e, "a tensor-core kernel gave up waiting (bounded wait expired)");
    }
    return NB_OK;
}
