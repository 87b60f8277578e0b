// BF16 tensor-core training step of the bounding network (Sec. 3.4 "Training"):
// forward, asymmetric BCE of Eq. (loss), backward and per-CTA gradient partials in one
// persistent kernel; the partials are then summed in CTA order and Adam updates the
// FP32 master weights (adam_kernel of the FP32 path).
//
// Every GEMM of the step runs on the tensor cores with BF16 operands and FP32
// accumulation (mma.sync m16n8k16): the forward Z = A W^T, the input gradient
// dA = dZ W and the weight gradient dW = dZ^T A, the last two contracting over the
// batch; ldmatrix(.trans) loads every operand in the orientation the MMA needs, so the
// activations of a tile are stored once, row-major, in shared memory.
// A CTA walks tiles of 64 samples; per tile it keeps the input and every hidden layer's
// activations (BF16) in shared memory for the backward pass, next to all layers' BF16
// weights.  The head (width 1), the loss and the bias gradients run in FP32.
// Weight-gradient partials go to the CTA's own slot with red.global.add (four adjacent
// columns per vector reduction where they are 16-byte aligned); each address has one
// owning thread per tile, so the slot's sums are in program order.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "group.cuh"
#include "tc.cuh"

namespace {

constexpr int TM = 64;           // samples per tile
constexpr int TPB = 512;         // threads of the resident-weight kernels: 16 warps
constexpr int NWARP = TPB / 32;
constexpr int K0 = 16;           // padded input width
constexpr int PAD = 8;           // row padding (elements) against ldmatrix bank conflicts
constexpr unsigned FULL = 0xffffffffu;

struct TrainDesc {
    int in, H, NH;
    const __nv_bfloat16 *img;    // per layer bf16 W[n][k], k padded to K0 (layer 0) or H
    const float *p;              // FP32 master parameters (biases and head)
    int off[NB_MAXL];
};

__host__ __device__ inline int kpad(int H, int l) { return l == 0 ? K0 : H; }
__host__ __device__ inline size_t img_off(int H, int l) {  // elements
    return l == 0 ? 0 : (size_t)H * K0 + (size_t)(l - 1) * H * H;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ void red_add(float *p, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
// p[0..3] += v0..v3 in one vector reduction (p 16-byte aligned)
__device__ __forceinline__ void red_add4(float *p, float v0, float v1, float v2, float v3) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v0), "f"(v1), "f"(v2), "f"(v3)
                 : "memory");
}
// every input coordinate of a sample is finite (BF16 keeps inf and NaN)
__device__ __forceinline__ bool row_finite(const __nv_bfloat16 *x, int in) {
    bool ok = true;
    for (int k = 0; k < in; k++) ok = ok && ((__bfloat16_as_ushort(x[k]) & 0x7f80u) != 0x7f80u);
    return ok;
}
__device__ __forceinline__ float softplusf(float u) { return u > 0.f ? u + log1pf(expf(-u)) : log1pf(expf(u)); }
__device__ __forceinline__ float sigmoidf(float u) {
    return u >= 0.f ? 1.f / (1.f + expf(-u)) : expf(u) / (1.f + expf(u));
}

// OUT[TM][N] = epilogue(X[TM][K] Y^T) with Y[N][K] row-major (forward, Y = W) or, with
// TRANS_Y, OUT = X Y with Y[K][N] (the input gradient, Y = W read transposed).
// Warps: 4 along the 64 rows x NWARP/4 along N.  RELU: out = relu(acc + bias) (forward);
// otherwise out = acc masked by mask[m][n] > 0 (backward through the ReLU).
template <int H, bool TRANS_Y, bool RELU>
__device__ __forceinline__ void tile_gemm(const __nv_bfloat16 *X, int xp, int K, const __nv_bfloat16 *Y, int yp,
                                          const float *bias, const __nv_bfloat16 *mask, int mp, __nv_bfloat16 *out,
                                          int op) {
    constexpr int NGN = NWARP / 4;        // warp groups along N
    constexpr int NT = H / (8 * NGN);     // n-tiles of 8 per warp (H / NGN columns)
    static_assert(NT % 2 == 0, "two n-tiles per B fragment load");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = (warp & 3) * 16, n0 = (warp >> 2) * (H / NGN);
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int mi = lane >> 3, r = lane & 7;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(smem_u32(X + (m0 + r + (mi & 1) * 8) * xp + k0 + (mi >> 1) * 8), a0, a1, a2, a3);
#pragma unroll
        for (int j = 0; j < NT; j += 2) {
            uint32_t b0, b1, b2, b3;
            if (!TRANS_Y) {
                // Y[n][k]: matrices (n0-7,k0-7) (n0-7,k8-15) (n8-15,k0-7) (n8-15,k8-15)
                ldsm_x4(smem_u32(Y + (n0 + 8 * j + r + (mi >> 1) * 8) * yp + k0 + (mi & 1) * 8), b0, b1, b2, b3);
            } else {
                // Y[k][n] read transposed: matrices (k0-7,n0-7) (k8-15,n0-7) (k0-7,n8-15) (k8-15,n8-15)
                ldsm_x4_t(smem_u32(Y + (k0 + r + (mi & 1) * 8) * yp + n0 + 8 * j + (mi >> 1) * 8), b0, b1, b2, b3);
            }
            mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
            mma_bf16(acc[j + 1], a0, a1, a2, a3, b2, b3);
        }
    }
    const int gr = lane >> 2, gc = (lane & 3) * 2;
#pragma unroll
    for (int j = 0; j < NT; j++) {
        const int nn = n0 + 8 * j + gc;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int m = m0 + gr + 8 * h;
            float v0 = acc[j][2 * h], v1 = acc[j][2 * h + 1];
            if (RELU) {
                v0 = fmaxf(v0 + bias[nn], 0.f);
                v1 = fmaxf(v1 + bias[nn + 1], 0.f);
            } else {
                const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + m * mp + nn);
                v0 = __low2float(mk) > 0.f ? v0 : 0.f;
                v1 = __high2float(mk) > 0.f ? v1 : 0.f;
            }
            *reinterpret_cast<uint32_t *>(out + m * op + nn) = pack2(v0, v1);
        }
    }
}

// slot[n][k] += sum_m DZ[m][n] A[m][k] for n < H, k < Kreal (weight gradient of one layer).
// Warps: n-blocks of 16 x column groups (as many as the columns allow in multiples of 8;
// warps beyond them sit out this layer).
template <int H>
__device__ __forceinline__ void tile_dw(const __nv_bfloat16 *DZ, int dp, const __nv_bfloat16 *A, int ap, int Kp,
                                        int Kreal, float *slotW) {
    constexpr int NB = H / 16, KG = NWARP / NB;  // n-blocks, column groups
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = (warp % NB) * 16, kg = warp / NB;
    const int kgs = max(1, min(KG, Kp / 8));  // column groups of this layer
    if (kg >= kgs) return;
    const int kw = Kp / kgs, kbeg = kg * kw;  // this warp's columns
    const int mi = lane >> 3, r = lane & 7;
    const int gr = lane >> 2, gc = (lane & 3) * 2;
    for (int kc = 0; kc < kw; kc += 64) {  // at most 64 columns (8 n8-tiles) of accumulators at a time
        const int cw = min(64, kw - kc);
        float acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
        for (int m0 = 0; m0 < TM; m0 += 16) {
            // A' = DZ^T (rows n, K' = m): matrices (n0-7,m0-7) (n8-15,m0-7) (n0-7,m8-15) (n8-15,m8-15)
            uint32_t a0, a1, a2, a3;
            ldsm_x4_t(smem_u32(DZ + (m0 + r + (mi >> 1) * 8) * dp + n0 + (mi & 1) * 8), a0, a1, a2, a3);
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                if (8 * j >= cw) break;
                const int k0 = kbeg + kc + 8 * j;
                // B' = A (K' = m, N' = k): matrices (m0-7,k0-7) (m8-15,k0-7) (m0-7,k8-15) (m8-15,k8-15)
                uint32_t b0, b1, b2, b3;
                ldsm_x4_t(smem_u32(A + (m0 + r + (mi & 1) * 8) * ap + k0 + (mi >> 1) * 8), b0, b1, b2, b3);
                mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
                if (8 * (j + 1) < cw) mma_bf16(acc[j + 1], a0, a1, a2, a3, b2, b3);
            }
        }
        // lanes 2i and 2i+1 hold columns k, k+1 and k+2, k+3 of rows gr and gr + 8: one
        // exchange gives the even lane four columns of row gr and the odd lane four of row
        // gr + 8, added with one vector reduction where the four are 16-byte aligned
        const bool odd = lane & 1;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            if (8 * j >= cw) break;
            const float s0 = odd ? acc[j][0] : acc[j][2], s1 = odd ? acc[j][1] : acc[j][3];
            const float r0 = __shfl_xor_sync(FULL, s0, 1), r1 = __shfl_xor_sync(FULL, s1, 1);
            const int k4 = kbeg + kc + 8 * j + (gc & ~2);  // first of the four columns
            const int nn = n0 + gr + (odd ? 8 : 0);
            float v[4];
            if (odd) {
                v[0] = r0; v[1] = r1; v[2] = acc[j][2]; v[3] = acc[j][3];
            } else {
                v[0] = acc[j][0]; v[1] = acc[j][1]; v[2] = r0; v[3] = r1;
            }
            float *dst = slotW + nn * Kreal + k4;
            if (k4 + 3 < Kreal && ((uintptr_t)dst & 15) == 0) {
                red_add4(dst, v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (k4 + u < Kreal) red_add(dst + u, v[u]);
            }
        }
    }
}

// shared-memory carve-up of the training kernels (see nb_train_bf16_smem)
#define NB_BF_SMEM                                                                                     \
    constexpr int HP = H + PAD, XP = K0 + PAD;                                                         \
    extern __shared__ __align__(16) uint8_t smem_raw[];                                                \
    const int NH = d.NH, t = threadIdx.x;                                                              \
    __nv_bfloat16 *Ws = reinterpret_cast<__nv_bfloat16 *>(smem_raw);                                   \
    __nv_bfloat16 *act = Ws + H * XP + (size_t)(NH - 1) * H * HP;                                      \
    __nv_bfloat16 *dz0 = act + TM * XP + (size_t)NH * TM * HP;                                         \
    __nv_bfloat16 *dz1 = dz0 + TM * HP;                                                                \
    float *bias = reinterpret_cast<float *>(dz1 + TM * HP);                                            \
    float *head = bias + NH * H;                                                                       \
    float *zs = head + H + 4, *gs = zs + TM, *ls = gs + TM;                                            \
    auto W_l = [&](int l) { return l == 0 ? Ws : Ws + H * XP + (size_t)(l - 1) * H * HP; };          \
    auto A_l = [&](int l) { return l == 0 ? act : act + TM * XP + (size_t)(l - 1) * TM * HP; };      \
    (void)HP;                                                                                          \
    (void)XP

// weights of one network (bf16 image -> padded rows), its biases and head; ends synchronised
template <int H>
__device__ __forceinline__ void bf_load(const TrainDesc &d, const __nv_bfloat16 *img, const float *p) {
    NB_BF_SMEM;
    (void)A_l;
    (void)zs;
    (void)gs;
    (void)ls;
    (void)dz0;
    // weights (bf16 image -> padded rows), biases, head
    for (int l = 0; l < NH; l++) {
        const int kp = kpad(H, l), pitch = l == 0 ? XP : HP;
        const __nv_bfloat16 *src = img + img_off(H, l);
        __nv_bfloat16 *dst = W_l(l);
        for (int e = t; e < H * kp / 8; e += blockDim.x) {
            const int row = (e * 8) / kp, col = (e * 8) % kp;
            *reinterpret_cast<uint4 *>(dst + row * pitch + col) = *reinterpret_cast<const uint4 *>(src + row * kp + col);
        }
    }
    for (int i = t; i < NH * H; i += blockDim.x) {
        const int l = i / H, j = i % H;
        bias[i] = p[d.off[l] + H * (l == 0 ? d.in : H) + j];
    }
    for (int i = t; i <= H; i += blockDim.x) head[i] = p[d.off[NH] + i];
    __syncthreads();

}

// one tile of TM samples starting at row base: forward, loss, backward, gradient partials
// into slot; ends synchronised
template <int H>
__device__ __forceinline__ void bf_tile(const TrainDesc &d, const float *__restrict__ q,
                                        const uint32_t *__restrict__ labels, long long base, int rows, float alpha,
                                        float beta, float inv_n, TauF tau, float *__restrict__ slot, float &lossacc,
                                        unsigned long long &c_fn, unsigned long long &c_fp, unsigned long long &c_nf) {
    NB_BF_SMEM;
    // input -> bf16, padded to K0
    for (int e = t; e < TM * K0; e += blockDim.x) {
        const int m = e / K0, k = e % K0;
        const float x = (m < rows && k < d.in) ? q[(base + m) * d.in + k] : 0.f;
        act[m * XP + k] = __float2bfloat16_rn(x);
    }
    __syncthreads();
    // forward
    for (int l = 0; l < NH; l++) {
        tile_gemm<H, false, true>(A_l(l), l == 0 ? XP : HP, kpad(H, l), W_l(l), l == 0 ? XP : HP, bias + l * H,
                                  nullptr, 0, A_l(l + 1), HP);
        __syncthreads();
    }
    // head (FP32) and loss: 4 threads per sample
    if (t < 4 * TM) {  // whole warps
        const __nv_bfloat16 *aL = A_l(NH);
        const int m = t >> 2, part = t & 3;
        float s = 0.f;
        for (int k = part; k < H; k += 4) s = fmaf(head[k], __bfloat162float(aL[m * HP + k]), s);
        s += __shfl_xor_sync(FULL, s, 1);
        s += __shfl_xor_sync(FULL, s, 2);
        if (part == 0) zs[m] = s + head[H];
    }
    __syncthreads();
    if (t < TM) {
        float g = 0.f, lv = 0.f;
        if (t < rows) {
            const long long i = base + t;
            const float y = (float)((labels[i >> 5] >> (i & 31)) & 1u);
            const float z = zs[t];
            if (isfinite(z) && row_finite(act + t * XP, d.in)) {
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
        gs[t] = g;
        ls[t] = lv;
        // a skipped sample must not meet its zero gradient with an inf or NaN activation
        if (t < rows && g == 0.f && !(isfinite(zs[t]) && row_finite(act + t * XP, d.in))) {
            for (int k = 0; k < K0; k++) act[t * XP + k] = __float2bfloat16_rn(0.f);
            for (int l = 1; l <= NH; l++)
                for (int k = 0; k < H; k++) A_l(l)[t * HP + k] = __float2bfloat16_rn(0.f);
        }
    }
    __syncthreads();
    if (t == 0)
        for (int m = 0; m < rows; m++) lossacc += ls[m];
    // head gradients and dZ of the last hidden layer
    {
        const __nv_bfloat16 *aL = A_l(NH);
        float *gW = slot + d.off[NH];
        for (int k = t; k <= H; k += blockDim.x) {
            float s = 0.f;
            if (k < H)
                for (int m = 0; m < TM; m++) s = fmaf(gs[m], __bfloat162float(aL[m * HP + k]), s);
            else
                for (int m = 0; m < TM; m++) s += gs[m];
            gW[k] += s;
        }
        for (int e = t; e < TM * H; e += blockDim.x) {
            const int m = e / H, k = e % H;
            const float a = __bfloat162float(aL[m * HP + k]);
            dz0[m * HP + k] = __float2bfloat16_rn(a > 0.f ? gs[m] * head[k] : 0.f);
        }
    }
    __syncthreads();
    __nv_bfloat16 *dzc = dz0, *dzn = dz1;
    for (int l = NH - 1; l >= 0; l--) {
        const int K = l == 0 ? d.in : H, kp = kpad(H, l);
        const __nv_bfloat16 *Al = A_l(l);
        float *gW = slot + d.off[l];
        tile_dw<H>(dzc, HP, Al, l == 0 ? XP : HP, kp, K, gW);
        for (int nn = t; nn < H; nn += blockDim.x) {
            float s = 0.f;
            for (int m = 0; m < TM; m++) s += __bfloat162float(dzc[m * HP + nn]);
            gW[(size_t)H * K + nn] += s;
        }
        if (l > 0) {
            // dA_{l} = dZ W_l, through the ReLU of layer l's input
            tile_gemm<H, true, false>(dzc, HP, H, W_l(l), HP, nullptr, Al, HP, dzn, HP);
            __syncthreads();
            __nv_bfloat16 *tp = dzc;
            dzc = dzn;
            dzn = tp;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void bf_counters(nb_step_stats *st, unsigned long long c_fn, unsigned long long c_fp,
                                            unsigned long long c_nf) {
    const int t = threadIdx.x;
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

template <int H>
__global__ void __launch_bounds__(TPB, 1)
    train_bf16_kernel(TrainDesc d, const float *__restrict__ q, const uint32_t *__restrict__ labels, long long n,
                      float alpha, float beta, float inv_n, TauF tau, float *__restrict__ partial,
                      float *loss_partial, long long stride, long long P, nb_step_stats *st) {
    bf_load<H>(d, d.img, d.p);
    float *slot = partial + (size_t)blockIdx.x * stride;
    const long long ntiles = (n + TM - 1) / TM;
    float lossacc = 0.f;
    unsigned long long c_fn = 0, c_fp = 0, c_nf = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long base = tile * TM;
        const int rows = (int)min((long long)TM, n - base);
        bf_tile<H>(d, q, labels, base, rows, alpha, beta, inv_n, tau, slot, lossacc, c_fn, c_fp, c_nf);
    }
    if (threadIdx.x == 0) loss_partial[blockIdx.x] = lossacc;
    bf_counters(st, c_fn, c_fp, c_nf);
}

// Grouped form: persistent CTAs walk the work items of a plan (rows of one object
// each); a CTA reloads weights only when its next item belongs to another object.
// Object o's parameters start at d.p + o * P and its bf16 image at d.img + o * img_elems.
template <int H>
__global__ void __launch_bounds__(TPB, 1)
    train_bf16_group_kernel(TrainDesc d, long long img_elems, const PlanItem *__restrict__ items, int n_items,
                            const long long *__restrict__ offsets, const float *__restrict__ q,
                            const uint32_t *__restrict__ labels, float alpha_arg, const float *sched_alpha,
                            const int *d_step, int sched_T, float beta, const TauF *taus, float *__restrict__ partial,
                            float *loss_partial, long long P, long long S, nb_step_stats *st) {
    float alpha = alpha_arg;
    if (sched_alpha) alpha = sched_alpha[min(*d_step, sched_T - 1)];
    unsigned long long c_fn = 0, c_fp = 0, c_nf = 0;
    int cur = -1;
    int k0, k1;
    item_range(n_items, k0, k1);
    for (int it = k0; it < k1; it++) {
        const PlanItem w = items[it];
        TrainDesc dd = d;
        dd.p = d.p + (size_t)w.obj * P;
        if (w.obj != cur) {
            __syncthreads();
            bf_load<H>(dd, d.img + (size_t)w.obj * img_elems, dd.p);
            cur = w.obj;
        }
        const float inv_n = 1.0f / (float)(offsets[w.obj + 1] - offsets[w.obj]);
        float *slot = partial + (size_t)it * S;
        float lossacc = 0.f;
        for (long long base = w.row0; base < w.row1; base += TM) {
            const int rows = (int)min((long long)TM, w.row1 - base);
            bf_tile<H>(dd, q, labels, base, rows, alpha, beta, inv_n, taus[w.obj], slot, lossacc, c_fn, c_fp, c_nf);
        }
        if (threadIdx.x == 0) loss_partial[it] = lossacc;
    }
    bf_counters(st, c_fn, c_fp, c_nf);
}

// FP32 master weights -> bf16 training image; blockIdx.y selects the object of a group
__global__ void pack_train_kernel(TrainDesc d, __nv_bfloat16 *img, long long total, long long P) {
    const int H = d.H;
    d.p += (size_t)blockIdx.y * P;
    img += (size_t)blockIdx.y * total;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int l;
        long long local;
        if (e < (long long)H * K0) {
            l = 0;
            local = e;
        } else {
            l = 1 + (int)((e - (long long)H * K0) / ((long long)H * H));
            local = (e - (long long)H * K0) % ((long long)H * H);
        }
        const int kp = kpad(H, l), K = l == 0 ? d.in : H;
        const int row = (int)(local / kp), col = (int)(local % kp);
        img[e] = __float2bfloat16_rn(col < K ? d.p[d.off[l] + (size_t)row * K + col] : 0.f);
    }
}

TrainDesc make_desc(const TcModel *tc, const MlpDesc &d) {
    TrainDesc t{};
    t.in = d.w[0];
    t.H = d.w[1];
    t.NH = d.L - 1;
    t.img = (const __nv_bfloat16 *)tc->train_img;
    t.p = d.p;
    for (int l = 0; l < d.L; l++) t.off[l] = d.off[l];
    return t;
}

size_t train_img_elems(int H, int NH) { return img_off(H, NH); }

int num_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// ------------------------------------------------------------------ width 256
// The BF16 weights of a 256-wide network (128 KB per hidden layer) do not fit in shared
// memory next to a tile's activations, so this form streams them: each layer's forward
// GEMM runs in two halves of 128 output neurons and each input-gradient GEMM in two halves
// of 128 contraction rows, every half loaded into one shared buffer just before use (the
// first layer, 256 x 16, in one piece).  Tiles of 32 samples; the head, the loss, the bias
// gradients and the weight-gradient partials (four-column vector reductions into the CTA's
// slot) as in the resident form.
constexpr int TW = 32, HW = 256, HPW = HW + PAD, XPW = K0 + PAD, HALFW = 128;

struct WideSmem {
    __nv_bfloat16 *x, *act, *dz0, *dz1, *wb;
    float *bias, *head, *zs, *gs, *ls;
};
__device__ __forceinline__ WideSmem wide_smem(int NH) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    WideSmem m;
    m.x = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
    m.act = m.x + TW * XPW;                      // A_1 .. A_NH, [TW][HPW] each
    m.dz0 = m.act + (size_t)NH * TW * HPW;
    m.dz1 = m.dz0 + TW * HPW;
    m.wb = m.dz1 + TW * HPW;                     // [HALFW][HPW], or the first layer [HW][XPW]
    m.bias = reinterpret_cast<float *>(m.wb + HALFW * HPW);
    m.head = m.bias + NH * HW;
    m.zs = m.head + HW + 4;
    m.gs = m.zs + TW;
    m.ls = m.gs + TW;
    return m;
}
__device__ __forceinline__ __nv_bfloat16 *wide_A(const WideSmem &m, int l) {
    return l == 0 ? m.x : m.act + (size_t)(l - 1) * TW * HPW;
}

// rows [row0, row0 + nrows) of layer l's image (kp columns) -> wb with row pitch `pitch`
__device__ __forceinline__ void wide_load(const __nv_bfloat16 *img_l, int kp, int row0, int nrows,
                                          __nv_bfloat16 *wb, int pitch) {
    const int cpr = kp / 8;  // 16-byte chunks per row
    for (int e = threadIdx.x; e < nrows * cpr; e += blockDim.x) {
        const int r = e / cpr, c = e % cpr;
        *reinterpret_cast<uint4 *>(wb + r * pitch + c * 8) =
            *reinterpret_cast<const uint4 *>(img_l + (size_t)(row0 + r) * kp + c * 8);
    }
}

// OUT[:, col0 .. col0+127] = relu(X W^T + b) for the 128 output rows of wb from wrow0
__device__ __forceinline__ void wide_fwd_half(const __nv_bfloat16 *X, int xp, int K, const __nv_bfloat16 *wb,
                                              int wp, int wrow0, const float *bias, int col0, __nv_bfloat16 *out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = (warp & 1) * 16, nb = (warp >> 1) * 32;
    const int mi = lane >> 3, r = lane & 7;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(smem_u32(X + (m0 + r + (mi & 1) * 8) * xp + k0 + (mi >> 1) * 8), a0, a1, a2, a3);
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
            uint32_t b0, b1, b2, b3;
            ldsm_x4(smem_u32(wb + (wrow0 + nb + 8 * j + r + (mi >> 1) * 8) * wp + k0 + (mi & 1) * 8), b0, b1, b2, b3);
            mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
            mma_bf16(acc[j + 1], a0, a1, a2, a3, b2, b3);
        }
    }
    const int gr = lane >> 2, gc = (lane & 3) * 2;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int nn = col0 + nb + 8 * j + gc;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int m = m0 + gr + 8 * h;
            const float v0 = fmaxf(acc[j][2 * h] + bias[nn], 0.f), v1 = fmaxf(acc[j][2 * h + 1] + bias[nn + 1], 0.f);
            *reinterpret_cast<uint32_t *>(out + m * HPW + nn) = pack2(v0, v1);
        }
    }
}

// acc += DZ[:, n0h .. n0h+127] W[n0h .. n0h+127][:] with wb holding those 128 rows of W
// (input gradient, 256 output columns; warps: 2 along the 32 rows x 4 along 64 columns)
__device__ __forceinline__ void wide_da_half(const __nv_bfloat16 *DZ, int n0h, const __nv_bfloat16 *wb,
                                             float (&acc)[8][4]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = (warp & 1) * 16, c0 = (warp >> 1) * 64;
    const int mi = lane >> 3, r = lane & 7;
    for (int k0 = 0; k0 < HALFW; k0 += 16) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(smem_u32(DZ + (m0 + r + (mi & 1) * 8) * HPW + n0h + k0 + (mi >> 1) * 8), a0, a1, a2, a3);
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            uint32_t b0, b1, b2, b3;
            // wb[n][k] read transposed: matrices (n0-7,k0-7) (n8-15,k0-7) (n0-7,k8-15) (n8-15,k8-15)
            ldsm_x4_t(smem_u32(wb + (k0 + r + (mi & 1) * 8) * HPW + c0 + 8 * j + (mi >> 1) * 8), b0, b1, b2, b3);
            mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
            mma_bf16(acc[j + 1], a0, a1, a2, a3, b2, b3);
        }
    }
}

// slot[n][k] += sum_m DZ[m][n] A[m][k], n < 256, k < Kreal (Kp padded columns of A)
__device__ __forceinline__ void wide_dw(const __nv_bfloat16 *DZ, const __nv_bfloat16 *A, int ap, int Kp, int Kreal,
                                        float *slotW) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mi = lane >> 3, r = lane & 7;
    const int gr = lane >> 2, gc = (lane & 3) * 2;
    const bool odd = lane & 1;
    for (int kc = 0; kc < Kp; kc += 64) {
        const int cw = min(64, Kp - kc);
        float acc[2][8][4];
#pragma unroll
        for (int b = 0; b < 2; b++)
#pragma unroll
            for (int j = 0; j < 8; j++) acc[b][j][0] = acc[b][j][1] = acc[b][j][2] = acc[b][j][3] = 0.f;
#pragma unroll
        for (int m0 = 0; m0 < TW; m0 += 16) {
            uint32_t a[2][4];
#pragma unroll
            for (int b = 0; b < 2; b++) {
                const int n0 = warp * 32 + 16 * b;
                ldsm_x4_t(smem_u32(DZ + (m0 + r + (mi >> 1) * 8) * HPW + n0 + (mi & 1) * 8), a[b][0], a[b][1], a[b][2],
                          a[b][3]);
            }
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                if (8 * j >= cw) break;
                uint32_t b0, b1, b2, b3;
                ldsm_x4_t(smem_u32(A + (m0 + r + (mi & 1) * 8) * ap + kc + 8 * j + (mi >> 1) * 8), b0, b1, b2, b3);
#pragma unroll
                for (int b = 0; b < 2; b++) {
                    mma_bf16(acc[b][j], a[b][0], a[b][1], a[b][2], a[b][3], b0, b1);
                    if (8 * (j + 1) < cw) mma_bf16(acc[b][j + 1], a[b][0], a[b][1], a[b][2], a[b][3], b2, b3);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const int n0 = warp * 32 + 16 * b;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                if (8 * j >= cw) break;
                const float s0 = odd ? acc[b][j][0] : acc[b][j][2], s1 = odd ? acc[b][j][1] : acc[b][j][3];
                const float r0 = __shfl_xor_sync(FULL, s0, 1), r1 = __shfl_xor_sync(FULL, s1, 1);
                const int k4 = kc + 8 * j + (gc & ~2);
                const int nn = n0 + gr + (odd ? 8 : 0);
                float v[4];
                if (odd) {
                    v[0] = r0; v[1] = r1; v[2] = acc[b][j][2]; v[3] = acc[b][j][3];
                } else {
                    v[0] = acc[b][j][0]; v[1] = acc[b][j][1]; v[2] = r0; v[3] = r1;
                }
                float *dst = slotW + (size_t)nn * Kreal + k4;
                if (k4 + 3 < Kreal && ((uintptr_t)dst & 15) == 0) {
                    red_add4(dst, v[0], v[1], v[2], v[3]);
                } else {
#pragma unroll
                    for (int u = 0; u < 4; u++)
                        if (k4 + u < Kreal) red_add(dst + u, v[u]);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256, 1)
    train_bf16_wide_kernel(TrainDesc d, const float *__restrict__ q, const uint32_t *__restrict__ labels, long long n,
                           float alpha, float beta, float inv_n, TauF tau, float *__restrict__ partial,
                           float *loss_partial, long long stride, nb_step_stats *st) {
    const int NH = d.NH, t = threadIdx.x;
    const WideSmem sm = wide_smem(NH);
    for (int i = t; i < NH * HW; i += blockDim.x) {
        const int l = i / HW, j = i % HW;
        sm.bias[i] = d.p[d.off[l] + HW * (l == 0 ? d.in : HW) + j];
    }
    for (int i = t; i <= HW; i += blockDim.x) sm.head[i] = d.p[d.off[NH] + i];
    float *slot = partial + (size_t)blockIdx.x * stride;
    const long long ntiles = (n + TW - 1) / TW;
    float lossacc = 0.f;
    unsigned long long c_fn = 0, c_fp = 0, c_nf = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long base = tile * TW;
        const int rows = (int)min((long long)TW, n - base);
        __syncthreads();
        for (int e = t; e < TW * K0; e += blockDim.x) {
            const int m = e / K0, k = e % K0;
            const float xv = (m < rows && k < d.in) ? q[(base + m) * d.in + k] : 0.f;
            sm.x[m * XPW + k] = __float2bfloat16_rn(xv);
        }
        // forward: the first layer in one piece, the hidden layers in two halves
        wide_load(d.img, K0, 0, HW, sm.wb, XPW);
        __syncthreads();
        wide_fwd_half(sm.x, XPW, K0, sm.wb, XPW, 0, sm.bias, 0, wide_A(sm, 1));
        wide_fwd_half(sm.x, XPW, K0, sm.wb, XPW, HALFW, sm.bias, HALFW, wide_A(sm, 1));
        for (int l = 1; l < NH; l++) {
            const __nv_bfloat16 *img_l = d.img + img_off(HW, l);
            for (int h = 0; h < 2; h++) {
                __syncthreads();  // the buffer is free and layer l's inputs are in place
                wide_load(img_l, HW, h * HALFW, HALFW, sm.wb, HPW);
                __syncthreads();
                wide_fwd_half(wide_A(sm, l), HPW, HW, sm.wb, HPW, 0, sm.bias + l * HW, h * HALFW, wide_A(sm, l + 1));
            }
        }
        __syncthreads();
        // head (FP32) and loss: 4 threads per sample
        if (t < 4 * TW) {
            const __nv_bfloat16 *aL = wide_A(sm, NH);
            const int m = t >> 2, part = t & 3;
            float sacc = 0.f;
            for (int k = part; k < HW; k += 4) sacc = fmaf(sm.head[k], __bfloat162float(aL[m * HPW + k]), sacc);
            sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
            sacc += __shfl_xor_sync(0xffffffffu, sacc, 2);
            if (part == 0) sm.zs[m] = sacc + sm.head[HW];
        }
        __syncthreads();
        if (t < TW) {
            float g = 0.f, lv = 0.f;
            if (t < rows) {
                const long long i = base + t;
                const float y = (float)((labels[i >> 5] >> (i & 31)) & 1u);
                const float z = sm.zs[t];
                if (isfinite(z) && row_finite(sm.x + t * XPW, d.in)) {
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
            sm.gs[t] = g;
            sm.ls[t] = lv;
            if (t < rows && !(isfinite(sm.zs[t]) && row_finite(sm.x + t * XPW, d.in))) {
                for (int k = 0; k < K0; k++) sm.x[t * XPW + k] = __float2bfloat16_rn(0.f);
                for (int l = 1; l <= NH; l++)
                    for (int k = 0; k < HW; k++) wide_A(sm, l)[t * HPW + k] = __float2bfloat16_rn(0.f);
            }
        }
        __syncthreads();
        if (t == 0)
            for (int m = 0; m < rows; m++) lossacc += sm.ls[m];
        // head gradients and dZ of the last hidden layer
        {
            const __nv_bfloat16 *aL = wide_A(sm, NH);
            float *gW = slot + d.off[NH];
            for (int k = t; k <= HW; k += blockDim.x) {
                float sacc = 0.f;
                if (k < HW)
                    for (int m = 0; m < TW; m++) sacc = fmaf(sm.gs[m], __bfloat162float(aL[m * HPW + k]), sacc);
                else
                    for (int m = 0; m < TW; m++) sacc += sm.gs[m];
                gW[k] += sacc;
            }
            for (int e = t; e < TW * HW; e += blockDim.x) {
                const int m = e / HW, k = e % HW;
                const float a = __bfloat162float(aL[m * HPW + k]);
                sm.dz0[m * HPW + k] = __float2bfloat16_rn(a > 0.f ? sm.gs[m] * sm.head[k] : 0.f);
            }
        }
        __syncthreads();
        __nv_bfloat16 *dzc = sm.dz0, *dzn = sm.dz1;
        for (int l = NH - 1; l >= 0; l--) {
            const int K = l == 0 ? d.in : HW, kp = kpad(HW, l);
            const __nv_bfloat16 *Al = wide_A(sm, l);
            float *gW = slot + d.off[l];
            wide_dw(dzc, Al, l == 0 ? XPW : HPW, kp, K, gW);
            for (int nn = t; nn < HW; nn += blockDim.x) {
                float sacc = 0.f;
                for (int m = 0; m < TW; m++) sacc += __bfloat162float(dzc[m * HPW + nn]);
                gW[(size_t)HW * K + nn] += sacc;
            }
            if (l > 0) {
                // dA_l = dZ W_l through the ReLU of layer l's input, W_l streamed in two halves
                float acc[8][4];
#pragma unroll
                for (int j = 0; j < 8; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
                const __nv_bfloat16 *img_l = d.img + img_off(HW, l);
                for (int h = 0; h < 2; h++) {
                    __syncthreads();
                    wide_load(img_l, HW, h * HALFW, HALFW, sm.wb, HPW);
                    __syncthreads();
                    wide_da_half(dzc, h * HALFW, sm.wb, acc);
                }
                const int warp = t >> 5, lane = t & 31;
                const int m0 = (warp & 1) * 16, c0 = (warp >> 1) * 64;
                const int gr = lane >> 2, gc = (lane & 3) * 2;
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int nn = c0 + 8 * j + gc;
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int m = m0 + gr + 8 * h;
                        const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(Al + m * HPW + nn);
                        const float v0 = __low2float(mk) > 0.f ? acc[j][2 * h] : 0.f;
                        const float v1 = __high2float(mk) > 0.f ? acc[j][2 * h + 1] : 0.f;
                        *reinterpret_cast<uint32_t *>(dzn + m * HPW + nn) = pack2(v0, v1);
                    }
                }
                __syncthreads();
                __nv_bfloat16 *tp = dzc;
                dzc = dzn;
                dzn = tp;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) loss_partial[blockIdx.x] = lossacc;
    bf_counters(st, c_fn, c_fp, c_nf);
}

size_t wide_smem_bytes(int NH) {
    const size_t bf = (size_t)TW * XPW + (size_t)NH * TW * HPW + 2 * (size_t)TW * HPW + (size_t)HALFW * HPW;
    return bf * 2 + ((size_t)NH * HW + HW + 4 + 3 * TW) * 4 + 64;
}

}  // namespace

size_t nb_train_bf16_smem(int H, int NH, long long P) {
    if (H == 256) return wide_smem_bytes(NH);
    const size_t HP = H + PAD, XP = K0 + PAD;
    const size_t w = (size_t)H * XP + (size_t)(NH - 1) * H * HP;
    const size_t a = (size_t)TM * XP + (size_t)NH * TM * HP;
    const size_t dz = 2 * (size_t)TM * HP;
    (void)P;
    return (w + a + dz) * 2 + ((size_t)NH * H + H + 4 + 3 * TM) * 4 + 64;
}

nb_status nb_train_bf16_check(const MlpDesc &d) {
    const int H = d.w[1], NH = d.L - 1;
    if (NH < 1) return nb_fail(NB_EUNSUPPORTED, "BF16 training needs at least one hidden layer");
    if (d.w[0] > K0) return nb_fail(NB_EUNSUPPORTED, "BF16 training: input width must be <= 16");
    if (H != 64 && H != 128 && H != 256)
        return nb_fail(NB_EUNSUPPORTED, "BF16 training: hidden width must be 64, 128 or 256");
    for (int l = 1; l < d.L; l++)
        if (d.w[l] != H) return nb_fail(NB_EUNSUPPORTED, "BF16 training: hidden widths must be equal");
    int dev = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    long long P = 0;
    for (int l = 0; l < d.L; l++) P += (long long)d.w[l + 1] * (d.w[l] + 1);
    if (nb_train_bf16_smem(H, NH, P) > (size_t)maxsm)
        return nb_fail(NB_EUNSUPPORTED, "BF16 training: the network does not fit in shared memory");
    return NB_OK;
}

size_t nb_train_bf16_img_bytes(const MlpDesc &d) { return train_img_elems(d.w[1], d.L - 1) * 2; }

nb_status nb_train_bf16_refresh(TcModel *tc, const MlpDesc &d, cudaStream_t s) {
    const TrainDesc t = make_desc(tc, d);
    const long long total = (long long)train_img_elems(t.H, t.NH);
    pack_train_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(t, (__nv_bfloat16 *)tc->train_img, total, 0);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

int nb_train_bf16_ctas(int64_t n) {
    const int64_t tiles = (n + TM - 1) / TM;
    int64_t g = num_sms();
    if (g > tiles) g = tiles;
    return (int)(g < 1 ? 1 : g);
}

nb_status nb_launch_train_bf16(TcModel *tc, const MlpDesc &d, const float *q, const uint32_t *labels, int64_t n,
                               float alpha, float beta, TauF tau, TrainWs ws, nb_step_stats *st, cudaStream_t s) {
    const TrainDesc t = make_desc(tc, d);
    long long P = 0;
    for (int l = 0; l < d.L; l++) P += (long long)d.w[l + 1] * (d.w[l] + 1);
    const long long stride = ws.stride > 0 ? ws.stride : P;  // slots 16-byte aligned when a multiple of 4
    NB_CUDA(cudaMemsetAsync(ws.partial, 0, (size_t)ws.G * stride * sizeof(float), s));
    if (st) NB_CUDA(cudaMemsetAsync(st, 0, sizeof(nb_step_stats), s));
    const size_t smem = nb_train_bf16_smem(t.H, t.NH, P);
    if (t.H == 256) {
        // weights streamed per half layer (tiles of 32 samples)
        NB_CUDA(cudaFuncSetAttribute(train_bf16_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        train_bf16_wide_kernel<<<ws.G, 256, smem, s>>>(t, q, labels, (long long)n, alpha, beta, 1.0f / (float)n, tau,
                                                       ws.partial, ws.loss_partial, stride, st);
    } else if (t.H == 128) {
        NB_CUDA(cudaFuncSetAttribute(train_bf16_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        train_bf16_kernel<128><<<ws.G, TPB, smem, s>>>(t, q, labels, (long long)n, alpha, beta, 1.0f / (float)n, tau,
                                                       ws.partial, ws.loss_partial, stride, P, st);
    } else {
        NB_CUDA(cudaFuncSetAttribute(train_bf16_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        train_bf16_kernel<64><<<ws.G, TPB, smem, s>>>(t, q, labels, (long long)n, alpha, beta, 1.0f / (float)n, tau,
                                                      ws.partial, ws.loss_partial, stride, P, st);
    }
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_train_bf16_group_init(TcModel *tc, const MlpDesc &d, int n_objects) {
    const nb_status st = nb_train_bf16_check(d);
    if (st != NB_OK) return st;
    if (d.w[1] == 256) return nb_fail(NB_EUNSUPPORTED, "grouped BF16 training: hidden width must be 64 or 128");
    tc->train_img_bytes = nb_train_bf16_img_bytes(d);
    if (cudaMalloc(&tc->train_img, tc->train_img_bytes * (size_t)n_objects) != cudaSuccess) {
        cudaGetLastError();
        return nb_fail(NB_ENOMEM, "grouped training image allocation failed");
    }
    return NB_OK;
}

nb_status nb_train_bf16_group_refresh(TcModel *tc, const MlpDesc &d, int n_objects, cudaStream_t s) {
    const TrainDesc t = make_desc(tc, d);
    const long long total = (long long)train_img_elems(t.H, t.NH);
    long long P = 0;
    for (int l = 0; l < d.L; l++) P += (long long)d.w[l + 1] * (d.w[l] + 1);
    pack_train_kernel<<<dim3((unsigned)((total + 255) / 256), n_objects), 256, 0, s>>>(
        t, (__nv_bfloat16 *)tc->train_img, total, P);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_launch_train_bf16_group(TcModel *tc, const MlpDesc &d, long long P, long long S, const nb_plan *pl,
                                     const float *q,
                                     const uint32_t *labels, float alpha, const float *sched_alpha, const int *d_step,
                                     int sched_T, float beta, const TauF *taus, float *partial, float *loss_partial,
                                     nb_step_stats *st, cudaStream_t s) {
    const TrainDesc t = make_desc(tc, d);
    const long long img_elems = (long long)train_img_elems(t.H, t.NH);
    const size_t smem = nb_train_bf16_smem(t.H, t.NH, P);
    int grid = num_sms();
    if (grid > pl->n_items) grid = pl->n_items;
    if (grid < 1) return NB_OK;
    if (t.H == 128) {
        NB_CUDA(cudaFuncSetAttribute(train_bf16_group_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        train_bf16_group_kernel<128><<<grid, TPB, smem, s>>>(t, img_elems, pl->items, pl->n_items, pl->offsets, q,
                                                             labels, alpha, sched_alpha, d_step, sched_T, beta, taus,
                                                             partial, loss_partial, P, S, st);
    } else {
        NB_CUDA(cudaFuncSetAttribute(train_bf16_group_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        train_bf16_group_kernel<64><<<grid, TPB, smem, s>>>(t, img_elems, pl->items, pl->n_items, pl->offsets, q,
                                                            labels, alpha, sched_alpha, d_step, sched_T, beta, taus,
                                                            partial, loss_partial, P, S, st);
    }
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}
