// Query sampler: Alg. 1 draws a fresh batch r ~ Uniform at every iteration.
//
// The draws come from the counter-based generator Philox4x64-10 (Salmon, Moraes,
// Dror and Shaw, SC 2011): query i of the stream (seed, kind) reads the blocks
// philox(counter = (i, j, p, 0), key = (seed, kind)), p = 0 for its scalars and
// p = 1, 2 for its first and second unit vector (j counts rejection attempts), so
// any range of a stream can be drawn by any launch in any order.  Every value is
// built in integers or in single IEEE float operations (division, square root,
// products and sums written with explicit round-to-nearest intrinsics, no
// contraction; FP32 rather than FP64, whose rate on this GPU is a small fraction of
// FP32's), then rounded to the 2^-qexp grid, so a stream is the same bits on every
// device.
#include "common.cuh"

namespace {

constexpr unsigned long long PH_M0 = 0xD2E7470EE14C6C93ull, PH_M1 = 0xCA5A826395121157ull;
constexpr unsigned long long PH_W0 = 0x9E3779B97F4A7C15ull, PH_W1 = 0xBB67AE8584CAA73Bull;
constexpr int TPB = 256;

struct Block4 {
    unsigned long long w[4];
};

__device__ __forceinline__ Block4 philox(unsigned long long c0, unsigned long long c1, unsigned long long c2,
                                         unsigned long long k0, unsigned long long k1) {
    unsigned long long x0 = c0, x1 = c1, x2 = c2, x3 = 0;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const unsigned long long hi0 = __umul64hi(PH_M0, x0), lo0 = PH_M0 * x0;
        const unsigned long long hi1 = __umul64hi(PH_M1, x2), lo1 = PH_M1 * x2;
        x0 = hi1 ^ x1 ^ k0;
        x1 = lo1;
        x2 = hi0 ^ x3 ^ k1;
        x3 = lo0;
        k0 += PH_W0;
        k1 += PH_W1;
    }
    return {{x0, x1, x2, x3}};
}

__device__ __forceinline__ long long field21(unsigned long long w, int s) {
    return (long long)((w >> (21 * s)) & 0x1FFFFFull) - 1048576ll;
}

// U[-1,1) in units of 2^-qexp: the top qexp+1 bits of the 21-bit field s
__device__ __forceinline__ float coord(unsigned long long w, int s, int qexp, float quantum) {
    const long long f = (long long)((w >> (21 * s)) & 0x1FFFFFull);
    return (float)((f >> (20 - qexp)) - (1ll << qexp)) * quantum;
}

__device__ __forceinline__ float grid_round(float x, float scale, float quantum) {
    return __fmul_rn(rintf(__fmul_rn(x, scale)), quantum);
}

// uniform direction: the first of up to 64 words whose three signed 21-bit fields
// lie in the shell 2^30 <= |v|^2 <= 2^40, normalised in FP32 (|v|^2 rounded to float,
// IEEE square root and division)
__device__ void unit_vector(unsigned long long seed, int kind, long long i, unsigned p, float u[3]) {
    for (unsigned j = 0; j < 16; j++) {
        const Block4 b = philox((unsigned long long)i, j, p, seed, (unsigned long long)kind);
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const long long v0 = field21(b.w[m], 0), v1 = field21(b.w[m], 1), v2 = field21(b.w[m], 2);
            const long long n2 = v0 * v0 + v1 * v1 + v2 * v2;
            if (n2 >= (1ll << 30) && n2 <= (1ll << 40)) {
                const float len = __fsqrt_rn(__ll2float_rn(n2));
                u[0] = __fdiv_rn((float)v0, len);
                u[1] = __fdiv_rn((float)v1, len);
                u[2] = __fdiv_rn((float)v2, len);
                return;
            }
        }
    }
    u[0] = 0.f;
    u[1] = 0.f;
    u[2] = 1.f;
}

// 2^y for 0 <= y < 8: 2^floor(y) times the degree-9 Taylor polynomial of exp(f ln 2),
// f = y - floor(y), coefficients 1/k! rounded to float, Horner form, one IEEE float
// operation per step
__device__ float exp2_taylor(float y) {
    constexpr float c[10] = {0x1p+0f, 0x1p+0f, 0x1p-1f, 0x1.555556p-3f, 0x1.555556p-5f,
                             0x1.111112p-7f, 0x1.6c16c2p-10f, 0x1.a01a02p-13f, 0x1.a01a02p-16f,
                             0x1.71de3ap-19f};
    const float n = floorf(y);
    const float t = __fmul_rn(__fsub_rn(y, n), 0x1.62e43p-1f);
    float p = c[9];
#pragma unroll
    for (int k = 8; k >= 0; k--) p = __fadd_rn(__fmul_rn(p, t), c[k]);
    return ldexpf(p, (int)n);
}

template <int KIND, int W>
__global__ void __launch_bounds__(TPB) sample_kernel(unsigned long long seed, int qexp, long long first,
                                                     long long n, float *__restrict__ q) {
    __shared__ float buf[TPB * W];
    const float quantum = ldexpf(1.0f, -qexp), scale = ldexpf(1.0f, qexp);
    for (long long base = (long long)blockIdx.x * TPB; base < n; base += (long long)gridDim.x * TPB) {
        const long long r = base + threadIdx.x;
        if (r < n) {
            const long long i = first + r;
            float *o = buf + threadIdx.x * W;
            if (KIND == NB_RAY3) {
                float u[3], v[3];
                unit_vector(seed, KIND, i, 1, u);
                unit_vector(seed, KIND, i, 2, v);
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    o[d] = grid_round(2.f * u[d], scale, quantum);
                    o[3 + d] = grid_round(v[d], scale, quantum);
                }
            } else {
                const Block4 b = philox((unsigned long long)i, 0, 0, seed, (unsigned long long)KIND);
                if (KIND == NB_POINT2) {
                    o[0] = coord(b.w[0], 0, qexp, quantum);
                    o[1] = coord(b.w[0], 1, qexp, quantum);
                } else if (KIND == NB_POINT3 || KIND == NB_POINT4T || KIND == NB_BOX3) {
#pragma unroll
                    for (int d = 0; d < 3; d++) o[d] = coord(b.w[0], d, qexp, quantum);
                    if (KIND == NB_POINT4T)
                        o[3] = (float)(long long)(b.w[1] & ((1ull << qexp) - 1)) * quantum;
                    if (KIND == NB_BOX3) {
#pragma unroll
                        for (int d = 0; d < 3; d++) {
                            const float x = __fmul_rn((float)(b.w[1 + d] >> 40), 0x1p-24f);
                            const float e = __fmul_rn(0x1.47ae14p-7f, exp2_taylor(__fmul_rn(x, 0x1.6934fp+2f)));
                            o[3 + d] = grid_round(e, scale, quantum);
                        }
                    }
                } else if (KIND == NB_PLANE3) {
                    float u[3];
                    unit_vector(seed, KIND, i, 1, u);
#pragma unroll
                    for (int d = 0; d < 3; d++) o[d] = grid_round(u[d], scale, quantum);
                    o[3] = coord(b.w[0], 0, qexp, quantum);
                }
            }
        }
        __syncthreads();
        // the block's rows are one contiguous range of q: store it coalesced
        const long long rows = min((long long)TPB, n - base);
        float *dst = q + base * W;
        for (int k = threadIdx.x; k < rows * W; k += TPB) dst[k] = buf[k];
        __syncthreads();
    }
}

template <int KIND, int W>
nb_status launch(uint64_t seed, int qexp, int64_t first, int64_t n, float *q, cudaStream_t s) {
    int dev = 0, sms = 148;
    NB_CUDA(cudaGetDevice(&dev));
    NB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long blocks_needed = (n + TPB - 1) / TPB;
    const int grid = (int)std::min<long long>(blocks_needed, (long long)sms * 8);
    sample_kernel<KIND, W><<<grid, TPB, 0, s>>>(seed, qexp, first, n, q);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

}  // namespace

extern "C" nb_status nb_sample(int32_t kind, int32_t qexp, uint64_t seed, int64_t first, int64_t n, float *q,
                               void *stream) {
    if (kind < NB_POINT2 || kind > NB_BOX3) return nb_fail(NB_EINVAL, "nb_sample: unknown kind");
    if (qexp < 8 || qexp > 20) return nb_fail(NB_EINVAL, "nb_sample: qexp must be in [8, 20]");
    if (first < 0 || n < 0 || first > (int64_t)1 << 62 || n > (int64_t)1 << 40)
        return nb_fail(NB_EINVAL, "nb_sample: bad range");
    if (n == 0) return NB_OK;
    if (!q) return nb_fail(NB_EINVAL, "nb_sample: null output");
    if ((uintptr_t)q % 4) return nb_fail(NB_EINVAL, "nb_sample: output not 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    switch (kind) {
    case NB_POINT2: return launch<NB_POINT2, 2>(seed, qexp, first, n, q, s);
    case NB_POINT3: return launch<NB_POINT3, 3>(seed, qexp, first, n, q, s);
    case NB_POINT4T: return launch<NB_POINT4T, 4>(seed, qexp, first, n, q, s);
    case NB_RAY3: return launch<NB_RAY3, 6>(seed, qexp, first, n, q, s);
    case NB_PLANE3: return launch<NB_PLANE3, 4>(seed, qexp, first, n, q, s);
    default: return launch<NB_BOX3, 6>(seed, qexp, first, n, q, s);
    }
}
