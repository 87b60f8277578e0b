// Query sampler: Alg. 1 draws a fresh batch r ~ Uniform at every iteration.
//
// The draws come from the counter-based generator Philox4x64-10 (Salmon, Moraes,
// Dror and Shaw, SC 2011): query i of the stream (seed, kind) reads the blocks
// philox(counter = (i, j, p, 0), key = (seed, kind)), p = 0 for its scalars and
// p = 1, 2 for its first and second unit vector (j counts rejection attempts), so
// any range of a stream can be drawn by any launch in any order.  Every value is
// built in integers or in correctly rounded IEEE operations (division, square root,
// products and sums written with explicit round-to-nearest intrinsics, no
// contraction), then rounded to the 2^-qexp grid, so a stream is the same bits on
// every device.
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

__device__ __forceinline__ float grid_round(double x, double scale, double quantum) {
    return (float)__dmul_rn(rint(__dmul_rn(x, scale)), quantum);
}

// uniform direction: the first of up to 64 words whose three signed 21-bit fields
// lie in the shell 2^30 <= |v|^2 <= 2^40, normalised in FP64
__device__ void unit_vector(unsigned long long seed, int kind, long long i, unsigned p, double u[3]) {
    for (unsigned j = 0; j < 16; j++) {
        const Block4 b = philox((unsigned long long)i, j, p, seed, (unsigned long long)kind);
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const long long v0 = field21(b.w[m], 0), v1 = field21(b.w[m], 1), v2 = field21(b.w[m], 2);
            const long long n2 = v0 * v0 + v1 * v1 + v2 * v2;
            if (n2 >= (1ll << 30) && n2 <= (1ll << 40)) {
                const double len = __dsqrt_rn((double)n2);
                u[0] = __ddiv_rn((double)v0, len);
                u[1] = __ddiv_rn((double)v1, len);
                u[2] = __ddiv_rn((double)v2, len);
                return;
            }
        }
    }
    u[0] = 0.0;
    u[1] = 0.0;
    u[2] = 1.0;
}

// 2^y for y >= 0: 2^floor(y) times the degree-20 Taylor polynomial of exp(f ln 2),
// f = y - floor(y), in the nested form p = 1 + (t/k) p, k = 20 .. 1
__device__ double exp2_taylor(double y) {
    const double n = floor(y);
    const double t = __dmul_rn(__dadd_rn(y, -n), 0.6931471805599453);
    double p = 1.0;
    for (int k = 20; k >= 1; k--) p = __dadd_rn(1.0, __dmul_rn(__ddiv_rn(t, (double)k), p));
    return scalbn(p, (int)n);
}

template <int KIND, int W>
__global__ void __launch_bounds__(TPB) sample_kernel(unsigned long long seed, int qexp, long long first,
                                                     long long n, float *__restrict__ q) {
    __shared__ float buf[TPB * W];
    const float quantum = ldexpf(1.0f, -qexp);
    const double dscale = ldexp(1.0, qexp), dquantum = ldexp(1.0, -qexp);
    for (long long base = (long long)blockIdx.x * TPB; base < n; base += (long long)gridDim.x * TPB) {
        const long long r = base + threadIdx.x;
        if (r < n) {
            const long long i = first + r;
            float *o = buf + threadIdx.x * W;
            if (KIND == NB_RAY3) {
                double u[3], v[3];
                unit_vector(seed, KIND, i, 1, u);
                unit_vector(seed, KIND, i, 2, v);
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    o[d] = grid_round(2.0 * u[d], dscale, dquantum);
                    o[3 + d] = grid_round(v[d], dscale, dquantum);
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
                            const double x = __dmul_rn((double)(b.w[1 + d] >> 11), 0x1p-53);
                            const double e = __dmul_rn(0.01, exp2_taylor(__dmul_rn(x, 5.643856189774724)));
                            o[3 + d] = grid_round(e, dscale, dquantum);
                        }
                    }
                } else if (KIND == NB_PLANE3) {
                    double u[3];
                    unit_vector(seed, KIND, i, 1, u);
#pragma unroll
                    for (int d = 0; d < 3; d++) o[d] = grid_round(u[d], dscale, dquantum);
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
