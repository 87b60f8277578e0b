// Exact labeler: y = g(r) of Sec. 3.1 for a union of closed balls.
//
// Alg. 1 labels a region by Any(f(SampleRegion(r))); here the region is tested
// against every ball analytically, in exact integer arithmetic on the 2^-qexp grid,
// so the label is the query function itself, inclusive of the surface (Sec. 3.1:
// the indicator is 1 inside and on the surface).
//
// Values are converted to integer grid units and must satisfy |v| < 2^29, which
// bounds every intermediate: differences < 2^30, squared sums < 2^62 (int64), and
// the ray / plane / moving-point products < 2^126 (unsigned 128-bit).
#include "common.cuh"

namespace {

struct SphI {
    int c[3];
    int r;
    int v[3];
    int pad;
};

constexpr float kGridLimit = 536870912.0f;  // 2^29

__device__ __forceinline__ bool to_grid(float x, float scale, int &out) {
    float s = x * scale;  // scaling by a power of two is exact
    if (!(fabsf(s) < kGridLimit)) return false;  // also rejects NaN and inf
    int k = __float2int_rn(s);
    if ((float)k != s) return false;
    out = k;
    return true;
}

__device__ __forceinline__ long long sq(int a) { return (long long)a * (long long)a; }

template <int KIND>
__device__ __forceinline__ int union_hit(const int *Q, const SphI *sph, int ns, int qexp) {
    if constexpr (KIND == NB_POINT2) {
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            long long d2 = sq(Q[0] - S.c[0]) + sq(Q[1] - S.c[1]);
            if (d2 <= sq(S.r)) return 1;
        }
    } else if constexpr (KIND == NB_POINT3) {
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            long long d2 = sq(Q[0] - S.c[0]) + sq(Q[1] - S.c[1]) + sq(Q[2] - S.c[2]);
            if (d2 <= sq(S.r)) return 1;
        }
    } else if constexpr (KIND == NB_POINT4T) {
        // centre at time t is c + v t; scaled by 2^qexp every term is an integer:
        // d = (x - c) 2^qexp - v t  (units 2^-2qexp), test |d|^2 <= (r 2^qexp)^2
        const long long T = Q[3];
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            unsigned __int128 d2 = 0;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                long long d = (long long)(Q[i] - S.c[i]) * (1LL << qexp) - (long long)S.v[i] * T;
                unsigned long long a = d < 0 ? (unsigned long long)(-d) : (unsigned long long)d;
                d2 += (unsigned __int128)a * a;
            }
            unsigned long long rs = (unsigned long long)S.r << qexp;
            if (d2 <= (unsigned __int128)rs * rs) return 1;
        }
    } else if constexpr (KIND == NB_RAY3) {
        // half-line o + s d, s >= 0; w = c - o.  Closest point is o when w.d <= 0,
        // otherwise the foot of the perpendicular: |w|^2 |d|^2 - (w.d)^2 <= r^2 |d|^2,
        // rearranged as (|w|^2 - r^2) |d|^2 <= (w.d)^2 once |w|^2 > r^2.
        const long long DD = sq(Q[3]) + sq(Q[4]) + sq(Q[5]);
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            int w0 = S.c[0] - Q[0], w1 = S.c[1] - Q[1], w2 = S.c[2] - Q[2];
            long long WW = sq(w0) + sq(w1) + sq(w2);
            long long RR = sq(S.r);
            if (WW <= RR) return 1;
            long long SD = (long long)w0 * Q[3] + (long long)w1 * Q[4] + (long long)w2 * Q[5];
            if (SD <= 0) continue;
            unsigned __int128 lhs = (unsigned __int128)(unsigned long long)(WW - RR) * (unsigned long long)DD;
            unsigned __int128 rhs = (unsigned __int128)(unsigned long long)SD * (unsigned long long)SD;
            if (lhs <= rhs) return 1;
        }
    } else if constexpr (KIND == NB_PLANE3) {
        // plane {x : n.x = off}: (n.c - off)^2 <= r^2 |n|^2 (units 2^-4qexp)
        const long long NN = sq(Q[0]) + sq(Q[1]) + sq(Q[2]);
        const long long OFF = (long long)Q[3] * (1LL << qexp);
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            long long d = (long long)Q[0] * S.c[0] + (long long)Q[1] * S.c[1] + (long long)Q[2] * S.c[2] - OFF;
            unsigned long long a = d < 0 ? (unsigned long long)(-d) : (unsigned long long)d;
            if ((unsigned __int128)a * a <= (unsigned __int128)(unsigned long long)sq(S.r) * (unsigned long long)NN)
                return 1;
        }
    } else if constexpr (KIND == NB_BOX3) {
        // closed box: squared distance from the centre c to the box <= r^2
        for (int s = 0; s < ns; s++) {
            const SphI S = sph[s];
            long long d2 = 0;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                int a = abs(S.c[i] - Q[i]) - Q[3 + i];
                if (a > 0) d2 += sq(a);
            }
            if (d2 <= sq(S.r)) return 1;
        }
    }
    return 0;
}

template <int KIND, int W>
__global__ void __launch_bounds__(256) label_kernel(const float *__restrict__ q, long long n, int ns, int dim,
                                                    int qexp, const float *__restrict__ cen,
                                                    const float *__restrict__ rad, const float *__restrict__ vel,
                                                    uint32_t *__restrict__ bits, nb_label_stats *st) {
    extern __shared__ SphI sph[];
    __shared__ int scene_bad;
    const float scale = ldexpf(1.0f, qexp);
    if (threadIdx.x == 0) scene_bad = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        SphI S = {{0, 0, 0}, 0, {0, 0, 0}, 0};
        bool ok = true;
        for (int i = 0; i < dim; i++) ok &= to_grid(cen[s * dim + i], scale, S.c[i]);
        ok &= to_grid(rad[s], scale, S.r) && S.r >= 0;
        if (vel)
            for (int i = 0; i < 3; i++) ok &= to_grid(vel[s * 3 + i], scale, S.v[i]);
        sph[s] = S;
        if (!ok) atomicOr(&scene_bad, 1);
    }
    __syncthreads();
    const bool bad = scene_bad != 0;

    const int lane = threadIdx.x & 31;
    const long long wpb = blockDim.x >> 5;
    const long long nwarps = (long long)gridDim.x * wpb;
    unsigned long long npos = 0, ninv = 0;
    for (long long wb = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); wb * 32 < n; wb += nwarps) {
        const long long i = wb * 32 + lane;
        int hit = 0;
        if (i < n) {
            int Q[W];
            bool ok = !bad;
#pragma unroll
            for (int k = 0; k < W; k++) ok &= to_grid(q[i * W + k], scale, Q[k]);
            if (KIND == NB_BOX3) ok = ok && Q[3] >= 0 && Q[4] >= 0 && Q[5] >= 0;
            if (!ok) {
                hit = 1;
                ninv++;
            } else {
                hit = union_hit<KIND>(Q, sph, ns, qexp);
            }
        }
        const unsigned b = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) {
            bits[wb] = b;
            npos += __popc(b);
        }
    }
    if (st) {
#pragma unroll
        for (int o = 16; o; o >>= 1) ninv += __shfl_xor_sync(0xffffffffu, ninv, o);
        if (lane == 0) {
            if (npos) atomicAdd(&st->n_positive, npos);
            if (ninv) atomicAdd(&st->n_invalid, ninv);
        }
    }
}

template <int KIND, int W>
nb_status launch(const nb_shape *sh, const float *q, int64_t n, uint32_t *bits, nb_label_stats *st,
                 cudaStream_t s) {
    auto k = label_kernel<KIND, W>;
    const size_t smem = (size_t)sh->n_spheres * sizeof(SphI);
    NB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 148;
    NB_CUDA(cudaGetDevice(&dev));
    NB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t warps = (n + 31) / 32;
    int64_t blocks = (warps + 7) / 8;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    if (blocks < 1) blocks = 1;
    k<<<(unsigned)blocks, 256, smem, s>>>(q, (long long)n, sh->n_spheres, sh->dim, sh->qexp, sh->centres, sh->radii,
                                          sh->vel, bits, st);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

}  // namespace

nb_status nb_launch_label(const nb_shape *sh, int kind, const float *q, int64_t n, uint32_t *bits,
                          nb_label_stats *st, cudaStream_t s) {
    if (st) NB_CUDA(cudaMemsetAsync(st, 0, sizeof(nb_label_stats), s));
    if (n == 0) return NB_OK;
    switch (kind) {
    case NB_POINT2: return launch<NB_POINT2, 2>(sh, q, n, bits, st, s);
    case NB_POINT3: return launch<NB_POINT3, 3>(sh, q, n, bits, st, s);
    case NB_POINT4T: return launch<NB_POINT4T, 4>(sh, q, n, bits, st, s);
    case NB_RAY3: return launch<NB_RAY3, 6>(sh, q, n, bits, st, s);
    case NB_PLANE3: return launch<NB_PLANE3, 4>(sh, q, n, bits, st, s);
    case NB_BOX3: return launch<NB_BOX3, 6>(sh, q, n, bits, st, s);
    default: return nb_fail(NB_EINVAL, "nb_label: unknown kind");
    }
}
