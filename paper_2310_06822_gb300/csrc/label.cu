// Exact labeler: y = g(r) of Sec. 3.1 for a union of closed balls.
//
// Alg. 1 labels a region by Any(f(SampleRegion(r))); here the region is tested
// against every ball analytically, in exact integer arithmetic on the 2^-qexp grid,
// so the label is the query function itself, inclusive of the surface (Sec. 3.1:
// the indicator is 1 inside and on the surface).  An FP32 pre-filter settles the
// tests that are far from tangency (exact.cuh); only the rest take the integer path.
#include "common.cuh"
#include "exact.cuh"

namespace {

using namespace nbexact;

template <int KIND, int W>
__global__ void __launch_bounds__(256) label_kernel(const float *__restrict__ q, long long n, int ns, int dim,
                                                    int qexp, const float *__restrict__ cen,
                                                    const float *__restrict__ rad, const float *__restrict__ vel,
                                                    uint32_t *__restrict__ bits, nb_label_stats *st) {
    extern __shared__ SphI sph[];
    SphF *sphf = reinterpret_cast<SphF *>(sph + ns);  // the same balls as exact floats for the filter
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
        SphF F;
        for (int i = 0; i < 3; i++) F.c[i] = i < dim ? cen[s * dim + i] : 0.f;
        F.rr = __fmul_rn(rad[s], rad[s]);
        sphf[s] = F;
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
            float qf[W];
            bool ok = !bad;
#pragma unroll
            for (int k = 0; k < W; k++) {
                qf[k] = q[i * W + k];
                ok &= to_grid(qf[k], scale, Q[k]);
            }
            if (KIND == NB_BOX3) ok = ok && Q[3] >= 0 && Q[4] >= 0 && Q[5] >= 0;
            if (!ok) {
                hit = 1;
                ninv++;
            } else {
                // FP32 pre-filter, the exact integer test where it cannot be sure
                hit = union_hit_filtered<KIND>(qf, Q, sphf, sph, ns, qexp);
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
    const size_t smem = (size_t)sh->n_spheres * (sizeof(SphI) + sizeof(SphF));
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
