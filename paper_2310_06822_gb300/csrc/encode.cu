// The paper's query parameterisation (Suppl. "Parameterization"): rays as start and
// direction, boxes as their two corners, planes as a point p0 on the plane and the normal.
// The library's own encodings carry the same information (box: centre and half-extents;
// plane: normal and offset of n . x = off); this converts them, one query per thread, for
// networks trained on the paper's inputs.  Box corners c -/+ e are exact for grid values
// (both terms are multiples of the grid step well inside FP32's 24 bits); the plane point
// p0 = off n / |n|^2 is the plane's point nearest the origin, each operation correctly
// rounded in FP32.
#include <algorithm>

#include "common.cuh"

namespace {

template <int KIND>
__global__ void encode_paper_kernel(const float *__restrict__ q, long long n, float *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (KIND == NB_BOX3) {
            const float *x = q + i * 6;
            float *o = out + i * 6;
            for (int d = 0; d < 3; d++) {
                o[d] = __fsub_rn(x[d], x[3 + d]);
                o[3 + d] = __fadd_rn(x[d], x[3 + d]);
            }
        } else {  // NB_PLANE3
            const float *x = q + i * 4;
            float *o = out + i * 6;
            const float nn = __fadd_rn(__fadd_rn(__fmul_rn(x[0], x[0]), __fmul_rn(x[1], x[1])), __fmul_rn(x[2], x[2]));
            const float s = __fdiv_rn(x[3], nn);
            for (int d = 0; d < 3; d++) {
                o[d] = __fmul_rn(s, x[d]);
                o[3 + d] = x[d];
            }
        }
    }
}

}  // namespace

extern "C" nb_status nb_encode_paper(int32_t kind, const float *q, int64_t n, float *out, void *stream) {
    if (kind < NB_POINT2 || kind > NB_BOX3) return nb_fail(NB_EINVAL, "nb_encode_paper: unknown kind");
    if (n < 0) return nb_fail(NB_EINVAL, "nb_encode_paper: n must be >= 0");
    if (n == 0) return NB_OK;
    if (!q || !out) return nb_fail(NB_EINVAL, "nb_encode_paper: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    static const int width[] = {2, 3, 4, 6, 4, 6};
    if (kind != NB_BOX3 && kind != NB_PLANE3) {  // points and rays: the same encoding
        NB_CUDA(cudaMemcpyAsync(out, q, (size_t)n * width[kind] * sizeof(float), cudaMemcpyDeviceToDevice, s));
        return NB_OK;
    }
    int dev = 0, sms = 148;
    NB_CUDA(cudaGetDevice(&dev));
    NB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long grid = std::min<long long>((n + 255) / 256, (long long)sms * 8);
    if (kind == NB_BOX3) encode_paper_kernel<NB_BOX3><<<(unsigned)grid, 256, 0, s>>>(q, (long long)n, out);
    else encode_paper_kernel<NB_PLANE3><<<(unsigned)grid, 256, 0, s>>>(q, (long long)n, out);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}
