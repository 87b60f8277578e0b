// Neural early-out (Sec. 3.3): a small network trained as a conservative bound of the
// complement 1 - g runs first; where it decides "outside the complement" the query is
// certainly inside (g = 1) and the late network is skipped.  The remaining rows are
// compacted, gathered and decided by the late network, and their bits scattered back.
#include "common.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

// out_bits <- rows the early network settles (inside), 0 elsewhere; idx <- the other rows
__global__ void early_compact_kernel(const uint32_t *__restrict__ bits_e, long long n, unsigned *count,
                                     unsigned *__restrict__ idx, uint32_t *__restrict__ out_bits) {
    const int lane = threadIdx.x & 31;
    const long long nw = (n + 31) / 32;
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw;
         w += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long i = w * 32 + lane;
        const bool valid = i < n;
        const bool late = valid && ((bits_e[w] >> lane) & 1u);
        const unsigned b = __ballot_sync(FULL, late);
        const unsigned v = __ballot_sync(FULL, valid);
        if (lane == 0) out_bits[w] = ~b & v;
        if (!b) continue;
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(count, (unsigned)__popc(b));
        base = __shfl_sync(FULL, base, 0);
        if (late) idx[base + __popc(b & ((1u << lane) - 1u))] = (unsigned)i;
    }
}

__global__ void early_gather_kernel(const float *__restrict__ q, int w, const unsigned *__restrict__ idx, long long m,
                                    float *__restrict__ qc) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m * w;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / w;
        qc[e] = q[(size_t)idx[j] * w + (e - j * w)];
    }
}

__global__ void early_scatter_kernel(const uint32_t *__restrict__ bits_c, const unsigned *__restrict__ idx, long long m,
                                     uint32_t *out_bits) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x)
        if ((bits_c[j >> 5] >> (j & 31)) & 1u) {
            const unsigned i = idx[j];
            atomicOr(out_bits + (i >> 5), 1u << (i & 31));
        }
}

int grid_for(long long work, int per_block) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long g = (work + per_block - 1) / per_block;
    if (g > (long long)sms * 8) g = (long long)sms * 8;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

nb_status nb_launch_early_compact(const uint32_t *bits_e, int64_t n, unsigned *count, unsigned *idx, uint32_t *out_bits,
                                  cudaStream_t s) {
    NB_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned), s));
    early_compact_kernel<<<grid_for((n + 31) / 32 * 32, 256), 256, 0, s>>>(bits_e, (long long)n, count, idx, out_bits);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_launch_early_gather(const float *q, int w, const unsigned *idx, int64_t m, float *qc, cudaStream_t s) {
    if (m == 0) return NB_OK;
    early_gather_kernel<<<grid_for(m * w, 256), 256, 0, s>>>(q, w, idx, (long long)m, qc);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status nb_launch_early_scatter(const uint32_t *bits_c, const unsigned *idx, int64_t m, uint32_t *out_bits,
                                  cudaStream_t s) {
    if (m == 0) return NB_OK;
    early_scatter_kernel<<<grid_for(m, 256), 256, 0, s>>>(bits_c, idx, (long long)m, out_bits);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

namespace {
__global__ void bits_not_kernel(const uint32_t *__restrict__ in, long long n, uint32_t *__restrict__ out) {
    const long long nw = (n + 31) / 32;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (long long)gridDim.x * blockDim.x) {
        const long long rest = n - w * 32;
        const uint32_t mask = rest >= 32 ? 0xffffffffu : ((1u << rest) - 1u);
        out[w] = ~in[w] & mask;
    }
}
}  // namespace

nb_status nb_launch_bits_not(const uint32_t *in, int64_t n, uint32_t *out, cudaStream_t s) {
    bits_not_kernel<<<grid_for((n + 31) / 32, 256), 256, 0, s>>>(in, (long long)n, out);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// Broad-phase three-way class (Sec. 4.4, inverted bounds): decision 0 of the outer bound is
// "certainly outside", decision 0 of the complement bound "certainly inside"; neither, or
// both (a conflict), leaves the query to the exact test.  One thread per query, one byte
// out; counts reduced per warp.
namespace {
__global__ void three_way_kernel(const uint32_t *__restrict__ bits_o, const uint32_t *__restrict__ bits_i, long long n,
                                 uint8_t *__restrict__ codes, nb_three_way_stats *st) {
    unsigned long long c_out = 0, c_in = 0, c_nei = 0, c_conf = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const bool out = !((bits_o[i >> 5] >> (i & 31)) & 1u);
        const bool in = !((bits_i[i >> 5] >> (i & 31)) & 1u);
        const uint8_t c = (out && !in) ? 0 : ((in && !out) ? 1 : 2);
        codes[i] = c;
        c_out += c == 0;
        c_in += c == 1;
        c_nei += c == 2;
        c_conf += in && out;
    }
    if (!st) return;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        c_out += __shfl_xor_sync(FULL, c_out, o);
        c_in += __shfl_xor_sync(FULL, c_in, o);
        c_nei += __shfl_xor_sync(FULL, c_nei, o);
        c_conf += __shfl_xor_sync(FULL, c_conf, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (c_out) atomicAdd((unsigned long long *)&st->n_out, c_out);
        if (c_in) atomicAdd((unsigned long long *)&st->n_in, c_in);
        if (c_nei) atomicAdd((unsigned long long *)&st->n_neither, c_nei);
        if (c_conf) atomicAdd((unsigned long long *)&st->n_conflict, c_conf);
    }
}
}  // namespace

nb_status nb_launch_three_way(const uint32_t *bits_outer, const uint32_t *bits_inner, int64_t n, uint8_t *codes,
                              nb_three_way_stats *st, cudaStream_t s) {
    three_way_kernel<<<grid_for(n, 256), 256, 0, s>>>(bits_outer, bits_inner, (long long)n, codes, st);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}
