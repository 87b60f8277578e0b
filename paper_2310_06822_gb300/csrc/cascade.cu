// Learned-culler cascade: a scene of many objects, each bounded by a trained network,
// queried by rays through a hierarchy of tests (Sec. 1: a cheap conservative test in
// front of an expensive exact one; Eq. (Benefit) prices the trade):
//   stage 1  axis-aligned box of each object (classical bound), then the ball of radius R
//            around the object's centre that contains all its spheres; the ray is moved
//            into the object's frame and its origin advanced to where it enters the ball
//            (the form the object's network was trained on);
//   stage 2  the object's network (nb_query_grouped on the binned pairs);
//   stage 3  the exact test of the ray against the object's spheres, only for pairs the
//            network did not exclude.
// The plain path is stage 1 without the ball, then stage 3 on every pair.
#include "common.cuh"
#include "exact.cuh"

#include <algorithm>
#include <cmath>
#include <new>
#include <utility>
#include <vector>

using namespace nbexact;

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned NO_RAY = 0xffffffffu;

struct ObjS {
    float lo[3], hi[3], c[3];
};

// slab test of the half-line o + s d, s >= 0, against the box [lo, hi]; inv = 1 / d.
// Monotone under box inclusion: every rounding step is monotone in lo and hi, so a ray
// that passes a box passes every box that contains it.
__device__ __forceinline__ bool slab_hit(const float o[3], const float d[3], const float inv[3], const float lo[3],
                                         const float hi[3]) {
    float t0 = 0.f, t1 = INFINITY;
    bool hit = true;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        if (d[i] == 0.f) {
            hit = hit && o[i] >= lo[i] && o[i] <= hi[i];
        } else {
            float ta = (lo[i] - o[i]) * inv[i], tb = (hi[i] - o[i]) * inv[i];
            if (ta > tb) {
                const float tmp = ta;
                ta = tb;
                tb = tmp;
            }
            t0 = fmaxf(t0, ta);
            t1 = fminf(t1, tb);
        }
    }
    return hit && t0 <= t1;
}

// the ray in the frame of an object centred at c and the discriminant of its entry into the
// ball |x| = R (R2 = R^2): the ray meets the ball iff disc >= 0 and dd > 0
struct BallFrame {
    float w[3], b, dd, ww, disc;
};

__device__ __forceinline__ BallFrame ball_frame(const float o[3], const float d[3], const float c[3], float R2) {
    // object frame: w = o - c (exact on the grid); entry into |x| = R:
    // |w + s d|^2 = R^2, s = (-b - sqrt(b^2 - |d|^2 (|w|^2 - R^2))) / |d|^2
    BallFrame f;
    for (int i = 0; i < 3; i++) f.w[i] = __fsub_rn(o[i], c[i]);
    const float *w = f.w;
    f.b = __fadd_rn(__fadd_rn(__fmul_rn(w[0], d[0]), __fmul_rn(w[1], d[1])), __fmul_rn(w[2], d[2]));
    f.dd = __fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])), __fmul_rn(d[2], d[2]));
    f.ww = __fadd_rn(__fadd_rn(__fmul_rn(w[0], w[0]), __fmul_rn(w[1], w[1])), __fmul_rn(w[2], w[2]));
    // b^2 - dd (ww - R^2) = dd R^2 - |w x d|^2 (Lagrange), free of the cancellation
    // between the two large terms when the origin is far from the object
    const float cx = fmaf(w[1], d[2], -__fmul_rn(w[2], d[1]));
    const float cy = fmaf(w[2], d[0], -__fmul_rn(w[0], d[2]));
    const float cz = fmaf(w[0], d[1], -__fmul_rn(w[1], d[0]));
    const float cr2 = __fadd_rn(__fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy)), __fmul_rn(cz, cz));
    f.disc = __fsub_rn(__fmul_rn(f.dd, R2), cr2);
    return f;
}

__device__ __forceinline__ bool ball_met(const BallFrame &f) { return f.disc >= 0.f && f.dd > 0.f; }

// q6 = (entry point into the ball, direction) of a ray that meets it
__device__ __forceinline__ void ball_entry(const BallFrame &f, const float d[3], float R2, float q6[6]) {
    // smaller root without cancellation: s = c / (-b + sqrt(disc)) when -b > 0
    const float sq_disc = __fsqrt_rn(f.disc);
    const float cc = __fsub_rn(f.ww, R2);
    float s = -f.b > 0.f ? __fdiv_rn(cc, __fadd_rn(-f.b, sq_disc)) : __fdiv_rn(__fsub_rn(-f.b, sq_disc), f.dd);
    s = fmaxf(s, 0.f);
    for (int i = 0; i < 3; i++) {
        q6[i] = __fadd_rn(f.w[i], __fmul_rn(s, d[i]));
        q6[3 + i] = d[i];
    }
}

// the ray in the frame of an object centred at c, its origin moved to where it enters the
// ball: q6 = (entry point, direction); false if it misses the ball
__device__ __forceinline__ bool canon_entry(const float o[3], const float d[3], const float c[3], float R2,
                                            float q6[6]) {
    const BallFrame f = ball_frame(o, d, c, R2);
    if (!ball_met(f)) return false;
    ball_entry(f, d, R2, q6);
    return true;
}

template <bool CANON, bool SCATTER>
__global__ void __launch_bounds__(256)
    bin_kernel(int K, float R2, const float *__restrict__ aabb, const float *__restrict__ oc,
               const float *__restrict__ rays, long long n, unsigned long long *counts,
               const long long *__restrict__ offsets, uint32_t *__restrict__ pair_ray, float *__restrict__ pair_q,
               nb_cascade_stats *st) {
    extern __shared__ ObjS objs[];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        ObjS o;
        for (int i = 0; i < 3; i++) {
            o.lo[i] = aabb[k * 6 + i];
            o.hi[i] = aabb[k * 6 + 3 + i];
            o.c[i] = oc[k * 3 + i];
        }
        objs[k] = o;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned long long n_aabb = 0, n_ball = 0;
    const long long wpb = blockDim.x >> 5, nw = (long long)gridDim.x * wpb;
    for (long long wb = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); wb * 32 < n; wb += nw) {
        const long long r = wb * 32 + lane;
        const bool valid = r < n;
        float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 1.f}, inv[3];
        if (valid)
            for (int i = 0; i < 3; i++) {
                o[i] = rays[r * 6 + i];
                d[i] = rays[r * 6 + 3 + i];
            }
        for (int i = 0; i < 3; i++) inv[i] = 1.0f / d[i];  // +-inf for a zero component
        for (int k = 0; k < K; k++) {
            const ObjS ob = objs[k];
            // slab test of the half-line against the box (the box is conservative: inflated)
            const bool hit = valid && slab_hit(o, d, inv, ob.lo, ob.hi);
            float q6[6];
            bool keep = hit;
            if (CANON && hit) keep = canon_entry(o, d, ob.c, R2, q6);
            const unsigned bh = __ballot_sync(FULL, hit), bk = __ballot_sync(FULL, keep);
            if (lane == 0) {
                n_aabb += __popc(bh);
                n_ball += __popc(bk);
            }
            if (!bk) continue;
            unsigned base = 0;
            if (lane == 0) base = (unsigned)atomicAdd(counts + k, (unsigned long long)__popc(bk));
            if (SCATTER) {
                base = __shfl_sync(FULL, base, 0);
                if (keep) {
                    const long long row = offsets[k] + base + __popc(bk & ((1u << lane) - 1u));
                    pair_ray[row] = (uint32_t)r;
                    if (CANON)
                        for (int i = 0; i < 6; i++) pair_q[row * 6 + i] = q6[i];
                }
            }
        }
    }
    if (st && lane == 0 && !SCATTER) {
        if (n_aabb) atomicAdd(&st->aabb_pairs, n_aabb);
        if (n_ball) atomicAdd(&st->ball_pairs, n_ball);
    }
}

// Stage 1 through the 4-wide tree of object boxes: one ray per thread, depth-first with a
// short stack (the builder bounds the depth, so the stack never fills; the guard only keeps
// the writes in bounds).  The counting call counts kept pairs per object in shared memory
// and adds the block's counts to counts[] once at the end; the scatter call reserves each
// pair's row with one global atomic on its object's count (a few hundred thousand pairs per
// object, spread over the L2 slices: cheaper than walking the tree a second time to
// reserve rows per tile).
constexpr int BVH_STACK = 32;
constexpr int BVH_TPB = 256;
// nodes sit in shared memory at an odd stride of 29 words (a node is 28): lanes reading
// the same field of different nodes then hit different banks (at 28 words they would
// share 8 banks)
constexpr int NODE_WORDS = (int)(sizeof(nb_bvh4_node) / 4), NODE_STRIDE = NODE_WORDS + 1;

template <bool CANON, bool SCATTER>
__global__ void __launch_bounds__(BVH_TPB)
    bin_bvh_kernel(int K, int n_nodes, float R2, const nb_bvh4_node *__restrict__ nodes_g, const float *__restrict__ oc,
                   const float *__restrict__ rays, long long n, unsigned long long *counts,
                   const long long *__restrict__ offsets, uint32_t *__restrict__ pair_ray, float *__restrict__ pair_q,
                   nb_cascade_stats *st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *nodes = reinterpret_cast<float *>(smem_raw);
    float *cen = nodes + n_nodes * NODE_STRIDE;          // [K][3] object centres (canonical call)
    unsigned *hist = reinterpret_cast<unsigned *>(cen + (CANON ? 3 * K : 0));  // counting call only
    {
        const float *src = reinterpret_cast<const float *>(nodes_g);
        for (int i = threadIdx.x; i < n_nodes * NODE_WORDS; i += blockDim.x)
            nodes[(i / NODE_WORDS) * NODE_STRIDE + i % NODE_WORDS] = src[i];
        if (CANON)
            for (int i = threadIdx.x; i < 3 * K; i += blockDim.x) cen[i] = oc[i];
        if (!SCATTER)
            for (int k = threadIdx.x; k < K; k += blockDim.x) hist[k] = 0;
    }
    __syncthreads();
    unsigned long long n_aabb = 0, n_ball = 0;
    // Each lane walks its ray's tree depth-first, one node per iteration; a lane whose walk
    // ends takes its next ray at once instead of idling until the warp's longest walk ends.
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float o[3], d[3], inv[3];
    int stack[BVH_STACK];
    int sp = 0, node = 0;
    bool live = r < n;
    auto load_ray = [&]() {
        for (int i = 0; i < 3; i++) {
            o[i] = rays[r * 6 + i];
            d[i] = rays[r * 6 + 3 + i];
        }
        for (int i = 0; i < 3; i++) inv[i] = 1.0f / d[i];  // +-inf for a zero component
        node = 0;
        sp = 0;
    };
    if (live) load_ray();
    while (__any_sync(FULL, live)) {
        if (!live) continue;
        const nb_bvh4_node &nd = *reinterpret_cast<const nb_bvh4_node *>(nodes + node * NODE_STRIDE);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int ch = nd.child[c];
            if (ch == NB_BVH_EMPTY) continue;
            const float lo[3] = {nd.lo[0][c], nd.lo[1][c], nd.lo[2][c]};
            const float hi[3] = {nd.hi[0][c], nd.hi[1][c], nd.hi[2][c]};
            if (!slab_hit(o, d, inv, lo, hi)) continue;
            if (ch >= 0) {
                if (sp < BVH_STACK) stack[sp++] = ch;
                continue;
            }
            const int k = -1 - ch;  // a leaf: the pair (r, k) passes the box
            if (!SCATTER) {
                bool keep = true;
                if (CANON) keep = ball_met(ball_frame(o, d, cen + 3 * k, R2));
                n_aabb++;
                n_ball += keep;
                if (keep) atomicAdd(hist + k, 1u);
            } else {
                float q6[6];
                if (CANON && !canon_entry(o, d, cen + 3 * k, R2, q6)) continue;
                const long long row = offsets[k] + (long long)atomicAdd(counts + k, 1ull);
                pair_ray[row] = (uint32_t)r;
                if (CANON)
                    for (int i = 0; i < 6; i++) pair_q[row * 6 + i] = q6[i];
            }
        }
        if (sp > 0) {
            node = stack[--sp];
        } else {
            r += stride;
            live = r < n;
            if (live) load_ray();
        }
    }
    if (SCATTER) return;
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        if (hist[k]) atomicAdd(counts + k, (unsigned long long)hist[k]);
    if (st) {
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            n_aabb += __shfl_xor_sync(FULL, n_aabb, off);
            n_ball += __shfl_xor_sync(FULL, n_ball, off);
        }
        if ((threadIdx.x & 31) == 0) {
            if (n_aabb) atomicAdd(&st->aabb_pairs, n_aabb);
            if (n_ball) atomicAdd(&st->ball_pairs, n_ball);
        }
    }
}

// the exact ray-sphere predicate on grid integers: w = C - O, hit iff |w|^2 <= r^2 or
// (w.d > 0 and |w|^2 |d|^2 - (w.d)^2 <= r^2 |d|^2), in 64- and 128-bit integers
__device__ __forceinline__ bool ray_sphere_exact(const int Q[6], long long DD, int c0, int c1, int c2, int rr) {
    const int w0 = c0 - Q[0], w1 = c1 - Q[1], w2 = c2 - Q[2];
    const long long WW = sq(w0) + sq(w1) + sq(w2), RR = sq(rr);
    if (WW <= RR) return true;
    const long long SD = (long long)w0 * Q[3] + (long long)w1 * Q[4] + (long long)w2 * Q[5];
    return SD > 0 && (unsigned __int128)(unsigned long long)(WW - RR) * (unsigned long long)DD <=
                         (unsigned __int128)(unsigned long long)SD * (unsigned long long)SD;
}

// One warp per 32 consecutive rows.  Rows are binned by object, so a warp's rows nearly
// always belong to one object: then its lanes convert 32 of the object's spheres to grid
// integers at a time, one each, and every lane tests its ray against them through warp
// shuffles.  Rows of several objects in one warp are tested lane by lane.  Either way a
// pair's test stops at its first hit, and sphere_tests counts the predicates up to it.
__global__ void __launch_bounds__(256)
    exact_kernel(int K, int qexp, const long long *__restrict__ sph_off, const float *__restrict__ cen,
                 const float *__restrict__ rad, const float *__restrict__ rays, const uint32_t *__restrict__ pair_ray,
                 const long long *__restrict__ offsets, long long rows, const uint32_t *__restrict__ pass,
                 uint32_t *__restrict__ hits, uint32_t *__restrict__ pair_hits, nb_cascade_stats *st) {
    const float scale = ldexpf(1.0f, qexp);
    const int lane = threadIdx.x & 31;
    unsigned long long n_pairs = 0, n_tests = 0, n_hit = 0;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long g = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g * 32 < rows; g += nwarps) {
        const long long row = g * 32 + lane;
        const uint32_t r = row < rows ? pair_ray[row] : NO_RAY;
        const bool live = r != NO_RAY && !(pass && !((pass[row >> 5] >> (row & 31)) & 1u));
        if (!__any_sync(FULL, live)) continue;
        const long long rr = min(row, rows - 1);
        int lo = 0, hi = K - 1;  // object of this row: last k with offsets[k] <= row
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offsets[mid] <= rr) lo = mid; else hi = mid - 1;
        }
        int Q[6] = {0, 0, 0, 0, 0, 0};
        bool ok = true;
        if (live)
            for (int i = 0; i < 6; i++) ok &= to_grid(rays[(size_t)r * 6 + i], scale, Q[i]);
        const long long DD = sq(Q[3]) + sq(Q[4]) + sq(Q[5]);
        int h = live && !ok;  // an off-grid ray is a hit (conservative)
        bool done = !live || !ok;
        unsigned long long tests = 0;
        const int obj0 = __shfl_sync(FULL, lo, 0);
        if (__all_sync(FULL, lo == obj0)) {
            const long long s0 = sph_off[obj0], s1 = sph_off[obj0 + 1];
            for (long long sb = s0; sb < s1; sb += 32) {
                if (__all_sync(FULL, done)) break;
                int C[3] = {0, 0, 0}, Rr = 0;
                int sok = 1;
                if (sb + lane < s1) {
                    const long long sj = sb + lane;
                    sok = to_grid(cen[sj * 3], scale, C[0]) && to_grid(cen[sj * 3 + 1], scale, C[1]) &&
                          to_grid(cen[sj * 3 + 2], scale, C[2]) && to_grid(rad[sj], scale, Rr);
                }
                const int cnt = (int)min(32LL, s1 - sb);
                for (int j = 0; j < cnt; j++) {
                    const int c0 = __shfl_sync(FULL, C[0], j), c1 = __shfl_sync(FULL, C[1], j);
                    const int c2 = __shfl_sync(FULL, C[2], j), rj = __shfl_sync(FULL, Rr, j);
                    const int okj = __shfl_sync(FULL, sok, j);
                    if (done) continue;
                    tests++;
                    if (!okj || ray_sphere_exact(Q, DD, c0, c1, c2, rj)) {
                        h = 1;  // an off-grid sphere counts as hit (conservative)
                        done = true;
                    }
                }
            }
        } else {
            for (long long sj = sph_off[lo]; !done && sj < sph_off[lo + 1]; sj++) {
                int C[3], Rr;
                const bool sok = to_grid(cen[sj * 3], scale, C[0]) && to_grid(cen[sj * 3 + 1], scale, C[1]) &&
                                 to_grid(cen[sj * 3 + 2], scale, C[2]) && to_grid(rad[sj], scale, Rr);
                tests++;
                if (!sok || ray_sphere_exact(Q, DD, C[0], C[1], C[2], Rr)) {
                    h = 1;
                    done = true;
                }
            }
        }
        if (live) {
            n_pairs++;
            n_tests += tests;
            if (h) {
                n_hit++;
                if (hits) atomicOr(hits + (r >> 5), 1u << (r & 31));
                if (pair_hits) atomicOr(pair_hits + (row >> 5), 1u << (row & 31));
            }
        }
    }
    if (st) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            n_pairs += __shfl_xor_sync(FULL, n_pairs, o);
            n_tests += __shfl_xor_sync(FULL, n_tests, o);
            n_hit += __shfl_xor_sync(FULL, n_hit, o);
        }
        if (lane == 0) {
            if (n_pairs) atomicAdd(&st->exact_pairs, n_pairs);
            if (n_tests) atomicAdd(&st->sphere_tests, n_tests);
            if (n_hit) atomicAdd(&st->hit_pairs, n_hit);
        }
    }
}

int num_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

nb_status check_scene(const nb_scene *sc) {
    if (!sc) return nb_fail(NB_EINVAL, "cascade: null scene");
    if (sc->n_objects < 1 || sc->n_objects > 4096) return nb_fail(NB_EINVAL, "cascade: n_objects must be 1..4096");
    if (sc->qexp < 8 || sc->qexp > 24) return nb_fail(NB_EINVAL, "cascade: qexp must be 8..24");
    if (!(sc->ball_radius > 0)) return nb_fail(NB_EINVAL, "cascade: ball_radius must be > 0");
    if (!sc->sphere_offsets || !sc->centres || !sc->radii || !sc->obj_centre || !sc->aabb)
        return nb_fail(NB_EINVAL, "cascade: null scene array");
    return NB_OK;
}

}  // namespace

extern "C" nb_status nb_cascade_bin(const nb_scene *scene, const float *rays, int64_t n, int32_t canonical,
                                    unsigned long long *counts, const int64_t *offsets, uint32_t *pair_ray,
                                    float *pair_q, nb_cascade_stats *dev_stats, void *stream) {
    nb_status st = check_scene(scene);
    if (st != NB_OK) return st;
    if (n < 0 || n >= ((int64_t)1 << 32) - 1) return nb_fail(NB_EINVAL, "nb_cascade_bin: n must be in [0, 2^32 - 1)");
    if (!counts || (n > 0 && !rays)) return nb_fail(NB_EINVAL, "nb_cascade_bin: null pointer");
    const bool scatter = offsets != nullptr;
    if (scatter && (!pair_ray || (canonical && !pair_q)))
        return nb_fail(NB_EINVAL, "nb_cascade_bin: scatter needs pair_ray (and pair_q when canonical)");
    cudaStream_t s = (cudaStream_t)stream;
    const int K = scene->n_objects;
    NB_CUDA(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * K, s));
    if (dev_stats && !scatter) NB_CUDA(cudaMemsetAsync(dev_stats, 0, sizeof(nb_cascade_stats), s));
    if (n == 0) return NB_OK;
    const size_t smem = sizeof(ObjS) * K;
    int64_t grid = (n + 255) / 256;
    if (grid > (int64_t)num_sms() * 8) grid = (int64_t)num_sms() * 8;
    const float R2 = scene->ball_radius * scene->ball_radius;
#define NB_BIN(C, S)                                                                                              \
    do {                                                                                                          \
        NB_CUDA(cudaFuncSetAttribute(bin_kernel<C, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        bin_kernel<C, S><<<(unsigned)grid, 256, smem, s>>>(K, R2, scene->aabb, scene->obj_centre, rays, (long long)n, \
                                                           counts, (const long long *)offsets, pair_ray, pair_q,   \
                                                           dev_stats);                                            \
    } while (0)
    if (canonical && scatter) NB_BIN(true, true);
    else if (canonical) NB_BIN(true, false);
    else if (scatter) NB_BIN(false, true);
    else NB_BIN(false, false);
#undef NB_BIN
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

extern "C" nb_status nb_cascade_exact(const nb_scene *scene, const float *rays, const uint32_t *pair_ray,
                                      const int64_t *offsets, int64_t rows, const uint32_t *pass_bits,
                                      uint32_t *ray_hits, uint32_t *pair_hits, nb_cascade_stats *dev_stats,
                                      void *stream) {
    nb_status st = check_scene(scene);
    if (st != NB_OK) return st;
    if (rows < 0) return nb_fail(NB_EINVAL, "nb_cascade_exact: negative rows");
    if (rows > 0 && (!rays || !pair_ray || !offsets || (!ray_hits && !pair_hits)))
        return nb_fail(NB_EINVAL, "nb_cascade_exact: null pointer");
    if (rows == 0) return NB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t grid = (rows + 255) / 256;
    if (grid > (int64_t)num_sms() * 8) grid = (int64_t)num_sms() * 8;
    exact_kernel<<<(unsigned)grid, 256, 0, s>>>(scene->n_objects, scene->qexp, (const long long *)scene->sphere_offsets,
                                               scene->centres, scene->radii, rays, pair_ray,
                                               (const long long *)offsets, (long long)rows, pass_bits, ray_hits, pair_hits,
                                               dev_stats);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// ------------------------------------------------------------------ spatial index of objects
// Host builder: Morton order of the object box centres, median splits two levels at a time
// (four children per node), child boxes the exact unions of the object boxes below them.
namespace {

constexpr int BVH_MAX_DEPTH = 10;  // 3 * depth + 1 <= BVH_STACK entries

uint32_t spread10(uint32_t v) {  // bits b9..b0 -> positions 27, 24, ..., 0
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

struct Bvh4Builder {
    const float *aabb;
    std::vector<int> order;
    std::vector<nb_bvh4_node> nodes;
    int depth = 0;

    void box(int a, int b, float lo[3], float hi[3]) const {
        for (int i = 0; i < 3; i++) {
            lo[i] = INFINITY;
            hi[i] = -INFINITY;
        }
        for (int j = a; j < b; j++) {
            const float *bx = aabb + (size_t)order[j] * 6;
            for (int i = 0; i < 3; i++) {
                lo[i] = std::min(lo[i], bx[i]);
                hi[i] = std::max(hi[i], bx[3 + i]);
            }
        }
    }

    int build(int a, int b, int level) {
        const int me = (int)nodes.size();
        nodes.push_back(nb_bvh4_node{});
        depth = std::max(depth, level);
        int cut[5], nc;
        if (b - a <= 4) {
            nc = b - a;
            for (int c = 0; c <= nc; c++) cut[c] = a + c;
        } else {
            const int m = a + (b - a) / 2;
            nc = 4;
            cut[0] = a;
            cut[1] = a + (m - a) / 2;
            cut[2] = m;
            cut[3] = m + (b - m) / 2;
            cut[4] = b;
        }
        nb_bvh4_node nd{};
        for (int c = 0; c < 4; c++) {
            if (c >= nc) {
                nd.child[c] = NB_BVH_EMPTY;
                continue;
            }
            float lo[3], hi[3];
            box(cut[c], cut[c + 1], lo, hi);
            for (int i = 0; i < 3; i++) {
                nd.lo[i][c] = lo[i];
                nd.hi[i][c] = hi[i];
            }
            nd.child[c] = cut[c + 1] - cut[c] == 1 ? -1 - order[cut[c]] : build(cut[c], cut[c + 1], level + 1);
        }
        nodes[me] = nd;
        return me;
    }
};

nb_status build_bvh4(const float *aabb, int K, std::vector<nb_bvh4_node> &nodes, int &depth) {
    for (int k = 0; k < K * 6; k++)
        if (!std::isfinite(aabb[k])) return nb_fail(NB_EINVAL, "cascade index: non-finite object box");
    double mn[3], mx[3];
    for (int i = 0; i < 3; i++) {
        mn[i] = INFINITY;
        mx[i] = -INFINITY;
    }
    std::vector<double> cen((size_t)K * 3);
    for (int k = 0; k < K; k++)
        for (int i = 0; i < 3; i++) {
            const double c = 0.5 * ((double)aabb[k * 6 + i] + (double)aabb[k * 6 + 3 + i]);
            cen[(size_t)k * 3 + i] = c;
            mn[i] = std::min(mn[i], c);
            mx[i] = std::max(mx[i], c);
        }
    std::vector<std::pair<uint32_t, int>> key((size_t)K);
    for (int k = 0; k < K; k++) {
        uint32_t code = 0;
        for (int i = 0; i < 3; i++) {
            const double u = mx[i] > mn[i] ? (cen[(size_t)k * 3 + i] - mn[i]) / (mx[i] - mn[i]) : 0.0;
            const uint32_t q = (uint32_t)std::min(1023.0, std::max(0.0, std::floor(u * 1024.0)));
            code |= spread10(q) << (2 - i);  // x in the highest bit of each triple
        }
        key[k] = {code, k};
    }
    std::sort(key.begin(), key.end());
    Bvh4Builder b;
    b.aabb = aabb;
    b.order.resize((size_t)K);
    for (int k = 0; k < K; k++) b.order[k] = key[k].second;
    b.nodes.reserve((size_t)std::max(1, K - 1));
    b.build(0, K, 1);
    if (b.depth > BVH_MAX_DEPTH) return nb_fail(NB_EINVAL, "cascade index: tree too deep");
    nodes.swap(b.nodes);
    depth = b.depth;
    return NB_OK;
}

}  // namespace

struct nb_cascade_index {
    int K = 0, n_nodes = 0, depth = 0;
    nb_bvh4_node *nodes = nullptr;  // device
};

extern "C" int32_t nb_cascade_index_max_nodes(int32_t n_objects) { return n_objects <= 2 ? 1 : n_objects - 1; }

extern "C" nb_status nb_cascade_index_build_host(const float *aabb, int32_t n_objects, nb_bvh4_node *nodes,
                                                 int32_t *n_nodes, int32_t *depth) {
    if (n_objects < 1 || n_objects > 4096) return nb_fail(NB_EINVAL, "cascade index: n_objects must be 1..4096");
    if (!aabb || !nodes || !n_nodes || !depth) return nb_fail(NB_EINVAL, "cascade index: null pointer");
    std::vector<nb_bvh4_node> v;
    int dep = 0;
    const nb_status st = build_bvh4(aabb, n_objects, v, dep);
    if (st != NB_OK) return st;
    std::copy(v.begin(), v.end(), nodes);
    *n_nodes = (int32_t)v.size();
    *depth = dep;
    return NB_OK;
}

extern "C" nb_status nb_cascade_index_create(const nb_scene *scene, nb_cascade_index **out) {
    nb_status st = check_scene(scene);
    if (st != NB_OK) return st;
    if (!out) return nb_fail(NB_EINVAL, "nb_cascade_index_create: null out");
    *out = nullptr;
    const int K = scene->n_objects;
    std::vector<float> h((size_t)K * 6);
    NB_CUDA(cudaMemcpy(h.data(), scene->aabb, h.size() * sizeof(float), cudaMemcpyDeviceToHost));
    std::vector<nb_bvh4_node> v;
    int dep = 0;
    st = build_bvh4(h.data(), K, v, dep);
    if (st != NB_OK) return st;
    nb_cascade_index *ix = new (std::nothrow) nb_cascade_index;
    if (!ix) return nb_fail(NB_ENOMEM, "nb_cascade_index_create: out of host memory");
    if (cudaMalloc(&ix->nodes, v.size() * sizeof(nb_bvh4_node)) != cudaSuccess) {
        cudaGetLastError();
        delete ix;
        return nb_fail(NB_ENOMEM, "nb_cascade_index_create: device allocation failed");
    }
    if (cudaMemcpy(ix->nodes, v.data(), v.size() * sizeof(nb_bvh4_node), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(ix->nodes);
        delete ix;
        return nb_fail(NB_ECUDA, "nb_cascade_index_create: upload failed");
    }
    ix->K = K;
    ix->n_nodes = (int)v.size();
    ix->depth = dep;
    *out = ix;
    return NB_OK;
}

extern "C" nb_status nb_cascade_index_destroy(nb_cascade_index *index) {
    if (!index) return NB_OK;
    cudaFree(index->nodes);
    delete index;
    return NB_OK;
}

extern "C" nb_status nb_cascade_bin_indexed(const nb_cascade_index *index, const nb_scene *scene, const float *rays,
                                            int64_t n, int32_t canonical, unsigned long long *counts,
                                            const int64_t *offsets, uint32_t *pair_ray, float *pair_q,
                                            nb_cascade_stats *dev_stats, void *stream) {
    nb_status st = check_scene(scene);
    if (st != NB_OK) return st;
    if (!index) return nb_fail(NB_EINVAL, "nb_cascade_bin_indexed: null index");
    if (index->K != scene->n_objects) return nb_fail(NB_EINVAL, "nb_cascade_bin_indexed: index of another scene");
    if (n < 0 || n >= ((int64_t)1 << 32) - 1)
        return nb_fail(NB_EINVAL, "nb_cascade_bin_indexed: n must be in [0, 2^32 - 1)");
    if (!counts || (n > 0 && !rays)) return nb_fail(NB_EINVAL, "nb_cascade_bin_indexed: null pointer");
    const bool scatter = offsets != nullptr;
    if (scatter && (!pair_ray || (canonical && !pair_q)))
        return nb_fail(NB_EINVAL, "nb_cascade_bin_indexed: scatter needs pair_ray (and pair_q when canonical)");
    cudaStream_t s = (cudaStream_t)stream;
    const int K = scene->n_objects;
    NB_CUDA(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * K, s));
    if (dev_stats && !scatter) NB_CUDA(cudaMemsetAsync(dev_stats, 0, sizeof(nb_cascade_stats), s));
    if (n == 0) return NB_OK;
    const size_t smem = (size_t)index->n_nodes * NODE_STRIDE * 4 + (canonical ? (size_t)K * 12 : 0) +
                        (scatter ? 0 : (size_t)K * 4);
    int dev = 0, optin = 0;
    NB_CUDA(cudaGetDevice(&dev));
    NB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (smem > (size_t)optin) return nb_fail(NB_EUNSUPPORTED, "nb_cascade_bin_indexed: tree exceeds shared memory");
    const float R2 = scene->ball_radius * scene->ball_radius;
    const long long blocks = (n + BVH_TPB - 1) / BVH_TPB;
#define NB_BIN_BVH(C, S)                                                                                           \
    do {                                                                                                           \
        NB_CUDA(cudaFuncSetAttribute(bin_bvh_kernel<C, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        int per_sm = 1;                                                                                            \
        NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bin_bvh_kernel<C, S>, BVH_TPB, smem));      \
        const long long grid = std::min<long long>(blocks, (long long)num_sms() * std::max(1, per_sm));             \
        bin_bvh_kernel<C, S><<<(unsigned)grid, BVH_TPB, smem, s>>>(K, index->n_nodes, R2, index->nodes,             \
                                                                   scene->obj_centre, rays, (long long)n, counts,   \
                                                                   (const long long *)offsets, pair_ray, pair_q,    \
                                                                   dev_stats);                                      \
    } while (0)
    if (canonical && scatter) NB_BIN_BVH(true, true);
    else if (canonical) NB_BIN_BVH(true, false);
    else if (scatter) NB_BIN_BVH(false, true);
    else NB_BIN_BVH(false, false);
#undef NB_BIN_BVH
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}
