// Grouped launches: many per-object bounding networks of one architecture, each with
// its own (uneven) number of samples, trained and queried in one persistent launch.
//
// The paper trains one network per object and rearranges objects without retraining
// (Sec. 2); its training loop is Sec. 3.4.  Here n_objects networks are stacked: the
// parameters of object o start at o * P.  A plan splits every object's rows (which are
// contiguous in one concatenated query array) into work items of at most `chunk` rows;
// persistent CTAs walk the items.  Training writes one gradient partial per item and a
// deterministic reduction sums each object's items in item order before its Adam step,
// so a step's result does not depend on scheduling.  An optional device-side schedule
// (alpha[t], Adam bias corrections[t], a device step counter) lets a whole training loop
// be captured in a CUDA graph with no host arguments changing between steps.
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "group.cuh"
#include "mlp_tile.cuh"

using namespace nbf32;

namespace {

int num_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

int nj_for(int maxw) {
    int nj = (maxw + 15) / 16;
    return nj <= 1 ? 1 : nj <= 2 ? 2 : nj <= 4 ? 4 : nj <= 8 ? 8 : 16;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------------------------------ training
template <int NJ, int TM>
__global__ void __launch_bounds__(256)
    group_train_kernel(MlpDesc d, long long P, const PlanItem *__restrict__ items, int n_items,
                       const long long *__restrict__ offsets, const float *__restrict__ q,
                       const uint32_t *__restrict__ labels, float alpha_arg, const float *sched_alpha,
                       const int *d_step, int sched_T, float beta, const TauF *taus, float *__restrict__ partial,
                       long long S, float *loss_partial, nb_step_stats *st) {
    extern __shared__ float smem[];
    __shared__ float zs[TM], dz[TM], ls[TM];
    const int t = threadIdx.x;
    float alpha = alpha_arg;
    if (sched_alpha) alpha = sched_alpha[min(*d_step, sched_T - 1)];
    unsigned long long c_fn = 0, c_fp = 0, c_nf = 0;
    int k0, k1;
    item_range(n_items, k0, k1);
    for (int it = k0; it < k1; it++) {
        const PlanItem w = items[it];
        MlpDesc dd = d;
        dd.p = d.p + (size_t)w.obj * P;
        const float inv_n = 1.0f / (float)(offsets[w.obj + 1] - offsets[w.obj]);
        float *slot = partial + (size_t)it * S;
        float lossacc = 0.f;
        for (long long base = w.row0; base < w.row1; base += TM) {
            const int rows = (int)min((long long)TM, w.row1 - base);
            train_tile<NJ, TM>(dd, q, labels, base, rows, alpha, beta, inv_n, taus[w.obj], slot, smem, zs, dz, ls,
                               lossacc, c_fn, c_fp, c_nf);
        }
        if (t == 0) loss_partial[it] = lossacc;
    }
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

// Per object: sum its items' partials in item order, keep the gradient, one Adam step.
__global__ void __launch_bounds__(256)
    group_adam_kernel(long long P, long long S, int n_objects, const int *__restrict__ obj_items,
                      const float *__restrict__ partial,
                      float *__restrict__ params, float *__restrict__ m, float *__restrict__ v,
                      float *__restrict__ grad, float lr, float b1, float b2, float eps, float c1_arg,
                      float sqrt_c2_arg, const float *sched_c1, const float *sched_sqrt_c2, const int *d_step,
                      int sched_T) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n_objects * P) return;
    const int o = (int)(idx / P);
    const long long p = idx % P;
    float c1 = c1_arg, sqrt_c2 = sqrt_c2_arg;
    if (sched_c1) {
        const int t = min(*d_step, sched_T - 1);
        c1 = sched_c1[t];
        sqrt_c2 = sched_sqrt_c2[t];
    }
    float g = 0.f;
    for (int it = obj_items[o]; it < obj_items[o + 1]; it++) g += partial[(size_t)it * S + p];
    grad[idx] = g;
    const float mm = b1 * m[idx] + (1.f - b1) * g;
    const float vv = b2 * v[idx] + (1.f - b2) * g * g;
    m[idx] = mm;
    v[idx] = vv;
    const float denom = sqrtf(vv) / sqrt_c2 + eps;
    params[idx] = params[idx] - (lr / c1) * (mm / denom);
}

// Mean over objects of each object's mean loss; advances the device step counter.
__global__ void group_loss_kernel(int n_objects, const int *__restrict__ obj_items,
                                  const long long *__restrict__ offsets, const float *__restrict__ loss_partial,
                                  nb_step_stats *st, int *d_step) {
    __shared__ float red[256];
    float acc = 0.f;
    for (int o = threadIdx.x; o < n_objects; o += blockDim.x) {
        float s = 0.f;
        for (int it = obj_items[o]; it < obj_items[o + 1]; it++) s += loss_partial[it];
        const long long cnt = offsets[o + 1] - offsets[o];
        if (cnt > 0) acc += s / (float)cnt;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (st) st->loss = red[0] / (float)n_objects;
        if (d_step) *d_step += 1;
    }
}

// ------------------------------------------------------------------ queries (FP32 form)
template <int NJ>
__global__ void __launch_bounds__(256)
    group_fwd_f32_kernel(MlpDesc d, long long P, const PlanItem *__restrict__ items, int n_items,
                         const float *__restrict__ q, const TauF *taus, float margin, uint32_t *__restrict__ bits,
                         float *__restrict__ logits, nb_query_stats *st, unsigned *flag_count, unsigned *flag_idx) {
    extern __shared__ float smem[];
    __shared__ float zs[TMF];
    const int t = threadIdx.x, lane = t & 31;
    unsigned long long c_in = 0, c_flag = 0, c_nf = 0;
    int k0, k1;
    item_range(n_items, k0, k1);
    for (int it = k0; it < k1; it++) {
        const PlanItem w = items[it];
        MlpDesc dd = d;
        dd.p = d.p + (size_t)w.obj * P;
        const TauF tau = taus[w.obj];
        for (long long base = w.row0; base < w.row1; base += TMF) {
            const int rows = (int)min((long long)TMF, w.row1 - base);
            fwd_tile<NJ>(dd, q, base, rows, tau, margin, bits, logits, flag_count, flag_idx, smem, zs, c_in, c_flag,
                         c_nf);
        }
    }
    if (st && lane == 0 && t < TMF) {
        if (c_in) atomicAdd(&st->n_inside, c_in);
        if (c_flag) atomicAdd(&st->n_flagged, c_flag);
        if (c_nf) atomicAdd(&st->n_nonfinite, c_nf);
    }
}

template <int NJ, int TM>
nb_status group_train_launch(const nb_group *g, const nb_plan *pl, const float *q, const uint32_t *labels,
                             float alpha, bool sched, float beta, float *partial, float *loss_partial,
                             nb_step_stats *st, cudaStream_t s) {
    constexpr int KP = 16 * NJ + 1;
    const size_t smem = (size_t)((g->L + 2) * TM * KP + KC * (16 * NJ + 1)) * sizeof(float);
    auto k = group_train_kernel<NJ, TM>;
    NB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 1;
    NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem));
    int grid = num_sms() * (per_sm < 1 ? 1 : per_sm);
    if (grid > pl->n_items) grid = pl->n_items;
    if (grid < 1) grid = 1;
    MlpDesc d = nb_group_desc(g);
    k<<<grid, 256, smem, s>>>(d, g->P, pl->items, pl->n_items, pl->offsets, q, labels, alpha,
                              sched ? g->sched_alpha : nullptr, g->d_step, g->sched_T, beta, g->d_tau, partial,
                              (long long)g->S, loss_partial, st);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

template <int NJ>
nb_status group_fwd_launch(const nb_group *g, const nb_plan *pl, const float *q, float margin, uint32_t *bits,
                           float *logits, nb_query_stats *st, QueryWs ws, cudaStream_t s) {
    constexpr int KP = 16 * NJ + 1;
    const size_t smem = (size_t)(2 * TMF * KP + KC * (16 * NJ + 1)) * sizeof(float);
    auto k = group_fwd_f32_kernel<NJ>;
    NB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 1;
    NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem));
    int grid = num_sms() * (per_sm < 1 ? 1 : per_sm);
    if (grid > pl->n_items) grid = pl->n_items;
    if (grid < 1) grid = 1;
    k<<<grid, 256, smem, s>>>(nb_group_desc(g), g->P, pl->items, pl->n_items, q, g->d_tau, margin, bits, logits, st,
                              ws.flag_count, ws.flag_idx);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status ensure_ws(nb_group *g, size_t bytes) {
    if (bytes <= g->ws_bytes) return NB_OK;
    if (g->ws) {
        NB_CUDA(cudaDeviceSynchronize());
        cudaFree(g->ws);
        g->ws = nullptr;
        g->ws_bytes = 0;
    }
    const size_t want = bytes + bytes / 4 + 4096;
    if (cudaMalloc(&g->ws, want) != cudaSuccess) {
        cudaGetLastError();
        return nb_fail(NB_ENOMEM, "grouped workspace allocation failed");
    }
    g->ws_bytes = want;
    return NB_OK;
}

void free_group(nb_group *g) {
    cudaFree(g->params);
    cudaFree(g->m);
    cudaFree(g->v);
    cudaFree(g->grad);
    cudaFree(g->paramsT);
    cudaFree(g->d_tau);
    cudaFree(g->ws);
    cudaFree(g->sched_alpha);
    cudaFree(g->sched_c1);
    cudaFree(g->sched_sqrt_c2);
    cudaFree(g->d_step);
    nb_tc_free(&g->tc);
    delete g;
}

nb_status upload_tau(nb_group *g) {
    std::vector<TauF> t(g->n_objects);
    for (int o = 0; o < g->n_objects; o++) t[o] = nb_tau_bracket(g->tau[o]);
    NB_CUDA(cudaMemcpy(g->d_tau, t.data(), sizeof(TauF) * g->n_objects, cudaMemcpyHostToDevice));
    return NB_OK;
}

}  // namespace

MlpDesc nb_group_desc(const nb_group *g) {
    MlpDesc d{};
    d.L = g->L;
    for (int l = 0; l <= g->L; l++) d.w[l] = g->widths[l];
    d.maxw = 0;
    for (int l = 0; l < g->L; l++) {
        d.off[l] = g->off[l];
        if (g->widths[l] > d.maxw) d.maxw = g->widths[l];
    }
    d.p = g->params;
    d.pT = g->paramsT;
    return d;
}

// ------------------------------------------------------------------ C ABI: plans
extern "C" nb_status nb_plan_create(const int64_t *host_offsets, int32_t n_objects, int32_t chunk_rows,
                                    nb_plan **out) {
    if (!host_offsets || !out) return nb_fail(NB_EINVAL, "nb_plan_create: null pointer");
    *out = nullptr;
    if (n_objects < 1) return nb_fail(NB_EINVAL, "nb_plan_create: n_objects must be >= 1");
    if (chunk_rows == 0) chunk_rows = 4096;
    if (chunk_rows < 64 || chunk_rows % 64) return nb_fail(NB_EINVAL, "nb_plan_create: chunk_rows must be a multiple of 64");
    if (host_offsets[0] < 0) return nb_fail(NB_EINVAL, "nb_plan_create: negative offset");
    for (int o = 0; o < n_objects; o++)
        if (host_offsets[o + 1] < host_offsets[o]) return nb_fail(NB_EINVAL, "nb_plan_create: offsets must not decrease");
    if (host_offsets[n_objects] >= ((int64_t)1 << 32)) return nb_fail(NB_EINVAL, "nb_plan_create: more than 2^32 rows");
    nb_plan *p = new nb_plan();
    p->n_objects = n_objects;
    p->chunk = chunk_rows;
    p->h_offsets.assign(host_offsets, host_offsets + n_objects + 1);
    p->aligned = true;
    std::vector<PlanItem> items;
    p->h_obj_items.resize(n_objects + 1);
    for (int o = 0; o < n_objects; o++) {
        p->h_obj_items[o] = (int)items.size();
        if (host_offsets[o] % 32) p->aligned = false;
        for (int64_t r = host_offsets[o]; r < host_offsets[o + 1]; r += chunk_rows) {
            PlanItem it{};
            it.obj = o;
            it.row0 = r;
            it.row1 = r + chunk_rows < host_offsets[o + 1] ? r + chunk_rows : host_offsets[o + 1];
            items.push_back(it);
        }
    }
    p->h_obj_items[n_objects] = (int)items.size();
    p->n_items = (int)items.size();
    p->n_rows = host_offsets[n_objects];
    if (cudaMalloc(&p->items, sizeof(PlanItem) * (items.size() + 1)) != cudaSuccess ||
        cudaMalloc(&p->obj_items, sizeof(int) * (n_objects + 1)) != cudaSuccess ||
        cudaMalloc(&p->offsets, sizeof(long long) * (n_objects + 1)) != cudaSuccess) {
        cudaGetLastError();
        nb_plan_destroy(p);
        return nb_fail(NB_ENOMEM, "nb_plan_create: allocation failed");
    }
    if (!items.empty())
        NB_CUDA(cudaMemcpy(p->items, items.data(), sizeof(PlanItem) * items.size(), cudaMemcpyHostToDevice));
    NB_CUDA(cudaMemcpy(p->obj_items, p->h_obj_items.data(), sizeof(int) * (n_objects + 1), cudaMemcpyHostToDevice));
    NB_CUDA(cudaMemcpy(p->offsets, host_offsets, sizeof(long long) * (n_objects + 1), cudaMemcpyHostToDevice));
    *out = p;
    return NB_OK;
}

extern "C" nb_status nb_plan_destroy(nb_plan *p) {
    if (!p) return NB_OK;
    cudaFree(p->items);
    cudaFree(p->obj_items);
    cudaFree(p->offsets);
    delete p;
    return NB_OK;
}

// ------------------------------------------------------------------ C ABI: groups
extern "C" nb_status nb_group_create(const int32_t *widths, int32_t n_layers, int32_t n_objects, int32_t infer_prec,
                                     int32_t train_prec, nb_group **out) {
    if (!widths || !out) return nb_fail(NB_EINVAL, "nb_group_create: null pointer");
    *out = nullptr;
    if (n_objects < 1) return nb_fail(NB_EINVAL, "nb_group_create: n_objects must be >= 1");
    if (n_layers < 1 || n_layers > NB_MAXL) return nb_fail(NB_EINVAL, "nb_group_create: n_layers must be 1..8");
    if (widths[n_layers] != 1) return nb_fail(NB_EINVAL, "nb_group_create: last width must be 1");
    for (int l = 0; l < n_layers; l++)
        if (widths[l] < 1 || widths[l] > NB_MAXW) return nb_fail(NB_EINVAL, "nb_group_create: widths must be 1..256");
    if (train_prec != NB_F32 && train_prec != NB_BF16)
        return nb_fail(NB_EUNSUPPORTED, "nb_group_create: grouped training runs in FP32 or BF16");
    if (infer_prec != NB_F32 && infer_prec != NB_F16X3)
        return nb_fail(NB_EUNSUPPORTED, "nb_group_create: grouped queries run in FP32 or split FP16");
    nb_group *g = new nb_group();
    g->L = n_layers;
    g->n_objects = n_objects;
    for (int l = 0; l <= n_layers; l++) g->widths[l] = widths[l];
    int64_t o = 0;
    for (int l = 0; l < n_layers; l++) {
        g->off[l] = (int)o;
        o += (int64_t)widths[l + 1] * (widths[l] + 1);
    }
    g->P = o;
    g->S = (o + 3) / 4 * 4;
    g->infer_prec = infer_prec;
    g->train_prec = train_prec;
    g->tau.assign(n_objects, 0.0);
    nb_fill_gamma(g->widths, g->L, &g->gamma);
    const size_t pb = (size_t)g->P * n_objects * sizeof(float);
    if (cudaMalloc(&g->params, pb) != cudaSuccess || cudaMalloc(&g->m, pb) != cudaSuccess ||
        cudaMalloc(&g->v, pb) != cudaSuccess || cudaMalloc(&g->grad, pb) != cudaSuccess ||
        cudaMalloc(&g->paramsT, pb) != cudaSuccess ||
        cudaMalloc(&g->d_tau, sizeof(TauF) * n_objects) != cudaSuccess || cudaMalloc(&g->d_step, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        free_group(g);
        return nb_fail(NB_ENOMEM, "nb_group_create: allocation failed");
    }
    cudaMemset(g->params, 0, pb);
    cudaMemset(g->m, 0, pb);
    cudaMemset(g->v, 0, pb);
    cudaMemset(g->grad, 0, pb);
    cudaMemset(g->paramsT, 0, pb);
    cudaMemset(g->d_step, 0, sizeof(int));
    if (upload_tau(g) != NB_OK) {
        free_group(g);
        return NB_ECUDA;
    }
    nb_status ts = NB_OK;
    if (infer_prec == NB_F16X3) ts = nb_tc_group_init(&g->tc, nb_group_desc(g), n_objects);
    if (ts == NB_OK && train_prec == NB_BF16) ts = nb_train_bf16_group_init(&g->tc, nb_group_desc(g), n_objects);
    if (ts != NB_OK) {
        std::string msg = nb_last_error();
        free_group(g);
        return nb_fail(ts, msg);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_group(g);
        return nb_fail(NB_ECUDA, "nb_group_create: device error");
    }
    *out = g;
    return NB_OK;
}

extern "C" nb_status nb_group_destroy(nb_group *g) {
    if (!g) return NB_OK;
    cudaDeviceSynchronize();
    free_group(g);
    return NB_OK;
}

extern "C" int64_t nb_group_param_count(const nb_group *g) { return g ? g->P : -1; }

static nb_status group_refresh(nb_group *g, cudaStream_t s) {
    const nb_status ts = nb_launch_transpose(nb_group_desc(g), g->paramsT, g->n_objects, g->P, s);
    if (ts != NB_OK) return ts;
    if (g->train_prec == NB_BF16) {
        const nb_status st = nb_train_bf16_group_refresh(&g->tc, nb_group_desc(g), g->n_objects, s);
        if (st != NB_OK) return st;
    }
    if (g->infer_prec != NB_F16X3) return NB_OK;
    return nb_tc_group_refresh(&g->tc, nb_group_desc(g), g->n_objects, s);
}

extern "C" nb_status nb_group_set_params(nb_group *g, const float *host_params, int64_t n) {
    if (!g || !host_params) return nb_fail(NB_EINVAL, "nb_group_set_params: null pointer");
    if (n != g->P * g->n_objects) return nb_fail(NB_EINVAL, "nb_group_set_params: expected n_objects * P values");
    const size_t pb = (size_t)n * sizeof(float);
    NB_CUDA(cudaMemcpy(g->params, host_params, pb, cudaMemcpyHostToDevice));
    NB_CUDA(cudaMemset(g->m, 0, pb));
    NB_CUDA(cudaMemset(g->v, 0, pb));
    NB_CUDA(cudaMemset(g->d_step, 0, sizeof(int)));
    g->step = 0;
    const nb_status st = group_refresh(g, 0);
    if (st != NB_OK) return st;
    NB_CUDA(cudaDeviceSynchronize());
    return NB_OK;
}

extern "C" nb_status nb_group_get_params(const nb_group *g, float *host_params, int64_t n) {
    if (!g || !host_params) return nb_fail(NB_EINVAL, "nb_group_get_params: null pointer");
    if (n != g->P * g->n_objects) return nb_fail(NB_EINVAL, "nb_group_get_params: expected n_objects * P values");
    NB_CUDA(cudaDeviceSynchronize());
    NB_CUDA(cudaMemcpy(host_params, g->params, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost));
    return NB_OK;
}

extern "C" nb_status nb_group_get_grad(const nb_group *g, float *host_grad, int64_t n) {
    if (!g || !host_grad) return nb_fail(NB_EINVAL, "nb_group_get_grad: null pointer");
    if (n != g->P * g->n_objects) return nb_fail(NB_EINVAL, "nb_group_get_grad: expected n_objects * P values");
    NB_CUDA(cudaDeviceSynchronize());
    NB_CUDA(cudaMemcpy(host_grad, g->grad, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost));
    return NB_OK;
}

extern "C" nb_status nb_group_set_tau(nb_group *g, const double *host_tau, int32_t n_objects) {
    if (!g || !host_tau) return nb_fail(NB_EINVAL, "nb_group_set_tau: null pointer");
    if (n_objects != g->n_objects) return nb_fail(NB_EINVAL, "nb_group_set_tau: wrong object count");
    for (int o = 0; o < n_objects; o++)
        if (isnan(host_tau[o])) return nb_fail(NB_EINVAL, "nb_group_set_tau: NaN");
    g->tau.assign(host_tau, host_tau + n_objects);
    return upload_tau(g);
}

extern "C" nb_status nb_group_get_tau(const nb_group *g, double *host_tau, int32_t n_objects) {
    if (!g || !host_tau) return nb_fail(NB_EINVAL, "nb_group_get_tau: null pointer");
    if (n_objects != g->n_objects) return nb_fail(NB_EINVAL, "nb_group_get_tau: wrong object count");
    memcpy(host_tau, g->tau.data(), sizeof(double) * n_objects);
    return NB_OK;
}

extern "C" nb_status nb_group_set_schedule(nb_group *g, const float *host_alpha, int32_t T) {
    if (!g || !host_alpha) return nb_fail(NB_EINVAL, "nb_group_set_schedule: null pointer");
    if (T < 1) return nb_fail(NB_EINVAL, "nb_group_set_schedule: T must be >= 1");
    cudaFree(g->sched_alpha);
    cudaFree(g->sched_c1);
    cudaFree(g->sched_sqrt_c2);
    g->sched_alpha = g->sched_c1 = g->sched_sqrt_c2 = nullptr;
    std::vector<float> c1(T), sc2(T);
    for (int t = 0; t < T; t++) {
        const double step = (double)(g->step + t + 1);
        c1[t] = (float)(1.0 - pow((double)g->b1, step));
        sc2[t] = (float)sqrt(1.0 - pow((double)g->b2, step));
    }
    if (cudaMalloc(&g->sched_alpha, sizeof(float) * T) != cudaSuccess ||
        cudaMalloc(&g->sched_c1, sizeof(float) * T) != cudaSuccess ||
        cudaMalloc(&g->sched_sqrt_c2, sizeof(float) * T) != cudaSuccess) {
        cudaGetLastError();
        return nb_fail(NB_ENOMEM, "nb_group_set_schedule: allocation failed");
    }
    NB_CUDA(cudaMemcpy(g->sched_alpha, host_alpha, sizeof(float) * T, cudaMemcpyHostToDevice));
    NB_CUDA(cudaMemcpy(g->sched_c1, c1.data(), sizeof(float) * T, cudaMemcpyHostToDevice));
    NB_CUDA(cudaMemcpy(g->sched_sqrt_c2, sc2.data(), sizeof(float) * T, cudaMemcpyHostToDevice));
    NB_CUDA(cudaMemset(g->d_step, 0, sizeof(int)));
    g->sched_T = T;
    g->sched_base = g->step;
    return NB_OK;
}

extern "C" nb_status nb_group_reserve(nb_group *g, const nb_plan *pl) {
    if (!g || !pl) return nb_fail(NB_EINVAL, "nb_group_reserve: null pointer");
    if (pl->n_objects != g->n_objects) return nb_fail(NB_EINVAL, "nb_group_reserve: plan and group differ in objects");
    const size_t train = align256((size_t)pl->n_items * g->S * sizeof(float)) + align256((size_t)pl->n_items * sizeof(float));
    const size_t query = 256 + 2 * align256((size_t)pl->n_rows * sizeof(unsigned));
    return ensure_ws(g, train > query ? train : query);
}

extern "C" nb_status nb_train_step_grouped(nb_group *g, const nb_plan *pl, const float *q, const uint32_t *label_bits,
                                           float alpha, float beta, nb_step_stats *dev_stats, void *stream) {
    if (!g || !pl) return nb_fail(NB_EINVAL, "nb_train_step_grouped: null group or plan");
    if (pl->n_objects != g->n_objects) return nb_fail(NB_EINVAL, "nb_train_step_grouped: plan and group differ in objects");
    if (!q || !label_bits) return nb_fail(NB_EINVAL, "nb_train_step_grouped: null pointer");
    const bool sched = alpha < 0;
    if (sched && !g->sched_alpha) return nb_fail(NB_EINVAL, "nb_train_step_grouped: alpha < 0 needs a schedule");
    if (!sched && (!(alpha >= 0) || isinf(alpha))) return nb_fail(NB_EINVAL, "nb_train_step_grouped: bad alpha");
    if (!(beta >= 0) || isinf(beta)) return nb_fail(NB_EINVAL, "nb_train_step_grouped: bad beta");
    if (pl->n_items == 0) return NB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    nb_status st = nb_group_reserve(g, pl);
    if (st != NB_OK) return st;
    float *partial = (float *)g->ws;
    float *loss_partial = (float *)((char *)g->ws + align256((size_t)pl->n_items * g->S * sizeof(float)));
    NB_CUDA(cudaMemsetAsync(partial, 0, (size_t)pl->n_items * g->S * sizeof(float), s));
    if (dev_stats) NB_CUDA(cudaMemsetAsync(dev_stats, 0, sizeof(nb_step_stats), s));
    const MlpDesc d = nb_group_desc(g);
    if (g->train_prec == NB_BF16)
        st = nb_launch_train_bf16_group(&g->tc, d, g->P, g->S, pl, q, label_bits, alpha, sched ? g->sched_alpha : nullptr,
                                        g->d_step, g->sched_T, beta, g->d_tau, partial, loss_partial, dev_stats, s);
    else switch (nj_for(d.maxw)) {
    case 1: st = group_train_launch<1, 32>(g, pl, q, label_bits, alpha, sched, beta, partial, loss_partial, dev_stats, s); break;
    case 2: st = group_train_launch<2, 32>(g, pl, q, label_bits, alpha, sched, beta, partial, loss_partial, dev_stats, s); break;
    case 4: st = group_train_launch<4, 32>(g, pl, q, label_bits, alpha, sched, beta, partial, loss_partial, dev_stats, s); break;
    case 8: st = group_train_launch<8, 32>(g, pl, q, label_bits, alpha, sched, beta, partial, loss_partial, dev_stats, s); break;
    default: st = group_train_launch<16, 16>(g, pl, q, label_bits, alpha, sched, beta, partial, loss_partial, dev_stats, s); break;
    }
    if (st != NB_OK) return st;
    float c1 = 1.f, sc2 = 1.f;
    if (!sched) {
        g->step += 1;
        c1 = (float)(1.0 - pow((double)g->b1, (double)g->step));
        sc2 = (float)sqrt(1.0 - pow((double)g->b2, (double)g->step));
    }
    const long long total = (long long)g->n_objects * g->P;
    group_adam_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        g->P, g->S, g->n_objects, pl->obj_items, partial, g->params, g->m, g->v, g->grad, g->lr, g->b1, g->b2, g->eps, c1,
        sc2, sched ? g->sched_c1 : nullptr, sched ? g->sched_sqrt_c2 : nullptr, g->d_step, g->sched_T);
    NB_CUDA(cudaGetLastError());
    group_loss_kernel<<<1, 256, 0, s>>>(g->n_objects, pl->obj_items, pl->offsets, loss_partial, dev_stats,
                                        sched ? g->d_step : nullptr);
    NB_CUDA(cudaGetLastError());
    return group_refresh(g, s);
}

extern "C" nb_status nb_group_sync_schedule(nb_group *g) {
    if (!g) return nb_fail(NB_EINVAL, "nb_group_sync_schedule: null group");
    int t = 0;
    NB_CUDA(cudaDeviceSynchronize());
    NB_CUDA(cudaMemcpy(&t, g->d_step, sizeof(int), cudaMemcpyDeviceToHost));
    g->step = g->sched_base + t;
    return NB_OK;
}

extern "C" nb_status nb_query_grouped(nb_group *g, const nb_plan *pl, const float *q, float margin, uint32_t *out_bits,
                                      float *opt_logits, nb_query_stats *dev_stats, void *stream) {
    if (!g || !pl) return nb_fail(NB_EINVAL, "nb_query_grouped: null group or plan");
    if (pl->n_objects != g->n_objects) return nb_fail(NB_EINVAL, "nb_query_grouped: plan and group differ in objects");
    if (!pl->aligned) return nb_fail(NB_EINVAL, "nb_query_grouped: every object's first row must be a multiple of 32");
    if (pl->n_rows > 0 && (!q || !out_bits)) return nb_fail(NB_EINVAL, "nb_query_grouped: null pointer");
    if (!(margin >= 0) || isinf(margin)) return nb_fail(NB_EINVAL, "nb_query_grouped: margin must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (dev_stats) NB_CUDA(cudaMemsetAsync(dev_stats, 0, sizeof(nb_query_stats), s));
    if (pl->n_rows == 0) return NB_OK;
    nb_status st = nb_group_reserve(g, pl);
    if (st != NB_OK) return st;
    const size_t list = align256((size_t)pl->n_rows * sizeof(unsigned));
    QueryWs ws;
    ws.flag_count = (unsigned *)g->ws;
    ws.ff_count = (unsigned *)((char *)g->ws + 64);
    ws.flag_idx = (unsigned *)((char *)g->ws + 256);
    ws.ff_idx = (unsigned *)((char *)g->ws + 256 + list);
    NB_CUDA(cudaMemsetAsync(ws.flag_count, 0, sizeof(unsigned), s));
    // rows outside every object's range keep 0 bits
    if (pl->h_offsets[0] > 0) NB_CUDA(cudaMemsetAsync(out_bits, 0, (size_t)(pl->h_offsets[0] / 32) * 4, s));
    const MlpDesc d = nb_group_desc(g);
    if (g->infer_prec == NB_F16X3) {
        st = nb_tc_group_query(&g->tc, d, g->P, pl, q, g->d_tau, margin, out_bits, opt_logits, dev_stats, ws, s);
    } else {
        switch (nj_for(d.maxw)) {
        case 1: st = group_fwd_launch<1>(g, pl, q, margin, out_bits, opt_logits, dev_stats, ws, s); break;
        case 2: st = group_fwd_launch<2>(g, pl, q, margin, out_bits, opt_logits, dev_stats, ws, s); break;
        case 4: st = group_fwd_launch<4>(g, pl, q, margin, out_bits, opt_logits, dev_stats, ws, s); break;
        case 8: st = group_fwd_launch<8>(g, pl, q, margin, out_bits, opt_logits, dev_stats, ws, s); break;
        default: st = group_fwd_launch<16>(g, pl, q, margin, out_bits, opt_logits, dev_stats, ws, s); break;
        }
    }
    if (st != NB_OK) return st;
    return nb_launch_recheck_grouped(d, g->gamma, q, pl->offsets, g->n_objects, g->P, g->d_tau, out_bits, dev_stats,
                                     ws, pl->n_rows, s);
}

extern "C" nb_status nb_calibrate_grouped(nb_group *g, const nb_plan *pl, const float *q, const uint32_t *label_bits,
                                          double eps, double *host_tau, void *stream) {
    if (!g || !pl || !host_tau) return nb_fail(NB_EINVAL, "nb_calibrate_grouped: null pointer");
    if (pl->n_objects != g->n_objects) return nb_fail(NB_EINVAL, "nb_calibrate_grouped: plan and group differ in objects");
    if (pl->n_rows > 0 && (!q || !label_bits)) return nb_fail(NB_EINVAL, "nb_calibrate_grouped: null pointer");
    if (!(eps >= 0) || isinf(eps)) return nb_fail(NB_EINVAL, "nb_calibrate_grouped: eps must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t maxn = 0;
    for (int o = 0; o < g->n_objects; o++) {
        const int64_t c = pl->h_offsets[o + 1] - pl->h_offsets[o];
        if (c > maxn) maxn = c;
    }
    const size_t head = 256, list = align256((size_t)(maxn > 0 ? maxn : 1) * sizeof(unsigned));
    nb_status st = ensure_ws(g, head + 2 * list);
    if (st != NB_OK) return st;
    CalibWs ws;
    ws.umin_bits = (unsigned *)g->ws;
    ws.zmin_bits = (unsigned long long *)((char *)g->ws + 64);
    ws.npos = (unsigned *)((char *)g->ws + 128);
    ws.pos_idx = (unsigned *)((char *)g->ws + head);
    ws.lo = (float *)((char *)g->ws + head + list);
    MlpDesc d = nb_group_desc(g);
    for (int o = 0; o < g->n_objects; o++) {
        const int64_t r0 = pl->h_offsets[o], r1 = pl->h_offsets[o + 1];
        double tau = INFINITY;
        if (r1 > r0) {
            d.p = g->params + (size_t)o * g->P;
            d.pT = g->paramsT + (size_t)o * g->P;
            st = nb_launch_calibrate(d, g->gamma, q, label_bits, r0, r1, ws, s);
            if (st != NB_OK) return st;
            unsigned long long zb = 0;
            unsigned npos = 0;
            NB_CUDA(cudaMemcpyAsync(&zb, ws.zmin_bits, 8, cudaMemcpyDeviceToHost, s));
            NB_CUDA(cudaMemcpyAsync(&npos, ws.npos, 4, cudaMemcpyDeviceToHost, s));
            NB_CUDA(cudaStreamSynchronize(s));
            tau = nb_tau_from_min_bits(zb, npos, eps);
        }
        g->tau[o] = tau;
        host_tau[o] = tau;
    }
    return upload_tau(g);
}

// ------------------------------------------------------------------ autotuner
// The grouped launches split every object's rows into work items of chunk_rows rows;
// small items balance uneven objects across the SMs, large ones load each object's
// weights into shared memory fewer times.  The best split depends on the widths, the
// object count and the spread of the counts, so it is measured: every candidate plan
// runs the operation (one untimed launch, then `reps` timed with CUDA events on the
// stream) and the fastest is returned.  Training trials run on a snapshot of the
// parameters, Adam moments, gradient and step counters, restored afterwards.
extern "C" nb_status nb_group_autotune(nb_group *g, const int64_t *host_offsets, int32_t n_objects, int32_t op,
                                       const float *q, const uint32_t *label_bits, const int32_t *candidates,
                                       int32_t n_candidates, int32_t reps, int32_t *best_chunk_rows, float *host_ms,
                                       void *stream) {
    if (!g || !host_offsets || !candidates || !best_chunk_rows) return nb_fail(NB_EINVAL, "nb_group_autotune: null pointer");
    if (n_objects != g->n_objects) return nb_fail(NB_EINVAL, "nb_group_autotune: wrong object count");
    if (op != NB_TUNE_QUERY && op != NB_TUNE_TRAIN) return nb_fail(NB_EINVAL, "nb_group_autotune: unknown operation");
    if (n_candidates < 1 || n_candidates > 64 || reps < 1 || reps > 1000)
        return nb_fail(NB_EINVAL, "nb_group_autotune: 1..64 candidates and 1..1000 repetitions");
    if (!q || (op == NB_TUNE_TRAIN && !label_bits)) return nb_fail(NB_EINVAL, "nb_group_autotune: null pointer");
    for (int c = 0; c < n_candidates; c++)
        if (candidates[c] < 64 || candidates[c] % 64)
            return nb_fail(NB_EINVAL, "nb_group_autotune: candidates must be multiples of 64");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_rows = host_offsets[n_objects];
    uint32_t *bits = nullptr;
    float *snap = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t pb = (size_t)g->P * g->n_objects * sizeof(float);
    nb_status st = NB_OK;
    int best = -1;
    float best_ms = INFINITY;
    const int64_t step0 = g->step;
    int dstep0 = 0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        st = nb_fail(NB_ECUDA, "nb_group_autotune: event creation failed");
        goto done;
    }
    if (op == NB_TUNE_QUERY) {
        if (cudaMalloc(&bits, (size_t)((n_rows + 31) / 32 + 1) * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            st = nb_fail(NB_ENOMEM, "nb_group_autotune: allocation failed");
            goto done;
        }
    } else {
        if (cudaMalloc(&snap, 4 * pb) != cudaSuccess) {
            cudaGetLastError();
            st = nb_fail(NB_ENOMEM, "nb_group_autotune: allocation failed");
            goto done;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess ||
            cudaMemcpy(&dstep0, g->d_step, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            st = nb_fail(NB_ECUDA, "nb_group_autotune: device error");
            goto done;
        }
        float *src[4] = {g->params, g->m, g->v, g->grad};
        for (int k = 0; k < 4; k++)
            if (cudaMemcpyAsync((char *)snap + k * pb, src[k], pb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                st = nb_fail(NB_ECUDA, "nb_group_autotune: snapshot failed");
                goto done;
            }
    }
    for (int c = 0; c < n_candidates && st == NB_OK; c++) {
        nb_plan *pl = nullptr;
        st = nb_plan_create(host_offsets, n_objects, candidates[c], &pl);
        if (st != NB_OK) break;
        float ms = 0.f;
        for (int r = 0; r <= reps && st == NB_OK; r++) {
            if (r == 1 && cudaEventRecord(e0, s) != cudaSuccess) st = nb_fail(NB_ECUDA, "nb_group_autotune: event");
            if (st != NB_OK) break;
            st = op == NB_TUNE_QUERY
                     ? nb_query_grouped(g, pl, q, 0.0f, bits, nullptr, nullptr, stream)
                     : nb_train_step_grouped(g, pl, q, label_bits, 1.0f, 1.0f, nullptr, stream);
        }
        if (st == NB_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = nb_fail(NB_ECUDA, "nb_group_autotune: timing failed");
        nb_plan_destroy(pl);
        if (st != NB_OK) break;
        ms /= (float)reps;
        if (host_ms) host_ms[c] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
done:
    if (snap) {
        // restore the training state whatever happened above
        float *dst[4] = {g->params, g->m, g->v, g->grad};
        for (int k = 0; k < 4; k++) cudaMemcpyAsync(dst[k], (char *)snap + k * pb, pb, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(g->d_step, &dstep0, sizeof(int), cudaMemcpyHostToDevice, s);
        g->step = step0;
        if (cudaStreamSynchronize(s) != cudaSuccess && st == NB_OK) st = nb_fail(NB_ECUDA, "nb_group_autotune: restore failed");
        const nb_status rs = group_refresh(g, s);
        if (st == NB_OK) st = rs;
        cudaStreamSynchronize(s);
        cudaFree(snap);
    }
    if (bits) {
        cudaStreamSynchronize(s);
        cudaFree(bits);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st == NB_OK) *best_chunk_rows = candidates[best];
    return st;
}
