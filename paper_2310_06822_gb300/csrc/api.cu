// C ABI of libnb (include/nb.h): argument checking, model state, workspace and the
// launch sequence of each hot-path call.
#include <fenv.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;

void nb_set_error(const std::string &msg) { g_err = msg; }

nb_status nb_fail(nb_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

nb_status nb_cuda_check(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return NB_ECUDA;
}

extern "C" const char *nb_last_error(void) { return g_err.c_str(); }

TauF nb_tau_bracket(double tau) {
    TauF t{};
    if (isinf(tau)) {
        t.dn = t.up = t.hi = (float)tau;
        return t;
    }
    // split tau = hi + lo + r: hi - tau is exact in double (Sterbenz), |r| <= err
    t.hi = (float)tau;
    const double r1 = tau - (double)t.hi;
    t.lo = (float)r1;
    const double r2 = fabs(r1 - (double)t.lo);
    t.err = (float)r2;
    if ((double)t.err < r2) t.err = nextafterf(t.err, INFINITY);
    float f = (float)tau;  // round to nearest
    if ((double)f == tau) {
        t.dn = t.up = f;
    } else if ((double)f < tau) {
        t.dn = f;
        t.up = nextafterf(f, INFINITY);
    } else {
        t.up = f;
        t.dn = nextafterf(f, -INFINITY);
    }
    return t;
}

void nb_fill_gamma(const int *widths, int L, GammaTab *gt) {
    // gamma_k = k u / (1 - k u), u = 2^-24, computed in double, then rounded up to float:
    // k = fan-in + 8 roundings per term (FP32 stage), k = 3 fan-in + 4 (compensated stage),
    // k = 4 fan-in + 4 (three-word stage)
    const double u = ldexp(1.0, -24);
    for (int l = 0; l < L; l++) {
        const double k = widths[l] + 8.0, gmm = k * u / (1.0 - k * u);
        float gf = (float)gmm;
        if ((double)gf < gmm) gf = nextafterf(gf, INFINITY);
        gt->g[l] = nextafterf(gf, INFINITY);
        const double k3 = 3.0 * widths[l] + 4.0, cd2 = k3 * u / (1.0 - k3 * u);
        float c2 = (float)cd2;
        if ((double)c2 < cd2) c2 = nextafterf(c2, INFINITY);
        gt->gd2[l] = nextafterf(c2, INFINITY);
        const double k4 = 4.0 * widths[l] + 4.0, cff = k4 * u / (1.0 - k4 * u);
        float cf = (float)cff;
        if ((double)cf < cff) cf = nextafterf(cf, INFINITY);
        gt->gff[l] = nextafterf(cf, INFINITY);
    }
}

double nb_tau_from_min_bits(unsigned long long zmin_bits, unsigned npos, double eps) {
    if (npos == 0) return INFINITY;
    if (zmin_bits == 0ull) return -INFINITY;  // a positive query had a NaN logit: everything is inside
    const unsigned long long u =
        (zmin_bits & 0x8000000000000000ull) ? (zmin_bits & 0x7fffffffffffffffull) : ~zmin_bits;
    double zmin;
    memcpy(&zmin, &u, 8);
    // tau = zmin - eps rounded toward -infinity; volatile operands keep the subtraction
    // between the two rounding-mode switches
    volatile double va = zmin, vb = eps;
    const int old = fegetround();
    fesetround(FE_DOWNWARD);
    volatile double t = va - vb;
    fesetround(old);
    return t;
}

// ---------------------------------------------------------------- model
struct nb_model {
    int device = 0;
    int L = 0;
    int widths[NB_MAXL + 1] = {0};
    int off[NB_MAXL] = {0};
    int64_t P = 0;
    int infer_prec = NB_F32, train_prec = NB_F32;
    int act = NB_ACT_RELU;
    float *params = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr;
    float *paramsT = nullptr;  // weights transposed, for the margin re-check and calibration
    bool pT_stale = false;     // paramsT lags the master weights (set by training steps)
    int64_t step = 0;
    double tau = 0.0;
    float lr = 1e-3f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    GammaTab gamma{};
    // library-owned scratch, grown on demand
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *eo_ws = nullptr;  // early-out scratch (this model as the late network) or three-way scratch (as the outer)
    size_t eo_bytes = 0;
    // low-precision weight images for the tensor-core paths
    TcModel tc{};
    // nb_query_host: two device staging chunks, a copy stream and its events
    cudaStream_t hq_stream = nullptr;
    cudaEvent_t hq_ready[2] = {nullptr, nullptr}, hq_done[2] = {nullptr, nullptr};
    float *hq_q[2] = {nullptr, nullptr};
    uint32_t *hq_bits[2] = {nullptr, nullptr};
    nb_query_stats *hq_stats = nullptr;  // [3]: one per chunk buffer and the running sum
    int64_t hq_chunk = 0;
    // nb_query_host reading pinned host queries in place: the device copy of the bits
    uint32_t *zc_bits = nullptr;
    int64_t zc_words = 0;
};

static MlpDesc desc_of(const nb_model *m) {
    MlpDesc d{};
    d.L = m->L;
    d.maxw = 0;
    for (int l = 0; l <= m->L; l++) d.w[l] = m->widths[l];
    for (int l = 0; l < m->L; l++) {
        d.off[l] = m->off[l];
        if (m->widths[l] > d.maxw) d.maxw = m->widths[l];
    }
    d.p = m->params;
    d.pT = m->paramsT;
    d.act = m->act;
    return d;
}

static nb_status ensure_ws(nb_model *m, size_t bytes) {
    if (bytes <= m->ws_bytes) return NB_OK;
    if (m->ws) {
        NB_CUDA(cudaDeviceSynchronize());
        cudaFree(m->ws);
        m->ws = nullptr;
        m->ws_bytes = 0;
    }
    size_t want = bytes + bytes / 4 + 4096;
    if (cudaMalloc(&m->ws, want) != cudaSuccess) {
        cudaGetLastError();
        m->ws = nullptr;
        return nb_fail(NB_ENOMEM, "workspace allocation failed");
    }
    m->ws_bytes = want;
    return NB_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

static void free_model(nb_model *m) {
    cudaFree(m->params);
    cudaFree(m->adam_m);
    cudaFree(m->adam_v);
    cudaFree(m->grad);
    cudaFree(m->paramsT);
    cudaFree(m->ws);
    cudaFree(m->eo_ws);
    for (int b = 0; b < 2; b++) {
        cudaFree(m->hq_q[b]);
        cudaFree(m->hq_bits[b]);
        if (m->hq_ready[b]) cudaEventDestroy(m->hq_ready[b]);
        if (m->hq_done[b]) cudaEventDestroy(m->hq_done[b]);
    }
    cudaFree(m->hq_stats);
    cudaFree(m->zc_bits);
    if (m->hq_stream) cudaStreamDestroy(m->hq_stream);
    nb_tc_free(&m->tc);
    delete m;
}

extern "C" nb_status nb_model_create(const int32_t *widths, int32_t n_layers, int32_t infer_prec, int32_t train_prec,
                                     nb_model **out) {
    return nb_model_create_act(widths, n_layers, infer_prec, train_prec, NB_ACT_RELU, out);
}

extern "C" nb_status nb_model_create_act(const int32_t *widths, int32_t n_layers, int32_t infer_prec,
                                         int32_t train_prec, int32_t activation, nb_model **out) {
    if (!widths || !out) return nb_fail(NB_EINVAL, "nb_model_create: null pointer");
    if (activation != NB_ACT_RELU && activation != NB_ACT_SINE)
        return nb_fail(NB_EINVAL, "nb_model_create: unknown activation");
    if (activation == NB_ACT_SINE && ((infer_prec != NB_F32 && infer_prec != NB_F16X3) || train_prec != NB_F32))
        return nb_fail(NB_EUNSUPPORTED,
                       "nb_model_create: sine networks infer in NB_F32 or NB_F16X3 and train in NB_F32");
    *out = nullptr;
    if (n_layers < 1 || n_layers > NB_MAXL) return nb_fail(NB_EINVAL, "nb_model_create: n_layers must be 1..8");
    if (widths[n_layers] != 1) return nb_fail(NB_EINVAL, "nb_model_create: last width must be 1");
    for (int l = 0; l < n_layers; l++)
        if (widths[l] < 1 || widths[l] > NB_MAXW)
            return nb_fail(NB_EINVAL, "nb_model_create: widths must be 1..256");
    if (infer_prec < NB_F32 || infer_prec > NB_F16X3 || train_prec < NB_F32 || train_prec > NB_BF16)
        return nb_fail(NB_EINVAL, "nb_model_create: bad precision");
    nb_model *m = new nb_model();
    cudaGetDevice(&m->device);
    m->L = n_layers;
    for (int l = 0; l <= n_layers; l++) m->widths[l] = widths[l];
    int64_t o = 0;
    for (int l = 0; l < n_layers; l++) {
        m->off[l] = (int)o;
        o += (int64_t)widths[l + 1] * (widths[l] + 1);
    }
    m->P = o;
    m->infer_prec = infer_prec;
    m->train_prec = train_prec;
    m->act = activation;
    nb_fill_gamma(m->widths, n_layers, &m->gamma);
    const size_t pb = (size_t)m->P * sizeof(float);
    if (cudaMalloc(&m->params, pb) != cudaSuccess || cudaMalloc(&m->adam_m, pb) != cudaSuccess ||
        cudaMalloc(&m->adam_v, pb) != cudaSuccess || cudaMalloc(&m->grad, pb) != cudaSuccess ||
        cudaMalloc(&m->paramsT, pb) != cudaSuccess) {
        cudaGetLastError();
        free_model(m);
        return nb_fail(NB_ENOMEM, "nb_model_create: allocation failed");
    }
    cudaMemset(m->params, 0, pb);
    cudaMemset(m->paramsT, 0, pb);
    cudaMemset(m->adam_m, 0, pb);
    cudaMemset(m->adam_v, 0, pb);
    cudaMemset(m->grad, 0, pb);
    if (infer_prec != NB_F32 || train_prec != NB_F32) {
        nb_status s = nb_tc_init(&m->tc, desc_of(m), infer_prec, train_prec);
        if (s != NB_OK) {
            std::string msg = nb_last_error();
            free_model(m);
            return nb_fail(s, msg);
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_model(m);
        return nb_fail(NB_ECUDA, "nb_model_create: device error");
    }
    *out = m;
    return NB_OK;
}

extern "C" nb_status nb_model_destroy(nb_model *m) {
    if (!m) return NB_OK;
    cudaDeviceSynchronize();
    free_model(m);
    return NB_OK;
}

extern "C" int64_t nb_model_param_count(const nb_model *m) { return m ? m->P : -1; }

// every copy derived from the FP32 master weights, after each change of them
static nb_status refresh_lowp(nb_model *m, cudaStream_t s) {
    const nb_status st = nb_launch_transpose(desc_of(m), m->paramsT, 1, m->P, s);
    if (st != NB_OK) return st;
    m->pT_stale = false;
    if (m->infer_prec == NB_F32 && m->train_prec == NB_F32) return NB_OK;
    return nb_tc_refresh(&m->tc, desc_of(m), s);
}

// after a training step: the copies the next step and the tensor-core queries read; the
// transposed copy (read by the re-check, the calibration and the thread-per-query
// forward) is brought up to date by the next call that reads it, on that call's stream
static nb_status refresh_after_step(nb_model *m, cudaStream_t s, bool train_img_written = false) {
    m->pT_stale = true;
    if (m->infer_prec == NB_F32 && m->train_prec == NB_F32) return NB_OK;
    return train_img_written ? nb_tc_refresh_query(&m->tc, desc_of(m), s) : nb_tc_refresh(&m->tc, desc_of(m), s);
}

static nb_status ensure_pT(nb_model *m, cudaStream_t s) {
    if (!m->pT_stale) return NB_OK;
    const nb_status st = nb_launch_transpose(desc_of(m), m->paramsT, 1, m->P, s);
    if (st == NB_OK) m->pT_stale = false;
    return st;
}

extern "C" nb_status nb_model_set_params(nb_model *m, const float *host_params, int64_t n_params) {
    if (!m || !host_params) return nb_fail(NB_EINVAL, "nb_model_set_params: null pointer");
    if (n_params != m->P) return nb_fail(NB_EINVAL, "nb_model_set_params: wrong parameter count");
    const size_t pb = (size_t)m->P * sizeof(float);
    NB_CUDA(cudaMemcpy(m->params, host_params, pb, cudaMemcpyHostToDevice));
    NB_CUDA(cudaMemset(m->adam_m, 0, pb));
    NB_CUDA(cudaMemset(m->adam_v, 0, pb));
    m->step = 0;
    nb_status st = refresh_lowp(m, 0);
    if (st != NB_OK) return st;
    NB_CUDA(cudaDeviceSynchronize());
    return NB_OK;
}

extern "C" nb_status nb_model_get_params(const nb_model *m, float *host_params, int64_t n_params) {
    if (!m || !host_params) return nb_fail(NB_EINVAL, "nb_model_get_params: null pointer");
    if (n_params != m->P) return nb_fail(NB_EINVAL, "nb_model_get_params: wrong parameter count");
    NB_CUDA(cudaDeviceSynchronize());
    NB_CUDA(cudaMemcpy(host_params, m->params, (size_t)m->P * sizeof(float), cudaMemcpyDeviceToHost));
    return NB_OK;
}

extern "C" nb_status nb_model_get_grad(const nb_model *m, float *host_grad, int64_t n_params) {
    if (!m || !host_grad) return nb_fail(NB_EINVAL, "nb_model_get_grad: null pointer");
    if (n_params != m->P) return nb_fail(NB_EINVAL, "nb_model_get_grad: wrong parameter count");
    NB_CUDA(cudaDeviceSynchronize());
    NB_CUDA(cudaMemcpy(host_grad, m->grad, (size_t)m->P * sizeof(float), cudaMemcpyDeviceToHost));
    return NB_OK;
}

extern "C" nb_status nb_model_set_tau(nb_model *m, double tau) {
    if (!m) return nb_fail(NB_EINVAL, "nb_model_set_tau: null model");
    if (isnan(tau)) return nb_fail(NB_EINVAL, "nb_model_set_tau: NaN");
    m->tau = tau;
    return NB_OK;
}

extern "C" nb_status nb_model_get_tau(const nb_model *m, double *tau) {
    if (!m || !tau) return nb_fail(NB_EINVAL, "nb_model_get_tau: null pointer");
    *tau = m->tau;
    return NB_OK;
}

extern "C" nb_status nb_model_set_adam(nb_model *m, float lr, float beta1, float beta2, float eps) {
    if (!m) return nb_fail(NB_EINVAL, "nb_model_set_adam: null model");
    if (!(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return nb_fail(NB_EINVAL, "nb_model_set_adam: bad hyper-parameter");
    m->lr = lr;
    m->b1 = beta1;
    m->b2 = beta2;
    m->eps = eps;
    return NB_OK;
}

// checkpoint layout: magic, P, step, tau, L, widths[L+1], then params, m, v (FP32)
static const uint64_t kMagic = 0x4e42434b50543031ull;  // "NBCKPT01"

static size_t state_bytes(const nb_model *m) {
    return 8 * 4 + 4 * (size_t)(NB_MAXL + 1) + 3 * (size_t)m->P * sizeof(float);
}

extern "C" nb_status nb_model_state_size(const nb_model *m, size_t *bytes) {
    if (!m || !bytes) return nb_fail(NB_EINVAL, "nb_model_state_size: null pointer");
    *bytes = state_bytes(m);
    return NB_OK;
}

extern "C" nb_status nb_model_get_state(const nb_model *m, void *host_buf, size_t bytes) {
    if (!m || !host_buf) return nb_fail(NB_EINVAL, "nb_model_get_state: null pointer");
    if (bytes < state_bytes(m)) return nb_fail(NB_EINVAL, "nb_model_get_state: buffer too small");
    NB_CUDA(cudaDeviceSynchronize());
    char *p = (char *)host_buf;
    uint64_t hdr[4] = {kMagic, (uint64_t)m->P, (uint64_t)m->step, 0};
    memcpy(&hdr[3], &m->tau, 8);
    memcpy(p, hdr, 32);
    int32_t w[NB_MAXL + 1] = {0};
    for (int l = 0; l <= m->L; l++) w[l] = m->widths[l];
    memcpy(p + 32, w, sizeof(w));
    char *q = p + 32 + sizeof(w);
    const size_t pb = (size_t)m->P * sizeof(float);
    NB_CUDA(cudaMemcpy(q, m->params, pb, cudaMemcpyDeviceToHost));
    NB_CUDA(cudaMemcpy(q + pb, m->adam_m, pb, cudaMemcpyDeviceToHost));
    NB_CUDA(cudaMemcpy(q + 2 * pb, m->adam_v, pb, cudaMemcpyDeviceToHost));
    return NB_OK;
}

extern "C" nb_status nb_model_set_state(nb_model *m, const void *host_buf, size_t bytes) {
    if (!m || !host_buf) return nb_fail(NB_EINVAL, "nb_model_set_state: null pointer");
    if (bytes < state_bytes(m)) return nb_fail(NB_EINVAL, "nb_model_set_state: buffer too small");
    const char *p = (const char *)host_buf;
    uint64_t hdr[4];
    memcpy(hdr, p, 32);
    if (hdr[0] != kMagic || hdr[1] != (uint64_t)m->P) return nb_fail(NB_EINVAL, "nb_model_set_state: not a checkpoint of this network");
    int32_t w[NB_MAXL + 1];
    memcpy(w, p + 32, sizeof(w));
    for (int l = 0; l <= m->L; l++)
        if (w[l] != m->widths[l]) return nb_fail(NB_EINVAL, "nb_model_set_state: widths differ");
    const char *q = p + 32 + sizeof(w);
    const size_t pb = (size_t)m->P * sizeof(float);
    NB_CUDA(cudaDeviceSynchronize());
    NB_CUDA(cudaMemcpy(m->params, q, pb, cudaMemcpyHostToDevice));
    NB_CUDA(cudaMemcpy(m->adam_m, q + pb, pb, cudaMemcpyHostToDevice));
    NB_CUDA(cudaMemcpy(m->adam_v, q + 2 * pb, pb, cudaMemcpyHostToDevice));
    m->step = (int64_t)hdr[2];
    memcpy(&m->tau, &hdr[3], 8);
    nb_status st = refresh_lowp(m, 0);
    if (st != NB_OK) return st;
    NB_CUDA(cudaDeviceSynchronize());
    return NB_OK;
}

// ---------------------------------------------------------------- hot path
static const int kEncW[6] = {2, 3, 4, 6, 4, 6};

extern "C" nb_status nb_label(const nb_shape *shape, int32_t kind, const float *q, int64_t n, uint32_t *out_bits,
                              nb_label_stats *dev_stats, void *stream) {
    if (!shape) return nb_fail(NB_EINVAL, "nb_label: null shape");
    if (kind < 0 || kind > 5) return nb_fail(NB_EINVAL, "nb_label: unknown kind");
    if (n < 0) return nb_fail(NB_EINVAL, "nb_label: negative n");
    if (n > 0 && (!q || !out_bits)) return nb_fail(NB_EINVAL, "nb_label: null query or output pointer");
    if (shape->dim != 2 && shape->dim != 3) return nb_fail(NB_EINVAL, "nb_label: dim must be 2 or 3");
    if ((kind == NB_POINT2) != (shape->dim == 2)) return nb_fail(NB_EINVAL, "nb_label: kind does not match the shape's dim");
    if (shape->n_spheres < 1 || shape->n_spheres > 4096) return nb_fail(NB_EINVAL, "nb_label: n_spheres must be 1..4096");
    if (shape->qexp < 8 || shape->qexp > 24) return nb_fail(NB_EINVAL, "nb_label: qexp must be 8..24");
    if (shape->reserved != 0) return nb_fail(NB_EINVAL, "nb_label: reserved field must be 0");
    if (!shape->centres || !shape->radii) return nb_fail(NB_EINVAL, "nb_label: null sphere arrays");
    if (kind == NB_POINT4T && !shape->vel) return nb_fail(NB_EINVAL, "nb_label: point4t needs velocities");
    (void)kEncW;
    return nb_launch_label(shape, kind, q, n, out_bits, dev_stats, (cudaStream_t)stream);
}

extern "C" nb_status nb_train_step(nb_model *m, const float *q, const uint32_t *label_bits, int64_t n, float alpha,
                                   float beta, nb_step_stats *dev_stats, void *stream) {
    if (!m) return nb_fail(NB_EINVAL, "nb_train_step: null model");
    if (n < 1) return nb_fail(NB_EINVAL, "nb_train_step: n must be >= 1");
    if (!q || !label_bits) return nb_fail(NB_EINVAL, "nb_train_step: null pointer");
    if (!(alpha >= 0) || !(beta >= 0) || isinf(alpha) || isinf(beta))
        return nb_fail(NB_EINVAL, "nb_train_step: alpha and beta must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const MlpDesc d = desc_of(m);
    const TauF tau = nb_tau_bracket(m->tau);
    m->step += 1;
    const double c1 = 1.0 - pow((double)m->b1, (double)m->step);
    const double c2 = 1.0 - pow((double)m->b2, (double)m->step);
    const bool bf16 = m->train_prec == NB_BF16, tcgen = bf16 && m->tc.train_tc;
    TrainWs tw{};
    tw.G = tcgen ? nb_train_tc_ctas(n) : bf16 ? nb_train_bf16_ctas(n) : nb_train_f32_ctas(d, n, sm_count());
    tw.stride = bf16 ? (m->P + 3) / 4 * 4 : m->P;  // BF16: 16-byte aligned slots for vector reductions
    const size_t need = align256((size_t)tw.G * tw.stride * sizeof(float)) + align256((size_t)tw.G * sizeof(float));
    nb_status st = ensure_ws(m, need);
    if (st != NB_OK) return st;
    tw.partial = (float *)m->ws;
    tw.loss_partial = (float *)((char *)m->ws + align256((size_t)tw.G * tw.stride * sizeof(float)));
    st = tcgen  ? nb_launch_train_tc(&m->tc, d, q, label_bits, n, alpha, beta, tau, tw, dev_stats, s)
         : bf16 ? nb_launch_train_bf16(&m->tc, d, q, label_bits, n, alpha, beta, tau, tw, dev_stats, s)
                : nb_launch_train_f32(d, q, label_bits, n, alpha, beta, tau, tw, dev_stats, s);
    if (st != NB_OK) return st;
    // the tcgen05 step's BF16 image is written by the Adam step itself
    TrainImgMap img{};
    if (tcgen) {
        img.img = (uint8_t *)m->tc.train_img;
        img.NH = m->L - 1;
        for (int l = 0; l <= m->L; l++) img.w[l] = m->widths[l];
        for (int l = 0; l < m->L; l++) img.off[l] = m->off[l];
    }
    st = nb_launch_adam(m->P, 1.0f / (float)n, m->params, m->adam_m, m->adam_v, m->grad, tw, m->lr, m->b1, m->b2,
                        m->eps, (float)c1, (float)sqrt(c2), dev_stats, s, img);
    if (st != NB_OK) return st;
    return refresh_after_step(m, s, tcgen);
}

extern "C" nb_status nb_query(nb_model *m, const float *q, int64_t n, float margin, uint32_t *out_bits,
                              float *opt_logits, nb_query_stats *dev_stats, void *stream) {
    if (!m) return nb_fail(NB_EINVAL, "nb_query: null model");
    if (n < 0 || n >= (int64_t)1 << 32) return nb_fail(NB_EINVAL, "nb_query: n must be in [0, 2^32)");
    if (n > 0 && (!q || !out_bits)) return nb_fail(NB_EINVAL, "nb_query: null pointer");
    if (!(margin >= 0) || isinf(margin)) return nb_fail(NB_EINVAL, "nb_query: margin must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (dev_stats) NB_CUDA(cudaMemsetAsync(dev_stats, 0, sizeof(nb_query_stats), s));
    if (n == 0) return NB_OK;
    const size_t list = align256((size_t)n * sizeof(unsigned));
    nb_status st = ensure_ws(m, 256 + 2 * list);
    if (st != NB_OK) return st;
    st = ensure_pT(m, s);
    if (st != NB_OK) return st;
    QueryWs ws;
    ws.flag_count = (unsigned *)m->ws;
    ws.ff_count = (unsigned *)((char *)m->ws + 64);
    ws.flag_idx = (unsigned *)((char *)m->ws + 256);
    ws.ff_idx = (unsigned *)((char *)m->ws + 256 + list);
    NB_CUDA(cudaMemsetAsync(ws.flag_count, 0, sizeof(unsigned), s));
    const MlpDesc d = desc_of(m);
    const TauF tau = nb_tau_bracket(m->tau);
    if (m->infer_prec == NB_F32)
        st = nb_narrow_eligible(d) ? nb_launch_fwd_narrow(d, q, n, tau, margin, out_bits, opt_logits, dev_stats, ws, s)
                                   : nb_launch_fwd_f32(d, q, n, tau, margin, out_bits, opt_logits, dev_stats, ws, s);
    else
        st = nb_tc_query(&m->tc, d, q, n, tau, margin, out_bits, opt_logits, dev_stats, ws, s);
    if (st != NB_OK) return st;
    return nb_launch_recheck(d, m->gamma, q, tau, out_bits, dev_stats, ws, n, s);
}

extern "C" nb_status nb_model_check(nb_model *m, void *stream) {
    if (!m) return nb_fail(NB_EINVAL, "nb_model_check: null model");
    NB_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    NB_CUDA(cudaGetLastError());
    return nb_tc_check(&m->tc);
}

// ---------------------------------------------------------------- queries from host memory
namespace {
__global__ void add_query_stats_kernel(nb_query_stats *sum, const nb_query_stats *part) {
    sum->n_inside += part->n_inside;
    sum->n_flagged += part->n_flagged;
    sum->n_resolved_f32 += part->n_resolved_f32;
    sum->n_resolved_ff += part->n_resolved_ff;
    sum->n_unresolved += part->n_unresolved;
    sum->n_nonfinite += part->n_nonfinite;
}
}  // namespace

static nb_status ensure_host_pipe(nb_model *m, int64_t chunk) {
    const int w = m->widths[0];
    // each piece is checked on its own, so a call after a failed set-up completes it
    // instead of using a part that does not exist
    if (!m->hq_stream) NB_CUDA(cudaStreamCreateWithFlags(&m->hq_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; b++) {
        if (!m->hq_ready[b]) NB_CUDA(cudaEventCreateWithFlags(&m->hq_ready[b], cudaEventDisableTiming));
        if (!m->hq_done[b]) NB_CUDA(cudaEventCreateWithFlags(&m->hq_done[b], cudaEventDisableTiming));
    }
    if (!m->hq_stats && cudaMalloc(&m->hq_stats, 3 * sizeof(nb_query_stats)) != cudaSuccess) {
        cudaGetLastError();
        m->hq_stats = nullptr;
        return nb_fail(NB_ENOMEM, "nb_query_host: allocation failed");
    }
    if (chunk <= m->hq_chunk) return NB_OK;
    NB_CUDA(cudaDeviceSynchronize());
    for (int b = 0; b < 2; b++) {
        cudaFree(m->hq_q[b]);
        cudaFree(m->hq_bits[b]);
        m->hq_q[b] = nullptr;
        m->hq_bits[b] = nullptr;
    }
    m->hq_chunk = 0;
    for (int b = 0; b < 2; b++)
        if (cudaMalloc(&m->hq_q[b], (size_t)chunk * w * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&m->hq_bits[b], (size_t)chunk / 32 * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return nb_fail(NB_ENOMEM, "nb_query_host: staging allocation failed");
        }
    m->hq_chunk = chunk;
    return NB_OK;
}

// The device address of pinned, mapped host memory when the link to the host is coherent
// (NVLink-C2C on a Grace-Blackwell node: native host atomics), else null.  Over C2C the
// forward reads its query rows from host memory at the rate it consumes them, so the
// staging copy buys nothing; over PCIe it would starve the forward.
static const float *mapped_host_rows(const float *host_q) {
    int dev = 0, coherent = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coherent, cudaDevAttrHostNativeAtomicSupported, dev) != cudaSuccess || !coherent) {
        cudaGetLastError();
        return nullptr;
    }
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host_q) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? (const float *)a.devicePointer : nullptr;
}

// nb_query on rows the device reads in place from mapped host memory; the bits go to a
// library-owned device buffer and are copied back once final.  Synchronous.
static nb_status query_in_place(nb_model *m, const float *dq, int64_t n, float margin, uint32_t *host_bits,
                                nb_query_stats *host_stats, cudaStream_t S) {
    const int64_t words = (n + 31) / 32;
    nb_status st = ensure_host_pipe(m, 32);  // the copy stream, events and statistics
    if (st != NB_OK) return st;
    if (words > m->zc_words) {
        NB_CUDA(cudaStreamSynchronize(S));
        cudaFree(m->zc_bits);
        m->zc_bits = nullptr;
        m->zc_words = 0;
        if (cudaMalloc(&m->zc_bits, (size_t)words * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return nb_fail(NB_ENOMEM, "nb_query_host: bits buffer allocation failed");
        }
        m->zc_words = words;
    }
    nb_query_stats *sum = m->hq_stats + 2;
    st = nb_query(m, dq, n, margin, m->zc_bits, nullptr, host_stats ? sum : nullptr, S);
    if (st != NB_OK) {
        cudaStreamSynchronize(S);  // kernels already queued may still read the caller's rows
        return st;
    }
    if (cudaMemcpyAsync(host_bits, m->zc_bits, (size_t)words * sizeof(uint32_t), cudaMemcpyDeviceToHost, S) !=
            cudaSuccess ||
        (host_stats &&
         cudaMemcpyAsync(host_stats, sum, sizeof(nb_query_stats), cudaMemcpyDeviceToHost, S) != cudaSuccess)) {
        cudaStreamSynchronize(S);
        return nb_fail(NB_ECUDA, "nb_query_host: copy failed");
    }
    NB_CUDA(cudaStreamSynchronize(S));
    return nb_tc_check(&m->tc);
}

extern "C" nb_status nb_query_host(nb_model *m, const float *host_q, int64_t n, float margin, uint32_t *host_bits,
                                   nb_query_stats *host_stats, int64_t chunk_rows, void *stream) {
    if (!m) return nb_fail(NB_EINVAL, "nb_query_host: null model");
    if (n < 0 || n >= (int64_t)1 << 32) return nb_fail(NB_EINVAL, "nb_query_host: n must be in [0, 2^32)");
    if (n > 0 && (!host_q || !host_bits)) return nb_fail(NB_EINVAL, "nb_query_host: null pointer");
    if (chunk_rows < 0) return nb_fail(NB_EINVAL, "nb_query_host: chunk_rows must be >= 0");
    if (host_stats) memset(host_stats, 0, sizeof(nb_query_stats));
    if (n == 0) return NB_OK;
    if (chunk_rows == 0) {
        const float *dq = mapped_host_rows(host_q);
        if (dq) return query_in_place(m, dq, n, margin, host_bits, host_stats, (cudaStream_t)stream);
    }
    const int w = m->widths[0];
    int64_t C = chunk_rows > 0 ? chunk_rows : ((int64_t)1 << 22);
    C = (C + 31) / 32 * 32;
    if (C > (n + 31) / 32 * 32) C = (n + 31) / 32 * 32;
    nb_status st = ensure_host_pipe(m, C);
    if (st != NB_OK) return st;
    cudaStream_t S = (cudaStream_t)stream, cs = m->hq_stream;
    nb_query_stats *sum = m->hq_stats + 2;
    if (host_stats) NB_CUDA(cudaMemsetAsync(sum, 0, sizeof(nb_query_stats), S));
    // Copy stream: H2D(0), then for each chunk i: H2D(i + 1), D2H(i).  H2D(i + 1) reuses the
    // buffer of chunk i - 1, whose D2H precedes it on the copy stream and waited for that
    // chunk's query; the query of chunk i runs on `stream` while chunk i + 1 is copied in.
    // chunk boundaries: the first chunk is a quarter of the others (a multiple of 32), so
    // the forward starts after a short first copy
    std::vector<int64_t> start;
    const int64_t first = std::max<int64_t>(32, C / 4 / 32 * 32);
    for (int64_t r0 = 0; r0 < n; r0 += (r0 == 0 ? first : C)) start.push_back(r0);
    start.push_back(n);
    const int64_t nch = (int64_t)start.size() - 1;
    auto rows_of = [&](int64_t i) { return start[i + 1] - start[i]; };
    auto h2d = [&](int64_t i) -> nb_status {
        const int b = (int)(i & 1);
        NB_CUDA(cudaMemcpyAsync(m->hq_q[b], host_q + (size_t)start[i] * w, (size_t)rows_of(i) * w * sizeof(float),
                                cudaMemcpyHostToDevice, cs));
        NB_CUDA(cudaEventRecord(m->hq_ready[b], cs));
        return NB_OK;
    };
    NB_CUDA(cudaStreamSynchronize(S));  // the staging buffers may still serve a query on `stream`
    // on any failure, let the copies already queued on the caller's host buffers finish
    // before returning
    auto drained = [&](nb_status e) {
        cudaStreamSynchronize(cs);
        cudaStreamSynchronize(S);
        return e;
    };
    st = h2d(0);
    if (st != NB_OK) return drained(st);
    for (int64_t i = 0; i < nch; i++) {
        const int b = (int)(i & 1);
        if (cudaStreamWaitEvent(S, m->hq_ready[b], 0) != cudaSuccess)
            return drained(nb_fail(NB_ECUDA, "nb_query_host: stream wait failed"));
        st = nb_query(m, m->hq_q[b], rows_of(i), margin, m->hq_bits[b], nullptr, host_stats ? m->hq_stats + b : nullptr,
                      S);
        if (st != NB_OK) return drained(st);
        if (host_stats) add_query_stats_kernel<<<1, 1, 0, S>>>(sum, m->hq_stats + b);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(m->hq_done[b], S) != cudaSuccess)
            return drained(nb_fail(NB_ECUDA, "nb_query_host: launch failed"));
        if (i + 1 < nch) {
            st = h2d(i + 1);
            if (st != NB_OK) return drained(st);
        }
        if (cudaStreamWaitEvent(cs, m->hq_done[b], 0) != cudaSuccess ||
            cudaMemcpyAsync(host_bits + (size_t)start[i] / 32, m->hq_bits[b],
                            (size_t)((rows_of(i) + 31) / 32) * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            cs) != cudaSuccess)
            return drained(nb_fail(NB_ECUDA, "nb_query_host: copy failed"));
    }
    NB_CUDA(cudaStreamSynchronize(cs));
    if (host_stats) {
        NB_CUDA(cudaMemcpyAsync(host_stats, sum, sizeof(nb_query_stats), cudaMemcpyDeviceToHost, S));
        NB_CUDA(cudaStreamSynchronize(S));
    }
    return nb_tc_check(&m->tc);  // synchronous already: report a forward that gave up waiting
}

// the workspace of the early-out and three-way queries, owned by one model; grows on demand
static nb_status ensure_eo_ws(nb_model *m, size_t need) {
    if (need <= m->eo_bytes) return NB_OK;
    NB_CUDA(cudaDeviceSynchronize());
    cudaFree(m->eo_ws);
    m->eo_ws = nullptr;
    m->eo_bytes = 0;
    if (cudaMalloc(&m->eo_ws, need) != cudaSuccess) {
        cudaGetLastError();
        return nb_fail(NB_ENOMEM, "workspace allocation failed");
    }
    m->eo_bytes = need;
    return NB_OK;
}

extern "C" nb_status nb_query_early_out(nb_model *early, nb_model *late, const float *q, int64_t n,
                                        float margin_early, float margin_late, uint32_t *out_bits,
                                        nb_early_stats *host_stats, void *stream) {
    if (!early || !late) return nb_fail(NB_EINVAL, "nb_query_early_out: null model");
    if (early->widths[0] != late->widths[0]) return nb_fail(NB_EINVAL, "nb_query_early_out: input widths differ");
    if (n < 0 || n >= (int64_t)1 << 32) return nb_fail(NB_EINVAL, "nb_query_early_out: n must be in [0, 2^32)");
    if (n > 0 && (!q || !out_bits)) return nb_fail(NB_EINVAL, "nb_query_early_out: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    if (host_stats) memset(host_stats, 0, sizeof(nb_early_stats));
    if (n == 0) return NB_OK;
    const int w = late->widths[0];
    const size_t words = align256((size_t)((n + 31) / 32) * 4), list = align256((size_t)n * 4);
    const size_t need = 256 + 2 * words + list + align256((size_t)n * w * sizeof(float));
    nb_status st = ensure_eo_ws(late, need);
    if (st != NB_OK) return st;
    char *base = (char *)late->eo_ws;
    unsigned *count = (unsigned *)base;
    uint32_t *bits_e = (uint32_t *)(base + 256);
    uint32_t *bits_c = (uint32_t *)(base + 256 + words);
    unsigned *idx = (unsigned *)(base + 256 + 2 * words);
    float *qc = (float *)(base + 256 + 2 * words + list);
    const MlpDesc de = desc_of(early);
    // a one-hidden-layer FP32 early network (the paper's early exit) settles rows and
    // gathers the others in one pass, its decisions certified by a rigorous bound
    const bool fused = early->infer_prec == NB_F32 && nb_early_settle_eligible(de);
    if (fused) {
        st = ensure_pT(early, s);
        if (st != NB_OK) return st;
        NB_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned), s));
        // bits_e holds each word's start in the gathered rows
        st = nb_launch_early_settle(de, q, n, nb_tau_bracket(early->tau), margin_early, out_bits, count, bits_e, qc,
                                    s);
        if (st != NB_OK) return st;
    } else {
        // 1. the early network on every row (certified decisions against its threshold)
        st = nb_query(early, q, n, margin_early, bits_e, nullptr, nullptr, stream);
        if (st != NB_OK) return st;
        // 2. rows it settles are inside; the others are listed
        st = nb_launch_early_compact(bits_e, n, count, idx, out_bits, s);
        if (st != NB_OK) return st;
    }
    unsigned m = 0;
    NB_CUDA(cudaMemcpyAsync(&m, count, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    // 3. the late network on the remaining rows only
    if (m > 0) {
        if (!fused) {
            st = nb_launch_early_gather(q, w, idx, m, qc, s);
            if (st != NB_OK) return st;
        }
        st = nb_query(late, qc, m, margin_late, bits_c, nullptr, nullptr, stream);
        if (st != NB_OK) return st;
        st = fused ? nb_launch_early_merge(bits_c, bits_e, n, out_bits, s)
                   : nb_launch_early_scatter(bits_c, idx, m, out_bits, s);
        if (st != NB_OK) return st;
    }
    if (host_stats) {
        host_stats->n_early_inside = (uint64_t)(n - m);
        host_stats->n_late = m;
    }
    st = nb_tc_check(&early->tc);
    return st != NB_OK ? st : nb_tc_check(&late->tc);
}

extern "C" nb_status nb_query_three_way(nb_model *outer, nb_model *inner, const float *q, int64_t n,
                                        float margin_outer, float margin_inner, uint8_t *codes,
                                        nb_three_way_stats *dev_stats, void *stream) {
    if (!outer || !inner) return nb_fail(NB_EINVAL, "nb_query_three_way: null model");
    if (outer->widths[0] != inner->widths[0]) return nb_fail(NB_EINVAL, "nb_query_three_way: input widths differ");
    if (n < 0 || n >= (int64_t)1 << 32) return nb_fail(NB_EINVAL, "nb_query_three_way: n must be in [0, 2^32)");
    if (n > 0 && (!q || !codes)) return nb_fail(NB_EINVAL, "nb_query_three_way: null pointer");
    if (n == 0) return NB_OK;
    const size_t words = align256((size_t)((n + 31) / 32) * 4);
    nb_status st = ensure_eo_ws(outer, 2 * words);
    if (st != NB_OK) return st;
    uint32_t *bits_o = (uint32_t *)outer->eo_ws;
    uint32_t *bits_i = (uint32_t *)((char *)outer->eo_ws + words);
    // both bounds, each certified against its own threshold
    st = nb_query(outer, q, n, margin_outer, bits_o, nullptr, nullptr, stream);
    if (st != NB_OK) return st;
    st = nb_query(inner, q, n, margin_inner, bits_i, nullptr, nullptr, stream);
    if (st != NB_OK) return st;
    return nb_launch_three_way(bits_o, bits_i, n, codes, dev_stats, (cudaStream_t)stream);
}

extern "C" nb_status nb_bits_not(const uint32_t *in, int64_t n, uint32_t *out, void *stream) {
    if (n < 0) return nb_fail(NB_EINVAL, "nb_bits_not: n must be >= 0");
    if (n == 0) return NB_OK;
    if (!in || !out) return nb_fail(NB_EINVAL, "nb_bits_not: null pointer");
    return nb_launch_bits_not(in, n, out, (cudaStream_t)stream);
}

extern "C" nb_status nb_calibrate(nb_model *m, const float *q, const uint32_t *label_bits, int64_t n, double eps,
                                  double *host_tau, void *stream) {
    if (!m || !host_tau) return nb_fail(NB_EINVAL, "nb_calibrate: null pointer");
    if (n < 0 || n >= (int64_t)1 << 32) return nb_fail(NB_EINVAL, "nb_calibrate: n must be in [0, 2^32)");
    if (n > 0 && (!q || !label_bits)) return nb_fail(NB_EINVAL, "nb_calibrate: null pointer");
    if (!(eps >= 0) || isinf(eps)) return nb_fail(NB_EINVAL, "nb_calibrate: eps must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        m->tau = INFINITY;
        *host_tau = m->tau;
        return NB_OK;
    }
    const size_t head = 256, list = align256((size_t)n * sizeof(unsigned));
    nb_status st = ensure_ws(m, head + 2 * list);
    if (st != NB_OK) return st;
    st = ensure_pT(m, s);
    if (st != NB_OK) return st;
    CalibWs ws;
    ws.umin_bits = (unsigned *)m->ws;
    ws.zmin_bits = (unsigned long long *)((char *)m->ws + 64);
    ws.npos = (unsigned *)((char *)m->ws + 128);
    ws.pos_idx = (unsigned *)((char *)m->ws + head);
    ws.lo = (float *)((char *)m->ws + head + list);
    st = nb_launch_calibrate(desc_of(m), m->gamma, q, label_bits, 0, n, ws, s);
    if (st != NB_OK) return st;
    unsigned long long h[2] = {0, 0};
    unsigned npos = 0;
    NB_CUDA(cudaMemcpyAsync(&h[0], ws.zmin_bits, 8, cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaMemcpyAsync(&npos, ws.npos, 4, cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    h[1] = npos;
    const double tau = nb_tau_from_min_bits(h[0], (unsigned)h[1], eps);
    m->tau = tau;
    *host_tau = tau;
    return NB_OK;
}

// ---------------------------------------------------------------- no-allocation training step
// Scratch for nb_train_step_noalloc: per-CTA gradient partials followed by the per-CTA
// loss partials.  Host code must not pass the symbol itself to a kernel (on the host
// it names a host-side stand-in); its device address is looked up once per device.
static __device__ __align__(256) float g_noalloc_scratch[NB_NOALLOC_SCRATCH_FLOATS];

static std::mutex g_noalloc_mu;
static float *g_noalloc_ptr[256] = {nullptr};

static nb_status noalloc_scratch(float **out) {
    int dev = 0;
    NB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return nb_fail(NB_EUNSUPPORTED, "nb_train_step_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return nb_cuda_check(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[dev] = (float *)p;
    }
    *out = g_noalloc_ptr[dev];
    return NB_OK;
}

extern "C" nb_status nb_train_step_noalloc(nb_model *m, const float *q, const uint32_t *label_bits, int64_t n,
                                           float alpha, float beta, nb_step_stats *dev_stats, void *stream) {
    if (!m) return nb_fail(NB_EINVAL, "nb_train_step_noalloc: null model");
    if (n < 1) return nb_fail(NB_EINVAL, "nb_train_step_noalloc: n must be >= 1");
    if (!q || !label_bits) return nb_fail(NB_EINVAL, "nb_train_step_noalloc: null pointer");
    if (!(alpha >= 0) || !(beta >= 0) || isinf(alpha) || isinf(beta))
        return nb_fail(NB_EINVAL, "nb_train_step_noalloc: alpha and beta must be finite and >= 0");
    if (m->train_prec != NB_F32)
        return nb_fail(NB_EUNSUPPORTED, "nb_train_step_noalloc: only the FP32 training precision is supported");
    if ((uint64_t)m->P + 1 > (uint64_t)NB_NOALLOC_SCRATCH_FLOATS)
        return nb_fail(NB_EINVAL, "nb_train_step_noalloc: the network has " + std::to_string(m->P) +
                                      " parameters; the static scratch holds networks of at most " +
                                      std::to_string(NB_NOALLOC_SCRATCH_FLOATS - 1));
    float *scratch = nullptr;
    nb_status st = noalloc_scratch(&scratch);
    if (st != NB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const MlpDesc d = desc_of(m);
    const TauF tau = nb_tau_bracket(m->tau);
    TrainWs tw{};
    const int64_t cap = (int64_t)NB_NOALLOC_SCRATCH_FLOATS / (m->P + 1);
    tw.G = nb_train_f32_ctas(d, n, sm_count());
    if (tw.G > cap) tw.G = (int)cap;
    tw.partial = scratch;
    tw.loss_partial = scratch + (size_t)tw.G * m->P;
    m->step += 1;
    const double c1 = 1.0 - pow((double)m->b1, (double)m->step);
    const double c2 = 1.0 - pow((double)m->b2, (double)m->step);
    st = nb_launch_train_f32(d, q, label_bits, n, alpha, beta, tau, tw, dev_stats, s);
    if (st != NB_OK) return st;
    st = nb_launch_adam(m->P, 1.0f / (float)n, m->params, m->adam_m, m->adam_v, m->grad, tw, m->lr, m->b1, m->b2,
                        m->eps, (float)c1, (float)sqrt(c2), dev_stats, s);
    if (st != NB_OK) return st;
    return refresh_after_step(m, s);
}
