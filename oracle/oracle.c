/*
 * oracle.c -- plain, slow, obviously correct FP64 / exact-integer CPU oracle for
 * the neural-bounding hot path (Liu et al., "Neural Bounding", SIGGRAPH 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only on the
 * seeded inputs drawn by paper_2310_06822_gb300/inputs.py.
 *
 * What it computes, each with the passage it follows:
 *   orc_label       exact query function g(r) (Sec. 3.1): 1 iff the region r
 *                   touches a point where the indicator f is 1, f being 1 inside
 *                   and ON the surface of a union of spheres.  Decided exactly in
 *                   128-bit integer arithmetic on grid-quantised inputs.
 *   orc_mc_label    Alg. 1's Any(f(SampleRegion(r))): g evaluated as "any" over
 *                   a lattice of sample points of the region (Sec. 4.2, "Query
 *                   types": any() over a sample of the indicator).  Test-only.
 *   orc_forward     bounding network h (Sec. 3.4 "Architecture"): MLP with ReLU
 *                   hidden layers (the configurations' activation) or, in the
 *                   _act forms with act = 1, the paper's sinusoidal hidden
 *                   activation sin(z); output logit z; sigmoid(z) rounded to
 *                   {0,1} is the decision z >= tau.
 *   orc_loss_grad   weighted binary cross-entropy of Eq. (loss) with weights
 *                   alpha(t) on y log(yhat) and beta(t) on (1-y) log(1-yhat),
 *                   mean over the batch, and its gradient by backpropagation.
 *   orc_adam        Adam (Sec. 3.4 "Training", Kingma & Ba), PyTorch defaults.
 *   orc_calibrate   output epsilon of Suppl. Sec. "Numerics": threshold
 *                   tau = (min over positives of z) - eps, rounded toward -inf.
 *   orc_count       FN / FP / TP / TN of the cost table of Sec. 3.1.
 *   orc_sample      Alg. 1's per-iteration draw of queries r ~ Uniform, made
 *                   reproducible by the counter-based Philox4x64-10 generator
 *                   (orc_philox4x64 exposes one block for its pin).
 *   orc_canonical_ray  the cascade's network input: a ray in an object's frame,
 *                   its origin moved to its entry into the ball around the
 *                   object (per-object networks, Sec. 2; hierarchy of tests,
 *                   Sec. 1), replaying the library's defined FP32 sequence;
 *                   orc_canonical_ray_f64 is the real-valued root it is pinned to.
 *
 * Number formats: every query and sphere value is an integer multiple of
 * 2^-qexp (see inputs.py).  Integer "units" below are multiples of 2^-qexp.
 * FP64 is used for the network; the weights are the FP32 master weights read
 * exactly.
 */
#include <fenv.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

enum { K_POINT2 = 0, K_POINT3, K_POINT4T, K_RAY3, K_PLANE3, K_BOX3 };
static const int ENC_W[6] = {2, 3, 4, 6, 4, 6};

/* x = v * 2^-qexp exactly, |v| < 2^50; returns 0 on success. */
static int units(float x, int qexp, int64_t *v) {
    double s = ldexp((double)x, qexp);
    if (!isfinite(s) || s != floor(s) || fabs(s) >= 1125899906842624.0) return -1;
    *v = (int64_t)s;
    return 0;
}

/* ---------------------------------------------------------------- scenes */
typedef struct {
    int dim;          /* 2 or 3 */
    int n;            /* number of spheres */
    const float *c;   /* [n][dim] centres */
    const float *r;   /* [n] radii */
    const float *v;   /* [n][3] velocities or NULL */
    int qexp;
} scene_t;

/* sphere s of the scene in integer units */
static int sphere_units(const scene_t *sc, int s, int64_t C[3], int64_t *R, int64_t V[3]) {
    for (int i = 0; i < 3; i++) { C[i] = 0; V[i] = 0; }
    for (int i = 0; i < sc->dim; i++)
        if (units(sc->c[s * sc->dim + i], sc->qexp, &C[i])) return -1;
    if (units(sc->r[s], sc->qexp, R) || *R < 0) return -1;
    if (sc->v)
        for (int i = 0; i < 3; i++)
            if (units(sc->v[s * 3 + i], sc->qexp, &V[i])) return -1;
    return 0;
}

/* ------------------------------------------------- exact predicates (Sec 3.1)
 * Each returns 1 iff the closed ball (C, R) meets the query region. */

/* point: |x - c|^2 <= r^2 */
static int hit_point(int dim, const int64_t X[], const int64_t C[], int64_t R) {
    i128 d2 = 0;
    for (int i = 0; i < dim; i++) { i128 d = (i128)X[i] - C[i]; d2 += d * d; }
    return d2 <= (i128)R * R;
}

/* space-time point (x, t) against a sphere whose centre moves as c + v t:
 * |x - c - v t|^2 <= r^2, everything scaled by 2^qexp so v t is an integer. */
static int hit_point4t(const int64_t X[], int64_t T, int qexp, const int64_t C[],
                       const int64_t V[], int64_t R) {
    i128 d2 = 0;
    for (int i = 0; i < 3; i++) {
        i128 d = ((i128)X[i] - C[i]) * ((i128)1 << qexp) - (i128)V[i] * T;
        d2 += d * d;
    }
    i128 rs = (i128)R * ((i128)1 << qexp);
    return d2 <= rs * rs;
}

/* half-line o + s d (s >= 0): squared distance from c to the half-line <= r^2.
 * With w = c - o: if w.d <= 0 the closest point is o; otherwise it is the foot
 * of the perpendicular, at squared distance |w|^2 - (w.d)^2/|d|^2. */
static int hit_ray(const int64_t O[], const int64_t D[], const int64_t C[], int64_t R) {
    i128 ww = 0, dd = 0, s = 0;
    for (int i = 0; i < 3; i++) {
        i128 w = (i128)C[i] - O[i];
        ww += w * w;
        dd += (i128)D[i] * D[i];
        s += w * D[i];
    }
    i128 rr = (i128)R * R;
    if (s <= 0) return ww <= rr;
    return ww * dd - s * s <= rr * dd;
}

/* plane {x : n.x = off}: distance |n.c - off| / |n| <= r */
static int hit_plane(const int64_t N[], int64_t OFF, int qexp, const int64_t C[], int64_t R) {
    i128 nc = 0, nn = 0;
    for (int i = 0; i < 3; i++) { nc += (i128)N[i] * C[i]; nn += (i128)N[i] * N[i]; }
    i128 d = nc - (i128)OFF * ((i128)1 << qexp);       /* units 2^-2qexp */
    i128 rr = (i128)R * R;                             /* units 2^-2qexp */
    return d * d <= rr * nn;                           /* units 2^-4qexp */
}

/* closed box centre b, half-extents e >= 0: squared distance from c to the box */
static int hit_box(const int64_t B[], const int64_t E[], const int64_t C[], int64_t R) {
    i128 d2 = 0;
    for (int i = 0; i < 3; i++) {
        i128 a = (i128)C[i] - B[i];
        if (a < 0) a = -a;
        a -= E[i];
        if (a > 0) d2 += a * a;
    }
    return d2 <= (i128)R * R;
}

/* query q (one encoding row) against the whole union: OR over spheres */
static int label_one(int kind, const float *q, const scene_t *sc) {
    int64_t Q[6];
    for (int i = 0; i < ENC_W[kind]; i++)
        if (units(q[i], sc->qexp, &Q[i])) return -1;
    if (kind == K_BOX3 && (Q[3] < 0 || Q[4] < 0 || Q[5] < 0)) return -1;
    for (int s = 0; s < sc->n; s++) {
        int64_t C[3], V[3], R;
        if (sphere_units(sc, s, C, &R, V)) return -1;
        int h = 0;
        switch (kind) {
        case K_POINT2: h = hit_point(2, Q, C, R); break;
        case K_POINT3: h = hit_point(3, Q, C, R); break;
        case K_POINT4T: h = hit_point4t(Q, Q[3], sc->qexp, C, V, R); break;
        case K_RAY3: h = hit_ray(Q, Q + 3, C, R); break;
        case K_PLANE3: h = hit_plane(Q, Q[3], sc->qexp, C, R); break;
        case K_BOX3: h = hit_box(Q, Q + 3, C, R); break;
        default: return -1;
        }
        if (h) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------ parallel for */
typedef struct {
    void (*fn)(void *ctx, int64_t lo, int64_t hi, int tid);
    void *ctx;
    int64_t lo, hi;
    int tid;
} job_t;

static void *job_run(void *p) {
    job_t *j = (job_t *)p;
    j->fn(j->ctx, j->lo, j->hi, j->tid);
    return NULL;
}

static void parallel_for(int64_t n, int nthreads, void (*fn)(void *, int64_t, int64_t, int), void *ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < nthreads) nthreads = n > 0 ? (int)n : 1;
    pthread_t th[256];
    job_t jobs[256];
    for (int t = 0; t < nthreads; t++) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].lo = n * t / nthreads;
        jobs[t].hi = n * (t + 1) / nthreads;
        jobs[t].tid = t;
    }
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, job_run, &jobs[t]);
    job_run(&jobs[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------- label */
typedef struct {
    int kind;
    const float *q;
    const scene_t *sc;
    uint8_t *out;
    int err;
} label_ctx;

static void label_range(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    label_ctx *c = (label_ctx *)p;
    for (int64_t i = lo; i < hi; i++) {
        int h = label_one(c->kind, c->q + i * ENC_W[c->kind], c->sc);
        if (h < 0) { c->err = 1; h = 1; }
        c->out[i] = (uint8_t)h;
    }
}

/* Exact labels y_i = g(q_i) for n queries.  Returns 0, or -1 if an input is
 * off the grid, non-finite, or a box has a negative half-extent. */
int orc_label(int kind, const float *q, int64_t n, int dim, int n_spheres, const float *centres,
              const float *radii, const float *vel, int qexp, uint8_t *out, int nthreads) {
    if (kind < 0 || kind > 5) return -1;
    scene_t sc = {dim, n_spheres, centres, radii, vel, qexp};
    if (kind == K_POINT2 && dim != 2) return -1;
    if (kind != K_POINT2 && dim != 3) return -1;
    if (kind == K_POINT4T && !vel) return -1;
    label_ctx c = {kind, q, &sc, out, 0};
    parallel_for(n, nthreads, label_range, &c);
    return c.err ? -1 : 0;
}

/* --------------------------------------------------------- MC labelling
 * Alg. 1 style: y = Any(f(samples of the region)), with sample points on an
 * exact lattice so f is evaluated exactly at each sample.
 *   ray:   points o + (k / 2^m) d for k = 0 .. kmax
 *   box:   points b + (j / J) e per axis, j in {-J..J}
 *   plane: the plane meets a ball iff the ball has lattice points on both
 *          closed sides of it; samples are c + (a,b,c) r / J with |(a,b,c)| <= J.
 * A sample set can only miss a contact, so MC = 1 implies exact = 1. */
int orc_mc_label(int kind, const float *q, int64_t n, int n_spheres, const float *centres,
                 const float *radii, int qexp, int density, uint8_t *out) {
    scene_t sc = {3, n_spheres, centres, radii, NULL, qexp};
    for (int64_t i = 0; i < n; i++) {
        int64_t Q[6];
        for (int k = 0; k < ENC_W[kind]; k++)
            if (units(q[i * ENC_W[kind] + k], qexp, &Q[k])) return -1;
        int hit = 0;
        for (int s = 0; s < n_spheres && !hit; s++) {
            int64_t C[3], V[3], R;
            if (sphere_units(&sc, s, C, &R, V)) return -1;
            if (kind == K_RAY3) {
                /* m = density, samples up to parameter 5 along d */
                int m = density;
                int64_t kmax = (int64_t)5 << m;
                for (int64_t k = 0; k <= kmax && !hit; k++) {
                    i128 d2 = 0;
                    for (int a = 0; a < 3; a++) {
                        i128 p = (i128)Q[a] * ((i128)1 << m) + (i128)k * Q[3 + a];
                        i128 dd = p - (i128)C[a] * ((i128)1 << m);
                        d2 += dd * dd;
                    }
                    i128 rs = (i128)R * ((i128)1 << m);
                    hit = d2 <= rs * rs;
                }
            } else if (kind == K_BOX3) {
                int J = density;
                for (int a = -J; a <= J && !hit; a++)
                    for (int b = -J; b <= J && !hit; b++)
                        for (int c = -J; c <= J && !hit; c++) {
                            int jj[3] = {a, b, c};
                            i128 d2 = 0;
                            for (int x = 0; x < 3; x++) {
                                i128 p = (i128)Q[x] * J + (i128)jj[x] * Q[3 + x];
                                i128 dd = p - (i128)C[x] * J;
                                d2 += dd * dd;
                            }
                            hit = d2 <= (i128)R * R * J * J;
                        }
            } else if (kind == K_PLANE3) {
                int J = density, pos = 0, neg = 0;
                for (int a = -J; a <= J && !(pos && neg); a++)
                    for (int b = -J; b <= J && !(pos && neg); b++)
                        for (int c = -J; c <= J && !(pos && neg); c++) {
                            if (a * a + b * b + c * c > J * J) continue;
                            int jj[3] = {a, b, c};
                            i128 sJ = 0; /* J * (n.p - off), units 2^-2qexp */
                            for (int x = 0; x < 3; x++)
                                sJ += (i128)Q[x] * ((i128)C[x] * J + (i128)jj[x] * R);
                            sJ -= (i128)Q[3] * J * ((i128)1 << qexp);
                            if (sJ >= 0) pos = 1;
                            if (sJ <= 0) neg = 1;
                        }
                hit = pos && neg;
            } else {
                return -1;
            }
        }
        out[i] = (uint8_t)hit;
    }
    return 0;
}

/* --------------------------------------------------------------- network
 * widths[0] = input width, widths[L] = 1; flat parameters: for each layer l,
 * W_l (widths[l+1] x widths[l], row-major) then b_l (widths[l+1]). */
#define MAXW 1024

static int64_t layer_offset(const int *widths, int l) {
    int64_t o = 0;
    for (int i = 0; i < l; i++) o += (int64_t)widths[i + 1] * (widths[i] + 1);
    return o;
}

int64_t orc_param_count(const int *widths, int L) { return layer_offset(widths, L); }

/* hidden activation: act 0 = ReLU max(z, 0) (the configurations), act 1 = sin(z), the
 * sinusoidal activation of Sec. 3.4 "Architecture" (no frequency factor is stated) */
static double activate(int act, double z) { return act ? sin(z) : (z > 0.0 ? z : 0.0); }
/* its derivative: ReLU'(z) = 1[z > 0], sin'(z) = cos(z) */
static double activate_d(int act, double z) { return act ? cos(z) : (z > 0.0 ? 1.0 : 0.0); }

/* forward pass of one query; keeps every layer's pre-activation z_l and
 * activation a_l (a_0 = x) in acts[l] / pre[l] when they are not NULL. */
static double forward_one(const int *widths, int L, int act, const float *params, const float *x,
                          double acts[][MAXW], double pre[][MAXW]) {
    double a[MAXW], z[MAXW];
    for (int k = 0; k < widths[0]; k++) a[k] = (double)x[k];
    if (acts) memcpy(acts[0], a, sizeof(double) * widths[0]);
    for (int l = 0; l < L; l++) {
        const float *W = params + layer_offset(widths, l);
        const float *b = W + (int64_t)widths[l + 1] * widths[l];
        for (int j = 0; j < widths[l + 1]; j++) {
            double s = (double)b[j];
            for (int k = 0; k < widths[l]; k++) s += (double)W[(int64_t)j * widths[l] + k] * a[k];
            z[j] = s;
        }
        if (pre) memcpy(pre[l + 1], z, sizeof(double) * widths[l + 1]);
        if (l < L - 1) {
            for (int j = 0; j < widths[l + 1]; j++) a[j] = activate(act, z[j]);
            if (acts) memcpy(acts[l + 1], a, sizeof(double) * widths[l + 1]);
        }
    }
    return z[0];
}

typedef struct {
    const int *widths;
    int L, act;
    const float *params;
    const float *X;
    double *z;
} fwd_ctx;

static void fwd_range(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    fwd_ctx *c = (fwd_ctx *)p;
    for (int64_t i = lo; i < hi; i++)
        c->z[i] = forward_one(c->widths, c->L, c->act, c->params, c->X + i * c->widths[0], NULL, NULL);
}

/* conditioning scale of the output logit: sum_k |W_L[k]| a_{L-1}[k] + |b_L|, the
 * magnitude the FP32 rounding error of the last layer is relative to */
int orc_forward_scale_act(const int *widths, int L, int act, const float *params, const float *X, int64_t n,
                          double *scale) {
    if (L < 1 || widths[L] != 1) return -1;
    double (*acts)[MAXW] = malloc(sizeof(double) * MAXW * (L + 1));
    const float *W = params + layer_offset(widths, L - 1);
    for (int64_t i = 0; i < n; i++) {
        forward_one(widths, L, act, params, X + i * widths[0], acts, NULL);
        double s = fabs((double)W[widths[L - 1]]);
        for (int k = 0; k < widths[L - 1]; k++) s += fabs((double)W[k]) * fabs(acts[L - 1][k]);
        scale[i] = s;
    }
    free(acts);
    return 0;
}

int orc_forward_scale(const int *widths, int L, const float *params, const float *X, int64_t n,
                      double *scale) {
    return orc_forward_scale_act(widths, L, 0, params, X, n, scale);
}

int orc_forward_act(const int *widths, int L, int act, const float *params, const float *X, int64_t n, double *z,
                    int nthreads) {
    if (L < 1 || widths[L] != 1 || act < 0 || act > 1) return -1;
    for (int l = 0; l <= L; l++)
        if (widths[l] < 1 || widths[l] > MAXW) return -1;
    fwd_ctx c = {widths, L, act, params, X, z};
    parallel_for(n, nthreads, fwd_range, &c);
    return 0;
}

int orc_forward(const int *widths, int L, const float *params, const float *X, int64_t n, double *z,
                int nthreads) {
    return orc_forward_act(widths, L, 0, params, X, n, z, nthreads);
}

/* softplus(u) = log(1 + e^u), evaluated without overflow */
static double softplus(double u) { return u > 0 ? u + log1p(exp(-u)) : log1p(exp(u)); }
static double sigmoid(double u) { return u >= 0 ? 1.0 / (1.0 + exp(-u)) : exp(u) / (1.0 + exp(u)); }

typedef struct {
    const int *widths;
    int L, act;
    const float *params;
    const float *X;
    const uint8_t *y;
    double alpha, beta;
    int64_t n, P;
    double *gpart;    /* [nthreads][P] */
    double *lpart;    /* [nthreads] */
} lg_ctx;

static void lg_range(void *p, int64_t lo, int64_t hi, int tid) {
    lg_ctx *c = (lg_ctx *)p;
    const int *w = c->widths;
    int L = c->L;
    double *g = c->gpart + (int64_t)tid * c->P;
    double (*acts)[MAXW] = malloc(sizeof(double) * MAXW * (L + 1));
    double (*pre)[MAXW] = malloc(sizeof(double) * MAXW * (L + 1));
    double delta[MAXW], dprev[MAXW];
    double loss = 0.0;
    for (int64_t i = lo; i < hi; i++) {
        double z = forward_one(w, L, c->act, c->params, c->X + i * w[0], acts, pre);
        double y = c->y[i] ? 1.0 : 0.0;
        /* Eq. (loss): -[alpha y log(s) + beta (1-y) log(1-s)], s = sigmoid(z)
         * -log(s) = softplus(-z), -log(1-s) = softplus(z) */
        loss += c->alpha * y * softplus(-z) + c->beta * (1.0 - y) * softplus(z);
        /* d/dz of the per-sample term, divided by n for the batch mean */
        double s = sigmoid(z);
        delta[0] = (c->alpha * y * (s - 1.0) + c->beta * (1.0 - y) * s) / (double)c->n;
        for (int l = L - 1; l >= 0; l--) {
            int64_t off = layer_offset(w, l);
            const float *W = c->params + off;
            double *gW = g + off, *gb = gW + (int64_t)w[l + 1] * w[l];
            for (int j = 0; j < w[l + 1]; j++) {
                gb[j] += delta[j];
                for (int k = 0; k < w[l]; k++) gW[(int64_t)j * w[l] + k] += delta[j] * acts[l][k];
            }
            if (l > 0) {
                for (int k = 0; k < w[l]; k++) {
                    double s2 = 0.0;
                    for (int j = 0; j < w[l + 1]; j++) s2 += (double)W[(int64_t)j * w[l] + k] * delta[j];
                    dprev[k] = s2 * activate_d(c->act, pre[l][k]);   /* dL/dz_k = dL/da_k act'(z_k) */
                }
                memcpy(delta, dprev, sizeof(double) * w[l]);
            }
        }
    }
    c->lpart[tid] = loss;
    free(acts);
    free(pre);
}

/* mean asymmetric BCE over the batch and its gradient w.r.t. the flat parameters */
int orc_loss_grad_act(const int *widths, int L, int act, const float *params, const float *X, const uint8_t *y,
                      int64_t n, double alpha, double beta, double *loss, double *grad, int nthreads) {
    if (L < 1 || widths[L] != 1 || n < 1 || act < 0 || act > 1) return -1;
    for (int l = 0; l <= L; l++)
        if (widths[l] < 1 || widths[l] > MAXW) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < nthreads) nthreads = (int)n;
    int64_t P = layer_offset(widths, L);
    double *gpart = calloc((size_t)nthreads * P, sizeof(double));
    double *lpart = calloc((size_t)nthreads, sizeof(double));
    lg_ctx c = {widths, L, act, params, X, y, alpha, beta, n, P, gpart, lpart};
    parallel_for(n, nthreads, lg_range, &c);
    double ls = 0.0;
    for (int64_t p = 0; p < P; p++) grad[p] = 0.0;
    for (int t = 0; t < nthreads; t++) {
        ls += lpart[t];
        for (int64_t p = 0; p < P; p++) grad[p] += gpart[(int64_t)t * P + p];
    }
    *loss = ls / (double)n;
    free(gpart);
    free(lpart);
    return 0;
}

int orc_loss_grad(const int *widths, int L, const float *params, const float *X, const uint8_t *y,
                  int64_t n, double alpha, double beta, double *loss, double *grad, int nthreads) {
    return orc_loss_grad_act(widths, L, 0, params, X, y, n, alpha, beta, loss, grad, nthreads);
}

/* Adam (Kingma & Ba) step t >= 1 with bias correction, in place */
void orc_adam(int64_t P, double *theta, double *m, double *v, const double *g, double lr, double b1,
              double b2, double eps, int64_t t) {
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t p = 0; p < P; p++) {
        m[p] = b1 * m[p] + (1.0 - b1) * g[p];
        v[p] = b2 * v[p] + (1.0 - b2) * g[p] * g[p];
        double mh = m[p] / c1, vh = v[p] / c2;
        theta[p] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* tau = (min over queries with y = 1 of z) - eps, rounded toward -infinity;
 * +inf when there is no positive.  Returns the number of positives. */
int64_t orc_calibrate(const double *z, const uint8_t *y, int64_t n, double eps, double *tau) {
    double mn = INFINITY;
    int64_t npos = 0;
    for (int64_t i = 0; i < n; i++)
        if (y[i]) { npos++; if (z[i] < mn) mn = z[i]; }
    if (npos == 0) { *tau = INFINITY; return 0; }
    int old = fegetround();
    fesetround(FE_DOWNWARD);
    volatile double t = mn - eps;
    fesetround(old);
    *tau = t;
    return npos;
}

/* cost-table counts of Sec. 3.1 for the decision z >= tau (out: FN FP TP TN) */
void orc_count(const double *z, const uint8_t *y, int64_t n, double tau, int64_t out[4]) {
    out[0] = out[1] = out[2] = out[3] = 0;
    for (int64_t i = 0; i < n; i++) {
        int d = z[i] >= tau;
        if (y[i] && !d) out[0]++;
        else if (!y[i] && d) out[1]++;
        else if (y[i] && d) out[2]++;
        else out[3]++;
    }
}

/* ----------------------------------------------------------- query sampling
 * Alg. 1 draws a fresh batch of queries r ~ Uniform every iteration.  The
 * uniform draws are made reproducible, independently of how they are computed,
 * by a counter-based generator: Philox4x64-10 (Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011), written here from
 * its published definition (round function, multipliers and Weyl key
 * increments of that paper).  Query i of a stream (seed, kind) reads the blocks
 *     philox(counter = (i, j, p, 0), key = (seed, kind)),
 * p = 0 for its scalars (j = 0) and p = 1, 2 for its first and second unit
 * vector (j = 0, 1, ... for the rejection attempts).
 *
 * From the 64-bit words w of a block (all values integer multiples of 2^-qexp,
 * 8 <= qexp <= 20):
 *   coordinate U[-1,1):  field s (21 bits at bit 21 s) of w, minus 2^20, read
 *                        in units of 2^-20 and truncated to the grid;
 *                        here: the top qexp+1 bits of the field, minus 2^qexp.
 *   time U[0,1):         the low qexp bits of w1 (4D points).
 *   unit vector:         v = three 21-bit fields minus 2^20 of one word,
 *                        accepted when 2^30 <= |v|^2 <= 2^40 (uniform in a
 *                        shell, so v/|v| is uniform on S^2); words are tried in
 *                        order w0..w3 of blocks j = 0..15, (0,0,1) if none is
 *                        accepted; u = v / sqrt(|v|^2) in FP32 (|v|^2 rounded to
 *                        float, IEEE square root and division), rounded to the
 *                        grid (nearest, ties to even).
 *   log-uniform [a, b]:  a * 2^(x log2(b/a)) in FP32, x = (w >> 40) 2^-24, with
 *                        2^f for the fractional part f evaluated as the degree-9
 *                        Taylor polynomial of exp(f ln 2) (coefficients 1/k!
 *                        rounded to float, Horner form); rounded to the grid.
 *                        Every constant is a float literal; every operation is
 *                        one IEEE float operation (no contraction).
 * Encodings: point (x from the fields of w0), 4D point (x, t), ray (2 u1, u2),
 * plane (u1, off from field 0 of w0), box (centre from w0, half-extent of axis
 * d log-uniform in [0.01, 0.5] from w_{1+d}).
 */
static const uint64_t PH_M0 = 0xD2E7470EE14C6C93ull, PH_M1 = 0xCA5A826395121157ull;
static const uint64_t PH_W0 = 0x9E3779B97F4A7C15ull, PH_W1 = 0xBB67AE8584CAA73Bull;

static void philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        unsigned __int128 p0 = (unsigned __int128)PH_M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)PH_M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        x0 = hi1 ^ x1 ^ k0;
        x1 = lo1;
        x2 = hi0 ^ x3 ^ k1;
        x3 = lo0;
        k0 += PH_W0;
        k1 += PH_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Test hook: one Philox4x64-10 block. */
void orc_philox4x64(const uint64_t *ctr, const uint64_t *key, uint64_t *out) { philox4x64_10(ctr, key, out); }

static void sample_block(uint64_t seed, int kind, int64_t i, uint64_t j, uint64_t p, uint64_t w[4]) {
    const uint64_t ctr[4] = {(uint64_t)i, j, p, 0};
    const uint64_t key[2] = {seed, (uint64_t)kind};
    philox4x64_10(ctr, key, w);
}

static int64_t field21(uint64_t w, int s) { return (int64_t)((w >> (21 * s)) & 0x1FFFFF) - 1048576; }

/* U[-1,1) coordinate in units of 2^-qexp */
static int64_t coord_units(uint64_t w, int s, int qexp) {
    const int64_t f = (int64_t)((w >> (21 * s)) & 0x1FFFFF);  /* [0, 2^21) */
    return (f >> (20 - qexp)) - ((int64_t)1 << qexp);
}

static float grid_round(float x, int qexp) { return ldexpf(rintf(ldexpf(x, qexp)), -qexp); }

static void unit_vector(uint64_t seed, int kind, int64_t i, uint64_t p, float u[3]) {
    for (uint64_t j = 0; j < 16; j++) {
        uint64_t w[4];
        sample_block(seed, kind, i, j, p, w);
        for (int m = 0; m < 4; m++) {
            const int64_t v0 = field21(w[m], 0), v1 = field21(w[m], 1), v2 = field21(w[m], 2);
            const int64_t n2 = v0 * v0 + v1 * v1 + v2 * v2;
            if (n2 >= ((int64_t)1 << 30) && n2 <= ((int64_t)1 << 40)) {
                const float len = sqrtf((float)n2);
                u[0] = (float)v0 / len;
                u[1] = (float)v1 / len;
                u[2] = (float)v2 / len;
                return;
            }
        }
    }
    u[0] = 0.0f; u[1] = 0.0f; u[2] = 1.0f;
}

/* 2^y for 0 <= y < 8: 2^floor(y) times the Taylor polynomial of exp(f ln 2) of degree 9,
 * f = y - floor(y), with the coefficients 1/k! rounded to float, in Horner form */
static float exp2_taylor(float y) {
    static const float c[10] = {0x1p+0f, 0x1p+0f, 0x1p-1f, 0x1.555556p-3f, 0x1.555556p-5f,
                                0x1.111112p-7f, 0x1.6c16c2p-10f, 0x1.a01a02p-13f, 0x1.a01a02p-16f,
                                0x1.71de3ap-19f};
    const float n = floorf(y);
    const float t = (y - n) * 0x1.62e43p-1f;
    float p = c[9];
    for (int k = 8; k >= 0; k--) p = p * t + c[k];
    return ldexpf(p, (int)n);
}

typedef struct {
    int kind, qexp;
    uint64_t seed;
    int64_t first;
    float *q;
} sample_ctx;

static void sample_range(void *pc, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    const sample_ctx *c = (const sample_ctx *)pc;
    const int qe = c->qexp;
    const double quantum = ldexp(1.0, -qe);
    for (int64_t r = lo; r < hi; r++) {
        const int64_t i = c->first + r;
        float *o = c->q + r * ENC_W[c->kind];
        uint64_t w[4];
        sample_block(c->seed, c->kind, i, 0, 0, w);
        float u[3], v[3];
        switch (c->kind) {
        case K_POINT2:
            for (int d = 0; d < 2; d++) o[d] = (float)((double)coord_units(w[0], d, qe) * quantum);
            break;
        case K_POINT3:
            for (int d = 0; d < 3; d++) o[d] = (float)((double)coord_units(w[0], d, qe) * quantum);
            break;
        case K_POINT4T:
            for (int d = 0; d < 3; d++) o[d] = (float)((double)coord_units(w[0], d, qe) * quantum);
            o[3] = (float)((double)(int64_t)(w[1] & (((uint64_t)1 << qe) - 1)) * quantum);
            break;
        case K_RAY3:
            unit_vector(c->seed, c->kind, i, 1, u);
            unit_vector(c->seed, c->kind, i, 2, v);
            for (int d = 0; d < 3; d++) {
                o[d] = grid_round(2.0f * u[d], qe);
                o[3 + d] = grid_round(v[d], qe);
            }
            break;
        case K_PLANE3:
            unit_vector(c->seed, c->kind, i, 1, u);
            for (int d = 0; d < 3; d++) o[d] = grid_round(u[d], qe);
            o[3] = (float)((double)coord_units(w[0], 0, qe) * quantum);
            break;
        case K_BOX3:
            for (int d = 0; d < 3; d++) {
                o[d] = (float)((double)coord_units(w[0], d, qe) * quantum);
                const float x = (float)(w[1 + d] >> 40) * 0x1p-24f;
                o[3 + d] = grid_round(0x1.47ae14p-7f * exp2_taylor(x * 0x1.6934fp+2f), qe);
            }
            break;
        }
    }
}

/* Queries first .. first+n-1 of the stream (seed, kind) into q[n][enc width].
 * Returns 0, or -1 for an unknown kind or qexp outside [8, 20]. */
int orc_sample(int kind, int qexp, uint64_t seed, int64_t first, int64_t n, float *q, int nthreads) {
    if (kind < 0 || kind > 5 || qexp < 8 || qexp > 20 || first < 0 || n < 0) return -1;
    sample_ctx c = {kind, qexp, seed, first, q};
    parallel_for(n, nthreads, sample_range, &c);
    return 0;
}

/* ------------------------------------------------ cascade: canonical ray
 * The learned-culler cascade (Sec. 1's hierarchy of a cheap conservative test in
 * front of an exact one; per-object networks, Sec. 2) hands each object's network
 * the ray in that object's frame with its origin moved to where it enters the ball
 * of radius R around the object's centre -- the distribution of ray origins the
 * network was trained on.  The paper leaves this frame open; the library defines
 * the transform as one fixed sequence of correctly rounded FP32 operations, and
 * this function replays that sequence (each line one IEEE float operation, fmaf
 * where the sequence fuses, -ffp-contract=off), so its results are the exact bits
 * the definition prescribes:
 *   w = o - c;  b = w.d;  dd = d.d;  ww = w.w            (sums left to right)
 *   x = w cross d, each component fmaf(w_i, d_j, -(w_j d_i))
 *   disc = dd R^2 - |x|^2     (Lagrange: equals b^2 - dd (ww - R^2))
 *   met  = disc >= 0 and dd > 0
 *   s = (ww - R^2) / (-b + sqrt(disc))   if -b > 0  (the smaller root, no cancellation)
 *     = (-b - sqrt(disc)) / dd            otherwise
 *   s = max(s, 0);  entry = w + s d
 * R2 is R^2 as a float (the caller squares R in FP32).  Output q6 = (entry, d) and
 * met (0: the ray misses the ball; q6 is then zero).
 * orc_canonical_ray_f64 computes the same entry point in FP64 from the same float
 * inputs; it exists only to pin the FP32 sequence against the real-valued root. */
static void canon_f32(const float o[3], const float d[3], const float c[3], float R2, float q6[6], uint8_t *met) {
    float w[3];
    for (int i = 0; i < 3; i++) w[i] = o[i] - c[i];
    const float b = ((w[0] * d[0]) + (w[1] * d[1])) + (w[2] * d[2]);
    const float dd = ((d[0] * d[0]) + (d[1] * d[1])) + (d[2] * d[2]);
    const float ww = ((w[0] * w[0]) + (w[1] * w[1])) + (w[2] * w[2]);
    const float cx = fmaf(w[1], d[2], -(w[2] * d[1]));
    const float cy = fmaf(w[2], d[0], -(w[0] * d[2]));
    const float cz = fmaf(w[0], d[1], -(w[1] * d[0]));
    const float cr2 = ((cx * cx) + (cy * cy)) + (cz * cz);
    const float disc = (dd * R2) - cr2;
    for (int i = 0; i < 6; i++) q6[i] = 0.f;
    *met = (disc >= 0.f && dd > 0.f) ? 1 : 0;
    if (!*met) return;
    const float sq = sqrtf(disc);
    const float cc = ww - R2;
    float s = (-b > 0.f) ? cc / ((-b) + sq) : ((-b) - sq) / dd;
    s = fmaxf(s, 0.f);
    for (int i = 0; i < 3; i++) {
        q6[i] = w[i] + (s * d[i]);
        q6[3 + i] = d[i];
    }
}

int orc_canonical_ray(const float *rays, const float *centres, int64_t n, float R2, float *q6, uint8_t *met) {
    if (n < 0 || !(R2 >= 0.f)) return -1;
    for (int64_t i = 0; i < n; i++) canon_f32(rays + 6 * i, rays + 6 * i + 3, centres + 3 * i, R2, q6 + 6 * i, met + i);
    return 0;
}

/* the same entry point in FP64 (smaller root of |w + s d|^2 = R^2, clamped at s = 0) */
int orc_canonical_ray_f64(const float *rays, const float *centres, int64_t n, double R, double *p3, uint8_t *met) {
    if (n < 0 || !(R >= 0.0)) return -1;
    for (int64_t i = 0; i < n; i++) {
        double w[3], d[3], b = 0, dd = 0, ww = 0;
        for (int k = 0; k < 3; k++) {
            w[k] = (double)rays[6 * i + k] - (double)centres[3 * i + k];
            d[k] = (double)rays[6 * i + 3 + k];
            b += w[k] * d[k];
            dd += d[k] * d[k];
            ww += w[k] * w[k];
        }
        const double x0 = w[1] * d[2] - w[2] * d[1], x1 = w[2] * d[0] - w[0] * d[2], x2 = w[0] * d[1] - w[1] * d[0];
        const double disc = dd * R * R - (x0 * x0 + x1 * x1 + x2 * x2);
        met[i] = (disc >= 0.0 && dd > 0.0) ? 1 : 0;
        double s = 0.0;
        if (met[i]) {
            s = (-b - sqrt(disc)) / dd;
            if (s < 0.0) s = 0.0;
        }
        for (int k = 0; k < 3; k++) p3[3 * i + k] = met[i] ? w[k] + s * d[k] : 0.0;
    }
    return 0;
}
