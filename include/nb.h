/*
 * nb.h -- C ABI of libnb, the GB300 (sm_103a) library for the data-parallel hot
 * path of Neural Bounding (Liu, Fischer, Yoo, Ritschel; SIGGRAPH 2024).
 *
 * The paper learns a function h(r) (Sec. 3.1) that is 1 wherever the query
 * function g(r) is 1 -- g(r) being 1 iff the region r (a point, space-time
 * point, ray, plane or box) touches a point where the indicator f is 1 -- and
 * may also be 1 elsewhere (false positives).  h is an MLP whose sigmoid output
 * is rounded to {0,1} (Sec. 3.4 "Architecture"), trained with the dynamically
 * weighted asymmetric binary cross-entropy of Eq. (loss) and Adam (Sec. 3.4
 * "Training"), with an output epsilon added for numerics (Suppl. "Numerics").
 *
 * Conventions shared by every entry point:
 *   - Pointers named q, out_bits, label_bits, opt_logits and every *_stats
 *     argument are DEVICE pointers owned by the caller; the library never frees
 *     them.  Host pointers are named host_*.
 *   - stream is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Calls enqueue work on it and return without synchronising,
 *     except where a call is documented as synchronous.
 *   - Queries are FP32, row-major, one encoding per row (widths: point2 2,
 *     point3 3, point4t 4 = (x,y,z,t), ray3 6 = (origin, direction),
 *     plane3 4 = (normal, offset) for {x : n.x = offset}, box3 6 =
 *     (centre, half-extents)).
 *   - Bit arrays hold query i in bit (i % 32) of word i / 32; the caller
 *     provides ceil(n / 32) words.  Bits past n in the last word are written 0.
 *   - Every call returns an nb_status.  Argument errors are detected on the
 *     host before anything is enqueued and leave outputs untouched; the message
 *     is available from nb_last_error() (thread-local).  Errors of earlier
 *     asynchronous work surface as NB_ECUDA on a later call.  No call traps,
 *     asserts or aborts on the device.
 */
#ifndef NB_H
#define NB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NB_OK = 0,
    NB_EINVAL = 1,       /* bad argument (null pointer, size, kind, width) */
    NB_ENOMEM = 2,       /* device or host allocation failed */
    NB_ECUDA = 3,        /* a CUDA runtime call failed */
    NB_ETIMEOUT = 4,     /* a bounded device wait gave up */
    NB_ENUMERIC = 5,     /* reserved: no call returns it (a training sample with a non-finite
                            logit is left out of the loss and gradient and counted instead) */
    NB_EUNSUPPORTED = 6  /* configuration not supported by this build or device */
} nb_status;

typedef enum { NB_POINT2 = 0, NB_POINT3 = 1, NB_POINT4T = 2, NB_RAY3 = 3, NB_PLANE3 = 4, NB_BOX3 = 5 } nb_kind;

/* Arithmetic of the fast forward path:
 *   NB_F32    FP32 FMA (CUDA cores), the plain single-object form (networks with input
 *             width <= 8 and every hidden layer but the last <= 128 wide run a query per
 *             thread with the weights in shared memory, others in tiles of queries);
 *   NB_BF16   tcgen05 tensor cores, BF16 operands, FP32 accumulation (one product);
 *   NB_FP8    tcgen05 tensor cores, E4M3 operands for the hidden-to-hidden layers with
 *             power-of-two scales per weight row and per query row (exact to apply),
 *             the first layer in split FP16, FP32 accumulation; hidden widths 128 or
 *             256 and at least two hidden layers;
 *   NB_F16X3  tcgen05 tensor cores, weights and activations split into FP16 hi + lo
 *             pairs and three products per layer (hi.hi + hi.lo + lo.hi), FP32
 *             accumulation: logits within a few FP32 roundings of the FP32 network. */
typedef enum { NB_F32 = 0, NB_BF16 = 1, NB_FP8 = 2, NB_F16X3 = 3 } nb_prec;

/* Indicator f of Sec. 3.1: a union of closed balls (disks when dim = 2).
 * All values must be integer multiples of 2^-qexp with magnitude below 2^(31-qexp)
 * (exact in FP32 and as 32-bit integers).  For NB_POINT4T the ball centre moves as
 * c + v t, so vel must be given.  All pointers are device pointers. */
typedef struct {
    int32_t dim;          /* 2 or 3 */
    int32_t n_spheres;    /* 1 .. 4096 */
    int32_t qexp;         /* grid quantum 2^-qexp, 8 .. 24 */
    int32_t reserved;     /* must be 0 */
    const float *centres; /* [n_spheres][dim] */
    const float *radii;   /* [n_spheres], >= 0 */
    const float *vel;     /* [n_spheres][3] or NULL */
} nb_shape;

/* Device-side counters, zeroed by the call that fills them. */
typedef struct {
    unsigned long long n_positive; /* queries labelled 1 */
    unsigned long long n_invalid;  /* off-grid / non-finite / out-of-range queries (labelled 1) */
} nb_label_stats;

typedef struct {
    unsigned long long n_inside;      /* decisions "maybe inside" (bit = 1) */
    unsigned long long n_flagged;     /* fast logit within the margin of tau: re-checked */
    unsigned long long n_resolved_f32;/* settled by the FP32 forward with its error bound */
    unsigned long long n_resolved_ff; /* settled by the float-float forward with its error bound */
    unsigned long long n_unresolved;  /* still ambiguous: decided inside (conservative) */
    unsigned long long n_nonfinite;   /* non-finite logit: decided inside and counted */
} nb_query_stats;

typedef struct {
    float loss;                    /* mean asymmetric BCE of the batch, Eq. (loss) */
    float reserved;
    unsigned long long fn;         /* batch false negatives at logit >= tau (added to) */
    unsigned long long fp;         /* batch false positives at logit >= tau (added to) */
    unsigned long long n_nonfinite;/* samples with a non-finite logit (added to) */
} nb_step_stats;  /* loss is written by each step; the counts accumulate until the caller zeroes them */

typedef struct nb_model nb_model;

/* ------------------------------------------------------------------ models */

/* Create a bounding network h (Sec. 3.4 "Architecture"): widths[0] is the query
 * encoding width, widths[1..n_layers-1] the hidden widths (ReLU), widths[n_layers]
 * must be 1 (the logit).  Hidden widths 1..256.  infer_prec selects the nb_query
 * fast path (see nb_prec; the tensor-core paths need equal hidden widths (at most 128
 * for NB_BF16 and NB_F16X3, which run widths other than 64 and 128 -- such as the
 * paper's 25-, 50- and 75-wide networks -- on a copy of the parameters zero-padded to
 * 64 or 128, computing the same logits; 128 or 256 for NB_FP8), an input width <= 16 and
 * weights that fit in shared memory, else NB_EUNSUPPORTED).  train_prec selects the training
 * step: NB_F32, or NB_BF16 (tensor cores; equal hidden widths of 64, 128 or 256, the
 * last with its weights streamed through shared memory).
 * Parameters start at zero; load them with nb_model_set_params.  Adam uses lr 1e-3,
 * betas (0.9, 0.999), eps 1e-8 (Sec. 3.4 "Training"); tau starts at 0, i.e. the
 * sigmoid rounded at 1/2 (Sec. 3.4).  The device is the current CUDA device. */
nb_status nb_model_create(const int32_t *widths, int32_t n_layers, int32_t infer_prec,
                          int32_t train_prec, nb_model **out);

/* Hidden activations: NB_ACT_RELU (the configurations') or NB_ACT_SINE, sin(z), the
 * sinusoidal activation of Sec. 3.4 "Architecture" (no frequency factor: sin of the
 * pre-activation itself).  nb_model_create_act is nb_model_create with the activation
 * chosen; nb_model_create makes ReLU networks.  Sine networks run the FP32 forward
 * (infer NB_F32) or the split-FP16 tensor-core forward (NB_F16X3, widths as there; padded
 * neurons stay 0 since sin 0 = 0), train in FP32 (train NB_F32), and are re-checked and
 * calibrated like ReLU networks, the rounding bounds adding the documented error of CUDA's
 * sinf (2 ulp) and sin (2 ulp) at each activation (sin is 1-Lipschitz).  Other precisions
 * return NB_EUNSUPPORTED; an unknown activation NB_EINVAL.  Checkpoints do not record the
 * activation: restore a state into a model of the same activation. */
#define NB_ACT_RELU 0
#define NB_ACT_SINE 1
nb_status nb_model_create_act(const int32_t *widths, int32_t n_layers, int32_t infer_prec, int32_t train_prec,
                              int32_t activation, nb_model **out);
nb_status nb_model_destroy(nb_model *m);
int64_t nb_model_param_count(const nb_model *m);

/* Flat FP32 parameters: for each layer l, W_l (widths[l+1] x widths[l], row-major)
 * then b_l.  set_params also resets Adam's moments and step counter and refreshes
 * the low-precision copies.  Both are synchronous. */
nb_status nb_model_set_params(nb_model *m, const float *host_params, int64_t n_params);
nb_status nb_model_get_params(const nb_model *m, float *host_params, int64_t n_params);
/* Gradient of the last nb_train_step (before the Adam update); synchronous. */
nb_status nb_model_get_grad(const nb_model *m, float *host_grad, int64_t n_params);

nb_status nb_model_set_tau(nb_model *m, double tau);
nb_status nb_model_get_tau(const nb_model *m, double *tau);
nb_status nb_model_set_adam(nb_model *m, float lr, float beta1, float beta2, float eps);

/* Checkpoint: parameters, Adam moments, step counter, tau.  Synchronous.
 * nb_model_state_size gives the byte count for host_buf. */
nb_status nb_model_state_size(const nb_model *m, size_t *bytes);
nb_status nb_model_get_state(const nb_model *m, void *host_buf, size_t bytes);
nb_status nb_model_set_state(nb_model *m, const void *host_buf, size_t bytes);

/* ------------------------------------------------------------- hot path */

/* Exact labels y_i = g(q_i) (Sec. 3.1; Alg. 1's Any(f(SampleRegion(r))) evaluated
 * analytically instead of by sampling).  Inclusive of the surface.  Each query is
 * tested against every ball in exact integer arithmetic on the 2^-qexp grid.
 * A query that is non-finite, off the grid or out of range is labelled 1
 * (conservative) and counted in n_invalid.  dev_stats may be NULL. */
nb_status nb_label(const nb_shape *shape, int32_t kind, const float *q, int64_t n, uint32_t *out_bits,
                   nb_label_stats *dev_stats, void *stream);

/* Query sampling: Alg. 1 draws a fresh batch r ~ Uniform at every training
 * iteration.  Writes queries first .. first+n-1 of the stream (seed, kind) as float
 * rows q[n][enc width] (2, 3, 4, 6, 4, 6 floats), every value on the 2^-qexp grid,
 * 8 <= qexp <= 20: points U[-1,1)^d; 4D points (x, t) with t U[0,1); rays with origin
 * on the radius-2 sphere and direction uniform on S^2; planes with normal uniform on
 * S^2 and offset U[-1,1); boxes with centre U[-1,1)^3 and half-extents log-uniform
 * in [0.01, 0.5].  Query i is a function of (seed, kind, i) alone: it reads the
 * counter-based generator Philox4x64-10 (Salmon et al., SC 2011) at counters
 * (i, j, p, 0) under key (seed, kind), and every transform is integer or correctly
 * rounded, so any split of a stream into calls gives the same bits.  q is a device
 * buffer owned by the caller (4-byte aligned).  Asynchronous on stream; EINVAL for an
 * unknown kind, qexp outside [8, 20], a negative range or a null q with n > 0. */
nb_status nb_sample(int32_t kind, int32_t qexp, uint64_t seed, int64_t first, int64_t n, float *q, void *stream);

/* The paper's query parameterisation (Suppl. "Parameterization") from the library's
 * encodings, for networks trained on the paper's inputs: rays (start, direction) and
 * points unchanged; boxes (centre c, half-extents e) -> corners (c - e, c + e), exact on
 * the grid; planes (normal n, offset of n . x = off) -> (p0, n) with p0 = off n / |n|^2,
 * the plane's point nearest the origin, in correctly rounded FP32 steps.  out holds n rows
 * of 2, 3, 4, 6, 6, 6 floats (point2, point3, point4t, ray3, plane3, box3); labels are
 * still computed on the library's encoding.  Device buffers, asynchronous on stream;
 * EINVAL for an unknown kind, n < 0 or null pointers with n > 0. */
nb_status nb_encode_paper(int32_t kind, const float *q, int64_t n, float *out, void *stream);

/* One training iteration of Sec. 3.4 on a batch of n queries with labels y:
 * forward, mean asymmetric BCE of Eq. (loss) with weights alpha (on y log yhat) and
 * beta (on (1-y) log(1-yhat)), backward, deterministic gradient reduction and one
 * Adam step on the FP32 master weights; the low-precision copies are refreshed.
 * A sample whose logit is not finite -- a non-finite input coordinate counts as such --
 * adds nothing to the loss or the gradient (the mean still divides by n) and is counted in
 * dev_stats->n_nonfinite.
 * dev_stats may be NULL.  n >= 1. */
nb_status nb_train_step(nb_model *m, const float *q, const uint32_t *label_bits, int64_t n, float alpha,
                        float beta, nb_step_stats *dev_stats, void *stream);

/* Decisions h(q_i) = [z_i >= tau] (sigmoid rounding of Sec. 3.4 shifted by the
 * calibrated threshold).  The fast path evaluates z in the model's infer precision;
 * every query whose fast logit lies within `margin` of tau is re-evaluated on the
 * FP32 master weights with a rigorous error bound, then in float-float if needed,
 * so decisions equal those of the exact real-valued network whenever the fast
 * logit's error is below margin.  opt_logits (may be NULL) receives the fast
 * logits.  dev_stats may be NULL.  Uses a library-owned workspace that grows on
 * demand (a growth synchronises the device). */
nb_status nb_query(nb_model *m, const float *q, int64_t n, float margin, uint32_t *out_bits, float *opt_logits,
                   nb_query_stats *dev_stats, void *stream);

/* Device status of a model's asynchronous work: synchronises `stream`, then returns
 * NB_ECUDA for a pending CUDA error and NB_ETIMEOUT if one of the model's tensor-core
 * kernels gave up a bounded wait since the last check (their waits on mbarriers poll a
 * bounded number of times; on expiry the kernel drains its copies and products, frees
 * tensor memory, returns and records the timeout, leaving the context usable).  The
 * record is cleared.  nb_query_host and nb_query_early_out check by themselves. */
nb_status nb_model_check(nb_model *m, void *stream);

/* Diagnostic of that mechanism without a fault: one thread waits, with the forward
 * kernels' bounded wait, on an mbarrier no one arrives at, gives up after `polls` polls
 * (1 .. 2^20) and returns.  Returns NB_ETIMEOUT (the expected outcome) once the stream has
 * drained; any other status is a failure of the mechanism. */
nb_status nb_selftest_bounded_wait(int32_t polls, void *stream);

/* nb_query for queries in host memory: host_q [n][enc width] and host_bits
 * ((n + 31) / 32 words) are host buffers; pinned (page-locked) ones let the copies overlap
 * the forward.  With chunk_rows 0, host_q pinned and a coherent host link (NVLink-C2C,
 * reported as native host atomics), the forward and the re-check read the rows in place
 * from host memory; the bits are decided into a library-owned device buffer and copied
 * back.  The caller must not write host_q during the call.  Otherwise (or with
 * chunk_rows > 0) the queries are streamed in chunks of chunk_rows (0: 2^22; rounded up to
 * a multiple of 32; the first chunk a quarter of that, so the forward starts early)
 * through two library-owned device staging buffers: while one chunk is
 * decided on `stream`, the next is copied in on a library-owned copy stream, and each
 * chunk's bits are copied back as soon as its decisions are final.  Decisions, margin
 * and re-check as nb_query.  host_stats (host memory, may be NULL) receives the sums over
 * all chunks.  Synchronous: returns when every bit is in host_bits.  The staging buffers
 * grow on demand (a growth synchronises the device). */
nb_status nb_query_host(nb_model *m, const float *host_q, int64_t n, float margin, uint32_t *host_bits,
                        nb_query_stats *host_stats, int64_t chunk_rows, void *stream);

/* Neural early-out (Sec. 3.3): `early` is a (small) network trained and calibrated as a
 * conservative bound of the complement 1 - g (labels inverted, e.g. by nb_bits_not), so
 * that where it decides 0 the query is certainly inside (g = 1); `late` is the bounding
 * network of g.  Every row is first decided by `early` (nb_query with margin_early); rows
 * it decides 0 get bit 1 without evaluating `late`; the other rows are compacted, gathered
 * into a library-owned buffer and decided by `late` (nb_query with margin_late), and
 * their bits scattered back.  When `early` has the paper's early-exit shape (one hidden
 * ReLU layer, input width 2, 3, 4, 6 or 8, NB_F32 inference), one pass settles and
 * gathers instead: a row is settled when its FP32 early logit plus a rigorous bound of
 * that logit's rounding error plus margin_early is below the early threshold; every
 * other row (non-finite ones included) goes to `late`.  Both networks take the same input
 * width.  host_stats (may
 * be NULL) receives how many rows each network decided.  Synchronous on stream (the
 * number of rows left for `late` is read back); the workspace, owned by `late`, grows on
 * demand (a growth synchronises the device). */
typedef struct {
    uint64_t n_early_inside;  /* rows settled by the early network (bit 1) */
    uint64_t n_late;          /* rows decided by the late network */
} nb_early_stats;
nb_status nb_query_early_out(nb_model *early, nb_model *late, const float *q, int64_t n, float margin_early,
                             float margin_late, uint32_t *out_bits, nb_early_stats *host_stats, void *stream);

/* Inverted bounds and the broad-phase three-way test (Sec. 4.4): swapping the asymmetry
 * weights gives a network that conservatively bounds where the object is certainly hit;
 * that network with its logit negated is a bound of the complement 1 - g, trained with the
 * usual weights on inverted labels (nb_bits_not) and calibrated on them.  `outer` is the
 * bounding network of g (decision 0: certainly outside), `inner` the bound of 1 - g
 * (decision 0: certainly inside).  codes[i] (one byte per query, caller-owned device
 * buffer of n bytes) is 0 certainly outside, 1 certainly inside, 2 neither: the queries a
 * collision test must still test exactly.  A query that both networks call certain, which
 * no query of either calibration set can be, gets 2 and is counted as a conflict.  Both
 * networks take the same input width; each is decided with its own margin and certified
 * re-check as in nb_query.  dev_stats (device memory, may be NULL) is added to.
 * Asynchronous on stream (no host synchronisation; capturable in a CUDA graph once the
 * workspace, owned by `outer`, has grown to n queries: a growth synchronises the device).
 * EINVAL for null models or pointers with n > 0, differing input widths, n outside
 * [0, 2^32). */
typedef struct {
    uint64_t n_out;       /* code 0 */
    uint64_t n_in;        /* code 1 */
    uint64_t n_neither;   /* code 2, conflicts included */
    uint64_t n_conflict;  /* both networks certain, contradicting each other */
} nb_three_way_stats;
nb_status nb_query_three_way(nb_model *outer, nb_model *inner, const float *q, int64_t n, float margin_outer,
                             float margin_inner, uint8_t *codes, nb_three_way_stats *dev_stats, void *stream);

/* out[i] = 1 - in[i] for the n bits of a label or decision array (bits past n cleared);
 * in and out may be the same buffer.  Asynchronous on stream. */
nb_status nb_bits_not(const uint32_t *in, int64_t n, uint32_t *out, void *stream);

/* Stepwise asymmetry schedule (Sec. 3.4; Suppl. "Weight schedule"), host logic.  The
 * loss weights change only at the end of a window of `period` iterations (10,000 in the
 * paper), and only if that window's training batches had false negatives (the fn count
 * the training steps add into one nb_step_stats, read once per window).  After k such
 * adjustments alpha (the false-negative weight of Eq. (loss)) is 1 + fn_step * k and beta
 * (the false-positive weight) is 1 / (dim_rate * k); both are 1 before the first.  The
 * paper's rates: dim_rate 20 (2D), 100 (3D), 200 (4D); fn_step 0.2.  The supplement
 * states the two series with the weights' roles exchanged; this reading makes the
 * false-negative cost grow without bound, as Sec. 3.1 requires.
 * nb_stepwise_window returns 1 when stop_windows (> 0) consecutive windows have had no
 * false negative (training may stop; Sec. 3.4 stops after six), 0 otherwise, -1 for an
 * uninitialised schedule. */
typedef struct {
    int32_t period;        /* iterations per window */
    int32_t dim_rate;      /* c in beta = 1 / (c k) */
    float fn_step;         /* growth of alpha per adjustment */
    int32_t stop_windows;  /* consecutive windows without a false negative that end training; 0: never */
    int32_t adjustments;   /* k */
    int32_t clean_windows; /* consecutive windows without a false negative so far */
    float alpha;           /* current false-negative weight */
    float beta;            /* current false-positive weight */
} nb_stepwise;
nb_status nb_stepwise_init(nb_stepwise *s, int32_t period, int32_t dim_rate, float fn_step, int32_t stop_windows);
int32_t nb_stepwise_window(nb_stepwise *s, uint64_t fn);

/* Threshold calibration (Suppl. "Numerics", output epsilon): tau = (minimum over
 * the queries labelled 1 of the network logit) - eps, rounded toward -infinity,
 * so the calibration set has no false negative.  The minimum is located with FP32
 * logits and rigorous bounds, and the candidates are re-evaluated in FP64.  With no
 * positive query, tau = +infinity.  Stores tau in the model and in *host_tau.
 * Synchronous on stream. */
nb_status nb_calibrate(nb_model *m, const float *q, const uint32_t *label_bits, int64_t n, double eps,
                       double *host_tau, void *stream);

/* ------------------------------------------------------- grouped launches
 * Many objects, one bounding network each (the paper trains one network per object and
 * rearranges objects without retraining, Sec. 2), all of one architecture, trained and
 * queried in one persistent launch per call.  The queries of all objects are concatenated
 * into one array: object o owns rows [offsets[o], offsets[o+1]).  A plan splits every
 * object's rows into work items of at most chunk_rows rows; grouped calls walk the items.
 * Per-object counts may be uneven.  Gradients are reduced per object in item order, so a
 * step does not depend on scheduling. */
typedef struct nb_plan nb_plan;
typedef struct nb_group nb_group;

/* host_offsets[0..n_objects], non-decreasing, total rows < 2^32.  chunk_rows: multiple of
 * 64, 0 = 4096.  Grouped queries additionally need every offsets[o] to be a multiple of 32
 * (each object's decision bits then start at a word).  Synchronous. */
nb_status nb_plan_create(const int64_t *host_offsets, int32_t n_objects, int32_t chunk_rows, nb_plan **out);
nb_status nb_plan_destroy(nb_plan *p);

/* widths as for nb_model_create; infer_prec NB_F32 (any widths) or NB_F16X3 (equal
 * hidden widths of exactly 64 or 128: the grouped forward has no padded form); train_prec
 * NB_F32 or NB_BF16 (equal hidden widths of 64 or 128).  EUNSUPPORTED otherwise. */
nb_status nb_group_create(const int32_t *widths, int32_t n_layers, int32_t n_objects, int32_t infer_prec,
                          int32_t train_prec, nb_group **out);
nb_status nb_group_destroy(nb_group *g);
int64_t nb_group_param_count(const nb_group *g); /* P of one object */
/* n_objects * P FP32 values, object-major; set resets Adam.  Synchronous. */
nb_status nb_group_set_params(nb_group *g, const float *host_params, int64_t n);
nb_status nb_group_get_params(const nb_group *g, float *host_params, int64_t n);
nb_status nb_group_get_grad(const nb_group *g, float *host_grad, int64_t n);
nb_status nb_group_set_tau(nb_group *g, const double *host_tau, int32_t n_objects);
nb_status nb_group_get_tau(const nb_group *g, double *host_tau, int32_t n_objects);
/* Device-side schedule for training loops captured in a CUDA graph: alpha[t] for the
 * next T steps (and the matching Adam bias corrections) live on the device and a device
 * step counter advances every step, so nb_train_step_grouped(..., alpha = -1, ...) needs
 * no host argument that changes between steps.  nb_group_sync_schedule copies the device
 * counter back to the host's step count (synchronous). */
nb_status nb_group_set_schedule(nb_group *g, const float *host_alpha, int32_t T);
nb_status nb_group_sync_schedule(nb_group *g);
/* Grows the group's workspace for the plan now (synchronous), so that later grouped calls
 * with this plan allocate nothing and can be captured in a CUDA graph. */
nb_status nb_group_reserve(nb_group *g, const nb_plan *plan);
/* One training step of every object on its rows (nb_train_step per object, in one
 * launch).  alpha < 0 takes alpha and the bias corrections from the device schedule.
 * dev_stats: loss = mean over objects of each object's mean loss; counts summed. */
nb_status nb_train_step_grouped(nb_group *g, const nb_plan *plan, const float *q, const uint32_t *label_bits,
                                float alpha, float beta, nb_step_stats *dev_stats, void *stream);
/* Decisions of every object's network on its rows against its threshold, with the margin
 * band re-checked in extended precision (as nb_query).  out_bits covers all rows. */
nb_status nb_query_grouped(nb_group *g, const nb_plan *plan, const float *q, float margin, uint32_t *out_bits,
                           float *opt_logits, nb_query_stats *dev_stats, void *stream);
/* nb_calibrate per object on its rows; host_tau[n_objects] receives the thresholds. */
nb_status nb_calibrate_grouped(nb_group *g, const nb_plan *plan, const float *q, const uint32_t *label_bits,
                               double eps, double *host_tau, void *stream);

/* Autotuner of the grouped launches' work split (the paper has no counterpart: its
 * networks are trained one at a time).  For each candidate chunk_rows (multiples of
 * 64) it builds the plan of host_offsets[n_objects + 1], runs op (NB_TUNE_QUERY: the
 * grouped query at margin 0 into a scratch bit buffer; NB_TUNE_TRAIN: grouped training
 * steps with alpha = beta = 1 on label_bits) once untimed and `reps` times timed with
 * CUDA events on stream, and returns the fastest candidate in *best_chunk_rows and,
 * when host_ms is not NULL, the mean milliseconds of every candidate in host_ms[].
 * Training trials run on a snapshot: parameters, Adam moments, gradient and step
 * counters are restored before returning, also on error.  Synchronous; allocates
 * a scratch buffer and the trial plans (not capturable in a CUDA graph). */
#define NB_TUNE_QUERY 0
#define NB_TUNE_TRAIN 1
nb_status nb_group_autotune(nb_group *g, const int64_t *host_offsets, int32_t n_objects, int32_t op, const float *q,
                            const uint32_t *label_bits, const int32_t *candidates, int32_t n_candidates, int32_t reps,
                            int32_t *best_chunk_rows, float *host_ms, void *stream);

/* ------------------------------------------------------- learned-culler cascade
 * Many objects in one scene, each a union of spheres with its own trained bounding
 * network, and rays asking "which rays hit any object".  Following the paper's premise
 * of a cheap conservative test in front of an expensive exact one (Sec. 1, Eq. (Benefit)),
 * the cascade is: axis-aligned box of the object -> the object's neural bound -> exact
 * sphere test; the plain path (box -> exact) is the reference: both must give the same hits.
 * All pointers are device pointers. */
typedef struct {
    int32_t n_objects;            /* K, 1 .. 4096 */
    int32_t qexp;                 /* world grid 2^-qexp of rays and spheres, 8 .. 24 */
    float ball_radius;            /* every sphere of object k lies inside this ball around obj_centre[k] */
    int32_t reserved;             /* 0 */
    const int64_t *sphere_offsets;/* [K+1]: spheres of object k are [sphere_offsets[k], sphere_offsets[k+1]) */
    const float *centres;         /* [S][3] world sphere centres */
    const float *radii;           /* [S] */
    const float *obj_centre;      /* [K][3] world centre of each object's frame (on the grid) */
    const float *aabb;            /* [K][6] min xyz, max xyz, containing every sphere of the object */
} nb_scene;

typedef struct {
    unsigned long long aabb_pairs;   /* (ray, object) pairs passing the box */
    unsigned long long ball_pairs;   /* ... and entering the object's ball (canonical binning) */
    unsigned long long exact_pairs;  /* pairs given to the exact test */
    unsigned long long sphere_tests; /* sphere predicates evaluated by the exact test */
    unsigned long long hit_pairs;    /* pairs whose exact test hit */
} nb_cascade_stats;

/* Stage 1 for n rays ([n][6], origin and direction on the grid) against every object.
 * Counting call (offsets == NULL): counts[k] = number of rays of object k passing the
 * box (and, if canonical, entering the ball); dev_stats (zeroed) gets the pair totals.
 * Scatter call (offsets = device [K+1], offsets[k+1] - offsets[k] >= counts[k]): object
 * k's rays go to rows offsets[k] .. of pair_ray (the ray index) and, if canonical, of
 * pair_q ([rows][6], the ray in the object's frame with its origin moved to where it
 * enters the ball -- the network's input); the caller pre-fills pair_ray with 0xffffffff
 * so padding rows are recognised.  counts is rewritten with the same counts. */
nb_status nb_cascade_bin(const nb_scene *scene, const float *rays, int64_t n, int32_t canonical,
                         unsigned long long *counts, const int64_t *offsets, uint32_t *pair_ray, float *pair_q,
                         nb_cascade_stats *dev_stats, void *stream);
/* Spatial index over the scene's objects for stage 1.  Sec. 3.2 stacks bounds into
 * hierarchies the way bounding boxes form a BVH; the tree here follows the linear builder
 * of the paper's BVH baseline (Sec. 4.1): objects in Morton order of their box centres
 * (10 bits per axis over the bounding box of the centres, ties by object index), split at
 * the median of that order, two median levels per node so that every node has up to four
 * children, and every node holds its children's boxes (exact unions of the object boxes
 * below them).  The floating-point slab test of stage 1 is monotone under box inclusion
 * (a ray that passes a box passes every box containing it), so the indexed stage 1 finds
 * exactly the pairs of nb_cascade_bin while testing only the boxes along the way.
 * nb_cascade_index_create copies scene->aabb to the host, builds there and uploads the
 * tree: synchronous.  EINVAL for a bad scene, ENOMEM, ECUDA. */
typedef struct nb_cascade_index nb_cascade_index;
nb_status nb_cascade_index_create(const nb_scene *scene, nb_cascade_index **out);
nb_status nb_cascade_index_destroy(nb_cascade_index *index);
/* Stage 1 through the index: arguments, results, padding rule and statistics as
 * nb_cascade_bin (the same pairs and counts; the rows of one object may come in another
 * order, as they may between two calls of nb_cascade_bin).  EINVAL if the index was
 * built for another object count. */
nb_status nb_cascade_bin_indexed(const nb_cascade_index *index, const nb_scene *scene, const float *rays, int64_t n,
                                 int32_t canonical, unsigned long long *counts, const int64_t *offsets,
                                 uint32_t *pair_ray, float *pair_q, nb_cascade_stats *dev_stats, void *stream);
/* The index's tree, built on the host from host boxes (no device involved), as
 * nb_cascade_index_create builds it.  nodes[0] is the root; a child slot c of a node holds
 * a box (lo[axis][c], hi[axis][c]) and child[c] >= 0 (a node index), -1 - k (object k)
 * or NB_BVH_EMPTY (unused slot, box zero).  nodes must hold
 * nb_cascade_index_max_nodes(n_objects) entries; *n_nodes receives the count used and
 * *depth the number of node levels.  EINVAL for n_objects outside 1 .. 4096 or null
 * pointers. */
#define NB_BVH_EMPTY (-2147483647 - 1)
typedef struct {
    float lo[3][4];
    float hi[3][4];
    int32_t child[4];
} nb_bvh4_node;
int32_t nb_cascade_index_max_nodes(int32_t n_objects);
nb_status nb_cascade_index_build_host(const float *aabb, int32_t n_objects, nb_bvh4_node *nodes, int32_t *n_nodes,
                                      int32_t *depth);
/* Stage 3: rows [0, rows) with pair_ray != 0xffffffff and (pass_bits == NULL or its bit
 * set) are tested exactly against their object's spheres (integer arithmetic on the
 * grid); a hit ORs the ray's bit into ray_hits and the row's bit into pair_hits (either
 * may be NULL, not both; the caller zeroes them).  pair_hits are the exact labels of the
 * pairs, e.g. for calibrating the objects' thresholds on the deployment distribution. */
nb_status nb_cascade_exact(const nb_scene *scene, const float *rays, const uint32_t *pair_ray,
                           const int64_t *offsets, int64_t rows, const uint32_t *pass_bits, uint32_t *ray_hits,
                           uint32_t *pair_hits, nb_cascade_stats *dev_stats, void *stream);

/* Training step that allocates nothing.  The paper has no counterpart; this is a
 * deployment variant of nb_train_step for callers that cannot call cudaMalloc:
 * hosts whose device memory is entirely reserved up front by another allocator
 * (a framework's caching allocator, a fixed arena), and real-time training loops
 * in which the implicit device-wide synchronisation of a cudaMalloc / cudaFree
 * would stall work on other streams.  nb_train_step grows a model-owned workspace
 * on demand; this variant instead keeps the per-CTA gradient partials in one
 * static device array of NB_NOALLOC_SCRATCH_FLOATS floats (8 MiB) that every GPU
 * loading libnb holds until the process exits.
 *   - Computes exactly what nb_train_step computes (FP32 training precision only;
 *     other precisions return NB_EUNSUPPORTED); the number of CTAs is capped to
 *     what the array holds, which can change the summation order of the gradient
 *     reduction, so results agree with nb_train_step within rounding.
 *   - Networks with more than NB_NOALLOC_SCRATCH_FLOATS - 1 parameters are
 *     rejected with NB_EINVAL.
 *   - The first call on a device looks up the array's device address for the
 *     current device (cudaGetSymbolAddress) and keeps it for the life of the
 *     process; make that first call before any stream capture.  The kept address
 *     belongs to the device's context at that time: after the application resets
 *     the device (cudaDeviceReset) it is stale, so do not call this entry point
 *     on that device again in the same process.
 *   - All calls share the one array (it keeps the last call's contents; the call
 *     clears what must start at zero), so calls whose work overlaps on the GPU --
 *     on different streams or different threads -- race and must be serialised
 *     by the caller.
 * Arguments, results and errors are those of nb_train_step. */
#define NB_NOALLOC_SCRATCH_FLOATS (2u << 20)
nb_status nb_train_step_noalloc(nb_model *m, const float *q, const uint32_t *label_bits, int64_t n, float alpha,
                                float beta, nb_step_stats *dev_stats, void *stream);

/* Thread-local message of the last failing call of this thread ("" if none). */
const char *nb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NB_H */
