// Internal definitions of the grouped (many-object) launches.
#pragma once

#include <vector>

#include "common.cuh"
#include "tc.cuh"

// One work item: rows [row0, row1) of the concatenated query array, all of object obj.
struct PlanItem {
    int obj;
    int pad;
    long long row0, row1;
};

// The contiguous range [k0, k1) of plan items a CTA of a grouped launch works through.
// A plan lists an object's items one after another, so a CTA meets each object in one run
// and loads that object's operands once per run (with CTAs striding over the items, nearly
// every item would belong to another object than the CTA's previous one).
__device__ __forceinline__ void item_range(int n_items, int &k0, int &k1) {
    k0 = (int)((long long)blockIdx.x * n_items / gridDim.x);
    k1 = (int)((long long)(blockIdx.x + 1) * n_items / gridDim.x);
}

struct nb_plan {
    int n_objects = 0;
    int n_items = 0;
    int chunk = 0;
    int64_t n_rows = 0;
    bool aligned = true;                 // every object's first row is a multiple of 32
    PlanItem *items = nullptr;           // device [n_items], object-major
    int *obj_items = nullptr;            // device [n_objects + 1]: items of object o
    long long *offsets = nullptr;        // device [n_objects + 1]
    std::vector<int64_t> h_offsets;
    std::vector<int> h_obj_items;
};

struct nb_group {
    int L = 0, n_objects = 0;
    int widths[NB_MAXL + 1] = {0};
    int off[NB_MAXL] = {0};
    int64_t P = 0;
    int64_t S = 0;                       // floats between two work items' gradient partials (P rounded up to 4)
    int infer_prec = NB_F32, train_prec = NB_F32;
    float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;  // [n_objects][P]
    float *paramsT = nullptr;            // [n_objects][P], weights transposed (re-check)
    std::vector<double> tau;
    TauF *d_tau = nullptr;               // device [n_objects]
    GammaTab gamma{};
    float lr = 1e-3f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    int64_t step = 0;
    // device-side schedule for graph-captured step loops
    float *sched_alpha = nullptr, *sched_c1 = nullptr, *sched_sqrt_c2 = nullptr;
    int sched_T = 0;
    int64_t sched_base = 0;
    int *d_step = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    TcModel tc{};                        // split-FP16 images of every object
};

MlpDesc nb_group_desc(const nb_group *g);

// split-FP16 grouped queries (tc_split.cu)
nb_status nb_tc_group_init(TcModel *tc, const MlpDesc &d, int n_objects);
nb_status nb_tc_group_refresh(TcModel *tc, const MlpDesc &d, int n_objects, cudaStream_t s);
nb_status nb_tc_group_query(TcModel *tc, const MlpDesc &d, int64_t P, const nb_plan *pl, const float *q,
                            const TauF *taus, float margin, uint32_t *bits, float *logits, nb_query_stats *st,
                            QueryWs ws, cudaStream_t s);

// BF16 tensor-core grouped training (train_bf16.cu)
nb_status nb_train_bf16_group_init(TcModel *tc, const MlpDesc &d, int n_objects);
nb_status nb_train_bf16_group_refresh(TcModel *tc, const MlpDesc &d, int n_objects, cudaStream_t s);
nb_status nb_launch_train_bf16_group(TcModel *tc, const MlpDesc &d, long long P, long long S, const nb_plan *pl,
                                     const float *q,
                                     const uint32_t *labels, float alpha, const float *sched_alpha, const int *d_step,
                                     int sched_T, float beta, const TauF *taus, float *partial, float *loss_partial,
                                     nb_step_stats *st, cudaStream_t s);
