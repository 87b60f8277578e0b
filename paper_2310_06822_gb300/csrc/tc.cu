// Tensor-core paths (placeholder until the tcgen05 kernels land).
#include "tc.cuh"

nb_status nb_tc_init(TcModel *tc, const MlpDesc &d, int infer_prec, int train_prec) {
    (void)tc; (void)d; (void)infer_prec; (void)train_prec;
    return nb_fail(NB_EUNSUPPORTED, "tensor-core precisions are not built yet");
}
void nb_tc_free(TcModel *tc) { (void)tc; }
nb_status nb_tc_refresh(TcModel *tc, const MlpDesc &d, cudaStream_t s) {
    (void)tc; (void)d; (void)s;
    return nb_fail(NB_EUNSUPPORTED, "tensor-core precisions are not built yet");
}
nb_status nb_tc_query(TcModel *, const MlpDesc &, const float *, int64_t, TauF, float, uint32_t *, float *,
                      nb_query_stats *, QueryWs, cudaStream_t) {
    return nb_fail(NB_EUNSUPPORTED, "tensor-core precisions are not built yet");
}
nb_status nb_tc_train_step(TcModel *, const MlpDesc &, const float *, const uint32_t *, int64_t, float, float, TauF,
                           float *, float *, float *, float *, float, float, float, float, float, float,
                           nb_step_stats *, cudaStream_t) {
    return nb_fail(NB_EUNSUPPORTED, "tensor-core precisions are not built yet");
}
