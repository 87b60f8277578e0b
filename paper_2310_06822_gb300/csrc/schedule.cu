// Stepwise asymmetry schedule of the loss weights (Sec. 3.1 / 3.4, Eq. (loss); the
// supplement's "Weight schedule"): the weights change only at the end of a window of
// `period` training iterations, and only if that window's batches still had false
// negatives.  After k such adjustments the weight on the positives' term (the cost of a
// false negative) is 1 + fn_step k and the weight on the negatives' term (the cost of a
// false positive) is 1 / (dim_rate k) -- 1 and 1 before the first.  The supplement states
// the two series with the roles of the two weights exchanged relative to Eq. (loss) (its
// false-negative weight would decrease); the reading kept here is the one under which
// the false-negative cost grows without bound, as the main text requires.  Host logic
// only: the caller lets the training steps add their false-negative counts into one
// nb_step_stats for the window and reads it once per window.
#include "common.cuh"

extern "C" nb_status nb_stepwise_init(nb_stepwise *s, int32_t period, int32_t dim_rate, float fn_step,
                                      int32_t stop_windows) {
    if (!s) return nb_fail(NB_EINVAL, "nb_stepwise_init: null schedule");
    if (period < 1 || dim_rate < 1 || !(fn_step >= 0.f) || !(fn_step < 1e6f) || stop_windows < 0)
        return nb_fail(NB_EINVAL, "nb_stepwise_init: period and dim_rate >= 1, fn_step >= 0, stop_windows >= 0");
    s->period = period;
    s->dim_rate = dim_rate;
    s->fn_step = fn_step;
    s->stop_windows = stop_windows;
    s->adjustments = 0;
    s->clean_windows = 0;
    s->alpha = 1.f;
    s->beta = 1.f;
    return NB_OK;
}

extern "C" int32_t nb_stepwise_window(nb_stepwise *s, uint64_t fn) {
    if (!s || s->period < 1 || s->dim_rate < 1) return -1;
    if (fn > 0) {
        s->adjustments++;
        s->clean_windows = 0;
        const double k = (double)s->adjustments;
        s->alpha = (float)(1.0 + (double)s->fn_step * k);
        s->beta = (float)(1.0 / ((double)s->dim_rate * k));
        return 0;
    }
    s->clean_windows++;
    return (s->stop_windows > 0 && s->clean_windows >= s->stop_windows) ? 1 : 0;
}
