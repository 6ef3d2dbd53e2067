// train.cu -- Algorithm 1 TRAIN step (forward and backward of one iteration).
#include "ht_internal.cuh"

extern "C" {

ht_status ht_train_create(ht_policy *p, const ht_train_desc *d, ht_train **out)
{
    (void)p;
    (void)d;
    if (out) *out = nullptr;
    ht_set_error("training step not built yet");
    return HT_ERR_UNSUPPORTED;
}

ht_status ht_train_destroy(ht_train *t)
{
    (void)t;
    return HT_OK;
}

ht_status ht_train_step_fwd(ht_train *t, const ht_image *crops, int n, const float *gray_levels, uint64_t seed,
                            double *losses_host, void *stream)
{
    (void)t; (void)crops; (void)n; (void)gray_levels; (void)seed; (void)losses_host; (void)stream;
    ht_set_error("training step not built yet");
    return HT_ERR_UNSUPPORTED;
}

ht_status ht_train_step_bwd(ht_train *t, float *grad_w, float *grad_b, void *stream)
{
    (void)t; (void)grad_w; (void)grad_b; (void)stream;
    ht_set_error("training step not built yet");
    return HT_ERR_UNSUPPORTED;
}

}  // extern "C"
