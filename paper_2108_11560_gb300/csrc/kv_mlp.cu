// The learned bracket (2-64-64-2 MLP) -- handle management, inference and training kernels.
#include <cuda_runtime.h>

#include "kv_internal.h"

struct kv_mlp {
    int magic;
};

namespace kvh {

int mlp_view(const kv_mlp* h, MlpView* out)
{
    (void)out;
    return h ? KV_ERR_HANDLE : KV_ERR_HANDLE;
}

int launch_mlp_path(const kv_args* a, int bins, double log_eps, int max_iter)
{
    (void)a;
    (void)bins;
    (void)log_eps;
    (void)max_iter;
    return KV_ERR_HANDLE;
}

}  // namespace kvh

extern "C" {
int kv_mlp_create(uint64_t, kv_mlp**) { return KV_ERR_HANDLE; }
int kv_mlp_free(kv_mlp*) { return KV_OK; }
int kv_mlp_save(const kv_mlp*, const char*) { return KV_ERR_HANDLE; }
int kv_mlp_load(const char*, kv_mlp**) { return KV_ERR_HANDLE; }
int kv_mlp_get_params(const kv_mlp*, float*, int64_t) { return KV_ERR_HANDLE; }
int kv_mlp_set_params(kv_mlp*, const float*, int64_t) { return KV_ERR_HANDLE; }
int kv_mlp_train(kv_mlp*, const kv_train_args*) { return KV_ERR_HANDLE; }
int kv_mlp_loss_grad(const kv_mlp*, const double*, const double*, const double*, const double*,
                     int64_t, double*, float*, void*)
{
    return KV_ERR_HANDLE;
}
int kv_mlp_predict(const kv_mlp*, const void*, const void*, void*, void*, int64_t, int, void*)
{
    return KV_ERR_HANDLE;
}
}
