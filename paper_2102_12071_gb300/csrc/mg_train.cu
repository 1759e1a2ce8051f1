// mg_train.cu -- training-loss kernels (placeholder until the adjoint kernels land).
#include "mg_internal.h"
#include "mgcnn.h"

struct mg_train_ctx {
  int unused;
};

extern "C" {
size_t mg_train_workspace_size(const mg_problem*, int, int, const mg_options*) { return 0; }
mg_status mg_train_setup(const mg_problem*, int, int, const mg_options*, void*, size_t, void*, mg_train_ctx** out) {
  if (out) *out = nullptr;
  return MG_ERR_UNSUPPORTED;
}
void mg_train_destroy(mg_train_ctx* ctx) { delete ctx; }
mg_status mg_train_step(mg_train_ctx*, const float*, const float*, float*, float*, void*) { return MG_ERR_UNSUPPORTED; }
}
