// Batched products in one persistent launch (step S9): placeholder.
#include "internal.h"

struct cht_batch {
  int dummy = 0;
};

namespace cht {

int batch_create(int32_t, const cht_plan_t *, const cht_mat_t *, const cht_mat_t *, int, int32_t,
                 cudaStream_t, cht_batch **) {
  set_error("batched products are not built yet");
  return CHT_ERR_UNSUPPORTED;
}
int batch_run(cht_batch *, cudaStream_t) { return CHT_ERR_UNSUPPORTED; }
int batch_output(cht_batch *, int32_t, cht_mat **) { return CHT_ERR_UNSUPPORTED; }
void batch_destroy(cht_batch *b) { delete b; }

}  // namespace cht
