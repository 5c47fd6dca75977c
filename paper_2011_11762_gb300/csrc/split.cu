// Split-precision numeric phase (step S7): placeholder until the tcgen05
// kernel lands.
#include "internal.h"

namespace cht {

int split_multiply(cht_plan *, cht_mat *, cht_mat *, int, cudaStream_t, double *, double *) {
  set_error("the split-precision form is not built yet");
  return CHT_ERR_UNSUPPORTED;
}

}  // namespace cht
