// Learned cardinality estimator (placeholder until the tensor-core MLP lands).
#include <string>

#include "internal.h"

struct huge_mlp {
    int dummy;
};

namespace huge {
int mlp_predict(const huge_mlp_t *m, const float *x, int rows, float *y, std::string *err) {
    (void)m; (void)x; (void)rows; (void)y;
    *err = "learned estimator not available";
    return HUGE_EINVAL;
}
}  // namespace huge
