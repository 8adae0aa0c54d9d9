// Learned output-size estimator: per-column features and the MLP that
// predicts nnz((AA)_*j) (filled in below).
#include <cuda_runtime.h>

#include "mcl.h"
#include "mcl_internal.h"

struct mcl_ctx;

mcl_status mcl_internal_estimate(mcl_ctx* c, const mcl_csc* A, const mcl::ExpandBuffers& b,
                                 cudaStream_t s) {
    (void)c;
    (void)A;
    (void)b;
    (void)s;
    return MCL_ERR_INVALID;
}
