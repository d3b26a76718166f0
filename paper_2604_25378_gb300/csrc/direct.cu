// Direct configuration of the affine-normal block (dense reduced solve).
#include "internal.h"
#include "mvsk.h"
#include "solver_kernels.cuh"

struct mvsk_ctx;
namespace {
mvsk_status direction_direct_impl(mvsk_ctx*) { return MVSK_EINVAL; }
}  // namespace
mvsk_status direction_direct(mvsk_ctx* c) { return direction_direct_impl(c); }

extern "C" mvsk_status mvsk_oracle_gram(mvsk_ctx*, const double*, double*) { return MVSK_EINVAL; }
