// Mixed-precision slab elimination (tensor cores); filled in by tc_gemm.cu.
#include "apf_internal.h"

struct MixedWork {};

int mixed_alloc(apf_ctx *c) { return set_err(c, APF_EINVAL, "mixed precision is not available in this build"); }
void mixed_free(apf_ctx *c) { (void)c; }
int mixed_eliminate(apf_ctx *c, cudaStream_t) { return set_err(c, APF_EINVAL, "mixed precision is not available"); }
int mixed_solve_fields(apf_ctx *c, cudaStream_t) { return set_err(c, APF_EINVAL, "mixed precision is not available"); }
void mixed_init_attrs() {}
