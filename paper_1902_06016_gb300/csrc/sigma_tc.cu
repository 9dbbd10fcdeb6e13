// Low-precision ring contraction on the tcgen05 tensor cores (mixed-precision inner solves).
#include "gfcc_internal.cuh"

namespace gfcc {

void build_low_precision(gfcc_ctx* c, int kind) {
  (void)c;
  (void)kind;
  throw Error{GFCC_ERR_ARG, "low-precision sigma is not available in this build"};
}

void ring_lowprec(gfcc_ctx* c, const double* ut, double* ct, int nb, cudaStream_t s) {
  (void)c; (void)ut; (void)ct; (void)nb; (void)s;
  throw Error{GFCC_ERR_STATE, "low-precision ring requested without operands"};
}

}  // namespace gfcc
