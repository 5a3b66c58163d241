// Tensor-core (tcgen05) form of the assembly contraction: see the kernel below.
#include "romb_internal.cuh"

romb_status launch_assemble_tc(romb_ctx* c) {
  (void)c;
  romb_set_error("tensor-core assembly not available in this build");
  return ROMB_E_ARG;
}
