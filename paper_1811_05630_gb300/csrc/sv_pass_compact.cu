// sv_pass_compact.cu — the fused pass for 1- and 2-qubit gates compiled with a register cap
// (1-qubit gates: 64 registers per thread, spilling, so that 4 CTAs of 256 threads fit on an
// SM; 2-qubit gates: 85 registers, 3 CTAs). A state selects it with sv_set_compact; results
// are identical, only the launch resources differ.
#include "sv_pass.cuh"

namespace sv {

cudaError_t launch_pass_compact(const PassArgs& a, int dtype, cudaStream_t st) {
  if (a.K > 4) return launch_pass(a, dtype, st);
  if (a.K > 2) return dtype == 1 ? launch_pass_k<float, 4, true>(a, st) : launch_pass_k<double, 4, true>(a, st);
  return dtype == 1 ? launch_pass_k<float, 2, true>(a, st) : launch_pass_k<double, 2, true>(a, st);
}

}  // namespace sv
