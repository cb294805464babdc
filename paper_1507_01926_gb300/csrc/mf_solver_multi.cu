// The solver kernel instances for batches and service unions (per-vertex label
// caps, per-instance global-relabel schedules); see mf_solver.cuh.
#include "mf_solver.cuh"

namespace mf {

// Kernel entry points of this unit for the launch code in mf_solver.cu, by
// register-budget variant (a template kernel's host stub is local to the unit
// that instantiates it).
const void *solver_multi_fn(int variant) {
  switch (variant) {
    case 0: return (const void *)solve_kernel<512, 1, KT, true>;
    case 1: return (const void *)solve_kernel<256, 3, KT, true>;
    case 2: return (const void *)solve_kernel<256, 4, KT, true>;
    case 3: return (const void *)solve_kernel<512, 2, KT, true>;
    case 4: return (const void *)solve_kernel<256, 1, 16, true>;
    default: return nullptr;
  }
}

template __global__ void solve_kernel<512, 1, KT, true>(Dev);
template __global__ void solve_kernel<256, 3, KT, true>(Dev);
template __global__ void solve_kernel<256, 4, KT, true>(Dev);
template __global__ void solve_kernel<512, 2, KT, true>(Dev);
template __global__ void solve_kernel<256, 1, 16, true>(Dev);

}  // namespace mf
