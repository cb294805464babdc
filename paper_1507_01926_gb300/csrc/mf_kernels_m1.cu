// Solver kernel instances for batches and service unions (per-vertex label caps, per-instance relabel schedules and phases), register-budget variants 3, 4; the kernel is
// mf_solver.cuh. The variants are spread over several units so that they compile in parallel.
#include "mf_solver.cuh"

namespace mf {

template __global__ void solve_kernel<512, 2, KT, true>(Dev);
template __global__ void solve_kernel<256, 1, 16, true>(Dev);

// Entry point of variant v if this unit holds it, else nullptr (a template kernel's host stub is local to
// the unit that instantiates it).
const void *solver_kernel_m1(int v) {
  switch (v) {
    case 3: return (const void *)solve_kernel<512, 2, KT, true>;
    case 4: return (const void *)solve_kernel<256, 1, 16, true>;
    default: return nullptr;
  }
}

}  // namespace mf
