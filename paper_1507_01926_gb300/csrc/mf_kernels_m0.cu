// Solver kernel instances for batches and service unions (per-vertex label caps, per-instance relabel schedules and phases), register-budget variants 0, 1, 2; the kernel is
// mf_solver.cuh. The variants are spread over several units so that they compile in parallel.
#include "mf_solver.cuh"

namespace mf {

template __global__ void solve_kernel<512, 1, KT, true>(Dev);
template __global__ void solve_kernel<256, 3, KT, true>(Dev);
template __global__ void solve_kernel<256, 4, KT, true>(Dev);

// Entry point of variant v if this unit holds it, else nullptr (a template kernel's host stub is local to
// the unit that instantiates it).
const void *solver_kernel_m0(int v) {
  switch (v) {
    case 0: return (const void *)solve_kernel<512, 1, KT, true>;
    case 1: return (const void *)solve_kernel<256, 3, KT, true>;
    case 2: return (const void *)solve_kernel<256, 4, KT, true>;
    default: return nullptr;
  }
}

}  // namespace mf
