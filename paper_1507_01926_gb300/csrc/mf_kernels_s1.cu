// Solver kernel instances for single graphs, register-budget variants 3, 4; the kernel is
// mf_solver.cuh. The variants are spread over several units so that they compile in parallel.
#include "mf_solver.cuh"

namespace mf {

template __global__ void solve_kernel<512, 2, KT, false>(Dev);
template __global__ void solve_kernel<256, 1, 16, false>(Dev);

// Entry point of variant v if this unit holds it, else nullptr (a template kernel's host stub is local to
// the unit that instantiates it).
const void *solver_kernel_s1(int v) {
  switch (v) {
    case 3: return (const void *)solve_kernel<512, 2, KT, false>;
    case 4: return (const void *)solve_kernel<256, 1, 16, false>;
    default: return nullptr;
  }
}

}  // namespace mf
