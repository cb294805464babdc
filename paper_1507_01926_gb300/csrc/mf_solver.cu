// Synchronous parallel push-relabel solver (arXiv:1507.01926, Section 3.1 and
// Algorithm 1, global relabels by Algorithm 2): the kernel instances for single
// graphs and the host side of the launch (register-budget variants, occupancy,
// cooperative launch). The kernel itself is in mf_solver.cuh; the instances for
// batches and service unions are compiled in mf_solver_multi.cu.
#include "mf_solver.cuh"

namespace mf {

template __global__ void solve_kernel<512, 1, KT, false>(Dev);
template __global__ void solve_kernel<256, 3, KT, false>(Dev);
template __global__ void solve_kernel<256, 4, KT, false>(Dev);
template __global__ void solve_kernel<512, 2, KT, false>(Dev);
template __global__ void solve_kernel<256, 1, 16, false>(Dev);

// ------------------------------------------------------------------ host side

const void *solver_multi_fn(int variant);  // mf_solver_multi.cu

struct Variant {
  const void *fn;  // single graphs (the batch and union instances: solver_multi_fn)
  int max_threads;
  int max_bin_thread;  // KTD
};

static const Variant kVariants[] = {
    {(const void *)solve_kernel<512, 1, KT, false>, 512, KT},  // up to 128 registers
    {(const void *)solve_kernel<256, 3, KT, false>, 256, KT},  // up to 85
    {(const void *)solve_kernel<256, 4, KT, false>, 256, KT},  // up to 64
    {(const void *)solve_kernel<512, 2, KT, false>, 512, KT},  // up to 64
    {(const void *)solve_kernel<256, 1, 16, false>, 256, 16},  // up to 255; one thread discharges up to 16 slots
};
constexpr int NUM_VARIANTS = sizeof(kVariants) / sizeof(kVariants[0]);

int solver_variants() { return NUM_VARIANTS; }

int solver_variant_max_threads(int variant) {
  return variant >= 0 && variant < NUM_VARIANTS ? kVariants[variant].max_threads : 0;
}

int solver_variant_max_bin_thread(int variant) {
  return variant >= 0 && variant < NUM_VARIANTS ? kVariants[variant].max_bin_thread : 0;
}

int keep_local_limit(const mf_options &o, long long max_degree, int block_threads) {
  if (!o.local_lists || o.simple_rounds) return 0;
  if (max_degree > o.bin_thread || max_degree > KT) return 0;  // not every vertex is thread-sized
  const int k = o.local_lists == 1 ? block_threads / 2 : o.local_lists;
  return k < block_threads ? k : block_threads;  // block_threads <= MAX_BLOCK
}

int solver_occupancy(int block_threads, int *blocks_per_sm, int variant, bool multi) {
  if (variant < 0 || variant >= NUM_VARIANTS) return -1;
  const void *fn = multi ? solver_multi_fn(variant) : kVariants[variant].fn;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block_threads, 0);
  return e == cudaSuccess ? 0 : -1;
}

cudaError_t launch_solver(const Dev &D, int grid, int block, cudaStream_t stream, int variant) {
  Dev d = D;
  void *args[] = {&d};
  const void *fn = D.vinst ? solver_multi_fn(variant) : kVariants[variant].fn;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, stream);
}

}  // namespace mf
