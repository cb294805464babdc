// Synchronous parallel push-relabel solver (arXiv:1507.01926, Section 3.1 and
// Algorithm 1, global relabels by Algorithm 2): the host side of the launch
// (register-budget variants, occupancy, cooperative launch). The kernel is in
// mf_solver.cuh; its instances (single graphs and unions, five register
// budgets each) are compiled in mf_kernels_*.cu.
#include "mf_solver.cuh"

namespace mf {

// ------------------------------------------------------------------ host side

// kernel entry points by variant, from the units that instantiate them (nullptr if the unit has not the variant)
const void *solver_kernel_s0(int v);
const void *solver_kernel_s1(int v);
const void *solver_kernel_m0(int v);
const void *solver_kernel_m1(int v);

static const void *kernel_fn(int variant, bool multi) {
  const void *f = multi ? solver_kernel_m0(variant) : solver_kernel_s0(variant);
  return f ? f : (multi ? solver_kernel_m1(variant) : solver_kernel_s1(variant));
}

struct Variant {
  int max_threads;
  int max_bin_thread;  // KTD
};

static const Variant kVariants[] = {
    {512, KT},  // 0: __launch_bounds__(512, 1), up to 128 registers
    {256, KT},  // 1: (256, 3), up to 85
    {256, KT},  // 2: (256, 4), up to 64
    {512, KT},  // 3: (512, 2), up to 64
    {256, 16},  // 4: (256, 1), up to 255; one thread discharges up to 16 slots
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
  const void *fn = kernel_fn(variant, multi);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block_threads, 0);
  return e == cudaSuccess ? 0 : -1;
}

cudaError_t launch_solver(const Dev &D, int grid, int block, cudaStream_t stream, int variant) {
  Dev d = D;
  void *args[] = {&d};
  const void *fn = kernel_fn(variant, D.vinst != nullptr);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, stream);
}

}  // namespace mf
