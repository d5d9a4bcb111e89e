// eq_gen_f64.cu - FP64 instances of the runtime-length passes.
#include "eq_gen_inst.cuh"
#include "eq_gen_host.h"

namespace eqg {
cudaError_t gen_occupancy_f64(int kind, int threads, size_t smem, int* blocks) {
  return GenInst<double>::occupancy(kind, threads, smem, blocks);
}
cudaError_t gen_launch_f64(int kind, const GenArgs& a, int grid, int threads, size_t smem, cudaStream_t s) {
  return GenInst<double>::launch(kind, a, grid, threads, smem, s);
}
}  // namespace eqg
