// eq_gen_f32.cu - FP32 instances of the runtime-length passes.
#include "eq_gen_inst.cuh"
#include "eq_gen_host.h"

namespace eqg {
cudaError_t gen_occupancy_f32(int kind, int threads, size_t smem, int* blocks) {
  return GenInst<float>::occupancy(kind, threads, smem, blocks);
}
cudaError_t gen_launch_f32(int kind, const GenArgs& a, int grid, int threads, size_t smem, cudaStream_t s) {
  return GenInst<float>::launch(kind, a, grid, threads, smem, s);
}
}  // namespace eqg
