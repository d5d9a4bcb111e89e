// eq_gen_dd.cu - the runtime-length passes of FP64 plans in double-float arithmetic (FP64 in HBM
// at the pipeline's ends, pairs of FP32 values between the passes): the warp-per-column strided
// kernel (kinds 4, 5) and the warp-per-row x kernel (kind 7); every axis length of such a plan
// has a 256- or 512-point register transform.
#include "eq_gen.cuh"
#include "eq_gen_host.h"

namespace eqg {
namespace {
const void* dd_fn(int kind) {
  if (kind == 7) return reinterpret_cast<const void*>(&k_gen_xdd<eqk::dd>);
  if (kind == 4) return reinterpret_cast<const void*>(&k_gen_scold<eqk::dd, false>);
  if (kind == 5) return reinterpret_cast<const void*>(&k_gen_scold<eqk::dd, true>);
  return nullptr;
}
}  // namespace

cudaError_t gen_occupancy_dd(int kind, int threads, size_t smem, int* blocks) {
  const void* f = dd_fn(kind);
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess && (!f || (size_t)optin < smem)) return cudaErrorInvalidValue;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, f, threads, smem);
}

cudaError_t gen_launch_dd(int kind, const GenArgs& a, int grid, int threads, size_t smem, cudaStream_t s) {
  if (kind == 7) k_gen_xdd<eqk::dd><<<grid, threads, smem, s>>>(a);
  else if (kind == 4) k_gen_scold<eqk::dd, false><<<grid, threads, smem, s>>>(a);
  else if (kind == 5) k_gen_scold<eqk::dd, true><<<grid, threads, smem, s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}
}  // namespace eqg
