// eq_gen_inst.cuh - launch wrappers of the runtime-length passes, included once per dtype.
#pragma once
#include <type_traits>

#include "eq_gen.cuh"

namespace eqg {

template <typename T> struct GenInst {
  static const void* fn(int kind) {
    if (kind == 0) return reinterpret_cast<const void*>(&k_gen_strided<T, false>);
    if (kind == 1) return reinterpret_cast<const void*>(&k_gen_strided<T, true>);
    if (kind == 3) return reinterpret_cast<const void*>(&k_gen_xrows<T>);
    if constexpr (std::is_same<T, float>::value) {       // the warp-per-column kernel is FP32
      if (kind == 4) return reinterpret_cast<const void*>(&k_gen_scols<false>);
      if (kind == 5) return reinterpret_cast<const void*>(&k_gen_scols<true>);
      if (kind == 6) return reinterpret_cast<const void*>(&k_gen_xpair<float>);
    } else if (kind == 4 || kind == 5 || kind == 6) {
      return nullptr;
    }
    return reinterpret_cast<const void*>(&k_gen_xproj<T>);
  }
  static cudaError_t occupancy(int kind, int threads, size_t smem, int* blocks) {
    // one kernel serves passes with different shared-memory sizes: allow the device maximum
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess && ((size_t)optin < smem || !fn(kind))) return cudaErrorInvalidValue;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn(kind), cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn(kind), threads, smem);
  }
  static cudaError_t launch(int kind, const GenArgs& a, int grid, int threads, size_t smem,
                            cudaStream_t s) {
    if (kind == 0) k_gen_strided<T, false><<<grid, threads, smem, s>>>(a);
    else if (kind == 1) k_gen_strided<T, true><<<grid, threads, smem, s>>>(a);
    else if (kind == 3) k_gen_xrows<T><<<grid, threads, smem, s>>>(a);
    else if (kind == 4 || kind == 5 || kind == 6) {
      if constexpr (std::is_same<T, float>::value) {
        if (kind == 4) k_gen_scols<false><<<grid, threads, smem, s>>>(a);
        else if (kind == 5) k_gen_scols<true><<<grid, threads, smem, s>>>(a);
        else k_gen_xpair<float><<<grid, threads, smem, s>>>(a);
      } else {
        return cudaErrorInvalidValue;
      }
    }
    else k_gen_xproj<T><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
  }
};

}  // namespace eqg
