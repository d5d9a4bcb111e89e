// eq_dispatch.cuh - runtime length -> template instance dispatch, included once per dtype.
#pragma once
#include "eq_internal.h"

namespace eqk {

template <typename T, int N> struct Inst {
  static cudaError_t info(PassKind kind, PassInfo* out) {
    using C = Cfg<T, N>;
    const void* fn;
    if (kind == PASS_XPROJ) {
      fn = reinterpret_cast<const void*>(&k_xproj<T, N>);
      out->threads = C::X_THREADS;
      out->smem = C::X_SMEM;
      // the potential x pass has the same shape
      cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_xpot<T, N>),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)out->smem);
      if (e != cudaSuccess) return e;
    } else {
      fn = kind == PASS_STRIDED_INV ? reinterpret_cast<const void*>(&k_strided<T, N, true>)
                                    : reinterpret_cast<const void*>(&k_strided<T, N, false>);
      out->threads = C::STRIDED_THREADS;
      out->smem = C::STRIDED_SMEM;
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)out->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out->blocks_per_sm, fn, out->threads,
                                                         out->smem);
  }
  static cudaError_t strided(bool inv, const StridedArgs& a, dim3 grid, cudaStream_t s) {
    using C = Cfg<T, N>;
    if (inv) k_strided<T, N, true><<<grid, C::STRIDED_THREADS, C::STRIDED_SMEM, s>>>(a);
    else k_strided<T, N, false><<<grid, C::STRIDED_THREADS, C::STRIDED_SMEM, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t xproj(const XArgs& a, dim3 grid, cudaStream_t s) {
    using C = Cfg<T, N>;
    k_xproj<T, N><<<grid, C::X_THREADS, C::X_SMEM, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t xpot(const XArgs& a, dim3 grid, cudaStream_t s) {
    using C = Cfg<T, N>;
    k_xpot<T, N><<<grid, C::X_THREADS, C::X_SMEM, s>>>(a);
    return cudaGetLastError();
  }
};

template <typename T, int N, int V> struct TmaInst {
  static cudaError_t info(TmaInfo* out) {
    using C = TmaCfg<T, N, V>;
    if constexpr (!C::OK) {
      return cudaErrorInvalidValue;
    } else {
      out->threads = C::THREADS;
      out->cols = C::B;
      out->box = C::BOX;
      out->smem = C::SMEM;
      const void* fns[5] = {reinterpret_cast<const void*>(&k_strided_tma<T, N, false, 1, V>),
                            reinterpret_cast<const void*>(&k_strided_tma<T, N, false, 0, V>),
                            reinterpret_cast<const void*>(&k_strided_tma<T, N, true, 0, V>),
                            reinterpret_cast<const void*>(&k_strided_tma<T, N, true, 2, V>),
                            reinterpret_cast<const void*>(&k_strided_tma<T, N, true, 3, V>)};
      cudaError_t e = cudaSuccess;
      for (const void* f : fns)
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
      int bl = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, fns[0], C::THREADS, C::SMEM);
      out->blocks_per_sm = bl;
      return e;
    }
  }
  static cudaError_t launch(bool inv, const CUtensorMap& map, const CUtensorMap& refmap,
                            const CUtensorMap& outmap, const TmaArgs& a, dim3 grid, cudaStream_t s) {
    using C = TmaCfg<T, N, V>;
    if constexpr (!C::OK) {
      return cudaErrorInvalidValue;
    } else {
      if (!inv && a.mode == 1)
        k_strided_tma<T, N, false, 1, V><<<grid, C::THREADS, C::SMEM, s>>>(map, refmap, outmap, a);
      else if (!inv)
        k_strided_tma<T, N, false, 0, V><<<grid, C::THREADS, C::SMEM, s>>>(map, refmap, outmap, a);
      else if (a.mode == 2)
        k_strided_tma<T, N, true, 2, V><<<grid, C::THREADS, C::SMEM, s>>>(map, refmap, outmap, a);
      else if (a.mode == 3)
        k_strided_tma<T, N, true, 3, V><<<grid, C::THREADS, C::SMEM, s>>>(map, refmap, outmap, a);
      else
        k_strided_tma<T, N, true, 0, V><<<grid, C::THREADS, C::SMEM, s>>>(map, refmap, outmap, a);
      return cudaGetLastError();
    }
  }
};

// shape variant 2 of the strided passes: 512-point FP32 columns, 16 x 32 (k_strided16)
struct Tma16Inst {
  static cudaError_t info(TmaInfo* out) {
    using C = Tma16Cfg;
    out->threads = C::THREADS;
    out->cols = C::B;
    out->box = C::BOX;
    out->smem = C::SMEM;
    const void* fns[5] = {reinterpret_cast<const void*>(&k_strided16<false, 1>),
                          reinterpret_cast<const void*>(&k_strided16<false, 0>),
                          reinterpret_cast<const void*>(&k_strided16<true, 0>),
                          reinterpret_cast<const void*>(&k_strided16<true, 2>),
                          reinterpret_cast<const void*>(&k_strided16<true, 3>)};
    cudaError_t e = cudaSuccess;
    for (const void* f : fns)
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    int bl = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, fns[0], C::THREADS, C::SMEM);
    out->blocks_per_sm = bl;
    return e;
  }
  static cudaError_t launch(bool inv, const CUtensorMap& map, const CUtensorMap& refmap,
                            const CUtensorMap& outmap, const TmaArgs& a, dim3 grid, cudaStream_t s) {
    using C = Tma16Cfg;
    if (!inv && a.mode == 1)
      k_strided16<false, 1><<<grid, C::THREADS, C::SMEM, s>>>(map, refmap, outmap, a);
    else if (!inv)
      k_strided16<false, 0><<<grid, C::THREADS, C::SMEM, s>>>(map, refmap, outmap, a);
    else if (a.mode == 2)
      k_strided16<true, 2><<<grid, C::THREADS, C::SMEM, s>>>(map, refmap, outmap, a);
    else if (a.mode == 3)
      k_strided16<true, 3><<<grid, C::THREADS, C::SMEM, s>>>(map, refmap, outmap, a);
    else
      k_strided16<true, 0><<<grid, C::THREADS, C::SMEM, s>>>(map, refmap, outmap, a);
    return cudaGetLastError();
  }
};

template <typename T, int N, int V> struct XTmaInst {
  static cudaError_t info(TmaInfo* out) {
    using C = XTmaCfg<T, N, V>;
    if constexpr (!C::OK) {
      return cudaErrorInvalidValue;
    } else {
      out->threads = C::THREADS;
      out->cols = C::P;
      out->box = 0;
      out->smem = C::SMEM;
      const void* f = reinterpret_cast<const void*>(&k_xproj_tma<T, N, V>);
      cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
      int bl = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, f, C::THREADS, C::SMEM);
      out->blocks_per_sm = bl;
      return e;
    }
  }
  static cudaError_t launch(const XTmaArgs& a, dim3 grid, cudaStream_t s) {
    using C = XTmaCfg<T, N, V>;
    if constexpr (!C::OK) {
      return cudaErrorInvalidValue;
    } else {
      k_xproj_tma<T, N, V><<<grid, C::THREADS, C::SMEM, s>>>(a);
      return cudaGetLastError();
    }
  }
};

template <typename T, int N, int MINB> struct XwInst {
  static cudaError_t info(TmaInfo* out) {
    using C = XwCfg<T, N, MINB>;
    if constexpr (!C::OK) {
      return cudaErrorInvalidValue;
    } else {
      out->threads = C::THREADS;
      out->cols = 1;
      out->box = 0;
      out->smem = C::SMEM;
      const void* f = reinterpret_cast<const void*>(&k_xproj_warp<T, N, MINB, false>);
      const void* fp = reinterpret_cast<const void*>(&k_xproj_warp<T, N, MINB, true>);
      cudaError_t e = cudaSuccess;
      for (const void* g : {f, fp}) {
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(g, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(g, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared);
      }
      int bl = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, f, C::THREADS, C::SMEM);
      out->blocks_per_sm = bl;
      return e;
    }
  }
  static cudaError_t launch(const XTmaArgs& a, dim3 grid, cudaStream_t s, bool pot = false) {
    using C = XwCfg<T, N, MINB>;
    if constexpr (!C::OK) {
      return cudaErrorInvalidValue;
    } else {
      if (pot) k_xproj_warp<T, N, MINB, true><<<grid, C::THREADS, C::SMEM, s>>>(a);
      else k_xproj_warp<T, N, MINB, false><<<grid, C::THREADS, C::SMEM, s>>>(a);
      return cudaGetLastError();
    }
  }
};

template <typename T, int N, int MINB, bool PF = false> struct XrInst {
  static cudaError_t info(TmaInfo* out) {
    using C = XrCfg<T, N>;
    if constexpr (!C::OK) {
      return cudaErrorInvalidValue;
    } else {
      out->threads = C::THREADS;
      out->cols = 1;
      out->box = 0;
      out->smem = C::SMEM;
      const void* f = reinterpret_cast<const void*>(&k_xproj_rows<T, N, MINB, false, PF>);
      const void* fp = reinterpret_cast<const void*>(&k_xproj_rows<T, N, MINB, true, PF>);
      cudaError_t e = cudaSuccess;
      for (const void* g : {f, fp}) {
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(g, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(g, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared);
      }
      int bl = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, f, C::THREADS, C::SMEM);
      out->blocks_per_sm = bl;
      return e;
    }
  }
  static cudaError_t launch(const XTmaArgs& a, dim3 grid, cudaStream_t s, bool pot = false) {
    using C = XrCfg<T, N>;
    if constexpr (!C::OK) {
      return cudaErrorInvalidValue;
    } else {
      if (pot) k_xproj_rows<T, N, MINB, true, PF><<<grid, C::THREADS, C::SMEM, s>>>(a);
      else k_xproj_rows<T, N, MINB, false, PF><<<grid, C::THREADS, C::SMEM, s>>>(a);
      return cudaGetLastError();
    }
  }
};

// the packed two-row x pass (k_xproj_pair): 512-point FP32 rows only
template <typename T, int N, int MINB, bool STAGED = false> struct XpInst {
  static constexpr bool OK = sizeof(T) == 4 && N == 512;
  using C = XpCfg<STAGED>;
  static cudaError_t info(TmaInfo* out) {
    if constexpr (!OK) {
      return cudaErrorInvalidValue;
    } else {
      out->threads = C::THREADS;
      out->cols = 1;
      out->box = 0;
      out->smem = C::SMEM;
      const void* f = reinterpret_cast<const void*>(&k_xproj_pair<MINB, STAGED>);
      const void* fp = reinterpret_cast<const void*>(&k_xproj_pair<MINB, STAGED, true>);
      cudaError_t e = cudaSuccess;
      for (const void* g : {f, fp}) {
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(g, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(g, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared);
      }
      int bl = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, f, C::THREADS, C::SMEM);
      out->blocks_per_sm = bl;
      return e;
    }
  }
  static cudaError_t launch(const XTmaArgs& a, dim3 grid, cudaStream_t s, bool pot = false) {
    if constexpr (!OK) {
      return cudaErrorInvalidValue;
    } else {
      if (pot) k_xproj_pair<MINB, STAGED, true><<<grid, C::THREADS, C::SMEM, s>>>(a);
      else k_xproj_pair<MINB, STAGED><<<grid, C::THREADS, C::SMEM, s>>>(a);
      return cudaGetLastError();
    }
  }
};

// blocks per SM asked of the register allocator for the warp-per-row x pass: FP32 variants 2 and
// 3 target three and four blocks; FP64 rows take twice the shared memory, so one and two
template <typename T> constexpr int XW_MINB(int fp32_blocks) {
  return sizeof(T) == 4 ? fp32_blocks : fp32_blocks - 2;
}

#define EQ_FOR_LENGTHS(X) X(1) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)

template <typename T> cudaError_t info_t(int n, PassKind kind, PassInfo* out) {
  switch (n) {
#define EQ_CASE(N) case N: return Inst<T, N>::info(kind, out);
    EQ_FOR_LENGTHS(EQ_CASE)
#undef EQ_CASE
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
cudaError_t strided_t(int n, bool inv, const StridedArgs& a, dim3 grid, cudaStream_t s) {
  switch (n) {
#define EQ_CASE(N) case N: return Inst<T, N>::strided(inv, a, grid, s);
    EQ_FOR_LENGTHS(EQ_CASE)
#undef EQ_CASE
    default: return cudaErrorInvalidValue;
  }
}
template <typename T> cudaError_t xpot_t(int n, const XArgs& a, dim3 grid, cudaStream_t s) {
  switch (n) {
#define EQ_CASE(N) case N: return Inst<T, N>::xpot(a, grid, s);
    EQ_FOR_LENGTHS(EQ_CASE)
#undef EQ_CASE
    default: return cudaErrorInvalidValue;
  }
}
template <typename T> cudaError_t xproj_t(int n, const XArgs& a, dim3 grid, cudaStream_t s) {
  switch (n) {
#define EQ_CASE(N) case N: return Inst<T, N>::xproj(a, grid, s);
    EQ_FOR_LENGTHS(EQ_CASE)
#undef EQ_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T> cudaError_t tma_info_t(int n, int v, TmaInfo* out) {
  if (v == 2) {
    if constexpr (sizeof(T) == 4) {
      if (n == 512) return Tma16Inst::info(out);
    }
    return cudaErrorInvalidValue;
  }
  switch (n) {
#define EQ_CASE(N) case N: return v ? TmaInst<T, N, 1>::info(out) : TmaInst<T, N, 0>::info(out);
    EQ_FOR_LENGTHS(EQ_CASE)
#undef EQ_CASE
    default: return cudaErrorInvalidValue;
  }
}
template <typename T>
cudaError_t tma_launch_t(int n, int v, bool inv, const CUtensorMap& map, const CUtensorMap& refmap,
                         const CUtensorMap& outmap, const TmaArgs& a, dim3 grid, cudaStream_t s) {
  if (v == 2) {
    if constexpr (sizeof(T) == 4) {
      if (n == 512) return Tma16Inst::launch(inv, map, refmap, outmap, a, grid, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (n) {
#define EQ_CASE(N)                                                              \
  case N:                                                                         \
    return v ? TmaInst<T, N, 1>::launch(inv, map, refmap, outmap, a, grid, s)    \
             : TmaInst<T, N, 0>::launch(inv, map, refmap, outmap, a, grid, s);
    EQ_FOR_LENGTHS(EQ_CASE)
#undef EQ_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T> cudaError_t xtma_info_t(int n, int v, TmaInfo* out) {
  switch (n) {
#define EQ_CASE(N)                                              \
  case N:                                                         \
    return v == 8   ? XpInst<T, N, 4, true>::info(out)                        \
           : v == 7 ? XpInst<T, N, 5>::info(out)                              \
           : v == 6 ? XrInst<T, N, XW_MINB<T>(3), true>::info(out)            \
           : v == 5 ? XrInst<T, N, XW_MINB<T>(5)>::info(out)                  \
           : v == 4 ? XrInst<T, N, XW_MINB<T>(4)>::info(out)                  \
           : v == 3 ? XwInst<T, N, XW_MINB<T>(4)>::info(out)                  \
           : v == 2 ? XwInst<T, N, XW_MINB<T>(3)>::info(out)                  \
                    : (v ? XTmaInst<T, N, 1>::info(out) : XTmaInst<T, N, 0>::info(out));
    EQ_FOR_LENGTHS(EQ_CASE)
#undef EQ_CASE
    default: return cudaErrorInvalidValue;
  }
}
// potential x pass in the warp-per-row and packed two-row kernels (variants 2 to 8)
template <typename T> cudaError_t xpot_warp_t(int n, int v, const XTmaArgs& a, dim3 grid, cudaStream_t s) {
  if (v < 2 || v > 8) return cudaErrorInvalidValue;
  switch (n) {
#define EQ_CASE(N)                                                                     \
  case N:                                                                                \
    return v == 8   ? XpInst<T, N, 4, true>::launch(a, grid, s, true)                   \
           : v == 7 ? XpInst<T, N, 5>::launch(a, grid, s, true)                         \
           : v == 6 ? XrInst<T, N, XW_MINB<T>(3), true>::launch(a, grid, s, true)       \
           : v == 5 ? XrInst<T, N, XW_MINB<T>(5)>::launch(a, grid, s, true)             \
           : v == 4 ? XrInst<T, N, XW_MINB<T>(4)>::launch(a, grid, s, true)             \
           : v == 3 ? XwInst<T, N, XW_MINB<T>(4)>::launch(a, grid, s, true)             \
                    : XwInst<T, N, XW_MINB<T>(3)>::launch(a, grid, s, true);
    EQ_FOR_LENGTHS(EQ_CASE)
#undef EQ_CASE
    default: return cudaErrorInvalidValue;
  }
}
template <typename T> cudaError_t xtma_launch_t(int n, int v, const XTmaArgs& a, dim3 grid, cudaStream_t s) {
  switch (n) {
#define EQ_CASE(N)                                                       \
  case N:                                                                  \
    return v == 8   ? XpInst<T, N, 4, true>::launch(a, grid, s)                        \
           : v == 7 ? XpInst<T, N, 5>::launch(a, grid, s)                              \
           : v == 6 ? XrInst<T, N, XW_MINB<T>(3), true>::launch(a, grid, s)            \
           : v == 5 ? XrInst<T, N, XW_MINB<T>(5)>::launch(a, grid, s)                  \
           : v == 4 ? XrInst<T, N, XW_MINB<T>(4)>::launch(a, grid, s)                  \
           : v == 3 ? XwInst<T, N, XW_MINB<T>(4)>::launch(a, grid, s)                  \
           : v == 2 ? XwInst<T, N, XW_MINB<T>(3)>::launch(a, grid, s)                  \
                    : (v ? XTmaInst<T, N, 1>::launch(a, grid, s) : XTmaInst<T, N, 0>::launch(a, grid, s));
    EQ_FOR_LENGTHS(EQ_CASE)
#undef EQ_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace eqk
