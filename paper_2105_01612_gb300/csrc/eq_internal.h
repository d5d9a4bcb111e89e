// eq_internal.h - host-side interface between the C ABI and the per-dtype kernel instances.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/eq.h"
#include "eq_kernels.cuh"
#include "eq_tma.cuh"
#include "eq_xrow.cuh"

namespace eqk {

struct PassInfo {
  int threads = 0;
  size_t smem = 0;
  int blocks_per_sm = 0;
};

enum PassKind { PASS_STRIDED_FWD = 0, PASS_STRIDED_INV = 1, PASS_XPROJ = 2 };

// Supported transform lengths of the compiled instances (powers of two 1..1024).
bool length_supported(int n);

// Launch shape of one pass for length n (sets the max dynamic shared memory attribute).
cudaError_t pass_info_f32(int n, PassKind kind, PassInfo* out);
cudaError_t pass_info_f64(int n, PassKind kind, PassInfo* out);

cudaError_t launch_strided_f32(int n, bool inv, const StridedArgs& a, dim3 grid, cudaStream_t s);
cudaError_t launch_strided_f64(int n, bool inv, const StridedArgs& a, dim3 grid, cudaStream_t s);
cudaError_t launch_xproj_f32(int n, const XArgs& a, dim3 grid, cudaStream_t s);
cudaError_t launch_xproj_f64(int n, const XArgs& a, dim3 grid, cudaStream_t s);
// potential x pass (reads the stress spectrum, writes the x-inverted y rows; XArgs::ydata)
cudaError_t launch_xpot_f32(int n, const XArgs& a, dim3 grid, cudaStream_t s);
cudaError_t launch_xpot_f64(int n, const XArgs& a, dim3 grid, cudaStream_t s);
// the same in the warp-per-row kernel (x variants 2 and 3; XTmaArgs::ydata)
cudaError_t launch_xpot_warp_f32(int n, int v, const XTmaArgs& a, dim3 grid, cudaStream_t s);
cudaError_t launch_xpot_warp_f64(int n, int v, const XTmaArgs& a, dim3 grid, cudaStream_t s);

// TMA-fed strided passes: info returns cudaErrorInvalidValue when no instance exists for n.
// v selects the shape variant (0: wide tiles, one block per SM; 1: narrow tiles, two blocks).
struct TmaInfo {
  int threads = 0, cols = 0, box = 0, blocks_per_sm = 0;
  size_t smem = 0;
};
cudaError_t tma_info_f32(int n, int v, TmaInfo* out);
cudaError_t tma_info_f64(int n, int v, TmaInfo* out);
cudaError_t launch_tma_f32(int n, int v, bool inv, const CUtensorMap& map, const CUtensorMap& refmap,
                           const CUtensorMap& outmap, const TmaArgs& a, dim3 grid, cudaStream_t s);
cudaError_t launch_tma_f64(int n, int v, bool inv, const CUtensorMap& map, const CUtensorMap& refmap,
                           const CUtensorMap& outmap, const TmaArgs& a, dim3 grid, cudaStream_t s);
// fused x pass variants (0, 1: bulk-copy row groups; 2, 3: warp per row through a bulk-copy stage,
// three / four blocks per SM; 4, 5: warp per row with direct loads and stores, four / five blocks
// per SM in FP32; 6: as 4 with the next row pair's loads issued early, three blocks): info fails
// when no instance exists for n
cudaError_t xtma_info_f32(int n, int v, TmaInfo* out);
cudaError_t xtma_info_f64(int n, int v, TmaInfo* out);
cudaError_t launch_xtma_f32(int n, int v, const XTmaArgs& a, dim3 grid, cudaStream_t s);
cudaError_t launch_xtma_f64(int n, int v, const XTmaArgs& a, dim3 grid, cudaStream_t s);

// Finalisation kernels of the power-of-two path (fixed-order FP64 reductions of block partials).
void finalize_mean(const double* part, int grid, int batch, double vol, double* mean,
                   double* instats, cudaStream_t s);
void finalize_norms(const double* partx, int gridx, const double* partl, int gridl, int batch,
                    double vol, const double* mean, const double* instats, int linf_flag,
                    eq_norms_t* out, cudaStream_t s);
void set_last_error(const std::string& msg);
// diagnostics on stderr when the environment's EQ_LOG level is at least `level` (eq_api.cu)
void log(int level, const char* fmt, ...);

}  // namespace eqk
