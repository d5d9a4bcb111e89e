// eq_f32.cu - FP32 instances of the pass kernels.
#include "eq_dispatch.cuh"

namespace eqk {
cudaError_t pass_info_f32(int n, PassKind kind, PassInfo* out) { return info_t<float>(n, kind, out); }
cudaError_t launch_strided_f32(int n, bool inv, const StridedArgs& a, dim3 grid, cudaStream_t s) {
  return strided_t<float>(n, inv, a, grid, s);
}
cudaError_t launch_xproj_f32(int n, const XArgs& a, dim3 grid, cudaStream_t s) {
  return xproj_t<float>(n, a, grid, s);
}
cudaError_t launch_xpot_warp_f32(int n, int v, const XTmaArgs& a, dim3 grid, cudaStream_t s) {
  return xpot_warp_t<float>(n, v, a, grid, s);
}
cudaError_t launch_xpot_f32(int n, const XArgs& a, dim3 grid, cudaStream_t s) {
  return xpot_t<float>(n, a, grid, s);
}
cudaError_t tma_info_f32(int n, int v, TmaInfo* out) { return tma_info_t<float>(n, v, out); }
cudaError_t launch_tma_f32(int n, int v, bool inv, const CUtensorMap& map, const CUtensorMap& refmap,
                           const CUtensorMap& outmap, const TmaArgs& a, dim3 grid, cudaStream_t s) {
  return tma_launch_t<float>(n, v, inv, map, refmap, outmap, a, grid, s);
}
cudaError_t xtma_info_f32(int n, int v, TmaInfo* out) { return xtma_info_t<float>(n, v, out); }
cudaError_t launch_xtma_f32(int n, int v, const XTmaArgs& a, dim3 grid, cudaStream_t s) {
  return xtma_launch_t<float>(n, v, a, grid, s);
}
}  // namespace eqk
