// eq_static.cu - eq_project_static: the FP32 projection of one field with every piece of scratch
// memory (tables, reduction partials, flags) taken from a fixed array that the library declares
// in device memory, so the call itself allocates nothing.
//
// Who needs it: callers that may not allocate device memory at the moment they project - code
// running under a strict memory budget or a custom allocator that owns all device memory, or a
// host whose CUDA allocation calls are forbidden in the hot loop.  They pass their own input and
// output buffers (and a device buffer for the norms); nothing else is requested from CUDA.
//
// The scratch array is a file-scope __device__ variable of EQ_STATIC_SCRATCH_BYTES bytes.  Every
// GPU that loads the library holds it until the process exits.  Host code cannot use the array's
// name as a device address (it is a host-side shadow), so on the first call on each device, with
// that device current, the address is looked up with cudaGetSymbolAddress and cached together with
// the identity of the CUDA context it belongs to.  A later call that finds another context current
// (after cudaDeviceReset, or another driver context made current) looks the address up again, so
// a stale address is never used.  That first call (and the first one after a context change)
// should come before any stream capture.  All calls share the array and it keeps the
// last call's contents: every call writes all the tables and reduction partials it later reads
// (no part of it has to start at zero).  Calls whose work overlaps on the GPU (different streams,
// or several host threads without ordering) race on the array; order them.
#include <mutex>
#include <string>

#include "../../include/eq.h"
#include "eq_internal.h"

static __device__ __align__(256) unsigned char eq_static_scratch[EQ_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_static_mu;
// per device: the context the cached address belongs to (its process-unique id) and the address
struct StaticSlot {
  unsigned long long ctx_id = 0;
  void* ptr = nullptr;
};
StaticSlot g_static_slot[64];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

template <typename F> F driver_fn(const char* name) {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<F>(f);
}

// Process-unique id of the calling thread's current context (0 when none is current yet).
unsigned long long current_ctx_id() {
  static const CtxGetCurrentFn get = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
  static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get || !get_id || get(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

eq_status sfail(eq_status st, const std::string& m) {
  eqk::set_last_error(m);
  return st;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Device-side tables: twiddles exp(-2 pi i m / n) and operator symbols per axis, and the x-pass
// row-pair list, computed in FP64 with the CUDA math library and rounded to FP32.
__global__ void k_static_tables(int nx, int ny, int nz, int op, double hx, double hy, double hz,
                                float2* tw, float* xi, int* pairs) {
  const int lens[3] = {nx, ny, nz};
  const double hs[3] = {hx, hy, hz};
  int tw_off = 0, xi_off = 0;
  for (int a = 0; a < 3; ++a) {
    const int n = lens[a];
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
      double sn, cs;
      sincospi(-2.0 * double(m) / double(n), &sn, &cs);
      tw[tw_off + m] = make_float2(float(cs), float(sn));
      const int sf = (2 * m < n) ? m : m - n;
      double v;
      if (2 * m == n) v = 0.0;
      else if (op == EQ_OP_CDO) v = 2.0 * 3.14159265358979323846 * double(sf) / (double(n) * hs[a]);
      else v = sinpi(2.0 * double(sf) / double(n)) / hs[a];
      xi[xi_off + m] = float(v);
    }
    tw_off += n;
    xi_off += n;
  }
  // canonical rows (kz, ky) with (kz, ky) <= (-kz, -ky), listed in (kz, ky) order
  const int half = nz / 2 + 1;
  for (int kz = blockIdx.x * blockDim.x + threadIdx.x; kz < half; kz += gridDim.x * blockDim.x) {
    // rows before kz: full rows for 0 < kz' < kz that are not self-mirror, half rows otherwise
    int before = 0;
    for (int k = 0; k < kz; ++k) {
      const bool self = (k == 0) || (2 * k == nz);
      before += self ? ny / 2 + 1 : ny;
    }
    const bool self = (kz == 0) || (2 * kz == nz);
    if (!self && 2 * kz > nz) continue;
    const int cnt = self ? ny / 2 + 1 : ny;
    for (int ky = 0; ky < cnt; ++ky) pairs[before + ky] = kz * ny + ky;
  }
}

}  // namespace

extern "C" eq_status eq_project_static(int nx, int ny, int nz, const eq_plan_opts* opts,
                                       const float* d_in, float* d_out, eq_norms_t* d_norms,
                                       void* cuda_stream) {
  if (!d_in || !d_out) return sfail(EQ_ERR_INVALID, "eq_project_static: NULL buffer");
  for (int n : {nx, ny, nz})
    if (n < 1 || n > EQ_STATIC_MAX_N || (n & (n - 1)))
      return sfail(EQ_ERR_INVALID, "eq_project_static: axis lengths must be powers of two 1.." +
                                       std::to_string(EQ_STATIC_MAX_N));
  eq_plan_opts o;
  eq_plan_opts_default(&o);
  if (opts) o = *opts;
  if ((o.op != EQ_OP_DDO && o.op != EQ_OP_CDO) || (o.nyq != EQ_NYQ_KEEP && o.nyq != EQ_NYQ_ZERO) ||
      (o.target != EQ_TARGET_EQUILIBRIUM && o.target != EQ_TARGET_COMPATIBILITY) ||
      !(o.hx > 0.0) || !(o.hy > 0.0) || !(o.hz > 0.0))
    return sfail(EQ_ERR_INVALID, "eq_project_static: bad options");
  const long long V = (long long)nx * ny * nz;
  const size_t bytes = (size_t)6 * V * sizeof(float);
  const uintptr_t i0 = (uintptr_t)d_in, o0 = (uintptr_t)d_out;
  if (i0 != o0 && i0 < o0 + bytes && o0 < i0 + bytes)
    return sfail(EQ_ERR_INVALID, "eq_project_static: d_in and d_out overlap without being equal");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess || dev < 0 || dev >= 64)
    return sfail(EQ_ERR_CUDA, "eq_project_static: no current device");
  // set-up once per device and context, with that device current: the scratch array's device
  // address (looked up again when the current context is not the one it was taken in)
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticSlot& slot = g_static_slot[dev];
    const unsigned long long ctx = current_ctx_id();
    if (!slot.ptr || ctx == 0 || ctx != slot.ctx_id) {
      void* ptr = nullptr;
      if ((e = cudaGetSymbolAddress(&ptr, eq_static_scratch)) != cudaSuccess)
        return sfail(EQ_ERR_CUDA, std::string("eq_project_static: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e));
      slot.ptr = ptr;
      slot.ctx_id = current_ctx_id();   // the lookup made the device's context current
    }
    scratch = slot.ptr;
  }
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return sfail(EQ_ERR_CUDA, "eq_project_static: device attribute");
  eqk::PassInfo iz, iy, ix, iyi, izi;
  if ((e = eqk::pass_info_f32(nz, eqk::PASS_STRIDED_FWD, &iz)) != cudaSuccess ||
      (e = eqk::pass_info_f32(ny, eqk::PASS_STRIDED_FWD, &iy)) != cudaSuccess ||
      (e = eqk::pass_info_f32(nx, eqk::PASS_XPROJ, &ix)) != cudaSuccess ||
      (e = eqk::pass_info_f32(ny, eqk::PASS_STRIDED_INV, &iyi)) != cudaSuccess ||
      (e = eqk::pass_info_f32(nz, eqk::PASS_STRIDED_INV, &izi)) != cudaSuccess)
    return sfail(EQ_ERR_CUDA, std::string("eq_project_static: kernel attributes: ") + cudaGetErrorString(e));
  auto grid_for = [&](const eqk::PassInfo& inf, long long units, int split) {
    long long g = (long long)sms * (inf.blocks_per_sm > 0 ? inf.blocks_per_sm : 1);
    g = (g + split - 1) / split;
    return (int)(g < 1 ? 1 : (g > units ? units : g));
  };
  const int tpc_z = nz / (nz < 8 ? nz : 8), tpc_y = ny / (ny < 8 ? ny : 8), tpc_x = nx / (nx < 8 ? nx : 8);
  const int Bz = iz.threads / tpc_z, By = iy.threads / tpc_y, P = ix.threads / (6 * tpc_x);
  const long long tz = ((long long)nx * ny + Bz - 1) / Bz, ty = ((long long)nx * nz + By - 1) / By;
  // canonical x-pass rows: the self-mirror kz rows (0 and nz/2) keep ky <= ny/2, the rows with
  // 0 < kz < nz/2 keep every ky (powers of two)
  const int self_z = (nz > 1) ? 2 : 1;
  const int half_y = ny / 2 + 1 > ny ? ny : ny / 2 + 1;
  const int npairs = ((nz - self_z) / 2) * ny + self_z * half_y;
  const int g1 = grid_for(iz, tz, 3), gy = grid_for(iy, ty, 3), gl = grid_for(izi, tz, 3);
  const int gx = grid_for(ix, (npairs + P - 1) / P, 1);
  // carve the scratch array
  size_t cur = 0;
  auto take = [&](size_t n) { size_t at = cur; cur = align256(cur + n); return at; };
  const size_t o_tw = take(sizeof(float2) * (nx + ny + nz));
  const size_t o_xi = take(sizeof(float) * (nx + ny + nz));
  const size_t o_pairs = take(sizeof(int) * npairs);
  const size_t o_p1 = take(sizeof(double) * 3 * g1 * 4);
  const size_t o_px = take(sizeof(double) * gx * 4);
  const size_t o_pl = take(sizeof(double) * 3 * gl);
  const size_t o_mean = take(sizeof(double) * 6);
  const size_t o_is = take(sizeof(double) * 2);
  const size_t o_norm = take(sizeof(eq_norms_t));
  if (cur > EQ_STATIC_SCRATCH_BYTES)
    return sfail(EQ_ERR_INVALID, "eq_project_static: grid needs " + std::to_string(cur) +
                                     " scratch bytes, more than the static array holds");
  unsigned char* b = static_cast<unsigned char*>(scratch);
  float2* tw = reinterpret_cast<float2*>(b + o_tw);
  float* xi = reinterpret_cast<float*>(b + o_xi);
  int* pairs = reinterpret_cast<int*>(b + o_pairs);
  double* part1 = reinterpret_cast<double*>(b + o_p1);
  double* partx = reinterpret_cast<double*>(b + o_px);
  double* partl = reinterpret_cast<double*>(b + o_pl);
  double* mean = reinterpret_cast<double*>(b + o_mean);
  double* instats = reinterpret_cast<double*>(b + o_is);
  eq_norms_t* norms = d_norms ? d_norms : reinterpret_cast<eq_norms_t*>(b + o_norm);

  k_static_tables<<<8, 256, 0, s>>>(nx, ny, nz, (int)o.op, o.hx, o.hy, o.hz, tw, xi, pairs);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return sfail(EQ_ERR_CUDA, std::string("eq_project_static: tables: ") + cudaGetErrorString(e));
  const float2* twx = tw;
  const float2* twy = tw + nx;
  const float2* twz = tw + nx + ny;
  eqk::StridedArgs a{};
  a.field_stride = 6 * V;
  a.V = V;
  a.in = d_in; a.out = d_out; a.ref = nullptr; a.tw = twz;
  a.nstride = (long long)nx * ny; a.inner = a.nstride; a.outer_stride = 0; a.ncols = a.inner;
  a.ntiles = tz; a.partials = part1; a.mode = 1; a.ncomp = 3;
  if ((e = eqk::launch_strided_f32(nz, false, a, dim3(g1, 3), s)) != cudaSuccess)
    return sfail(EQ_ERR_CUDA, std::string("eq_project_static: z forward: ") + cudaGetErrorString(e));
  eqk::finalize_mean(part1, g1, 1, double(V), mean, instats, s);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return sfail(EQ_ERR_CUDA, std::string("eq_project_static: mean finalisation: ") +
                                  cudaGetErrorString(e));
  eqk::StridedArgs ay{};
  ay.field_stride = 6 * V; ay.V = V; ay.in = d_out; ay.out = d_out; ay.tw = twy;
  ay.nstride = nx; ay.inner = nx; ay.outer_stride = (long long)nx * ny; ay.ncols = (long long)nz * nx;
  ay.ntiles = ty; ay.mode = 0; ay.ncomp = 3;
  if ((e = eqk::launch_strided_f32(ny, false, ay, dim3(gy, 3), s)) != cudaSuccess)
    return sfail(EQ_ERR_CUDA, std::string("eq_project_static: y forward: ") + cudaGetErrorString(e));
  eqk::XArgs x{};
  x.data = d_out; x.tw = twx; x.xi_x = xi; x.xi_y = xi + nx; x.xi_z = xi + nx + ny;
  x.pairs = pairs; x.mean = mean; x.partials = partx; x.field_stride = 6 * V; x.V = V;
  x.nx = nx; x.ny = ny; x.nz = nz; x.npairs = npairs; x.ngroups = (npairs + P - 1) / P;
  x.nyq_zero = o.nyq == EQ_NYQ_ZERO; x.inv_v = 1.0 / double(V);
  x.compat = o.target == EQ_TARGET_COMPATIBILITY;
  if ((e = eqk::launch_xproj_f32(nx, x, dim3(gx, 1), s)) != cudaSuccess)
    return sfail(EQ_ERR_CUDA, std::string("eq_project_static: x pass: ") + cudaGetErrorString(e));
  if ((e = eqk::launch_strided_f32(ny, true, ay, dim3(gy, 3), s)) != cudaSuccess)
    return sfail(EQ_ERR_CUDA, std::string("eq_project_static: y inverse: ") + cudaGetErrorString(e));
  const bool linf = o.want_linf && d_in != d_out;
  eqk::StridedArgs az = a;
  az.in = d_out; az.ref = linf ? d_in : nullptr; az.partials = partl; az.mode = 2;
  if ((e = eqk::launch_strided_f32(nz, true, az, dim3(gl, 3), s)) != cudaSuccess)
    return sfail(EQ_ERR_CUDA, std::string("eq_project_static: z inverse: ") + cudaGetErrorString(e));
  eqk::finalize_norms(partx, gx, linf ? partl : nullptr, gl, 1, double(V), mean, instats,
                      linf ? 0 : EQ_FLAG_NO_LINF, norms, s);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return sfail(EQ_ERR_CUDA, std::string("eq_project_static: norms: ") + cudaGetErrorString(e));
  return EQ_OK;
}
