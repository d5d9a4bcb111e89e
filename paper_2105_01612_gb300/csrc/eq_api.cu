// eq_api.cu - plans and the C ABI entry points of include/eq.h (host runtime).
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cstdarg>
#include <cstdio>

#include <nvtx3/nvToolsExt.h>

#include "../../include/eq.h"
#include "eq_gen_host.h"
#include "eq_internal.h"

namespace {

thread_local std::string g_last_error;

// Host-side trace ranges (NVTX: no-ops unless a profiler is attached): one per call and one per
// pass launch, so that a timeline shows which call and pass each kernel belongs to.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

eq_status fail(eq_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}
eq_status fail_cuda(cudaError_t e, const char* where) {
  return fail(EQ_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

namespace eqk {
bool length_supported(int n) { return is_pow2(n) && n <= 1024; }
void set_last_error(const std::string& msg) { g_last_error = msg; }

// Diagnostics on stderr, by the level in the environment variable EQ_LOG (read once): 0 or unset
// silent, 1 plan decisions (kernel variants, grids, workspace), 2 also every call and every
// serving admission, completion and plan release.
int log_level() {
  static const int lv = [] {
    const char* e = getenv("EQ_LOG");
    return e && e[0] >= '0' && e[0] <= '9' ? e[0] - '0' : 0;
  }();
  return lv;
}
void log(int level, const char* fmt, ...) {
  if (log_level() < level) return;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  fprintf(stderr, "[eq] %s\n", buf);
}
}  // namespace eqk

// ---------------------------------------------------------------- finalisation kernels

// c0 and ||S_in||^2 per field from the first pass's block partials (fixed order, FP64).
// One block per field; each thread sums a fixed stride of the block partials in order, then a
// fixed shuffle/shared-memory tree: the result does not depend on timing.
__global__ void k_finalize_mean(const double* __restrict__ part, int grid, int batch, double vol,
                                double* __restrict__ mean, double* __restrict__ instats) {
  __shared__ double red[32 * 8];
  const int f = blockIdx.x;
  if (f >= batch) return;
  double v[8] = {};                                  // sa, sb of each component, sq, nonfinite
  for (int c = 0; c < 3; ++c) {
    const double* p = part + ((long long)(f * 3 + c) * grid) * 4;
    for (int g = threadIdx.x; g < grid; g += blockDim.x) {
      v[2 * c] += p[g * 4 + 0];
      v[2 * c + 1] += p[g * 4 + 1];
      v[6] += p[g * 4 + 2];
      v[7] += p[g * 4 + 3];
    }
  }
  eqk::block_sum<8>(v, red);
  if (threadIdx.x == 0) {
    for (int j = 0; j < 6; ++j) mean[f * 6 + j] = v[j] / vol;
    instats[f * 2 + 0] = v[6];
    instats[f * 2 + 1] = v[7];
  }
}

// eq_norms_t per field from the x-pass spectral sums (Parseval) and the last pass's L-inf.
__global__ void k_finalize_norms(const double* __restrict__ partx, int gridx,
                                 const double* __restrict__ partl, int gridl, int batch,
                                 double vol, const double* __restrict__ mean,
                                 const double* __restrict__ instats, int linf_flag,
                                 eq_norms_t* __restrict__ out) {
  __shared__ double red[32 * 4];
  const int f = blockIdx.x;
  if (f >= batch) return;
  double v[4] = {};                                  // r2, div in, div out, o2
  const double* p = partx + (long long)f * gridx * 4;
  for (int g = threadIdx.x; g < gridx; g += blockDim.x)
    for (int j = 0; j < 4; ++j) v[j] += p[g * 4 + j];
  eqk::block_sum<4>(v, red);
  double lm = 0.0;
  if (partl) {
    const double* q = partl + (long long)f * 3 * gridl;
    for (int g = threadIdx.x; g < 3 * gridl; g += blockDim.x) lm = fmax(lm, q[g]);
  }
  lm = eqk::block_max(lm, red);
  if (threadIdx.x == 0) {
    const double v2 = vol * vol;
    eq_norms_t n;
    for (int j = 0; j < 6; ++j) n.mean[j] = mean[f * 6 + j];
    n.norm_in = sqrt(instats[f * 2 + 0] / vol);
    n.norm_out = sqrt(v[3] / v2);
    n.resid_l2 = sqrt(v[0] / v2);
    n.resid_rel = n.norm_in > 0.0 ? n.resid_l2 / n.norm_in : 0.0;
    n.div_in_l2 = sqrt(v[1] / v2);
    n.div_out_l2 = sqrt(v[2] / v2);
    n.resid_linf = lm;
    n.flags = (instats[f * 2 + 1] > 0.0 ? EQ_FLAG_NONFINITE : 0) | linf_flag;
    out[f] = n;
  }
}

// The plan's norms and error flag into its mapped host mirror, last on the stream of every call:
// eq_norms then waits for the call's event and reads host memory, with no copy of its own that
// could queue behind another stream's transfers on a copy engine.
static_assert(sizeof(eq_norms_t) % 8 == 0, "eq_norms_t is copied as 8-byte words");
__global__ void k_publish(const eq_norms_t* __restrict__ src, int batch, const int* err,
                          eq_norms_t* hdst, int* herr) {
  const unsigned long long* a = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* b = reinterpret_cast<unsigned long long*>(hdst);
  const int words = batch * (int)(sizeof(eq_norms_t) / 8);
  for (int i = threadIdx.x; i < words; i += blockDim.x) b[i] = a[i];
  if (threadIdx.x == 0) *herr = err ? *err : 0;
}

// Failure-detection self-test: the bounded mbarrier wait of the TMA passes, on a barrier that no
// copy and no thread ever completes, with a short limit; when it runs out the kernel raises the
// plan's error flag exactly as a pass does, and returns.
__global__ void k_wait_selftest(int* err, long long polls) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    eqk::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !eqk::mbar_wait(&bar, 0u, polls)) atomicOr(err, 1);
}

// ---- non-periodic specimens in a zero-stress buffer (Sec. 5.2) ---------------------------------

constexpr int PAD_GRID = 1216;  // blocks per field of the crop pass (8 x 152 SMs)

// Copy the specimen planes (sx, sy, sz) into the corner of the grid planes (nx, ny, nz) and zero
// the rest.  One warp per grid row (plane, z, y), lanes along x, four loads in flight per lane.
template <typename T>
__global__ void __launch_bounds__(256)
k_pad(const T* __restrict__ in, T* __restrict__ out, int sx, int sy, int sz, int nx, int ny, int nz,
      long long rows) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = w0; r < rows; r += nw) {
    const long long pl = r / ((long long)ny * nz);
    const int zy = (int)(r - pl * ny * nz), z = zy / ny, y = zy - z * ny;
    T* o = out + r * nx;
    const int lim = (z < sz && y < sy) ? sx : 0;     // specimen columns of this row
    const T* src = in + ((pl * sz + z) * sy + y) * sx;
    for (int x0 = lane; x0 < nx; x0 += 128) {
      T v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int x = x0 + 32 * k;
        v[k] = x < lim ? src[x] : T(0);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (x0 + 32 * k < nx) o[x0 + 32 * k] = v[k];
    }
  }
}

// Cut the specimen region of the projected grid into out, and the largest |in - out| over it per
// block (grid (PAD_GRID, batch): warps of a field's blocks walk its 6 sz sy specimen rows, four
// loads of each kind in flight per lane).  `in` may equal `out`: each element is read before it
// is written, by the same thread.
template <typename T>
__global__ void __launch_bounds__(256)
k_crop_linf(const T* __restrict__ work, const T* in, T* out, int sx, int sy, int sz, int nx, int ny,
            int nz, double* __restrict__ partials) {
  __shared__ double red[32];
  const int f = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const long long rows = 6LL * sz * sy;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  T m = T(0);                 // in the working precision, as the last pass of eq_project
  for (long long r = w0; r < rows; r += nw) {
    const int pl = (int)(r / ((long long)sz * sy));
    const int zy = (int)(r - (long long)pl * sz * sy), z = zy / sy, y = zy - z * sy;
    const long long splane = (long long)f * 6 + pl;
    const T* wr = work + ((splane * nz + z) * ny + y) * nx;
    const long long so = ((splane * sz + z) * sy + y) * sx;
    for (int x0 = lane; x0 < sx; x0 += 128) {
      T v[4], ref[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int x = x0 + 32 * k;
        v[k] = x < sx ? wr[x] : T(0);
        ref[k] = x < sx ? in[so + x] : T(0);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int x = x0 + 32 * k;
        if (x < sx) {
          m = fmax(m, fabs(ref[k] - v[k]));
          out[so + x] = v[k];
        }
      }
    }
  }
  const double mb = eqk::block_max(double(m), red);
  if (threadIdx.x == 0) partials[(long long)f * gridDim.x + blockIdx.x] = mb;
}

// L-inf of each field into its norms (fixed order), clearing the no-L-inf flag of the in-place run
__global__ void k_pad_linf(const double* __restrict__ partials, int grid, int batch,
                           eq_norms_t* __restrict__ norms) {
  for (int f = threadIdx.x; f < batch; f += blockDim.x) {
    double m = 0.0;
    for (int g = 0; g < grid; ++g) m = fmax(m, partials[(long long)f * grid + g]);
    norms[f].resid_linf = m;
    norms[f].flags &= ~EQ_FLAG_NO_LINF;
  }
}

namespace eqk {
void finalize_mean(const double* part, int grid, int batch, double vol, double* mean,
                   double* instats, cudaStream_t s) {
  k_finalize_mean<<<batch, 256, 0, s>>>(part, grid, batch, vol, mean, instats);
}
void finalize_norms(const double* partx, int gridx, const double* partl, int gridl, int batch,
                    double vol, const double* mean, const double* instats, int linf_flag,
                    eq_norms_t* out, cudaStream_t s) {
  k_finalize_norms<<<batch, 256, 0, s>>>(partx, gridx, partl, gridl, batch, vol, mean, instats,
                                         linf_flag, out);
}
}  // namespace eqk

// ---------------------------------------------------------------- plan

struct eq_plan {
  int nx = 0, ny = 0, nz = 0, batch = 0;
  eq_dtype dtype = EQ_F32;
  eq_plan_opts opts{};
  long long V = 0;
  size_t esize = 4;
  int device = 0;
  int sms = 0;
  // device tables and reduction buffers (one allocation)
  void* dmem = nullptr;
  size_t dbytes = 0;
  void* tw[3] = {nullptr, nullptr, nullptr};   // x, y, z twiddles
  void* xi[3] = {nullptr, nullptr, nullptr};   // x, y, z operator symbols
  void* twst = nullptr;                        // per-stage x twiddles (cos table, sin table)
  int* pairs = nullptr;
  int npairs = 0;
  double* part1 = nullptr;     // [batch][3][g1][4]
  double* partx = nullptr;     // [batch][gx][4]
  double* partl = nullptr;     // [batch][3][gl]
  double* mean = nullptr;      // [batch][6]
  double* instats = nullptr;   // [batch][2]
  eq_norms_t* norms = nullptr; // [batch]
  int g1 = 1, gy = 1, gx = 1, gl = 1;
  eqk::PassInfo info_z_f, info_y_f, info_x, info_y_i, info_z_i;
  // TMA-fed strided passes (used when an instance exists and the x extent tiles evenly)
  eqk::TmaInfo tz, ty, tx;
  bool tma_allow = false;
  bool tma_z = false, tma_y = false, tma_x = false;
  bool avail_z = false, avail_y = false, avail_x = false;   // instances exist for these sizes
  int vz = 0, vy = 0, vx = 0;                               // shape variants in use
  int gtz = 1, gty = 1, gtx = 1, gtz_max = 1, gtx_max = 1;
  int* err = nullptr;          // raised by a kernel whose bounded wait ran out
  cudaEvent_t done = nullptr;
  // mapped pinned host mirror of the norms ([batch]) and of the error flag, written by k_publish
  void* mirror = nullptr;
  eq_norms_t* hnorms = nullptr;
  int* herr = nullptr;
  eq_norms_t* hnorms_dev = nullptr;   // the same memory as the device addresses it
  int* herr_dev = nullptr;
  bool have_result = false;
  // staging for eq_project_host
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // workspace of eq_project_padded: the padded fields, then one L-inf partial per block and field
  void* pad_ws = nullptr;
  double* pad_part = nullptr;
  // optional per-pass timing: one set of EQ_NUM_PASSES + 1 events per timed call
  std::vector<cudaEvent_t> tev;
  int tcap = 0, tused = 0;
  // runtime-length path (sizes other than powers of two, uneven batches); null = fast path
  eqg::GenPlan* gen = nullptr;
  // FP64 plans with every length 512 or at most 256: plain projections run the runtime-length
  // passes in double-float arithmetic (this sub-plan); the Hodge and padded forms keep the FP64
  // passes of this plan
  eqg::GenPlan* ddgen = nullptr;
  bool native_only = false;   // set while a padded projection runs: FP64 instructions throughout
  bool g_dd = false;          // the captured graph's passes were the double-float ones
  long long total_elems = 0;   // elements of one call's buffer (all fields, 6 planes)
  // captured CUDA graph of the passes for one (d_in, d_out) pair
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* g_in = nullptr;
  void* g_out = nullptr;
  void* g_y = nullptr;
  int g_spec[3] = {0, 0, 0};
};

namespace {

cudaError_t pass_info(eq_dtype dt, int n, eqk::PassKind k, eqk::PassInfo* out) {
  return dt == EQ_F32 ? eqk::pass_info_f32(n, k, out) : eqk::pass_info_f64(n, k, out);
}

template <typename T> void fill_tables(int n, double h, eq_op op, std::vector<unsigned char>& tw,
                                       std::vector<unsigned char>& xi) {
  using T2 = typename eqk::V2<T>::t;
  tw.resize(sizeof(T2) * n);
  xi.resize(sizeof(T) * n);
  T2* w = reinterpret_cast<T2*>(tw.data());
  T* s = reinterpret_cast<T*>(xi.data());
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < n; ++m) {
    const double ang = -two_pi * double(m) / double(n);
    w[m].x = T(std::cos(ang));
    w[m].y = T(std::sin(ang));
    // signed frequency; the Nyquist index of an even length gets symbol 0 (CDO and DDO)
    const int sf = (2 * m < n) ? m : m - n;
    double v;
    if (2 * m == n) v = 0.0;
    else if (op == EQ_OP_CDO) v = two_pi * double(sf) / (double(n) * h);
    else v = std::sin(two_pi * double(sf) / double(n)) / h;
    s[m] = T(v);
  }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Per-stage twiddles W_{Ns R}^{r k} (k < Ns, r = 1..R-1) of the power-of-two schedule of
// length n, stages with Ns > 1 in order, as a cos table followed by a sin table.
template <typename T> void staged_twiddles(int n, std::vector<unsigned char>& out) {
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<double> c, sn;
  int ns = 1, st = 0;
  while (ns < n) {
    const int R = eqk::stage_radix(n, st);
    if (ns > 1)
      for (int k = 0; k < ns; ++k)
        for (int r = 1; r < R; ++r) {
          const double ang = -two_pi * double(r * k) / double(ns * R);
          c.push_back(std::cos(ang));
          sn.push_back(std::sin(ang));
        }
    ns *= R;
    ++st;
  }
  // n = 512: the warp-per-row x pass factors 512 = 16 x 32 and takes W512^(l k1) as a table
  // [k1][l] (k1 < 16, l < 32) of complex values after the per-stage tables
  const size_t staged = sizeof(T) * 2 * std::max<size_t>(1, c.size());
  out.resize(staged + (n == 512 ? 2 * sizeof(T) * 512 : 0));   // (read by the FP32 instance)
  T* o = reinterpret_cast<T*>(out.data());
  for (size_t i = 0; i < c.size(); ++i) {
    o[i] = T(c[i]);
    o[c.size() + i] = T(sn[i]);
  }
  if (n == 512) {
    T* w = reinterpret_cast<T*>(out.data() + staged);
    for (int k1 = 0; k1 < 16; ++k1)
      for (int l = 0; l < 32; ++l) {
        const double ang = -two_pi * double(l * k1) / 512.0;
        w[2 * (k1 * 32 + l)] = T(std::cos(ang));
        w[2 * (k1 * 32 + l) + 1] = T(std::sin(ang));
      }
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiled>(f);
  }();
  return fn;
}

// 4-D view (x, y, z, plane) of a buffer of `planes` planes (6 per stress field, 4 per potential
// field); box of `cols` x values and `box` points along the transformed axis (2 = z, 1 = y).
// `spec` (nullable): the buffer holds specimen-sized planes (sx, sy, sz) instead of the plan's grid;
// a copy that reaches past them reads zeros and a store there is cut off.
bool make_map(CUtensorMap* m, const void* base, const eq_plan* p, int axis, int cols, int box,
              int planes, const int* spec = nullptr) {
  EncodeTiled enc = encode_fn();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  const cuuint64_t es = p->esize;
  const cuuint64_t dx = spec ? spec[0] : p->nx, dy = spec ? spec[1] : p->ny, dz = spec ? spec[2] : p->nz;
  if ((dx * es) % 16) return false;
  const cuuint64_t dims[4] = {dx, dy, dz, (cuuint64_t)planes};
  const cuuint64_t strides[3] = {dx * es, dx * dy * es, dx * dy * dz * es};
  const cuuint32_t boxd[4] = {(cuuint32_t)cols, axis == 1 ? (cuuint32_t)box : 1u,
                              axis == 2 ? (cuuint32_t)box : 1u, 1u};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, p->esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
             const_cast<void*>(base), dims, strides, boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Select shape variants for the TMA / bulk-copy passes and compute their grids (occupancy x SMs,
// split over fields and components, capped by the work).
void tma_setup(eq_plan* p, int vz, int vy, int vx) {
  p->vz = vz; p->vy = vy; p->vx = vx;
  p->tma_z = p->tma_y = p->tma_x = false;
  if (p->tma_allow) {
    const bool f32 = p->dtype == EQ_F32;
    // strided variant 2 exists for some lengths only: fall back to the wide tiles elsewhere
    auto strided = [&](int n, int& v, eqk::TmaInfo* ti) {
      cudaError_t te = f32 ? eqk::tma_info_f32(n, v, ti) : eqk::tma_info_f64(n, v, ti);
      if (te != cudaSuccess && v == 2) {
        cudaGetLastError();
        v = 0;
        te = f32 ? eqk::tma_info_f32(n, v, ti) : eqk::tma_info_f64(n, v, ti);
      }
      return te == cudaSuccess && ti->cols > 0 && p->nx % ti->cols == 0 && ti->blocks_per_sm > 0;
    };
    p->tma_z = strided(p->nz, p->vz, &p->tz);
    p->tma_y = strided(p->ny, p->vy, &p->ty);
    cudaError_t te;
    te = f32 ? eqk::xtma_info_f32(p->nx, vx, &p->tx) : eqk::xtma_info_f64(p->nx, vx, &p->tx);
    p->tma_x = te == cudaSuccess && p->tx.blocks_per_sm > 0;
    cudaGetLastError();
  }
  const long long b3 = 3LL * p->batch;
  p->gtz = p->tma_z ? (int)std::max(1LL, std::min<long long>((long long)p->sms * p->tz.blocks_per_sm / b3,
                                                             (long long)p->ny * (p->nx / p->tz.cols)))
                    : 1;
  p->gty = p->tma_y ? (int)std::max(1LL, std::min<long long>((long long)p->sms * p->ty.blocks_per_sm / b3,
                                                             (long long)p->nz * (p->nx / p->ty.cols)))
                    : 1;
  p->gtx = p->tma_x ? (int)std::max(1LL, std::min<long long>((long long)p->sms * p->tx.blocks_per_sm / p->batch,
                                                             (p->npairs + p->tx.cols - 1) / p->tx.cols))
                    : 1;
  p->avail_z = p->tma_z; p->avail_y = p->tma_y; p->avail_x = p->tma_x;
}

// TMA stores through the exchange buffer: measured faster for the z passes (the 16 x 32 kernel:
// both; the wide tiles: the last one) and slower for the y passes.  EQ_TMA_STORE overrides for
// measurements (0 never, 1 last z pass, 2 every z pass, 3 every pass).
bool tma_store_for(const eq_plan* p, int axis, int mode) {
  static const int ts = [] {
    const char* e = getenv("EQ_TMA_STORE");
    return e && e[0] >= '0' && e[0] <= '3' ? e[0] - '0' : -1;
  }();
  if (ts < 0) return axis == 2 && (p->vz == 2 || mode == 2);
  return ts == 3 || (axis == 2 && (ts == 2 || (ts == 1 && mode == 2)));
}

// Strided pass along `axis` through the TMA kernel; false if not applicable for these buffers.
// ncomp: complex fields per field of the buffers (3 for stress fields, 2 for the potential).
// spec (nullable): specimen size (sx, sy, sz) of the source (spec_src) and of the reference and
// destination (spec_dst) buffers, inside the plan's grid (eq_project_padded fused into the passes).
bool try_tma(eq_plan* p, bool on, int axis, bool inv, int mode, const void* src, void* dst,
             const void* ref, double* partials, cudaStream_t s, cudaError_t* e, int ncomp = 3,
             const int* spec = nullptr, bool spec_src = false, bool spec_dst = false) {
  if (!on) return false;
  const eqk::TmaInfo& ti = axis == 2 ? p->tz : p->ty;
  CUtensorMap map, refmap, outmap;
  const int planes = 2 * ncomp * p->batch;
  const int* ss = spec_src ? spec : nullptr;
  const int* sd = spec_dst ? spec : nullptr;
  if (!make_map(&map, src, p, axis, ti.cols, ti.box, planes, ss) ||
      (ref && !make_map(&refmap, ref, p, axis, ti.cols, ti.box, planes, sd)) ||
      (dst != src && !make_map(&outmap, dst, p, axis, ti.cols, ti.box, planes, sd))) {
    *e = cudaErrorInvalidValue;
    return true;
  }
  if (!ref) refmap = map;
  if (dst == src) outmap = map;
  eqk::TmaArgs t{};
  t.ref = ref; t.out = dst; t.tw = p->tw[axis]; t.partials = partials; t.err = p->err;
  t.field_stride = 2LL * ncomp * p->V; t.V = p->V;
  t.nx = p->nx; t.ny = p->ny; t.nz = p->nz;
  t.axis = axis; t.mode = mode; t.ncomp = ncomp;
  t.tma_store = tma_store_for(p, axis, mode);
  if (sd) {                                 // cut the stores and the residual to the specimen
    t.lim_x = sd[0]; t.lim_y = sd[1]; t.lim_z = sd[2];
    if (mode == 2) t.mode = 3;
    if (!t.tma_store) {                     // the per-thread stores do not cut
      *e = cudaErrorInvalidValue;
      return true;
    }
  }
  t.ntiles = (axis == 2 ? (long long)p->ny : (long long)p->nz) * (p->nx / ti.cols);
  // one resident wave over (field, component) pairs: the plan's grid is sized for three
  const long long g3 = axis == 2 ? p->gtz : p->gty;
  const long long gx = std::max(1LL, std::min<long long>(g3 * 3 / ncomp, t.ntiles));
  dim3 grid((unsigned)(ncomp == 3 ? g3 : gx), p->batch * ncomp);
  const int n = axis == 2 ? p->nz : p->ny;
  const int v = axis == 2 ? p->vz : p->vy;
  *e = p->dtype == EQ_F32 ? eqk::launch_tma_f32(n, v, inv, map, refmap, outmap, t, grid, s)
                          : eqk::launch_tma_f64(n, v, inv, map, refmap, outmap, t, grid, s);
  return true;
}

// d_y (nullable): also write the Hodge potential y into this 4-plane-per-field buffer (a
// potential x pass before the projector, then y and z inverse passes over the buffer).
// spec (nullable): d_in and d_final are specimens of (sx, sy, sz) inside the plan's grid
// (eq_project_padded): the first z pass reads d_in with zeros past its edges into the plan's
// padded workspace, the middle passes work there, and the last z pass writes the specimen region
// of the result into d_final.  Needs the TMA z passes with tiled stores (checked by the caller).
// Plain projections of FP64 plans with a double-float sub-plan run its passes.
bool use_dd(const eq_plan* p, const void* d_y, const int* spec) {
  return p->ddgen && !p->native_only && !d_y && !spec;
}

eq_status enqueue_passes(eq_plan* p, const void* d_in, void* d_final, cudaStream_t s, void* d_y,
                         const int* spec) {
  const bool f32 = p->dtype == EQ_F32;
  void* d_out = spec ? p->pad_ws : d_final;
  cudaEvent_t* ev = nullptr;
  if (p->tused < p->tcap) ev = &p->tev[(size_t)p->tused++ * (EQ_NUM_PASSES + 1)];
  if (p->gen || use_dd(p, d_y, spec)) {
    std::string err;
    eq_status st = eqg::gen_enqueue(p->gen ? p->gen : p->ddgen, d_in, d_out, s, ev, &err);
    if (st != EQ_OK) return fail(st, "eq_project: " + err);
    return EQ_OK;
  }
  static const char* kPassNames[EQ_NUM_PASSES] = {"eq z forward", "eq mean", "eq y forward",
                                                   "eq x project", "eq y inverse", "eq z inverse",
                                                   "eq norms"};
  int open_range = -1;
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev[i], s);
    if (open_range >= 0) nvtxRangePop();
    open_range = i < EQ_NUM_PASSES ? i : -1;
    if (open_range >= 0) nvtxRangePushA(kPassNames[i]);
  };
  struct CloseRange {
    int* r;
    ~CloseRange() { if (*r >= 0) nvtxRangePop(); }
  } close_range{&open_range};
  mark(0);
  // the TMA passes need 16-byte aligned buffers; decide once per call so the reductions and
  // their finalisation agree on the grid
  const bool aligned = !(reinterpret_cast<uintptr_t>(d_in) & 15) && !(reinterpret_cast<uintptr_t>(d_out) & 15) &&
                       !(reinterpret_cast<uintptr_t>(d_final) & 15);
  const bool on_z = p->tma_z && aligned, on_y = p->tma_y && aligned;
  const int gz_used = on_z ? p->gtz : p->g1, gl_used = on_z ? p->gtz : p->gl;
  const long long V = p->V;
  const long long fstride = 6 * V;
  cudaError_t e;
  // pass 1: z forward, d_in -> d_out, input statistics
  eqk::StridedArgs a{};
  a.field_stride = fstride;
  a.V = V;
  a.err = p->err;
  {
    a.in = d_in; a.out = d_out; a.ref = nullptr; a.tw = p->tw[2];
    a.nstride = (long long)p->ny * p->nx; a.inner = a.nstride; a.outer_stride = 0;
    a.ncols = a.inner;
    const int B = p->info_z_f.threads / std::max(1, p->nz / std::min(8, p->nz));
    a.ntiles = (a.ncols + B - 1) / B;
    a.partials = p->part1; a.mode = 1; a.ncomp = 3;
    dim3 grid(p->g1, p->batch * 3);
    if (spec) {
      if (!try_tma(p, on_z, 2, false, 1, d_in, d_out, nullptr, p->part1, s, &e, 3, spec, true, false))
        return fail(EQ_ERR_INVALID, "padded projection: the z passes need the TMA kernels");
    } else if (!try_tma(p, on_z, 2, false, 1, d_in, d_out, nullptr, p->part1, s, &e)) {
      e = f32 ? eqk::launch_strided_f32(p->nz, false, a, grid, s)
              : eqk::launch_strided_f64(p->nz, false, a, grid, s);
    }
    if (e != cudaSuccess) return fail_cuda(e, "z forward pass");
  }
  mark(1);
  k_finalize_mean<<<p->batch, 256, 0, s>>>(p->part1, gz_used, p->batch, double(V),
                                           p->mean, p->instats);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "mean finalisation");
  mark(2);
  // pass 2: y forward
  eqk::StridedArgs ay{};
  ay.field_stride = fstride; ay.V = V; ay.err = p->err;
  ay.in = d_out; ay.out = d_out; ay.ref = nullptr; ay.tw = p->tw[1];
  ay.nstride = p->nx; ay.inner = p->nx; ay.outer_stride = (long long)p->ny * p->nx;
  ay.ncols = (long long)p->nz * p->nx;
  {
    const int B = p->info_y_f.threads / std::max(1, p->ny / std::min(8, p->ny));
    ay.ntiles = (ay.ncols + B - 1) / B;
  }
  ay.partials = nullptr; ay.mode = 0; ay.ncomp = 3;
  {
    dim3 grid(p->gy, p->batch * 3);
    if (!try_tma(p, on_y, 1, false, 0, d_out, d_out, nullptr, nullptr, s, &e))
      e = f32 ? eqk::launch_strided_f32(p->ny, false, ay, grid, s)
              : eqk::launch_strided_f64(p->ny, false, ay, grid, s);
    if (e != cudaSuccess) return fail_cuda(e, "y forward pass");
  }
  mark(3);
  // potential x pass (reads the spectrum before the projector rewrites it): the warp-per-row
  // kernel when the x pass runs it and the buffers allow bulk copies, else the plain-load kernel
  const int pot_vx = p->vx;
  const bool pot_warp = d_y && p->tma_x && pot_vx >= 2 && pot_vx <= 8 &&
                        !(reinterpret_cast<uintptr_t>(d_out) & 15) &&
                        !(reinterpret_cast<uintptr_t>(d_y) & 15);
  if (pot_warp) {
    eqk::XTmaArgs x{};
    x.data = d_out; x.tws = p->twst;
    x.xi_x = p->xi[0]; x.xi_y = p->xi[1]; x.xi_z = p->xi[2];
    x.pairs = p->pairs; x.err = p->err;
    x.field_stride = fstride; x.V = V;
    x.nx = p->nx; x.ny = p->ny; x.nz = p->nz;
    x.npairs = p->npairs;
    x.ngroups = (p->npairs + p->tx.cols - 1) / p->tx.cols;
    x.inv_v = 1.0 / double(V);
    x.ydata = d_y; x.yfield_stride = 4 * V;
    dim3 grid(p->gtx, p->batch);
    e = f32 ? eqk::launch_xpot_warp_f32(p->nx, pot_vx, x, grid, s)
            : eqk::launch_xpot_warp_f64(p->nx, pot_vx, x, grid, s);
    if (e != cudaSuccess) return fail_cuda(e, "potential x pass");
  } else if (d_y) {
    eqk::XArgs x{};
    x.data = d_out; x.tw = p->tw[0]; x.err = p->err;
    x.xi_x = p->xi[0]; x.xi_y = p->xi[1]; x.xi_z = p->xi[2];
    x.pairs = p->pairs;
    x.field_stride = fstride; x.V = V;
    x.nx = p->nx; x.ny = p->ny; x.nz = p->nz;
    x.npairs = p->npairs;
    const int tpc = p->nx / std::min(8, p->nx);
    const int P = p->info_x.threads / (6 * tpc);
    x.ngroups = (p->npairs + P - 1) / P;
    x.inv_v = 1.0 / double(V);
    x.ydata = d_y; x.yfield_stride = 4 * V;
    dim3 grid(p->gx, p->batch);
    e = f32 ? eqk::launch_xpot_f32(p->nx, x, grid, s) : eqk::launch_xpot_f64(p->nx, x, grid, s);
    if (e != cudaSuccess) return fail_cuda(e, "potential x pass");
  }
  // pass 3: x forward + projector + x inverse
  const bool on_x = p->tma_x && !(reinterpret_cast<uintptr_t>(d_out) & 15);
  const int gx_used = on_x ? p->gtx : p->gx;
  if (on_x) {
    eqk::XTmaArgs x{};
    x.data = d_out; x.tws = p->twst;
    x.xi_x = p->xi[0]; x.xi_y = p->xi[1]; x.xi_z = p->xi[2];
    x.pairs = p->pairs; x.mean = p->mean; x.partials = p->partx; x.err = p->err;
    x.field_stride = fstride; x.V = V;
    x.nx = p->nx; x.ny = p->ny; x.nz = p->nz;
    x.npairs = p->npairs;
    x.ngroups = (p->npairs + p->tx.cols - 1) / p->tx.cols;
    x.nyq_zero = p->opts.nyq == EQ_NYQ_ZERO;
    x.compat = p->opts.target == EQ_TARGET_COMPATIBILITY;
    x.inv_v = 1.0 / double(V);
    dim3 grid(p->gtx, p->batch);
    e = f32 ? eqk::launch_xtma_f32(p->nx, p->vx, x, grid, s) : eqk::launch_xtma_f64(p->nx, p->vx, x, grid, s);
    if (e != cudaSuccess) return fail_cuda(e, "x projection pass");
  } else {
    eqk::XArgs x{};
    x.data = d_out; x.tw = p->tw[0]; x.err = p->err;
    x.xi_x = p->xi[0]; x.xi_y = p->xi[1]; x.xi_z = p->xi[2];
    x.pairs = p->pairs; x.mean = p->mean; x.partials = p->partx;
    x.field_stride = fstride; x.V = V;
    x.nx = p->nx; x.ny = p->ny; x.nz = p->nz;
    x.npairs = p->npairs;
    const int tpc = p->nx / std::min(8, p->nx);
    const int P = p->info_x.threads / (6 * tpc);
    x.ngroups = (p->npairs + P - 1) / P;
    x.nyq_zero = p->opts.nyq == EQ_NYQ_ZERO;
    x.compat = p->opts.target == EQ_TARGET_COMPATIBILITY;
    x.inv_v = 1.0 / double(V);
    dim3 grid(p->gx, p->batch);
    e = f32 ? eqk::launch_xproj_f32(p->nx, x, grid, s) : eqk::launch_xproj_f64(p->nx, x, grid, s);
    if (e != cudaSuccess) return fail_cuda(e, "x projection pass");
  }
  mark(4);
  const bool linf = p->opts.want_linf && d_in != d_out && d_in != d_final;
  // pass 4: y inverse
  {
    dim3 grid(p->gy, p->batch * 3);
    if (!try_tma(p, on_y, 1, true, 0, d_out, d_out, nullptr, nullptr, s, &e))
      e = f32 ? eqk::launch_strided_f32(p->ny, true, ay, grid, s)
              : eqk::launch_strided_f64(p->ny, true, ay, grid, s);
    if (e != cudaSuccess) return fail_cuda(e, "y inverse pass");
  }
  mark(5);
  // pass 5: z inverse (+ residual L-inf against d_in)
  {
    eqk::StridedArgs az = a;
    az.in = d_out; az.out = d_out; az.ref = linf ? d_in : nullptr;
    az.partials = p->partl; az.mode = 2;
    dim3 grid(p->gl, p->batch * 3);
    if (spec) {
      if (!try_tma(p, on_z, 2, true, 2, d_out, d_final, linf ? d_in : nullptr, p->partl, s, &e, 3,
                   spec, false, true))
        return fail(EQ_ERR_INVALID, "padded projection: the z passes need the TMA kernels");
    } else if (!try_tma(p, on_z, 2, true, 2, d_out, d_out, linf ? d_in : nullptr, p->partl, s, &e)) {
      e = f32 ? eqk::launch_strided_f32(p->nz, true, az, grid, s)
              : eqk::launch_strided_f64(p->nz, true, az, grid, s);
    }
    if (e != cudaSuccess) return fail_cuda(e, "z inverse pass");
  }
  // potential: y and z inverse over the y buffer (two complex fields per field), in place
  if (d_y) {
    const bool on_ypot = !(reinterpret_cast<uintptr_t>(d_y) & 15);
    eqk::StridedArgs py = ay;
    py.in = d_y; py.out = d_y; py.field_stride = 4 * V; py.ncomp = 2;
    if (!try_tma(p, p->tma_y && on_ypot, 1, true, 0, d_y, d_y, nullptr, nullptr, s, &e, 2))
      e = f32 ? eqk::launch_strided_f32(p->ny, true, py, dim3(p->gy, p->batch * 2), s)
              : eqk::launch_strided_f64(p->ny, true, py, dim3(p->gy, p->batch * 2), s);
    if (e != cudaSuccess) return fail_cuda(e, "potential y inverse pass");
    eqk::StridedArgs pz = a;
    pz.in = d_y; pz.out = d_y; pz.ref = nullptr; pz.partials = nullptr; pz.mode = 0;
    pz.field_stride = 4 * V; pz.ncomp = 2;
    if (!try_tma(p, p->tma_z && on_ypot, 2, true, 0, d_y, d_y, nullptr, nullptr, s, &e, 2))
      e = f32 ? eqk::launch_strided_f32(p->nz, true, pz, dim3(p->gl, p->batch * 2), s)
              : eqk::launch_strided_f64(p->nz, true, pz, dim3(p->gl, p->batch * 2), s);
    if (e != cudaSuccess) return fail_cuda(e, "potential z inverse pass");
  }
  mark(6);
  k_finalize_norms<<<p->batch, 256, 0, s>>>(p->partx, gx_used, linf ? p->partl : nullptr, gl_used,
                                            p->batch, double(V), p->mean, p->instats,
                                            linf ? 0 : EQ_FLAG_NO_LINF, p->norms);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "norm finalisation");
  mark(7);
  return EQ_OK;
}

// The norms of the last call (and the error flag) into the plan's host mirror.
eq_status publish(eq_plan* p, cudaStream_t s, bool dd = false) {
  const eq_norms_t* src = p->gen ? eqg::gen_norms_device(p->gen)
                                 : (dd ? eqg::gen_norms_device(p->ddgen) : p->norms);
  int* err = dd ? eqg::gen_err_device(p->ddgen) : p->err;
  k_publish<<<1, 128, 0, s>>>(src, p->batch, err, p->hnorms_dev, p->herr_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EQ_OK : fail_cuda(e, "norms publish");
}

// All passes of one projection, then the norms into the host mirror.
eq_status enqueue(eq_plan* p, const void* d_in, void* d_final, cudaStream_t s, void* d_y = nullptr,
                  const int* spec = nullptr) {
  eq_status st = enqueue_passes(p, d_in, d_final, s, d_y, spec);
  return st == EQ_OK ? publish(p, s, use_dd(p, d_y, spec)) : st;
}

// Mapped pinned memory for the host mirror of the norms and the error flag.
eq_status alloc_mirror(eq_plan* p) {
  const size_t nb = sizeof(eq_norms_t) * (size_t)p->batch;
  cudaError_t e = cudaHostAlloc(&p->mirror, nb + 64, cudaHostAllocMapped);
  if (e != cudaSuccess) {
    p->mirror = nullptr;
    return fail_cuda(e, "cudaHostAlloc (norms mirror)");
  }
  std::memset(p->mirror, 0, nb + 64);
  void* dev = nullptr;
  if ((e = cudaHostGetDevicePointer(&dev, p->mirror, 0)) != cudaSuccess)
    return fail_cuda(e, "cudaHostGetDevicePointer (norms mirror)");
  p->hnorms = static_cast<eq_norms_t*>(p->mirror);
  p->herr = reinterpret_cast<int*>(static_cast<unsigned char*>(p->mirror) + nb);
  p->hnorms_dev = static_cast<eq_norms_t*>(dev);
  p->herr_dev = reinterpret_cast<int*>(static_cast<unsigned char*>(dev) + nb);
  return EQ_OK;
}

// Enqueue one projection: replay the plan's captured CUDA graph when the buffers are the ones it
// was captured with (capturing it first if not), or launch the passes directly when timing.
eq_status run(eq_plan* p, const void* d_in, void* d_out, cudaStream_t s, void* d_y = nullptr,
              const int* spec = nullptr) {
  cudaError_t e;
  const bool timed = p->tused < p->tcap;
  const int sp[3] = {spec ? spec[0] : 0, spec ? spec[1] : 0, spec ? spec[2] : 0};
  if (p->opts.graph && !timed) {
    const bool dd = use_dd(p, d_y, spec);
    if (!p->gexec || p->g_in != d_in || p->g_out != d_out || p->g_y != d_y || p->g_dd != dd ||
        p->g_spec[0] != sp[0] || p->g_spec[1] != sp[1] || p->g_spec[2] != sp[2]) {
      if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
      if (!p->cap && (e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return fail_cuda(e, "capture stream");
      if ((e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return fail_cuda(e, "begin capture");
      eq_status st = enqueue(p, d_in, d_out, p->cap, d_y, spec);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(p->cap, &graph);
      if (st != EQ_OK) { if (graph) cudaGraphDestroy(graph); return st; }
      if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return fail_cuda(e, "end capture"); }
      e = cudaGraphInstantiate(&p->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) { p->gexec = nullptr; return fail_cuda(e, "graph instantiate"); }
      p->g_in = d_in;
      p->g_out = d_out;
      p->g_y = d_y;
      p->g_dd = dd;
      for (int i = 0; i < 3; ++i) p->g_spec[i] = sp[i];
    }
    if ((e = cudaGraphLaunch(p->gexec, s)) != cudaSuccess) return fail_cuda(e, "graph launch");
  } else {
    eq_status st = enqueue(p, d_in, d_out, s, d_y, spec);
    if (st != EQ_OK) return st;
  }
  if ((e = cudaEventRecord(p->done, s)) != cudaSuccess) return fail_cuda(e, "event record");
  p->have_result = true;
  return EQ_OK;
}

void release(eq_plan* p) {
  if (!p) return;
  for (cudaEvent_t e : p->tev) cudaEventDestroy(e);
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->done) cudaEventDestroy(p->done);
  if (p->mirror) cudaFreeHost(p->mirror);
  if (p->dmem) cudaFree(p->dmem);
  if (p->stage) cudaFree(p->stage);
  if (p->pad_ws) cudaFree(p->pad_ws);
  if (p->gen) eqg::gen_destroy(p->gen);
  if (p->ddgen) eqg::gen_destroy(p->ddgen);
  delete p;
}

}  // namespace

extern "C" {

void eq_plan_opts_default(eq_plan_opts* o) {
  if (!o) return;
  o->op = EQ_OP_DDO;
  o->hx = o->hy = o->hz = 1.0;
  o->nyq = EQ_NYQ_KEEP;
  o->want_linf = 1;
  o->graph = 1;
  o->target = EQ_TARGET_EQUILIBRIUM;
}

const char* eq_last_error(void) { return g_last_error.c_str(); }

static eq_status check_opts(const eq_plan_opts* opts, eq_plan_opts* o, const char* who) {
  eq_plan_opts_default(o);
  if (opts) *o = *opts;
  if (o->op != EQ_OP_DDO && o->op != EQ_OP_CDO) return fail(EQ_ERR_INVALID, std::string(who) + ": bad op");
  if (o->nyq != EQ_NYQ_KEEP && o->nyq != EQ_NYQ_ZERO)
    return fail(EQ_ERR_INVALID, std::string(who) + ": bad nyquist policy");
  if (o->target != EQ_TARGET_EQUILIBRIUM && o->target != EQ_TARGET_COMPATIBILITY)
    return fail(EQ_ERR_INVALID, std::string(who) + ": bad target");
  if (!(o->hx > 0.0) || !(o->hy > 0.0) || !(o->hz > 0.0) || !std::isfinite(o->hx) ||
      !std::isfinite(o->hy) || !std::isfinite(o->hz))
    return fail(EQ_ERR_INVALID, std::string(who) + ": spacing must be finite and > 0");
  return EQ_OK;
}

static eq_status create_generic(const int* dims, int count, eq_dtype dtype, const eq_plan_opts& o,
                                eq_plan** out) {
  eq_plan* p = new (std::nothrow) eq_plan();
  if (!p) return fail(EQ_ERR_OOM, "eq_plan_create: host allocation failed");
  p->dtype = dtype; p->opts = o; p->batch = count;
  p->nx = dims[0]; p->ny = dims[1]; p->nz = dims[2];
  p->esize = dtype == EQ_F32 ? 4 : 8;
  cudaError_t e;
  if ((e = cudaGetDevice(&p->device)) != cudaSuccess) { release(p); return fail_cuda(e, "cudaGetDevice"); }
  if ((e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess) {
    release(p);
    return fail_cuda(e, "cudaDeviceGetAttribute");
  }
  std::string err;
  eq_status st = eqg::gen_plan_create(dims, count, dtype, o, p->sms, &p->gen, &err);
  if (st != EQ_OK) { release(p); return fail(st, "eq_plan_create: " + err); }
  p->total_elems = eqg::gen_total_elems(p->gen);
  p->dbytes = eqg::gen_device_bytes(p->gen);
  p->err = eqg::gen_err_device(p->gen);
  if (alloc_mirror(p) != EQ_OK) {
    release(p);
    return EQ_ERR_CUDA;
  }
  if ((e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming)) != cudaSuccess) {
    release(p);
    return fail_cuda(e, "cudaEventCreate");
  }
  *out = p;
  return EQ_OK;
}

eq_status eq_plan_create(int nx, int ny, int nz, eq_dtype dtype, int batch,
                         const eq_plan_opts* opts, eq_plan** out) {
  if (!out) return fail(EQ_ERR_INVALID, "eq_plan_create: out is NULL");
  *out = nullptr;
  if (dtype != EQ_F32 && dtype != EQ_F64) return fail(EQ_ERR_INVALID, "eq_plan_create: bad dtype");
  if (batch < 1) return fail(EQ_ERR_INVALID, "eq_plan_create: batch must be >= 1");
  bool fast = true;
  for (int n : {nx, ny, nz}) {
    if (!eqg::gen_length_supported(n))
      return fail(EQ_ERR_INVALID, "eq_plan_create: axis length " + std::to_string(n) +
                                      " unsupported (1..1024; lengths with a prime factor above 13"
                                      " need 2n-1 <= 1024)");
    fast = fast && eqk::length_supported(n);
  }
  eq_plan_opts o;
  eq_status st = check_opts(opts, &o, "eq_plan_create");
  if (st != EQ_OK) return st;
  if (!fast) {
    std::vector<int> dims;
    for (int b = 0; b < batch; ++b) { dims.push_back(nx); dims.push_back(ny); dims.push_back(nz); }
    return create_generic(dims.data(), batch, dtype, o, out);
  }

  eq_plan* p = new (std::nothrow) eq_plan();
  if (!p) return fail(EQ_ERR_OOM, "eq_plan_create: host allocation failed");
  p->nx = nx; p->ny = ny; p->nz = nz; p->batch = batch; p->dtype = dtype; p->opts = o;
  p->V = (long long)nx * ny * nz;
  p->total_elems = (long long)batch * 6 * p->V;
  p->esize = dtype == EQ_F32 ? 4 : 8;
  cudaError_t e;
  if ((e = cudaGetDevice(&p->device)) != cudaSuccess) { release(p); return fail_cuda(e, "cudaGetDevice"); }
  if ((e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess) {
    release(p);
    return fail_cuda(e, "cudaDeviceGetAttribute");
  }
  if ((e = pass_info(dtype, nz, eqk::PASS_STRIDED_FWD, &p->info_z_f)) != cudaSuccess ||
      (e = pass_info(dtype, ny, eqk::PASS_STRIDED_FWD, &p->info_y_f)) != cudaSuccess ||
      (e = pass_info(dtype, nx, eqk::PASS_XPROJ, &p->info_x)) != cudaSuccess ||
      (e = pass_info(dtype, ny, eqk::PASS_STRIDED_INV, &p->info_y_i)) != cudaSuccess ||
      (e = pass_info(dtype, nz, eqk::PASS_STRIDED_INV, &p->info_z_i)) != cudaSuccess) {
    release(p);
    return fail_cuda(e, "kernel attributes");
  }
  // canonical row pairs of the x pass: rows (kz, ky) whose mirror (-kz, -ky) is not smaller
  std::vector<int> pairs;
  for (int kz = 0; kz < nz; ++kz) {
    const int mz = kz == 0 ? 0 : nz - kz;
    if (mz < kz) continue;
    for (int ky = 0; ky < ny; ++ky) {
      const int my = ky == 0 ? 0 : ny - ky;
      if (mz == kz && my < ky) continue;
      pairs.push_back(kz * ny + ky);
    }
  }
  p->npairs = (int)pairs.size();
  // grids: one resident wave, split over (field, component)
  auto grid_for = [&](const eqk::PassInfo& inf, long long units, int split) {
    long long g = (long long)p->sms * std::max(1, inf.blocks_per_sm);
    g = (g + split - 1) / split;
    g = std::max(1LL, std::min(g, units));
    return (int)g;
  };
  {
    const int Bz = p->info_z_f.threads / std::max(1, nz / std::min(8, nz));
    const int By = p->info_y_f.threads / std::max(1, ny / std::min(8, ny));
    const long long tz = ((long long)nx * ny + Bz - 1) / Bz;
    const long long ty = ((long long)nx * nz + By - 1) / By;
    const int tpc = nx / std::min(8, nx);
    const int P = p->info_x.threads / (6 * tpc);
    const long long gxn = (p->npairs + P - 1) / P;
    p->g1 = grid_for(p->info_z_f, tz, batch * 3);
    p->gy = grid_for(p->info_y_f, ty, batch * 3);
    p->gx = grid_for(p->info_x, gxn, batch);
    p->gl = grid_for(p->info_z_i, tz, batch * 3);
    // TMA / bulk-copy passes: shape variant 0 (wide tiles) unless overridden; grids sized for
    // both variants so that the autotuner can switch between them later
    const char* no_tma = getenv("EQ_NO_TMA");
    p->tma_allow = !(no_tma && no_tma[0] == '1') && encode_fn() != nullptr &&
                   ((size_t)nx * p->esize) % 16 == 0;
    int gmax_z = 1, gmax_x = 1;
    for (int v = 8; v >= 0; --v) {
      tma_setup(p, v <= 2 ? v : 0, v <= 2 ? v : 0, v);
      gmax_z = std::max(gmax_z, std::max(p->gtz, p->gty));
      gmax_x = std::max(gmax_x, p->gtx);
    }
    // defaults measured on GB300 at 256^3 and 512^3: the 16 x 32 column kernel for 512-point FP32
    // strided passes (z: with TMA stores), wide tiles for the others (eq_plan_autotune re-decides
    // per plan)
    const char* vs = getenv("EQ_TMA_VARIANT");
    const char* vxs = getenv("EQ_X_VARIANT");
    const char* vzs = getenv("EQ_TMA_VARIANT_Z");
    const int v0 = vs && vs[0] >= '0' && vs[0] <= '2' ? vs[0] - '0' : 2;
    const int vz0 = vzs && vzs[0] >= '0' && vzs[0] <= '2' ? vzs[0] - '0' : v0;
    // x pass: the packed two-row kernel with cp.async staging (8) where it exists (512-point
    // FP32 rows), else the warp-per-row kernel with direct loads (4), measured faster than the
    // bulk-copy staged forms (3, 2)
    const int vx0 = vxs && vxs[0] >= '0' && vxs[0] <= '8' ? vxs[0] - '0' : 8;
    tma_setup(p, vz0, v0, vx0);
    if (!p->tma_x && vx0 >= 7) tma_setup(p, vz0, v0, 4);
    for (int v = vx0 - 1; !p->tma_x && v >= 0; --v) tma_setup(p, vz0, v0, v);   // fall back
    p->gtz_max = gmax_z;
    p->gtx_max = gmax_x;
  }
  // tables
  std::vector<unsigned char> tw[3], xi[3];
  const int lens[3] = {nx, ny, nz};
  const double hs[3] = {o.hx, o.hy, o.hz};
  for (int a = 0; a < 3; ++a) {
    if (dtype == EQ_F32) fill_tables<float>(lens[a], hs[a], o.op, tw[a], xi[a]);
    else fill_tables<double>(lens[a], hs[a], o.op, tw[a], xi[a]);
  }
  std::vector<unsigned char> twst;
  if (dtype == EQ_F32) staged_twiddles<float>(nx, twst);
  else staged_twiddles<double>(nx, twst);
  size_t off = 0;
  size_t o_tw[3], o_xi[3];
  const size_t o_twst = off; off = align_up(off + twst.size(), 256);
  for (int a = 0; a < 3; ++a) { o_tw[a] = off; off = align_up(off + tw[a].size(), 256); }
  for (int a = 0; a < 3; ++a) { o_xi[a] = off; off = align_up(off + xi[a].size(), 256); }
  const size_t o_pairs = off; off = align_up(off + sizeof(int) * pairs.size(), 256);
  const size_t o_p1 = off; off = align_up(off + sizeof(double) * batch * 3 * std::max(p->g1, p->gtz_max) * 4, 256);
  const size_t o_px = off; off = align_up(off + sizeof(double) * batch * std::max(p->gx, p->gtx_max) * 4, 256);
  const size_t o_pl = off; off = align_up(off + sizeof(double) * batch * 3 * std::max(p->gl, p->gtz_max), 256);
  const size_t o_err = off; off = align_up(off + sizeof(int), 256);
  const size_t o_mean = off; off = align_up(off + sizeof(double) * batch * 6, 256);
  const size_t o_is = off; off = align_up(off + sizeof(double) * batch * 2, 256);
  const size_t o_nr = off; off = align_up(off + sizeof(eq_norms_t) * batch, 256);
  p->dbytes = off;
  if ((e = cudaMalloc(&p->dmem, off)) != cudaSuccess) {
    release(p);
    cudaGetLastError();
    return fail(EQ_ERR_OOM, std::string("eq_plan_create: cudaMalloc: ") + cudaGetErrorString(e));
  }
  unsigned char* base = static_cast<unsigned char*>(p->dmem);
  for (int a = 0; a < 3; ++a) {
    p->tw[a] = base + o_tw[a];
    p->xi[a] = base + o_xi[a];
    if ((e = cudaMemcpy(p->tw[a], tw[a].data(), tw[a].size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->xi[a], xi[a].data(), xi[a].size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
      release(p);
      return fail_cuda(e, "table upload");
    }
  }
  p->twst = base + o_twst;
  if ((e = cudaMemcpy(p->twst, twst.data(), twst.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    release(p);
    return fail_cuda(e, "twiddle upload");
  }
  p->pairs = reinterpret_cast<int*>(base + o_pairs);
  p->part1 = reinterpret_cast<double*>(base + o_p1);
  p->partx = reinterpret_cast<double*>(base + o_px);
  p->partl = reinterpret_cast<double*>(base + o_pl);
  p->mean = reinterpret_cast<double*>(base + o_mean);
  p->instats = reinterpret_cast<double*>(base + o_is);
  p->norms = reinterpret_cast<eq_norms_t*>(base + o_nr);
  p->err = reinterpret_cast<int*>(base + o_err);
  if ((e = cudaMemset(p->err, 0, sizeof(int))) != cudaSuccess) {
    release(p);
    return fail_cuda(e, "error flag");
  }
  if ((e = cudaMemcpy(p->pairs, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    release(p);
    return fail_cuda(e, "pair table upload");
  }
  if (alloc_mirror(p) != EQ_OK) {
    release(p);
    return EQ_ERR_CUDA;
  }
  if ((e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming)) != cudaSuccess) {
    release(p);
    return fail_cuda(e, "cudaEventCreate");
  }
  if (dtype == EQ_F64) {                 // the double-float sub-plan of plain projections
    std::vector<int> dims;
    for (int b = 0; b < batch; ++b) { dims.push_back(nx); dims.push_back(ny); dims.push_back(nz); }
    std::string err;
    eqg::GenPlan* g = nullptr;
    if (eqg::gen_plan_create(dims.data(), batch, dtype, o, p->sms, &g, &err) == EQ_OK) {
      if (eqg::gen_is_dd(g)) {
        p->ddgen = g;
        p->dbytes += eqg::gen_device_bytes(g);
      } else {
        eqg::gen_destroy(g);
      }
    } else {
      cudaGetLastError();
      eqk::log(1, "eq_plan_create: no double-float sub-plan (%s)", err.c_str());
    }
  }
  eqk::log(1, "eq_plan_create %dx%dx%d %s batch %d: z %s variant %d grid %d, y %s variant %d grid %d, "
              "x %s variant %d grid %d, %zu workspace bytes",
           nx, ny, nz, dtype == EQ_F32 ? "f32" : "f64", batch, p->tma_z ? "tma" : "plain", p->vz,
           p->tma_z ? p->gtz : p->g1, p->tma_y ? "tma" : "plain", p->vy, p->tma_y ? p->gty : p->gy,
           p->tma_x ? "fused" : "plain", p->vx, p->tma_x ? p->gtx : p->gx, p->dbytes);
  *out = p;
  return EQ_OK;
}

eq_status eq_plan_create_varlen(const int* dims, int count, eq_dtype dtype,
                                const eq_plan_opts* opts, eq_plan** out) {
  if (!out) return fail(EQ_ERR_INVALID, "eq_plan_create_varlen: out is NULL");
  *out = nullptr;
  if (!dims || count < 1) return fail(EQ_ERR_INVALID, "eq_plan_create_varlen: need dims and count >= 1");
  if (dtype != EQ_F32 && dtype != EQ_F64) return fail(EQ_ERR_INVALID, "eq_plan_create_varlen: bad dtype");
  for (int i = 0; i < 3 * count; ++i)
    if (!eqg::gen_length_supported(dims[i]))
      return fail(EQ_ERR_INVALID, "eq_plan_create_varlen: axis length " + std::to_string(dims[i]) +
                                      " unsupported");
  eq_plan_opts o;
  eq_status st = check_opts(opts, &o, "eq_plan_create_varlen");
  if (st != EQ_OK) return st;
  return create_generic(dims, count, dtype, o, out);
}

eq_status eq_project(eq_plan* p, const void* d_in, void* d_out, void* stream) {
  if (!p || !d_in || !d_out) return fail(EQ_ERR_INVALID, "eq_project: NULL argument");
  const size_t bytes = (size_t)p->total_elems * p->esize;
  const uintptr_t i0 = (uintptr_t)d_in, o0 = (uintptr_t)d_out;
  if (i0 != o0 && i0 < o0 + bytes && o0 < i0 + bytes)
    return fail(EQ_ERR_INVALID, "eq_project: d_in and d_out overlap without being equal");
  if ((i0 % p->esize) || (o0 % p->esize))
    return fail(EQ_ERR_INVALID, "eq_project: buffers not aligned to the element size");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return fail(EQ_ERR_INVALID, "eq_project: current device differs from the plan's");
  TraceRange tr("eq_project");
  eqk::log(2, "eq_project %dx%dx%d batch %d", p->nx, p->ny, p->nz, p->batch);
  return run(p, d_in, d_out, static_cast<cudaStream_t>(stream));
}

eq_status eq_project_hodge(eq_plan* p, const void* d_in, void* d_out, void* d_y, void* stream) {
  if (!p || !d_in || !d_out || !d_y) return fail(EQ_ERR_INVALID, "eq_project_hodge: NULL argument");
  if (p->gen)
    return fail(EQ_ERR_INVALID, "eq_project_hodge: needs a plan with power-of-two axis lengths");
  const size_t bytes = (size_t)p->total_elems * p->esize;
  const size_t ybytes = bytes / 6 * 4;
  const uintptr_t i0 = (uintptr_t)d_in, o0 = (uintptr_t)d_out, y0 = (uintptr_t)d_y;
  if (i0 != o0 && i0 < o0 + bytes && o0 < i0 + bytes)
    return fail(EQ_ERR_INVALID, "eq_project_hodge: d_in and d_out overlap without being equal");
  if ((y0 < i0 + bytes && i0 < y0 + ybytes) || (y0 < o0 + bytes && o0 < y0 + ybytes))
    return fail(EQ_ERR_INVALID, "eq_project_hodge: d_y overlaps d_in or d_out");
  if ((i0 % p->esize) || (o0 % p->esize) || (y0 % p->esize))
    return fail(EQ_ERR_INVALID, "eq_project_hodge: buffers not aligned to the element size");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return fail(EQ_ERR_INVALID, "eq_project_hodge: current device differs from the plan's");
  return run(p, d_in, d_out, static_cast<cudaStream_t>(stream), d_y);
}

eq_status eq_project_padded(eq_plan* p, int sx, int sy, int sz, const void* d_in, void* d_out,
                            void* stream) {
  if (!p || !d_in || !d_out) return fail(EQ_ERR_INVALID, "eq_project_padded: NULL argument");
  if (p->gen)
    return fail(EQ_ERR_INVALID, "eq_project_padded: needs a plan with power-of-two axis lengths");
  if (sx < 1 || sy < 1 || sz < 1 || sx > p->nx || sy > p->ny || sz > p->nz)
    return fail(EQ_ERR_INVALID, "eq_project_padded: the specimen must fit the plan's grid");
  const size_t sbytes = (size_t)p->batch * 6 * sx * sy * sz * p->esize;
  const uintptr_t i0 = (uintptr_t)d_in, o0 = (uintptr_t)d_out;
  if (i0 != o0 && i0 < o0 + sbytes && o0 < i0 + sbytes)
    return fail(EQ_ERR_INVALID, "eq_project_padded: d_in and d_out overlap without being equal");
  if ((i0 % p->esize) || (o0 % p->esize))
    return fail(EQ_ERR_INVALID, "eq_project_padded: buffers not aligned to the element size");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return fail(EQ_ERR_INVALID, "eq_project_padded: current device differs from the plan's");
  cudaError_t e;
  const size_t wbytes = (size_t)p->total_elems * p->esize;
  if (!p->pad_ws) {
    const size_t pbytes = sizeof(double) * (size_t)p->batch * PAD_GRID;
    if ((e = cudaMalloc(&p->pad_ws, wbytes + pbytes)) != cudaSuccess) {
      p->pad_ws = nullptr;
      cudaGetLastError();
      return fail(EQ_ERR_OOM, std::string("eq_project_padded: cudaMalloc: ") + cudaGetErrorString(e));
    }
    p->pad_part = reinterpret_cast<double*>(static_cast<unsigned char*>(p->pad_ws) + wbytes);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // fused: the first z pass reads the specimen (zeros past its edges, from the copy engine) and
  // the last z pass writes it back cut out, with no pass of its own for either.  Needs the TMA z
  // passes with tiled stores on 16-byte aligned specimen rows; EQ_PAD_UNFUSED=1 forces the
  // separate pad and cut kernels (for measurements).
  {
    const char* uf = getenv("EQ_PAD_UNFUSED");
    const bool fused = !(uf && uf[0] == '1') && p->tma_z && tma_store_for(p, 2, 2) &&
                       ((size_t)sx * p->esize) % 16 == 0 && !(i0 & 15) && !(o0 & 15);
    if (fused) {
      const int spec[3] = {sx, sy, sz};
      return run(p, d_in, d_out, s, nullptr, spec);
    }
  }
  const long long rows = 6LL * p->batch * p->nz * p->ny;
  const int pgrid = (int)std::min<long long>((rows + 7) / 8, (long long)p->sms * 8);
  if (p->dtype == EQ_F32)
    k_pad<float><<<pgrid, 256, 0, s>>>(static_cast<const float*>(d_in), static_cast<float*>(p->pad_ws),
                                        sx, sy, sz, p->nx, p->ny, p->nz, rows);
  else
    k_pad<double><<<pgrid, 256, 0, s>>>(static_cast<const double*>(d_in), static_cast<double*>(p->pad_ws),
                                         sx, sy, sz, p->nx, p->ny, p->nz, rows);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "eq_project_padded: pad");
  p->native_only = true;                 // padded projections: FP64 instructions in both forms
  eq_status st = run(p, p->pad_ws, p->pad_ws, s);
  p->native_only = false;
  if (st != EQ_OK) return st;
  dim3 cgrid(PAD_GRID, p->batch);
  if (p->dtype == EQ_F32)
    k_crop_linf<float><<<cgrid, 256, 0, s>>>(static_cast<const float*>(p->pad_ws),
                                              static_cast<const float*>(d_in), static_cast<float*>(d_out),
                                              sx, sy, sz, p->nx, p->ny, p->nz, p->pad_part);
  else
    k_crop_linf<double><<<cgrid, 256, 0, s>>>(static_cast<const double*>(p->pad_ws),
                                               static_cast<const double*>(d_in), static_cast<double*>(d_out),
                                               sx, sy, sz, p->nx, p->ny, p->nz, p->pad_part);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "eq_project_padded: crop");
  if (p->opts.want_linf) {
    k_pad_linf<<<1, 128, 0, s>>>(p->pad_part, PAD_GRID, p->batch, p->norms);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "eq_project_padded: L-inf");
    eq_status pst = publish(p, s);
    if (pst != EQ_OK) return pst;
  }
  // eq_norms waits for the last kernel of this call
  if ((e = cudaEventRecord(p->done, s)) != cudaSuccess) return fail_cuda(e, "event record");
  return EQ_OK;
}

eq_status eq_project_host_async(eq_plan* p, const void* h_in, void* h_out, void* stream) {
  if (!p || !h_in || !h_out) return fail(EQ_ERR_INVALID, "eq_project_host_async: NULL argument");
  const size_t bytes = (size_t)p->total_elems * p->esize;
  cudaError_t e;
  if (!p->stage) {
    if ((e = cudaMalloc(&p->stage, 2 * bytes)) != cudaSuccess) {
      p->stage = nullptr;
      cudaGetLastError();
      return fail(EQ_ERR_OOM, std::string("eq_project_host_async: cudaMalloc: ") + cudaGetErrorString(e));
    }
    p->stage_bytes = 2 * bytes;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* d_in = p->stage;
  void* d_out = static_cast<unsigned char*>(p->stage) + bytes;
  if ((e = cudaMemcpyAsync(d_in, h_in, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail_cuda(e, "eq_project_host_async: H2D");
  eq_status st = run(p, d_in, d_out, s);
  if (st != EQ_OK) return st;
  if ((e = cudaMemcpyAsync(h_out, d_out, bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail_cuda(e, "eq_project_host_async: D2H");
  // eq_norms (and the caller's stream) then cover the copy back as well
  if ((e = cudaEventRecord(p->done, s)) != cudaSuccess) return fail_cuda(e, "event record");
  return EQ_OK;
}

eq_status eq_project_host(eq_plan* p, const void* h_in, void* h_out, void* stream) {
  if (!p || !h_in || !h_out) return fail(EQ_ERR_INVALID, "eq_project_host: NULL argument");
  const size_t bytes = (size_t)p->total_elems * p->esize;
  cudaError_t e;
  if (!p->stage) {
    if ((e = cudaMalloc(&p->stage, 2 * bytes)) != cudaSuccess) {
      p->stage = nullptr;
      cudaGetLastError();
      return fail(EQ_ERR_OOM, std::string("eq_project_host: cudaMalloc: ") + cudaGetErrorString(e));
    }
    p->stage_bytes = 2 * bytes;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* d_in = p->stage;
  void* d_out = static_cast<unsigned char*>(p->stage) + bytes;
  if ((e = cudaMemcpyAsync(d_in, h_in, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail_cuda(e, "eq_project_host: H2D");
  eq_status st = run(p, d_in, d_out, s);
  if (st != EQ_OK) return st;
  if ((e = cudaMemcpyAsync(h_out, d_out, bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail_cuda(e, "eq_project_host: D2H");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_cuda(e, "eq_project_host: sync");
  return EQ_OK;
}

eq_status eq_norms(eq_plan* p, eq_norms_t* host_out) {
  if (!p || !host_out) return fail(EQ_ERR_INVALID, "eq_norms: NULL argument");
  if (!p->have_result) return fail(EQ_ERR_INVALID, "eq_norms: no projection enqueued yet");
  cudaError_t e;
  if ((e = cudaEventSynchronize(p->done)) != cudaSuccess) return fail_cuda(e, "eq_norms: wait");
  // the call's last kernel has written the host mirror
  volatile int* herr = p->herr;
  if (const int flags = *herr) {
    *herr = 0;
    if (p->err && (e = cudaMemset(p->err, 0, sizeof(int))) != cudaSuccess)
      return fail_cuda(e, "eq_norms: error flag");
    if (flags & EQ_ERRBIT_BOUNDS)
      return fail(EQ_ERR_CUDA, "eq_norms: an index out of range was caught (bounds-checked build); "
                               "results are invalid");
    return fail(EQ_ERR_TIMEOUT, "eq_norms: a bounded wait inside a kernel ran out; results are invalid");
  }
  std::memcpy(host_out, p->hnorms, sizeof(eq_norms_t) * p->batch);
  return EQ_OK;
}

eq_status eq_selftest_wait_timeout(eq_plan* p, long long polls, void* stream) {
  if (!p || polls < 1 || polls > (1LL << 24))
    return fail(EQ_ERR_INVALID, "eq_selftest_wait_timeout: NULL plan or polls outside 1..2^24");
  if (!p->err || p->gen)
    return fail(EQ_ERR_INVALID, "eq_selftest_wait_timeout: this plan's kernels have no bounded waits");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_wait_selftest<<<1, 32, 0, s>>>(p->err, polls);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(e, "eq_selftest_wait_timeout: launch");
  eq_status st = publish(p, s);
  if (st != EQ_OK) return st;
  if ((e = cudaEventRecord(p->done, s)) != cudaSuccess) return fail_cuda(e, "event record");
  p->have_result = true;
  return EQ_OK;
}

eq_status eq_plan_set_timing(eq_plan* p, int max_calls) {
  if (!p || max_calls < 0) return fail(EQ_ERR_INVALID, "eq_plan_set_timing: bad argument");
  const size_t need = (size_t)max_calls * (EQ_NUM_PASSES + 1);
  while (p->tev.size() < need) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return fail_cuda(err, "eq_plan_set_timing: cudaEventCreate");
    p->tev.push_back(e);
  }
  p->tcap = max_calls;
  p->tused = 0;
  return EQ_OK;
}

eq_status eq_plan_pass_ms(eq_plan* p, double* ms_out, int* ncalls_out) {
  if (!p || !ms_out) return fail(EQ_ERR_INVALID, "eq_plan_pass_ms: NULL argument");
  for (int i = 0; i < EQ_NUM_PASSES; ++i) ms_out[i] = 0.0;
  cudaError_t e;
  if (p->tused > 0) {
    cudaEvent_t last = p->tev[(size_t)(p->tused - 1) * (EQ_NUM_PASSES + 1) + EQ_NUM_PASSES];
    if ((e = cudaEventSynchronize(last)) != cudaSuccess) return fail_cuda(e, "eq_plan_pass_ms: wait");
  }
  for (int c = 0; c < p->tused; ++c) {
    cudaEvent_t* ev = &p->tev[(size_t)c * (EQ_NUM_PASSES + 1)];
    for (int i = 0; i < EQ_NUM_PASSES; ++i) {
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, ev[i], ev[i + 1])) != cudaSuccess)
        return fail_cuda(e, "eq_plan_pass_ms: elapsed");
      ms_out[i] += ms;
    }
  }
  if (ncalls_out) *ncalls_out = p->tused;
  p->tused = 0;
  p->tcap = 0;                         // timing off again: later calls replay the graph
  return EQ_OK;
}

// Per-pass times (ms) of the second of two direct runs with the plan's current choices.
eq_status time_passes(eq_plan* p, const void* d_in, void* d_out, cudaStream_t s, cudaEvent_t* ev,
                      float* ms) {
  for (int rep = 0; rep < 2; ++rep) {
    std::vector<cudaEvent_t> keep(p->tev);
    p->tev.assign(ev, ev + EQ_NUM_PASSES + 1);
    p->tcap = 1; p->tused = 0;
    eq_status st = enqueue(p, d_in, d_out, s);
    p->tev.swap(keep);
    if (st != EQ_OK) return st;
    cudaEventSynchronize(ev[EQ_NUM_PASSES]);
    for (int i = 0; i < EQ_NUM_PASSES; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  }
  return EQ_OK;
}

eq_status eq_plan_autotune(eq_plan* p, const void* d_in, void* d_out, void* stream) {
  if (!p || !d_in || !d_out) return fail(EQ_ERR_INVALID, "eq_plan_autotune: NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
  if (p->gen) {
    std::string err;
    eq_status st = eqg::gen_autotune(p->gen, d_in, d_out, s, &err);
    if (st != EQ_OK) return fail(st, "eq_plan_autotune: " + err);
    return EQ_OK;
  }
  // power-of-two plans: per pass, keep the fastest of the wide-tile TMA / bulk-copy variant, the
  // narrow-tile variant and the plain-load kernels (events between the passes, second of two runs)
  cudaEvent_t ev[EQ_NUM_PASSES + 1];
  for (auto& x : ev)
    if ((e = cudaEventCreate(&x)) != cudaSuccess) return fail_cuda(e, "eq_plan_autotune: events");
  constexpr int NCFG = 11;
  float ms[NCFG][EQ_NUM_PASSES] = {};
  bool ok[NCFG][3] = {};                                // [config][axis z, y, x] available
  const int saved_cap = p->tcap, saved_used = p->tused;
  // the variants are those of this plan's own passes (an FP64 plan's double-float sub-plan, which
  // runs its plain projections, has none to choose): time them
  p->native_only = true;
  struct Restore {
    eq_plan* p;
    ~Restore() { p->native_only = false; }
  } restore{p};
  // configs: 0 wide tiles, 1 narrow tiles, 2 plain kernels, 3 and 4 warp-per-row x pass through
  // a bulk-copy stage (three and four blocks per SM asked of the register allocator), 5 the 16 x 32
  // strided kernel (where it exists; its config counts for an axis only if the axis really ran
  // it), 6 and 7 the warp-per-row x pass with direct loads and stores (four and five blocks),
  // 8 the same with the next row pair's loads issued early (three blocks), 9 the packed two-row
  // x pass (512-point FP32 rows), 10 the same with the next rows staged by cp.async
  auto xvar = [](int cfg) {
    return cfg == 1 ? 1 : (cfg == 3 ? 2 : (cfg == 4 ? 3 : (cfg >= 6 ? cfg - 2 : 0)));
  };
  auto svar = [](int cfg) { return cfg == 1 ? 1 : (cfg == 5 ? 2 : 0); };
  for (int cfg = 0; cfg < NCFG; ++cfg) {
    tma_setup(p, svar(cfg), svar(cfg), xvar(cfg));
    if (cfg == 2) p->tma_z = p->tma_y = p->tma_x = false;
    if (cfg == 3 || cfg == 4 || cfg >= 6) p->tma_z = p->tma_y = false;
    if (cfg == 5) {
      p->tma_x = false;
      if (p->vz != 2) p->tma_z = false;
      if (p->vy != 2) p->tma_y = false;
    }
    ok[cfg][0] = cfg == 2 || p->tma_z;
    ok[cfg][1] = cfg == 2 || p->tma_y;
    ok[cfg][2] = cfg == 2 || p->tma_x;
    const eq_status st = time_passes(p, d_in, d_out, s, ev, ms[cfg]);
    if (st != EQ_OK) {
      p->tcap = saved_cap; p->tused = saved_used;
      for (auto& x : ev) cudaEventDestroy(x);
      return st;
    }
  }
  // pass indices: 0 z forward, 2 y forward, 3 x, 4 y inverse, 5 z inverse
  auto pick = [&](int axis, int ncfg, float (*cost)(const float*)) {
    int best = 2;
    for (int c = 0; c < ncfg; ++c)
      if (c != 2 && ok[c][axis] && cost(ms[c]) < cost(ms[best])) best = c;
    return best;
  };
  const int bz = pick(0, NCFG, [](const float* m) { return m[0] + m[5]; });
  const int by = pick(1, NCFG, [](const float* m) { return m[2] + m[4]; });
  const int bx = pick(2, NCFG, [](const float* m) { return m[3]; });
  tma_setup(p, svar(bz), svar(by), xvar(bx));
  if (bz == 2) p->tma_z = false;
  if (by == 2) p->tma_y = false;
  if (bx == 2) p->tma_x = false;
  p->tcap = saved_cap; p->tused = saved_used;
  for (auto& x : ev) cudaEventDestroy(x);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "eq_plan_autotune");
  return EQ_OK;
}

size_t eq_plan_workspace_bytes(const eq_plan* p) { return p ? p->dbytes + p->stage_bytes : 0; }

void eq_plan_destroy(eq_plan* p) {
  if (!p) return;
  if (p->done) cudaEventSynchronize(p->done);
  release(p);
}

}  // extern "C"
