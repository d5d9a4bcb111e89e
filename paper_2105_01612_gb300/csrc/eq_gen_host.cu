// eq_gen_host.cu - plans of the runtime-length path: axis schedules, Bluestein tables, field
// descriptors, work-item prefix sums, launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <complex>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "eq_gen_host.h"

namespace eqg {

namespace {

bool factorize(int m, std::vector<int>& r) {
  r.clear();
  int x = m;
  while (x % 8 == 0) { r.push_back(8); x /= 8; }
  if (x % 4 == 0) { r.push_back(4); x /= 4; }
  if (x % 2 == 0) { r.push_back(2); x /= 2; }
  for (int p : {13, 11, 7, 5, 3})
    while (x % p == 0) { r.push_back(p); x /= p; }
  return x == 1;
}

constexpr int MAX_M = 1024;

}  // namespace

bool gen_length_supported(int n) {
  if (n < 1 || n > MAX_M) return false;
  std::vector<int> r;
  if (factorize(n, r)) return true;
  for (int m = 2 * n - 1; m <= MAX_M; ++m)
    if (factorize(m, r)) return true;
  return false;
}

// ---- finalisation: one block per field; each thread sums a fixed strided share of the
// field's partial records, then a fixed-shape tree (bitwise reproducible for a given launch).

constexpr int FIN_THREADS = 256;

template <int K>
__device__ __forceinline__ void fin_block_sum(double (&v)[K], double* red) {
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp * K + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < FIN_THREADS / 32; ++w) s += red[w * K + k];
      v[k] = s;
    }
}

__global__ void __launch_bounds__(FIN_THREADS)
k_gen_finalize_mean(const double* __restrict__ part, const long long* __restrict__ item0,
                    const FieldDesc* __restrict__ fields, int nf, double* __restrict__ mean,
                    double* __restrict__ instats) {
  __shared__ double red[(FIN_THREADS / 32) * 8];
  const int f = blockIdx.x;
  if (f >= nf) return;
  const long long i0 = item0[f], i1 = item0[f + 1];
  const long long per_comp = (i1 - i0) / 3;
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // sa, sb per component, sq, nonfinite
  for (int c = 0; c < 3; ++c) {
    const long long r0 = (i0 + c * per_comp) * WARPS_MAX, r1 = (i0 + (c + 1) * per_comp) * WARPS_MAX;
    for (long long r = r0 + threadIdx.x; r < r1; r += FIN_THREADS) {
      const double* p = part + r * 4;
      v[2 * c] += p[0];
      v[2 * c + 1] += p[1];
      v[6] += p[2];
      v[7] += p[3];
    }
  }
  fin_block_sum<8>(v, red);
  if (threadIdx.x == 0) {
    const double vol = double(fields[f].V);
    for (int j = 0; j < 6; ++j) mean[f * 6 + j] = v[j] / vol;
    instats[f * 2] = v[6];
    instats[f * 2 + 1] = v[7];
  }
}

__global__ void __launch_bounds__(FIN_THREADS)
k_gen_finalize_norms(const double* __restrict__ partx, const long long* __restrict__ itemx,
                     const double* __restrict__ partl, const long long* __restrict__ iteml,
                     const FieldDesc* __restrict__ fields, int nf, const double* __restrict__ mean,
                     const double* __restrict__ instats, int linf_flag, eq_norms_t* __restrict__ out) {
  __shared__ double red[(FIN_THREADS / 32) * 4];
  __shared__ double redm[FIN_THREADS / 32];
  const int f = blockIdx.x;
  if (f >= nf) return;
  double v[4] = {0, 0, 0, 0};   // resid^2, div_in^2, div_out^2, out^2 (spectral sums)
  for (long long r = itemx[f] * WARPS_MAX + threadIdx.x; r < itemx[f + 1] * WARPS_MAX; r += FIN_THREADS) {
    const double* p = partx + r * 4;
    v[0] += p[0]; v[1] += p[1]; v[2] += p[2]; v[3] += p[3];
  }
  double lm = 0.0;
  if (partl)
    for (long long r = iteml[f] * WARPS_MAX * 4 + threadIdx.x; r < iteml[f + 1] * WARPS_MAX * 4; r += FIN_THREADS)
      lm = fmax(lm, partl[r]);
  fin_block_sum<4>(v, red);
  for (int o = 16; o > 0; o >>= 1) lm = fmax(lm, __shfl_down_sync(0xffffffffu, lm, o));
  if ((threadIdx.x & 31) == 0) redm[threadIdx.x >> 5] = lm;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < FIN_THREADS / 32; ++w) lm = fmax(lm, redm[w]);
    const double vol = double(fields[f].V), v2 = vol * vol;
    eq_norms_t n;
    for (int j = 0; j < 6; ++j) n.mean[j] = mean[f * 6 + j];
    n.norm_in = sqrt(instats[f * 2] / vol);
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

// ---- plan ------------------------------------------------------------------------------

struct PassShape {
  int kind = 0;            // strided passes: 0 (k_gen_strided) or 4 (k_gen_scols / k_gen_scold),
                           // the inverse launching kind + 1; x pass: 2 (k_gen_xproj), 3
                           // (k_gen_xrows), 6 (k_gen_xpair) or 7 (k_gen_xdd)
  int cols = 16, pitch = 16, tpi = 1, threads = 256, mmax = 1, grid = 1;
  size_t smem = 0;
  long long nitems = 0;
  long long* item0 = nullptr;   // device [F + 1]
};

struct GenPlan {
  eq_dtype dtype = EQ_F32;
  eq_plan_opts opts{};
  int F = 0;
  int sms = 0;
  long long total_elems = 0;
  void* dmem = nullptr;
  size_t dbytes = 0;
  FieldDesc* fields = nullptr;
  AxisPlan* axes = nullptr;
  void* cpool = nullptr;
  void* xipool = nullptr;
  int* pairpool = nullptr;
  double* part_first = nullptr;
  double* part_x = nullptr;
  double* part_last = nullptr;
  double* mean = nullptr;
  double* instats = nullptr;
  eq_norms_t* norms = nullptr;
  int* err = nullptr;          // error word (bounds-checked builds raise it)
  PassShape z, y, x;
  std::vector<FieldDesc> fh;
  std::vector<AxisPlan> ah;
  int mx[3] = {1, 1, 1};       // largest transform length per axis (x, y, z)
  void* wmem = nullptr;        // work allocation: item prefix sums and partials
  size_t wbytes = 0;
  GenTune tune;
  std::string key;             // tuning-cache key
  int tw256 = -1, w512 = -1;   // complex-pool offsets of the paired-transform tables
  bool dd = false;             // FP64 plan in double-float arithmetic (tables, kernels, HBM pairs)
};

namespace {

template <typename T>
void push_complex(std::vector<unsigned char>& pool, std::complex<double> v) {
  T re = T(v.real()), im = T(v.imag());
  const unsigned char* a = reinterpret_cast<const unsigned char*>(&re);
  const unsigned char* b = reinterpret_cast<const unsigned char*>(&im);
  pool.insert(pool.end(), a, a + sizeof(T));
  pool.insert(pool.end(), b, b + sizeof(T));
}
template <typename T> void push_real(std::vector<unsigned char>& pool, double v) {
  T t = T(v);
  const unsigned char* a = reinterpret_cast<const unsigned char*>(&t);
  pool.insert(pool.end(), a, a + sizeof(T));
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// DFT_m(b) / m of the wrapped conjugate chirp, computed once per (n, m) in the process (a direct
// O(m^2) sum in FP64) and kept for later plans.
const std::vector<std::complex<double>>& chirp_transform(int n, int m,
                                                         const std::vector<std::complex<double>>& b) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, std::vector<std::complex<double>>> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find({n, m});
  if (it != cache.end()) return it->second;
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<std::complex<double>> w(m), out(m);
  for (int j = 0; j < m; ++j) w[j] = std::polar(1.0, -two_pi * double(j) / double(m));
  for (int k = 0; k < m; ++k) {
    std::complex<double> acc = 0.0;
    for (int d = 0; d < m; ++d) acc += b[d] * w[(long long)k * d % m];
    out[k] = acc / double(m);
  }
  return cache.emplace(std::make_pair(n, m), std::move(out)).first->second;
}

template <typename T>
void build_tables(GenPlan* g, const std::vector<int>& lens, std::vector<unsigned char>& cpool,
                  std::map<int, int>& axis_of_len) {
  const double two_pi = 6.283185307179586476925286766559, pi = two_pi / 2;
  std::map<int, int> tw_of_m;
  auto twiddles = [&](int m) {
    auto it = tw_of_m.find(m);
    if (it != tw_of_m.end()) return it->second;
    const int off = int(cpool.size() / (2 * sizeof(T)));
    for (int j = 0; j < m; ++j) push_complex<T>(cpool, std::polar(1.0, -two_pi * j / m));
    tw_of_m[m] = off;
    return off;
  };
  // staged twiddles W_{Ns R}^{r k} of the radix-8 schedule of a power-of-two length M (stages with
  // Ns > 1 in order, k < Ns, r = 1..R-1), as complex (cos, sin) entries
  std::map<int, int> staged_of_m;
  auto staged = [&](int M) {
    auto it = staged_of_m.find(M);
    if (it != staged_of_m.end()) return it->second;
    const int off = int(cpool.size() / (2 * sizeof(T)));
    int ns = 1, st = 0;
    while (ns < M) {
      const int R = eqk::stage_radix(M, st);
      if (ns > 1)
        for (int k = 0; k < ns; ++k)
          for (int r = 1; r < R; ++r)
            push_complex<T>(cpool, std::polar(1.0, -two_pi * double(r * k) / double(ns * R)));
      ns *= R;
      ++st;
    }
    staged_of_m[M] = off;
    return off;
  };
  for (int n : lens) {
    if (axis_of_len.count(n)) continue;
    AxisPlan ap{};
    std::vector<int> r;
    ap.n = n;
    if (factorize(n, r)) {
      ap.m = n;
      ap.blue = 0;
      ap.fast = (n >= 128 && n <= 1024 && (n & (n - 1)) == 0) ? 1 : 0;
    } else {
      // Bluestein: up to n = 256 a power-of-two length (served by the register FFT) although a
      // smooth length can be shorter; beyond, the smallest smooth length (shared memory)
      int m = 2 * n - 1;
      int p2 = 1;
      while (p2 < m) p2 <<= 1;
      if (p2 <= 512) {
        m = p2;
        factorize(m, r);
        ap.fast = 1;
      } else {
        while (!factorize(m, r)) ++m;
        ap.fast = 0;
      }
      ap.m = m;
      ap.blue = 1;
    }
    ap.nst = (int)r.size();
    for (int s = 0; s < ap.nst; ++s) ap.radix[s] = r[s];
    ap.tw = twiddles(ap.m);
    ap.chirp = ap.bhat = -1;
    if (ap.blue) {
      // chirp c_j = exp(-pi i j^2 / n) with j^2 reduced mod 2n; bhat = DFT_m(b) / m where
      // b_d = conj(c_d) for d in [0, n) and b_{m-d} = conj(c_d) for d in [1, n)
      std::vector<std::complex<double>> c(n), b(ap.m, 0.0);
      for (int j = 0; j < n; ++j) {
        const long long q = (long long)j * j % (2LL * n);
        c[j] = std::polar(1.0, -pi * double(q) / n);
      }
      for (int d = 0; d < n; ++d) {
        b[d] = std::conj(c[d]);
        if (d > 0) b[ap.m - d] = std::conj(c[d]);
      }
      ap.chirp = int(cpool.size() / (2 * sizeof(T)));
      for (int j = 0; j < n; ++j) push_complex<T>(cpool, c[j]);
      ap.bhat = int(cpool.size() / (2 * sizeof(T)));
      for (const std::complex<double>& v : chirp_transform(n, ap.m, b)) push_complex<T>(cpool, v);
    }
    // warp-per-row x pass: a power-of-two transform of 256 or 512 points in registers, directly
    // for n = 256, 512, else Bluestein with the power of two >= max(256, 2 n - 1)
    ap.wm = 0;
    ap.wchirp = ap.wbhat = ap.wtw = -1;
    if (n == 256 || n == 512) {
      ap.wm = n;
    } else {
      int p2 = 256;
      while (p2 < 2 * n - 1) p2 <<= 1;
      if (p2 <= 512) ap.wm = p2;
    }
    if (ap.wm) {
      ap.wtw = staged(ap.wm);
      if (ap.wm != n) {
        if (ap.blue && ap.m == ap.wm) {
          ap.wchirp = ap.chirp;
          ap.wbhat = ap.bhat;
        } else {
          std::vector<std::complex<double>> c(n), b(ap.wm, 0.0);
          for (int j = 0; j < n; ++j) {
            const long long q = (long long)j * j % (2LL * n);
            c[j] = std::polar(1.0, -pi * double(q) / n);
          }
          for (int d = 0; d < n; ++d) {
            b[d] = std::conj(c[d]);
            if (d > 0) b[ap.wm - d] = std::conj(c[d]);
          }
          ap.wchirp = int(cpool.size() / (2 * sizeof(T)));
          for (int j = 0; j < n; ++j) push_complex<T>(cpool, c[j]);
          ap.wbhat = int(cpool.size() / (2 * sizeof(T)));
          for (const std::complex<double>& v : chirp_transform(n, ap.wm, b)) push_complex<T>(cpool, v);
        }
      }
    }
    axis_of_len[n] = (int)g->ah.size();
    g->ah.push_back(ap);
  }
  // tables of the paired 256-point transforms of the warp-per-column strided kernel: staged
  // twiddles of length 256 and W512^j (j < 256), the twiddle of a 512-point transform's
  // even / odd split
  g->tw256 = staged(256);
  g->w512 = int(cpool.size() / (2 * sizeof(T)));
  for (int j = 0; j < 256; ++j) push_complex<T>(cpool, std::polar(1.0, -two_pi * j / 512.0));
}

template <typename T>
void xi_table(std::vector<unsigned char>& pool, int n, double h, eq_op op) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < n; ++m) {
    const int sf = (2 * m < n) ? m : m - n;
    double v;
    if (2 * m == n) v = 0.0;
    else if (op == EQ_OP_CDO) v = two_pi * double(sf) / (double(n) * h);
    else v = std::sin(two_pi * double(sf) / double(n)) / h;
    push_real<T>(pool, v);
  }
}

void canonical_pairs(int ny, int nz, std::vector<int>& out) {
  for (int kz = 0; kz < nz; ++kz) {
    const int mz = kz == 0 ? 0 : nz - kz;
    if (mz < kz) continue;
    for (int ky = 0; ky < ny; ++ky) {
      const int my = ky == 0 ? 0 : ny - ky;
      if (mz == kz && my < ky) continue;
      out.push_back(kz * ny + ky);
    }
  }
}

cudaError_t occupancy(const GenPlan* g, int kind, int threads, size_t smem, int* blocks) {
  if (g->dd) return gen_occupancy_dd(kind, threads, smem, blocks);
  return g->dtype == EQ_F32 ? gen_occupancy_f32(kind, threads, smem, blocks)
                            : gen_occupancy_f64(kind, threads, smem, blocks);
}

}  // namespace

eq_status gen_plan_create(const int* dims, int count, eq_dtype dtype, const eq_plan_opts& o,
                          int sms, GenPlan** out, std::string* err) {
  *out = nullptr;
  GenPlan* g = new (std::nothrow) GenPlan();
  if (!g) { *err = "host allocation failed"; return EQ_ERR_OOM; }
  g->dtype = dtype;
  g->opts = o;
  g->F = count;
  g->sms = sms;
  const size_t es = dtype == EQ_F32 ? 4 : 8;
  std::vector<int> lens;
  for (int i = 0; i < 3 * count; ++i) lens.push_back(dims[i]);
  std::vector<unsigned char> cpool, xipool;
  std::map<int, int> axis_of_len;
  // FP64 in double-float arithmetic where every length has a 256- or 512-point register
  // transform (512, or at most 256); EQ_F64_ARITH=native keeps FP64 instructions (measurements)
  if (dtype == EQ_F64) {
    const char* ar = getenv("EQ_F64_ARITH");
    bool ok = !(ar && std::string(ar) == "native");
    for (int n : lens) ok = ok && (n == 512 || n <= 256);
    g->dd = ok;
  }
  if (dtype == EQ_F32) build_tables<float>(g, lens, cpool, axis_of_len);
  else if (g->dd) build_tables<eqk::dd>(g, lens, cpool, axis_of_len);
  else build_tables<double>(g, lens, cpool, axis_of_len);
  std::map<std::pair<int, int>, int> xi_of;   // (axis, n) -> offset
  std::map<std::pair<int, int>, std::pair<int, int>> pairs_of;   // (ny, nz) -> (offset, count)
  std::vector<int> pairpool;
  const double hs[3] = {o.hx, o.hy, o.hz};
  long long off = 0;
  int mx[3] = {1, 1, 1};
  for (int f = 0; f < count; ++f) {
    FieldDesc fd{};
    fd.nx = dims[3 * f]; fd.ny = dims[3 * f + 1]; fd.nz = dims[3 * f + 2];
    fd.V = (long long)fd.nx * fd.ny * fd.nz;
    fd.in_off = fd.out_off = off;
    off += 6 * fd.V;
    const int n3[3] = {fd.nx, fd.ny, fd.nz};
    for (int a = 0; a < 3; ++a) {
      fd.ax[a] = axis_of_len[n3[a]];
      mx[a] = std::max(mx[a], g->ah[fd.ax[a]].m);
      auto key = std::make_pair(a, n3[a]);
      if (!xi_of.count(key)) {
        xi_of[key] = int(xipool.size() / es);
        if (dtype == EQ_F32) xi_table<float>(xipool, n3[a], hs[a], o.op);
        else if (g->dd) xi_table<eqk::dd>(xipool, n3[a], hs[a], o.op);
        else xi_table<double>(xipool, n3[a], hs[a], o.op);
      }
      fd.xi[a] = xi_of[key];
    }
    auto pk = std::make_pair(fd.ny, fd.nz);
    if (!pairs_of.count(pk)) {
      const int start = (int)pairpool.size();
      canonical_pairs(fd.ny, fd.nz, pairpool);
      pairs_of[pk] = {start, (int)pairpool.size() - start};
    }
    fd.pairs = pairs_of[pk].first;
    fd.npairs = pairs_of[pk].second;
    g->fh.push_back(fd);
  }
  g->total_elems = off;
  g->mx[0] = mx[0]; g->mx[1] = mx[1]; g->mx[2] = mx[2];
  {
    // tuning-cache key: sizes (FNV-1a of the dims list), dtype, options, GPU
    unsigned long long h = 1469598103934665603ULL;
    for (int i = 0; i < 3 * count; ++i) {
      h ^= (unsigned long long)dims[i];
      h *= 1099511628211ULL;
    }
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    std::string gpu = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "gpu";
    for (char& c : gpu) if (c == '"' || c == '\\') c = '_';
    char buf[512];
    snprintf(buf, sizeof(buf), "gen|%s|op%d|nyq%d|%.6g,%.6g,%.6g|n%d|%016llx|%s|%d",
             dtype == EQ_F32 ? "f32" : (g->dd ? "f64dd" : "f64"), (int)o.op, (int)o.nyq, o.hx, o.hy, o.hz, count, h,
             gpu.c_str(), sms);
    g->key = buf;
  }
  // tables: one device allocation
  size_t cur = 0;
  auto take = [&](size_t bytes) { size_t at = cur; cur = align_up(cur + bytes, 256); return at; };
  const size_t o_f = take(sizeof(FieldDesc) * count);
  const size_t o_a = take(sizeof(AxisPlan) * g->ah.size());
  const size_t o_c = take(cpool.size());
  const size_t o_xi = take(xipool.size());
  const size_t o_pp = take(sizeof(int) * std::max<size_t>(1, pairpool.size()));
  const size_t o_m = take(sizeof(double) * 6 * count);
  const size_t o_is = take(sizeof(double) * 2 * count);
  const size_t o_n = take(sizeof(eq_norms_t) * count);
  const size_t o_err = take(sizeof(int));
  g->dbytes = cur;
  cudaError_t e = cudaMalloc(&g->dmem, cur);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    delete g;
    return EQ_ERR_OOM;
  }
  unsigned char* b = static_cast<unsigned char*>(g->dmem);
  g->fields = reinterpret_cast<FieldDesc*>(b + o_f);
  g->axes = reinterpret_cast<AxisPlan*>(b + o_a);
  g->cpool = b + o_c;
  g->xipool = b + o_xi;
  g->pairpool = reinterpret_cast<int*>(b + o_pp);
  g->mean = reinterpret_cast<double*>(b + o_m);
  g->instats = reinterpret_cast<double*>(b + o_is);
  g->norms = reinterpret_cast<eq_norms_t*>(b + o_n);
  g->err = reinterpret_cast<int*>(b + o_err);
  if ((e = cudaMemset(g->err, 0, sizeof(int))) != cudaSuccess) {
    *err = std::string("error word: ") + cudaGetErrorString(e);
    gen_destroy(g);
    return EQ_ERR_CUDA;
  }
  struct Up { void* d; const void* h; size_t n; } ups[] = {
      {g->fields, g->fh.data(), sizeof(FieldDesc) * count},
      {g->axes, g->ah.data(), sizeof(AxisPlan) * g->ah.size()},
      {g->cpool, cpool.data(), cpool.size()},
      {g->xipool, xipool.data(), xipool.size()},
      {g->pairpool, pairpool.data(), sizeof(int) * pairpool.size()}};
  for (const Up& u : ups) {
    if (u.n == 0) continue;
    if ((e = cudaMemcpy(u.d, u.h, u.n, cudaMemcpyHostToDevice)) != cudaSuccess) {
      *err = std::string("table upload: ") + cudaGetErrorString(e);
      gen_destroy(g);
      return EQ_ERR_CUDA;
    }
  }
  // pass shapes: the tuning cache if it knows this plan, else the defaults
  GenTune t = gen_default_tune(g);
  eq_status st = EQ_ERR_INVALID;
  if (gen_cache_lookup(g, &t)) {
    std::string stale;
    st = gen_configure(g, t, &stale);                      // an entry that no longer fits is
    if (st != EQ_OK) t = gen_default_tune(g);              // passed over for the defaults
  }
  if (st != EQ_OK) st = gen_configure(g, t, err);
  if (st != EQ_OK) {
    gen_destroy(g);
    return st;
  }
  *out = g;
  return EQ_OK;
}

// Every field's x length is served by the warp-per-row x pass (a 256- or 512-point transform).
bool xrows_supported(const GenPlan* g) {
  for (const FieldDesc& fd : g->fh)
    if (g->ah[fd.ax[0]].wm == 0) return false;
  return true;
}

// An FP32 plan whose every field's length on this axis (1 = y, 2 = z) is served by the
// warp-per-column strided kernel (transform length wm of 256 or 512).
bool scols_supported(const GenPlan* g, int axis) {
  if (g->dtype != EQ_F32) return false;                   // the kernel is FP32
  for (const FieldDesc& fd : g->fh)
    if (g->ah[fd.ax[axis]].wm == 0) return false;
  return true;
}

GenTune gen_default_tune(const GenPlan* g) {
  const size_t es = g->dtype == EQ_F32 ? 4 : 8;
  GenTune t;
  t.zc = es == 4 ? (g->mx[2] > 256 ? 8 : 16) : (g->mx[2] > 256 ? 4 : 8);
  t.yc = es == 4 ? (g->mx[1] > 256 ? 8 : 16) : (g->mx[1] > 256 ? 4 : 8);
  if (scols_supported(g, 2) || g->dd) t.zc = 0;
  if (scols_supported(g, 1) || g->dd) t.yc = 0;
  t.zt = t.yt = 256;
  t.xp = xrows_supported(g) ? (es == 4 ? 4 : 0) : (g->mx[0] > 256 ? 1 : 2);
  if (g->dd) t.zt = t.yt = SD_THREADS;
  return t;
}

// Set the pass shapes (tile columns, threads, row pairs) and rebuild the work-item tables and
// the partial buffers for them.
eq_status gen_configure(GenPlan* g, const GenTune& t, std::string* err) {
  const size_t cs = g->dtype == EQ_F32 ? 8 : 16;
  const size_t limit = 227 * 1024;
  PassShape z = g->z, y = g->y, x = g->x;
  z.kind = 0; z.mmax = g->mx[2]; z.cols = t.zc; z.pitch = t.zc; z.threads = t.zt;
  y.kind = 0; y.mmax = g->mx[1]; y.cols = t.yc; y.pitch = t.yc; y.threads = t.yt;
  if (g->dd && (t.zc != 0 || t.yc != 0 || t.xp != 0)) {
    *err = "double-float plans run the warp-per-column strided and warp-per-row x kernels only";
    return EQ_ERR_INVALID;
  }
  for (int axis = 1; axis <= 2 && g->dd; ++axis) {
    PassShape& p = axis == 2 ? z : y;
    p.kind = 4; p.cols = SD_COLS; p.pitch = SD_PITCH; p.threads = SD_THREADS;
  }
  for (int axis = 1; axis <= 2 && !g->dd; ++axis) {
    PassShape& p = axis == 2 ? z : y;
    if ((axis == 2 ? t.zc : t.yc) != 0) continue;
    if (!scols_supported(g, axis)) {
      *err = "strided pass: the warp-per-column kernel serves lengths up to 256 and 512 only";
      return EQ_ERR_INVALID;
    }
    p.kind = 4; p.cols = 32; p.pitch = 33; p.threads = SC_THREADS;   // columns per field: scols_cols
  }
  if ((t.xp == 0 || t.xp == 4) && !xrows_supported(g)) {
    *err = "x pass: the warp-per-row kernels serve x lengths up to 256 and 512 only";
    return EQ_ERR_INVALID;
  }
  if (t.xp == 4 && g->dtype != EQ_F32) {
    *err = "x pass: the warp-per-plane-pair kernel is FP32";
    return EQ_ERR_INVALID;
  }
  if (t.xp < 0 || t.xp > 4) {
    *err = "x pass: unknown kernel choice";
    return EQ_ERR_INVALID;
  }
  if (t.xp == 0 && g->dd) {
    x.kind = 7; x.mmax = g->mx[0]; x.cols = 6; x.pitch = 0; x.threads = XD_THREADS;
  } else if (t.xp == 0) {
    x.kind = 3; x.mmax = g->mx[0]; x.cols = 6; x.pitch = 0; x.threads = XR_THREADS;
  } else if (t.xp == 4) {
    x.kind = 6; x.mmax = g->mx[0]; x.cols = 6; x.pitch = 0; x.threads = XQ_THREADS;
  } else {
    x.kind = 2; x.mmax = g->mx[0]; x.cols = 6 * t.xp; x.pitch = 6 * t.xp + 1; x.threads = 32 * x.cols;
  }
  PassShape* ps[3] = {&z, &y, &x};
  for (PassShape* p : ps) {
    p->smem = p->kind == 3   ? (g->dtype == EQ_F32 ? xrows_smem<float>()
                                : g->dd ? xrows_smem<eqk::dd>() : xrows_smem<double>())
              : p->kind == 4 ? (g->dd ? scold_smem<eqk::dd>() : scols_smem())
              : p->kind == 6 ? xpair_smem()
              : p->kind == 7 ? xdd_smem<eqk::dd>()
                             : (2 * (size_t)p->mmax * p->pitch + 3 * (size_t)p->mmax) * cs;
    if (p->smem > limit || p->threads > 512 || p->threads % p->cols != 0 || p->cols < 1) {
      *err = "pass shape does not fit (tile columns, threads or shared memory)";
      return EQ_ERR_INVALID;
    }
  }
  const int count = g->F;
  std::vector<long long> pre[3];
  for (int pi = 0; pi < 3; ++pi) {
    PassShape* p = ps[pi];
    int blocks = 0;
    cudaError_t e = occupancy(g, p->kind, p->threads, p->smem, &blocks);
    if (e == cudaSuccess && pi < 2) e = occupancy(g, p->kind + 1, p->threads, p->smem, &blocks);
    if (e != cudaSuccess || blocks < 1) {
      cudaGetLastError();
      *err = std::string("occupancy: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "0 blocks");
      return EQ_ERR_INVALID;
    }
    const long long resident = (long long)g->sms * blocks;
    long long total_tiles = 0;
    for (const FieldDesc& fd : g->fh) {
      if (pi == 2) total_tiles += (fd.npairs + (p->cols / 6) - 1) / (p->cols / 6);
      else {
        const long long ncols = pi == 0 ? (long long)fd.nx * fd.ny : (long long)fd.nz * fd.nx;
        const int cols = p->kind == 4 && !g->dd ? scols_cols(g->ah[fd.ax[pi == 0 ? 2 : 1]].n) : p->cols;
        total_tiles += 3 * ((ncols + cols - 1) / cols);
      }
    }
    p->tpi = (int)std::max(1LL, total_tiles / (8 * resident));
    pre[pi].assign(count + 1, 0);
    for (int f = 0; f < count; ++f) {
      const FieldDesc& fd = g->fh[f];
      long long items;
      if (pi == 2) {
        const long long groups = (fd.npairs + (p->cols / 6) - 1) / (p->cols / 6);
        items = (groups + p->tpi - 1) / p->tpi;
      } else {
        const long long ncols = pi == 0 ? (long long)fd.nx * fd.ny : (long long)fd.nz * fd.nx;
        const int cols = p->kind == 4 && !g->dd ? scols_cols(g->ah[fd.ax[pi == 0 ? 2 : 1]].n) : p->cols;
        const long long ntiles = (ncols + cols - 1) / cols;
        items = 3 * ((ntiles + p->tpi - 1) / p->tpi);
      }
      pre[pi][f + 1] = pre[pi][f] + items;
    }
    p->nitems = pre[pi][count];
    p->grid = (int)std::max(1LL, std::min(resident, p->nitems));
  }
  // work allocation: item prefix sums and per-warp partial records
  size_t cur = 0;
  auto take = [&](size_t bytes) { size_t at = cur; cur = align_up(cur + bytes, 256); return at; };
  const size_t o_iz = take(sizeof(long long) * (count + 1));
  const size_t o_iy = take(sizeof(long long) * (count + 1));
  const size_t o_ix = take(sizeof(long long) * (count + 1));
  const size_t o_pf = take(sizeof(double) * z.nitems * WARPS_MAX * 4);
  const size_t o_px = take(sizeof(double) * x.nitems * WARPS_MAX * 4);
  const size_t o_pl = take(sizeof(double) * z.nitems * WARPS_MAX * 4);
  if (cur > g->wbytes) {
    void* w = nullptr;
    cudaError_t e = cudaMalloc(&w, cur);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
      return EQ_ERR_OOM;
    }
    if (g->wmem) cudaFree(g->wmem);
    g->wmem = w;
    g->wbytes = cur;
  }
  unsigned char* b = static_cast<unsigned char*>(g->wmem);
  z.item0 = reinterpret_cast<long long*>(b + o_iz);
  y.item0 = reinterpret_cast<long long*>(b + o_iy);
  x.item0 = reinterpret_cast<long long*>(b + o_ix);
  cudaError_t e;
  if ((e = cudaMemcpy(z.item0, pre[0].data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(y.item0, pre[1].data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(x.item0, pre[2].data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice)) != cudaSuccess) {
    *err = std::string("item tables: ") + cudaGetErrorString(e);
    return EQ_ERR_CUDA;
  }
  g->part_first = reinterpret_cast<double*>(b + o_pf);
  g->part_x = reinterpret_cast<double*>(b + o_px);
  g->part_last = reinterpret_cast<double*>(b + o_pl);
  g->z = z; g->y = y; g->x = x;
  g->tune = t;
  return EQ_OK;
}

eq_status gen_enqueue(GenPlan* g, const void* d_in, void* d_out, cudaStream_t s, cudaEvent_t* ev,
                      std::string* err) {
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], s); };
  const bool f32 = g->dtype == EQ_F32;
  auto launch = [&](int kind, const GenArgs& a, const PassShape& p) {
    if (g->dd) return gen_launch_dd(kind, a, p.grid, p.threads, p.smem, s);
    return f32 ? gen_launch_f32(kind, a, p.grid, p.threads, p.smem, s)
               : gen_launch_f64(kind, a, p.grid, p.threads, p.smem, s);
  };
  GenArgs a{};
  a.fields = g->fields; a.axes = g->axes; a.cpool = g->cpool; a.xipool = g->xipool;
  a.pairpool = g->pairpool; a.mean = g->mean; a.nfields = g->F;
  a.nyq_zero = g->opts.nyq == EQ_NYQ_ZERO;
  a.err = g->err;
  a.tw256 = g->tw256; a.w512 = g->w512;
  a.compat = g->opts.target == EQ_TARGET_COMPATIBILITY;
  auto shape = [&](const PassShape& p) {
    a.item0 = p.item0; a.nitems = p.nitems; a.tiles_per_item = p.tpi; a.cols = p.cols;
    a.pitch = p.pitch; a.mmax = p.mmax;
  };
  cudaError_t e;
  mark(0);
  // z forward (d_in -> d_out) with input statistics
  shape(g->z);
  a.in = d_in; a.out = d_out; a.ref = nullptr; a.partials = g->part_first; a.axis = 2; a.mode = 1;
  a.io = g->dd ? 1 : 0;
  if ((e = launch(g->z.kind, a, g->z)) != cudaSuccess) { *err = std::string("z forward: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(1);
  k_gen_finalize_mean<<<g->F, FIN_THREADS, 0, s>>>(g->part_first, g->z.item0, g->fields, g->F,
                                                   g->mean, g->instats);
  if ((e = cudaGetLastError()) != cudaSuccess) { *err = std::string("mean: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(2);
  shape(g->y);
  a.in = d_out; a.partials = nullptr; a.axis = 1; a.mode = 0; a.io = 0;
  if ((e = launch(g->y.kind, a, g->y)) != cudaSuccess) { *err = std::string("y forward: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(3);
  shape(g->x);
  a.partials = g->part_x; a.mode = 0;
  if ((e = launch(g->x.kind, a, g->x)) != cudaSuccess) { *err = std::string("x pass: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(4);
  shape(g->y);
  a.partials = nullptr; a.axis = 1; a.mode = 0;
  if ((e = launch(g->y.kind + 1, a, g->y)) != cudaSuccess) { *err = std::string("y inverse: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(5);
  const bool linf = g->opts.want_linf && d_in != d_out;
  shape(g->z);
  a.ref = linf ? d_in : nullptr; a.partials = g->part_last; a.axis = 2; a.mode = linf ? 2 : 0;
  a.io = g->dd ? 2 : 0;
  if ((e = launch(g->z.kind + 1, a, g->z)) != cudaSuccess) { *err = std::string("z inverse: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(6);
  k_gen_finalize_norms<<<g->F, FIN_THREADS, 0, s>>>(
      g->part_x, g->x.item0, linf ? g->part_last : nullptr, g->z.item0, g->fields, g->F, g->mean,
      g->instats, linf ? 0 : EQ_FLAG_NO_LINF, g->norms);
  if ((e = cudaGetLastError()) != cudaSuccess) { *err = std::string("norms: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(7);
  return EQ_OK;
}

const eq_norms_t* gen_norms_device(const GenPlan* g) { return g->norms; }
int* gen_err_device(const GenPlan* g) { return g->err; }
GenTune gen_current_tune(const GenPlan* g) { return g->tune; }

// ---- tuning cache: a JSON object {"key": [zc, zt, yc, yt, xp], ...} in the file $EQ_TUNE_CACHE

namespace {

std::string read_file(const char* path) {
  std::ifstream f(path);
  if (!f) return "";
  std::stringstream ss;
  ss << f.rdbuf();
  return ss.str();
}

// entries of the cache file as (key, values) pairs
std::vector<std::pair<std::string, std::vector<int>>> parse_cache(const std::string& txt) {
  std::vector<std::pair<std::string, std::vector<int>>> out;
  size_t pos = 0;
  while (true) {
    const size_t q0 = txt.find('"', pos);
    if (q0 == std::string::npos) break;
    const size_t q1 = txt.find('"', q0 + 1);
    if (q1 == std::string::npos) break;
    const size_t b0 = txt.find('[', q1);
    const size_t b1 = txt.find(']', b0 == std::string::npos ? q1 : b0);
    if (b0 == std::string::npos || b1 == std::string::npos) break;
    std::vector<int> vals;
    std::stringstream ss(txt.substr(b0 + 1, b1 - b0 - 1));
    std::string tok;
    while (std::getline(ss, tok, ',')) vals.push_back(std::atoi(tok.c_str()));
    out.emplace_back(txt.substr(q0 + 1, q1 - q0 - 1), vals);
    pos = b1 + 1;
  }
  return out;
}

void cache_store(const GenPlan* g) {
  const char* path = getenv("EQ_TUNE_CACHE");
  if (!path || !*path) return;
  auto entries = parse_cache(read_file(path));
  const std::vector<int> v = {g->tune.zc, g->tune.zt, g->tune.yc, g->tune.yt, g->tune.xp};
  bool found = false;
  for (auto& e : entries)
    if (e.first == g->key) { e.second = v; found = true; }
  if (!found) entries.emplace_back(g->key, v);
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp);
    f << "{\n";
    for (size_t i = 0; i < entries.size(); ++i) {
      f << "  \"" << entries[i].first << "\": [";
      for (size_t k = 0; k < entries[i].second.size(); ++k) f << (k ? ", " : "") << entries[i].second[k];
      f << "]" << (i + 1 < entries.size() ? "," : "") << "\n";
    }
    f << "}\n";
  }
  std::rename(tmp.c_str(), path);
}

}  // namespace

bool gen_cache_lookup(const GenPlan* g, GenTune* t) {
  const char* path = getenv("EQ_TUNE_CACHE");
  if (!path || !*path) return false;
  for (const auto& e : parse_cache(read_file(path)))
    if (e.first == g->key && e.second.size() == 5) {
      t->zc = e.second[0]; t->zt = e.second[1]; t->yc = e.second[2]; t->yt = e.second[3];
      t->xp = e.second[4];
      return true;
    }
  return false;
}

// time one pass (z forward, y forward or x) with the current shapes; median of 3 runs, ms
static float time_pass(GenPlan* g, int which, const void* d_in, void* d_out, cudaStream_t s) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  GenArgs a{};
  a.fields = g->fields; a.axes = g->axes; a.cpool = g->cpool; a.xipool = g->xipool;
  a.pairpool = g->pairpool; a.mean = g->mean; a.nfields = g->F;
  a.nyq_zero = g->opts.nyq == EQ_NYQ_ZERO;
  a.err = g->err;
  a.tw256 = g->tw256; a.w512 = g->w512;
  a.compat = g->opts.target == EQ_TARGET_COMPATIBILITY;
  const PassShape& p = which == 0 ? g->z : (which == 1 ? g->y : g->x);
  a.item0 = p.item0; a.nitems = p.nitems; a.tiles_per_item = p.tpi; a.cols = p.cols;
  a.pitch = p.pitch; a.mmax = p.mmax;
  a.in = which == 0 ? d_in : d_out;
  a.out = d_out;
  a.axis = which == 0 ? 2 : 1;
  a.mode = which == 0 ? 1 : 0;
  a.partials = which == 0 ? g->part_first : (which == 2 ? g->part_x : nullptr);
  a.io = g->dd && which == 0 ? 1 : 0;
  const int kind = p.kind;
  float best[3];
  for (int r = 0; r < 4; ++r) {
    cudaEventRecord(e0, s);
    if (g->dd) gen_launch_dd(kind, a, p.grid, p.threads, p.smem, s);
    else if (g->dtype == EQ_F32) gen_launch_f32(kind, a, p.grid, p.threads, p.smem, s);
    else gen_launch_f64(kind, a, p.grid, p.threads, p.smem, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0) best[r - 1] = ms;              // first run warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::sort(best, best + 3);
  return best[1];
}

eq_status gen_autotune(GenPlan* g, const void* d_in, void* d_out, cudaStream_t s, std::string* err) {
  GenTune best = g->tune;
  const bool f32 = g->dtype == EQ_F32;
  const int cols[4] = {f32 ? 4 : 2, f32 ? 8 : 4, f32 ? 16 : 8, f32 ? 32 : 16};
  const int threads[3] = {128, 256, 512};
  for (int which = 0; which < 3; ++which) {
    float best_ms = 1e30f;
    GenTune keep = best;
    std::vector<GenTune> cands;
    if (which < 2) {
      for (int c : cols)
        for (int t : threads) {
          GenTune u = best;
          if (which == 0) { u.zc = c; u.zt = t; } else { u.yc = c; u.yt = t; }
          cands.push_back(u);
        }
      if (scols_supported(g, which == 0 ? 2 : 1)) {      // the warp-per-column kernel
        GenTune u = best;
        if (which == 0) { u.zc = 0; u.zt = SC_THREADS; } else { u.yc = 0; u.yt = SC_THREADS; }
        cands.push_back(u);
      }
    } else {
      for (int xp : {0, 1, 2, 3, 4}) {
        GenTune u = best;
        u.xp = xp;
        cands.push_back(u);
      }
    }
    for (const GenTune& u : cands) {
      std::string e2;
      if (gen_configure(g, u, &e2) != EQ_OK) continue;     // shape does not fit: skip
      const float ms = time_pass(g, which, d_in, d_out, s);
      if (cudaGetLastError() != cudaSuccess) continue;
      if (ms < best_ms) { best_ms = ms; keep = u; }
    }
    best = keep;
  }
  eq_status st = gen_configure(g, best, err);
  if (st != EQ_OK) return st;
  cache_store(g);
  return EQ_OK;
}
size_t gen_device_bytes(const GenPlan* g) { return g->dbytes + g->wbytes; }
bool gen_is_dd(const GenPlan* g) { return g->dd; }
long long gen_total_elems(const GenPlan* g) { return g->total_elems; }
int gen_count(const GenPlan* g) { return g->F; }

void gen_destroy(GenPlan* g) {
  if (!g) return;
  if (g->dmem) cudaFree(g->dmem);
  if (g->wmem) cudaFree(g->wmem);
  delete g;
}

}  // namespace eqg
