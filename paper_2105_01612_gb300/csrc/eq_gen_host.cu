// eq_gen_host.cu - plans of the runtime-length path: axis schedules, Bluestein tables, field
// descriptors, work-item prefix sums, launches.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
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

// ---- finalisation (one thread per field, fixed order) -------------------------------------

__global__ void k_gen_finalize_mean(const double* __restrict__ part, const long long* __restrict__ item0,
                                    const FieldDesc* __restrict__ fields, int nf,
                                    double* __restrict__ mean, double* __restrict__ instats) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const long long i0 = item0[f], i1 = item0[f + 1];
    const long long per_comp = (i1 - i0) / 3;
    double sq = 0.0, nfin = 0.0;
    for (int c = 0; c < 3; ++c) {
      double sa = 0.0, sb = 0.0;
      for (long long it = i0 + c * per_comp; it < i0 + (c + 1) * per_comp; ++it)
        for (int w = 0; w < WARPS_MAX; ++w) {
          const double* p = part + (it * WARPS_MAX + w) * 4;
          sa += p[0]; sb += p[1]; sq += p[2]; nfin += p[3];
        }
      const double vol = double(fields[f].V);
      mean[f * 6 + 2 * c] = sa / vol;
      mean[f * 6 + 2 * c + 1] = sb / vol;
    }
    instats[f * 2] = sq;
    instats[f * 2 + 1] = nfin;
  }
}

__global__ void k_gen_finalize_norms(const double* __restrict__ partx, const long long* __restrict__ itemx,
                                     const double* __restrict__ partl, const long long* __restrict__ iteml,
                                     const FieldDesc* __restrict__ fields, int nf,
                                     const double* __restrict__ mean, const double* __restrict__ instats,
                                     int linf_flag, eq_norms_t* __restrict__ out) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    double r2 = 0.0, di = 0.0, dout = 0.0, o2 = 0.0;
    for (long long it = itemx[f]; it < itemx[f + 1]; ++it)
      for (int w = 0; w < WARPS_MAX; ++w) {
        const double* p = partx + (it * WARPS_MAX + w) * 4;
        r2 += p[0]; di += p[1]; dout += p[2]; o2 += p[3];
      }
    const double vol = double(fields[f].V), v2 = vol * vol;
    eq_norms_t n;
    for (int j = 0; j < 6; ++j) n.mean[j] = mean[f * 6 + j];
    n.norm_in = sqrt(instats[f * 2] / vol);
    n.norm_out = sqrt(o2 / v2);
    n.resid_l2 = sqrt(r2 / v2);
    n.resid_rel = n.norm_in > 0.0 ? n.resid_l2 / n.norm_in : 0.0;
    n.div_in_l2 = sqrt(di / v2);
    n.div_out_l2 = sqrt(dout / v2);
    double lm = 0.0;
    if (partl)
      for (long long it = iteml[f]; it < iteml[f + 1]; ++it)
        for (int w = 0; w < WARPS_MAX * 4; ++w) lm = fmax(lm, partl[it * WARPS_MAX * 4 + w]);
    n.resid_linf = lm;
    n.flags = (instats[f * 2 + 1] > 0.0 ? EQ_FLAG_NONFINITE : 0) | linf_flag;
    out[f] = n;
  }
}

// ---- plan ------------------------------------------------------------------------------

struct PassShape {
  int kind = 0;            // 0 strided fwd, 1 strided inv, 2 x
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
  PassShape z, y, x;
  std::vector<FieldDesc> fh;
  std::vector<AxisPlan> ah;
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
  for (int n : lens) {
    if (axis_of_len.count(n)) continue;
    AxisPlan ap{};
    std::vector<int> r;
    ap.n = n;
    if (factorize(n, r)) {
      ap.m = n;
      ap.blue = 0;
    } else {
      int m = 2 * n - 1;
      while (!factorize(m, r)) ++m;
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
      for (int k = 0; k < ap.m; ++k) {
        std::complex<double> acc = 0.0;
        for (int d = 0; d < ap.m; ++d)
          acc += b[d] * std::polar(1.0, -two_pi * double((long long)k * d % ap.m) / ap.m);
        push_complex<T>(cpool, acc / double(ap.m));
      }
    }
    axis_of_len[n] = (int)g->ah.size();
    g->ah.push_back(ap);
  }
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

cudaError_t occupancy(eq_dtype dt, int kind, int threads, size_t smem, int* blocks) {
  return dt == EQ_F32 ? gen_occupancy_f32(kind, threads, smem, blocks)
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
  const size_t es = dtype == EQ_F32 ? 4 : 8, cs = 2 * es;
  std::vector<int> lens;
  for (int i = 0; i < 3 * count; ++i) lens.push_back(dims[i]);
  std::vector<unsigned char> cpool, xipool;
  std::map<int, int> axis_of_len;
  if (dtype == EQ_F32) build_tables<float>(g, lens, cpool, axis_of_len);
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
  // pass shapes
  const size_t budget = 200 * 1024;
  auto strided_cols = [&](int m) {
    int C = es == 4 ? 16 : 8;
    while (C > 1 && 2 * (size_t)m * C * cs > budget) C /= 2;
    return C;
  };
  PassShape* ps[3] = {&g->z, &g->y, &g->x};
  g->z.kind = 0; g->z.mmax = mx[2];
  g->y.kind = 0; g->y.mmax = mx[1];
  g->x.kind = 2; g->x.mmax = mx[0];
  for (PassShape* p : {&g->z, &g->y}) {
    p->cols = strided_cols(p->mmax);
    p->pitch = p->cols;
    p->threads = 256;
    p->smem = 2 * (size_t)p->mmax * p->pitch * cs;
  }
  {
    int P = 2;
    while (P > 1 && 2 * (size_t)g->x.mmax * (6 * P + 1) * cs > budget) --P;
    g->x.cols = 6 * P;
    g->x.pitch = 6 * P + 1;
    g->x.threads = 256;
    g->x.smem = 2 * (size_t)g->x.mmax * g->x.pitch * cs;
    if (g->x.smem > 227 * 1024) {
      *err = "x length too large for the runtime-length path";
      delete g;
      return EQ_ERR_INVALID;
    }
  }
  // work items per field and pass; tiles per item chosen for about 8 items per resident block
  std::vector<long long> iz(count + 1), iy(count + 1), ix(count + 1);
  for (int pi = 0; pi < 3; ++pi) {
    PassShape* p = ps[pi];
    int blocks = 0;
    cudaError_t e = occupancy(dtype, pi == 2 ? 2 : 0, p->threads, p->smem, &blocks);
    if (e == cudaSuccess) e = occupancy(dtype, pi == 2 ? 2 : 1, p->threads, p->smem, &blocks);
    if (e != cudaSuccess || blocks < 1) {
      *err = std::string("occupancy: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "0 blocks");
      delete g;
      return EQ_ERR_CUDA;
    }
    const long long resident = (long long)sms * blocks;
    long long total_tiles = 0;
    for (const FieldDesc& fd : g->fh) {
      if (pi == 2) total_tiles += (fd.npairs + (p->cols / 6) - 1) / (p->cols / 6);
      else {
        const long long ncols = pi == 0 ? (long long)fd.nx * fd.ny : (long long)fd.nz * fd.nx;
        total_tiles += 3 * ((ncols + p->cols - 1) / p->cols);
      }
    }
    p->tpi = (int)std::max(1LL, total_tiles / (8 * resident));
    std::vector<long long>& pre = pi == 0 ? iz : (pi == 1 ? iy : ix);
    pre[0] = 0;
    for (int f = 0; f < count; ++f) {
      const FieldDesc& fd = g->fh[f];
      long long items;
      if (pi == 2) {
        const long long groups = (fd.npairs + (p->cols / 6) - 1) / (p->cols / 6);
        items = (groups + p->tpi - 1) / p->tpi;
      } else {
        const long long ncols = pi == 0 ? (long long)fd.nx * fd.ny : (long long)fd.nz * fd.nx;
        const long long ntiles = (ncols + p->cols - 1) / p->cols;
        items = 3 * ((ntiles + p->tpi - 1) / p->tpi);
      }
      pre[f + 1] = pre[f] + items;
    }
    p->nitems = pre[count];
    p->grid = (int)std::max(1LL, std::min(resident, p->nitems));
  }
  // one device allocation for everything
  size_t o_f = 0, cur = 0;
  auto take = [&](size_t bytes) { size_t at = cur; cur = align_up(cur + bytes, 256); return at; };
  o_f = take(sizeof(FieldDesc) * count);
  const size_t o_a = take(sizeof(AxisPlan) * g->ah.size());
  const size_t o_c = take(cpool.size());
  const size_t o_xi = take(xipool.size());
  const size_t o_pp = take(sizeof(int) * std::max<size_t>(1, pairpool.size()));
  const size_t o_iz = take(sizeof(long long) * (count + 1));
  const size_t o_iy = take(sizeof(long long) * (count + 1));
  const size_t o_ix = take(sizeof(long long) * (count + 1));
  const size_t o_pf = take(sizeof(double) * g->z.nitems * WARPS_MAX * 4);
  const size_t o_px = take(sizeof(double) * g->x.nitems * WARPS_MAX * 4);
  const size_t o_pl = take(sizeof(double) * g->z.nitems * WARPS_MAX * 4);
  const size_t o_m = take(sizeof(double) * 6 * count);
  const size_t o_is = take(sizeof(double) * 2 * count);
  const size_t o_n = take(sizeof(eq_norms_t) * count);
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
  g->z.item0 = reinterpret_cast<long long*>(b + o_iz);
  g->y.item0 = reinterpret_cast<long long*>(b + o_iy);
  g->x.item0 = reinterpret_cast<long long*>(b + o_ix);
  g->part_first = reinterpret_cast<double*>(b + o_pf);
  g->part_x = reinterpret_cast<double*>(b + o_px);
  g->part_last = reinterpret_cast<double*>(b + o_pl);
  g->mean = reinterpret_cast<double*>(b + o_m);
  g->instats = reinterpret_cast<double*>(b + o_is);
  g->norms = reinterpret_cast<eq_norms_t*>(b + o_n);
  struct Up { void* d; const void* h; size_t n; } ups[] = {
      {g->fields, g->fh.data(), sizeof(FieldDesc) * count},
      {g->axes, g->ah.data(), sizeof(AxisPlan) * g->ah.size()},
      {g->cpool, cpool.data(), cpool.size()},
      {g->xipool, xipool.data(), xipool.size()},
      {g->pairpool, pairpool.data(), sizeof(int) * pairpool.size()},
      {g->z.item0, iz.data(), sizeof(long long) * (count + 1)},
      {g->y.item0, iy.data(), sizeof(long long) * (count + 1)},
      {g->x.item0, ix.data(), sizeof(long long) * (count + 1)}};
  for (const Up& u : ups) {
    if (u.n == 0) continue;
    if ((e = cudaMemcpy(u.d, u.h, u.n, cudaMemcpyHostToDevice)) != cudaSuccess) {
      *err = std::string("table upload: ") + cudaGetErrorString(e);
      gen_destroy(g);
      return EQ_ERR_CUDA;
    }
  }
  *out = g;
  return EQ_OK;
}

eq_status gen_enqueue(GenPlan* g, const void* d_in, void* d_out, cudaStream_t s, cudaEvent_t* ev,
                      std::string* err) {
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], s); };
  const bool f32 = g->dtype == EQ_F32;
  auto launch = [&](int kind, const GenArgs& a, const PassShape& p) {
    return f32 ? gen_launch_f32(kind, a, p.grid, p.threads, p.smem, s)
               : gen_launch_f64(kind, a, p.grid, p.threads, p.smem, s);
  };
  GenArgs a{};
  a.fields = g->fields; a.axes = g->axes; a.cpool = g->cpool; a.xipool = g->xipool;
  a.pairpool = g->pairpool; a.mean = g->mean; a.nfields = g->F;
  a.nyq_zero = g->opts.nyq == EQ_NYQ_ZERO;
  auto shape = [&](const PassShape& p) {
    a.item0 = p.item0; a.nitems = p.nitems; a.tiles_per_item = p.tpi; a.cols = p.cols;
    a.pitch = p.pitch; a.mmax = p.mmax;
  };
  cudaError_t e;
  mark(0);
  // z forward (d_in -> d_out) with input statistics
  shape(g->z);
  a.in = d_in; a.out = d_out; a.ref = nullptr; a.partials = g->part_first; a.axis = 2; a.mode = 1;
  if ((e = launch(0, a, g->z)) != cudaSuccess) { *err = std::string("z forward: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(1);
  k_gen_finalize_mean<<<(g->F + 127) / 128, 128, 0, s>>>(g->part_first, g->z.item0, g->fields, g->F,
                                                         g->mean, g->instats);
  if ((e = cudaGetLastError()) != cudaSuccess) { *err = std::string("mean: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(2);
  shape(g->y);
  a.in = d_out; a.partials = nullptr; a.axis = 1; a.mode = 0;
  if ((e = launch(0, a, g->y)) != cudaSuccess) { *err = std::string("y forward: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(3);
  shape(g->x);
  a.partials = g->part_x; a.mode = 0;
  if ((e = launch(2, a, g->x)) != cudaSuccess) { *err = std::string("x pass: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(4);
  shape(g->y);
  a.partials = nullptr; a.axis = 1; a.mode = 0;
  if ((e = launch(1, a, g->y)) != cudaSuccess) { *err = std::string("y inverse: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(5);
  const bool linf = g->opts.want_linf && d_in != d_out;
  shape(g->z);
  a.ref = linf ? d_in : nullptr; a.partials = g->part_last; a.axis = 2; a.mode = linf ? 2 : 0;
  if ((e = launch(1, a, g->z)) != cudaSuccess) { *err = std::string("z inverse: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(6);
  k_gen_finalize_norms<<<(g->F + 127) / 128, 128, 0, s>>>(
      g->part_x, g->x.item0, linf ? g->part_last : nullptr, g->z.item0, g->fields, g->F, g->mean,
      g->instats, linf ? 0 : EQ_FLAG_NO_LINF, g->norms);
  if ((e = cudaGetLastError()) != cudaSuccess) { *err = std::string("norms: ") + cudaGetErrorString(e); return EQ_ERR_CUDA; }
  mark(7);
  return EQ_OK;
}

const eq_norms_t* gen_norms_device(const GenPlan* g) { return g->norms; }
size_t gen_device_bytes(const GenPlan* g) { return g->dbytes; }
long long gen_total_elems(const GenPlan* g) { return g->total_elems; }
int gen_count(const GenPlan* g) { return g->F; }

void gen_destroy(GenPlan* g) {
  if (!g) return;
  if (g->dmem) cudaFree(g->dmem);
  delete g;
}

}  // namespace eqg
