// eq_grains.cu - grain means and the grain-averaged field over a fixed grain map (Sec. 5.1: the
// synthetic measurement of Table 1 averages the equilibrated stress over each grain).
//
// The grain map is fixed across the fields averaged with it, so eq_grains_create sorts the voxel
// indices by grain once, on the host, keeping voxel order within a grain (a counting sort), and
// uploads the per-grain lists.  A means launch then gives each (grain, field) one block that
// walks its grain's list in a fixed order and reduces in FP64 with a fixed tree: the means do
// not depend on timing.  The fill launch writes every voxel's grain mean, coalesced along the
// voxel index.
#include <cuda_runtime.h>

#include <new>
#include <string>
#include <vector>

#include "eq_internal.h"

struct eq_grains {
  int nx = 0, ny = 0, nz = 0, ngrains = 0;
  long long V = 0;
  int device = 0;
  int sms = 0;
  long long* d_off = nullptr;   // [ngrains + 1] start of each grain's voxel list
  int* d_vox = nullptr;         // [V] voxel indices grouped by grain, increasing within a grain
  int* d_map = nullptr;         // [V] grain id of each voxel
  void* d_mt = nullptr;         // means in the fields' dtype for the fill, [cap][ngrains][6]
  size_t mt_bytes = 0;
};

namespace {

eq_status gfail(eq_status st, const std::string& msg) {
  eqk::set_last_error(msg);
  return st;
}

void release(eq_grains* g) {
  if (!g) return;
  if (g->d_off) cudaFree(g->d_off);
  if (g->d_vox) cudaFree(g->d_vox);
  if (g->d_map) cudaFree(g->d_map);
  if (g->d_mt) cudaFree(g->d_mt);
  delete g;
}

// Per-thread running sum: FP64 for FP64 data; for FP32 data a compensated FP32 sum (error about
// 2 eps of the summed magnitudes, whatever the count; FP64 arithmetic is scarce on GB300).
template <typename T> struct GrainAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(T v) { s += double(v); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct GrainAcc<float> {
  eqk::Kahan<float> k;
  __device__ __forceinline__ void add(float v) { k.add(v); }
  __device__ __forceinline__ double value() const { return k.value(); }
};

// grid (ngrains, batch), 256 threads: means[f][g][c] = (sum over grain g of field f, plane c) / n_g
template <typename T>
__global__ void __launch_bounds__(256)
k_grain_means(const T* __restrict__ in, long long field_stride, long long V,
              const long long* __restrict__ off, const int* __restrict__ vox, int ngrains,
              double* __restrict__ means, T* __restrict__ means_t) {
  __shared__ double red[32 * 6];
  const int g = blockIdx.x, f = blockIdx.y;
  const T* s = in + f * field_stride;
  const long long b = off[g], e = off[g + 1];
  GrainAcc<T> acc[6];
  // four list entries per step (their loads in flight together), in list order per thread
  const long long bs = blockDim.x;
  long long i = b + threadIdx.x;
  for (; i + 3 * bs < e; i += 4 * bs) {
    long long p[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) p[k] = vox[i + k * bs];
    T x[4][6];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 6; ++c) x[k][c] = s[c * V + p[k]];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[c].add(x[k][c]);
  }
  for (; i < e; i += bs) {
    const long long p = vox[i];
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c].add(s[c * V + p]);
  }
  double v[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) v[c] = acc[c].value();
  eqk::block_sum<6>(v, red);
  if (threadIdx.x == 0) {
    const double n = double(e - b);
    double* m = means + ((long long)f * ngrains + g) * 6;
    T* mt = means_t ? means_t + ((long long)f * ngrains + g) * 6 : nullptr;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      m[c] = n > 0.0 ? v[c] / n : 0.0;
      if (mt) mt[c] = T(m[c]);
    }
  }
}

// out[f][c][p] = means[f][map[p]][c]; grid (blocks, batch).  Each warp takes chunks of 128
// consecutive voxels, lane l the voxels l + 32 k (k < 4): every load and store instruction covers
// 32 consecutive voxels, four in flight per lane.
template <typename T>
__global__ void __launch_bounds__(256)
k_grain_fill(T* __restrict__ out, long long field_stride, long long V, const int* __restrict__ map,
             int ngrains, const T* __restrict__ means_t) {
  const int f = blockIdx.y;
  const T* mf = means_t + (long long)f * ngrains * 6;
  T* of = out + f * field_stride;
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = w0 * 128; base < V; base += nw * 128) {
    int gs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long p = base + lane + 32 * k;
      gs[k] = p < V ? map[p] : 0;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      T v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = mf[gs[k] * 6 + c];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long long p = base + lane + 32 * k;
        if (p < V) of[c * V + p] = v[k];
      }
    }
  }
}

}  // namespace

extern "C" eq_status eq_grains_create(const int* grain_map, int nx, int ny, int nz, int ngrains,
                                      eq_grains** out) {
  if (!out) return gfail(EQ_ERR_INVALID, "eq_grains_create: out is NULL");
  *out = nullptr;
  if (!grain_map) return gfail(EQ_ERR_INVALID, "eq_grains_create: grain_map is NULL");
  if (nx < 1 || ny < 1 || nz < 1 || nx > 1024 || ny > 1024 || nz > 1024 || ngrains < 1)
    return gfail(EQ_ERR_INVALID, "eq_grains_create: sizes must be 1..1024 and ngrains >= 1");
  const long long V = (long long)nx * ny * nz;
  // counting sort of the voxel indices by grain id (stable: voxel order within a grain)
  std::vector<long long> off((size_t)ngrains + 1, 0);
  for (long long v = 0; v < V; ++v) {
    const int g = grain_map[v];
    if (g < 0 || g >= ngrains)
      return gfail(EQ_ERR_INVALID, "eq_grains_create: grain id " + std::to_string(g) +
                                       " at voxel " + std::to_string(v) + " outside [0, ngrains)");
    ++off[(size_t)g + 1];
  }
  for (int g = 0; g < ngrains; ++g) off[(size_t)g + 1] += off[(size_t)g];
  std::vector<int> vox((size_t)V);
  {
    std::vector<long long> pos(off.begin(), off.end() - 1);
    for (long long v = 0; v < V; ++v) vox[(size_t)pos[(size_t)grain_map[v]]++] = (int)v;
  }
  eq_grains* g = new (std::nothrow) eq_grains();
  if (!g) return gfail(EQ_ERR_OOM, "eq_grains_create: host allocation failed");
  g->nx = nx; g->ny = ny; g->nz = nz; g->ngrains = ngrains; g->V = V;
  cudaError_t e;
  if ((e = cudaGetDevice(&g->device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device)) != cudaSuccess) {
    release(g);
    return gfail(EQ_ERR_CUDA, std::string("eq_grains_create: ") + cudaGetErrorString(e));
  }
  if ((e = cudaMalloc(&g->d_off, sizeof(long long) * off.size())) != cudaSuccess ||
      (e = cudaMalloc(&g->d_vox, sizeof(int) * (size_t)V)) != cudaSuccess ||
      (e = cudaMalloc(&g->d_map, sizeof(int) * (size_t)V)) != cudaSuccess) {
    release(g);
    cudaGetLastError();
    return gfail(EQ_ERR_OOM, std::string("eq_grains_create: cudaMalloc: ") + cudaGetErrorString(e));
  }
  if ((e = cudaMemcpy(g->d_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(g->d_vox, vox.data(), sizeof(int) * (size_t)V, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(g->d_map, grain_map, sizeof(int) * (size_t)V, cudaMemcpyHostToDevice)) != cudaSuccess) {
    release(g);
    return gfail(EQ_ERR_CUDA, std::string("eq_grains_create: upload: ") + cudaGetErrorString(e));
  }
  *out = g;
  return EQ_OK;
}

extern "C" eq_status eq_grain_average(eq_grains* g, eq_dtype dtype, int batch, const void* d_in,
                                      double* d_means, void* d_avg, void* stream) {
  if (!g || !d_in || !d_means) return gfail(EQ_ERR_INVALID, "eq_grain_average: NULL argument");
  if (batch < 1 || batch > 65535) return gfail(EQ_ERR_INVALID, "eq_grain_average: batch must be 1..65535");
  if (dtype != EQ_F32 && dtype != EQ_F64) return gfail(EQ_ERR_INVALID, "eq_grain_average: bad dtype");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != g->device)
    return gfail(EQ_ERR_INVALID, "eq_grain_average: current device differs from the grain map's");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long fs = 6 * g->V;
  cudaError_t e;
  if (d_avg) {
    // the fill reads the means in the fields' dtype (converted once per grain, not per voxel):
    // an object-owned buffer, grown on a call with a larger batch or dtype
    const size_t need = (size_t)batch * g->ngrains * 6 * (dtype == EQ_F32 ? 4 : 8);
    if (need > g->mt_bytes) {
      if (g->d_mt) cudaFree(g->d_mt);
      g->d_mt = nullptr;
      g->mt_bytes = 0;
      if ((e = cudaMalloc(&g->d_mt, need)) != cudaSuccess) {
        g->d_mt = nullptr;
        cudaGetLastError();
        return gfail(EQ_ERR_OOM, std::string("eq_grain_average: cudaMalloc: ") + cudaGetErrorString(e));
      }
      g->mt_bytes = need;
    }
  }
  dim3 grid((unsigned)g->ngrains, (unsigned)batch);
  if (dtype == EQ_F32)
    k_grain_means<float><<<grid, 256, 0, s>>>(static_cast<const float*>(d_in), fs, g->V, g->d_off,
                                                g->d_vox, g->ngrains, d_means,
                                                d_avg ? static_cast<float*>(g->d_mt) : nullptr);
  else
    k_grain_means<double><<<grid, 256, 0, s>>>(static_cast<const double*>(d_in), fs, g->V, g->d_off,
                                                 g->d_vox, g->ngrains, d_means,
                                                 d_avg ? static_cast<double*>(g->d_mt) : nullptr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gfail(EQ_ERR_CUDA, std::string("eq_grain_average: means: ") + cudaGetErrorString(e));
  if (d_avg) {
    const long long chunks = (g->V + 127) / 128;              // one warp each
    dim3 fgrid((unsigned)std::max<long long>(1, std::min<long long>((long long)g->sms * 8 / batch + 1,
                                                                    (chunks + 7) / 8)),
               (unsigned)batch);
    if (dtype == EQ_F32)
      k_grain_fill<float><<<fgrid, 256, 0, s>>>(static_cast<float*>(d_avg), fs, g->V, g->d_map,
                                                 g->ngrains, static_cast<const float*>(g->d_mt));
    else
      k_grain_fill<double><<<fgrid, 256, 0, s>>>(static_cast<double*>(d_avg), fs, g->V, g->d_map,
                                                  g->ngrains, static_cast<const double*>(g->d_mt));
    if ((e = cudaGetLastError()) != cudaSuccess)
      return gfail(EQ_ERR_CUDA, std::string("eq_grain_average: fill: ") + cudaGetErrorString(e));
  }
  return EQ_OK;
}

extern "C" void eq_grains_destroy(eq_grains* g) { release(g); }
