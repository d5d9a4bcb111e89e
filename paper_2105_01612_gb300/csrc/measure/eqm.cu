// eqm.cu - measurement kernels for the benchmark (libeqm.so): arithmetic-throughput probes that
// give the roofline denominators no copy or GEMM measures (FP64 and FP32 FMA), and the per-mode
// projector over a cuFFT half spectrum, the elementwise half of the "cuFFT plus one kernel"
// comparison baseline.  None of this is on the projection path of libeq.so.
//
// C entry points (all enqueue on `stream` and return a cudaError_t value as int):
//   eqm_fma_probe(dtype, out, blocks, threads, iters, stream)
//       dtype 1: FP64, 0: FP32.  Every thread runs 8 independent FMA chains for `iters` rounds
//       (2 * 8 * iters flops a thread); out (device, blocks * threads elements of dtype) receives
//       the chains' sums so that no chain is dead code.
//   eqm_project_half(dtype, spec, nz, ny, nxh, xi_x, xi_y, xi_z, stream)
//       spec: device, complex (interleaved re, im) array [6][nz][ny][nxh] of dtype, the r2c
//       spectrum of the six Voigt planes (xx, yy, zz, yz, xz, xy) of one field; xi_*: device
//       operator symbols (nxh, ny, nz entries).  In place, at every mode with |xi| > 0:
//       S <- S - n (x) v - v (x) n + (n . v) n (x) n with n = xi / |xi|, v = S n (the projector
//       Q S Q of Sec. 3.2 with Q = I - n n^T); modes with xi = 0 are kept.
#include <cuda_runtime.h>

namespace {

template <typename T>
__global__ void k_fma_probe(T* out, long long iters) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x) * T(1e-6) + T(k);
  const T a = T(0.9999), b = T(1e-4);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <typename T>
__global__ void __launch_bounds__(256)
k_project_half(typename C2<T>::t* spec, int nz, int ny, int nxh, const T* __restrict__ xi_x,
               const T* __restrict__ xi_y, const T* __restrict__ xi_z) {
  using T2 = typename C2<T>::t;
  const long long plane = (long long)nz * ny * nxh;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < plane;
       m += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(m % nxh);
    const long long r = m / nxh;
    const int ky = (int)(r % ny), kz = (int)(r / ny);
    const T x0 = xi_x[kx], x1 = xi_y[ky], x2 = xi_z[kz];
    const T k2 = x0 * x0 + x1 * x1 + x2 * x2;
    if (!(k2 > T(0))) continue;
    const T rn = T(1) / sqrt(k2);
    const T n0 = x0 * rn, n1 = x1 * rn, n2 = x2 * rn;
    T2 s[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) s[j] = spec[j * plane + m];
    // v = S n with S = [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]], Voigt slots 0..5
    T2 v0, v1, v2;
    v0.x = s[0].x * n0 + s[5].x * n1 + s[4].x * n2;  v0.y = s[0].y * n0 + s[5].y * n1 + s[4].y * n2;
    v1.x = s[5].x * n0 + s[1].x * n1 + s[3].x * n2;  v1.y = s[5].y * n0 + s[1].y * n1 + s[3].y * n2;
    v2.x = s[4].x * n0 + s[3].x * n1 + s[2].x * n2;  v2.y = s[4].y * n0 + s[3].y * n1 + s[2].y * n2;
    T2 q;
    q.x = n0 * v0.x + n1 * v1.x + n2 * v2.x;
    q.y = n0 * v0.y + n1 * v1.y + n2 * v2.y;
    const T nn[3] = {n0, n1, n2};
    const T2 vv[3] = {v0, v1, v2};
    const int I[6] = {0, 1, 2, 1, 0, 0}, J[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int i = I[j], l = J[j];
      T2 o;
      o.x = s[j].x - nn[i] * vv[l].x - vv[i].x * nn[l] + q.x * nn[i] * nn[l];
      o.y = s[j].y - nn[i] * vv[l].y - vv[i].y * nn[l] + q.y * nn[i] * nn[l];
      spec[j * plane + m] = o;
    }
  }
}

int grid_for(long long work, int threads) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long g = (work + threads - 1) / threads;
  const long long cap = (long long)sms * 8;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

extern "C" int eqm_fma_probe(int dtype, void* out, int blocks, int threads, long long iters,
                             void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == 1) k_fma_probe<double><<<blocks, threads, 0, s>>>(static_cast<double*>(out), iters);
  else k_fma_probe<float><<<blocks, threads, 0, s>>>(static_cast<float*>(out), iters);
  return (int)cudaGetLastError();
}

extern "C" int eqm_project_half(int dtype, void* spec, int nz, int ny, int nxh, const void* xi_x,
                                const void* xi_y, const void* xi_z, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long plane = (long long)nz * ny * nxh;
  const int g = grid_for(plane, 256);
  if (dtype == 1)
    k_project_half<double><<<g, 256, 0, s>>>(static_cast<double2*>(spec), nz, ny, nxh,
                                              static_cast<const double*>(xi_x),
                                              static_cast<const double*>(xi_y),
                                              static_cast<const double*>(xi_z));
  else
    k_project_half<float><<<g, 256, 0, s>>>(static_cast<float2*>(spec), nz, ny, nxh,
                                             static_cast<const float*>(xi_x),
                                             static_cast<const float*>(xi_y),
                                             static_cast<const float*>(xi_z));
  return (int)cudaGetLastError();
}
