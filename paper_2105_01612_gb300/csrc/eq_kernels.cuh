// eq_kernels.cuh - the five HBM passes of the projection and their launch configuration.
//
// Data layout: the caller's output buffer holds the spectrum during the call.  The six real
// Voigt planes of a field are read as three complex fields Z_c = S_{2c} + i S_{2c+1}
// ((xx, yy), (zz, yz), (xz, xy)), stored split-complex (real part in plane 2c, imaginary part in
// plane 2c+1).  Every pass reads a tile and writes the same positions, so the whole pipeline
// runs in place in d_out and d_out may alias d_in.  Pass order:
//   1. z forward  (reads d_in, writes d_out; FP64 mean / norm partials of the input)
//   2. y forward
//   3. x forward + per-mode projector + x inverse (row pairs k, -k together; norm partials)
//   4. y inverse
//   5. z inverse  (optional residual L-infinity against d_in)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "eq_fft.cuh"
#include "eq_dd.cuh"

namespace eqk {

// Bounds-checked builds (compiled with EQ_BOUNDS_CHECK defined; libeq_check.so): an index outside
// [0, n) raises bit EQ_ERRBIT_BOUNDS of the plan's error word and the access is skipped, so a
// wrong index shows up as an error status at eq_norms instead of a fault.  Other builds compile
// the check away.  Checked: the global loads and stores of the plain strided and x passes, of the
// warp-per-row x passes and of the runtime-length passes, and the shared-memory work-buffer
// indices of the runtime-length transforms.
#define EQ_ERRBIT_BOUNDS 2
__device__ __forceinline__ bool in_bounds(long long i, long long n, int* err) {
#ifdef EQ_BOUNDS_CHECK
  if (i >= 0 && i < n) return true;
  if (err) atomicOr(err, EQ_ERRBIT_BOUNDS);
  return false;
#else
  (void)i; (void)n; (void)err;
  return true;
#endif
}

template <typename T, int N> struct Cfg {
  static constexpr int E = N >= 8 ? 8 : N;
  static constexpr int TPC = N / E;
  static constexpr int B0 = sizeof(T) == 4 ? 16 : 8;
  static constexpr int BW = (256 / TPC > B0) ? 256 / TPC : B0;
  static constexpr int B = (BW * TPC > 1024) ? 1024 / TPC : BW;          // strided columns
  static constexpr int STRIDED_THREADS = B * TPC;
  // x pass: P row pairs (6 P transforms) per block; 6 P TPC must be a multiple of 32
  static constexpr int PM_ = TPC >= 16 ? 1 : 16 / TPC;
  static constexpr int PW0 = (256 + 6 * TPC - 1) / (6 * TPC) > 2 ? (256 + 6 * TPC - 1) / (6 * TPC) : 2;
  static constexpr int PW = (PW0 + PM_ - 1) / PM_ * PM_;
  static constexpr int PM = 1024 / (6 * TPC) > 0 ? 1024 / (6 * TPC) : 1;
  static constexpr int P = PW < PM ? PW : PM;                               // x-pass row pairs
  static constexpr int XCOLS = 6 * P;
  static constexpr int X_THREADS = XCOLS * TPC;
  static constexpr int PITCH = N + (N >> 3);
  using T2 = typename V2<T>::t;
  static constexpr size_t STRIDED_SMEM = sizeof(T2) * (size_t(N) + size_t(N) * B);
  static constexpr size_t X_SMEM = sizeof(T2) * (size_t(N) + size_t(XCOLS) * PITCH) + sizeof(T) * N;
};

struct StridedArgs {
  const void* in;          // field 0, plane 0 of the source
  void* out;               // field 0, plane 0 of the destination
  const void* ref;         // last pass: original input for resid_linf (nullptr = skip)
  const void* tw;          // N twiddles exp(-2 pi i m / N)
  long long field_stride;  // elements between fields (6 V)
  long long V;             // elements per plane
  long long nstride;       // elements between consecutive points of one transform
  long long inner;         // columns per outer slab (contiguous index range)
  long long outer_stride;  // elements between outer slabs
  long long ncols;         // outer * inner
  long long ntiles;        // ceil(ncols / B)
  double* partials;        // first: [batch][3][grid][4]; last: [batch][3][grid] (linf)
  int mode;                // 0 = middle pass, 1 = first (reductions), 2 = last
  int ncomp;               // complex fields (pairs of planes) per field: 3 (stress), 2 (potential)
  int* err;                // plan error word (bounds-checked builds; nullable)
};

struct XArgs {
  void* data;              // field 0, plane 0 (spectrum, split complex)
  const void* tw;          // nx twiddles
  const void* xi_x;        // operator symbol per axis (nx, ny, nz entries)
  const void* xi_y;
  const void* xi_z;
  const int* pairs;        // canonical rows kz * ny + ky whose mirror row is >= itself
  const double* mean;      // [batch][6] FP64 mean (c0)
  double* partials;        // [batch][grid][4]
  long long field_stride;
  long long V;
  int nx, ny, nz;
  int npairs;
  int ngroups;
  int nyq_zero;
  int compat;              // 1: return the compatible part c0 + (S - S_equil)
  double inv_v;            // 1 / (nx ny nz)
  void* ydata;             // potential pass: field 0, plane 0 of the 4-plane y buffer
  long long yfield_stride; // elements between fields of the y buffer (4 V)
  int* err;                // plan error word (bounds-checked builds; nullable)
};

// deterministic block sum of K doubles per thread; result valid in thread 0
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* red /* >= 32*K */) {
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
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[w * K + k];
      v[k] = s;
    }
  }
}

__device__ __forceinline__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) v = fmax(v, red[w]);
  }
  return v;
}

struct IdxStrided {
  int b, B;
  __device__ __forceinline__ int operator()(int i) const { return i * B + b; }
};
struct IdxRow {
  int base;
  __device__ __forceinline__ int operator()(int i) const { return base + i + (i >> 3); }
};

// Transform along a strided axis (z or y) of all three complex fields of every field.
// grid = (G, batch * 3); block = Cfg::STRIDED_THREADS.
template <typename T, int N, bool INV>
__global__ void __launch_bounds__(Cfg<T, N>::STRIDED_THREADS)
k_strided(const StridedArgs a) {
  using C = Cfg<T, N>;
  using T2 = typename C::T2;
  constexpr int E = C::E, TPC = C::TPC, B = C::B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* tw = reinterpret_cast<T2*>(smem_raw);
  T2* buf = tw + N;
  __shared__ double red[32 * 4];

  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = reinterpret_cast<const T2*>(a.tw)[i];
  __syncthreads();

  const int b = threadIdx.x % B, t = threadIdx.x / B;
  const int field = blockIdx.y / a.ncomp, comp = blockIdx.y % a.ncomp;
  const long long fbase = field * a.field_stride + (2LL * comp) * a.V;
  const T* in_re = reinterpret_cast<const T*>(a.in) + fbase;
  const T* in_im = in_re + a.V;
  T* out_re = reinterpret_cast<T*>(a.out) + fbase;
  T* out_im = out_re + a.V;
  const T* ref_re = a.ref ? reinterpret_cast<const T*>(a.ref) + fbase : nullptr;
  const T* ref_im = ref_re ? ref_re + a.V : nullptr;
  // Voigt weights of the two planes of complex field `comp`: (1,1), (1,2), (2,2)
  const T wa = comp == 2 ? T(2) : T(1), wb = comp == 0 ? T(1) : T(2);

  Kahan<T> sa, sb, sq;
  T nonfinite = T(0);
  T linf = T(0);
  const IdxStrided idx{b, B};

  for (long long tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const long long col = tile * B + b;
    const bool valid = col < a.ncols;
    const long long o = valid ? col / a.inner : 0, ii = valid ? col - o * a.inner : 0;
    const long long base = o * a.outer_stride + ii;
    T2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const long long off = base + (long long)(t + TPC * e) * a.nstride;
      x[e] = valid && in_bounds(off, a.V, a.err) ? T2{in_re[off], in_im[off]} : T2{T(0), T(0)};
    }
    if (a.mode == 1 && valid) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        if (!isfinite(x[e].x) || !isfinite(x[e].y)) nonfinite += T(1);
        sa.add(x[e].x);
        sb.add(x[e].y);
        sq.add(wa * x[e].x * x[e].x + wb * x[e].y * x[e].y);
      }
    }
    fft_column<N, E, INV>(x, t, buf, idx, tw);
    if (valid) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const long long off = base + (long long)(t + TPC * e) * a.nstride;
        if (!in_bounds(off, a.V, a.err)) continue;
        out_re[off] = x[e].x;
        out_im[off] = x[e].y;
        if (a.mode == 2 && ref_re) {
          linf = fmax(linf, fabs(ref_re[off] - x[e].x));
          linf = fmax(linf, fabs(ref_im[off] - x[e].y));
        }
      }
    }
  }
  if (a.mode == 1) {
    double v[4] = {sa.value(), sb.value(), sq.value(), double(nonfinite)};
    block_sum<4>(v, red);
    if (threadIdx.x == 0) {
      double* p = a.partials + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * 4;
      p[0] = v[0]; p[1] = v[1]; p[2] = v[2]; p[3] = v[3];
    }
  } else if (a.mode == 2 && ref_re) {
    double m = block_max(double(linf), red);
    if (threadIdx.x == 0) a.partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = m;
  }
}

// 2 c0_j V of field `mean` (FP64 means, V voxels) in the working precision, computed once per
// field outside the mode loops; false (and nothing written) when there is no mean.
template <typename T>
__device__ __forceinline__ bool zero_mode_values(const double* mean, double vol, T (&zm)[6]) {
  if (!mean) return false;
#pragma unroll
  for (int j = 0; j < 6; ++j) zm[j] = T(2.0 * mean[j] * vol);
  return true;
}

// rsqrt in the kernel's precision (library calls)
__device__ __forceinline__ float rsqrt_t(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_t(double v) { return rsqrt(v); }

// The per-mode projector and its norm terms for one mode pair (k, -k).
//   in:  a[c] = Z_c(k), bb[c] = Z_c(-k)  (c = 0..2)
//   out: a[c] <- Zout_c(k) / V,  bb[c] <- Zout_c(-k) / V
// Zout is the projected field Q S Q, or with `compat` its complement S - Q S Q (the mean, at
// k = 0, is kept either way).  zm (nullable): the k = 0 values of the doubled Voigt components,
// 2 c0_j V, set in place of the transformed mean at the zero mode (zero_mode_values below).
// Works on twice the Voigt components (the unpack's 1/2 is folded into the repack and into the
// norm weights).  With n = xi / |xi|, v = S n and s = n . v, the projector removes
// D = n (x) v + v (x) n - s n (x) n, whose squared Frobenius norm is 2 |v|^2 - s^2 (no
// cancellation: |v|^2 >= s^2), and |xi . S|^2 = |xi|^2 |v|^2.
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }

// FP32 form of project_pair below, the same arithmetic with the real and imaginary parts of each
// doubled Voigt component held as one pair P_j = {Re, Im} and worked by packed two-lane
// instructions (one instruction for both parts wherever they meet the same real factor).
// ACC: the running sums of the four norm terms (anything with add(float): a Kahan sum, or a plain
// sum that the caller folds into a compensated one).
template <typename ACC>
__device__ __forceinline__ void project_pair_f32x2(float2 (&a)[3], float2 (&bb)[3], float xi0,
                                                   float xi1, float xi2, bool zero_mode,
                                                   const float* zm, bool nyq_zero,
                                                   bool compat, float inv_v, float mult,
                                                   ACC& r2, ACC& di2, ACC& do2, ACC& o2) {
  // 2 S_2c = A + conj B, 2 S_2c+1 = -i (A - conj B)
  float2 P[6];
  const float2 pm = make_float2(1.f, -1.f);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    P[2 * c] = __ffma2_rn(bb[c], pm, a[c]);
    P[2 * c + 1] = make_float2(a[c].y + bb[c].y, bb[c].x - a[c].x);
  }
  if (zero_mode && zm) {
#pragma unroll
    for (int j = 0; j < 6; ++j) P[j] = make_float2(zm[j], 0.f);
  }
  const float k2 = xi0 * xi0 + xi1 * xi1 + xi2 * xi2;
  float2 O[6];
  float rr = 0.f, din = 0.f;
  if (k2 > 0.f) {
    const float rn = rsqrtf(k2);
    const float n0 = xi0 * rn, n1 = xi1 * rn, n2 = xi2 * rn;
    const float2 N0 = bc2(n0), N1 = bc2(n1), N2 = bc2(n2);
    // v = S n, s = n . v (Voigt slots: 0 xx, 1 yy, 2 zz, 3 yz, 4 xz, 5 xy)
    const float2 V0 = __ffma2_rn(P[4], N2, __ffma2_rn(P[5], N1, __fmul2_rn(P[0], N0)));
    const float2 V1 = __ffma2_rn(P[3], N2, __ffma2_rn(P[1], N1, __fmul2_rn(P[5], N0)));
    const float2 V2 = __ffma2_rn(P[2], N2, __ffma2_rn(P[3], N1, __fmul2_rn(P[4], N0)));
    const float2 S = __ffma2_rn(N2, V2, __ffma2_rn(N1, V1, __fmul2_rn(N0, V0)));
    const float2 VV = __ffma2_rn(V2, V2, __ffma2_rn(V1, V1, __fmul2_rn(V0, V0)));
    const float2 R = __ffma2_rn(__fmul2_rn(S, bc2(-1.f)), S, __fadd2_rn(VV, VV));   // 2|v|^2 - s^2
    rr = R.x + R.y;
    din = k2 * (VV.x + VV.y);
    O[0] = __ffma2_rn(S, bc2(n0 * n0), __ffma2_rn(V0, bc2(-2.f * n0), P[0]));
    O[1] = __ffma2_rn(S, bc2(n1 * n1), __ffma2_rn(V1, bc2(-2.f * n1), P[1]));
    O[2] = __ffma2_rn(S, bc2(n2 * n2), __ffma2_rn(V2, bc2(-2.f * n2), P[2]));
    O[3] = __ffma2_rn(S, bc2(n1 * n2), __ffma2_rn(V1, bc2(-n2), __ffma2_rn(V2, bc2(-n1), P[3])));
    O[4] = __ffma2_rn(S, bc2(n0 * n2), __ffma2_rn(V0, bc2(-n2), __ffma2_rn(V2, bc2(-n0), P[4])));
    O[5] = __ffma2_rn(S, bc2(n0 * n1), __ffma2_rn(V0, bc2(-n1), __ffma2_rn(V1, bc2(-n0), P[5])));
  } else {
    // the zero mode and the all-Nyquist corners: kept, or dropped (literal route, not the mean)
    const bool drop = nyq_zero && !zero_mode;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float w = j < 3 ? 1.f : 2.f;
      if (drop) rr += w * (P[j].x * P[j].x + P[j].y * P[j].y);
      O[j] = drop ? make_float2(0.f, 0.f) : P[j];
    }
  }
  // sum over j of w_j |X_j|^2 (w = 1 for the normal, 2 for the shear slots), both parts
  auto wnorm = [](const float2 (&X)[6]) {
    const float2 d = __ffma2_rn(X[2], X[2], __ffma2_rn(X[1], X[1], __fmul2_rn(X[0], X[0])));
    const float2 o = __ffma2_rn(X[5], X[5], __ffma2_rn(X[4], X[4], __fmul2_rn(X[3], X[3])));
    const float2 q = __ffma2_rn(o, bc2(2.f), d);
    return q.x + q.y;
  };
  // compatible part: out = S - O away from k = 0; the residual S - out is then O
  if (compat && !zero_mode) {
    const float o2n = wnorm(O);
#pragma unroll
    for (int j = 0; j < 6; ++j) O[j] = csub(P[j], O[j]);
    rr = o2n;
  }
  // norm terms (sums of |.|^2 over modes; Parseval turns them into voxel means)
  {
    const float oo = wnorm(O);
    const float2 X0 = bc2(xi0), X1 = bc2(xi1), X2 = bc2(xi2);
    const float2 D0 = __ffma2_rn(X2, O[4], __ffma2_rn(X1, O[5], __fmul2_rn(X0, O[0])));
    const float2 D1 = __ffma2_rn(X2, O[3], __ffma2_rn(X1, O[1], __fmul2_rn(X0, O[5])));
    const float2 D2 = __ffma2_rn(X2, O[2], __ffma2_rn(X1, O[3], __fmul2_rn(X0, O[4])));
    const float2 DD = __ffma2_rn(D2, D2, __ffma2_rn(D1, D1, __fmul2_rn(D0, D0)));
    const float dout = DD.x + DD.y;
    const float m4 = 0.25f * mult;                    // (1/2)^2 of the doubled components
    r2.add(m4 * rr);
    o2.add(m4 * oo);
    di2.add(m4 * din);
    do2.add(m4 * dout);
  }
  // repack: Zout_c(k) = O_2c + i O_2c+1, Zout_c(-k) = conj(O_2c) + i conj(O_2c+1), halved
  const float2 hv = bc2(0.5f * inv_v);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 A = O[2 * c], B = O[2 * c + 1];
    a[c] = __fmul2_rn(make_float2(A.x - B.y, A.y + B.x), hv);
    bb[c] = __fmul2_rn(make_float2(A.x + B.y, B.x - A.y), hv);
  }
}

template <typename T, typename T2, typename ACC>
__device__ __forceinline__ void project_pair(T2 (&a)[3], T2 (&bb)[3], T xi0, T xi1, T xi2,
                                             bool zero_mode, const T* zm,
                                             bool nyq_zero, bool compat, T inv_v, T mult,
                                             ACC& r2, ACC& di2, ACC& do2, ACC& o2) {
  if constexpr (sizeof(T) == 4) {
    project_pair_f32x2(a, bb, xi0, xi1, xi2, zero_mode, zm, nyq_zero, compat, inv_v, mult,
                       r2, di2, do2, o2);
  } else if constexpr (std::is_same<T, double>::value) {
    // FP64: the same arithmetic in double-float (FP32 instructions, about 2^-48 relative per
    // operation), inputs and outputs converted on the bits.  FP64 instructions issue at a small
    // fraction of the FP32 rate on this GPU, and this is the FP64 path's densest arithmetic.
    dd2 ad[3], bd[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ad[c] = dd2{dd_from_bits(a[c].x), dd_from_bits(a[c].y)};
      bd[c] = dd2{dd_from_bits(bb[c].x), dd_from_bits(bb[c].y)};
    }
    dd zmd[6];
    const bool zmode = zero_mode && zm;
    if (zmode) {
#pragma unroll
      for (int j = 0; j < 6; ++j) zmd[j] = dd_from_bits(zm[j]);
    }
    PlainSum<dd> pr, pdi, pdo, po;
    project_pair<dd, dd2>(ad, bd, dd_from_bits(xi0), dd_from_bits(xi1), dd_from_bits(xi2),
                          zero_mode, zmode ? zmd : nullptr, nyq_zero, compat, dd_from_bits(inv_v),
                          dd_from_bits(mult), pr, pdi, pdo, po);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a[c] = T2{dd_to_bits(ad[c].x), dd_to_bits(ad[c].y)};
      bb[c] = T2{dd_to_bits(bd[c].x), dd_to_bits(bd[c].y)};
    }
    r2.add(dd_to_bits(pr.s));
    di2.add(dd_to_bits(pdi.s));
    do2.add(dd_to_bits(pdo.s));
    o2.add(dd_to_bits(po.s));
  } else {
    // 2 S_2c = A + conj B, 2 S_2c+1 = -i (A - conj B)
    T sr[6], si[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sr[2 * c] = a[c].x + bb[c].x;
      si[2 * c] = a[c].y - bb[c].y;
      sr[2 * c + 1] = a[c].y + bb[c].y;
      si[2 * c + 1] = bb[c].x - a[c].x;
    }
    if (zero_mode && zm) {
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        sr[j] = zm[j];
        si[j] = T(0);
      }
    }
    const T k2 = xi0 * xi0 + xi1 * xi1 + xi2 * xi2;
    T orr[6], oi[6];
    T rr = T(0), din = T(0);
    if (k2 > T(0)) {
      const T rn = rsqrt_t(k2);
      const T n0 = xi0 * rn, n1 = xi1 * rn, n2 = xi2 * rn;
      // Voigt slots: 0 xx, 1 yy, 2 zz, 3 yz, 4 xz, 5 xy
  #define EQ_PROJ(S, O)                                                         \
      {                                                                          \
        const T v0 = S[0] * n0 + S[5] * n1 + S[4] * n2;                          \
        const T v1 = S[5] * n0 + S[1] * n1 + S[3] * n2;                          \
        const T v2 = S[4] * n0 + S[3] * n1 + S[2] * n2;                          \
        const T s = n0 * v0 + n1 * v1 + n2 * v2;                                 \
        const T vv = v0 * v0 + v1 * v1 + v2 * v2;                               \
        rr += T(2) * vv - s * s;                                                 \
        din += k2 * vv;                                                          \
        O[0] = S[0] - T(2) * n0 * v0 + s * n0 * n0;                              \
        O[1] = S[1] - T(2) * n1 * v1 + s * n1 * n1;                              \
        O[2] = S[2] - T(2) * n2 * v2 + s * n2 * n2;                              \
        O[3] = S[3] - n1 * v2 - v1 * n2 + s * n1 * n2;                           \
        O[4] = S[4] - n0 * v2 - v0 * n2 + s * n0 * n2;                           \
        O[5] = S[5] - n0 * v1 - v0 * n1 + s * n0 * n1;                           \
      }
      EQ_PROJ(sr, orr)
      EQ_PROJ(si, oi)
  #undef EQ_PROJ
    } else {
      // the zero mode and the all-Nyquist corners: kept, or dropped (literal route, not the mean)
      const bool drop = nyq_zero && !zero_mode;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const T w = j < 3 ? T(1) : T(2);
        if (drop) rr += w * (sr[j] * sr[j] + si[j] * si[j]);
        orr[j] = drop ? T(0) : sr[j];
        oi[j] = drop ? T(0) : si[j];
      }
    }
    // compatible part: out = S - O away from k = 0; the residual S - out is then O
    if (compat && !zero_mode) {
      T o2n = T(0);
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const T w = j < 3 ? T(1) : T(2);
        o2n += w * (orr[j] * orr[j] + oi[j] * oi[j]);
        orr[j] = sr[j] - orr[j];
        oi[j] = si[j] - oi[j];
      }
      rr = o2n;
    }
    // norm terms (sums of |.|^2 over modes; Parseval turns them into voxel means)
    {
      T oo = T(0), dout = T(0);
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const T w = j < 3 ? T(1) : T(2);
        oo += w * (orr[j] * orr[j] + oi[j] * oi[j]);
      }
  #define EQ_DIV(S, ACC)                                                          \
      {                                                                          \
        const T d0 = xi0 * S[0] + xi1 * S[5] + xi2 * S[4];                       \
        const T d1 = xi0 * S[5] + xi1 * S[1] + xi2 * S[3];                       \
        const T d2 = xi0 * S[4] + xi1 * S[3] + xi2 * S[2];                       \
        ACC += d0 * d0 + d1 * d1 + d2 * d2;                                      \
      }
      EQ_DIV(orr, dout) EQ_DIV(oi, dout)
  #undef EQ_DIV
      const T m4 = T(0.25) * mult;                      // (1/2)^2 of the doubled components
      r2.add(m4 * rr);
      o2.add(m4 * oo);
      di2.add(m4 * din);
      do2.add(m4 * dout);
    }
    // repack: Zout_c(k) = O_2c + i O_2c+1, Zout_c(-k) = conj(O_2c) + i conj(O_2c+1), halved
    const T hv = T(0.5) * inv_v;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T or_ = orr[2 * c], oi_ = oi[2 * c], pr = orr[2 * c + 1], pi_ = oi[2 * c + 1];
      a[c] = T2{(or_ - pi_) * hv, (oi_ + pr) * hv};
      bb[c] = T2{(or_ + pi_) * hv, (pr - oi_) * hv};
    }
  }
}

// The Hodge potential y of one mode pair (k, -k) (Theorem 2): with n = xi / |xi|, v = S n and
// s = n . v, sym grad y reaches the part the projector removes when
// y_hat = -(i / |xi|) (2 v - s n); y_hat = 0 where xi = 0 (k = 0 and the Nyquist corners).
//   in:  a[c] = Z_c(k), bb[c] = Z_c(-k) of the stress spectrum (c = 0..2), as in project_pair
//   out: packed y spectra scaled by 1 / V: y01 = y0 + i y1 and y2 at k (yk[0], yk[1]) and at -k
//        (ym[0], ym[1]); y real gives y_c(-k) = conj(y_c(k)).
template <typename T, typename T2>
__device__ __forceinline__ void potential_pair(const T2 (&a)[3], const T2 (&bb)[3], T xi0, T xi1,
                                               T xi2, T inv_v, T2 (&yk)[2], T2 (&ym)[2]) {
  const T k2 = xi0 * xi0 + xi1 * xi1 + xi2 * xi2;
  if (!(k2 > T(0))) {
    yk[0] = yk[1] = ym[0] = ym[1] = T2{T(0), T(0)};
    return;
  }
  // doubled Voigt components, as in project_pair
  T sr[6], si[6];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    sr[2 * c] = a[c].x + bb[c].x;
    si[2 * c] = a[c].y - bb[c].y;
    sr[2 * c + 1] = a[c].y + bb[c].y;
    si[2 * c + 1] = bb[c].x - a[c].x;
  }
  const T rn = rsqrt_t(k2);
  const T n0 = xi0 * rn, n1 = xi1 * rn, n2 = xi2 * rn;
  // with the doubled S: 2 v - s n = V - (n . V / 2) n, V = (2 S) n; y_hat = (w_i - i w_r) / |xi|
  T wr[3], wi[3];
#define EQ_W(S, W)                                                              \
  {                                                                            \
    const T v0 = S[0] * n0 + S[5] * n1 + S[4] * n2;                            \
    const T v1 = S[5] * n0 + S[1] * n1 + S[3] * n2;                            \
    const T v2 = S[4] * n0 + S[3] * n1 + S[2] * n2;                            \
    const T hs = T(0.5) * (n0 * v0 + n1 * v1 + n2 * v2);                       \
    W[0] = v0 - hs * n0;                                                       \
    W[1] = v1 - hs * n1;                                                       \
    W[2] = v2 - hs * n2;                                                       \
  }
  EQ_W(sr, wr)
  EQ_W(si, wi)
#undef EQ_W
  const T f = rn * inv_v;                           // 1 / (|xi| V)
  T2 y[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) y[c] = T2{wi[c] * f, -wr[c] * f};
  yk[0] = T2{y[0].x - y[1].y, y[0].y + y[1].x};     // y0 + i y1 at k
  ym[0] = T2{y[0].x + y[1].y, y[1].x - y[0].y};     // conj(y0) + i conj(y1) at -k
  yk[1] = y[2];
  ym[1] = T2{y[2].x, -y[2].y};
}

// Fused x pass: forward transform of row pairs (k_y, k_z) and (-k_y, -k_z), projector on every
// mode pair (k, -k), inverse transform, store.  grid = (G, batch); block = Cfg::X_THREADS.
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<T, N>::X_THREADS)
k_xproj(const XArgs a) {
  using C = Cfg<T, N>;
  using T2 = typename C::T2;
  constexpr int E = C::E, TPC = C::TPC, P = C::P, PITCH = C::PITCH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* tw = reinterpret_cast<T2*>(smem_raw);
  T2* buf = tw + N;
  T* xix = reinterpret_cast<T*>(buf + C::XCOLS * PITCH);
  __shared__ double red[32 * 4];

  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tw[i] = reinterpret_cast<const T2*>(a.tw)[i];
    xix[i] = reinterpret_cast<const T*>(a.xi_x)[i];
  }
  __syncthreads();
  const T* xiy = reinterpret_cast<const T*>(a.xi_y);
  const T* xiz = reinterpret_cast<const T*>(a.xi_z);

  const int col = threadIdx.x / TPC, t = threadIdx.x % TPC;
  const int slot = col / 6, side = (col % 6) / 3, comp = col % 3;
  const int field = blockIdx.y;
  T* fdata = reinterpret_cast<T*>(a.data) + field * a.field_stride;
  T* pre = fdata + (2LL * comp) * a.V;
  T* pim = pre + a.V;
  T zmv[6];
  const T* zm = zero_mode_values(a.mean ? a.mean + field * 6 : nullptr, 1.0 / a.inv_v, zmv)
                    ? zmv : nullptr;
  const IdxRow idx{col * PITCH};
  const T inv_v = T(a.inv_v);

  Kahan<T> r2, di2, do2, o2;

  for (int g = blockIdx.x; g < a.ngroups; g += gridDim.x) {
    const int p = g * P + slot;
    const bool valid = p < a.npairs;
    int rowA = 0, rowB = 0;
    if (valid) {
      rowA = a.pairs[p];
      const int kz = rowA / a.ny, ky = rowA - kz * a.ny;
      const int mz = kz == 0 ? 0 : a.nz - kz, my = ky == 0 ? 0 : a.ny - ky;
      rowB = mz * a.ny + my;
    }
    const bool selfrow = rowA == rowB;
    const bool active = valid && !(side == 1 && selfrow);
    const long long roff = (long long)(side == 0 ? rowA : rowB) * N;
    T2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const long long off = roff + t + TPC * e;
      x[e] = active && in_bounds(off, a.V, a.err) ? T2{pre[off], pim[off]} : T2{T(0), T(0)};
    }
    fft_column<N, E, false>(x, t, buf, idx, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) buf[idx(t + TPC * e)] = x[e];
    __syncthreads();

    for (int item = threadIdx.x; item < P * N; item += blockDim.x) {
      const int s2 = item / N, kx = item - s2 * N;
      const int p2 = g * P + s2;
      if (p2 >= a.npairs) continue;
      const int rA = a.pairs[p2];
      const int kz = rA / a.ny, ky = rA - kz * a.ny;
      const int mz = kz == 0 ? 0 : a.nz - kz, my = ky == 0 ? 0 : a.ny - ky;
      const bool self2 = (mz * a.ny + my) == rA;
      const int kxm = kx == 0 ? 0 : N - kx;
      if (self2 && kx > kxm) continue;
      const int colA = s2 * 6, colB = self2 ? s2 * 6 : s2 * 6 + 3;
      T2 av[3], bv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        av[c] = buf[(colA + c) * PITCH + kx + (kx >> 3)];
        bv[c] = buf[(colB + c) * PITCH + kxm + (kxm >> 3)];
      }
      const bool selfmode = self2 && kx == kxm;
      const bool zero_mode = (rA == 0) && kx == 0;
      project_pair<T>(av, bv, xix[kx], xiy[ky], xiz[kz], zero_mode, zm, a.nyq_zero != 0,
                      a.compat != 0, inv_v, selfmode ? T(1) : T(2), r2, di2, do2, o2);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        buf[(colA + c) * PITCH + kx + (kx >> 3)] = av[c];
        if (!selfmode) buf[(colB + c) * PITCH + kxm + (kxm >> 3)] = bv[c];
      }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = buf[idx(t + TPC * e)];
    __syncthreads();
    fft_column<N, E, true>(x, t, buf, idx, tw);
    if (active) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const long long off = roff + t + TPC * e;
        if (!in_bounds(off, a.V, a.err)) continue;
        pre[off] = x[e].x;
        pim[off] = x[e].y;
      }
    }
  }
  double v[4] = {r2.value(), di2.value(), do2.value(), o2.value()};
  block_sum<4>(v, red);
  if (threadIdx.x == 0) {
    double* q = a.partials + ((long long)field * gridDim.x + blockIdx.x) * 4;
    q[0] = v[0]; q[1] = v[1]; q[2] = v[2]; q[3] = v[3];
  }
}


// Potential x pass: reads the stress spectrum after the z and y forward passes (not modifying
// it), takes the forward x transform of each row pair, forms the packed y spectra per mode pair
// (potential_pair) and writes their inverse x transforms into the 4-plane y buffer (y0 + i y1 in
// planes 0/1, y2 + i 0 in planes 2/3).  Same row-pair layout as k_xproj; only the columns of
// components 0 and 1 of each side carry y back out.
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<T, N>::X_THREADS)
k_xpot(const XArgs a) {
  using C = Cfg<T, N>;
  using T2 = typename C::T2;
  constexpr int E = C::E, TPC = C::TPC, P = C::P, PITCH = C::PITCH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* tw = reinterpret_cast<T2*>(smem_raw);
  T2* buf = tw + N;
  T* xix = reinterpret_cast<T*>(buf + C::XCOLS * PITCH);

  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tw[i] = reinterpret_cast<const T2*>(a.tw)[i];
    xix[i] = reinterpret_cast<const T*>(a.xi_x)[i];
  }
  __syncthreads();
  const T* xiy = reinterpret_cast<const T*>(a.xi_y);
  const T* xiz = reinterpret_cast<const T*>(a.xi_z);

  const int col = threadIdx.x / TPC, t = threadIdx.x % TPC;
  const int slot = col / 6, side = (col % 6) / 3, comp = col % 3;
  const int field = blockIdx.y;
  const T* fdata = reinterpret_cast<const T*>(a.data) + field * a.field_stride;
  const T* pre = fdata + (2LL * comp) * a.V;
  const T* pim = pre + a.V;
  T* yre = reinterpret_cast<T*>(a.ydata) + field * a.yfield_stride + (2LL * (comp & 1)) * a.V;
  T* yim = yre + a.V;
  const IdxRow idx{col * PITCH};
  const T inv_v = T(a.inv_v);

  for (int g = blockIdx.x; g < a.ngroups; g += gridDim.x) {
    const int p = g * P + slot;
    const bool valid = p < a.npairs;
    int rowA = 0, rowB = 0;
    if (valid) {
      rowA = a.pairs[p];
      const int kz = rowA / a.ny, ky = rowA - kz * a.ny;
      const int mz = kz == 0 ? 0 : a.nz - kz, my = ky == 0 ? 0 : a.ny - ky;
      rowB = mz * a.ny + my;
    }
    const bool selfrow = rowA == rowB;
    const bool active = valid && !(side == 1 && selfrow);
    const long long roff = (long long)(side == 0 ? rowA : rowB) * N;
    T2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const long long off = roff + t + TPC * e;
      x[e] = active && in_bounds(off, a.V, a.err) ? T2{pre[off], pim[off]} : T2{T(0), T(0)};
    }
    fft_column<N, E, false>(x, t, buf, idx, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) buf[idx(t + TPC * e)] = x[e];
    __syncthreads();

    for (int item = threadIdx.x; item < P * N; item += blockDim.x) {
      const int s2 = item / N, kx = item - s2 * N;
      const int p2 = g * P + s2;
      if (p2 >= a.npairs) continue;
      const int rA = a.pairs[p2];
      const int kz = rA / a.ny, ky = rA - kz * a.ny;
      const int mz = kz == 0 ? 0 : a.nz - kz, my = ky == 0 ? 0 : a.ny - ky;
      const bool self2 = (mz * a.ny + my) == rA;
      const int kxm = kx == 0 ? 0 : N - kx;
      if (self2 && kx > kxm) continue;
      const int colA = s2 * 6, colB = self2 ? s2 * 6 : s2 * 6 + 3;
      T2 av[3], bv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        av[c] = buf[(colA + c) * PITCH + kx + (kx >> 3)];
        bv[c] = buf[(colB + c) * PITCH + kxm + (kxm >> 3)];
      }
      T2 yk[2], ym[2];
      potential_pair<T>(av, bv, xix[kx], xiy[ky], xiz[kz], inv_v, yk, ym);
      // this mode pair owns (row A, kx) and (row B, kxm) of every column: store in place
      const bool selfmode = self2 && kx == kxm;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        buf[(colA + c) * PITCH + kx + (kx >> 3)] = yk[c];
        if (!selfmode) buf[(colB + c) * PITCH + kxm + (kxm >> 3)] = ym[c];
      }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = buf[idx(t + TPC * e)];
    __syncthreads();
    fft_column<N, E, true>(x, t, buf, idx, tw);
    if (active && comp < 2) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const long long off = roff + t + TPC * e;
        if (!in_bounds(off, a.V, a.err)) continue;
        yre[off] = x[e].x;
        yim[off] = x[e].y;
      }
    }
  }
}

}  // namespace eqk
