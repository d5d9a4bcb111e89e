// eq_fft.cuh - register/shared-memory FFT core for power-of-two lengths (device code).
//
// One transform of length N is held by TPC = N / E threads, E complex elements each: thread t
// holds element t + TPC * e in register slot e.  A Stockham autosort schedule runs log_R(N)
// stages of radix R in {8, 4, 2}; in the stage with span Ns the butterfly j reads elements
// j + r N/R (which are exactly register slots q + r E/R of thread t = j mod TPC), multiplies
// leg r by W_{Ns R}^{r (j mod Ns)} and writes its outputs to (j / Ns) Ns R + (j mod Ns) + r Ns.
// Between stages the outputs go through shared memory; after the last stage every output is
// back in the register slot of its natural index, so the caller can store it directly.
//
// The forward transform is unnormalised with exp(-2 pi i m x / N); the inverse uses
// exp(+2 pi i m x / N) without the 1/N factor (the projector applies 1/(nx ny nz) once).
#pragma once
#include <cuda_runtime.h>

namespace eqk {

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return {a.x + b.x, a.y + b.y}; }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return {a.x - b.x, a.y - b.y}; }
// FP32: one packed two-lane instruction (sm_100 and later) for both parts, rounded like the
// scalar operations
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
// r + s * v for a real s, both parts
template <typename T2, typename T> __device__ __forceinline__ T2 cfma_s(T s, T2 v, T2 r) {
  return {r.x + s * v.x, r.y + s * v.y};
}
__device__ __forceinline__ float2 cfma_s(float s, float2 v, float2 r) {
  return __ffma2_rn(make_float2(s, s), v, r);
}
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename T2> __device__ __forceinline__ T2 mul_mi(T2 a) {
  return INV ? T2{-a.y, a.x} : T2{a.y, -a.x};
}

template <bool INV, typename T2> __device__ __forceinline__ void dft2(T2* v) {
  T2 a = v[0];
  v[0] = cadd(a, v[1]);
  v[1] = csub(a, v[1]);
}

// X_r = sum_m v_m W4^{r m}, W4 = exp(-+ 2 pi i / 4)
template <bool INV, typename T2> __device__ __forceinline__ void dft4(T2* v) {
  T2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  T2 s13 = cadd(v[1], v[3]), d13 = mul_mi<INV>(csub(v[1], v[3]));
  v[0] = cadd(s02, s13);
  v[2] = csub(s02, s13);
  v[1] = cadd(d02, d13);
  v[3] = csub(d02, d13);
}

// radix 8 as two radix-4 transforms of the sums / twiddled differences of v_m and v_{m+4}
template <bool INV, typename T2> __device__ __forceinline__ void dft8(T2* v) {
  using T = decltype(v[0].x);
  const T h = T(0.70710678118654752440);
  T2 a[4], b[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    a[m] = cadd(v[m], v[m + 4]);
    b[m] = csub(v[m], v[m + 4]);
  }
  // b_m *= W8^m
  b[1] = INV ? T2{h * (b[1].x - b[1].y), h * (b[1].x + b[1].y)}
             : T2{h * (b[1].x + b[1].y), h * (b[1].y - b[1].x)};
  b[2] = mul_mi<INV>(b[2]);
  b[3] = INV ? T2{-h * (b[3].x + b[3].y), h * (b[3].x - b[3].y)}
             : T2{h * (b[3].y - b[3].x), -h * (b[3].x + b[3].y)};
  dft4<INV>(a);
  dft4<INV>(b);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[2 * q] = a[q];
    v[2 * q + 1] = b[q];
  }
}

// cos(pi j / 16), j = 0..8; W32^q = cos(2 pi q / 32) -+ i sin(2 pi q / 32) follows by symmetry
__host__ __device__ constexpr double cos_pi16(int j) {
  constexpr double c[9] = {1.0,
                           0.9807852804032304491262,
                           0.9238795325112867561282,
                           0.8314696123025452370788,
                           0.7071067811865475244008,
                           0.5555702330196022247428,
                           0.3826834323650897717285,
                           0.1950903220161282678483,
                           0.0};
  return j <= 8 ? c[j] : -c[16 - j];                // j in 0..16
}
__host__ __device__ constexpr double sin_pi16(int j) {  // j in 0..16
  return j <= 8 ? cos_pi16(8 - j) : cos_pi16(j - 8);
}
// v * W32^q (forward: exp(-2 pi i q / 32); INV: the conjugate), q in 0..15, trivial q skip the
// multiply
template <int Q, bool INV, typename T2> __device__ __forceinline__ T2 mul_w32(T2 v) {
  using T = decltype(v.x);
  if constexpr (Q == 0) {
    return v;
  } else if constexpr (Q == 8) {
    return mul_mi<INV>(v);
  } else {
    constexpr T c = T(cos_pi16(Q));
    constexpr T s = INV ? T(sin_pi16(Q)) : T(-sin_pi16(Q));
    return T2{v.x * c - v.y * s, v.x * s + v.y * c};
  }
}

// v * W32^q for a q known after unrolling (dispatch to the constant forms)
template <bool INV, typename T2> __device__ __forceinline__ T2 mul_w32_rt(int q, T2 v) {
  switch (q) {
    case 1: return mul_w32<1, INV>(v);
    case 2: return mul_w32<2, INV>(v);
    case 3: return mul_w32<3, INV>(v);
    case 4: return mul_w32<4, INV>(v);
    case 5: return mul_w32<5, INV>(v);
    case 6: return mul_w32<6, INV>(v);
    case 7: return mul_w32<7, INV>(v);
    case 8: return mul_w32<8, INV>(v);
    case 9: return mul_w32<9, INV>(v);
    case 10: return mul_w32<10, INV>(v);
    case 11: return mul_w32<11, INV>(v);
    case 12: return mul_w32<12, INV>(v);
    case 13: return mul_w32<13, INV>(v);
    case 14: return mul_w32<14, INV>(v);
    case 15: return mul_w32<15, INV>(v);
    default: return v;
  }
}

// radix 16 as two radix-8 transforms of the sums / W16-twiddled differences of v_m and v_{m+8};
// outputs in natural order
template <bool INV, typename T2> __device__ __forceinline__ void dft16(T2* v) {
  T2 a[8], b[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    a[m] = cadd(v[m], v[m + 8]);
    b[m] = csub(v[m], v[m + 8]);
  }
  b[1] = mul_w32<2, INV>(b[1]);
  b[2] = mul_w32<4, INV>(b[2]);
  b[3] = mul_w32<6, INV>(b[3]);
  b[4] = mul_w32<8, INV>(b[4]);
  b[5] = mul_w32<10, INV>(b[5]);
  b[6] = mul_w32<12, INV>(b[6]);
  b[7] = mul_w32<14, INV>(b[7]);
  dft8<INV>(a);
  dft8<INV>(b);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    v[2 * q] = a[q];
    v[2 * q + 1] = b[q];
  }
}

template <int R, bool INV, typename T2> __device__ __forceinline__ void dftR(T2* v) {
  if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v);
  else if constexpr (R == 2) dft2<INV>(v);
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
// radix of stage s for N = 2^L: 8 while three or more bits remain, then 4 or 2
__host__ __device__ constexpr int stage_radix(int N, int s) {
  int rem = ilog2(N);
  for (int i = 0; i < s; ++i) rem -= (rem >= 3 ? 3 : rem);
  return rem >= 3 ? 8 : (rem == 2 ? 4 : (rem == 1 ? 2 : 1));
}
__host__ __device__ constexpr int num_stages(int N) {
  int rem = ilog2(N), s = 0;
  while (rem > 0) { rem -= (rem >= 3 ? 3 : rem); ++s; }
  return s;
}
__host__ __device__ constexpr int stage_span(int N, int s) {  // Ns before stage s
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= stage_radix(N, i);
  return ns;
}

// Per-stage twiddle tables: offset of the table of the stage with span NS (stages with NS > 1
// hold NS (R - 1) entries) and their total size.
__host__ __device__ constexpr int staged_offset(int N, int NS) {
  int off = 0, ns = 1, s = 0;
  while (ns < NS) {
    const int R = stage_radix(N, s);
    if (ns > 1) off += ns * (R - 1);
    ns *= R;
    ++s;
  }
  return off;
}
__host__ __device__ constexpr int staged_size(int N) { return staged_offset(N, N); }

// Twiddle sources of a stage: the plain table tw[m] = W_N^m (any layout), or per-stage tables
// laid out [k][r - 1] for k < Ns (consecutive k are consecutive threads in the x pass, so a warp
// reads consecutive words: no shared-memory bank conflicts), split into cos and sin arrays.
template <typename T2> struct TwPlain {
  const T2* tw;
  template <int N, int NS, int R>
  __device__ __forceinline__ T2 get(int k, int r) const { return tw[(r * k) * (N / (NS * R))]; }
};
template <typename T> struct TwStaged {
  const T* c;   // cos, all stages back to back
  const T* s;   // sin
  // offset of stage table with span NS: sum of NS' (R' - 1) over earlier stages
  template <int N, int NS, int R>
  __device__ __forceinline__ typename V2<T>::t get(int k, int r) const {
    constexpr int off = staged_offset(N, NS);
    const int i = off + k * (R - 1) + (r - 1);
    return {c[i], s[i]};
  }
};



// One Stockham stage on the thread's registers; leaves outputs in the same slots.
template <int N, int E, int S, bool INV, typename T2, typename TW>
__device__ __forceinline__ void fft_stage(T2 (&x)[E], int t, const TW& tw) {
  constexpr int R = stage_radix(N, S);
  constexpr int NS = stage_span(N, S);
  constexpr int TPC = N / E;
  constexpr int Q = E / R;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    T2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[q + r * Q];
    if constexpr (NS > 1) {
      const int k = (t + TPC * q) & (NS - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        T2 w = tw.template get<N, NS, R>(k, r);
        if (INV) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    dftR<R, INV>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) x[q + r * Q] = v[r];
  }
}

// Output position of register slot (q, r) after stage S, for thread t.
template <int N, int E, int S>
__device__ __forceinline__ int stage_out_pos(int t, int q, int r) {
  constexpr int R = stage_radix(N, S);
  constexpr int NS = stage_span(N, S);
  constexpr int TPC = N / E;
  const int j = t + TPC * q;
  return (j / NS) * NS * R + (j & (NS - 1)) + r * NS;
}

// Exchange storage between stages: interleaved complex through an index map, or split real and
// imaginary arrays with a bank swizzle (for the x pass, whose warps run along one transform).
template <typename T2, typename IDX> struct AosAcc {
  T2* buf;
  IDX idx;
  __device__ __forceinline__ void put(int i, T2 v) const { buf[idx(i)] = v; }
  __device__ __forceinline__ T2 get(int i) const { return buf[idx(i)]; }
};
// Split real/imaginary rows of N words, element i stored at swz(i): an XOR of the low five bits
// with bits 5..7 of i, so the contiguous, stage-output and projector access patterns of a warp
// (32 consecutive threads of one transform) touch 32 distinct banks.
__host__ __device__ __forceinline__ int swz(int i) { return i ^ ((i >> 5) & 7) ^ (((i >> 6) & 3) << 3); }
// Spectrum rows of the 512-point warp transform, interleaved complex (8-byte words, served 16
// lanes per wavefront): element i at i ^ (bit 8 of i moved to bit 3), so that the transform's
// output stores (lanes 2 kap + h write kap + 16 q + 256 h), its input loads (l + 32 e) and the
// projector's runs of consecutive modes touch 16 distinct word pairs in each half-warp.
__host__ __device__ __forceinline__ int sx512(int i) { return i ^ (((i >> 8) & 1) << 3); }
template <typename T> struct SoaAcc {
  T* re;
  T* im;
  __device__ __forceinline__ void put(int i, typename V2<T>::t v) const {
    const int j = swz(i);
    re[j] = v.x;
    im[j] = v.y;
  }
  __device__ __forceinline__ typename V2<T>::t get(int i) const {
    const int j = swz(i);
    return {re[j], im[j]};
  }
};

// Full transform of one column through the accessor `acc`.  WARP = false synchronises the block
// between exchange writes and reads; WARP = true only the warp (the column's TPC = 32 threads are
// one warp and its exchange storage is private to it).  On entry the caller guarantees that the
// exchange storage is no longer being read from any earlier use.
template <int N, int E, bool INV, int S = 0, bool WARP = false, typename T2, typename ACC, typename TW>
__device__ __forceinline__ void fft_column_acc(T2 (&x)[E], int t, const ACC& acc, const TW& tw) {
  if constexpr (S < num_stages(N)) {
    fft_stage<N, E, S, INV>(x, t, tw);
    if constexpr (S + 1 < num_stages(N)) {
      constexpr int R = stage_radix(N, S);
      constexpr int Q = E / R;
#pragma unroll
      for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) acc.put(stage_out_pos<N, E, S>(t, q, r), x[q + r * Q]);
      if constexpr (WARP) __syncwarp(); else __syncthreads();
      constexpr int TPC = N / E;
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = acc.get(t + TPC * e);
      if constexpr (WARP) __syncwarp(); else __syncthreads();
      fft_column_acc<N, E, INV, S + 1, WARP>(x, t, acc, tw);
    }
  }
}

// Interleaved-complex exchange through `idx(i)`, twiddles from the plain table.
template <int N, int E, bool INV, typename T2, typename IDX>
__device__ __forceinline__ void fft_column(T2 (&x)[E], int t, T2* buf, const IDX& idx,
                                           const T2* __restrict__ tw) {
  fft_column_acc<N, E, INV>(x, t, AosAcc<T2, IDX>{buf, idx}, TwPlain<T2>{tw});
}

// 512-point transform of one row held by one warp, lane l holding point l + 32 e in slot e
// (e < 16).  With n = l + 32 e and k = k1 + 16 k2 (k1 < 16, k2 < 32):
//   1. a 16-point DFT over e in registers: Y_l[k1];
//   2. Y_l[k1] *= W512^(l k1) (tw = 16 x 32 table [k1][l] of the forward factors);
//   3. one exchange through the warp's row (512 interleaved complex values): Y_l[k1] stored at
//      32 k1 + (l ^ 2 k1), so that both the store (fixed k1) and the load below are
//      conflict-free in each half-warp;
//   4. lane L = 2 kap + h loads Y_{h + 2 m}[kap], m < 16, and takes a 16-point DFT over m:
//      Z_h[q] for the even (h = 0) and odd (h = 1) halves of the 32-point DFT over l;
//   5. lanes L and L ^ 1 combine by shuffle: X[kap + 16 q + 256 h] = Z_0[q] +- W32^q Z_1[q].
// On return slot q of lane L holds output kap + 16 q + 256 h.  The caller guarantees that no lane
// still reads the row on entry; the row is free again on return.
template <bool INV, typename T2>
__device__ __forceinline__ void fft512_warp(T2 (&v)[16], int lane, T2* buf,
                                            const T2* __restrict__ tw) {
  using T = decltype(v[0].x);
  dft16<INV>(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) {
    T2 w = tw[k1 * 32 + lane];
    if (INV) w.y = -w.y;
    v[k1] = cmul(v[k1], w);
  }
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) {
    buf[k1 * 32 + (lane ^ (2 * k1))] = v[k1];
  }
  __syncwarp();
  const int kap = lane >> 1, h = lane & 1;
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    v[m] = buf[kap * 32 + h + 2 * (m ^ kap)];
  }
  __syncwarp();
  dft16<INV>(v);
  const T sg = h ? T(-1) : T(1);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    // lane h = 1 sends W32^q Z_1[q], lane h = 0 sends Z_0[q]; each adds +- its own value
    const T2 t = mul_w32_rt<INV>(q, v[q]);
    const T2 send = h ? t : v[q];
    T2 recv;
    recv.x = __shfl_xor_sync(0xffffffffu, send.x, 1);
    recv.y = __shfl_xor_sync(0xffffffffu, send.y, 1);
    v[q] = cfma_s(sg, send, recv);
  }
}

// Plain running sum (a short per-thread partial, folded into a Kahan sum by the caller).
template <typename T> struct PlainSum {
  T s = T(0);
  __device__ __forceinline__ void add(T v) { s += v; }
};

// Kahan-compensated FP32/FP64 running sum (per-thread partial of a global FP64 reduction).
template <typename T> struct Kahan {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T v) {
    T y = v - c;
    T tt = s + y;
    c = (tt - s) - y;
    s = tt;
  }
  __device__ __forceinline__ double value() const { return double(s) - double(c); }
};

}  // namespace eqk
