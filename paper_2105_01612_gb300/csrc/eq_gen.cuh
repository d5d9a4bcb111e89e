// eq_gen.cuh - runtime-length FFT passes for any grid size and for batches of uneven fields.
//
// Lengths whose prime factors are all in {2, 3, 5, 7, 11, 13} run a mixed-radix Stockham
// schedule; any other length n runs Bluestein's chirp-z algorithm: with c_j = exp(-pi i j^2/n),
// X_k = c_k sum_j (x_j c_j) conj(c_{k-j}), a circular convolution of length m >= 2n - 1 done with
// two length-m transforms and the precomputed transform of the chirp.  Inverse transforms use
// X = conj(DFT(conj(x))).  A block holds C transforms ("columns") in shared memory laid out
// [element][column] with a padded pitch and ping-pongs between two buffers, one barrier per stage.
//
// Work items: a pass over a list of fields enumerates (field, component, chunk of column tiles)
// or (field, chunk of x-row pairs); each item's warps write their own FP64 partial records, so
// every reduction is a fixed-order sum (bitwise reproducible, independent of the other fields).
#pragma once
#include <cuda_runtime.h>

#include "../../include/eq.h"
#include "eq_kernels.cuh"
#include "eq_pfft.cuh"
#include "eq_dd.cuh"

namespace eqg {

using eqk::cadd;
using eqk::cmul;
using eqk::csub;
using eqk::Kahan;

constexpr int MAXST = 20;
constexpr int WARPS_MAX = 32;

struct AxisPlan {
  int n;              // logical length
  int m;              // transform length (n, or the Bluestein length)
  int blue;           // 1 = Bluestein
  int nst;            // number of stages of the length-m schedule
  int radix[MAXST];
  int tw;             // offset (complex entries) of exp(-2 pi i j / m), j < m, in the pool
  int chirp;          // Bluestein: n entries c_j = exp(-pi i j^2 / n)
  int bhat;           // Bluestein: m entries DFT_m(conj c, wrapped) / m
  int fast;           // 1: m is a power of two served by the fixed-size register FFT when the
                      //    pass shape gives it a compiled (m, points per thread) instance
  // warp-per-row x pass (k_gen_xrows): transform length wm (256 or 512; 0 = not served), n itself
  // for n = wm, else Bluestein with the tables below
  int wm;
  int wchirp;         // n entries c_j (complex pool), -1 when wm == n
  int wbhat;          // wm entries DFT_wm(conj c, wrapped) / wm, -1 when wm == n
  int wtw;            // staged twiddles of the length-wm radix-8 schedule as complex (cos, sin)
};

struct FieldDesc {
  long long in_off;   // element offset of the field (plane 0) in the input buffer
  long long out_off;  // element offset in the output buffer
  long long V;        // nx ny nz
  int nx, ny, nz;
  int ax[3];          // axis plans of x, y, z
  int xi[3];          // offsets of the operator symbol tables (real entries) in the xi pool
  int pairs;          // offset of the canonical x-row pairs in the pair pool
  int npairs;
};

struct GenArgs {
  const void* in;          // input buffer base (first pass) / output base (others)
  void* out;
  const void* ref;         // last pass: input for L-inf (nullptr = skip)
  const FieldDesc* fields;
  const AxisPlan* axes;
  const void* cpool;       // complex pool: twiddles, chirps, chirp transforms
  const void* xipool;      // real pool: operator symbols
  const int* pairpool;
  const double* mean;      // [F][6]
  const long long* item0;  // [F + 1] first work item of each field for this pass
  double* partials;        // [items][WARPS][4]
  int nfields;
  long long nitems;
  int axis;                // 1 = y, 2 = z for strided passes
  int mode;                // 0 middle, 1 first, 2 last (strided)
  int tiles_per_item;      // strided: column tiles of C columns per item; x: row-pair groups
  int cols;                // C: columns per tile
  int pitch;               // shared-memory pitch (>= C)
  int mmax;                // largest transform length among the fields
  int nyq_zero;
  int compat;              // 1: return the compatible part c0 + (S - S_equil)
  int* err;                // plan error word (bounds-checked builds)
  int tw256;               // complex pool: staged twiddles of length 256 (k_gen_scols)
  int w512;                // complex pool: W512^j, j < 256 (k_gen_scols)
  int io;                  // double-float plans: bit 0 this pass reads FP64, bit 1 it writes FP64
                           // (the pipeline's ends); the passes between hold double-float pairs
};

// FP64 at the ends of a double-float pipeline (the first pass's loads are converted on the bits
// in k_gen_scold): the last pass's re-read of the input and its stores, converted on the FP64
// units (the faster form for each, as measured); between the passes, double-float pairs.
__device__ __forceinline__ eqk::dd ld_f64(const eqk::dd* p, long long i) {
  return eqk::dd_from_f64(reinterpret_cast<const double*>(p)[i]);
}
__device__ __forceinline__ void st_dd(eqk::dd* p, long long i, eqk::dd v, bool f64) {
  if (f64) reinterpret_cast<double*>(p)[i] = eqk::dd_to_f64(v);
  else p[i] = v;
}

// ---- small DFTs -------------------------------------------------------------------------

template <int R, bool INV, typename T2>
__device__ __forceinline__ void dft_small(T2 (&v)[R], const T2 (&wr)[R]) {
  if constexpr (R == 2) eqk::dft2<INV>(v);
  else if constexpr (R == 4) eqk::dft4<INV>(v);
  else if constexpr (R == 8) eqk::dft8<INV>(v);
  else {
    // direct R-point DFT with the R-th roots wr[q] = W_R^q (already conjugated for INV)
    T2 o[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      T2 acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], wr[(r * q) % R]));
      o[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = o[q];
  }
}

// one Stockham stage of radix R over C columns: src -> dst.  blockDim.x must be a multiple of C;
// thread t works on column t % C and butterflies t / C, t / C + blockDim.x / C, ...
template <int R, bool INV, typename T2>
__device__ __forceinline__ void gen_stage(const T2* __restrict__ src, T2* __restrict__ dst, int m,
                                          int ns, int C, int pitch, const T2* __restrict__ tw,
                                          int* err = nullptr) {
  const int nb = m / R;
  const int tstep = m / (ns * R);
  const int col = threadIdx.x % C, jstep = blockDim.x / C;
  T2 wr[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    T2 w = tw[q * nb];
    if (INV) w.y = -w.y;
    wr[q] = w;
  }
  for (int j = threadIdx.x / C; j < nb; j += jstep) {
    T2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int ix = (j + r * nb) * pitch + col;
      v[r] = eqk::in_bounds(ix, (long long)m * pitch, err) ? src[ix] : T2{};
    }
    const int k = j % ns;
    if (ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        T2 t = tw[r * k * tstep];
        if (INV) t.y = -t.y;
        v[r] = cmul(v[r], t);
      }
    }
    dft_small<R, INV>(v, wr);
    const int base = (j / ns) * ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int ix = (base + r * ns) * pitch + col;
      if (eqk::in_bounds(ix, (long long)m * pitch, err)) dst[ix] = v[r];
    }
  }
}

// Length-m transform of C columns; data starts in a, returns the buffer holding the result.
template <bool INV, typename T2>
__device__ T2* gen_fft(T2* a, T2* b, const AxisPlan& ap, int C, int pitch, const T2* tw,
                       int* err = nullptr) {
  int ns = 1;
  for (int s = 0; s < ap.nst; ++s) {
    const int R = ap.radix[s];
    switch (R) {
      case 2: gen_stage<2, INV>(a, b, ap.m, ns, C, pitch, tw, err); break;
      case 3: gen_stage<3, INV>(a, b, ap.m, ns, C, pitch, tw, err); break;
      case 4: gen_stage<4, INV>(a, b, ap.m, ns, C, pitch, tw, err); break;
      case 5: gen_stage<5, INV>(a, b, ap.m, ns, C, pitch, tw, err); break;
      case 7: gen_stage<7, INV>(a, b, ap.m, ns, C, pitch, tw, err); break;
      case 8: gen_stage<8, INV>(a, b, ap.m, ns, C, pitch, tw, err); break;
      case 11: gen_stage<11, INV>(a, b, ap.m, ns, C, pitch, tw, err); break;
      case 13: gen_stage<13, INV>(a, b, ap.m, ns, C, pitch, tw, err); break;
      default: break;
    }
    __syncthreads();
    ns *= R;
    T2* t = a; a = b; b = t;
  }
  return a;
}

// Per-item copy of an axis plan's tables into shared memory: twiddles (m), chirp (n), chirp
// transform (m).
template <typename T2>
__device__ __forceinline__ void load_tables(const AxisPlan& ap, const T2* __restrict__ cpool,
                                            T2* tws, T2* chs, T2* bhs) {
  for (int i = threadIdx.x; i < ap.m; i += blockDim.x) {
    tws[i] = cpool[ap.tw + i];
    if (ap.blue) bhs[i] = cpool[ap.bhat + i];
  }
  if (ap.blue)
    for (int i = threadIdx.x; i < ap.n; i += blockDim.x) chs[i] = cpool[ap.chirp + i];
}

// Power-of-two length M with the fixed-size register FFT of the compile-time passes: thread
// (col, t) = (tid % C, tid / C) holds elements t + (M / E) e of column col (E per thread, so
// blockDim = C M / E), exchanging through b.  Bluestein: forward, times the chirp transform,
// inverse (the inverse direction is handled by the caller's conjugation); otherwise one transform.
// Leaves the outputs in a (natural order) behind a barrier and returns a.
template <int M, int E, typename T2>
__device__ __noinline__ T2* fast_transform(T2* a, T2* b, int C, int pitch, const T2* tws,
                                           const T2* bhs, bool blue, bool inv) {
  constexpr int TPC = M / E;
  const int col = threadIdx.x % C, t = threadIdx.x / C;
  T2 x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) x[e] = a[(t + TPC * e) * pitch + col];
  const eqk::IdxStrided idx{col, pitch};
  if (blue) {
    eqk::fft_column<M, E, false>(x, t, b, idx, tws);
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = cmul(x[e], bhs[t + TPC * e]);
    eqk::fft_column<M, E, true>(x, t, b, idx, tws);
  } else if (inv) {
    eqk::fft_column<M, E, true>(x, t, b, idx, tws);
  } else {
    eqk::fft_column<M, E, false>(x, t, b, idx, tws);
  }
#pragma unroll
  for (int e = 0; e < E; ++e) a[(t + TPC * e) * pitch + col] = x[e];
  __syncthreads();
  return a;
}

// The compiled (M, E) instances; nullptr when the pass shape has none (runtime stages then).
template <typename T2>
__device__ __forceinline__ T2* fast_dispatch(T2* a, T2* b, const AxisPlan& ap, int C, int pitch,
                                             const T2* tws, const T2* bhs, bool inv) {
  const int tpc = blockDim.x / C;
  const int e = ap.m / tpc;
  if (tpc * C != (int)blockDim.x || e * tpc != ap.m) return nullptr;
  const bool blue = ap.blue != 0;
  switch (ap.m * 64 + e) {
    case 128 * 64 + 8: return fast_transform<128, 8>(a, b, C, pitch, tws, bhs, blue, inv);
    case 256 * 64 + 8: return fast_transform<256, 8>(a, b, C, pitch, tws, bhs, blue, inv);
    case 256 * 64 + 16: return fast_transform<256, 16>(a, b, C, pitch, tws, bhs, blue, inv);
    case 512 * 64 + 8: return fast_transform<512, 8>(a, b, C, pitch, tws, bhs, blue, inv);
    case 512 * 64 + 16: return fast_transform<512, 16>(a, b, C, pitch, tws, bhs, blue, inv);
    case 1024 * 64 + 16: return fast_transform<1024, 16>(a, b, C, pitch, tws, bhs, blue, inv);
    default: return nullptr;
  }
}

// Full axis transform of the C columns held in `a` (element-major, pitch `pitch`).  For Bluestein
// the caller has already multiplied by the chirp and zero-filled [n, m).  Returns the buffer with
// the outputs (before the Bluestein post-chirp, see post()).
template <typename T2>
__device__ T2* axis_transform(T2* a, T2* b, const AxisPlan& ap, int C, int pitch, const T2* tws,
                              const T2* bhs, bool inv, int* err = nullptr) {
  if (ap.fast) {
    T2* r = fast_dispatch(a, b, ap, C, pitch, tws, bhs, inv);
    if (r) return r;
  }
  if (!ap.blue)
    return inv ? gen_fft<true>(a, b, ap, C, pitch, tws, err) : gen_fft<false>(a, b, ap, C, pitch, tws, err);
  T2* r = gen_fft<false>(a, b, ap, C, pitch, tws, err);
  T2* o = (r == a) ? b : a;
  const int col = threadIdx.x % C, jstep = blockDim.x / C;
  for (int k = threadIdx.x / C; k < ap.m; k += jstep) r[k * pitch + col] = cmul(r[k * pitch + col], bhs[k]);
  __syncthreads();
  return gen_fft<true>(r, o, ap, C, pitch, tws, err);
}

// value to place in the work buffer for input element j of a transform (pre-chirp, conj trick)
template <typename T2>
__device__ __forceinline__ T2 pre(T2 x, int j, const AxisPlan& ap, const T2* chs, bool inv) {
  if (!ap.blue) return x;
  if (inv) x.y = -x.y;
  return cmul(x, chs[j]);
}
template <typename T2>
__device__ __forceinline__ T2 post(T2 y, int k, const AxisPlan& ap, const T2* chs, bool inv) {
  if (!ap.blue) return y;
  T2 r = cmul(y, chs[k]);
  if (inv) r.y = -r.y;
  return r;
}

__device__ __forceinline__ int find_field(const long long* item0, int nf, long long item) {
  int lo = 0, hi = nf - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (item0[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int K>
__device__ __forceinline__ void warp_partials(double (&v)[K], double* dst) {
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) dst[(threadIdx.x >> 5) * K + k] = v[k];
}

// Shared memory of the runtime-length kernels: two work buffers of mmax x pitch, then the
// per-item tables (twiddles, chirp, chirp transform: mmax entries each).
template <typename T2> struct GenSmem {
  T2 *a, *b, *tw, *ch, *bh;
  __device__ GenSmem(unsigned char* raw, int mmax, int pitch) {
    a = reinterpret_cast<T2*>(raw);
    b = a + (size_t)mmax * pitch;
    tw = b + (size_t)mmax * pitch;
    ch = tw + mmax;
    bh = ch + mmax;
  }
};

// Strided pass (axis y or z) over a list of fields, any lengths.
// Item = (field, component, chunk of tiles_per_item tiles of C consecutive columns).
// blockDim.x must be a multiple of C.
template <typename T, bool INV>
__global__ void __launch_bounds__(512) k_gen_strided(const GenArgs a) {
  using T2 = typename eqk::V2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GenSmem<T2> sm(smem_raw, a.mmax, a.pitch);
  const T2* cpool = reinterpret_cast<const T2*>(a.cpool);
  const int C = a.cols, pitch = a.pitch;
  const int nw = blockDim.x >> 5;
  const int col = threadIdx.x % C, j0 = threadIdx.x / C, jstep = blockDim.x / C;
  int cur_ax = -1;

  for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const int f = find_field(a.item0, a.nfields, item);
    const FieldDesc fd = a.fields[f];
    const int axi = fd.ax[a.axis];
    const AxisPlan& ap = a.axes[axi];
    if (axi != cur_ax) {                       // tables of this axis length into shared memory
      __syncthreads();
      load_tables(ap, cpool, sm.tw, sm.ch, sm.bh);
      __syncthreads();
      cur_ax = axi;
    }
    const int n = ap.n, m = ap.m;
    long long inner, nstride, outer_stride, ncols;
    if (a.axis == 2) { inner = (long long)fd.nx * fd.ny; nstride = inner; outer_stride = 0; ncols = inner; }
    else { inner = fd.nx; nstride = fd.nx; outer_stride = (long long)fd.nx * fd.ny; ncols = (long long)fd.nz * fd.nx; }
    const long long ntiles = (ncols + C - 1) / C;
    const long long chunks = (ntiles + a.tiles_per_item - 1) / a.tiles_per_item;
    const long long local = item - a.item0[f];
    const int comp = (int)(local / chunks);
    const long long chunk = local - comp * chunks;
    const T* in_re = reinterpret_cast<const T*>(a.in) + (a.mode == 1 ? fd.in_off : fd.out_off) + 2LL * comp * fd.V;
    const T* in_im = in_re + fd.V;
    T* out_re = reinterpret_cast<T*>(a.out) + fd.out_off + 2LL * comp * fd.V;
    T* out_im = out_re + fd.V;
    const T* ref_re = a.ref ? reinterpret_cast<const T*>(a.ref) + fd.in_off + 2LL * comp * fd.V : nullptr;
    const T wa = comp == 2 ? T(2) : T(1), wb = comp == 0 ? T(1) : T(2);
    Kahan<T> sa, sb, sq;
    T nonfinite = T(0), linf = T(0);
    const bool inv = INV;
    for (long long tile = chunk * a.tiles_per_item;
         tile < ntiles && tile < (chunk + 1) * a.tiles_per_item; ++tile) {
      const long long c = tile * C + col;
      const bool valid = c < ncols;
      const long long o = valid ? c / inner : 0;
      const long long base = o * outer_stride + (valid ? c - o * inner : 0);
      // loads in batches of LB independent loads per thread (several in flight), then the
      // statistics, the pre-chirp and the stores into the work buffer
      constexpr int LB = 8;
      for (int jb = j0; jb < m; jb += LB * jstep) {
        T2 xb[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int j = jb + u * jstep;
          const long long off = base + (long long)j * nstride;
          xb[u] = (j < n && valid && eqk::in_bounds(off, fd.V, a.err))
                      ? T2{in_re[off], in_im[off]} : T2{T(0), T(0)};
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int j = jb + u * jstep;
          if (j >= m) break;
          T2 x = xb[u];
          if (j < n && valid) {
            if (a.mode == 1) {
              if (!isfinite(x.x) || !isfinite(x.y)) nonfinite += T(1);
              sa.add(x.x);
              sb.add(x.y);
              sq.add(wa * x.x * x.x + wb * x.y * x.y);
            }
            x = pre(x, j, ap, sm.ch, inv);
          }
          sm.a[j * pitch + col] = x;
        }
      }
      __syncthreads();
      T2* r = axis_transform(sm.a, sm.b, ap, C, pitch, sm.tw, sm.bh, inv, a.err);
      if (valid) {
        constexpr int SB = 8;
        for (int kb = j0; kb < n; kb += SB * jstep) {
          T2 rb[SB];                                   // residual reference, loaded ahead
          if (ref_re) {
#pragma unroll
            for (int u = 0; u < SB; ++u) {
              const int k = kb + u * jstep;
              const long long off = base + (long long)k * nstride;
              rb[u] = (k < n && eqk::in_bounds(off, fd.V, a.err))
                          ? T2{ref_re[off], ref_re[off + fd.V]} : T2{T(0), T(0)};
            }
          }
#pragma unroll
          for (int u = 0; u < SB; ++u) {
            const int k = kb + u * jstep;
            if (k >= n) break;
            const long long off = base + (long long)k * nstride;
            if (!eqk::in_bounds(off, fd.V, a.err)) continue;
            const T2 y = post(r[k * pitch + col], k, ap, sm.ch, inv);
            out_re[off] = y.x;
            out_im[off] = y.y;
            if (ref_re) {
              linf = fmax(linf, fabs(rb[u].x - y.x));
              linf = fmax(linf, fabs(rb[u].y - y.y));
            }
          }
        }
      }
      __syncthreads();
    }
    if (a.mode == 1) {
      double v[4] = {sa.value(), sb.value(), sq.value(), double(nonfinite)};
      warp_partials<4>(v, a.partials + item * WARPS_MAX * 4);
      for (int k = nw * 4 + threadIdx.x; k < WARPS_MAX * 4; k += blockDim.x)
        a.partials[item * WARPS_MAX * 4 + k] = 0.0;
    } else if (a.mode == 2) {
      double v = double(linf);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
      if ((threadIdx.x & 31) == 0) a.partials[item * WARPS_MAX * 4 + (threadIdx.x >> 5)] = v;
      for (int k = nw + threadIdx.x; k < WARPS_MAX * 4; k += blockDim.x)
        a.partials[item * WARPS_MAX * 4 + k] = 0.0;
    }
  }
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

// ---- strided pass, a warp per column (lengths served by a 256- or 512-point transform) ------
//
// FP32.  Same items, partial records and modes as k_gen_strided.  A tile of C adjacent columns
// (n points each; C = 32 for n <= 256, else 16) comes into shared memory by 4-byte asynchronous
// copies (C consecutive elements of a plane per point, all of a thread's points in flight); the
// warps then
// transform whole columns with paired 256-point transforms (two sequences in one warp, packed
// two-lane arithmetic, eq_pfft.cuh; one compiled forward transform, the inverse by conjugation)
// and write the n outputs back into the tile, which leaves by coalesced stores (with the
// L-infinity residual of the last pass).  Two blocks of 8 warps per SM.  Every field of a launch has
// its axis served by a transform length wm in {256, 512}:
//   wm = 256: a warp takes two adjacent columns as the pair, either transformed directly (n = 256)
//     or by Bluestein's chirp-z convolution (n <= 128: pre-chirp, forward transform, product with
//     the chirp transform, inverse transform, post-chirp);
//   wm = 512: a warp takes one column at a time, its 512-point transform split into the 256-point
//     transforms of the even and odd outputs (the decimation-in-frequency step
//     a_j = u_j + u_{j+256}, b_j = (u_j - u_{j+256}) W512^j) as the pair.  Directly for n = 512;
//     for Bluestein (n <= 256, so u_{j+256} = 0) the convolution's inverse transform needs only
//     the outputs j < 256, y_j = P_j + W512^-j Q_j from the inverse transforms P, Q of the even
//     and odd halves of the product.
// The inverse direction of a Bluestein length goes by conjugation of input and output.
constexpr int SC_WARPS = 8, SC_THREADS = 32 * SC_WARPS;
constexpr int SC_MAXN = 512;          // longest column (n = wm = 512)
constexpr int SC_TILE = SC_MAXN * 17; // tile entries: 16 columns of 512 points or 32 of 256, pitch
                                      // columns + 1
// columns of a tile for axis length n
__host__ __device__ constexpr int scols_cols(int n) { return n <= 256 ? 32 : 16; }
constexpr size_t scols_smem() {
  return sizeof(float4) * size_t(SC_WARPS) * 256 +                          // exchange rows
         sizeof(float2) * (size_t(SC_TILE) + 256 + 512 + 256) +             // tile, chirp, chirp
                                                                             // transform, W512^j
         2 * sizeof(float) * size_t(eqk::staged_size(256));                 // staged twiddles
}

__device__ __forceinline__ eqk::CPair cpair(float2 a, float2 b) {
  return eqk::CPair{make_float2(a.x, b.x), make_float2(a.y, b.y)};
}
__device__ __forceinline__ float2 pair_lo(const eqk::CPair& v) { return make_float2(v.r.x, v.i.x); }
__device__ __forceinline__ float2 pair_hi(const eqk::CPair& v) { return make_float2(v.r.y, v.i.y); }
// lane 0 times w0, lane 1 times w1 (complex)
__device__ __forceinline__ eqk::CPair pmul_lanes(eqk::CPair v, float2 w0, float2 w1) {
  const float2 C = make_float2(w0.x, w1.x), S = make_float2(w0.y, w1.y);
  return eqk::CPair{eqk::fsub2(__fmul2_rn(v.r, C), __fmul2_rn(v.i, S)),
                    __ffma2_rn(v.r, S, __fmul2_rn(v.i, C))};
}

// The paired 256-point transform, forward, or with inv the unnormalised inverse as the conjugate
// of the forward transform of the conjugate: one compiled transform serves both directions (a
// small instruction working set)
__device__ __forceinline__ void pfft256(eqk::CPair (&v)[8], bool inv, int lane, const eqk::PairAcc& acc,
                                        const eqk::TwStaged<float>& tw) {
  const float2 m1 = make_float2(-1.f, -1.f);
  if (inv) {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e].i = __fmul2_rn(v[e].i, m1);
  }
  eqk::pfft_column<256, 8, false>(v, lane, acc, tw);
  if (inv) {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e].i = __fmul2_rn(v[e].i, m1);
  }
}

// Length-n DFT of one sequence through the 512-point split (wm = 512: n = 512 directly, or
// Bluestein for n <= 256).  in(j) gives x_j (j < n); out(k, X_k) takes the n outputs; INV: the
// exponent's sign is +, unnormalised.  All reads of in() precede every call of out().  On entry no
// lane reads `acc`; it is free again on return.
template <bool INV, typename IN, typename OUT>
__device__ __forceinline__ void dft_split512(int n, IN in, OUT out, const eqk::PairAcc& acc,
                                             const eqk::TwStaged<float>& tw, const float2* w512,
                                             const float2* chs, const float4* bhs2, int lane) {
  const bool blue = n != 512;
  eqk::CPair v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int j = lane + 32 * e;
    float2 u0 = make_float2(0.f, 0.f), u1 = make_float2(0.f, 0.f);
    if (j < n) u0 = in(j);
    float2 w = w512[j];
    if (blue) {
      if (INV) u0.y = -u0.y;
      u0 = cmul(u0, chs[j < n ? j : 0]);
    } else {
      u1 = in(j + 256);
      if (INV) w.y = -w.y;
    }
    v[e] = cpair(cadd(u0, u1), cmul(csub(u0, u1), w));
  }
  if (blue) {
    pfft256(v, false, lane, acc, tw);
#pragma unroll
    for (int e = 0; e < 8; ++e) {                 // U_{2k} (lane 0) and U_{2k+1} (lane 1) times b^
      const float4 b = bhs2[lane + 32 * e];
      v[e] = pmul_lanes(v[e], make_float2(b.x, b.y), make_float2(b.z, b.w));
    }
    pfft256(v, true, lane, acc, tw);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = lane + 32 * e;
      if (j < n) {
        const float2 w = w512[j];
        float2 y = cadd(pair_lo(v[e]), cmul(pair_hi(v[e]), make_float2(w.x, -w.y)));
        y = cmul(y, chs[j]);
        if (INV) y.y = -y.y;
        out(j, y);
      }
    }
  } else {
    pfft256(v, INV, lane, acc, tw);
#pragma unroll
    for (int e = 0; e < 8; ++e) {                 // outputs 2k and 2k + 1, k = lane + 32 e
      const int k = lane + 32 * e;
      out(2 * k, pair_lo(v[e]));
      out(2 * k + 1, pair_hi(v[e]));
    }
  }
}

// Length-n DFTs of two sequences at once (wm = 256: n = 256 directly, or Bluestein for
// n <= 128); in0 / in1 and out0 / out1 as in dft_split512.
template <bool INV, typename IN0, typename IN1, typename OUT0, typename OUT1>
__device__ __forceinline__ void dft_pair256(int n, IN0 in0, IN1 in1, OUT0 out0, OUT1 out1,
                                            const eqk::PairAcc& acc, const eqk::TwStaged<float>& tw,
                                            const float2* chs, const float2* bhs, int lane) {
  const bool blue = n != 256;
  eqk::CPair v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int j = lane + 32 * e;
    float2 x0 = make_float2(0.f, 0.f), x1 = x0;
    if (j < n) {
      x0 = in0(j);
      x1 = in1(j);
      if (blue) {
        if (INV) { x0.y = -x0.y; x1.y = -x1.y; }
        const float2 c = chs[j];
        x0 = cmul(x0, c);
        x1 = cmul(x1, c);
      }
    }
    v[e] = cpair(x0, x1);
  }
  if (blue) {
    pfft256(v, false, lane, acc, tw);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float2 b = bhs[lane + 32 * e];
      v[e] = eqk::pmul_cs(v[e], b.x, b.y);
    }
    pfft256(v, true, lane, acc, tw);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = lane + 32 * e;
      if (j < n) {
        const float2 c = chs[j];
        float2 y0 = cmul(pair_lo(v[e]), c), y1 = cmul(pair_hi(v[e]), c);
        if (INV) { y0.y = -y0.y; y1.y = -y1.y; }
        out0(j, y0);
        out1(j, y1);
      }
    }
  } else {
    pfft256(v, INV, lane, acc, tw);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = lane + 32 * e;
      out0(k, pair_lo(v[e]));
      out1(k, pair_hi(v[e]));
    }
  }
}

// A column of the tile (wm = 512), and columns c0, c0 + 1 (wm = 256), transformed in place.
template <bool INV>
__device__ __forceinline__ void scol512(float2* tile, int pitch, int col, int n,
                                        const eqk::PairAcc& acc, const eqk::TwStaged<float>& tw,
                                        const float2* w512, const float2* chs, const float4* bhs2,
                                        int lane, int* err) {
  auto in = [&](int j) {
    return eqk::in_bounds((long long)j * pitch + col, SC_TILE, err) ? tile[j * pitch + col]
                                                                     : make_float2(0.f, 0.f);
  };
  auto out = [&](int k, float2 y) { tile[k * pitch + col] = y; };
  dft_split512<INV>(n, in, out, acc, tw, w512, chs, bhs2, lane);
}
template <bool INV>
__device__ __forceinline__ void scol256(float2* tile, int pitch, int c0, int n,
                                        const eqk::PairAcc& acc, const eqk::TwStaged<float>& tw,
                                        const float2* chs, const float2* bhs, int lane, int* err) {
  auto in0 = [&](int j) {
    return eqk::in_bounds((long long)j * pitch + c0 + 1, SC_TILE, err) ? tile[j * pitch + c0]
                                                                        : make_float2(0.f, 0.f);
  };
  auto in1 = [&](int j) {
    return eqk::in_bounds((long long)j * pitch + c0 + 1, SC_TILE, err) ? tile[j * pitch + c0 + 1]
                                                                        : make_float2(0.f, 0.f);
  };
  auto out0 = [&](int k, float2 y) { tile[k * pitch + c0] = y; };
  auto out1 = [&](int k, float2 y) { tile[k * pitch + c0 + 1] = y; };
  dft_pair256<INV>(n, in0, in1, out0, out1, acc, tw, chs, bhs, lane);
}

template <bool INV>
__global__ void __launch_bounds__(SC_THREADS, 2) k_gen_scols(const GenArgs a) {
  using T = float;
  using T2 = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int TWS = eqk::staged_size(256);
  float4* rows = reinterpret_cast<float4*>(smem_raw);      // [warp][256] exchange entries
  T2* tile = reinterpret_cast<T2*>(rows + SC_WARPS * 256); // [point][pitch]
  T2* chs = tile + SC_TILE;                     // chirp (n <= 256)
  T2* bhs = chs + 256;                                     // chirp transform (wm entries)
  T2* w512 = bhs + 512;                                    // W512^j, j < 256
  T* twc = reinterpret_cast<T*>(w512 + 256);
  T* tws = twc + TWS;
  const T2* cpool = reinterpret_cast<const T2*>(a.cpool);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (int i = tid; i < TWS; i += blockDim.x) {
    const T2 t = cpool[a.tw256 + i];
    twc[i] = t.x;
    tws[i] = t.y;
  }
  for (int i = tid; i < 256; i += blockDim.x) w512[i] = cpool[a.w512 + i];
  const eqk::TwStaged<T> tw{twc, tws};
  const eqk::PairAcc acc{rows + w * 256};
  int cur_ax = -1;
  for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const int f = find_field(a.item0, a.nfields, item);
    const FieldDesc fd = a.fields[f];
    const int axi = fd.ax[a.axis];
    const AxisPlan& ap = a.axes[axi];
    const int n = ap.n, wm = ap.wm;
    const int C = scols_cols(n), pitch = C + 1;
    const int lc = tid % C, lj = tid / C, jstep = SC_THREADS / C;
    if (axi != cur_ax) {                  // chirp tables of this axis length into shared memory
      __syncthreads();
      if (wm != n) {
        for (int i = tid; i < n; i += blockDim.x) chs[i] = cpool[ap.wchirp + i];
        for (int i = tid; i < wm; i += blockDim.x) bhs[i] = cpool[ap.wbhat + i];
      }
      __syncthreads();
      cur_ax = axi;
    }
    long long inner, nstride, outer_stride, ncols;
    if (a.axis == 2) { inner = (long long)fd.nx * fd.ny; nstride = inner; outer_stride = 0; ncols = inner; }
    else { inner = fd.nx; nstride = fd.nx; outer_stride = (long long)fd.nx * fd.ny; ncols = (long long)fd.nz * fd.nx; }
    const long long ntiles = (ncols + C - 1) / C;
    const long long chunks = (ntiles + a.tiles_per_item - 1) / a.tiles_per_item;
    const long long local = item - a.item0[f];
    const int comp = (int)(local / chunks);
    const long long chunk = local - comp * chunks;
    const T* in_re = reinterpret_cast<const T*>(a.in) + (a.mode == 1 ? fd.in_off : fd.out_off) + 2LL * comp * fd.V;
    const T* in_im = in_re + fd.V;
    T* out_re = reinterpret_cast<T*>(a.out) + fd.out_off + 2LL * comp * fd.V;
    T* out_im = out_re + fd.V;
    const T* ref_re = a.ref ? reinterpret_cast<const T*>(a.ref) + fd.in_off + 2LL * comp * fd.V : nullptr;
    const T wa = comp == 2 ? T(2) : T(1), wb = comp == 0 ? T(1) : T(2);
    Kahan<T> sa, sb, sq;
    T nonfinite = T(0), linf = T(0);
    for (long long tl = chunk * a.tiles_per_item; tl < ntiles && tl < (chunk + 1) * a.tiles_per_item; ++tl) {
      const long long c = tl * C + lc;
      const bool valid = c < ncols;
      const long long o = valid ? c / inner : 0;
      const long long base = o * outer_stride + (valid ? c - o * inner : 0);
      constexpr int LB = 8;                  // store phase: residual loads in flight a thread
      // the tile by 4-byte asynchronous copies, all of this thread's points in flight at once;
      // then the first pass's statistics from the thread's own points
      if (valid) {
        for (int j = lj; j < n; j += jstep) {
          const long long off = base + (long long)j * nstride;
          if (eqk::in_bounds(off, fd.V, a.err) && eqk::in_bounds((long long)j * pitch + lc, SC_TILE, a.err)) {
            cp_async4(&tile[j * pitch + lc].x, in_re + off);
            cp_async4(&tile[j * pitch + lc].y, in_im + off);
          }
        }
      }
      asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
      if (valid && a.mode == 1) {
        for (int j = lj; j < n; j += jstep) {
          const T2 x = tile[j * pitch + lc];
          if (!isfinite(x.x) || !isfinite(x.y)) nonfinite += T(1);
          sa.add(x.x);
          sb.add(x.y);
          sq.add(wa * x.x * x.x + wb * x.y * x.y);
        }
      }
      __syncthreads();
      if (wm == 512) {
        for (int cc = w; cc < C; cc += SC_WARPS)
          if (tl * C + cc < ncols)                          // warp-uniform
            scol512<INV>(tile, pitch, cc, n, acc, tw, w512, chs, reinterpret_cast<const float4*>(bhs),
                         lane, a.err);
      } else {
        for (int c0 = 2 * w; c0 < C; c0 += 2 * SC_WARPS)
          if (tl * C + c0 < ncols)
            scol256<INV>(tile, pitch, c0, n, acc, tw, chs, bhs, lane, a.err);
      }
      __syncthreads();
      // coalesced tile store (+ the residual of the last pass against the input)
      if (valid) {
        for (int kb = lj; kb < n; kb += LB * jstep) {
          T2 rb[LB];
          if (ref_re) {
#pragma unroll
            for (int u = 0; u < LB; ++u) {
              const int k = kb + u * jstep;
              const long long off = base + (long long)k * nstride;
              rb[u] = (k < n && eqk::in_bounds(off, fd.V, a.err)) ? T2{ref_re[off], ref_re[off + fd.V]}
                                                                   : T2{T(0), T(0)};
            }
          }
#pragma unroll
          for (int u = 0; u < LB; ++u) {
            const int k = kb + u * jstep;
            const long long off = base + (long long)k * nstride;
            if (k < n && eqk::in_bounds(off, fd.V, a.err)) {
              const T2 y = tile[k * pitch + lc];
              out_re[off] = y.x;
              out_im[off] = y.y;
              if (ref_re) {
                linf = fmax(linf, fabs(rb[u].x - y.x));
                linf = fmax(linf, fabs(rb[u].y - y.y));
              }
            }
          }
        }
      }
      __syncthreads();                                      // the tile is free for the next one
    }
    if (a.mode == 1) {
      double v[4] = {sa.value(), sb.value(), sq.value(), double(nonfinite)};
      warp_partials<4>(v, a.partials + item * WARPS_MAX * 4);
      for (int k = SC_WARPS * 4 + tid; k < WARPS_MAX * 4; k += blockDim.x)
        a.partials[item * WARPS_MAX * 4 + k] = 0.0;
    } else if (a.mode == 2) {
      double v = double(linf);
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o2));
      if (lane == 0) a.partials[item * WARPS_MAX * 4 + w] = v;
      for (int k = SC_WARPS + tid; k < WARPS_MAX * 4; k += blockDim.x)
        a.partials[item * WARPS_MAX * 4 + k] = 0.0;
    }
  }
}

// ---- strided pass of double-float plans, a warp per column (wm in {256, 512}) -------------
//
// FP64 plans in double-float arithmetic (FP64 in HBM at the pipeline's ends: the first pass
// converts its loads, the last its stores and the residual's re-read input; double-float pairs
// between the passes).  Same items, partial records and modes as k_gen_strided.  Two blocks of
// SD_WARPS warps per SM (one loads while the other transforms).  A tile of SD_COLS adjacent
// columns (n points each) comes into shared memory by 8-byte asynchronous copies (SD_COLS
// consecutive elements of a plane per point, all of a thread's points in flight at once); each
// warp then transforms a
// column in place with dd_seq (below) and the tile leaves by coalesced stores (with the
// L-infinity residual of the last pass).  All fields of a launch have their axis served (wm in
// {256, 512}); Bluestein lengths are at most 256, so their chirp tables sit in the tile's upper
// rows, reloaded with every item.
constexpr int SD_COLS = 8, SD_WARPS = 8, SD_THREADS = 32 * SD_WARPS, SD_PITCH = SD_COLS + 1;
constexpr int SD_MAXN = 512;          // longest column (n = wm = 512)
template <typename T> constexpr size_t scold_smem() {
  return 2 * sizeof(T) * (size_t(SD_MAXN) * SD_PITCH + 256) +
         sizeof(T) * (size_t(SD_WARPS) * 2 * 256 + 2 * eqk::staged_size(256));
}

// One sequence of a double-float pass (a tile column, or an x row), element j at base[j pitch]
// (j pitch < lim), transformed in place through a single compiled 256-point forward transform
// (its code, executed for each half, keeps the instruction working set small): the inverse
// direction (INV) by conjugation of input and output; a 512-point column through
// the decimation-in-frequency split a_j = u_j + u_{j+256}, b_j = (u_j - u_{j+256}) W512^j, the two
// halves one after the other (outputs 2k and 2k + 1); Bluestein's convolution (n <= 256) with
// transform length wm = 512 from the same split (u_{j+256} = 0), keeping only the outputs j < n
// of its inverse transform, y_j = P_j + W512^-j Q_j, or with wm = 256 directly.
__device__ __forceinline__ void dd_seq(bool INV, eqk::dd2* base, int pitch, long long lim, int n, int wm,
                                       const eqk::SoaAcc<eqk::dd>& acc,
                                       const eqk::TwStaged<eqk::dd>& tw, const eqk::dd2* w512,
                                       const eqk::dd2* chs, const eqk::dd2* bhs, int* err) {
  using T = eqk::dd;
  using T2 = eqk::dd2;
  const int lane = threadIdx.x & 31;
  const bool blue = n != wm, split = wm == 512;
  auto conj = [](T2 v) { return T2{v.x, -v.y}; };
  auto ld = [&](int j) {
    return eqk::in_bounds((long long)j * pitch, lim, err) ? base[j * pitch] : T2{T(0), T(0)};
  };
  // the forward 256-point transform of x, or with inv the unnormalised inverse by conjugation
  auto fft = [&](T2 (&x)[8], bool inv) {
    if (inv) {
#pragma unroll
      for (int e = 0; e < 8; ++e) x[e] = conj(x[e]);
    }
    __syncwarp();                                          // the warp's row is free
    eqk::fft_column_acc<256, 8, false, 0, true>(x, lane, acc, tw);
    if (inv) {
#pragma unroll
      for (int e = 0; e < 8; ++e) x[e] = conj(x[e]);
    }
  };
  T2 keep[8];
#pragma unroll 1
  for (int h = 0; h < (split ? 2 : 1); ++h) {
    T2 x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = lane + 32 * e;
      T2 u0 = j < n ? ld(j) : T2{T(0), T(0)}, u1 = T2{T(0), T(0)};
      if (blue) {
        if (INV) u0 = conj(u0);
        u0 = cmul(u0, chs[j < n ? j : 0]);
      } else if (split) {
        u1 = ld(j + 256);
      }
      if (split && h == 1) {
        const T2 w = w512[j];
        x[e] = cmul(csub(u0, u1), (INV && !blue) ? conj(w) : w);
      } else {
        x[e] = split ? cadd(u0, u1) : u0;
      }
    }
    if (blue) {
      fft(x, false);
#pragma unroll
      for (int e = 0; e < 8; ++e) {                    // the chirp transform at k (or 2k + h)
        const int k = lane + 32 * e;
        x[e] = cmul(x[e], bhs[split ? 2 * k + h : k]);
      }
      fft(x, true);
    } else {
      fft(x, INV);
    }
    if (h == 0) {
#pragma unroll
      for (int e = 0; e < 8; ++e) keep[e] = x[e];
    }
    if (!split || h == 1) {                            // all reads of the column are done
      __syncwarp();
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = lane + 32 * e;
        if (blue) {
          if (k < n) {
            T2 y = split ? cadd(keep[e], cmul(x[e], conj(w512[k]))) : x[e];
            y = cmul(y, chs[k]);
            base[k * pitch] = INV ? conj(y) : y;
          }
        } else if (split) {
          base[(2 * k) * pitch] = keep[e];
          base[(2 * k + 1) * pitch] = x[e];
        } else {
          base[k * pitch] = x[e];
        }
      }
    }
  }
  __syncwarp();
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

// running double-float sum (its 48-bit significand holds a thread's partial sums of a pass
// without compensation); read out as FP64
struct DdSum {
  eqk::dd s = eqk::dd(0.f, 0.f);
  __device__ __forceinline__ void add(eqk::dd v) { s = s + v; }
  __device__ __forceinline__ double value() const { return double(s); }
};

template <typename T, bool INV>
__global__ void __launch_bounds__(SD_THREADS, 2) k_gen_scold(const GenArgs a) {
  using T2 = typename eqk::V2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int TWS = eqk::staged_size(256);
  T2* tile = reinterpret_cast<T2*>(smem_raw);               // [point][SD_PITCH]
  T2* chs = tile + 256 * SD_PITCH;                          // Bluestein (n <= 256): rows 256..
  T2* bhs = chs + 256;                                       //   of the tile hold the chirps
  T2* w512 = tile + SD_MAXN * SD_PITCH;
  T* rows = reinterpret_cast<T*>(w512 + 256);               // [warp][re 256 | im 256]
  T* twc = rows + SD_WARPS * 2 * 256;
  T* tws = twc + TWS;
  const T2* cpool = reinterpret_cast<const T2*>(a.cpool);
  const int tid = threadIdx.x, w = tid >> 5;
  const int lc = tid % SD_COLS, lj = tid / SD_COLS, jstep = SD_THREADS / SD_COLS;
  const eqk::SoaAcc<T> acc{rows + w * 2 * 256, rows + w * 2 * 256 + 256};
  for (int i = tid; i < TWS; i += blockDim.x) {          // the 256-point transform's twiddles
    const T2 t = cpool[a.tw256 + i];
    twc[i] = t.x;
    tws[i] = t.y;
  }
  for (int i = tid; i < 256; i += blockDim.x) w512[i] = cpool[a.w512 + i];
  const eqk::TwStaged<T> tw{twc, tws};
  for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const int f = find_field(a.item0, a.nfields, item);
    const FieldDesc fd = a.fields[f];
    const int axi = fd.ax[a.axis];
    const AxisPlan& ap = a.axes[axi];
    const int n = ap.n, wm = ap.wm;
    if (wm != n) {                        // chirps into the tile's upper rows, every item
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) chs[i] = cpool[ap.wchirp + i];
      for (int i = tid; i < wm; i += blockDim.x) bhs[i] = cpool[ap.wbhat + i];
      __syncthreads();
    }
    long long inner, nstride, outer_stride, ncols;
    if (a.axis == 2) { inner = (long long)fd.nx * fd.ny; nstride = inner; outer_stride = 0; ncols = inner; }
    else { inner = fd.nx; nstride = fd.nx; outer_stride = (long long)fd.nx * fd.ny; ncols = (long long)fd.nz * fd.nx; }
    const long long ntiles = (ncols + SD_COLS - 1) / SD_COLS;
    const long long chunks = (ntiles + a.tiles_per_item - 1) / a.tiles_per_item;
    const long long local = item - a.item0[f];
    const int comp = (int)(local / chunks);
    const long long chunk = local - comp * chunks;
    const T* in_re = reinterpret_cast<const T*>(a.in) + (a.mode == 1 ? fd.in_off : fd.out_off) + 2LL * comp * fd.V;
    const T* in_im = in_re + fd.V;
    T* out_re = reinterpret_cast<T*>(a.out) + fd.out_off + 2LL * comp * fd.V;
    T* out_im = out_re + fd.V;
    const T* ref_re = a.ref ? reinterpret_cast<const T*>(a.ref) + fd.in_off + 2LL * comp * fd.V : nullptr;
    const T wa = comp == 2 ? T(2) : T(1), wb = comp == 0 ? T(1) : T(2);
    DdSum sa, sb, sq;                     // double-float sums: 48 bits need no compensation
    T nonfinite = T(0), linf = T(0);
    const bool in64 = a.io & 1, out64 = a.io & 2;
    for (long long tl = chunk * a.tiles_per_item; tl < ntiles && tl < (chunk + 1) * a.tiles_per_item; ++tl) {
      const long long c = tl * SD_COLS + lc;
      const bool valid = c < ncols;
      const long long o = valid ? c / inner : 0;
      const long long base = o * outer_stride + (valid ? c - o * inner : 0);
      constexpr int LB = 8;                  // store phase: residual loads in flight a thread
      // the tile by 8-byte asynchronous copies, every point of this thread in flight at once (the
      // raw bytes: FP64 values in the first pass, double-float pairs otherwise); then each thread
      // converts its own points in place and takes the first pass's statistics
      if (valid) {
        for (int j = lj; j < n; j += jstep) {
          const long long off = base + (long long)j * nstride;
          if (eqk::in_bounds(off, fd.V, a.err) && eqk::in_bounds((long long)j * SD_PITCH + lc, SD_MAXN * SD_PITCH, a.err)) {
            cp_async8(&tile[j * SD_PITCH + lc].x, in_re + off);
            cp_async8(&tile[j * SD_PITCH + lc].y, in_im + off);
          }
        }
      }
      asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
      if (valid && (in64 || a.mode == 1)) {
        for (int j = lj; j < n; j += jstep) {
          T2 x = tile[j * SD_PITCH + lc];
          if (in64) {
            const double2 raw = *reinterpret_cast<const double2*>(&tile[j * SD_PITCH + lc]);
            x = T2{eqk::dd_from_bits(raw.x), eqk::dd_from_bits(raw.y)};
            tile[j * SD_PITCH + lc] = x;
          }
          if (a.mode == 1) {
            if (!isfinite(x.x) || !isfinite(x.y)) nonfinite += T(1);
            sa.add(x.x);
            sb.add(x.y);
            sq.add(wa * x.x * x.x + wb * x.y * x.y);
          }
        }
      }
      __syncthreads();
      for (int cc = w; cc < SD_COLS; cc += SD_WARPS) {
        if (tl * SD_COLS + cc >= ncols) continue;             // warp-uniform
        dd_seq(INV, tile + cc, SD_PITCH, (long long)SD_MAXN * SD_PITCH - cc, n, wm, acc, tw, w512, chs,
                    bhs, a.err);
      }
      __syncthreads();
      // coalesced tile store (+ the residual of the last pass against the input)
      if (valid) {
        for (int kb = lj; kb < n; kb += LB * jstep) {
          T2 rb[LB];
          if (ref_re) {
#pragma unroll
            for (int u = 0; u < LB; ++u) {
              const int k = kb + u * jstep;
              const long long off = base + (long long)k * nstride;
              rb[u] = (k < n && eqk::in_bounds(off, fd.V, a.err))
                          ? T2{ld_f64(ref_re, off), ld_f64(ref_re, off + fd.V)}
                          : T2{T(0), T(0)};
            }
          }
#pragma unroll
          for (int u = 0; u < LB; ++u) {
            const int k = kb + u * jstep;
            if (k >= n) break;
            const long long off = base + (long long)k * nstride;
            if (!eqk::in_bounds(off, fd.V, a.err)) continue;
            const T2 y = tile[k * SD_PITCH + lc];
            st_dd(out_re, off, y.x, out64);
            st_dd(out_im, off, y.y, out64);
            if (ref_re) {
              linf = fmax(linf, fabs(rb[u].x - y.x));
              linf = fmax(linf, fabs(rb[u].y - y.y));
            }
          }
        }
      }
      __syncthreads();                                      // the tile is free for the next one
    }
    if (a.mode == 1) {
      double v[4] = {sa.value(), sb.value(), sq.value(), double(nonfinite)};
      warp_partials<4>(v, a.partials + item * WARPS_MAX * 4);
      for (int k = SD_WARPS * 4 + threadIdx.x; k < WARPS_MAX * 4; k += blockDim.x)
        a.partials[item * WARPS_MAX * 4 + k] = 0.0;
    } else if (a.mode == 2) {
      double v = double(linf);
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o2));
      if ((threadIdx.x & 31) == 0) a.partials[item * WARPS_MAX * 4 + (threadIdx.x >> 5)] = v;
      for (int k = SD_WARPS + threadIdx.x; k < WARPS_MAX * 4; k += blockDim.x)
        a.partials[item * WARPS_MAX * 4 + k] = 0.0;
    }
  }
}

// ---- x pass of double-float plans, a warp per row (wm in {256, 512}) --------------------------
//
// Item = (field, tiles_per_item row pairs), the items of k_gen_xrows.  A block of six warps takes
// a row pair (k, -k): warp w copies row A (w < 3) or B of plane pair w mod 3 into its shared row,
// transforms it in place with dd_seq (one compiled 256-point transform, both halves of a 512-point
// row in turn), the block meets, the mode pairs are projected across the six rows (the generic
// projector in double-float), the block meets again, and every warp takes its row's inverse
// transform in place and stores it.  Rows are double-float pairs in HBM (a middle pass).
constexpr int XD_THREADS = 192, XD_MAXN = 512;
template <typename T> constexpr size_t xdd_smem() {
  return 2 * sizeof(T) * (6 * size_t(XD_MAXN) + 256 + 512 + 256) +     // rows, chirps, W512^j
         sizeof(T) * (6 * 2 * 256 + 2 * eqk::staged_size(256) + XD_MAXN);  // exchange, twiddles, xi_x
}

template <typename T>
__global__ void __launch_bounds__(XD_THREADS, 2) k_gen_xdd(const GenArgs a) {
  static_assert(sizeof(T) == 8, "double-float kernel");
  using T2 = eqk::dd2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int TWS = eqk::staged_size(256);
  T2* rows = reinterpret_cast<T2*>(smem_raw);                // [warp][XD_MAXN]
  T2* chs = rows + 6 * XD_MAXN;
  T2* bhs = chs + 256;
  T2* w512 = bhs + 512;
  T* xch = reinterpret_cast<T*>(w512 + 256);                 // [warp][re 256 | im 256]
  T* twc = xch + 6 * 2 * 256;
  T* tws = twc + TWS;
  T* xix = tws + TWS;
  const T2* cpool = reinterpret_cast<const T2*>(a.cpool);
  const T* xipool = reinterpret_cast<const T*>(a.xipool);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int side = w / 3, comp = w % 3;
  for (int i = tid; i < TWS; i += blockDim.x) {
    const T2 t = cpool[a.tw256 + i];
    twc[i] = t.x;
    tws[i] = t.y;
  }
  for (int i = tid; i < 256; i += blockDim.x) w512[i] = cpool[a.w512 + i];
  const eqk::TwStaged<T> tw{twc, tws};
  const eqk::SoaAcc<T> acc{xch + w * 2 * 256, xch + w * 2 * 256 + 256};
  T2* row = rows + w * XD_MAXN;
  int cur_f = -1;
  for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const int f = find_field(a.item0, a.nfields, item);
    const FieldDesc fd = a.fields[f];
    const AxisPlan& ap = a.axes[fd.ax[0]];
    const int n = fd.nx, wm = ap.wm, ny = fd.ny, nz = fd.nz;
    if (f != cur_f) {                     // this field's x tables into shared memory
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) xix[i] = xipool[fd.xi[0] + i];
      if (wm != n) {
        for (int i = tid; i < n; i += blockDim.x) chs[i] = cpool[ap.wchirp + i];
        for (int i = tid; i < wm; i += blockDim.x) bhs[i] = cpool[ap.wbhat + i];
      }
      __syncthreads();
      cur_f = f;
    }
    T* base = reinterpret_cast<T*>(a.out) + fd.out_off;
    const T* xiy = xipool + fd.xi[1];
    const T* xiz = xipool + fd.xi[2];
    T zmv[6];
    eqk::zero_mode_values(a.mean + f * 6, double(fd.V), zmv);
    const T inv_v = T(1.0 / double(fd.V));
    DdSum r2, di2, do2, o2;
    const long long local = item - a.item0[f];
    const long long lim = 6 * fd.V;
    for (int g = (int)(local * a.tiles_per_item);
         g < fd.npairs && g < (local + 1) * a.tiles_per_item; ++g) {
      const int rA = a.pairpool[fd.pairs + g];
      const int kz = rA / ny, ky = rA - kz * ny;
      const int rB = (kz == 0 ? 0 : nz - kz) * ny + (ky == 0 ? 0 : ny - ky);
      const bool self = rA == rB;
      const bool active = !(side == 1 && self);              // warp-uniform
      const long long roff = (long long)(side == 0 ? rA : rB) * n + 2LL * comp * fd.V;
      const T xi_y = xiy[ky], xi_z = xiz[kz];
      // phase 0: load and forward transform, then the projector; phase 1: inverse transform and
      // store (one call site of the transform: one inlined copy of its code)
#pragma unroll 1
      for (int ph = 0; ph < 2; ++ph) {
        if (active) {
          if (ph == 0) {                  // the row by 8-byte asynchronous copies, all in flight
            for (int j = lane; j < n; j += 32) {
              if (eqk::in_bounds(roff + j + fd.V, lim, a.err)) {
                cp_async8(&row[j].x, base + roff + j);
                cp_async8(&row[j].y, base + roff + j + fd.V);
              }
            }
            asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
            __syncwarp();
          }
          dd_seq(ph == 1, row, 1, XD_MAXN, n, wm, acc, tw, w512, chs, bhs, a.err);
          if (ph == 1) {
            for (int j = lane; j < n; j += 32) {
              if (eqk::in_bounds(roff + j + fd.V, lim, a.err)) {
                base[roff + j] = row[j].x;
                base[roff + j + fd.V] = row[j].y;
              }
            }
            __syncwarp();
          }
        }
        if (ph == 1) break;
        __syncthreads();
        for (int kx = tid; kx < n; kx += blockDim.x) {
          const int kxm = kx == 0 ? 0 : n - kx;
          if (self && kx > kxm) continue;
          T2 av[3], bv[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            av[c] = rows[c * XD_MAXN + kx];
            bv[c] = rows[(self ? c : 3 + c) * XD_MAXN + kxm];
          }
          const bool selfmode = self && kx == kxm;
          eqk::project_pair<T>(av, bv, xix[kx], xi_y, xi_z, rA == 0 && kx == 0, zmv,
                               a.nyq_zero != 0, a.compat != 0, inv_v, selfmode ? T(1) : T(2), r2,
                               di2, do2, o2);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            rows[c * XD_MAXN + kx] = av[c];
            if (!selfmode) rows[(self ? c : 3 + c) * XD_MAXN + kxm] = bv[c];
          }
        }
        __syncthreads();
      }
    }
    double v[4] = {r2.value(), di2.value(), do2.value(), o2.value()};
    warp_partials<4>(v, a.partials + item * WARPS_MAX * 4);
    for (int k = 6 * 4 + tid; k < WARPS_MAX * 4; k += blockDim.x)
      a.partials[item * WARPS_MAX * 4 + k] = 0.0;
  }
}

// ---- x pass, a warp per Voigt pair (FP32; every x length served by wm in {256, 512}) ----------
//
// Item = (field, tiles_per_item row pairs).  A block of three warps takes a row pair (k, -k):
// warp c loads rows A and B of complex plane pair c, takes their x transforms with the paired
// 256-point transforms (dft_pair256 for both rows at once when wm = 256; dft_split512 for one row
// after the other when wm = 512) and leaves the n spectrum values of each row in shared memory;
// the block meets; the mode pairs are projected across the three planes; the block meets again;
// every warp takes the inverse transforms of its two rows and stores them.
constexpr int XQ_THREADS = 96, XQ_MAXN = 512;
constexpr size_t xpair_smem() {
  return sizeof(float4) * 3 * 256 +                                 // exchange rows
         sizeof(float2) * (6 * XQ_MAXN + 256 + 512 + 256) +         // spectra, chirp, chirp
                                                                    // transform, W512^j
         2 * sizeof(float) * size_t(eqk::staged_size(256)) + sizeof(float) * XQ_MAXN;
}

template <typename T>
__global__ void __launch_bounds__(XQ_THREADS, 4) k_gen_xpair(const GenArgs a) {
  static_assert(sizeof(T) == 4, "FP32 kernel");
  using T2 = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int TWS = eqk::staged_size(256);
  float4* rows = reinterpret_cast<float4*>(smem_raw);       // [warp][256] exchange entries
  T2* spec = reinterpret_cast<T2*>(rows + 3 * 256);         // [plane pair][side][XQ_MAXN]
  T2* chs = spec + 6 * XQ_MAXN;
  T2* bhs = chs + 256;
  T2* w512 = bhs + 512;
  T* twc = reinterpret_cast<T*>(w512 + 256);
  T* tws = twc + TWS;
  T* xix = tws + TWS;
  const T2* cpool = reinterpret_cast<const T2*>(a.cpool);
  const T* xipool = reinterpret_cast<const T*>(a.xipool);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (int i = tid; i < TWS; i += blockDim.x) {
    const T2 t = cpool[a.tw256 + i];
    twc[i] = t.x;
    tws[i] = t.y;
  }
  for (int i = tid; i < 256; i += blockDim.x) w512[i] = cpool[a.w512 + i];
  const eqk::TwStaged<T> tw{twc, tws};
  const eqk::PairAcc acc{rows + w * 256};
  T2* sA = spec + (2 * w) * XQ_MAXN;                         // this warp's spectra
  T2* sB = sA + XQ_MAXN;
  int cur_f = -1;
  for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const int f = find_field(a.item0, a.nfields, item);
    const FieldDesc fd = a.fields[f];
    const AxisPlan& ap = a.axes[fd.ax[0]];
    const int n = fd.nx, wm = ap.wm, ny = fd.ny, nz = fd.nz;
    if (f != cur_f) {                     // this field's x tables into shared memory
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) xix[i] = xipool[fd.xi[0] + i];
      if (wm != n) {
        for (int i = tid; i < n; i += blockDim.x) chs[i] = cpool[ap.wchirp + i];
        for (int i = tid; i < wm; i += blockDim.x) bhs[i] = cpool[ap.wbhat + i];
      }
      __syncthreads();
      cur_f = f;
    }
    T* base = reinterpret_cast<T*>(a.out) + fd.out_off;
    const T* xiy = xipool + fd.xi[1];
    const T* xiz = xipool + fd.xi[2];
    T zmv[6];
    eqk::zero_mode_values(a.mean + f * 6, double(fd.V), zmv);
    const T inv_v = T(1.0 / double(fd.V));
    Kahan<T> r2, di2, do2, o2;
    const long long local = item - a.item0[f];
    const long long lim = 6 * fd.V;
    for (int g = (int)(local * a.tiles_per_item);
         g < fd.npairs && g < (local + 1) * a.tiles_per_item; ++g) {
      const int rA = a.pairpool[fd.pairs + g];
      const int kz = rA / ny, ky = rA - kz * ny;
      const int rB = (kz == 0 ? 0 : nz - kz) * ny + (ky == 0 ? 0 : ny - ky);
      const bool self = rA == rB;
      const long long oA = (long long)rA * n + 2LL * w * fd.V, oB = (long long)rB * n + 2LL * w * fd.V;
      auto load = [&](long long o) {
        return [=](int j) {
          return eqk::in_bounds(o + j + fd.V, lim, a.err) ? make_float2(base[o + j], base[o + j + fd.V])
                                                          : make_float2(0.f, 0.f);
        };
      };
      auto keep = [](T2* s) { return [=](int k, float2 y) { s[k] = y; }; };
      // forward transforms of rows A and B of plane pair w into sA, sB
      __syncwarp();
      if (wm == 256) {
        dft_pair256<false>(n, load(oA), load(oB), keep(sA), keep(sB), acc, tw, chs, bhs, lane);
      } else {
        const float4* bh2 = reinterpret_cast<const float4*>(bhs);
#pragma unroll 1
        for (int r = 0; r < (self ? 1 : 2); ++r)                // rows A and B in turn
          dft_split512<false>(n, load(r ? oB : oA), keep(r ? sB : sA), acc, tw, w512, chs, bh2, lane);
      }
      __syncthreads();
      // projector over the mode pairs (kx, B at -kx)
      const T xi_y = xiy[ky], xi_z = xiz[kz];
      eqk::PlainSum<T> ps[4];
      for (int kx = tid; kx < n; kx += blockDim.x) {
        const int kxm = kx == 0 ? 0 : n - kx;
        if (self && kx > kxm) continue;
        T2 av[3], bv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          av[c] = spec[(2 * c) * XQ_MAXN + kx];
          bv[c] = spec[(2 * c + (self ? 0 : 1)) * XQ_MAXN + kxm];
        }
        const bool selfmode = self && kx == kxm;
        eqk::project_pair<T>(av, bv, xix[kx], xi_y, xi_z, rA == 0 && kx == 0, zmv, a.nyq_zero != 0,
                             a.compat != 0, inv_v, selfmode ? T(1) : T(2), ps[0], ps[1], ps[2], ps[3]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          spec[(2 * c) * XQ_MAXN + kx] = av[c];
          if (!selfmode) spec[(2 * c + (self ? 0 : 1)) * XQ_MAXN + kxm] = bv[c];
        }
      }
      r2.add(ps[0].s);
      di2.add(ps[1].s);
      do2.add(ps[2].s);
      o2.add(ps[3].s);
      __syncthreads();
      // inverse transforms of the two rows, stored
      auto read = [](const T2* s) { return [=](int k) { return s[k]; }; };
      auto store = [&](long long o) {
        return [=](int j, float2 y) {
          if (eqk::in_bounds(o + j + fd.V, lim, a.err)) {
            base[o + j] = y.x;
            base[o + j + fd.V] = y.y;
          }
        };
      };
      if (wm == 256) {
        auto skip = [](int, float2) {};
        if (self) dft_pair256<true>(n, read(sA), read(sA), store(oA), skip, acc, tw, chs, bhs, lane);
        else dft_pair256<true>(n, read(sA), read(sB), store(oA), store(oB), acc, tw, chs, bhs, lane);
      } else {
        const float4* bh2 = reinterpret_cast<const float4*>(bhs);
#pragma unroll 1
        for (int r = 0; r < (self ? 1 : 2); ++r)
          dft_split512<true>(n, read(r ? sB : sA), store(r ? oB : oA), acc, tw, w512, chs, bh2, lane);
      }
    }
    double v[4] = {r2.value(), di2.value(), do2.value(), o2.value()};
    warp_partials<4>(v, a.partials + item * WARPS_MAX * 4);
    for (int k = 3 * 4 + tid; k < WARPS_MAX * 4; k += blockDim.x)
      a.partials[item * WARPS_MAX * 4 + k] = 0.0;
  }
}

// Fused x pass over a list of fields, any lengths.  Item = (field, tiles_per_item groups of P
// row pairs); C = 6 P columns; blockDim.x = 32 C (one warp per row for the global loads).
template <typename T>
__global__ void __launch_bounds__(512) k_gen_xproj(const GenArgs a) {
  using T2 = typename eqk::V2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GenSmem<T2> sm(smem_raw, a.mmax, a.pitch);
  const T2* cpool = reinterpret_cast<const T2*>(a.cpool);
  const T* xipool = reinterpret_cast<const T*>(a.xipool);
  const int C = a.cols, pitch = a.pitch, P = C / 6;
  const int nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, wrow = threadIdx.x >> 5;       // one warp per row
  int cur_ax = -1;

  for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const int f = find_field(a.item0, a.nfields, item);
    const FieldDesc fd = a.fields[f];
    const AxisPlan& ap = a.axes[fd.ax[0]];
    if (fd.ax[0] != cur_ax) {
      __syncthreads();
      load_tables(ap, cpool, sm.tw, sm.ch, sm.bh);
      __syncthreads();
      cur_ax = fd.ax[0];
    }
    const int nx = fd.nx, ny = fd.ny, nz = fd.nz, m = ap.m;
    const long long local = item - a.item0[f];
    const int* pairs = a.pairpool + fd.pairs;
    T* base = reinterpret_cast<T*>(a.out) + fd.out_off;
    const T* xix = xipool + fd.xi[0];
    const T* xiy = xipool + fd.xi[1];
    const T* xiz = xipool + fd.xi[2];
    T zmv[6];
    eqk::zero_mode_values(a.mean + f * 6, double(fd.V), zmv);
    const T inv_v = T(1.0 / double(fd.V));
    Kahan<T> r2, di2, do2, o2;
    const int ngroups = (fd.npairs + P - 1) / P;
    // row handled by this warp: column wrow = slot * 6 + side * 3 + comp
    const int slot = wrow / 6, side = (wrow % 6) / 3, comp = wrow % 3;
    for (int g = (int)(local * a.tiles_per_item);
         g < ngroups && g < (local + 1) * a.tiles_per_item; ++g) {
      const int p = g * P + slot;
      long long roff = -1;
      if (p < fd.npairs) {
        const int rA = pairs[p];
        const int kz = rA / ny, ky = rA - kz * ny;
        const int rB = (kz == 0 ? 0 : nz - kz) * ny + (ky == 0 ? 0 : ny - ky);
        if (!(side == 1 && rA == rB)) roff = (long long)(side == 0 ? rA : rB) * nx + 2LL * comp * fd.V;
      }
      for (int j = lane; j < m; j += 32) {
        T2 x = {T(0), T(0)};
        if (j < nx && roff >= 0 && eqk::in_bounds(roff + j + fd.V, 6 * fd.V, a.err))
          x = pre(T2{base[roff + j], base[roff + j + fd.V]}, j, ap, sm.ch, false);
        sm.a[j * pitch + wrow] = x;
      }
      __syncthreads();
      T2* r = axis_transform(sm.a, sm.b, ap, C, pitch, sm.tw, sm.bh, false, a.err);
      if (ap.blue) {
        const int col = threadIdx.x % C, jstep = blockDim.x / C;
        for (int k = threadIdx.x / C; k < nx; k += jstep)
          r[k * pitch + col] = post(r[k * pitch + col], k, ap, sm.ch, false);
        __syncthreads();
      }
      for (int it = threadIdx.x; it < P * nx; it += blockDim.x) {
        const int s2 = it / nx, kx = it - s2 * nx;
        const int p2 = g * P + s2;
        if (p2 >= fd.npairs) continue;
        const int rA = pairs[p2];
        const int kz = rA / ny, ky = rA - kz * ny;
        const bool self2 = ((kz == 0 ? 0 : nz - kz) * ny + (ky == 0 ? 0 : ny - ky)) == rA;
        const int kxm = kx == 0 ? 0 : nx - kx;
        if (self2 && kx > kxm) continue;
        const int colA = s2 * 6, colB = self2 ? s2 * 6 : s2 * 6 + 3;
        T2 av[3], bv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          av[c] = r[kx * pitch + colA + c];
          bv[c] = r[kxm * pitch + colB + c];
        }
        const bool selfmode = self2 && kx == kxm;
        eqk::project_pair<T>(av, bv, xix[kx], xiy[ky], xiz[kz], rA == 0 && kx == 0, zmv,
                             a.nyq_zero != 0, a.compat != 0, inv_v, selfmode ? T(1) : T(2), r2, di2, do2, o2);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          r[kx * pitch + colA + c] = av[c];
          if (!selfmode) r[kxm * pitch + colB + c] = bv[c];
        }
      }
      __syncthreads();
      // inverse: move to the other buffer (pre-chirp for Bluestein), transform, store
      T2* other = (r == sm.a) ? sm.b : sm.a;
      {
        const int col = threadIdx.x % C, jstep = blockDim.x / C;
        for (int j = threadIdx.x / C; j < m; j += jstep)
          other[j * pitch + col] = j < nx ? pre(r[j * pitch + col], j, ap, sm.ch, true) : T2{T(0), T(0)};
      }
      __syncthreads();
      T2* q = axis_transform(other, r, ap, C, pitch, sm.tw, sm.bh, true, a.err);
      if (roff >= 0)
        for (int j = lane; j < nx; j += 32) {
          if (!eqk::in_bounds(roff + j + fd.V, 6 * fd.V, a.err)) continue;
          const T2 y = post(q[j * pitch + wrow], j, ap, sm.ch, true);
          base[roff + j] = y.x;
          base[roff + j + fd.V] = y.y;
        }
      __syncthreads();
    }
    double v[4] = {r2.value(), di2.value(), do2.value(), o2.value()};
    warp_partials<4>(v, a.partials + item * WARPS_MAX * 4);
    for (int k = nw * 4 + threadIdx.x; k < WARPS_MAX * 4; k += blockDim.x)
      a.partials[item * WARPS_MAX * 4 + k] = 0.0;
  }
}

// ---- x pass, one warp per row (lengths served by a 256- or 512-point register transform) --------
//
// As eqk::k_xproj_rows for one row pair at a time, with the row length n of the item's field: a
// block of six warps, warp (side, component) loads its row of n points straight into registers
// (lane l holds points l + 32 e, zero beyond n), takes the length-wm transform through its own
// shared row (radix-8 stages, warp barriers only) - directly when wm = n, else as Bluestein's
// chirp-z convolution (pre-chirp, transform, chirp transform, inverse transform, post-chirp) -
// and leaves the n spectrum values in that row; the block meets; the mode pairs are projected
// across the six rows; the block meets again; every warp takes the inverse transform and stores
// its row.  All fields of an item share wm (one item = one field).
constexpr int XR_MAXN = 256;         // longest Bluestein row (wm = 512 >= 2 n - 1)
constexpr int XR_MAXM = 512;
constexpr int XR_THREADS = 192;
template <typename T> constexpr size_t xrows_smem() {
  return sizeof(T) * (12 * XR_MAXM + 2 * eqk::staged_size(XR_MAXM) + XR_MAXN) +
         2 * sizeof(T) * (XR_MAXN + XR_MAXM);
}

template <typename T, int M>
__device__ __forceinline__ void xrows_pair(const GenArgs& a, const FieldDesc& fd, int g, T* rows,
                                           const eqk::TwStaged<T>& tw,
                                           const typename eqk::V2<T>::t* chs,
                                           const typename eqk::V2<T>::t* bhs, const T* xix,
                                           const T* xiy, const T* xiz, const T* zm, T inv_v,
                                           T* base, eqk::PlainSum<T> (&ps)[4]) {
  using T2 = typename eqk::V2<T>::t;
  constexpr int E = M / 32;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, side = w / 3, comp = w % 3;
  const int n = fd.nx, ny = fd.ny, nz = fd.nz;
  const bool blue = M != n;
  const int rA = a.pairpool[fd.pairs + g];
  const int kz = rA / ny, ky = rA - kz * ny;
  const int rB = (kz == 0 ? 0 : nz - kz) * ny + (ky == 0 ? 0 : ny - ky);
  const bool self = rA == rB;
  const bool active = !(side == 1 && self);                 // warp-uniform
  const long long roff = (long long)(side == 0 ? rA : rB) * n + 2LL * comp * fd.V;
  T* wre = rows + (2 * w) * XR_MAXM;
  T* wim = wre + XR_MAXM;
  const eqk::SoaAcc<T> acc{wre, wim};
  // Bluestein convolution of the pre-chirped row in x (length-M transforms): X_k = conv * c_k
  auto chirpz = [&](T2 (&x)[E]) {
    eqk::fft_column_acc<M, E, false, 0, true>(x, lane, acc, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = cmul(x[e], bhs[lane + 32 * e]);
    __syncwarp();
    eqk::fft_column_acc<M, E, true, 0, true>(x, lane, acc, tw);
  };
  if (active) {
    T2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = lane + 32 * e;
      x[e] = T2{T(0), T(0)};
      if (j < n && eqk::in_bounds(roff + j + fd.V, 6 * fd.V, a.err)) {
        x[e] = T2{base[roff + j], base[roff + j + fd.V]};
        if (blue) x[e] = cmul(x[e], chs[j]);
      }
    }
    __syncwarp();                                           // the row is free (last pair read)
    if (blue) {
      chirpz(x);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = lane + 32 * e;
        if (k < n) x[e] = cmul(x[e], chs[k]);
      }
    } else {
      eqk::fft_column_acc<M, E, false, 0, true>(x, lane, acc, tw);
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (lane + 32 * e < n) acc.put(lane + 32 * e, x[e]);
  }
  __syncthreads();
  const T xi_y = xiy[ky], xi_z = xiz[kz];
  for (int kx = tid; kx < n; kx += blockDim.x) {
    const int kxm = kx == 0 ? 0 : n - kx;
    if (self && kx > kxm) continue;
    const int ja = eqk::swz(kx), jb = eqk::swz(kxm);
    T2 av[3], bv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T* ra = rows + (2 * c) * XR_MAXM;
      const T* rb = rows + (2 * (self ? c : 3 + c)) * XR_MAXM;
      av[c] = T2{ra[ja], ra[XR_MAXM + ja]};
      bv[c] = T2{rb[jb], rb[XR_MAXM + jb]};
    }
    const bool selfmode = self && kx == kxm;
    eqk::project_pair<T>(av, bv, xix[kx], xi_y, xi_z, rA == 0 && kx == 0, zm, a.nyq_zero != 0,
                         a.compat != 0, inv_v, selfmode ? T(1) : T(2), ps[0], ps[1], ps[2], ps[3]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T* ra = rows + (2 * c) * XR_MAXM;
      T* rb = rows + (2 * (self ? c : 3 + c)) * XR_MAXM;
      ra[ja] = av[c].x;
      ra[XR_MAXM + ja] = av[c].y;
      if (!selfmode) {
        rb[jb] = bv[c].x;
        rb[XR_MAXM + jb] = bv[c].y;
      }
    }
  }
  __syncthreads();
  if (active) {
    T2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = lane + 32 * e;
      x[e] = T2{T(0), T(0)};
      if (k < n) {
        x[e] = acc.get(k);
        if (blue) x[e] = cmul(T2{x[e].x, -x[e].y}, chs[k]);   // inverse by conjugation
      }
    }
    __syncwarp();
    if (blue) {
      chirpz(x);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const T2 r = cmul(x[e], chs[(lane + 32 * e) < n ? lane + 32 * e : 0]);
        x[e] = T2{r.x, -r.y};
      }
    } else {
      eqk::fft_column_acc<M, E, true, 0, true>(x, lane, acc, tw);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = lane + 32 * e;
      if (j < n && eqk::in_bounds(roff + j + fd.V, 6 * fd.V, a.err)) {
        base[roff + j] = x[e].x;
        base[roff + j + fd.V] = x[e].y;
      }
    }
    __syncwarp();
  }
}

// Item = (field, tiles_per_item row pairs); every field's x length has wm in {256, 512}.
template <typename T>
__global__ void __launch_bounds__(XR_THREADS, 2) k_gen_xrows(const GenArgs a) {
  using T2 = typename eqk::V2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int TWS = eqk::staged_size(XR_MAXM);
  T* rows = reinterpret_cast<T*>(smem_raw);                 // [warp][re M | im M]
  T* twc = rows + 12 * XR_MAXM;
  T* tws = twc + TWS;
  T* xix = tws + TWS;
  T2* chs = reinterpret_cast<T2*>(xix + XR_MAXN);
  T2* bhs = chs + XR_MAXN;
  const T2* cpool = reinterpret_cast<const T2*>(a.cpool);
  const T* xipool = reinterpret_cast<const T*>(a.xipool);
  const int nw = blockDim.x >> 5;
  int cur_f = -1;
  for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const int f = find_field(a.item0, a.nfields, item);
    const FieldDesc fd = a.fields[f];
    const AxisPlan& ap = a.axes[fd.ax[0]];
    const int wm = ap.wm;
    if (f != cur_f) {                       // tables of this field's x length into shared memory
      __syncthreads();
      const int ts = eqk::staged_size(wm);
      for (int i = threadIdx.x; i < ts; i += blockDim.x) {
        const T2 t = cpool[ap.wtw + i];
        twc[i] = t.x;
        tws[i] = t.y;
      }
      for (int i = threadIdx.x; i < fd.nx; i += blockDim.x) xix[i] = xipool[fd.xi[0] + i];
      if (wm != fd.nx) {
        for (int i = threadIdx.x; i < fd.nx; i += blockDim.x) chs[i] = cpool[ap.wchirp + i];
        for (int i = threadIdx.x; i < wm; i += blockDim.x) bhs[i] = cpool[ap.wbhat + i];
      }
      __syncthreads();
      cur_f = f;
    }
    const eqk::TwStaged<T> tw{twc, tws};
    T* base = reinterpret_cast<T*>(a.out) + fd.out_off;
    const T* xiy = xipool + fd.xi[1];
    const T* xiz = xipool + fd.xi[2];
    T zmv[6];
    eqk::zero_mode_values(a.mean + f * 6, double(fd.V), zmv);
    const T inv_v = T(1.0 / double(fd.V));
    Kahan<T> r2, di2, do2, o2;
    const long long local = item - a.item0[f];
    for (int g = (int)(local * a.tiles_per_item);
         g < fd.npairs && g < (local + 1) * a.tiles_per_item; ++g) {
      eqk::PlainSum<T> ps[4];
      if (wm == 512)
        xrows_pair<T, 512>(a, fd, g, rows, tw, chs, bhs, xix, xiy, xiz, zmv, inv_v, base, ps);
      else
        xrows_pair<T, 256>(a, fd, g, rows, tw, chs, bhs, xix, xiy, xiz, zmv, inv_v, base, ps);
      r2.add(ps[0].s);
      di2.add(ps[1].s);
      do2.add(ps[2].s);
      o2.add(ps[3].s);
    }
    double v[4] = {r2.value(), di2.value(), do2.value(), o2.value()};
    warp_partials<4>(v, a.partials + item * WARPS_MAX * 4);
    for (int k = nw * 4 + threadIdx.x; k < WARPS_MAX * 4; k += blockDim.x)
      a.partials[item * WARPS_MAX * 4 + k] = 0.0;
  }
}

}  // namespace eqg
