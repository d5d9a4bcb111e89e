// eq_tma.cuh - strided passes (z, y) with TMA-fed double buffering (sm_100+ bulk tensor copies).
//
// One block per SM walks its tiles (B consecutive x columns x all N points of one complex field).
// Thread 0 issues cp.async.bulk.tensor loads of tile k+2 into the shared-memory stage that tile k
// has just been read from, completing on that stage's mbarrier, so two tiles of loads are in
// flight while the block transforms tile k (register Stockham stages, exchange buffer) and
// stores it with plain coalesced stores.  Every mbarrier wait is bounded: if it runs out the
// block raises the plan's error flag, waits (bounded) for its own copies in flight and leaves.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "eq_kernels.cuh"

namespace eqk {

constexpr long long TMA_WAIT_LIMIT = 1LL << 24;   // polls of one mbarrier phase (> 1 s)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// true once the phase with the given parity has completed; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          long long limit = TMA_WAIT_LIMIT) {
  const unsigned a = smem_u32(bar);
  for (long long i = 0; i < limit; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (i > 64) __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, unsigned long long* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_u32(bar))
      : "memory");
}

// tiled store from shared memory (bulk group; the caller commits and waits)
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1,
                                             int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
          reinterpret_cast<unsigned long long>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
      : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// V = 0: 64-byte tile rows (16 FP32 / 8 FP64 columns), one block per SM; V = 1: 32-byte rows,
// half the shared memory, two blocks per SM.
template <typename T, int N, int V = 0> struct TmaCfg {
  static constexpr int E = 8;
  static constexpr int TPC = N / E;
  static constexpr int BW = (sizeof(T) == 4 ? 16 : 8) >> V;
  static constexpr int B = BW * TPC <= 1024 ? BW : 1024 / TPC;
  static constexpr int MINB = V == 0 ? 1 : 2;
  static constexpr int THREADS = B * TPC;
  static constexpr int BOX = N < 256 ? N : 256;       // points per TMA box along the axis
  static constexpr int NBOX = N / BOX;
  using T2 = typename V2<T>::t;
  static constexpr size_t STAGE_BYTES = 2 * sizeof(T) * size_t(N) * B;   // re + im planes
  // alignment + barriers, twiddles, two stages, exchange, per-thread running sums
  static constexpr size_t SMEM = 1024 + sizeof(T2) * N + 2 * STAGE_BYTES +
                                 sizeof(T2) * size_t(N) * B + 6 * sizeof(T) * size_t(THREADS);
  static constexpr bool OK = N >= 64 && SMEM * MINB <= 227 * 1024 && (V == 0 || B * TPC <= 512);
};

struct TmaArgs {
  const void* ref;         // last pass: input field for the L-inf residual (nullptr = skip)
  void* out;               // destination field 0, plane 0
  const void* tw;
  double* partials;        // mode 1: [batch][3][grid][4]; mode 2: [batch][3][grid]
  int* err;                // raised when a bounded wait runs out
  long long field_stride, V;
  int nx, ny, nz;
  int axis;                // 2 = z, 1 = y
  int mode;                // 0 middle, 1 first (statistics), 2 last
  int tma_store;           // 1: store tiles by TMA through the exchange buffer
  int ncomp;               // complex fields (pairs of planes) per field: 3 (stress), 2 (potential)
  int lim_x, lim_y, lim_z; // > 0: the destination and reference hold only this specimen region
                           // (TMA stores only; boxes outside it are skipped, L-inf is cut to it)
  long long ntiles;        // tiles per (field, component)
};

// Inside the specimen limits of a TmaArgs (no limits: always); x column, y row, z point.
__device__ __forceinline__ bool in_spec(const TmaArgs& a, int x, int y, int z) {
  return a.lim_x == 0 || (x < a.lim_x && y < a.lim_y && z < a.lim_z);
}

// MODE: 0 middle pass, 1 first pass (input statistics), 2 last pass (L-inf against a.ref, whose
// tile streams through `refmap` into the stage the transform has just read, while it computes),
// 3 the last pass of a specimen inside the grid (as 2, with the L-inf cut to the specimen).
// At 1024 threads a thread has 64 registers; the running statistics of MODE 1 (three compensated
// sums) and the L-inf of MODE 2 live in a per-thread slot of shared memory instead, so that no
// register spills to local memory (whose reloads would go to L2 every tile).  The transformed
// tile leaves by per-thread stores or, with a.tma_store, through the exchange buffer by tiled TMA
// stores (`outmap`); the host takes the latter for the last z pass, where it measured faster.
template <typename T, int N, bool INV, int MODE, int V>
__global__ void __launch_bounds__(TmaCfg<T, N, V>::THREADS, TmaCfg<T, N, V>::MINB)
k_strided_tma(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap refmap,
              const __grid_constant__ CUtensorMap outmap, const TmaArgs a) {
  using C = TmaCfg<T, N, V>;
  using T2 = typename C::T2;
  constexpr int E = C::E, TPC = C::TPC, B = C::B, BOX = C::BOX, NBOX = C::NBOX;
  constexpr int THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_tma[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_tma) + 127) & ~uintptr_t(127));
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(base);
  T* stage0 = reinterpret_cast<T*>(base + 128);      // stage s at stage0 + s * 2 N B
  T2* tw = reinterpret_cast<T2*>(stage0 + 4 * N * B);
  T2* xbuf = tw + N;
  T* acc = reinterpret_cast<T*>(xbuf + N * B);       // [6][THREADS] running sums (MODE 1, 2)
  __shared__ double red[32 * 4];
  __shared__ int abort_flag, nonfinite;

  const int tid = threadIdx.x;
  const int b = tid % B, t = tid / B;
  const int field = blockIdx.y / a.ncomp, comp = blockIdx.y % a.ncomp;
  const int plane_re = field * 2 * a.ncomp + 2 * comp;
  const int tiles_x = a.nx / B;
  const int ntiles = (int)a.ntiles;

  for (int i = tid; i < N; i += blockDim.x) tw[i] = reinterpret_cast<const T2*>(a.tw)[i];
  if constexpr (MODE != 0) {
#pragma unroll
    for (int j = 0; j < 6; ++j) acc[j * THREADS + tid] = T(0);
  }
  if (tid == 0) {
    abort_flag = 0;
    nonfinite = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // coordinates of tile u: (x0, row) with row = y (z pass) or z (y pass)
  int issued0 = 0, issued1 = 0;                        // loads issued per stage (thread 0)
  auto issue = [&](int u, int s, const CUtensorMap* m) {
    const int x0 = (u % tiles_x) * B;
    const int row = u / tiles_x;
    if (s) ++issued1; else ++issued0;
    mbar_expect_tx(&bar[s], (unsigned)C::STAGE_BYTES);
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < NBOX; ++q) {
        T* dst = stage0 + s * 2 * N * B + p * N * B + q * BOX * B;
        if (a.axis == 2) tma_load_4d(dst, m, &bar[s], x0, row, q * BOX, plane_re + p);
        else tma_load_4d(dst, m, &bar[s], x0, q * BOX, row, plane_re + p);
      }
  };
  int ph0 = 0, ph1 = 0;                                  // completed phases per stage

  const int first = blockIdx.x, step = gridDim.x;
  if (tid == 0) {
    if (first < ntiles) issue(first, 0, &map);
    if (first + step < ntiles) issue(first + step, 1, &map);
  }

  const IdxStrided idx{b, B};
  int k = 0;
  for (int u = first; u < ntiles; u += step, ++k) {
    const int s = k & 1;
    // one thread polls the barrier; the block barrier then publishes the stage to everyone
    if (tid == 0 && !mbar_wait(&bar[s], (unsigned)((s ? ph1 : ph0) & 1))) {
      atomicOr(a.err, 1);
      abort_flag = 1;
    }
    if (s) ++ph1; else ++ph0;
    __syncthreads();
    if (abort_flag) break;
    T2 x[E];
    {
      const T* sre = stage0 + s * 2 * N * B;
#pragma unroll
      for (int e = 0; e < E; ++e)
        x[e] = T2{sre[(t + TPC * e) * B + b], sre[N * B + (t + TPC * e) * B + b]};
    }
    // the previous tile's stores must have read the exchange buffer before the transform reuses it
    if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncthreads();                                   // stage s is free again
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (MODE >= 2 && a.ref) issue(u, s, &refmap);    // this tile's input, for the residual
      else if (u + 2 * step < ntiles) issue(u + 2 * step, s, &map);
    }
    if constexpr (MODE == 1) {
      // plain sums over the thread's E points, compensated across tiles in the thread's slot.
      // A NaN or infinity in any point makes its tile sum non-finite (so does a sum beyond the
      // type's range, which the flag then reports as well)
      const T wa = comp == 2 ? T(2) : T(1), wb = comp == 0 ? T(1) : T(2);
      T tsum[3] = {T(0), T(0), T(0)};
      T sx2 = T(0), sy2 = T(0);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        tsum[0] += x[e].x;
        tsum[1] += x[e].y;
        sx2 = fma(x[e].x, x[e].x, sx2);
        sy2 = fma(x[e].y, x[e].y, sy2);
      }
      tsum[2] = wa * sx2 + wb * sy2;
      if (!isfinite(tsum[0]) || !isfinite(tsum[1])) nonfinite = 1;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Kahan<T> kh{acc[(2 * j) * THREADS + tid], acc[(2 * j + 1) * THREADS + tid]};
        kh.add(tsum[j]);
        acc[(2 * j) * THREADS + tid] = kh.s;
        acc[(2 * j + 1) * THREADS + tid] = kh.c;
      }
    }
    fft_column<N, E, INV>(x, t, xbuf, idx, tw);      // ends after a barrier past its last read
    if (!a.tma_store) {
      const int x0 = (u % tiles_x) * B;
      const int row = u / tiles_x;
      // offsets within one plane (nx ny nz < 2^31); the plane bases are 64-bit pointers
      const int col0 = a.axis == 2 ? row * a.nx + x0 + b : row * a.nx * a.ny + x0 + b;
      const int nstride = a.axis == 2 ? a.nx * a.ny : a.nx;
      T* out_re = reinterpret_cast<T*>(a.out) + field * a.field_stride + (2LL * comp) * a.V;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int off = col0 + (t + TPC * e) * nstride;
        out_re[off] = x[e].x;
        out_re[a.V + off] = x[e].y;
      }
    } else {
      // the tile in box layout ([point][column], re plane then im plane) into the exchange
      // buffer, then out by tiled stores
      T* ore = reinterpret_cast<T*>(xbuf);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        ore[(t + TPC * e) * B + b] = x[e].x;
        ore[N * B + (t + TPC * e) * B + b] = x[e].y;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        const int x0 = (u % tiles_x) * B;
        const int row = u / tiles_x;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int q = 0; q < NBOX; ++q) {
            // a box starting outside the specimen region (when one is set) is skipped; one that
            // reaches past its edge is cut by the copy
            if (a.lim_x && (x0 >= a.lim_x || row >= (a.axis == 2 ? a.lim_y : a.lim_z) ||
                            q * BOX >= (a.axis == 2 ? a.lim_z : a.lim_y)))
              continue;
            const T* src = ore + p * N * B + q * BOX * B;
            if (a.axis == 2) tma_store_4d(&outmap, src, x0, row, q * BOX, plane_re + p);
            else tma_store_4d(&outmap, src, x0, q * BOX, row, plane_re + p);
          }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    if constexpr (MODE >= 2) {
      if (a.ref) {
        if (tid == 0 && !mbar_wait(&bar[s], (unsigned)((s ? ph1 : ph0) & 1))) {
          atomicOr(a.err, 1);
          abort_flag = 1;
        }
        if (s) ++ph1; else ++ph0;
        __syncthreads();
        if (abort_flag) break;
        const T* sre = stage0 + s * 2 * N * B;
        T linf = acc[tid];
        const int x0 = (u % tiles_x) * B + b, row = u / tiles_x;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int pt = t + TPC * e;
          if (MODE == 3 && !in_spec(a, x0, a.axis == 2 ? row : pt, a.axis == 2 ? pt : row)) continue;
          linf = fmax(linf, fabs(sre[pt * B + b] - x[e].x));
          linf = fmax(linf, fabs(sre[N * B + pt * B + b] - x[e].y));
        }
        acc[tid] = linf;
        __syncthreads();                               // stage s read: refill with tile k + 2
        if (abort_flag) break;
        if (tid == 0 && u + 2 * step < ntiles) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue(u + 2 * step, s, &map);
        }
      }
    }
  }
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // stores complete
  if (abort_flag) {
    // leave no copy in flight: wait (bounded) for every phase this block issued
    if (tid == 0) {
      if (issued0 > 0) mbar_wait(&bar[0], (unsigned)((issued0 - 1) & 1));
      if (issued1 > 0) mbar_wait(&bar[1], (unsigned)((issued1 - 1) & 1));
    }
    __syncthreads();
    return;
  }
  if constexpr (MODE == 1) {
    double v[4];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      v[j] = double(acc[(2 * j) * THREADS + tid]) - double(acc[(2 * j + 1) * THREADS + tid]);
    v[3] = 0.0;
    block_sum<4>(v, red);                              // starts with a block barrier
    if (tid == 0) {
      double* p = a.partials + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * 4;
      p[0] = v[0]; p[1] = v[1]; p[2] = v[2]; p[3] = nonfinite ? 1.0 : 0.0;
    }
  } else if constexpr (MODE >= 2) {
    if (a.ref) {
      double m = block_max(double(acc[tid]), red);
      if (tid == 0) a.partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = m;
    }
  }
}

// ---- strided passes for 512-point FP32 columns: 16 x 32 per column ----------------------
//
// Same tiles, stages and modes as k_strided_tma (16 columns x 512 points, TMA double buffering),
// with 512 threads: thread (b, t) = (tid % 16, tid / 16) holds points t + 32 e (e < 16) of
// column b.  Per column (the factorisation of fft512_warp): a 16-point DFT in registers, the
// twiddle W512^(t k1), one exchange through a column-padded buffer (pitch 513 complex words:
// conflict-free per half-warp), a 16-point DFT over the even / odd halves of the 32-point DFTs and
// a radix-2 combine of threads t and t ^ 1 (lanes l and l ^ 16 of one warp) by shuffle.  Thread
// (b, 2 kap + h) then holds output kap + 16 q + 256 h in slot q.  The next tile's copy is issued
// after the exchange barrier, so a tile costs two block barriers (four with the L-inf residual,
// two more with TMA stores through the exchange buffer).
struct Tma16Cfg {
  static constexpr int N = 512, E = 16, TPC = 32, B = 16, THREADS = 512, BOX = 256, NBOX = 2;
  static constexpr int XP = 513;                                  // complex words per column
  static constexpr size_t STAGE_BYTES = 2 * sizeof(float) * size_t(N) * B;
  static constexpr size_t SMEM = 1024 + sizeof(float2) * 512 + 2 * STAGE_BYTES +
                                 sizeof(float2) * size_t(XP) * B + 6 * sizeof(float) * THREADS;
};

template <bool INV, int MODE>
__global__ void __launch_bounds__(Tma16Cfg::THREADS, 1)
k_strided16(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap refmap,
            const __grid_constant__ CUtensorMap outmap, const TmaArgs a) {
  using C = Tma16Cfg;
  using T = float;
  using T2 = float2;
  constexpr int N = C::N, B = C::B, BOX = C::BOX, NBOX = C::NBOX, XP = C::XP, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_t16[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_t16) + 127) & ~uintptr_t(127));
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(base);
  T* stage0 = reinterpret_cast<T*>(base + 128);      // stage s at stage0 + s * 2 N B
  T2* tw = reinterpret_cast<T2*>(stage0 + 4 * N * B);   // W512^(t k1) at [k1][t]
  T2* xbuf = tw + 512;
  T* acc = reinterpret_cast<T*>(xbuf + XP * B);     // [6][THREADS] running sums (MODE 1, 2)
  __shared__ double red[32 * 4];
  __shared__ int abort_flag, nonfinite;

  const int tid = threadIdx.x;
  const int b = tid % B, t = tid / B;
  const int kap = t >> 1, h = t & 1;
  const int field = blockIdx.y / a.ncomp, comp = blockIdx.y % a.ncomp;
  const int plane_re = field * 2 * a.ncomp + 2 * comp;
  const int tiles_x = a.nx / B;
  const int ntiles = (int)a.ntiles;

  // W512^(t k1) from the plain table W512^m (m < 512)
  for (int i = tid; i < 512; i += blockDim.x)
    tw[i] = reinterpret_cast<const T2*>(a.tw)[((i & 31) * (i >> 5)) & 511];
  if constexpr (MODE != 0) {
#pragma unroll
    for (int j = 0; j < 6; ++j) acc[j * THREADS + tid] = T(0);
  }
  if (tid == 0) {
    abort_flag = 0;
    nonfinite = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  int issued0 = 0, issued1 = 0;                      // loads issued per stage (thread 0)
  auto issue = [&](int u, int s, const CUtensorMap* m) {
    const int x0 = (u % tiles_x) * B;
    const int row = u / tiles_x;
    if (s) ++issued1; else ++issued0;
    mbar_expect_tx(&bar[s], (unsigned)C::STAGE_BYTES);
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < NBOX; ++q) {
        T* dst = stage0 + s * 2 * N * B + p * N * B + q * BOX * B;
        if (a.axis == 2) tma_load_4d(dst, m, &bar[s], x0, row, q * BOX, plane_re + p);
        else tma_load_4d(dst, m, &bar[s], x0, q * BOX, row, plane_re + p);
      }
  };
  int ph0 = 0, ph1 = 0;                              // completed phases per stage
  const int first = blockIdx.x, step = gridDim.x;
  if (tid == 0) {
    if (first < ntiles) issue(first, 0, &map);
    if (first + step < ntiles) issue(first + step, 1, &map);
  }
  const T sg = h ? T(-1) : T(1);

  int k = 0;
  for (int u = first; u < ntiles; u += step, ++k) {
    const int s = k & 1;
    if (tid == 0 && !mbar_wait(&bar[s], (unsigned)((s ? ph1 : ph0) & 1))) {
      atomicOr(a.err, 1);
      abort_flag = 1;
    }
    if (s) ++ph1; else ++ph0;
    // first pass with tiled stores: the tile's output leaves from its own load stage (free once
    // the exchange is written), so no later tile waits for the stores before its exchange; the
    // stage is refilled one tile later, once those stores have read it.  Otherwise the stores
    // leave from the exchange buffer, which the last tile's stores must have read by now.
    const bool OS = MODE == 1 && a.tma_store;
    if (tid == 0 && !OS) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncthreads();                                 // stage s ready; the last tile fully done
    if (abort_flag) break;
    T2 v[16];
    {
      const T* sre = stage0 + s * 2 * N * B;
#pragma unroll
      for (int e = 0; e < 16; ++e)
        v[e] = T2{sre[(t + 32 * e) * B + b], sre[N * B + (t + 32 * e) * B + b]};
    }
    // last pass: stage s is read, so this tile's input (for the residual) can start loading into
    // it now rather than behind the exchange; the other passes refill it there instead (an extra
    // barrier measured slower for them)
    constexpr bool EARLY = MODE >= 2;
    if (EARLY && a.ref) {
      __syncthreads();
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(u, s, &refmap);
      }
    }
    T sx2 = T(0), sy2 = T(0);
    if constexpr (MODE == 1) {
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        sx2 = fma(v[e].x, v[e].x, sx2);
        sy2 = fma(v[e].y, v[e].y, sy2);
      }
    }
    // transform: 16-point DFT over e, twiddle, exchange
    dft16<INV>(v);
    if constexpr (MODE == 1) {
      // statistics of the 16 points: sums from the DFT's zero-frequency output (their plain sum),
      // squares weighted by the Voigt multiplicity of each plane (xx yy | zz yz | xz xy)
      const T wa = comp == 2 ? T(2) : T(1), wb = comp == 0 ? T(1) : T(2);
      const T tsum[3] = {v[0].x, v[0].y, wa * sx2 + wb * sy2};
      if (!isfinite(tsum[0]) || !isfinite(tsum[1])) nonfinite = 1;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Kahan<T> kh{acc[(2 * j) * THREADS + tid], acc[(2 * j + 1) * THREADS + tid]};
        kh.add(tsum[j]);
        acc[(2 * j) * THREADS + tid] = kh.s;
        acc[(2 * j + 1) * THREADS + tid] = kh.c;
      }
    }
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
      T2 w = tw[k1 * 32 + t];
      if (INV) w.y = -w.y;
      v[k1] = cmul(v[k1], w);
    }
    T2* xc = xbuf + b * XP;
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) xc[k1 * 32 + (t ^ (2 * k1))] = v[k1];
    __syncthreads();                                 // exchange written; stage s fully read
    if (tid == 0 && !OS && !(EARLY && a.ref) && u + 2 * step < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(u + 2 * step, s, &map);
    }
    // stage s ^ 1 takes tile u + step once the last tile's stores have read it
    if (tid == 0 && OS && k >= 1 && u + step < ntiles) {
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(u + step, s ^ 1, &map);
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = xc[kap * 32 + h + 2 * (m ^ kap)];
    dft16<INV>(v);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const T2 tq = mul_w32_rt<INV>(q, v[q]);
      const T2 send = h ? tq : v[q];
      T2 recv;
      recv.x = __shfl_xor_sync(0xffffffffu, send.x, 16);
      recv.y = __shfl_xor_sync(0xffffffffu, send.y, 16);
      v[q] = cfma_s(sg, send, recv);
    }
    // slot q holds point kap + 16 q + 256 h of column b
    if (!a.tma_store) {
      const int x0 = (u % tiles_x) * B;
      const int row = u / tiles_x;
      const int col0 = a.axis == 2 ? row * a.nx + x0 + b : row * a.nx * a.ny + x0 + b;
      const int nstride = a.axis == 2 ? a.nx * a.ny : a.nx;
      T* out_re = reinterpret_cast<T*>(a.out) + field * a.field_stride + (2LL * comp) * a.V;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int off = col0 + (kap + 16 * q + 256 * h) * nstride;
        out_re[off] = v[q].x;
        out_re[a.V + off] = v[q].y;
      }
    } else {
      // the tile in box layout ([point][column], re plane then im plane) into the tile's load
      // stage (first pass) or the exchange buffer (every read of it is behind the barrier
      // below), then out by tiled stores
      if (!OS) __syncthreads();
      T* ore = OS ? stage0 + s * 2 * N * B : reinterpret_cast<T*>(xbuf);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int pnt = (kap + 16 * q + 256 * h) * B + b;
        ore[pnt] = v[q].x;
        ore[N * B + pnt] = v[q].y;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        const int x0 = (u % tiles_x) * B;
        const int row = u / tiles_x;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int q = 0; q < NBOX; ++q) {
            // a box starting outside the specimen region (when one is set) is skipped; one that
            // reaches past its edge is cut by the copy
            if (a.lim_x && (x0 >= a.lim_x || row >= (a.axis == 2 ? a.lim_y : a.lim_z) ||
                            q * BOX >= (a.axis == 2 ? a.lim_z : a.lim_y)))
              continue;
            const T* src = ore + p * N * B + q * BOX * B;
            if (a.axis == 2) tma_store_4d(&outmap, src, x0, row, q * BOX, plane_re + p);
            else tma_store_4d(&outmap, src, x0, q * BOX, row, plane_re + p);
          }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    if constexpr (MODE >= 2) {
      if (a.ref) {
        if (tid == 0 && !mbar_wait(&bar[s], (unsigned)((s ? ph1 : ph0) & 1))) {
          atomicOr(a.err, 1);
          abort_flag = 1;
        }
        if (s) ++ph1; else ++ph0;
        __syncthreads();
        if (abort_flag) break;
        const T* sre = stage0 + s * 2 * N * B;
        T linf = acc[tid];
        const int x0 = (u % tiles_x) * B + b, row = u / tiles_x;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int pt = kap + 16 * q + 256 * h;
          if (MODE == 3 && !in_spec(a, x0, a.axis == 2 ? row : pt, a.axis == 2 ? pt : row)) continue;
          const int pnt = pt * B + b;
          linf = fmax(linf, fabs(sre[pnt] - v[q].x));
          linf = fmax(linf, fabs(sre[N * B + pnt] - v[q].y));
        }
        acc[tid] = linf;
        __syncthreads();                             // stage s read: refill with tile k + 2
        if (tid == 0 && u + 2 * step < ntiles) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue(u + 2 * step, s, &map);
        }
      }
    }
  }
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // stores complete
  if (abort_flag) {
    if (tid == 0) {
      if (issued0 > 0) mbar_wait(&bar[0], (unsigned)((issued0 - 1) & 1));
      if (issued1 > 0) mbar_wait(&bar[1], (unsigned)((issued1 - 1) & 1));
    }
    __syncthreads();
    return;
  }
  if constexpr (MODE == 1) {
    double r[4];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      r[j] = double(acc[(2 * j) * THREADS + tid]) - double(acc[(2 * j + 1) * THREADS + tid]);
    r[3] = 0.0;
    block_sum<4>(r, red);
    if (tid == 0) {
      double* p = a.partials + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * 4;
      p[0] = r[0]; p[1] = r[1]; p[2] = r[2]; p[3] = nonfinite ? 1.0 : 0.0;
    }
  } else if constexpr (MODE >= 2) {
    if (a.ref) {
      double m = block_max(double(acc[tid]), red);
      if (tid == 0) a.partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = m;
    }
  }
}

// ---- fused x pass with bulk-copy double buffering --------------------------------------
//
// Same work as k_xproj (forward x transform of P row pairs, projector per mode pair, inverse x
// transform).  The rows of group g + 2 stream into shared memory with cp.async.bulk (one 1-D copy
// per row and plane) while the block works on group g; the results leave through a shared
// staging buffer with cp.async.bulk stores (one per row and plane), so the store traffic costs
// the threads nothing.  The exchanges use split real/imaginary arrays and per-stage twiddle
// tables, both laid out so that a warp's accesses hit distinct banks.

__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(
                   reinterpret_cast<unsigned long long>(gdst)),
               "r"(smem_u32(ssrc)), "r"(bytes)
               : "memory");
}

// V = 0: two row pairs per block (FP32, N <= 512), one block per SM; V = 1: one row pair per
// block, two blocks per SM.
template <typename T, int N, int V = 0> struct XTmaCfg {
  static constexpr int E = 8;
  static constexpr int TPC = N / E;
  static constexpr int P = (V == 0 && sizeof(T) == 4 && N <= 512) ? 2 : 1;
  static constexpr int MINB = V == 0 ? 1 : 2;
  static constexpr int XCOLS = 6 * P;
  static constexpr int THREADS = XCOLS * TPC;
  static constexpr int PF = N;                                          // exchange row (swizzled)
  static constexpr int TWS = staged_size(N);
  using T2 = typename V2<T>::t;
  static constexpr size_t STAGE_BYTES = 2 * sizeof(T) * size_t(N) * XCOLS;   // re + im rows
  static constexpr size_t SMEM = 1024 + 3 * STAGE_BYTES + 2 * sizeof(T) * size_t(XCOLS) * PF +
                                 2 * sizeof(T) * TWS + sizeof(T) * N;
  static constexpr bool OK = N >= 64 && THREADS * MINB <= 1024 && SMEM * MINB <= 227 * 1024 &&
                            (V == 0 || P == 1);
};

struct XTmaArgs {
  void* data;
  const void* tws;         // per-stage twiddles of the x length: cos[TWS] then sin[TWS]; for
                           // N = 512 followed by W512^(l k1) as complex [16][32]
  const void* xi_x;
  const void* xi_y;
  const void* xi_z;
  const int* pairs;
  const double* mean;
  double* partials;        // [batch][grid][4]
  int* err;
  long long field_stride, V;
  int nx, ny, nz;
  int npairs, ngroups;
  int nyq_zero;
  int compat;              // 1: return the compatible part c0 + (S - S_equil)
  double inv_v;
  void* ydata;             // potential mode: field 0, plane 0 of the 4-plane y buffer
  long long yfield_stride; // elements between fields of the y buffer (4 V)
};

template <typename T, int N, int V>
__global__ void __launch_bounds__(XTmaCfg<T, N, V>::THREADS, XTmaCfg<T, N, V>::MINB)
k_xproj_tma(const XTmaArgs a) {
  using C = XTmaCfg<T, N, V>;
  using T2 = typename C::T2;
  constexpr int E = C::E, TPC = C::TPC, P = C::P, PF = C::PF, XCOLS = C::XCOLS, TWS = C::TWS;
  extern __shared__ __align__(16) unsigned char smem_xt[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_xt) + 127) & ~uintptr_t(127));
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(base);
  T* stage0 = reinterpret_cast<T*>(base + 128);       // stage s at stage0 + s * 2 N XCOLS
  T* outs = stage0 + 4 * N * XCOLS;                     // bulk-store source, [col][plane][N]
  T* xre = outs + 2 * N * XCOLS;                        // exchange, [col][PF]
  T* xim = xre + XCOLS * PF;
  T* twc = xim + XCOLS * PF;
  T* tws = twc + TWS;
  T* xix = tws + TWS;
  __shared__ double red[32 * 4];
  __shared__ int abort_flag;
  __shared__ int rinfo[2][P][6];                        // rowA, rowB, self, valid, kz, ky
  __shared__ T rxi[2][P][2];                            // Xi_y(ky), Xi_z(kz)

  const int tid = threadIdx.x;
  for (int i = tid; i < TWS; i += blockDim.x) {
    twc[i] = reinterpret_cast<const T*>(a.tws)[i];
    tws[i] = reinterpret_cast<const T*>(a.tws)[TWS + i];
  }
  for (int i = tid; i < N; i += blockDim.x) xix[i] = reinterpret_cast<const T*>(a.xi_x)[i];
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const TwStaged<T> tw{twc, tws};
  const T* xiy = reinterpret_cast<const T*>(a.xi_y);
  const T* xiz = reinterpret_cast<const T*>(a.xi_z);
  const int col = tid / TPC, t = tid % TPC;
  const int slot = col / 6, side = (col % 6) / 3;
  const int field = blockIdx.y;
  T* fdata = reinterpret_cast<T*>(a.data) + field * a.field_stride;
  T zmv[6];
  const T* zm = zero_mode_values(a.mean ? a.mean + field * 6 : nullptr, 1.0 / a.inv_v, zmv)
                    ? zmv : nullptr;
  const SoaAcc<T> acc{xre + col * PF, xim + col * PF};
  const T inv_v = T(a.inv_v);

  auto mirror = [&](int r) {
    const int kz = r / a.ny, ky = r - kz * a.ny;
    return (kz == 0 ? 0 : a.nz - kz) * a.ny + (ky == 0 ? 0 : a.ny - ky);
  };
  int issued0 = 0, issued1 = 0;
  // thread 0: stream the rows of group g into stage s (skipping absent and mirror-of-self rows)
  auto issue = [&](int g, int s) {
    unsigned bytes = 0;
    int rows[2 * P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int p = g * P + q;
      rows[2 * q] = rows[2 * q + 1] = -1;
      if (p < a.npairs) {
        const int rA = a.pairs[p], rB = mirror(rA);
        rows[2 * q] = rA;
        rows[2 * q + 1] = rB == rA ? -1 : rB;
      }
      bytes += ((rows[2 * q] >= 0 ? 6u : 0u) + (rows[2 * q + 1] >= 0 ? 6u : 0u)) * N * sizeof(T);
    }
    if (s) ++issued1; else ++issued0;
    mbar_expect_tx(&bar[s], bytes);
    T* st = stage0 + s * 2 * N * XCOLS;
#pragma unroll
    for (int q = 0; q < P; ++q)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int r = rows[2 * q + sd];
        if (r < 0) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int pl = 0; pl < 2; ++pl) {
            const int cc = q * 6 + sd * 3 + c;
            bulk_load(st + (2 * cc + pl) * N, fdata + (2LL * c + pl) * a.V + (long long)r * N,
                      N * sizeof(T), &bar[s]);
          }
      }
  };
  const int first = blockIdx.x, step = gridDim.x;
  if (tid == 0) {
    if (first < a.ngroups) issue(first, 0);
    if (first + step < a.ngroups) issue(first + step, 1);
  }

  Kahan<T> r2, di2, do2, o2;
  int k = 0;
  for (int g = first; g < a.ngroups; g += step, ++k) {
    const int s = k & 1;
    if (tid < P) {                                      // row information of this group
      const int p = g * P + tid;
      const int rA = p < a.npairs ? a.pairs[p] : 0;
      const int rB = mirror(rA);
      const int kz = rA / a.ny, ky = rA - kz * a.ny;
      rinfo[s][tid][0] = rA;
      rinfo[s][tid][1] = rB;
      rinfo[s][tid][2] = rA == rB;
      rinfo[s][tid][3] = p < a.npairs;
      rinfo[s][tid][4] = kz;
      rinfo[s][tid][5] = ky;
      rxi[s][tid][0] = xiy[ky];
      rxi[s][tid][1] = xiz[kz];
    }
    if (tid == 0 && !mbar_wait(&bar[s], (k >> 1) & 1)) {
      atomicOr(a.err, 1);
      abort_flag = 1;
    }
    __syncthreads();
    if (abort_flag) break;
    const bool active = rinfo[s][slot][3] && !(side == 1 && rinfo[s][slot][2]);
    T2 x[E];
    {
      const T* sre = stage0 + s * 2 * N * XCOLS + (2 * col) * N;
      const T* sim = sre + N;
#pragma unroll
      for (int e = 0; e < E; ++e)
        x[e] = active ? T2{sre[t + TPC * e], sim[t + TPC * e]} : T2{T(0), T(0)};
    }
    __syncthreads();                                   // stage s is free again
    if (tid == 0 && g + 2 * step < a.ngroups) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(g + 2 * step, s);
    }
    fft_column_acc<N, E, false>(x, t, acc, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) acc.put(t + TPC * e, x[e]);
    __syncthreads();
    for (int item = tid; item < P * N; item += blockDim.x) {
      const int s2 = item / N, kx = item - s2 * N;
      if (!rinfo[s][s2][3]) continue;
      const int rA = rinfo[s][s2][0];
      const bool self2 = rinfo[s][s2][2];
      const int kxm = kx == 0 ? 0 : N - kx;
      if (self2 && kx > kxm) continue;
      const int colA = s2 * 6, colB = self2 ? s2 * 6 : s2 * 6 + 3;
      const int ja = swz(kx), jb = swz(kxm);
      T2 av[3], bv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        av[c] = T2{xre[(colA + c) * PF + ja], xim[(colA + c) * PF + ja]};
        bv[c] = T2{xre[(colB + c) * PF + jb], xim[(colB + c) * PF + jb]};
      }
      const bool selfmode = self2 && kx == kxm;
      project_pair<T>(av, bv, xix[kx], rxi[s][s2][0], rxi[s][s2][1], rA == 0 && kx == 0, zm,
                      a.nyq_zero != 0, a.compat != 0, inv_v, selfmode ? T(1) : T(2), r2, di2, do2, o2);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        xre[(colA + c) * PF + ja] = av[c].x;
        xim[(colA + c) * PF + ja] = av[c].y;
        if (!selfmode) {
          xre[(colB + c) * PF + jb] = bv[c].x;
          xim[(colB + c) * PF + jb] = bv[c].y;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = acc.get(t + TPC * e);
    __syncthreads();
    fft_column_acc<N, E, true>(x, t, acc, tw);
    // results -> staging -> bulk stores; the previous group's stores must have read it first
    if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncthreads();
    if (active) {
      T* ore = outs + (2 * col) * N;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        ore[t + TPC * e] = x[e].x;
        ore[N + t + TPC * e] = x[e].y;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
#pragma unroll
      for (int q = 0; q < P; ++q) {
        if (!rinfo[s][q][3]) continue;
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          if (sd == 1 && rinfo[s][q][2]) continue;
          const int r = rinfo[s][q][sd];
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int pl = 0; pl < 2; ++pl) {
              const int cc = q * 6 + sd * 3 + c;
              bulk_store(fdata + (2LL * c + pl) * a.V + (long long)r * N, outs + (2 * cc + pl) * N,
                         N * sizeof(T));
            }
        }
      }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  if (abort_flag) {
    if (tid == 0) {
      if (issued0 > 0) mbar_wait(&bar[0], (unsigned)((issued0 - 1) & 1));
      if (issued1 > 0) mbar_wait(&bar[1], (unsigned)((issued1 - 1) & 1));
    }
    __syncthreads();
    return;
  }
  double v[4] = {r2.value(), di2.value(), do2.value(), o2.value()};
  block_sum<4>(v, red);
  if (tid == 0) {
    double* q = a.partials + ((long long)field * gridDim.x + blockIdx.x) * 4;
    q[0] = v[0]; q[1] = v[1]; q[2] = v[2]; q[3] = v[3];
  }
}

// ---- fused x pass, one warp per row -------------------------------------------------------
//
// A block holds one row pair: six warps, one per (row, component), each holding its row of N
// points as 32 lanes x E = N / 32 registers.  The x transforms exchange through warp-private
// shared rows (split real / imaginary, bank swizzle) with warp barriers only; the block meets
// three times per row pair (rows read from the bulk-copy stage; forward results in place; modes
// projected).  Rows arrive by cp.async.bulk into a single stage that is refilled for the next row
// pair as soon as it has been read, and leave by cp.async.bulk stores from each warp's row.
// Several blocks share an SM, so one block's barriers overlap the others' work.

template <typename T, int N, int MINB = 1> struct XwCfg {
  static constexpr int E = N / 32;
  static constexpr int THREADS = 6 * 32;
  static constexpr int TWS = staged_size(N);
  // 16 x 32 transform (fft512_warp) in FP32; in FP64 (ALU-bound on GB300) the radix-8 stages
  // measured faster
  static constexpr bool F16 = N == 512 && sizeof(T) == 4;
  static constexpr size_t ROWS_BYTES = 12 * sizeof(T) * size_t(N);      // 6 rows x (re, im)
  static constexpr size_t TW_BYTES = F16 ? 2 * sizeof(T) * 512 : 2 * sizeof(T) * TWS;
  static constexpr size_t SMEM = 256 + 2 * ROWS_BYTES + TW_BYTES + sizeof(T) * N;
  static constexpr bool OK = (N == 256 || N == 512) && SMEM <= 227 * 1024;
};

// POT: the potential x pass of eq_project_hodge instead (reads the spectrum rows, forms the packed
// y spectra per mode pair with potential_pair in the rows of components 0 and 1, and those two
// warps of each side store their inverse transforms into the y buffer; nothing else is written).
template <typename T, int N, int MINB, bool POT>
__global__ void __launch_bounds__(XwCfg<T, N, MINB>::THREADS, MINB)
k_xproj_warp(const XTmaArgs a) {
  using C = XwCfg<T, N, MINB>;
  using T2 = typename V2<T>::t;
  constexpr int E = C::E, TWS = C::TWS;
  constexpr bool F16 = C::F16;
  extern __shared__ __align__(16) unsigned char smem_xw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_xw) + 127) & ~uintptr_t(127));
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(base);
  T* stage = reinterpret_cast<T*>(base + 128);          // [warp][plane][N], bulk-copy target
  T* rows = stage + 12 * N;                             // [warp][plane][N], exchange + store source
  T* twc = rows + 12 * N;                               // staged cos, or the W512 table (F16)
  T* tws = twc + TWS;
  T2* tw16 = reinterpret_cast<T2*>(twc);
  T* xix = F16 ? reinterpret_cast<T*>(tw16 + 512) : tws + TWS;
  __shared__ double red[32 * 4];
  __shared__ int abort_flag;
  __shared__ int rinfo[2][6];                           // rowA, rowB, self, valid, kz, ky
  __shared__ T rxi[2][2];                               // Xi_y(ky), Xi_z(kz)

  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int side = w / 3, comp = w % 3;
  if constexpr (F16) {
    const T2* src = reinterpret_cast<const T2*>(reinterpret_cast<const T*>(a.tws) + 2 * TWS);
    for (int i = tid; i < 512; i += blockDim.x) tw16[i] = src[i];
  } else {
    for (int i = tid; i < TWS; i += blockDim.x) {
      twc[i] = reinterpret_cast<const T*>(a.tws)[i];
      tws[i] = reinterpret_cast<const T*>(a.tws)[TWS + i];
    }
  }
  for (int i = tid; i < N; i += blockDim.x) xix[i] = reinterpret_cast<const T*>(a.xi_x)[i];
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const TwStaged<T> tw{twc, tws};
  const T* xiy = reinterpret_cast<const T*>(a.xi_y);
  const T* xiz = reinterpret_cast<const T*>(a.xi_z);
  const int field = blockIdx.y;
  T* fdata = reinterpret_cast<T*>(a.data) + field * a.field_stride;
  T zmv[6];
  const T* zm = zero_mode_values(a.mean ? a.mean + field * 6 : nullptr, 1.0 / a.inv_v, zmv)
                    ? zmv : nullptr;
  T* wre = rows + (2 * w) * N;
  T* wim = wre + N;
  const SoaAcc<T> acc{wre, wim};
  const T inv_v = T(a.inv_v);

  // thread 0: rows of row pair g into info slot s, then stream them into the stage
  int issued = 0;
  auto issue = [&](int g, int s) {
    const int rA = a.pairs[g];
    const int kz = rA / a.ny, ky = rA - kz * a.ny;
    const int rB = (kz == 0 ? 0 : a.nz - kz) * a.ny + (ky == 0 ? 0 : a.ny - ky);
    rinfo[s][0] = rA; rinfo[s][1] = rB; rinfo[s][2] = rA == rB; rinfo[s][3] = 1;
    rinfo[s][4] = kz; rinfo[s][5] = ky;
    rxi[s][0] = xiy[ky];
    rxi[s][1] = xiz[kz];
    const int nrows = rA == rB ? 3 : 6;
    ++issued;
    mbar_expect_tx(bar, (unsigned)(nrows * 2 * N * sizeof(T)));
    for (int r = 0; r < nrows; ++r) {
      const int row = r < 3 ? rA : rB, c = r % 3;
      for (int pl = 0; pl < 2; ++pl)
        bulk_load(stage + (2 * r + pl) * N, fdata + (2LL * c + pl) * a.V + (long long)row * N,
                  N * sizeof(T), bar);
    }
  };
  __syncthreads();
  const int first = blockIdx.x, step = gridDim.x;
  if (tid == 0 && first < a.npairs) issue(first, 0);

  Kahan<T> r2, di2, do2, o2;
  int k = 0;
  for (int g = first; g < a.npairs; g += step, ++k) {
    const int s = k & 1;
    if (tid == 0 && !mbar_wait(bar, k & 1)) {
      atomicOr(a.err, 1);
      abort_flag = 1;
    }
    __syncthreads();
    if (abort_flag) break;
    const bool self = rinfo[s][2];
    const bool active = !(side == 1 && self);
    T2 x[E];
    {
      const T* sre = stage + (2 * w) * N;
#pragma unroll
      for (int e = 0; e < E; ++e)
        x[e] = active ? T2{sre[lane + 32 * e], sre[N + lane + 32 * e]} : T2{T(0), T(0)};
    }
    __syncthreads();                                    // stage free: refill for the next pair
    if (tid == 0 && g + step < a.npairs) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(g + step, s ^ 1);
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncwarp();                                       // this warp's row no longer being stored
    if constexpr (F16) {
      // spectrum as interleaved complex values in the warp's row
      T2* wrow = reinterpret_cast<T2*>(wre);
      fft512_warp<false>(x, lane, wrow, tw16);
      const int kap = lane >> 1, h = lane & 1;
#pragma unroll
      for (int q = 0; q < 16; ++q) wrow[sx512(kap + 16 * q + 256 * h)] = x[q];
    } else {
      fft_column_acc<N, E, false, 0, true>(x, lane, acc, tw);
#pragma unroll
      for (int e = 0; e < E; ++e) acc.put(lane + 32 * e, x[e]);
    }
    __syncthreads();
    const int rA = rinfo[s][0];
    for (int kx = tid; kx < N; kx += blockDim.x) {
      const int kxm = kx == 0 ? 0 : N - kx;
      if (self && kx > kxm) continue;
      const int ja = F16 ? sx512(kx) : swz(kx), jb = F16 ? sx512(kxm) : swz(kxm);
      T2 av[3], bv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T* ra = rows + (2 * c) * N;
        const T* rb = rows + (2 * (self ? c : 3 + c)) * N;
        if constexpr (F16) {
          av[c] = reinterpret_cast<const T2*>(ra)[ja];
          bv[c] = reinterpret_cast<const T2*>(rb)[jb];
        } else {
          av[c] = T2{ra[ja], ra[N + ja]};
          bv[c] = T2{rb[jb], rb[N + jb]};
        }
      }
      const bool selfmode = self && kx == kxm;
      if constexpr (POT) {
        T2 yk[2], ym[2];
        potential_pair<T>(av, bv, xix[kx], rxi[s][0], rxi[s][1], inv_v, yk, ym);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          av[c] = yk[c];
          bv[c] = ym[c];
        }
      } else {
        project_pair<T>(av, bv, xix[kx], rxi[s][0], rxi[s][1], rA == 0 && kx == 0, zm,
                        a.nyq_zero != 0, a.compat != 0, inv_v, selfmode ? T(1) : T(2), r2, di2,
                        do2, o2);
      }
#pragma unroll
      for (int c = 0; c < (POT ? 2 : 3); ++c) {
        T* ra = rows + (2 * c) * N;
        T* rb = rows + (2 * (self ? c : 3 + c)) * N;
        if constexpr (F16) {
          reinterpret_cast<T2*>(ra)[ja] = av[c];
          if (!selfmode) reinterpret_cast<T2*>(rb)[jb] = bv[c];
        } else {
          ra[ja] = av[c].x;
          ra[N + ja] = av[c].y;
          if (!selfmode) {
            rb[jb] = bv[c].x;
            rb[N + jb] = bv[c].y;
          }
        }
      }
    }
    __syncthreads();
    if (POT && comp == 2) continue;                    // no y row for this warp (warp-uniform)
    if constexpr (F16) {
      T2* wrow = reinterpret_cast<T2*>(wre);
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = wrow[sx512(lane + 32 * e)];
      fft512_warp<true>(x, lane, wrow, tw16);
      // results in natural order into this warp's row, then one bulk store per plane
      const int kap = lane >> 1, h = lane & 1;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        wre[kap + 16 * q + 256 * h] = x[q].x;
        wim[kap + 16 * q + 256 * h] = x[q].y;
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = acc.get(lane + 32 * e);
      __syncwarp();
      fft_column_acc<N, E, true, 0, true>(x, lane, acc, tw);
      // results in natural order (unswizzled) into this warp's row, then one bulk store per plane
#pragma unroll
      for (int e = 0; e < E; ++e) {
        wre[lane + 32 * e] = x[e].x;
        wim[lane + 32 * e] = x[e].y;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0 && active) {
      const int row = side == 0 ? rA : rinfo[s][1];
      T* dst = POT ? reinterpret_cast<T*>(a.ydata) + field * a.yfield_stride : fdata;
      bulk_store(dst + (2LL * comp) * a.V + (long long)row * N, wre, N * sizeof(T));
      bulk_store(dst + (2LL * comp + 1) * a.V + (long long)row * N, wim, N * sizeof(T));
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  if (abort_flag) {
    if (tid == 0 && issued > 0) mbar_wait(bar, (unsigned)((issued - 1) & 1));
    __syncthreads();
    return;
  }
  if constexpr (!POT) {
    double v[4] = {r2.value(), di2.value(), do2.value(), o2.value()};
    block_sum<4>(v, red);
    if (tid == 0) {
      double* q = a.partials + ((long long)field * gridDim.x + blockIdx.x) * 4;
      q[0] = v[0]; q[1] = v[1]; q[2] = v[2]; q[3] = v[3];
    }
  }
}

}  // namespace eqk
