// eq_xrow.cuh - fused x pass, one warp per row, rows read from and written to global memory by
// the threads themselves (no staging copy through shared memory).
//
// Work per row pair (rows (ky, kz) and (-ky, -kz), three complex fields each, as in k_xproj_warp):
// every warp loads its row of N points straight into registers (lane l holds points l + 32 e, one
// coalesced 128-byte load per plane and e), takes the forward x transform through its own shared
// row, and leaves the spectrum there; the block meets once; every thread projects its mode pairs
// (k, -k) across the six rows (project_pair, norm terms summed per row pair in the working
// precision and folded into compensated per-thread sums); the block meets again; every warp
// takes the inverse transform of its row and stores the result from registers.  Two block
// barriers per row pair and no bulk copies: shared memory carries only the transform exchange and
// the projection, about a third less traffic than staging the rows through it, and no thread
// waits on a copy barrier.  Several blocks share an SM, so one block's loads and barriers overlap
// the others' arithmetic.
#pragma once
#include <type_traits>

#include "eq_fft_pair.cuh"
#include "eq_tma.cuh"

namespace eqk {

template <typename T, int N> struct XrCfg {
  static constexpr int E = N / 32;
  static constexpr int THREADS = 6 * 32;
  static constexpr int TWS = staged_size(N);
  // 16 x 32 warp transform for 512-point FP32 rows, radix-8 stages otherwise (as k_xproj_warp)
  static constexpr bool F16 = N == 512 && sizeof(T) == 4;
  static constexpr size_t ROWS_BYTES = 12 * sizeof(T) * size_t(N);       // 6 rows x (re, im)
  static constexpr size_t TW_BYTES = F16 ? 2 * sizeof(T) * 512 : 2 * sizeof(T) * TWS;
  static constexpr size_t SMEM = ROWS_BYTES + TW_BYTES + sizeof(T) * N;
  static constexpr bool OK = (N == 256 || N == 512) && SMEM <= 227 * 1024;
};

// POT: the potential x pass of eq_project_hodge (reads the stress spectrum, forms the packed y
// spectra per mode pair with potential_pair in the rows of components 0 and 1, and those warps
// of each side store their inverse transforms into the y buffer; the stress spectrum is not
// written).
// PF: each warp loads its row of the next row pair into registers as soon as its forward
// transform is done, so those loads are in flight during the projection and the inverse
// transform (about 2 N / 32 more registers a thread).
template <typename T, int N, int MINB, bool POT, bool PF = false>
__global__ void __launch_bounds__(XrCfg<T, N>::THREADS, MINB)
k_xproj_rows(const XTmaArgs a) {
  using C = XrCfg<T, N>;
  using T2 = typename V2<T>::t;
  constexpr int E = C::E, TWS = C::TWS;
  constexpr bool F16 = C::F16;
  extern __shared__ __align__(16) unsigned char smem_xr[];
  T* rows = reinterpret_cast<T*>(smem_xr);            // [warp][re N | im N], or [warp][N] T2 (F16)
  T* twc = rows + 12 * N;                              // staged cos, or the W512 table (F16)
  T* tws = twc + TWS;
  T2* tw16 = reinterpret_cast<T2*>(twc);
  T* xix = F16 ? reinterpret_cast<T*>(tw16 + 512) : tws + TWS;
  __shared__ double red[32 * 4];

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
  __syncthreads();
  const TwStaged<T> tw{twc, tws};
  const T* xiy = reinterpret_cast<const T*>(a.xi_y);
  const T* xiz = reinterpret_cast<const T*>(a.xi_z);
  const int field = blockIdx.y;
  T* fdata = reinterpret_cast<T*>(a.data) + field * a.field_stride;
  T* ydst = POT ? reinterpret_cast<T*>(a.ydata) + field * a.yfield_stride : nullptr;
  T zmv[6];
  const T* zm = zero_mode_values(a.mean ? a.mean + field * 6 : nullptr, 1.0 / a.inv_v, zmv)
                    ? zmv : nullptr;
  T* wre = rows + (2 * w) * N;
  T* wim = wre + N;
  T2* wrow = reinterpret_cast<T2*>(wre);
  const SoaAcc<T> acc{wre, wim};
  const T inv_v = T(a.inv_v);
  const int kap = lane >> 1, hh = lane & 1;

  // row of row pair g handled by this warp: rows (ky, kz) and (-ky, -kz); a self-mirror pair
  // has one row, and the warps of side 1 sit out
  struct RowOf {
    int rA, kz, ky;
    bool self, active;
    long long off;
  };
  auto row_of = [&](int g) {
    RowOf r;
    r.rA = a.pairs[g];
    r.kz = r.rA / a.ny;
    r.ky = r.rA - r.kz * a.ny;
    const int rB = (r.kz == 0 ? 0 : a.nz - r.kz) * a.ny + (r.ky == 0 ? 0 : a.ny - r.ky);
    r.self = r.rA == rB;
    r.active = !(side == 1 && r.self);                  // warp-uniform
    r.off = (long long)(side == 0 ? r.rA : rB) * N;
    return r;
  };
  const T* src_re = fdata + (2LL * comp) * a.V;
  const T* src_im = src_re + a.V;
  T2 xn[PF ? E : 1];                                    // the next pair's row (PF)
  bool have_next = false;

  Kahan<T> r2, di2, do2, o2;
  for (int g = blockIdx.x; g < a.npairs; g += gridDim.x) {
    const RowOf ro = row_of(g);
    const int rA = ro.rA, kz = ro.kz, ky = ro.ky;
    const bool self = ro.self, active = ro.active;
    const long long rowoff = ro.off;
    if (active) {
      T2 x[E];
      if (PF && have_next) {
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = xn[PF ? e : 0];
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const long long off = rowoff + lane + 32 * e;
          x[e] = in_bounds(off, a.V, a.err) ? T2{src_re[off], src_im[off]} : T2{T(0), T(0)};
        }
      }
      if constexpr (F16) {
        fft512_warp<false>(x, lane, wrow, tw16);
#pragma unroll
        for (int q = 0; q < 16; ++q) wrow[sx512(kap + 16 * q + 256 * hh)] = x[q];
      } else {
        __syncwarp();
        fft_column_acc<N, E, false, 0, true>(x, lane, acc, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) acc.put(lane + 32 * e, x[e]);
      }
    }
    if constexpr (PF) {
      have_next = false;
      if (g + (int)gridDim.x < a.npairs) {
        const RowOf nx = row_of(g + gridDim.x);
        if (nx.active) {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const long long off = nx.off + lane + 32 * e;
            xn[e] = in_bounds(off, a.V, a.err) ? T2{src_re[off], src_im[off]} : T2{T(0), T(0)};
          }
          have_next = true;
        }
      }
    }
    __syncthreads();
    const T xi_y = xiy[ky], xi_z = xiz[kz];
    PlainSum<T> pr2, pdi2, pdo2, po2;
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
        potential_pair<T>(av, bv, xix[kx], xi_y, xi_z, inv_v, yk, ym);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          av[c] = yk[c];
          bv[c] = ym[c];
        }
      } else {
        project_pair<T>(av, bv, xix[kx], xi_y, xi_z, rA == 0 && kx == 0, zm,
                        a.nyq_zero != 0, a.compat != 0, inv_v, selfmode ? T(1) : T(2), pr2,
                        pdi2, pdo2, po2);
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
    if constexpr (!POT) {
      r2.add(pr2.s);
      di2.add(pdi2.s);
      do2.add(pdo2.s);
      o2.add(po2.s);
    }
    __syncthreads();
    if (active && !(POT && comp == 2)) {                  // warp-uniform
      T* dre = POT ? ydst + (2LL * comp) * a.V + rowoff : fdata + (2LL * comp) * a.V + rowoff;
      T* dim = dre + a.V;
      T2 x[E];
      if constexpr (F16) {
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = wrow[sx512(lane + 32 * e)];
        fft512_warp<true>(x, lane, wrow, tw16);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int pos = kap + 16 * q + 256 * hh;
          if (!in_bounds(rowoff + pos, a.V, a.err)) continue;
          dre[pos] = x[q].x;
          dim[pos] = x[q].y;
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = acc.get(lane + 32 * e);
        __syncwarp();
        fft_column_acc<N, E, true, 0, true>(x, lane, acc, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (!in_bounds(rowoff + lane + 32 * e, a.V, a.err)) continue;
          dre[lane + 32 * e] = x[e].x;
          dim[lane + 32 * e] = x[e].y;
        }
      }
      __syncwarp();                                       // the row is free for the next pair
    }
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


// ---- fused x pass, one warp per component and row pair, both rows as packed pairs ---------------
//
// 512-point FP32 rows.  A block of three warps holds one row pair; warp c holds rows (ky, kz) and
// (-ky, -kz) of complex field c together, point p of both rows as one CPair (fft512_pair), so each
// transform instruction serves both rows.  The rows come from global memory straight into
// registers and leave from registers; the warp's 8 KB row buffer carries the transform exchange
// and then the spectrum of both rows ({Re A, Re B, Im A, Im B} per mode, sp512 order).  Between
// the two block barriers each thread takes modes kx and 512 - kx of all three fields: both mode
// pairs (kx, -kx) and (512 - kx, kx - 512) of the row pair from six 16-byte loads.  A self-mirror
// row pair (one row) is loaded into both halves and only its first half is stored.
//
// STAGED: each warp copies its two rows of the next row pair into a staging area of shared memory
// with cp.async as soon as it has read the current ones, so the loads of the next pair are in
// flight during this pair's transforms and projection (the twiddle table is then kept as {c, s}
// to stay at four blocks per SM).
template <bool STAGED = false> struct XpCfg {
  static constexpr int N = 512, THREADS = 96;
  static constexpr size_t SPEC_BYTES = 3 * sizeof(float4) * N;        // three warps' rows
  static constexpr size_t TW_BYTES = (STAGED ? sizeof(float2) : sizeof(float4)) * 512;
  static constexpr size_t STAGE_BYTES = STAGED ? 3 * 4 * sizeof(float) * N : 0;  // 4 planes a warp
  static constexpr size_t SMEM = SPEC_BYTES + TW_BYTES + sizeof(float) * N + STAGE_BYTES;
};

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)),
               "l"(reinterpret_cast<unsigned long long>(gsrc))
               : "memory");
}

// POT: the potential x pass of eq_project_hodge instead (reads the stress spectrum and does not
// write it; forms y's spectra per mode pair with potential_pair in the rows of fields 0 and 1,
// y0 + i y1 and y2 + i 0, rows A and B as pairs; warps 0 and 1 store their inverse transforms
// into the 4-plane y buffer; no norm partials).
template <int MINB, bool STAGED = false, bool POT = false>
__global__ void __launch_bounds__(XpCfg<STAGED>::THREADS, MINB)
k_xproj_pair(const XTmaArgs a) {
  using C = XpCfg<STAGED>;
  constexpr int N = C::N;
  using TWE = typename std::conditional<STAGED, float2, float4>::type;
  extern __shared__ __align__(16) unsigned char smem_xp[];
  float4* spec = reinterpret_cast<float4*>(smem_xp);     // [warp][512]
  TWE* tw4 = reinterpret_cast<TWE*>(spec + 3 * N);       // W512^(l k1): {c, c, s, s} or {c, s}
  float* xix = reinterpret_cast<float*>(tw4 + 512);
  float* stage = xix + N;                                // STAGED: [warp][re A, im A, re B, im B][N]
  __shared__ double red[32 * 4];

  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  {
    constexpr int TWS = staged_size(N);
    const float2* src = reinterpret_cast<const float2*>(reinterpret_cast<const float*>(a.tws) + 2 * TWS);
    for (int i = tid; i < 512; i += blockDim.x) {
      const float2 t = src[i];
      if constexpr (STAGED) tw4[i] = t;
      else tw4[i] = make_float4(t.x, t.x, t.y, t.y);
    }
    for (int i = tid; i < N; i += blockDim.x) xix[i] = reinterpret_cast<const float*>(a.xi_x)[i];
  }
  __syncthreads();
  const float* xiy = reinterpret_cast<const float*>(a.xi_y);
  const float* xiz = reinterpret_cast<const float*>(a.xi_z);
  const int field = blockIdx.y;
  float* fdata = reinterpret_cast<float*>(a.data) + field * a.field_stride;
  float zmv[6];
  const float* zm = zero_mode_values(a.mean ? a.mean + field * 6 : nullptr, 1.0 / a.inv_v, zmv)
                        ? zmv : nullptr;
  float4* wrow = spec + w * N;
  const float inv_v = float(a.inv_v);
  const int kap = lane >> 1, hh = lane & 1;
  float* pre = fdata + (2LL * w) * a.V;                  // this warp's field: planes 2 w, 2 w + 1
  float* pim = pre + a.V;
  float* wst = stage + w * 4 * N;                        // STAGED: this warp's staging planes
  // STAGED: this warp's rows of row pair g into the staging planes (16-byte copies)
  auto stage_rows = [&](int g) {
    const int rA = a.pairs[g];
    const int kz = rA / a.ny, ky = rA - kz * a.ny;
    const int rB = (kz == 0 ? 0 : a.nz - kz) * a.ny + (ky == 0 ? 0 : a.ny - ky);
    const long long o[2] = {(long long)rA * N, (long long)rB * N};
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int chunk = lane + 32 * i;                   // 512 chunks of 4 floats: plane, offset
      const int pl = chunk >> 7, off = (chunk & 127) * 4;
      const float* src = (pl & 1 ? pim : pre) + o[pl >> 1] + off;
      if (in_bounds(o[pl >> 1] + off + 3, a.V, a.err)) cp_async16(wst + pl * N + off, src);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (STAGED && (int)blockIdx.x < a.npairs) stage_rows(blockIdx.x);

  Kahan<float> r2, di2, do2, o2;
  for (int g = blockIdx.x; g < a.npairs; g += gridDim.x) {
    const int rA = a.pairs[g];
    const int kz = rA / a.ny, ky = rA - kz * a.ny;
    const int rB = (kz == 0 ? 0 : a.nz - kz) * a.ny + (ky == 0 ? 0 : a.ny - ky);
    const bool self = rA == rB;
    const long long oA = (long long)rA * N, oB = (long long)rB * N;
    {
      CPair v[16];
      if constexpr (STAGED) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int p = lane + 32 * e;
          v[e] = CPair{make_float2(wst[p], wst[2 * N + p]), make_float2(wst[N + p], wst[3 * N + p])};
        }
        __syncwarp();                                    // staging read: refill with the next pair
        if (g + (int)gridDim.x < a.npairs) stage_rows(g + gridDim.x);
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int p = lane + 32 * e;
          const bool okA = in_bounds(oA + p, a.V, a.err), okB = in_bounds(oB + p, a.V, a.err);
          const float ra = okA ? pre[oA + p] : 0.f, ia = okA ? pim[oA + p] : 0.f;
          const float rb = self || !okB ? ra : pre[oB + p], ib = self || !okB ? ia : pim[oB + p];
          v[e] = CPair{make_float2(ra, rb), make_float2(ia, ib)};
        }
      }
      fft512_pair<false>(v, lane, wrow, tw4);
#pragma unroll
      for (int q = 0; q < 16; ++q)
        wrow[sp512(kap + 16 * q + 256 * hh)] = make_float4(v[q].r.x, v[q].r.y, v[q].i.x, v[q].i.y);
    }
    __syncthreads();
    const float xi_y = xiy[ky], xi_z = xiz[kz];
    PlainSum<float> pr2, pdi2, pdo2, po2;
    for (int kx = tid; kx <= N / 2; kx += blockDim.x) {
      const int kxm = kx == 0 ? 0 : N - kx;
      const int j1 = sp512(kx), j2 = sp512(kxm);
      float4 e1[3], e2[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        e1[c] = spec[c * N + j1];
        e2[c] = spec[c * N + j2];
      }
      // mode pair 1: A(kx) with B(-kx) = B(kxm)
      float2 av[3], bv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        av[c] = make_float2(e1[c].x, e1[c].z);
        bv[c] = make_float2(self ? e2[c].x : e2[c].y, self ? e2[c].z : e2[c].w);
      }
      const bool same = kx == kxm;                       // kx = 0 or N / 2
      if constexpr (POT) {
        // y replaces the spectra of fields 0 and 1, laid out as the projection's outputs below
        float2 yk[2], ym[2];
        potential_pair<float>(av, bv, xix[kx], xi_y, xi_z, inv_v, yk, ym);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          av[c] = yk[c];
          bv[c] = ym[c];
        }
      } else {
        project_pair<float>(av, bv, xix[kx], xi_y, xi_z, rA == 0 && kx == 0, zm, a.nyq_zero != 0,
                            a.compat != 0, inv_v, (self && same) ? 1.f : 2.f, pr2, pdi2, pdo2, po2);
      }
      if (self) {
        // one row: the pair's outputs are that row at kx and at kxm (copied into both halves)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          e1[c] = make_float4(av[c].x, av[c].x, av[c].y, av[c].y);
          if (!same) e2[c] = make_float4(bv[c].x, bv[c].x, bv[c].y, bv[c].y);
        }
      } else if (same) {
#pragma unroll
        for (int c = 0; c < 3; ++c) e1[c] = make_float4(av[c].x, bv[c].x, av[c].y, bv[c].y);
      } else {
        // mode pair 2: A(kxm) with B(-kxm) = B(kx)
        float2 av2[3], bv2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          av2[c] = make_float2(e2[c].x, e2[c].z);
          bv2[c] = make_float2(e1[c].y, e1[c].w);
        }
        if constexpr (POT) {
          float2 yk[2], ym[2];
          potential_pair<float>(av2, bv2, xix[kxm], xi_y, xi_z, inv_v, yk, ym);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            av2[c] = yk[c];
            bv2[c] = ym[c];
          }
        } else {
          project_pair<float>(av2, bv2, xix[kxm], xi_y, xi_z, false, zm, a.nyq_zero != 0,
                              a.compat != 0, inv_v, 2.f, pr2, pdi2, pdo2, po2);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          e1[c] = make_float4(av[c].x, bv2[c].x, av[c].y, bv2[c].y);
          e2[c] = make_float4(av2[c].x, bv[c].x, av2[c].y, bv[c].y);
        }
      }
#pragma unroll
      for (int c = 0; c < (POT ? 2 : 3); ++c) {
        spec[c * N + j1] = e1[c];
        if (!same) spec[c * N + j2] = e2[c];
      }
    }
    r2.add(pr2.s);
    di2.add(pdi2.s);
    do2.add(pdo2.s);
    o2.add(po2.s);
    __syncthreads();
    if (!(POT && w == 2)) {                              // warp-uniform: no y row for warp 2
      float* dre = POT ? reinterpret_cast<float*>(a.ydata) + field * a.yfield_stride + (2LL * w) * a.V
                       : pre;
      float* dim = dre + a.V;
      CPair v[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const float4 t = wrow[sp512(lane + 32 * e)];
        v[e] = CPair{make_float2(t.x, t.y), make_float2(t.z, t.w)};
      }
      fft512_pair<true>(v, lane, wrow, tw4);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int p = kap + 16 * q + 256 * hh;
        if (!in_bounds(oA + p, a.V, a.err) || !in_bounds(oB + p, a.V, a.err)) continue;
        dre[oA + p] = v[q].r.x;
        dim[oA + p] = v[q].i.x;
        if (!self) {
          dre[oB + p] = v[q].r.y;
          dim[oB + p] = v[q].i.y;
        }
      }
      __syncwarp();                                      // the row buffer is free for the next pair
    }
  }
  if constexpr (!POT) {
    double v4[4] = {r2.value(), di2.value(), do2.value(), o2.value()};
    block_sum<4>(v4, red);
    if (tid == 0) {
      double* q = a.partials + ((long long)field * gridDim.x + blockIdx.x) * 4;
      q[0] = v4[0]; q[1] = v4[1]; q[2] = v4[2]; q[3] = v4[3];
    }
  }
}

}  // namespace eqk
