// eq_pfft.cuh - Stockham transforms of two sequences at once, the sequences' values held as
// packed pairs (CPair, eq_fft_pair.cuh) (device code).
#pragma once
#include "eq_fft_pair.cuh"

namespace eqk {

// ---- Stockham transforms of two sequences at once ----------------------------------------
//
// The schedule of fft_column_acc (eq_fft.cuh) on CPair values: one transform of length N held by
// the TPC = N / E = 32 lanes of a warp, lane t holding points t + 32 e of both sequences in slot
// e, radix-8 stages (then 4 or 2) with the outputs of each stage exchanged through the warp's
// own buffer of 16-byte entries; after the last stage slot e holds output t + 32 e.

template <int R, bool INV> __device__ __forceinline__ void pdftR(CPair* v) {
  if constexpr (R == 8) {
    pdft8<INV>(v);
  } else if constexpr (R == 4) {
    pdft4<INV>(v);
  } else {
    const CPair a = v[0];
    v[0] = padd(a, v[1]);
    v[1] = psub(a, v[1]);
  }
}

// 16-byte exchange entries, entry i at i ^ ((i >> 3) & 7): the stage outputs of eight
// consecutive lanes (a quarter-warp, one wavefront) and their contiguous reloads fall in eight
// distinct 16-byte slots
struct PairAcc {
  float4* buf;
  __device__ __forceinline__ void put(int i, CPair v) const {
    buf[i ^ ((i >> 3) & 7)] = make_float4(v.r.x, v.r.y, v.i.x, v.i.y);
  }
  __device__ __forceinline__ CPair get(int i) const {
    const float4 e = buf[i ^ ((i >> 3) & 7)];
    return CPair{make_float2(e.x, e.y), make_float2(e.z, e.w)};
  }
};

template <int N, int E, int S, bool INV, typename TW>
__device__ __forceinline__ void pfft_stage(CPair (&x)[E], int t, const TW& tw) {
  constexpr int R = stage_radix(N, S);
  constexpr int NS = stage_span(N, S);
  constexpr int TPC = N / E;
  constexpr int Q = E / R;
  static_assert(Q >= 1 && TPC == 32, "one warp per transform, at least R points a lane");
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    CPair v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[q + r * Q];
    if constexpr (NS > 1) {
      const int k = (t + TPC * q) & (NS - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = tw.template get<N, NS, R>(k, r);
        v[r] = pmul_cs(v[r], w.x, INV ? -w.y : w.y);
      }
    }
    pdftR<R, INV>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) x[q + r * Q] = v[r];
  }
}

// Full transform of both sequences (unnormalised; INV: exp(+2 pi i m x / N)).  No lane may still
// read `acc` on entry; it is free again on return.
template <int N, int E, bool INV, int S = 0, typename TW>
__device__ __forceinline__ void pfft_column(CPair (&x)[E], int t, const PairAcc& acc, const TW& tw) {
  if constexpr (S < num_stages(N)) {
    pfft_stage<N, E, S, INV>(x, t, tw);
    if constexpr (S + 1 < num_stages(N)) {
      constexpr int R = stage_radix(N, S);
      constexpr int Q = E / R;
#pragma unroll
      for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) acc.put(stage_out_pos<N, E, S>(t, q, r), x[q + r * Q]);
      __syncwarp();
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = acc.get(t + 32 * e);
      __syncwarp();
      pfft_column<N, E, INV, S + 1>(x, t, acc, tw);
    }
  }
}

}  // namespace eqk
