// eq_fft_pair.cuh - 512-point FP32 transforms of two rows at once, the rows' values held as packed
// pairs (device code).
//
// A CPair holds the same point of two rows: r = {Re row 0, Re row 1}, i = {Im row 0, Im row 1}.
// Every add, subtract and multiply of a transform then acts on both rows with one packed two-lane
// FP32 instruction (add/sub/mul/fma .f32x2, rounded like the scalar operations), so a warp
// transforms two rows for the instructions one row takes in eq_fft.cuh.  The factorisation is
// that of fft512_warp: 512 = 16 x 32, lane l holding points l + 32 e (e < 16); a 16-point DFT in
// registers, the twiddle W512^(l k1), one exchange through the warp's row buffer (16-byte
// entries), a 16-point DFT over the even / odd halves of the 32-point DFTs and a radix-2 combine
// of lanes 2 kap and 2 kap + 1 by shuffle.  Lane 2 kap + h ends with output kap + 16 q + 256 h of
// both rows in slot q.
#pragma once
#include <cuda_runtime.h>

#include "eq_fft.cuh"

namespace eqk {

struct CPair {
  float2 r, i;
};

__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 bcast(float s) { return make_float2(s, s); }

__device__ __forceinline__ CPair padd(CPair a, CPair b) { return {__fadd2_rn(a.r, b.r), __fadd2_rn(a.i, b.i)}; }
__device__ __forceinline__ CPair psub(CPair a, CPair b) { return {fsub2(a.r, b.r), fsub2(a.i, b.i)}; }
// a + W4 b and a - W4 b with W4 = -i (forward) or +i (inverse), no separate negation
template <bool INV> __device__ __forceinline__ CPair padd_w4(CPair a, CPair b) {
  return INV ? CPair{fsub2(a.r, b.i), __fadd2_rn(a.i, b.r)} : CPair{__fadd2_rn(a.r, b.i), fsub2(a.i, b.r)};
}
template <bool INV> __device__ __forceinline__ CPair psub_w4(CPair a, CPair b) {
  return INV ? CPair{__fadd2_rn(a.r, b.i), fsub2(a.i, b.r)} : CPair{fsub2(a.r, b.i), __fadd2_rn(a.i, b.r)};
}
// v * (c + i s) for real constants: Re = r c - i s, Im = r s + i c
__device__ __forceinline__ CPair pmul_cs(CPair v, float c, float s) {
  return {__ffma2_rn(v.i, bcast(-s), __fmul2_rn(v.r, bcast(c))),
          __ffma2_rn(v.r, bcast(s), __fmul2_rn(v.i, bcast(c)))};
}
// v * W32^Q (forward: exp(-2 pi i Q / 32); INV: the conjugate), Q in 0..15
template <int Q, bool INV> __device__ __forceinline__ CPair pmul_w32(CPair v) {
  if constexpr (Q == 0) {
    return v;
  } else if constexpr (Q == 8) {                       // -i (forward), +i (inverse)
    return INV ? CPair{__fmul2_rn(v.i, bcast(-1.f)), v.r} : CPair{v.i, __fmul2_rn(v.r, bcast(-1.f))};
  } else if constexpr (Q == 4 || Q == 12) {            // h (1 -+ i) and h (-1 -+ i)
    constexpr float h = float(cos_pi16(4));
    // forward Q = 4: h (r + i, i - r); Q = 12: h (i - r, -(r + i)); inverse conjugates
    const float2 s = __fadd2_rn(v.r, v.i), d = fsub2(v.i, v.r);
    if constexpr (Q == 4) {
      return INV ? CPair{__fmul2_rn(d, bcast(-h)), __fmul2_rn(s, bcast(h))}
                 : CPair{__fmul2_rn(s, bcast(h)), __fmul2_rn(d, bcast(h))};
    } else {
      return INV ? CPair{__fmul2_rn(s, bcast(-h)), __fmul2_rn(d, bcast(-h))}
                 : CPair{__fmul2_rn(d, bcast(h)), __fmul2_rn(s, bcast(-h))};
    }
  } else {
    constexpr float c = float(cos_pi16(Q));
    constexpr float s = INV ? float(sin_pi16(Q)) : float(-sin_pi16(Q));
    return pmul_cs(v, c, s);
  }
}
template <bool INV> __device__ __forceinline__ CPair pmul_w32_rt(int q, CPair v) {
  switch (q) {
    case 1: return pmul_w32<1, INV>(v);
    case 2: return pmul_w32<2, INV>(v);
    case 3: return pmul_w32<3, INV>(v);
    case 4: return pmul_w32<4, INV>(v);
    case 5: return pmul_w32<5, INV>(v);
    case 6: return pmul_w32<6, INV>(v);
    case 7: return pmul_w32<7, INV>(v);
    case 8: return pmul_w32<8, INV>(v);
    case 9: return pmul_w32<9, INV>(v);
    case 10: return pmul_w32<10, INV>(v);
    case 11: return pmul_w32<11, INV>(v);
    case 12: return pmul_w32<12, INV>(v);
    case 13: return pmul_w32<13, INV>(v);
    case 14: return pmul_w32<14, INV>(v);
    case 15: return pmul_w32<15, INV>(v);
    default: return v;
  }
}

// X_r = sum_m v_m W4^{r m}
template <bool INV> __device__ __forceinline__ void pdft4(CPair* v) {
  const CPair s02 = padd(v[0], v[2]), d02 = psub(v[0], v[2]);
  const CPair s13 = padd(v[1], v[3]), d13 = psub(v[1], v[3]);
  v[0] = padd(s02, s13);
  v[2] = psub(s02, s13);
  v[1] = padd_w4<INV>(d02, d13);
  v[3] = psub_w4<INV>(d02, d13);
}

// radix 8: two radix-4 transforms of the sums / W8-twiddled differences of v_m and v_{m+4}
template <bool INV> __device__ __forceinline__ void pdft8(CPair* v) {
  CPair a[4], b[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    a[m] = padd(v[m], v[m + 4]);
    b[m] = psub(v[m], v[m + 4]);
  }
  b[1] = pmul_w32<4, INV>(b[1]);
  b[2] = pmul_w32<8, INV>(b[2]);
  b[3] = pmul_w32<12, INV>(b[3]);
  pdft4<INV>(a);
  pdft4<INV>(b);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[2 * q] = a[q];
    v[2 * q + 1] = b[q];
  }
}

// radix 16: two radix-8 transforms of the sums / W16-twiddled differences of v_m and v_{m+8};
// outputs in natural order
template <bool INV> __device__ __forceinline__ void pdft16(CPair* v) {
  CPair a[8], b[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    a[m] = padd(v[m], v[m + 8]);
    b[m] = psub(v[m], v[m + 8]);
  }
  b[1] = pmul_w32<2, INV>(b[1]);
  b[2] = pmul_w32<4, INV>(b[2]);
  b[3] = pmul_w32<6, INV>(b[3]);
  b[4] = pmul_w32<8, INV>(b[4]);
  b[5] = pmul_w32<10, INV>(b[5]);
  b[6] = pmul_w32<12, INV>(b[6]);
  b[7] = pmul_w32<14, INV>(b[7]);
  pdft8<INV>(a);
  pdft8<INV>(b);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    v[2 * q] = a[q];
    v[2 * q + 1] = b[q];
  }
}

// 512-point transform of the two rows held by one warp (see the file comment).  tw: W512^(l k1)
// as [k1][l] entries {cos, cos, sin, sin} or {cos, sin} (forward factors; the inverse conjugates
// them).  buf:
// the warp's 512 16-byte entries; no lane may still read it on entry, and it is free on return.
// twiddle pair registers {c, c} and {s, s} from a table of {c, c, s, s} or of {c, s} entries
__device__ __forceinline__ void tw_pair(const float4* tw, int i, float2& C, float2& S) {
  const float4 w = tw[i];
  C = make_float2(w.x, w.y);
  S = make_float2(w.z, w.w);
}
__device__ __forceinline__ void tw_pair(const float2* tw, int i, float2& C, float2& S) {
  const float2 w = tw[i];
  C = bcast(w.x);
  S = bcast(w.y);
}

template <bool INV, typename TWE>
__device__ __forceinline__ void fft512_pair(CPair (&v)[16], int lane, float4* buf,
                                            const TWE* __restrict__ tw) {
  pdft16<INV>(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) {
    float2 C, S;
    tw_pair(tw, k1 * 32 + lane, C, S);
    const CPair x = v[k1];
    if (INV) {   // (r + i i)(c - i s) = (r c + i s) + i (i c - r s)
      v[k1] = CPair{__ffma2_rn(x.i, S, __fmul2_rn(x.r, C)), fsub2(__fmul2_rn(x.i, C), __fmul2_rn(x.r, S))};
    } else {     // (r + i i)(c + i s) = (r c - i s) + i (r s + i c)
      v[k1] = CPair{fsub2(__fmul2_rn(x.r, C), __fmul2_rn(x.i, S)), __ffma2_rn(x.r, S, __fmul2_rn(x.i, C))};
    }
  }
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1)
    buf[k1 * 32 + (lane ^ (2 * k1))] = make_float4(v[k1].r.x, v[k1].r.y, v[k1].i.x, v[k1].i.y);
  __syncwarp();
  const int kap = lane >> 1, h = lane & 1;
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const float4 e = buf[kap * 32 + h + 2 * (m ^ kap)];
    v[m] = CPair{make_float2(e.x, e.y), make_float2(e.z, e.w)};
  }
  __syncwarp();
  pdft16<INV>(v);
  const float2 sg = bcast(h ? -1.f : 1.f);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    // lane h = 1 sends W32^q Z_1[q], lane h = 0 sends Z_0[q]; each adds +- its own value
    const CPair t = pmul_w32_rt<INV>(q, v[q]);
    const CPair send = h ? t : v[q];
    CPair recv;
    recv.r.x = __shfl_xor_sync(0xffffffffu, send.r.x, 1);
    recv.r.y = __shfl_xor_sync(0xffffffffu, send.r.y, 1);
    recv.i.x = __shfl_xor_sync(0xffffffffu, send.i.x, 1);
    recv.i.y = __shfl_xor_sync(0xffffffffu, send.i.y, 1);
    v[q] = CPair{__ffma2_rn(sg, send.r, recv.r), __ffma2_rn(sg, send.i, recv.i)};
  }
}

// Position of spectrum entry k (k < 512) in a row of 16-byte entries: bit 8 of k flipped into
// bit 2, so that the transform's output stores (lanes 2 kap + h write kap + 16 q + 256 h), its
// inverse loads (l + 32 e) and runs of consecutive modes hit 8 distinct 16-byte slots in every
// quarter-warp.
__host__ __device__ __forceinline__ int sp512(int k) { return k ^ (((k >> 8) & 1) << 2); }

}  // namespace eqk
