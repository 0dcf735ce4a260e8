// Precision form of the radix-16 Stockham pass: the 16-point DFTs of a pass are
// evaluated on the tensor cores as a real matrix product
//
//     [Re y | Im y] (16 x 32) = [Re v | Im v] (16 x 32) . F (32 x 32),
//     F = [[ C, -S ], [ S, C ]] with C_kn = cos(2 pi k n/16), S_kn = sin(2 pi k n/16),
//
// for tiles of 16 vectors (one warp, mma.sync m16n8k16, FP32 accumulation).
// FP16X2: operands split into a high and a low fp16 part (x = hi + lo, 22
// significand bits), product hi.hi + hi.lo + lo.hi (3 MMAs).
// BF16X3: operands split into three bf16 parts (x = x0 + x1 + x2, 24 bits),
// product x0.y0 + x0.y1 + x1.y0 + x0.y2 + x1.y1 + x2.y0 (6 MMAs): every term of
// order below 2^-24 relative is dropped, so both forms carry FP32 accuracy.
// Each tile is scaled by a power of two so that its largest input lies in
// [2^14, 2^15) before the split (fp16 range), and unscaled after the product.
// Stage twiddles are applied in FP32 before the split, from the FP64-derived
// table.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fused.cuh"

namespace adfft {

enum PrecisionMode : int { kPrecNative = 0, kPrecFp16x2 = 1, kPrecBf16x3 = 2 };

template <int PREC>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if constexpr (PREC == kPrecFp16x2) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}
template <int PREC>
__device__ __forceinline__ float2 unpack2(uint32_t v) {
  if constexpr (PREC == kPrecFp16x2) {
    return __half22float2(*reinterpret_cast<__half2*>(&v));
  } else {
    return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&v));
  }
}
// hi = round(x), lo = round(x - hi), two values per 32-bit register.
template <int PREC>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  hi = pack2<PREC>(a, b);
  const float2 h = unpack2<PREC>(hi);
  lo = pack2<PREC>(a - h.x, b - h.y);
}
// x0 = round(x), x1 = round(x - x0), x2 = round(x - x0 - x1) (each subtraction exact in FP32).
template <int PREC>
__device__ __forceinline__ void split3(float a, float b, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
  p0 = pack2<PREC>(a, b);
  const float2 h0 = unpack2<PREC>(p0);
  const float ra = a - h0.x, rb = b - h0.y;
  p1 = pack2<PREC>(ra, rb);
  const float2 h1 = unpack2<PREC>(p1);
  p2 = pack2<PREC>(ra - h1.x, rb - h1.y);
}
// Split of an operand pair into the parts the form multiplies: [0] high, [1] low (FP16X2) or
// [0] x0, [1] x1, [2] x2 (BF16X3).
template <int PREC> struct Parts { static constexpr int n = (PREC == 2) ? 3 : 2; };
template <int PREC>
__device__ __forceinline__ void split_parts(float a, float b, uint32_t (&p)[Parts<PREC>::n]) {
  if constexpr (Parts<PREC>::n == 3) split3<PREC>(a, b, p[0], p[1], p[2]);
  else split2<PREC>(a, b, p[0], p[1]);
}

template <int PREC>
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
  if constexpr (PREC == kPrecFp16x2) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
}

// F[k][n] of the real 32 x 32 form above (k: input index, n: output index).
__device__ __forceinline__ float dft16_real_entry(int k, int n) {
  const int kk = k & 15, nn = n & 15;
  const int t = (kk * nn) & 15;                     // angle 2 pi t / 16 = 2 pi (2t) / 32
  const int u = (2 * t) & 31;
  // cos and sin of 2 pi u / 32 from the octant table
  float c, s;
  {
    const int q = u >> 3, r = u & 7;
    const float c0 = (float)kCos32(r), s0 = (float)kSin32(r);
    // rotate (c0, s0) by q quarter turns
    c = (q == 0) ? c0 : (q == 1) ? -s0 : (q == 2) ? -c0 : s0;
    s = (q == 0) ? s0 : (q == 1) ? c0 : (q == 2) ? -s0 : -c0;
  }
  const bool kre = k < 16, nre = n < 16;
  if (kre && nre) return c;        // Re v -> Re y :  cos
  if (!kre && nre) return s;       // Im v -> Re y :  sin
  if (kre && !nre) return -s;      // Re v -> Im y : -sin
  return c;                        // Im v -> Im y :  cos
}

// B fragments of F for this lane, split into parts: [part][kstep 2][ntile 4][2 regs].
template <int PREC>
__device__ __forceinline__ void load_dft16_fragments(uint32_t (&bp)[Parts<PREC>::n][2][4][2]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  constexpr int NP = Parts<PREC>::n;
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int n = 8 * nt + g;
      const int k0 = 16 * ks + 2 * t;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        uint32_t q[NP];
        split_parts<PREC>(dft16_real_entry(k0 + 8 * r, n), dft16_real_entry(k0 + 8 * r + 1, n), q);
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) bp[pp][ks][nt][r] = q[pp];
      }
    }
  }
}

// One in-place radix-16 Stockham pass with the DFTs on the tensor cores.
// Same data movement as stockham_pass<16>: row (rl, j) reads j + i*Np/16 and
// writes (j / Ns)*16 Ns + (j mod Ns) + i*Ns.  A warp owns tiles of 16 rows;
// lane (g, t) holds the elements i in {2t, 2t+1, 2t+8, 2t+9} of rows g and g+8.
// TPT: tiles per warp held in registers across the barrier.
template <int PREC, int TPT, typename V>
__device__ void stockham_pass_tc(const FusedArgs& a, V* buf, const TwTable<V>& tab, int Ns,
                                                 int logNs) {
  static_assert(sizeof(V) == 8, "tensor-core passes take complex64 data");
  const int log_items = a.logNp - 4;
  const int items_res = 1 << log_items;
  const int items = a.RPC * items_res;
  const int ntiles = (items + 15) >> 4;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const unsigned tw_step = (unsigned)a.Mt / ((unsigned)Ns << 4);
  const int in_step = items_res + (items_res >> 4);       // pad16(j + i S) = pad16(j) + i (S + S/16)
  constexpr int NPART = Parts<PREC>::n;
  uint32_t bp[NPART][2][4][2];
  load_dft16_fragments<PREC>(bp);
  // element slot e -> DFT index i
  const int idx4[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
  float2 res[TPT][2][4];                                  // [tile][row g / g+8][slot]
#pragma unroll
  for (int tt = 0; tt < TPT; ++tt) {
    const int tile = warp + tt * nwarps;
    float2 x[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = tile * 16 + g + 8 * h;
      const bool ok = tile < ntiles && row < items;
      const int rl = row >> log_items, j = row & (items_res - 1);
      const float2* src = reinterpret_cast<const float2*>(buf) + rl * a.region + pad16(j);
      // twiddles W_{16 Ns}^{k i}, k = j mod Ns
      const unsigned k = (unsigned)(j & (Ns - 1));
      const float2 w1 = tab(k * tw_step);
      const float2 wa = tab(k * (unsigned)idx4[0] * tw_step);
      const float2 wb = tab(k * (unsigned)idx4[2] * tw_step);
      const float2 w[4] = {wa, cmul(wa, w1), wb, cmul(wb, w1)};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        // pad16(j + i S) = pad16(j) + i (S + S/16) needs S a multiple of 16; shorter
        // transforms index every element through pad16
        float2 v = make_float2(0.f, 0.f);
        if (ok)
          v = (items_res >= 16) ? src[idx4[e] * in_step]
                                : reinterpret_cast<const float2*>(buf)[rl * a.region + pad16(j + idx4[e] * items_res)];
        x[h][e] = cmul(v, w[e]);
      }
    }
    // power-of-two tile scale: the tile's largest magnitude goes to [2^14, 2^15)
    float m = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int e = 0; e < 4; ++e) m = fmaxf(m, fmaxf(fabsf(x[h][e].x), fabsf(x[h][e].y)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int ex = 0;
    if (m > 0.f) ex = ((__float_as_int(m) >> 23) & 0xff) - 127;   // floor(log2 m) for normal m
    ex = max(-100, min(100, ex));
    const float up = __int_as_float((127 + 14 - ex) << 23);     // 2^(14 - ex)
    const float down = __int_as_float((127 - 14 + ex) << 23);   // 2^(ex - 14)
    // A fragments: kstep 0 = real parts, kstep 1 = imaginary parts
    uint32_t ap[NPART][2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      // a0:(g, 2t..2t+1) a1:(g+8, 2t..) a2:(g, 2t+8..) a3:(g+8, 2t+8..)
      const float p00 = (ks ? x[0][0].y : x[0][0].x) * up, p01 = (ks ? x[0][1].y : x[0][1].x) * up;
      const float p10 = (ks ? x[1][0].y : x[1][0].x) * up, p11 = (ks ? x[1][1].y : x[1][1].x) * up;
      const float p02 = (ks ? x[0][2].y : x[0][2].x) * up, p03 = (ks ? x[0][3].y : x[0][3].x) * up;
      const float p12 = (ks ? x[1][2].y : x[1][2].x) * up, p13 = (ks ? x[1][3].y : x[1][3].x) * up;
      const float pv[4][2] = {{p00, p01}, {p10, p11}, {p02, p03}, {p12, p13}};
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        uint32_t q[NPART];
        split_parts<PREC>(pv[f][0], pv[f][1], q);
#pragma unroll
        for (int pp = 0; pp < NPART; ++pp) ap[pp][ks][f] = q[pp];
      }
    }
    float d[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
      for (int q = 0; q < 4; ++q) d[nt][q] = 0.f;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        // smallest terms first: the FP32 accumulator adds them before the dominant product
        if constexpr (NPART == 3) {
          mma16816<PREC>(d[nt], ap[2][ks], bp[0][ks][nt]);
          mma16816<PREC>(d[nt], ap[1][ks], bp[1][ks][nt]);
          mma16816<PREC>(d[nt], ap[0][ks], bp[2][ks][nt]);
        }
        mma16816<PREC>(d[nt], ap[1][ks], bp[0][ks][nt]);
        mma16816<PREC>(d[nt], ap[0][ks], bp[1][ks][nt]);
        mma16816<PREC>(d[nt], ap[0][ks], bp[0][ks][nt]);
      }
    }
    // D fragment (row g: d[.][0..1], row g+8: d[.][2..3]) at columns 8 nt + 2t + {0,1}:
    // ntile 0 -> Re y[2t..2t+1], 1 -> Re y[2t+8..], 2 -> Im y[2t..], 3 -> Im y[2t+8..]
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      res[tt][h][0] = make_float2(d[0][2 * h] * down, d[2][2 * h] * down);
      res[tt][h][1] = make_float2(d[0][2 * h + 1] * down, d[2][2 * h + 1] * down);
      res[tt][h][2] = make_float2(d[1][2 * h] * down, d[3][2 * h] * down);
      res[tt][h][3] = make_float2(d[1][2 * h + 1] * down, d[3][2 * h + 1] * down);
    }
  }
  __syncthreads();
  const int out_step = Ns + (Ns >> 4);
#pragma unroll
  for (int tt = 0; tt < TPT; ++tt) {
    const int tile = warp + tt * nwarps;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = tile * 16 + g + 8 * h;
      if (tile < ntiles && row < items) {
        const int rl = row >> log_items, j = row & (items_res - 1);
        const int k = j & (Ns - 1);
        const int base = ((j >> logNs) << (logNs + 4)) + k;
        float2* dst = reinterpret_cast<float2*>(buf) + rl * a.region;
        if (Ns >= 16) {
          float2* p0 = dst + pad16(base);
#pragma unroll
          for (int e = 0; e < 4; ++e) p0[idx4[e] * out_step] = res[tt][h][e];
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) dst[pad16(base + idx4[e] * Ns)] = res[tt][h][e];
        }
      }
    }
  }
  __syncthreads();
}

}  // namespace adfft
