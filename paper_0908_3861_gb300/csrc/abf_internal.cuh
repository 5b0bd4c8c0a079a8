// Internal definitions shared by the abf CUDA translation units.
//
// Exact arithmetic: integers modulo 2^(64 L) held as L little-endian uint64
// limbs.  Running sums (Sec. 7 (1)) and the mesh numerator (Eq. (final_eqn))
// are formed in this ring; only the final numerator, whose true size is bounded
// (abf_plan_create checks the bound), is read back as a signed integer.
#pragma once
#include <type_traits>
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/abf.h"

namespace abf {

constexpr int kMaxLimbs = 4;

// Lattice direction vectors of Sec. 7 (theta = 0, pi/4, pi/2, 3pi/4; b_k r_k = v_k).
// v1 = (1,0), v2 = (1,1), v3 = (0,1), v4 = (-1,1).

template <int L>
struct Wide {
  uint64_t w[L];
};

template <int L>
__device__ __forceinline__ void wzero(Wide<L>& a) {
#pragma unroll
  for (int i = 0; i < L; ++i) a.w[i] = 0;
}

// a += b (mod 2^(64L))
template <int L>
__device__ __forceinline__ void wadd(Wide<L>& a, const Wide<L>& b) {
  if constexpr (L == 1) {
    a.w[0] += b.w[0];
  } else {
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
      uint64_t s = a.w[i] + b.w[i];
      uint64_t c1 = s < b.w[i];
      uint64_t t = s + carry;
      uint64_t c2 = t < carry;
      a.w[i] = t;
      carry = c1 | c2;
    }
  }
}

// a -= b (mod 2^(64L))
template <int L>
__device__ __forceinline__ void wsub(Wide<L>& a, const Wide<L>& b) {
  if constexpr (L == 1) {
    a.w[0] -= b.w[0];
  } else {
    uint64_t borrow = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
      uint64_t d = a.w[i] - b.w[i];
      uint64_t b1 = a.w[i] < b.w[i];
      uint64_t t = d - borrow;
      uint64_t b2 = d < borrow;
      a.w[i] = t;
      borrow = b1 | b2;
    }
  }
}

// a += b (mod 2^(64L)) as one add-with-carry chain (the scans: fewer ALU
// operations than the compare-and-carry form, which the mesh schedules better).
template <int L>
__device__ __forceinline__ void waddc(Wide<L>& a, const Wide<L>& b) {
  if constexpr (L == 1) {
    a.w[0] += b.w[0];
  } else if constexpr (L == 2) {
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.w[0]), "+l"(a.w[1]) : "l"(b.w[0]), "l"(b.w[1]));
  } else if constexpr (L == 3) {
    asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
        : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2])
        : "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]));
  } else {
    static_assert(L == 4, "1..4 limbs");
    asm("add.cc.u64 %0, %0, %4;\n\taddc.cc.u64 %1, %1, %5;\n\taddc.cc.u64 %2, %2, %6;\n\taddc.u64 %3, %3, %7;"
        : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2]), "+l"(a.w[3])
        : "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]), "l"(b.w[3]));
  }
}

// a -= b (mod 2^(64L)) as one subtract-with-borrow chain.
template <int L>
__device__ __forceinline__ void wsubc(Wide<L>& a, const Wide<L>& b) {
  if constexpr (L == 1) {
    a.w[0] -= b.w[0];
  } else if constexpr (L == 2) {
    asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;" : "+l"(a.w[0]), "+l"(a.w[1]) : "l"(b.w[0]), "l"(b.w[1]));
  } else if constexpr (L == 3) {
    asm("sub.cc.u64 %0, %0, %3;\n\tsubc.cc.u64 %1, %1, %4;\n\tsubc.u64 %2, %2, %5;"
        : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2])
        : "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]));
  } else {
    static_assert(L == 4, "1..4 limbs");
    asm("sub.cc.u64 %0, %0, %4;\n\tsubc.cc.u64 %1, %1, %5;\n\tsubc.cc.u64 %2, %2, %6;\n\tsubc.u64 %3, %3, %7;"
        : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2]), "+l"(a.w[3])
        : "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]), "l"(b.w[3]));
  }
}

// acc += g * w (mod 2^(64L)), w an unsigned 64-bit factor.
template <int L>
__device__ __forceinline__ void wmac(Wide<L>& acc, const Wide<L>& g, uint64_t w) {
  if constexpr (L == 1) {
    acc.w[0] += g.w[0] * w;
  } else {
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
      uint64_t lo = g.w[i] * w;
      uint64_t s = acc.w[i] + lo;
      uint64_t c1 = s < lo;
      uint64_t t = s + carry;
      uint64_t c2 = t < carry;
      acc.w[i] = t;
      if (i + 1 < L) carry = __umul64hi(g.w[i], w) + c1 + c2;
    }
  }
}

// acc += g * (wlo + 2^64 whi) (mod 2^(64L)): a 128-bit factor.
template <int L>
__device__ __forceinline__ void wmac128(Wide<L>& acc, const Wide<L>& g, uint64_t wlo, uint64_t whi) {
  wmac<L>(acc, g, wlo);
  if constexpr (L > 1) {
    if (whi) {
      Wide<L - 1> a1, g1;
#pragma unroll
      for (int i = 0; i < L - 1; ++i) {
        a1.w[i] = acc.w[i + 1];
        g1.w[i] = g.w[i];
      }
      wmac<L - 1>(a1, g1, whi);
#pragma unroll
      for (int i = 0; i < L - 1; ++i) acc.w[i + 1] = a1.w[i];
    }
  }
}

// acc += g * w (mod 2^128) for a two-limb g and a 64-bit w, as one chain of
// 32-bit multiply-adds with carry (the twelve partial products of a
// 4 x 2 word product that land below bit 128).
__device__ __forceinline__ void wmac2_u64(Wide<2>& acc, const Wide<2>& g, uint64_t w) {
  uint32_t r0 = (uint32_t)acc.w[0], r1 = (uint32_t)(acc.w[0] >> 32);
  uint32_t r2 = (uint32_t)acc.w[1], r3 = (uint32_t)(acc.w[1] >> 32);
  const uint32_t a0 = (uint32_t)g.w[0], a1 = (uint32_t)(g.w[0] >> 32);
  const uint32_t a2 = (uint32_t)g.w[1], a3 = (uint32_t)(g.w[1] >> 32);
  const uint32_t w0 = (uint32_t)w, w1 = (uint32_t)(w >> 32);
  asm("{\n\t"
      "mad.lo.cc.u32  %0, %4, %8, %0;\n\t"
      "madc.hi.cc.u32 %1, %4, %8, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %8, %2;\n\t"
      "madc.hi.u32    %3, %6, %8, %3;\n\t"
      "mad.lo.cc.u32  %1, %5, %8, %1;\n\t"
      "madc.lo.cc.u32 %2, %6, %8, %2;\n\t"
      "madc.lo.u32    %3, %7, %8, %3;\n\t"
      "mad.lo.cc.u32  %1, %4, %9, %1;\n\t"
      "madc.hi.cc.u32 %2, %4, %9, %2;\n\t"
      "madc.hi.u32    %3, %5, %9, %3;\n\t"
      "mad.lo.cc.u32  %2, %5, %9, %2;\n\t"
      "madc.lo.u32    %3, %6, %9, %3;\n\t"
      "}"
      : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3)
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(w0), "r"(w1));
  acc.w[0] = ((uint64_t)r1 << 32) | r0;
  acc.w[1] = ((uint64_t)r3 << 32) | r2;
}

// Carry-chained multiply-accumulates for wider limbs and weights (written by
// gen_mac_chains.py beside this file; the build re-checks their schedule and
// that this file holds exactly what the generator writes).
// acc += g * w (mod 2^192): 3-limb g, 64-bit w; 20 multiply-adds in carry chains.
__device__ __forceinline__ void wmac_w6_b2(Wide<3>& acc, const Wide<3>& g, uint32_t w0, uint32_t w1) {
  uint32_t r[6], a[6];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r[2 * i] = (uint32_t)acc.w[i]; r[2 * i + 1] = (uint32_t)(acc.w[i] >> 32);
    a[2 * i] = (uint32_t)g.w[i]; a[2 * i + 1] = (uint32_t)(g.w[i] >> 32);
  }
  asm("{\n\t"
      "mad.lo.cc.u32   %0, %6, %12, %0;\n\t"
      "madc.hi.cc.u32  %1, %6, %12, %1;\n\t"
      "madc.hi.cc.u32  %2, %7, %12, %2;\n\t"
      "madc.hi.cc.u32  %3, %8, %12, %3;\n\t"
      "madc.hi.cc.u32  %4, %9, %12, %4;\n\t"
      "madc.hi.u32     %5, %10, %12, %5;\n\t"
      "mad.lo.cc.u32   %1, %7, %12, %1;\n\t"
      "madc.lo.cc.u32  %2, %8, %12, %2;\n\t"
      "madc.lo.cc.u32  %3, %9, %12, %3;\n\t"
      "madc.lo.cc.u32  %4, %10, %12, %4;\n\t"
      "madc.lo.u32     %5, %11, %12, %5;\n\t"
      "mad.lo.cc.u32   %1, %6, %13, %1;\n\t"
      "madc.hi.cc.u32  %2, %6, %13, %2;\n\t"
      "madc.hi.cc.u32  %3, %7, %13, %3;\n\t"
      "madc.hi.cc.u32  %4, %8, %13, %4;\n\t"
      "madc.hi.u32     %5, %9, %13, %5;\n\t"
      "mad.lo.cc.u32   %2, %7, %13, %2;\n\t"
      "madc.lo.cc.u32  %3, %8, %13, %3;\n\t"
      "madc.lo.cc.u32  %4, %9, %13, %4;\n\t"
      "madc.lo.u32     %5, %10, %13, %5;\n\t"
      "}"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(w0), "r"(w1));
#pragma unroll
  for (int i = 0; i < 3; ++i) acc.w[i] = ((uint64_t)r[2 * i + 1] << 32) | r[2 * i];
}

// acc += g * w (mod 2^256): 4-limb g, 64-bit w; 28 multiply-adds in carry chains.
__device__ __forceinline__ void wmac_w8_b2(Wide<4>& acc, const Wide<4>& g, uint32_t w0, uint32_t w1) {
  uint32_t r[8], a[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    r[2 * i] = (uint32_t)acc.w[i]; r[2 * i + 1] = (uint32_t)(acc.w[i] >> 32);
    a[2 * i] = (uint32_t)g.w[i]; a[2 * i + 1] = (uint32_t)(g.w[i] >> 32);
  }
  asm("{\n\t"
      "mad.lo.cc.u32   %0, %8, %16, %0;\n\t"
      "madc.hi.cc.u32  %1, %8, %16, %1;\n\t"
      "madc.hi.cc.u32  %2, %9, %16, %2;\n\t"
      "madc.hi.cc.u32  %3, %10, %16, %3;\n\t"
      "madc.hi.cc.u32  %4, %11, %16, %4;\n\t"
      "madc.hi.cc.u32  %5, %12, %16, %5;\n\t"
      "madc.hi.cc.u32  %6, %13, %16, %6;\n\t"
      "madc.hi.u32     %7, %14, %16, %7;\n\t"
      "mad.lo.cc.u32   %1, %9, %16, %1;\n\t"
      "madc.lo.cc.u32  %2, %10, %16, %2;\n\t"
      "madc.lo.cc.u32  %3, %11, %16, %3;\n\t"
      "madc.lo.cc.u32  %4, %12, %16, %4;\n\t"
      "madc.lo.cc.u32  %5, %13, %16, %5;\n\t"
      "madc.lo.cc.u32  %6, %14, %16, %6;\n\t"
      "madc.lo.u32     %7, %15, %16, %7;\n\t"
      "mad.lo.cc.u32   %1, %8, %17, %1;\n\t"
      "madc.hi.cc.u32  %2, %8, %17, %2;\n\t"
      "madc.hi.cc.u32  %3, %9, %17, %3;\n\t"
      "madc.hi.cc.u32  %4, %10, %17, %4;\n\t"
      "madc.hi.cc.u32  %5, %11, %17, %5;\n\t"
      "madc.hi.cc.u32  %6, %12, %17, %6;\n\t"
      "madc.hi.u32     %7, %13, %17, %7;\n\t"
      "mad.lo.cc.u32   %2, %9, %17, %2;\n\t"
      "madc.lo.cc.u32  %3, %10, %17, %3;\n\t"
      "madc.lo.cc.u32  %4, %11, %17, %4;\n\t"
      "madc.lo.cc.u32  %5, %12, %17, %5;\n\t"
      "madc.lo.cc.u32  %6, %13, %17, %6;\n\t"
      "madc.lo.u32     %7, %14, %17, %7;\n\t"
      "}"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(w0), "r"(w1));
#pragma unroll
  for (int i = 0; i < 4; ++i) acc.w[i] = ((uint64_t)r[2 * i + 1] << 32) | r[2 * i];
}

// acc += g * w (mod 2^128): 2-limb g, 128-bit w; 16 multiply-adds in carry chains.
__device__ __forceinline__ void wmac_w4_b4(Wide<2>& acc, const Wide<2>& g, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  uint32_t r[4], a[4];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    r[2 * i] = (uint32_t)acc.w[i]; r[2 * i + 1] = (uint32_t)(acc.w[i] >> 32);
    a[2 * i] = (uint32_t)g.w[i]; a[2 * i + 1] = (uint32_t)(g.w[i] >> 32);
  }
  asm("{\n\t"
      "mad.lo.cc.u32   %0, %4, %8, %0;\n\t"
      "madc.hi.cc.u32  %1, %4, %8, %1;\n\t"
      "madc.hi.cc.u32  %2, %5, %8, %2;\n\t"
      "madc.hi.u32     %3, %6, %8, %3;\n\t"
      "mad.lo.cc.u32   %1, %5, %8, %1;\n\t"
      "madc.lo.cc.u32  %2, %6, %8, %2;\n\t"
      "madc.lo.u32     %3, %7, %8, %3;\n\t"
      "mad.lo.cc.u32   %1, %4, %9, %1;\n\t"
      "madc.hi.cc.u32  %2, %4, %9, %2;\n\t"
      "madc.hi.u32     %3, %5, %9, %3;\n\t"
      "mad.lo.cc.u32   %2, %5, %9, %2;\n\t"
      "madc.lo.u32     %3, %6, %9, %3;\n\t"
      "mad.lo.cc.u32   %2, %4, %10, %2;\n\t"
      "madc.hi.u32     %3, %4, %10, %3;\n\t"
      "mad.lo.u32      %3, %5, %10, %3;\n\t"
      "mad.lo.u32      %3, %4, %11, %3;\n\t"
      "}"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(w0), "r"(w1), "r"(w2), "r"(w3));
#pragma unroll
  for (int i = 0; i < 2; ++i) acc.w[i] = ((uint64_t)r[2 * i + 1] << 32) | r[2 * i];
}

// acc += g * w (mod 2^192): 3-limb g, 128-bit w; 32 multiply-adds in carry chains.
__device__ __forceinline__ void wmac_w6_b4(Wide<3>& acc, const Wide<3>& g, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  uint32_t r[6], a[6];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r[2 * i] = (uint32_t)acc.w[i]; r[2 * i + 1] = (uint32_t)(acc.w[i] >> 32);
    a[2 * i] = (uint32_t)g.w[i]; a[2 * i + 1] = (uint32_t)(g.w[i] >> 32);
  }
  asm("{\n\t"
      "mad.lo.cc.u32   %0, %6, %12, %0;\n\t"
      "madc.hi.cc.u32  %1, %6, %12, %1;\n\t"
      "madc.hi.cc.u32  %2, %7, %12, %2;\n\t"
      "madc.hi.cc.u32  %3, %8, %12, %3;\n\t"
      "madc.hi.cc.u32  %4, %9, %12, %4;\n\t"
      "madc.hi.u32     %5, %10, %12, %5;\n\t"
      "mad.lo.cc.u32   %1, %7, %12, %1;\n\t"
      "madc.lo.cc.u32  %2, %8, %12, %2;\n\t"
      "madc.lo.cc.u32  %3, %9, %12, %3;\n\t"
      "madc.lo.cc.u32  %4, %10, %12, %4;\n\t"
      "madc.lo.u32     %5, %11, %12, %5;\n\t"
      "mad.lo.cc.u32   %1, %6, %13, %1;\n\t"
      "madc.hi.cc.u32  %2, %6, %13, %2;\n\t"
      "madc.hi.cc.u32  %3, %7, %13, %3;\n\t"
      "madc.hi.cc.u32  %4, %8, %13, %4;\n\t"
      "madc.hi.u32     %5, %9, %13, %5;\n\t"
      "mad.lo.cc.u32   %2, %7, %13, %2;\n\t"
      "madc.lo.cc.u32  %3, %8, %13, %3;\n\t"
      "madc.lo.cc.u32  %4, %9, %13, %4;\n\t"
      "madc.lo.u32     %5, %10, %13, %5;\n\t"
      "mad.lo.cc.u32   %2, %6, %14, %2;\n\t"
      "madc.hi.cc.u32  %3, %6, %14, %3;\n\t"
      "madc.hi.cc.u32  %4, %7, %14, %4;\n\t"
      "madc.hi.u32     %5, %8, %14, %5;\n\t"
      "mad.lo.cc.u32   %3, %7, %14, %3;\n\t"
      "madc.lo.cc.u32  %4, %8, %14, %4;\n\t"
      "madc.lo.u32     %5, %9, %14, %5;\n\t"
      "mad.lo.cc.u32   %3, %6, %15, %3;\n\t"
      "madc.hi.cc.u32  %4, %6, %15, %4;\n\t"
      "madc.hi.u32     %5, %7, %15, %5;\n\t"
      "mad.lo.cc.u32   %4, %7, %15, %4;\n\t"
      "madc.lo.u32     %5, %8, %15, %5;\n\t"
      "}"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(w0), "r"(w1), "r"(w2), "r"(w3));
#pragma unroll
  for (int i = 0; i < 3; ++i) acc.w[i] = ((uint64_t)r[2 * i + 1] << 32) | r[2 * i];
}

// acc += g * w (mod 2^256): 4-limb g, 128-bit w; 48 multiply-adds in carry chains.
__device__ __forceinline__ void wmac_w8_b4(Wide<4>& acc, const Wide<4>& g, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  uint32_t r[8], a[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    r[2 * i] = (uint32_t)acc.w[i]; r[2 * i + 1] = (uint32_t)(acc.w[i] >> 32);
    a[2 * i] = (uint32_t)g.w[i]; a[2 * i + 1] = (uint32_t)(g.w[i] >> 32);
  }
  asm("{\n\t"
      "mad.lo.cc.u32   %0, %8, %16, %0;\n\t"
      "madc.hi.cc.u32  %1, %8, %16, %1;\n\t"
      "madc.hi.cc.u32  %2, %9, %16, %2;\n\t"
      "madc.hi.cc.u32  %3, %10, %16, %3;\n\t"
      "madc.hi.cc.u32  %4, %11, %16, %4;\n\t"
      "madc.hi.cc.u32  %5, %12, %16, %5;\n\t"
      "madc.hi.cc.u32  %6, %13, %16, %6;\n\t"
      "madc.hi.u32     %7, %14, %16, %7;\n\t"
      "mad.lo.cc.u32   %1, %9, %16, %1;\n\t"
      "madc.lo.cc.u32  %2, %10, %16, %2;\n\t"
      "madc.lo.cc.u32  %3, %11, %16, %3;\n\t"
      "madc.lo.cc.u32  %4, %12, %16, %4;\n\t"
      "madc.lo.cc.u32  %5, %13, %16, %5;\n\t"
      "madc.lo.cc.u32  %6, %14, %16, %6;\n\t"
      "madc.lo.u32     %7, %15, %16, %7;\n\t"
      "mad.lo.cc.u32   %1, %8, %17, %1;\n\t"
      "madc.hi.cc.u32  %2, %8, %17, %2;\n\t"
      "madc.hi.cc.u32  %3, %9, %17, %3;\n\t"
      "madc.hi.cc.u32  %4, %10, %17, %4;\n\t"
      "madc.hi.cc.u32  %5, %11, %17, %5;\n\t"
      "madc.hi.cc.u32  %6, %12, %17, %6;\n\t"
      "madc.hi.u32     %7, %13, %17, %7;\n\t"
      "mad.lo.cc.u32   %2, %9, %17, %2;\n\t"
      "madc.lo.cc.u32  %3, %10, %17, %3;\n\t"
      "madc.lo.cc.u32  %4, %11, %17, %4;\n\t"
      "madc.lo.cc.u32  %5, %12, %17, %5;\n\t"
      "madc.lo.cc.u32  %6, %13, %17, %6;\n\t"
      "madc.lo.u32     %7, %14, %17, %7;\n\t"
      "mad.lo.cc.u32   %2, %8, %18, %2;\n\t"
      "madc.hi.cc.u32  %3, %8, %18, %3;\n\t"
      "madc.hi.cc.u32  %4, %9, %18, %4;\n\t"
      "madc.hi.cc.u32  %5, %10, %18, %5;\n\t"
      "madc.hi.cc.u32  %6, %11, %18, %6;\n\t"
      "madc.hi.u32     %7, %12, %18, %7;\n\t"
      "mad.lo.cc.u32   %3, %9, %18, %3;\n\t"
      "madc.lo.cc.u32  %4, %10, %18, %4;\n\t"
      "madc.lo.cc.u32  %5, %11, %18, %5;\n\t"
      "madc.lo.cc.u32  %6, %12, %18, %6;\n\t"
      "madc.lo.u32     %7, %13, %18, %7;\n\t"
      "mad.lo.cc.u32   %3, %8, %19, %3;\n\t"
      "madc.hi.cc.u32  %4, %8, %19, %4;\n\t"
      "madc.hi.cc.u32  %5, %9, %19, %5;\n\t"
      "madc.hi.cc.u32  %6, %10, %19, %6;\n\t"
      "madc.hi.u32     %7, %11, %19, %7;\n\t"
      "mad.lo.cc.u32   %4, %9, %19, %4;\n\t"
      "madc.lo.cc.u32  %5, %10, %19, %5;\n\t"
      "madc.lo.cc.u32  %6, %11, %19, %6;\n\t"
      "madc.lo.u32     %7, %12, %19, %7;\n\t"
      "}"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(w0), "r"(w1), "r"(w2), "r"(w3));
#pragma unroll
  for (int i = 0; i < 4; ++i) acc.w[i] = ((uint64_t)r[2 * i + 1] << 32) | r[2 * i];
}

// acc += g * w (mod 2^128) for a two-limb g and a 32-bit w (seven partial products).
__device__ __forceinline__ void wmac2_u32(Wide<2>& acc, const Wide<2>& g, uint32_t w0) {
  uint32_t r0 = (uint32_t)acc.w[0], r1 = (uint32_t)(acc.w[0] >> 32);
  uint32_t r2 = (uint32_t)acc.w[1], r3 = (uint32_t)(acc.w[1] >> 32);
  const uint32_t a0 = (uint32_t)g.w[0], a1 = (uint32_t)(g.w[0] >> 32);
  const uint32_t a2 = (uint32_t)g.w[1], a3 = (uint32_t)(g.w[1] >> 32);
  asm("{\n\t"
      "mad.lo.cc.u32  %0, %4, %8, %0;\n\t"
      "madc.hi.cc.u32 %1, %4, %8, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %8, %2;\n\t"
      "madc.hi.u32    %3, %6, %8, %3;\n\t"
      "mad.lo.cc.u32  %1, %5, %8, %1;\n\t"
      "madc.lo.cc.u32 %2, %6, %8, %2;\n\t"
      "madc.lo.u32    %3, %7, %8, %3;\n\t"
      "}"
      : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3)
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(w0));
  acc.w[0] = ((uint64_t)r1 << 32) | r0;
  acc.w[1] = ((uint64_t)r3 << 32) | r2;
}

// Weight table element types per order: D < 2^32 (n = 1), < 2^60 (n = 2), < 2^121 (n = 3)
// (room for the FD weight |w_j| <= 16, resp. 81, folded into the table weight).
template <int N> struct WeightT;
template <> struct WeightT<1> { using T = uint32_t; };
template <> struct WeightT<2> { using T = uint64_t; };
template <> struct WeightT<3> { using T = ulonglong2; };

// acc += g * w for the table word types.
template <int L, typename WT>
__device__ __forceinline__ void mac_weight(Wide<L>& acc, const Wide<L>& gv, const WT w) {
  if constexpr (sizeof(WT) == 16) {
    if constexpr (L == 1) wmac<1>(acc, gv, w.x);
    else if constexpr (L == 2) wmac_w4_b4(acc, gv, (uint32_t)w.x, (uint32_t)(w.x >> 32), (uint32_t)w.y, (uint32_t)(w.y >> 32));
    else if constexpr (L == 3) wmac_w6_b4(acc, gv, (uint32_t)w.x, (uint32_t)(w.x >> 32), (uint32_t)w.y, (uint32_t)(w.y >> 32));
    else wmac_w8_b4(acc, gv, (uint32_t)w.x, (uint32_t)(w.x >> 32), (uint32_t)w.y, (uint32_t)(w.y >> 32));
  } else if constexpr (sizeof(WT) == 8) {
    if constexpr (L == 1) wmac<1>(acc, gv, w);
    else if constexpr (L == 2) wmac2_u64(acc, gv, w);
    else if constexpr (L == 3) wmac_w6_b2(acc, gv, (uint32_t)w, (uint32_t)(w >> 32));
    else wmac_w8_b2(acc, gv, (uint32_t)w, (uint32_t)(w >> 32));
  } else if constexpr (L == 2) {
    wmac2_u32(acc, gv, w);
  } else {
    wmac<L>(acc, gv, (uint64_t)w);
  }
}

// -a (mod 2^(64L))
template <int L>
__device__ __forceinline__ Wide<L> wneg(const Wide<L>& a) {
  Wide<L> r;
  uint64_t carry = 1;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const uint64_t v = ~a.w[i] + carry;
    carry = (carry && v == 0) ? 1 : 0;
    r.w[i] = v;
  }
  return r;
}

// acc += w * t for a small signed integer w.
template <int L>
__device__ __forceinline__ void wmac_signed(Wide<L>& acc, const Wide<L>& t, int w) {
  if (w >= 0) {
    wmac<L>(acc, t, (uint64_t)w);
  } else {
    Wide<L> p;
    wzero<L>(p);
    wmac<L>(p, t, (uint64_t)(-w));
    wsub<L>(acc, p);
  }
}

// Signed value of a two's complement L-limb integer, rounded to binary64
// (a few roundings; the exact value is available from the numerator API).
template <int L>
__device__ __forceinline__ double wto_double(const Wide<L>& a) {
  Wide<L> m = a;
  const bool neg = (m.w[L - 1] >> 63) != 0;
  if (neg) {
    uint64_t carry = 1;
#pragma unroll
    for (int i = 0; i < L; ++i) {
      uint64_t v = ~m.w[i] + carry;
      carry = (carry && v == 0) ? 1 : 0;
      m.w[i] = v;
    }
  }
  double v = 0.0;
#pragma unroll
  for (int i = L - 1; i >= 0; --i) v = v * 18446744073709551616.0 + (double)m.w[i];
  return neg ? -v : v;
}

template <int L>
__device__ __forceinline__ Wide<L> wload(const uint64_t* p) {
  Wide<L> r;
  if constexpr (L == 2) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
    r.w[0] = v.x;
    r.w[1] = v.y;
  } else if constexpr (L == 4) {
    const ulonglong2 v0 = reinterpret_cast<const ulonglong2*>(p)[0];
    const ulonglong2 v1 = reinterpret_cast<const ulonglong2*>(p)[1];
    r.w[0] = v0.x; r.w[1] = v0.y; r.w[2] = v1.x; r.w[3] = v1.y;
  } else {
#pragma unroll
    for (int i = 0; i < L; ++i) r.w[i] = p[i];
  }
  return r;
}

template <int L>
__device__ __forceinline__ void wstore(uint64_t* p, const Wide<L>& a) {
  if constexpr (L == 2) {
    *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(a.w[0], a.w[1]);
  } else if constexpr (L == 4) {
    reinterpret_cast<ulonglong2*>(p)[0] = make_ulonglong2(a.w[0], a.w[1]);
    reinterpret_cast<ulonglong2*>(p)[1] = make_ulonglong2(a.w[2], a.w[3]);
  } else {
#pragma unroll
    for (int i = 0; i < L; ++i) p[i] = a.w[i];
  }
}

// Sign-extend a signed 64-bit integer into L limbs.
template <int L>
__device__ __forceinline__ Wide<L> wfrom_i64(int64_t v) {
  Wide<L> r;
  r.w[0] = (uint64_t)v;
  const uint64_t ext = v < 0 ? ~0ull : 0ull;
#pragma unroll
  for (int i = 1; i < L; ++i) r.w[i] = ext;
  return r;
}

// Acquire / release accesses for the scan look-back flags.
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// After relaxed loads that observed release stores: the data those stores
// published is visible to the loads that follow.
__device__ __forceinline__ void fence_acquire() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// ------------------------------------------------------- interpolation stencil
// A tap y = p + r has r in [0,1)^2 (even n, p = floor y) or [-1/2,1/2)^2 (odd
// n, p = nearest); its lattice neighbours are p + d, d in [dmin, dmin + 3n)^2.
// The weight of neighbour d is ZP^{*n}(r - d), whose support is the open
// octagon |x|, |y| < 3n/2, |x +- y| < 2n.  A neighbour whose weight is zero for
// every r is dropped: the box of possible r - d and the octagon are convex, so
// they meet iff their projections on x, y, x + y and x - y overlap (worked in
// doubled coordinates).  9, 32 and 69 neighbours remain for n = 1, 2, 3.
template <int N>
__host__ __device__ constexpr bool stencil_keeps(int ix, int iy) {
  const int dmin = (N % 2 == 0) ? (-(3 * N) / 2 + 1) : (-(3 * N - 1) / 2);
  const int off = (N % 2 == 0) ? 0 : -1;  // 2 x (lower end of r)
  const int lx = -2 * (dmin + ix) + off, hx = lx + 2;
  const int ly = -2 * (dmin + iy) + off, hy = ly + 2;
  return lx < 3 * N && -3 * N < hx && ly < 3 * N && -3 * N < hy && lx + ly < 4 * N && -4 * N < hx + hy &&
         lx - hy < 4 * N && -4 * N < hx - ly;
}

template <int N>
__host__ __device__ constexpr int stencil_count() {
  int c = 0;
  for (int iy = 0; iy < 3 * N; ++iy)
    for (int ix = 0; ix < 3 * N; ++ix) c += stencil_keeps<N>(ix, iy) ? 1 : 0;
  return c;
}

template <int N>
struct Stencil {
  static constexpr int kN3 = 3 * N;
  static constexpr int kDmin = (N % 2 == 0) ? (-(3 * N) / 2 + 1) : (-(3 * N - 1) / 2);
  int count;
  int dx[9 * N * N];
  int dy[9 * N * N];
  constexpr Stencil() : count(0), dx(), dy() {
    for (int iy = 0; iy < kN3; ++iy)
      for (int ix = 0; ix < kN3; ++ix)
        if (stencil_keeps<N>(ix, iy)) {
          dx[count] = kDmin + ix;
          dy[count] = kDmin + iy;
          ++count;
        }
  }
};

// ---------------------------------------------------------------- host side

// Everything a kernel needs to know about one plan (passed by value).
// Row-pass input types beyond abf_dtype: integer coefficients staged on the
// device (the 1-D prefilter's output), read without conversion or checks.
constexpr int kStageI32 = 16;
constexpr int kStageI64 = 17;

struct PlanView {
  int W, H, n, Q, P, F;
  int left, right, above;         // lattice box margins (rows start at k2 = 0)
  int Gw, Gh;                     // lattice box width / height
  long long Gp;                   // row pitch of g, elements
  int Cmax, Cmin;                 // integer step bounds (units 2^-Q)
  int scale_kind, in_dtype, out_dtype;
  int limbs;
  double value_bound;             // bound on |f|
  double log2D;                   // log2 of the weight denominator
  float log2_base;                // log2(D |f|max 2^F): the pixel-independent part of the bound
  double Dd;                      // D as binary64
  int table_bytes_per_w;          // 4, 8 or 16
  const void* table;              // (2^P)^2 rows of (3n)^2 weights
  const void* table_fold;         // n = 3: the table folded by the square's symmetries, else null
  // Running sums per direction v1..v4 (n each for the four-direction filter;
  // (n, 0, n, 0) for N = 2), and, for the generalised mesh, the unit boxes E
  // per axis of the model phi, the kernel's stencil and the output origin.
  int r[4];
  int E;                          // 0: phi = delta
  int R, dminx, dminy;            // generalised table: neighbours per row, stencil box origin
  const int2* stencil;            // generalised table: the R neighbours (dx, dy)
  const void* gtaps;              // generalised mesh: the taps grouped by FD weight
  double out_scale;               // generalised mesh: 2^(Q sum r - F) / D
  int den_int;                    // generalised mesh: prod_k C_k^{r_k} fits 63 bits
  unsigned long long* dbg;        // ABF_FLAG_DEBUG_BOUNDS: first violating pixel + 1, else null
  int ox, oy;                     // output pixel m sits at lattice point m + (ox, oy)
};

// ------------------------------------------------------ per-pixel scale reading
// Paper scales a_k (Sec. 7) -> lattice steps c_k (c2 = a2 / sqrt2, c4 = a4 / sqrt2),
// or the ellipse moment rule; then C_k = rint(c_k 2^Q).  binary64 with explicit
// round-to-nearest intrinsics (no contraction into fused multiply-adds), so the
// integers agree with any other IEEE implementation of the same sequence.
constexpr double kInvSqrt2 = 0.7071067811865476;

// Lattice steps from one pixel's scale record; returns false on invalid input.
__device__ __forceinline__ bool read_steps(int kind, float4 sc, int n, double cmax, double c[4]) {
  const double a0 = sc.x, a1 = sc.y, a2 = sc.z, a3 = sc.w;
  if (kind == ABF_SCALES_C4) {
    c[0] = a0; c[1] = a1; c[2] = a2; c[3] = a3;
  } else if (kind == ABF_SCALES_A4) {
    c[0] = a0;
    c[1] = __dmul_rn(a1, kInvSqrt2);
    c[2] = a2;
    c[3] = __dmul_rn(a3, kInvSqrt2);
  } else {
    // Ellipse (sigma, elongation, cos t, sin t) -> covariance -> moment rule.
    const double sigma = a0, elong = a1, ct = a2, st = a3;
    if (!(sigma > 0.0) || !(elong > 0.0) || !isfinite(sigma) || !isfinite(elong) || !isfinite(ct) ||
        !isfinite(st))
      return false;
    const double s2 = __dmul_rn(sigma, sigma);
    const double ev1 = __dmul_rn(s2, elong);
    const double ev2 = __ddiv_rn(s2, elong);
    const double cc = __dmul_rn(ct, ct);
    const double ss = __dmul_rn(st, st);
    const double cs = __dmul_rn(ct, st);
    const double c11 = __dadd_rn(__dmul_rn(ev1, cc), __dmul_rn(ev2, ss));
    const double c22 = __dadd_rn(__dmul_rn(ev1, ss), __dmul_rn(ev2, cc));
    const double c12 = __dmul_rn(__dsub_rn(ev1, ev2), cs);
    const double a12 = fabs(c12);
    const double mn = c11 < c22 ? c11 : c22;
    const double t = (a12 <= mn) ? __dmul_rn(0.25, __dadd_rn(a12, mn)) : __dmul_rn(0.5, mn);
    const double h = __dmul_rn(0.5, c12);
    double u[4];
    u[0] = __dsub_rn(c11, __dmul_rn(2.0, t));
    u[1] = __dadd_rn(t, h);
    u[2] = __dsub_rn(c22, __dmul_rn(2.0, t));
    u[3] = __dsub_rn(t, h);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double uk = u[k] < 0.0 ? 0.0 : u[k];
      // 12 u_k / n: for n = 1, 2 the quotient is the correctly rounded product
      // with 1/n (exact), the same double as the division gives
      const double t12 = __dmul_rn(12.0, uk);
      const double q = n == 1 ? t12 : (n == 2 ? __dmul_rn(t12, 0.5) : __ddiv_rn(t12, (double)n));
      double ck = __dsqrt_rn(q);
      if (ck < 1.0) ck = 1.0;
      if (ck > cmax) ck = cmax;
      c[k] = ck;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (!isfinite(c[k]) || !(c[k] > 0.0)) return false;
  return true;
}

// C_k = rint(c_k 2^Q), validated against the plan's bounds.
__device__ __forceinline__ bool pixel_steps(const PlanView& pv, const float4* scales, size_t scale_pitch,
                                            int x, int y, int C[4]) {
  const float4 sc = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(scales) +
                                                     (size_t)y * scale_pitch + (size_t)x * sizeof(float4));
  if (pv.scale_kind == ABF_SCALES_C4) {
    // direct steps: c 2^Q is exact in binary32 (a power-of-two scaling; inf
    // when it overflows) and rintf rounds it as rint would in binary64, so the
    // same integers come out without the binary64 pipe
    const float cf[4] = {sc.x, sc.y, sc.z, sc.w};
    const float q = ldexpf(1.0f, pv.Q);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (!isfinite(cf[k]) || !(cf[k] > 0.0f)) return false;
      const float v = cf[k] * q;
      if (!(v < 2147483648.0f)) return false;
      const int r = __float2int_rn(v);
      if (r < 1 || r > pv.Cmax) return false;
      C[k] = r;
    }
    return C[0] >= pv.Cmin && C[2] >= pv.Cmin;
  }
  double c[4];
  const double cmax = ldexp((double)pv.Cmax, -pv.Q);
  if (!read_steps(pv.scale_kind, sc, pv.n, cmax, c)) return false;
  const double q = ldexp(1.0, pv.Q);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double v = c[k] * q;  // exact (power of two)
    if (!(v < 2147483648.0)) return false;
    const long long r = __double2ll_rn(v);
    if (r < 1 || r > pv.Cmax) return false;  // Cmax = rint(max_scale 2^Q): rint is monotone
    C[k] = (int)r;
  }
  if (C[0] < pv.Cmin || C[2] < pv.Cmin) return false;
  return true;
}


// Device status word bits are the ABF_DEV_* values of abf.h.
__device__ __forceinline__ void raise_status(int32_t* st, int32_t bits) {
  atomicOr(st, bits);
}

// ABF_FLAG_DEBUG_BOUNDS: whether the reads of a tap whose lattice point is box
// column cx, row py, with stencil offsets dx in [dxlo, dxhi] and dy <= dyhi,
// stay in the lattice box (rows below 0 are never read).  On a violation the
// status gets ABF_DEV_BOUNDS and the first pixel is recorded; the caller
// skips the tap.
__device__ __forceinline__ bool dbg_tap_ok(const PlanView& pv, int32_t* status, int cx, int py, int dxlo, int dxhi,
                                           int dyhi, int x, int y) {
  if (cx + dxlo >= 0 && cx + dxhi < pv.Gw && py + dyhi < pv.Gh) return true;
  raise_status(status, ABF_DEV_BOUNDS);
  atomicCAS(pv.dbg, 0ull, (unsigned long long)y * (unsigned long long)pv.W + (unsigned long long)x + 1ull);
  return false;
}

// Input element -> integer f 2^F; raises ABF_DEV_BAD_INPUT (and reads 0) when
// a floating-point value is off the 2^-F grid or beyond the value bound
// (bound_i = floor(value_bound 2^F)).  binary32 inputs are checked in binary32
// (scaling by 2^F is exact, rintf is exact) and integers, keeping the per-sample
// work off the slow binary64 pipe.
template <typename TIn>
__device__ __forceinline__ int64_t convert_f(TIn raw, double scale, long long bound_i, int32_t* status) {
  if constexpr (std::is_integral<TIn>::value) {
    if constexpr (sizeof(TIn) <= 2) return (int64_t)raw * (int64_t)scale;  // u8 / u16 samples
    else return (int64_t)raw;  // integer coefficients staged by the 1-D prefilter: already c 2^F
  } else if constexpr (sizeof(TIn) == 4) {
    const float v = raw * (float)scale;  // exact: scale is a power of two (inf if it overflows)
    if (!(rintf(v) == v) || !(fabsf(v) < 4.0e18f)) {
      raise_status(status, ABF_DEV_BAD_INPUT);
      return 0;
    }
    // a 32-bit conversion where it fits: the 64-bit one issues on the binary64 pipe
    const long long r = fabsf(v) < 2147483648.0f ? (long long)__float2int_rn(v) : __float2ll_rn(v);
    if (r > bound_i || r < -bound_i) {
      raise_status(status, ABF_DEV_BAD_INPUT);
      return 0;
    }
    return r;
  } else {
    const double v = (double)raw * scale;  // exact: scale is a power of two
    const double r = rint(v);
    if (!(r == v) || !(fabs(r) < 4.0e18)) {
      raise_status(status, ABF_DEV_BAD_INPUT);
      return 0;
    }
    const long long ri = (long long)r;
    if (ri > bound_i || ri < -bound_i) {
      raise_status(status, ABF_DEV_BAD_INPUT);
      return 0;
    }
    return ri;
  }
}


}  // namespace abf

// A plan (opaque in the C ABI).
struct abf_plan_s {
  abf_desc desc;
  abf::PlanView pv;
  void* real_table = nullptr;  // tile forms: pair weight table (D0 ZP^{*n})
  double D0 = 0.0;             // tile forms: D = D0 2^((4n-2)P)
  double tol_abs = 0.0;        // tile forms: error tolerance times the value bound
  unsigned __int128 D;
  int device;
  int32_t* d_status = nullptr;
  size_t g_bytes = 0, ws_bytes = 0;
  int mesh_warps = 8;          // rows per CTA of the exact mesh (abf_plan_autotune)
  // Generalised plans (N = 2, or a B-spline model phi): pv is the mesh's view
  // (output pixels, origin); sv the running sums' view of their input (the
  // image, or the model coefficients staged on an extended frame).
  bool general = false;
  abf::PlanView sv{};
  void* d_stage = nullptr;     // model coefficients c_q (int64), sv.W x sv.H
  void* d_pf_tmp = nullptr;    // prefilter intermediate (int64), H rows x sv.W, and the column pass' state
  size_t pf_tmp_bytes = 0;
  void* pf = nullptr;          // prefilter constants (host copy)
  void* d_gtaps = nullptr;     // generalised mesh: the taps grouped by FD weight
  void* d_dbg = nullptr;       // ABF_FLAG_DEBUG_BOUNDS: the first violating pixel + 1
};

namespace abf {
// The 1-D interpolation prefilter's constants (Sec. 3; its kernels are in
// line1d.cu), shared with the 2-D model's separable prefilter.
constexpr int kPfHalo = 64;                         // >= every warm-up length W_p
constexpr int kPfMaxPoles = 2;
struct PrefilterView {
  int length, Gw, left, G, npoles;
  int W[kPfMaxPoles];            // warm-up samples per pole
  long long Z[kPfMaxPoles];      // rint(z_p 2^64)
  long long A[kPfMaxPoles];      // rint(A_p 2^60)
  double scale;                  // 2^F
  long long bound;               // floor(value_bound 2^F)
};
abf_status prefilter2d_setup(int n1, double xmax, PrefilterView* pf, double* hnorm, int* tail);
// Host-side fault injection (abf_debug_inject_fault, ABF_FAULT): take one
// armed fault of a kind (true if one was armed), or test whether a kind is armed.
bool fault_take(int kind);
bool fault_active(int kind);
cudaError_t run_prefilter_rows_raw(const PrefilterView& v, int count, int in_dtype, const void* f, size_t f_pitch,
                                   long long* c, long long c_pitch, int32_t* status, cudaStream_t st);

// One image of a batched adaptive step (run_mesh_batch).
struct BatchIn {
  PlanView pv;
  const uint64_t* g;
  const void* scales;
  size_t scale_pitch;
  void* s;
  size_t s_pitch;
  int32_t* status;
};
int batch_max_jobs();
// Persistent launches of the adaptive step over many images, one per (order,
// limbs, fast path) group; counter: 32 64-bit device counters.
cudaError_t run_mesh_batch(const BatchIn* in, int njobs, unsigned long long* counter, int warps, cudaStream_t st);

// abf_integrate / abf_filter (exact form) with the device status word given by
// the caller instead of the plan's own: the serving loop gives every slot its
// own word, so that jobs sharing a plan do not see each other's flags.
abf_status integrate_with_status(abf_plan p, const void* d_f, size_t f_pitch, void* d_g, void* d_ws,
                                 int32_t* d_status, cudaStream_t st);
abf_status filter_with_status(abf_plan p, const void* d_g, const void* d_scales, size_t scale_pitch, void* d_s,
                              size_t s_pitch, int32_t* d_status, cudaStream_t st);
}  // namespace abf
