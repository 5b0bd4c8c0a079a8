// Adaptive step of Sec. 7 (2), Eq. (final_eqn), exact form:
//
//   s[m] = (c1 c2 c3 c4)^-n sum_j w_j g_I(m + tau - sum_k j_k c_k v_k)
//
// with j in {0..n}^4, w_j = prod_k (-1)^{j_k} binom(n, j_k) (for n = 1 the 16
// vertices and signs of Table "Mesh Vertices"), tau = (n/2) sum_k (c_k - 1) v_k
// (Sec. 7; times n at order n), and g_I(y) = sum_k g[k] ZP^{*n}(y - k) the ZP
// interpolation of the integrated image.
//
// Exact arithmetic: c_k = C_k 2^-Q with integer C_k, so every tap y_j is on the
// 2^-P grid (P = Q for even n, Q + 1 for odd n), and D ZP^{*n} is an integer
// there (table built by the plan).  The numerator
//   S[m] = D sum_j w_j g_I(y_j)
// is formed modulo 2^(64 L); its true size is bounded by
//   D (prod c)^n |f|max 2^F (1 + 1/c1)(1 + 1/c3)
// (|s| <= |f|max times the lattice sum of the kernel), checked per pixel.
// s = S 2^(4 Q n) / (D (prod C)^n 2^F) in binary64.
//
// Per-pixel scale readings (a5): the kind-specific map to lattice steps and the
// rounding C_k = rint(c_k 2^Q) use binary64 with explicit round-to-nearest
// intrinsics (no contraction into fused multiply-adds), so the integers agree
// with any other IEEE implementation of the same operation sequence.
#include "abf_internal.cuh"

namespace abf {

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
      double ck = __dsqrt_rn(__ddiv_rn(__dmul_rn(12.0, uk), (double)n));
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
  double c[4];
  const double cmax = ldexp((double)pv.Cmax, -pv.Q);
  if (!read_steps(pv.scale_kind, sc, pv.n, cmax, c)) return false;
  const double q = ldexp(1.0, pv.Q);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double v = c[k] * q;  // exact (power of two)
    if (!(v <= (double)pv.Cmax)) return false;
    const long long r = __double2ll_rn(v);
    if (r < 1) return false;
    C[k] = (int)r;
  }
  if (C[0] < pv.Cmin || C[2] < pv.Cmin) return false;
  return true;
}

// log2 of the numerator bound for this pixel (see file header).
__device__ __forceinline__ double numerator_log2_bound(const PlanView& pv, const int C[4]) {
  double lp = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) lp += log2((double)C[k]);
  const double q = ldexp(1.0, pv.Q);
  const double kappa = (1.0 + q / C[0]) * (1.0 + q / C[2]);
  return pv.log2D + pv.n * (lp - 4.0 * pv.Q) + log2(pv.value_bound) + pv.F + log2(kappa) + 1e-6;
}

// (-1)^j binom(N, j) for N <= 3: binom is 1 at the ends and N inside.
template <int N>
__device__ __forceinline__ int signed_binom(int j) {
  const int c = (j == 0 || j == N) ? 1 : N;
  return (j & 1) ? -c : c;
}

// Weight table element types per order: D < 2^32 (n = 1), < 2^64 (n = 2), < 2^128 (n = 3).
template <int N> struct WeightT;
template <> struct WeightT<1> { using T = uint32_t; };
template <> struct WeightT<2> { using T = uint64_t; };
template <> struct WeightT<3> { using T = ulonglong2; };

template <int L, typename WT>
__device__ __forceinline__ void mac_weight(Wide<L>& acc, const Wide<L>& gv, const WT w) {
  if constexpr (sizeof(WT) == 16) {
    wmac128<L>(acc, gv, w.x, w.y);
  } else {
    wmac<L>(acc, gv, (uint64_t)w);
  }
}

template <typename WT>
__device__ __forceinline__ bool wnonzero(const WT w) {
  if constexpr (sizeof(WT) == 16) return (w.x | w.y) != 0;
  else return w != 0;
}

// The numerator S for pixel (x, y) with integer steps C.
template <int N, int L>
__device__ __forceinline__ Wide<L> mesh_numerator(const PlanView& pv, const uint64_t* __restrict__ g,
                                                  int x, int y, const int C[4]) {
  using WT = typename WeightT<N>::T;
  constexpr int N3 = 3 * N;
  constexpr int DMIN = (N % 2 == 0) ? (-(3 * N) / 2 + 1) : (-(3 * N - 1) / 2);
  const WT* __restrict__ table = reinterpret_cast<const WT*>(pv.table);
  const int P = pv.P;
  const int sh = (N % 2 == 0) ? 0 : 1;        // 2^(P-Q)
  const int one = 1 << pv.Q;
  const int half = (N % 2 == 0) ? 0 : (1 << (P - 1));
  const int mask = (1 << P) - 1;
  // tau in units of 2^-P: (n/2) sum_k (C_k - 2^Q) v_k 2^(P-Q)
  const int tx = (N * (C[0] + C[1] - C[3] - one)) << sh >> 1;
  const int ty = (N * (C[1] + C[2] + C[3] - 3 * one)) << sh >> 1;
  const int y0x = (x << P) + tx;
  const int y0y = (y << P) + ty;
  const int s1 = C[0] << sh, s2 = C[1] << sh, s3 = C[2] << sh, s4 = C[3] << sh;
  const long long rowpitch = pv.Gp;
  const int left = pv.left;

  Wide<L> S;
  wzero<L>(S);
#pragma unroll 1
  for (int j4 = 0; j4 <= N; ++j4) {
#pragma unroll 1
    for (int j2 = 0; j2 <= N; ++j2) {
#pragma unroll 1
      for (int j3 = 0; j3 <= N; ++j3) {
#pragma unroll 1
        for (int j1 = 0; j1 <= N; ++j1) {
          const int w = signed_binom<N>(j1) * signed_binom<N>(j2) * signed_binom<N>(j3) * signed_binom<N>(j4);
          // y_j = y0 - j1 c1 v1 - j2 c2 v2 - j3 c3 v3 - j4 c4 v4
          const int Yx = y0x - j1 * s1 - j2 * s2 + j4 * s4;
          const int Yy = y0y - j2 * s2 - j3 * s3 - j4 * s4;
          const int px = (Yx + half) >> P;
          const int py = (Yy + half) >> P;
          const int rx = (Yx + half) & mask;
          const int ry = (Yy + half) & mask;
          const WT* __restrict__ wrow = table + (size_t)((ry << P) | rx) * (N3 * N3);
          Wide<L> acc;
          wzero<L>(acc);
#pragma unroll
          for (int iy = 0; iy < N3; ++iy) {
            const int k2 = py + DMIN + iy;
            if (k2 < 0) continue;  // rows below the image: g = 0
            const uint64_t* __restrict__ grow = g + ((size_t)k2 * rowpitch + (size_t)(px + DMIN + left)) * L;
#pragma unroll
            for (int ix = 0; ix < N3; ++ix) {
              const WT wt = wrow[iy * N3 + ix];
              if (wnonzero(wt)) {
                const Wide<L> gv = wload<L>(grow + (size_t)ix * L);
                mac_weight<L, WT>(acc, gv, wt);
              }
            }
          }
          wmac_signed<L>(S, acc, w);
        }
      }
    }
  }
  return S;
}

template <typename TOut>
__device__ __forceinline__ void store_out(void* s, size_t s_pitch, int x, int y, double v) {
  TOut* row = reinterpret_cast<TOut*>(reinterpret_cast<char*>(s) + (size_t)y * s_pitch);
  row[x] = (TOut)v;
}

template <int N, int L, typename TOut>
__global__ void __launch_bounds__(128) mesh_exact_kernel(const PlanView pv, const uint64_t* __restrict__ g,
                                                         const float4* __restrict__ scales, size_t scale_pitch,
                                                         void* __restrict__ s, size_t s_pitch,
                                                         uint64_t* __restrict__ num, size_t num_pitch,
                                                         int32_t* status) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= pv.W || y >= pv.H) return;
  int C[4];
  if (!pixel_steps(pv, scales, scale_pitch, x, y, C)) {
    raise_status(status, ABF_DEV_BAD_SCALE);
    if (s) store_out<TOut>(s, s_pitch, x, y, __longlong_as_double(0x7ff8000000000000ll));
    return;
  }
  if (numerator_log2_bound(pv, C) >= 64.0 * L - 1.0) {
    raise_status(status, ABF_DEV_RANGE);
    if (s) store_out<TOut>(s, s_pitch, x, y, __longlong_as_double(0x7ff8000000000000ll));
    return;
  }
  const Wide<L> S = mesh_numerator<N, L>(pv, g, x, y, C);
  if (num) {
    uint64_t* p = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(num) + (size_t)y * num_pitch) + (size_t)x * L;
#pragma unroll
    for (int i = 0; i < L; ++i) p[i] = S.w[i];
  }
  if (s) {
    // s = S 2^(4Qn - F) / (D prod C^n)
    double den = pv.Dd;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double ck = (double)C[k];
      double p = 1.0;
#pragma unroll
      for (int e = 0; e < N; ++e) p *= ck;
      den *= p;
    }
    const double v = ldexp(wto_double<L>(S), 4 * pv.Q * N - pv.F) / den;
    store_out<TOut>(s, s_pitch, x, y, v);
  }
}

__global__ void prepare_scales_kernel(const PlanView pv, const float4* __restrict__ scales, size_t scale_pitch,
                                      int4* __restrict__ Cout, size_t C_pitch, int32_t* status) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= pv.W || y >= pv.H) return;
  int C[4];
  int4* row = reinterpret_cast<int4*>(reinterpret_cast<char*>(Cout) + (size_t)y * C_pitch);
  if (!pixel_steps(pv, scales, scale_pitch, x, y, C)) {
    raise_status(status, ABF_DEV_BAD_SCALE);
    row[x] = make_int4(0, 0, 0, 0);
    return;
  }
  row[x] = make_int4(C[0], C[1], C[2], C[3]);
}

// Maxima over the image of max_k c_k and of c1 c2 c3 c4 (after rounding to the
// 2^-Q grid), as the bit patterns of positive doubles (ordered like integers).
__global__ void measure_scales_kernel(const PlanView pv, const float4* __restrict__ scales, size_t scale_pitch,
                                      unsigned long long* out2, int32_t* status) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  double cm = 0.0, pr = 0.0;
  if (x < pv.W && y < pv.H) {
    const float4 sc = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(scales) +
                                                       (size_t)y * scale_pitch + (size_t)x * sizeof(float4));
    double c[4];
    if (read_steps(pv.scale_kind, sc, pv.n, ldexp((double)pv.Cmax, -pv.Q), c)) {
      const double q = ldexp(1.0, pv.Q);
      pr = 1.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double ck = rint(c[k] * q) / q;
        cm = fmax(cm, ck);
        pr *= ck;
      }
    } else {
      raise_status(status, ABF_DEV_BAD_SCALE);
    }
  }
  // warp reduction, then one atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    cm = fmax(cm, __shfl_xor_sync(0xffffffffu, cm, o));
    pr = fmax(pr, __shfl_xor_sync(0xffffffffu, pr, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out2 + 0, (unsigned long long)__double_as_longlong(cm));
    atomicMax(out2 + 1, (unsigned long long)__double_as_longlong(pr));
  }
}

cudaError_t run_measure_scales(const PlanView& pv, const void* scales, size_t scale_pitch,
                               unsigned long long* out2, int32_t* status, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  dim3 block(32, 4);
  dim3 grid((pv.W + 31) / 32, (pv.H + 3) / 4);
  measure_scales_kernel<<<grid, block, 0, st>>>(pv, (const float4*)scales, scale_pitch, out2, status);
  return cudaGetLastError();
}

template <int N, int L>
static cudaError_t launch_mesh_NL(const PlanView& pv, const uint64_t* g, const void* scales, size_t scale_pitch,
                                  void* s, size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status,
                                  cudaStream_t st) {
  dim3 block(32, 4);
  dim3 grid((pv.W + 31) / 32, (pv.H + 3) / 4);
  if (pv.out_dtype == ABF_F64)
    mesh_exact_kernel<N, L, double><<<grid, block, 0, st>>>(pv, g, (const float4*)scales, scale_pitch, s, s_pitch,
                                                            num, num_pitch, status);
  else
    mesh_exact_kernel<N, L, float><<<grid, block, 0, st>>>(pv, g, (const float4*)scales, scale_pitch, s, s_pitch,
                                                           num, num_pitch, status);
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_mesh_N(const PlanView& pv, const uint64_t* g, const void* scales, size_t scale_pitch,
                                 void* s, size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status,
                                 cudaStream_t st) {
  switch (pv.limbs) {
    case 1: return launch_mesh_NL<N, 1>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
    case 2: return launch_mesh_NL<N, 2>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
    case 3: return launch_mesh_NL<N, 3>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
    default: return launch_mesh_NL<N, 4>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
  }
}

cudaError_t run_mesh_exact(const PlanView& pv, const uint64_t* g, const void* scales, size_t scale_pitch, void* s,
                           size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status, cudaStream_t st) {
  switch (pv.n) {
    case 1: return launch_mesh_N<1>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
    case 2: return launch_mesh_N<2>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
    default: return launch_mesh_N<3>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
  }
}

cudaError_t run_prepare_scales(const PlanView& pv, const void* scales, size_t scale_pitch, void* C, size_t C_pitch,
                               int32_t* status, cudaStream_t st) {
  dim3 block(32, 4);
  dim3 grid((pv.W + 31) / 32, (pv.H + 3) / 4);
  prepare_scales_kernel<<<grid, block, 0, st>>>(pv, (const float4*)scales, scale_pitch, (int4*)C, C_pitch, status);
  return cudaGetLastError();
}

}  // namespace abf
