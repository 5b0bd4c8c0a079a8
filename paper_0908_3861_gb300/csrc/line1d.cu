// The 1-D scale-adaptive B-spline filter of Sec. 3 (Proposition "prop"), exact
// form, on a batch of signals (one per row).
//
//   Non-adaptive step: g = u_1^{(n2+1)} * c, n2+1 causal running sums of the
//     model coefficients c 2^F.  For model degree n1 in {0, 1} the
//     interpolation prefilter (b^{n1})^-1 is the identity and c = f; for n1 in
//     2..5 `prefilter_kernel` computes c = f * (b^{n1})^-1 rounded to the 2^-F
//     grid (below).  The row pass of scan.cu runs the sums, on rows extended by
//     `left` samples before the signal (the prefilter's tail; 0 for n1 <= 1)
//     and `right` samples past its end (the sums keep changing there while the
//     adaptive step reads them).
//   Adaptive step: s[m] = Delta_a^{n2+1} F(m), F(x) = sum_k g[k] beta^N(x +
//     tau - k), N = n1 + n2 + 1, tau = (a - 1)(n2 + 1)/2 (Eq. (link)): the FD
//     mask d^{n2+1}_a of Eq. (FD) at the points y_j = m + tau - a j, each
//     interpolated with the degree-N B-spline.
//
// Exact arithmetic: a = A 2^-Q, so y_j lies on the 2^-P grid, P = Q + 1, and
// D beta^N is an integer there for D = N! 2^(N P).  The table holds
// D beta^N(r - d) for r = R 2^-P in [0, 1) and the N+1 or N+2 integers d that
// can carry weight; it is built on the host from the B-spline recurrence of
// degree n from degree n-1 (two shifted copies weighted by linear factors) in
// integers, and every row is checked to sum to D (partition of unity).
//   S[m] = sum_j (-1)^j binom(n2+1, j) sum_d g[p_j + d] T[r_j][d]  (mod 2^(64 L))
//   s[m] = S[m] 2^(Q (n2+1)) / (D A^(n2+1) 2^F)  in binary64, as S[m] times a
//   per-plan table of the normaliser's reciprocal per integer scale A (one
//   binary64 multiply per sample instead of a division and a power).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "abf_internal.cuh"

namespace abf {

cudaError_t run_row_scan(const PlanView& pv, const void* f, size_t f_pitch, uint64_t* g, int32_t* status,
                         cudaStream_t st);

struct Line1dView {
  int length, count, n1, n2, N, Q, P, F, K, dmin;
  int left;          // samples of g before the signal (g index = k + left)
  int Amax;
  long long Gp;      // row pitch of g, elements
  int limbs;
  int out_dtype;
  float log2_base;   // log2(D |f|max 2^F)
  double Dd;         // D
  const uint64_t* table;  // 2^P rows x K entries
  const double* rtab;     // R[A] = 2^(Q(n2+1) - F) / (D A^(n2+1)), A = 0..Amax, or null
};

// acc += g * w (mod 2^(64 L)) for a 64-bit table weight, as carry chains.
template <int L>
__device__ __forceinline__ void mac64(Wide<L>& acc, const Wide<L>& gv, uint64_t w) {
  if constexpr (L == 1) wmac<1>(acc, gv, w);
  else if constexpr (L == 2) wmac2_u64(acc, gv, w);
  else if constexpr (L == 3) wmac_w6_b2(acc, gv, (uint32_t)w, (uint32_t)(w >> 32));
  else wmac_w8_b2(acc, gv, (uint32_t)w, (uint32_t)(w >> 32));
}

template <int N2>
__device__ __forceinline__ int binom_n2p1(int j) {
  // binom(N2 + 1, j)
  int c = 1;
#pragma unroll
  for (int i = 0; i < N2 + 1; ++i)
    if (i < j) c = c * (N2 + 1 - i) / (i + 1);
  return c;
}

// One thread per output sample.  KK = K, the table's neighbours per row, so
// the neighbour loop unrolls; g holds zeros for the adaptive step's whole
// reach before the signal, so no read needs a bounds check.
template <int L, int N2, int KK>
__global__ void __launch_bounds__(256) mesh1d_kernel(const Line1dView v, const uint64_t* __restrict__ g,
                                                     const float* __restrict__ a, size_t a_pitch, void* s,
                                                     size_t s_pitch, uint64_t* num, size_t num_pitch,
                                                     int32_t* status) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y;
  if (m >= v.length) return;
  const float av = reinterpret_cast<const float*>(reinterpret_cast<const char*>(a) + (size_t)row * a_pitch)[m];
  // a 2^Q is exact in binary32 (a power-of-two scaling), so its rint there is
  // the binary64 rint of the same value; this keeps the per-sample work off
  // the binary64 pipe, a thirty-second of the integer rate on GB300
  const float x = av * (float)(1 << v.Q);
  int ok = 1;
  long long A = 0;
  if (!(x > 0.0f) || !(x < 2147483648.0f)) {
    ok = 0;
  } else {
    A = __float2ll_rn(x);
    if (A < 1 || A > v.Amax) ok = 0;
  }
  if (ok) {
    const float lb = v.log2_base + (float)(N2 + 1) * (__log2f((float)A) - (float)v.Q) + 0.05f;
    if (!(lb < 64.0f * L - 1.0f)) ok = 2;
  }
  const bool f64 = v.out_dtype == ABF_F64;
  if (ok != 1) {
    raise_status(status, ok == 0 ? ABF_DEV_BAD_SCALE : ABF_DEV_RANGE);
    if (s) {
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      char* srow = reinterpret_cast<char*>(s) + (size_t)row * s_pitch;
      if (f64) reinterpret_cast<double*>(srow)[m] = nan;
      else reinterpret_cast<float*>(srow)[m] = (float)nan;
    }
    return;
  }
  const int P = v.P;
  const long long mask = (1ll << P) - 1;
  const long long tauP = (A - (1ll << v.Q)) * (N2 + 1);  // tau in units of 2^-P
  const uint64_t* grow = g + (size_t)row * (size_t)v.Gp * L;
  Wide<L> acc;
  wzero<L>(acc);
#pragma unroll
  for (int j = 0; j < N2 + 2; ++j) {
    const long long Y = ((long long)m << P) + tauP - 2 * A * j;  // y_j in units of 2^-P
    const long long p = Y >> P;
    const int r = (int)(Y & mask);
    const uint64_t* trow = v.table + (size_t)r * KK;
    const uint64_t* gk = grow + (size_t)(p + v.dmin + v.left) * L;
    Wide<L> Fj;
    wzero<L>(Fj);
#pragma unroll
    for (int d = 0; d < KK; ++d) mac64<L>(Fj, wload<L>(gk + (size_t)d * L), __ldg(trow + d));
    Wide<L> t;
    wzero<L>(t);
    wmac<L>(t, Fj, (uint64_t)binom_n2p1<N2>(j));
    if (j & 1) wsub<L>(acc, t);
    else wadd<L>(acc, t);
  }
  if (num) {
    uint64_t* q8 = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(num) + (size_t)row * num_pitch) + (size_t)m * L;
#pragma unroll
    for (int i = 0; i < L; ++i) q8[i] = acc.w[i];
  }
  if (s) {
    double val;
    if (v.rtab) {
      val = wto_double<L>(acc) * __ldg(v.rtab + A);  // R[A] = 2^(Q(n2+1) - F) / (D A^(n2+1))
    } else {
      double den = v.Dd;
#pragma unroll
      for (int e = 0; e < N2 + 1; ++e) den *= (double)A;
      val = ldexp(wto_double<L>(acc), v.Q * (N2 + 1) - v.F) / den;
    }
    char* srow = reinterpret_cast<char*>(s) + (size_t)row * s_pitch;
    if (f64) reinterpret_cast<double*>(srow)[m] = val;
    else reinterpret_cast<float*>(srow)[m] = (float)val;
  }
}

template <int L, int N2, int KK>
static cudaError_t launch_mesh1d_K(const Line1dView& v, const uint64_t* g, const float* a, size_t a_pitch, void* s,
                                   size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status,
                                   cudaStream_t st) {
  dim3 grid((v.length + 255) / 256, v.count);
  mesh1d_kernel<L, N2, KK><<<grid, 256, 0, st>>>(v, g, a, a_pitch, s, s_pitch, num, num_pitch, status);
  return cudaGetLastError();
}

// K = N + 1 (N odd) or N + 2 (N even), N = n1 + n2 + 1 with n1 in 0..5: the
// pairs (n2, K) that occur.
template <int L>
static cudaError_t launch_mesh1d_L(const Line1dView& v, const uint64_t* g, const float* a, size_t a_pitch, void* s,
                                   size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status,
                                   cudaStream_t st) {
#define ABF_MESH1D(N2, KK) \
  if (v.n2 == N2 && v.K == KK) return launch_mesh1d_K<L, N2, KK>(v, g, a, a_pitch, s, s_pitch, num, num_pitch, status, st)
  ABF_MESH1D(0, 2); ABF_MESH1D(0, 4); ABF_MESH1D(0, 6); ABF_MESH1D(0, 8);
  ABF_MESH1D(1, 4); ABF_MESH1D(1, 6); ABF_MESH1D(1, 8);
  ABF_MESH1D(2, 4); ABF_MESH1D(2, 6); ABF_MESH1D(2, 8); ABF_MESH1D(2, 10);
  ABF_MESH1D(3, 6); ABF_MESH1D(3, 8); ABF_MESH1D(3, 10);
#undef ABF_MESH1D
  return cudaErrorInvalidValue;
}

static cudaError_t run_mesh1d(const Line1dView& v, const uint64_t* g, const float* a, size_t a_pitch, void* s,
                              size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status, cudaStream_t st) {
  switch (v.limbs) {
    case 1: return launch_mesh1d_L<1>(v, g, a, a_pitch, s, s_pitch, num, num_pitch, status, st);
    case 2: return launch_mesh1d_L<2>(v, g, a, a_pitch, s, s_pitch, num, num_pitch, status, st);
    case 3: return launch_mesh1d_L<3>(v, g, a, a_pitch, s, s_pitch, num, num_pitch, status, st);
    default: return launch_mesh1d_L<4>(v, g, a, a_pitch, s, s_pitch, num, num_pitch, status, st);
  }
}

// ----------------------------------------- interpolation prefilter (n1 >= 2)
// c = f * (b^{n1})^-1 (Sec. 3).  The inverse of the symmetric B-spline
// interpolation filter is, by partial fractions over the poles z_p in (-1, 0)
// of its symbol (one for n1 = 2, 3, two for n1 = 4, 5), a sum of two-sided
// exponentials h[k] = sum_p A_p z_p^|k|, so
//   c[k] = sum_p A_p (y+_p[k] + y-_p[k] - x[k]),
//   y+_p[k] = x[k] + z_p y+_p[k-1]  (causal),  y-_p[k] = x[k] + z_p y-_p[k+1]  (anti-causal),
// with x = f 2^F zero outside the signal.  The exact form takes c on the 2^-F
// grid, c_q = rint(c 2^F) (ties to even), so the recursions need only a bounded
// error below that grid: they run in 64-bit fixed point with G guard bits
// (x 2^G; z_p as rint(z_p 2^64) through the high half of a signed 64 x 64
// product; A_p as rint(A_p 2^60)), on the integer pipe rather than the binary64
// one (a thirty-second of the integer multiply-add rate on GB300).  A thread
// owns kPfSeg consecutive outputs and starts each recursion W_p samples early
// from a zero state (|z_p|^W_p 2^63 < 1/8 unit); the CTA stages its tile of x
// with both halos in shared memory (one pad word per 32 keeps the threads'
// strided reads off a common bank) and stores c_q through it, coalesced.
constexpr int kPfThreads = 128;
constexpr int kPfSeg = 32;                          // outputs per thread
constexpr int kPfTile = kPfThreads * kPfSeg;        // outputs per CTA
constexpr int kPfStage = kPfTile + 2 * kPfHalo;     // staged samples
constexpr int kPfSmem = kPfStage + kPfStage / 32 + 1;

__device__ __forceinline__ int pf_pad(int j) { return j + (j >> 5); }

// ROUND = false (the first, row-wise pass of the 2-D model's separable
// prefilter): the sums are written as they are, c 2^(F + G - 4), for the
// column pass to continue from.
template <typename TIn, typename TOut, bool ROUND = true>
__global__ void __launch_bounds__(kPfThreads, 3) prefilter_kernel(const PrefilterView v, const TIn* __restrict__ f,
                                                                  size_t f_pitch, TOut* __restrict__ c,
                                                                  long long c_pitch, int32_t* status) {
  __shared__ long long sx[kPfSmem];  // x 2^G
  const int row = blockIdx.y;
  const long long i0 = (long long)blockIdx.x * kPfTile;  // first output (g index; k = i - left)
  const TIn* frow = reinterpret_cast<const TIn*>(reinterpret_cast<const char*>(f) + (size_t)row * f_pitch);
  const long long one = 1ll << v.G;
  for (int j = threadIdx.x; j < kPfStage; j += kPfThreads) {
    const long long k = i0 - kPfHalo + j - v.left;
    long long xv = 0;
    if (k >= 0 && k < v.length) xv = convert_f<TIn>(frow[k], v.scale, v.bound, status);
    sx[pf_pad(j)] = xv * one;
  }
  __syncthreads();
  long long acc[kPfSeg];  // c 2^F in units of 2^-(G-4)
#pragma unroll
  for (int e = 0; e < kPfSeg; ++e) acc[e] = 0;
  const int jb = kPfHalo + threadIdx.x * kPfSeg;
#pragma unroll
  for (int p = 0; p < kPfMaxPoles; ++p) {
    if (p >= v.npoles) break;
    const long long Z = v.Z[p], A = v.A[p];
    const int W = v.W[p];
    // the causal and the anti-causal recursion advance together: two
    // independent dependency chains per thread
    long long yf = 0, yb = 0;
    for (int i = 0; i < W; ++i) {
      yf = sx[pf_pad(jb - W + i)] + __mul64hi(yf, Z);
      yb = sx[pf_pad(jb + kPfSeg - 1 + W - i)] + __mul64hi(yb, Z);
    }
#pragma unroll
    for (int i = 0; i < kPfSeg; ++i) {
      const long long xf = sx[pf_pad(jb + i)];
      yf = xf + __mul64hi(yf, Z);
      acc[i] += __mul64hi(yf - xf, A);
      yb = sx[pf_pad(jb + kPfSeg - 1 - i)] + __mul64hi(yb, Z);
      acc[kPfSeg - 1 - i] += __mul64hi(yb, A);
    }
  }
  __syncthreads();  // every thread is done with x
  const int sh = v.G - 4;
  const long long half = 1ll << (sh - 1);
#pragma unroll
  for (int e = 0; e < kPfSeg; ++e) {
    long long q = acc[e];
    if (ROUND) {
      q = acc[e] >> sh;  // floor
      const long long r = acc[e] - q * (1ll << sh);
      if (r > half || (r == half && (q & 1))) ++q;
    }
    sx[pf_pad(threadIdx.x * kPfSeg + e)] = q;
  }
  __syncthreads();
  TOut* crow = c + (size_t)row * (size_t)c_pitch;
  for (int j = threadIdx.x; j < kPfTile; j += kPfThreads) {
    const long long i = i0 + j;
    if (i < v.Gw) crow[i] = (TOut)sx[pf_pad(j)];
  }
}

template <typename TIn>
static cudaError_t launch_prefilter_in(const PrefilterView& v, int count, const void* f, size_t f_pitch,
                                       void* c, long long c_pitch, bool wide, int32_t* status, cudaStream_t st) {
  dim3 grid((unsigned)((v.Gw + kPfTile - 1) / kPfTile), (unsigned)count);
  if (wide)
    prefilter_kernel<TIn, long long><<<grid, kPfThreads, 0, st>>>(v, (const TIn*)f, f_pitch, (long long*)c, c_pitch,
                                                                  status);
  else
    prefilter_kernel<TIn, int32_t><<<grid, kPfThreads, 0, st>>>(v, (const TIn*)f, f_pitch, (int32_t*)c, c_pitch,
                                                                status);
  return cudaGetLastError();
}

// The row-wise first pass of the 2-D model's prefilter: unrounded sums
// c_row 2^(F + G - 4) as int64, rows of v.Gw elements (pitch c_pitch elements).
template <typename TIn>
static cudaError_t launch_prefilter_raw(const PrefilterView& v, int count, const void* f, size_t f_pitch,
                                        long long* c, long long c_pitch, int32_t* status, cudaStream_t st) {
  dim3 grid((unsigned)((v.Gw + kPfTile - 1) / kPfTile), (unsigned)count);
  prefilter_kernel<TIn, long long, false><<<grid, kPfThreads, 0, st>>>(v, (const TIn*)f, f_pitch, c, c_pitch, status);
  return cudaGetLastError();
}

cudaError_t run_prefilter_rows_raw(const PrefilterView& v, int count, int in_dtype, const void* f, size_t f_pitch,
                                   long long* c, long long c_pitch, int32_t* status, cudaStream_t st) {
  switch (in_dtype) {
    case ABF_U8: return launch_prefilter_raw<uint8_t>(v, count, f, f_pitch, c, c_pitch, status, st);
    case ABF_U16: return launch_prefilter_raw<uint16_t>(v, count, f, f_pitch, c, c_pitch, status, st);
    case ABF_F32: return launch_prefilter_raw<float>(v, count, f, f_pitch, c, c_pitch, status, st);
    default: return launch_prefilter_raw<double>(v, count, f, f_pitch, c, c_pitch, status, st);
  }
}

static cudaError_t run_prefilter(const PrefilterView& v, int count, int in_dtype, const void* f, size_t f_pitch,
                                 void* c, long long c_pitch, bool wide, int32_t* status, cudaStream_t st) {
  switch (in_dtype) {
    case ABF_U8: return launch_prefilter_in<uint8_t>(v, count, f, f_pitch, c, c_pitch, wide, status, st);
    case ABF_U16: return launch_prefilter_in<uint16_t>(v, count, f, f_pitch, c, c_pitch, wide, status, st);
    case ABF_F32: return launch_prefilter_in<float>(v, count, f, f_pitch, c, c_pitch, wide, status, st);
    default: return launch_prefilter_in<double>(v, count, f, f_pitch, c, c_pitch, wide, status, st);
  }
}

}  // namespace abf

using i128 = __int128;

// D beta^N(R 2^-P - d) for R in [0, 2^P) and d = dmin .. dmin + K - 1, by the
// degree recurrence in integers: with B_n(X) = n! 2^(n P) beta^n(X 2^-P),
//   B_0(X) = 1 on (-2^(P-1), 2^(P-1)]  (beta^0 of Sec. 2),
//   B_n(X) = (X + (n+1) 2^(P-1)) B_{n-1}(X + 2^(P-1)) + ((n+1) 2^(P-1) - X) B_{n-1}(X - 2^(P-1)).
static bool build_table_1d(int N, int P, int K, int dmin, std::vector<uint64_t>& out, unsigned long long* D) {
  const long long h = 1ll << (P - 1);
  // B_n tabulated on X in [-(N+1) h - h, (N+1) h + h]
  const long long lo = -(N + 2) * h, hi = (N + 2) * h;
  const size_t span = (size_t)(hi - lo + 1);
  std::vector<i128> prev(span, 0), cur(span, 0);
  for (long long X = lo; X <= hi; ++X) prev[(size_t)(X - lo)] = (X > -h && X <= h) ? 1 : 0;
  for (int n = 1; n <= N; ++n) {
    for (long long X = lo; X <= hi; ++X) {
      const long long Xa = X + h, Xb = X - h;
      const i128 ba = (Xa >= lo && Xa <= hi) ? prev[(size_t)(Xa - lo)] : 0;
      const i128 bb = (Xb >= lo && Xb <= hi) ? prev[(size_t)(Xb - lo)] : 0;
      cur[(size_t)(X - lo)] = (i128)(X + (n + 1) * h) * ba + (i128)((n + 1) * h - X) * bb;
    }
    prev.swap(cur);
  }
  i128 Dv = 1;
  for (int i = 2; i <= N; ++i) Dv *= i;
  Dv <<= (N * P);
  if (Dv >= ((i128)1 << 63)) return false;
  const long long rows = 1ll << P;
  out.assign((size_t)rows * K, 0);
  for (long long R = 0; R < rows; ++R) {
    i128 sum = 0;
    for (int c = 0; c < K; ++c) {
      const long long X = R - (long long)(dmin + c) * (1ll << P);
      const i128 w = (X >= lo && X <= hi) ? prev[(size_t)(X - lo)] : 0;
      if (w < 0) return false;
      out[(size_t)R * K + c] = (uint64_t)w;
      sum += w;
    }
    if (sum != Dv) return false;  // partition of unity, and no weight outside the K neighbours
  }
  *D = (unsigned long long)Dv;
  return true;
}

// Neighbours d with beta^N(r - d) != 0 for some r in [0, 1): -(N+1)/2 < d < (N+3)/2.
static void table_shape(int N, int* dmin, int* K) {
  *dmin = (N % 2) ? -(N + 1) / 2 + 1 : -N / 2;
  *K = (N % 2) ? N + 1 : N + 2;
}

// Poles z_p and partial-fraction weights A_p of (b^{n1})^-1, n1 = 2..5:
// h[k] = sum_p A_p z_p^|k|.  With w = q + 1/q the symbol
// b_0 + sum_{k>=1} b_k (q^k + q^-k) is a polynomial of degree M = n1/2 in w
// (q^2 + q^-2 = w^2 - 2); each root w_p < -2 gives z_p + 1/z_p = w_p, and
// 1/(w - w_p) = -z_p / ((1 - z_p q^-1)(1 - z_p q)) expands to
// -z_p / (1 - z_p^2) sum_k z_p^|k| q^k.
struct PoleSet {
  int M;
  double z[2], A[2];
  double hnorm;  // sum_p |A_p| (1 + |z_p|) / (1 - |z_p|) >= ||h||_1
};

static bool interp_poles(int n1, PoleSet& ps) {
  if (n1 < 2 || n1 > 5) return false;
  // b^{n1}[k] = beta^{n1}(k) from the degree recurrence at P = 1 (row r = 0)
  int dmin = 0, K = 0;
  table_shape(n1, &dmin, &K);
  std::vector<uint64_t> t;
  unsigned long long D = 0;
  if (!build_table_1d(n1, 1, K, dmin, t, &D)) return false;
  double b[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k <= n1 / 2; ++k) b[k] = (double)t[(size_t)(-k - dmin)] / (double)D;  // beta(k) = beta(-k)
  ps.M = n1 / 2;
  double w[2];
  if (ps.M == 1) {
    w[0] = -b[0] / b[1];
  } else {
    const double disc = b[1] * b[1] - 4.0 * b[2] * (b[0] - 2.0 * b[2]);
    if (!(disc > 0.0)) return false;
    const double q = -0.5 * (b[1] + std::sqrt(disc));  // b[1] > 0: no cancellation
    w[0] = (b[0] - 2.0 * b[2]) / q;
    w[1] = q / b[2];
  }
  ps.hnorm = 0.0;
  for (int p = 0; p < ps.M; ++p) {
    if (!(w[p] < -2.0)) return false;
    ps.z[p] = 2.0 / (w[p] - std::sqrt(w[p] * w[p] - 4.0));  // the root inside (-1, 0), no cancellation
    const double res = -ps.z[p] / (1.0 - ps.z[p] * ps.z[p]);
    if (ps.M == 1) ps.A[p] = res / b[1];
    else ps.A[p] = (p == 0 ? 1.0 : -1.0) * res / (b[2] * (w[0] - w[1]));
    const double az = std::fabs(ps.z[p]);
    ps.hnorm += std::fabs(ps.A[p]) * (1.0 + az) / (1.0 - az);
  }
  return true;
}

namespace abf {
// Constants of the 2-D model's separable prefilter (degree n1 in 2..5; the
// same recursions as the 1-D filter's, run along rows and then along
// columns): poles and weights in 64-bit fixed point, guard bits G for samples
// up to xmax = |f|max 2^F, and the tail T of coefficients kept beyond each
// image edge (beyond it |c| 2^F < 1/4, counting the other axis' gain hnorm).
abf_status prefilter2d_setup(int n1, double xmax, PrefilterView* pf, double* hnorm, int* tail) {
  PoleSet ps{};
  if (!interp_poles(n1, ps)) return ABF_ERR_UNSUPPORTED;
  double zmax = 0.0;
  for (int q = 0; q < ps.M; ++q) zmax = std::max(zmax, std::fabs(ps.z[q]));
  const double x2 = xmax * ps.hnorm;  // the column pass' input bound
  const int G = (int)std::floor(61.0 - std::log2(std::max(xmax, x2) * (2.0 / (1.0 - zmax) + 1.0)));
  if (G < 24) return ABF_ERR_RANGE;
  *pf = PrefilterView{};
  pf->G = std::min(G, 40);
  pf->npoles = ps.M;
  for (int q = 0; q < ps.M; ++q) {
    const double az = std::fabs(ps.z[q]);
    pf->W[q] = std::min(kPfHalo, (int)std::ceil(66.0 / -std::log2(az)));
    pf->Z[q] = std::llrint(std::ldexp(ps.z[q], 64));
    pf->A[q] = std::llrint(std::ldexp(ps.A[q], 60));
    if (!(std::fabs(ps.A[q]) < 7.0)) return ABF_ERR_UNSUPPORTED;
  }
  int T = 0;
  for (; T < 4096; ++T) {
    double t = 0.0;
    for (int q = 0; q < ps.M; ++q) {
      const double az = std::fabs(ps.z[q]);
      t += std::fabs(ps.A[q]) * std::pow(az, T + 1) / (1.0 - az);
    }
    if (x2 * t < 0.25) break;
  }
  *hnorm = ps.hnorm;
  *tail = T;
  return ABF_OK;
}
}  // namespace abf

struct abf1d_plan_s {
  abf1d_desc desc;
  abf::Line1dView v;
  abf::PlanView rows;   // the row pass over the extended signals
  abf::PrefilterView pf;
  uint64_t* d_table = nullptr;
  int32_t* d_status = nullptr;
  void* d_stage = nullptr;   // n1 >= 2: c_q per row (int32 or int64, g's pitch)
  double* d_rtab = nullptr;  // normalisation per integer scale
  bool stage_wide = false;
  size_t g_bytes = 0;
  int right = 0;
};

extern "C" {

abf_status abf1d_plan_create(const abf1d_desc* d, abf1d_plan* out) {
  if (!d || !out) return ABF_ERR_INVALID;
  *out = nullptr;
  if (d->length < 1 || d->count < 1 || d->count > 65535) return ABF_ERR_INVALID;
  if (d->n1 < 0 || d->n2 < 0 || d->n2 > 3) return ABF_ERR_INVALID;
  if (d->n1 > 5) return ABF_ERR_UNSUPPORTED;
  if (d->in_dtype < ABF_U8 || d->in_dtype > ABF_F64) return ABF_ERR_INVALID;
  if (d->out_dtype != ABF_F32 && d->out_dtype != ABF_F64) return ABF_ERR_INVALID;
  if (d->q_bits < 1 || d->q_bits > 10 || d->in_frac_bits < 0 || d->in_frac_bits > 40) return ABF_ERR_INVALID;
  const double qd = std::ldexp(1.0, d->q_bits);
  if (!(d->max_scale > 0) || !(d->max_scale * qd < 1e9)) return ABF_ERR_INVALID;
  const int Amax = (int)std::lrint(d->max_scale * qd);
  if (Amax < 1) return ABF_ERR_INVALID;
  double vb = d->value_bound;
  if (!(vb > 0)) {
    if (d->in_dtype == ABF_U8) vb = 255.0;
    else if (d->in_dtype == ABF_U16) vb = 65535.0;
    else return ABF_ERR_INVALID;
  }
  const int N = d->n1 + d->n2 + 1, P = d->q_bits + 1;
  int dmin = 0, K = 0;
  table_shape(N, &dmin, &K);
  std::vector<uint64_t> tab;
  unsigned long long D = 0;
  try {
    if (!build_table_1d(N, P, K, dmin, tab, &D)) return ABF_ERR_UNSUPPORTED;
  } catch (const std::bad_alloc&) {
    return ABF_ERR_OOM;
  }
  // Model coefficients: c = f (n1 <= 1) or c = f * (b^{n1})^-1 rounded to the
  // 2^-F grid, |c_q| <= hnorm |f|max + 2^-(F+1).
  const double xmax = std::ldexp(vb, d->in_frac_bits);  // bound on |f 2^F|
  PoleSet ps{};
  abf::PrefilterView pf{};
  double cmax = vb;
  int left = 0;
  bool wide = false;
  if (d->n1 >= 2) {
    if (!interp_poles(d->n1, ps)) return ABF_ERR_UNSUPPORTED;
    double zmax = 0.0;
    for (int q = 0; q < ps.M; ++q) zmax = std::max(zmax, std::fabs(ps.z[q]));
    // guard bits: |x 2^G|, |y+ 2^G|, |y- 2^G| and their combination stay below 2^61
    const int G = (int)std::floor(61.0 - std::log2(xmax * (2.0 / (1.0 - zmax) + 1.0)));
    if (G < 24) return ABF_ERR_RANGE;
    pf.G = std::min(G, 40);
    pf.npoles = ps.M;
    for (int q = 0; q < ps.M; ++q) {
      const double az = std::fabs(ps.z[q]);
      pf.W[q] = std::min(abf::kPfHalo, (int)std::ceil(66.0 / -std::log2(az)));
      pf.Z[q] = std::llrint(std::ldexp(ps.z[q], 64));
      pf.A[q] = std::llrint(std::ldexp(ps.A[q], 60));
      if (!(std::fabs(ps.A[q]) < 7.0)) return ABF_ERR_UNSUPPORTED;
    }
    // left tail: for k <= -(left+1), |c[k]| <= xmax sum_p |A_p| |z_p|^(left+1) / (1 - |z_p|) < 1/4
    for (left = 0; left < 4096; ++left) {
      double t = 0.0;
      for (int q = 0; q < ps.M; ++q) {
        const double az = std::fabs(ps.z[q]);
        t += std::fabs(ps.A[q]) * std::pow(az, left + 1) / (1.0 - az);
      }
      if (xmax * t < 0.25) break;
    }
    cmax = ps.hnorm * vb + std::ldexp(1.0, -d->in_frac_bits);
    wide = !(ps.hnorm * xmax + 1.0 < 2147483647.0);
  }
  // |s| <= |c|max (non-negative kernel, unit lattice sum), so
  // |S| <= D max_scale^(n2+1) |c|max 2^F.
  const double lb = std::log2((double)D) + (d->n2 + 1) * std::log2((double)Amax / qd) + std::log2(cmax) +
                    d->in_frac_bits + 1e-6;
  const int L = (int)std::floor((lb + 1.0) / 64.0) + 1;
  if (L > abf::kMaxLimbs) return ABF_ERR_RANGE;
  abf1d_plan p = new (std::nothrow) abf1d_plan_s();
  if (!p) return ABF_ERR_OOM;
  p->desc = *d;
  // samples past the end read by the adaptive step: tau_max + (N+1)/2, plus margin
  const double tau_max = std::max(0.0, ((double)Amax / qd - 1.0) * (d->n2 + 1) / 2.0);
  p->right = (int)std::ceil(tau_max + (N + 1) / 2.0) + 2;
  abf::Line1dView& v = p->v;
  v.length = d->length; v.count = d->count; v.n1 = d->n1; v.n2 = d->n2; v.N = N; v.Q = d->q_bits; v.P = P;
  v.F = d->in_frac_bits; v.K = K; v.dmin = dmin; v.Amax = Amax; v.limbs = L; v.out_dtype = d->out_dtype;
  // g keeps zeros before the signal for the adaptive step's reach there
  // (y_j >= -(a + 1)(n2 + 1)/2 >= -(tau_max + n2 + 1), and (N+1)/2 + 1 more
  // for the B-spline's neighbours), so its reads need no bounds check
  left = std::max(left, (int)std::ceil(tau_max + (d->n2 + 1) + (N + 1) / 2.0) + 2);
  v.left = left;
  v.log2_base = (float)(std::log2((double)D) + std::log2(cmax) + d->in_frac_bits);
  v.Dd = (double)D;
  const long long Gw = (long long)left + d->length + p->right;
  if (Gw >= (1ll << 31)) {
    delete p;
    return ABF_ERR_INVALID;
  }
  v.Gp = (Gw + 3) / 4 * 4;
  abf::PlanView& r = p->rows;
  r = abf::PlanView{};
  r.H = d->count; r.n = d->n2 + 1; r.Q = d->q_bits; r.P = P; r.F = d->in_frac_bits;
  r.r[0] = d->n2 + 1;  // the row pass: n2 + 1 cascaded sums
  r.above = 0; r.Gw = (int)Gw; r.Gh = d->count; r.Gp = v.Gp;
  r.out_dtype = d->out_dtype; r.limbs = L; r.value_bound = vb;
  if (d->n1 >= 2) {
    // the row pass reads the staged c_q: the whole extended row is its input
    r.W = (int)Gw; r.left = 0; r.right = 0;
    r.in_dtype = wide ? abf::kStageI64 : abf::kStageI32;
    pf.length = d->length; pf.Gw = (int)Gw; pf.left = left;
    pf.scale = std::ldexp(1.0, d->in_frac_bits);
    const double bd = std::floor(xmax);
    pf.bound = bd < 4.0e18 ? (long long)bd : 4000000000000000000ll;
    p->pf = pf;
    p->stage_wide = wide;
  } else {
    r.W = d->length; r.left = left; r.right = p->right;
    r.in_dtype = d->in_dtype;
  }
  p->g_bytes = (size_t)v.Gp * (size_t)d->count * (size_t)L * 8;
  if (cudaMalloc(&p->d_table, tab.size() * sizeof(uint64_t)) != cudaSuccess) {
    delete p;
    return ABF_ERR_OOM;
  }
  if (d->n1 >= 2 &&
      cudaMalloc(&p->d_stage, (size_t)v.Gp * (size_t)d->count * (wide ? 8 : 4)) != cudaSuccess) {
    cudaFree(p->d_table);
    delete p;
    return ABF_ERR_OOM;
  }
  if (cudaMemcpy(p->d_table, tab.data(), tab.size() * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMalloc(&p->d_status, sizeof(int32_t)) != cudaSuccess) {
    cudaFree(p->d_table);
    if (p->d_stage) cudaFree(p->d_stage);
    delete p;
    return ABF_ERR_CUDA;
  }
  if (cudaMemset(p->d_status, 0, sizeof(int32_t)) != cudaSuccess) {
    cudaFree(p->d_table);
    cudaFree(p->d_status);
    if (p->d_stage) cudaFree(p->d_stage);
    delete p;
    return ABF_ERR_CUDA;
  }
  v.table = p->d_table;
  v.rtab = nullptr;
  if (Amax <= (1 << 22)) {
    // the normalisation per integer scale, in the kernel's former operation order
    std::vector<double> rt((size_t)Amax + 1, 0.0);
    const double e2 = std::ldexp(1.0, d->q_bits * (d->n2 + 1) - d->in_frac_bits);
    for (int A = 1; A <= Amax; ++A) {
      double den = (double)D;
      for (int e = 0; e < d->n2 + 1; ++e) den *= (double)A;
      rt[(size_t)A] = e2 / den;
    }
    double* d_rt = nullptr;
    if (cudaMalloc(&d_rt, rt.size() * sizeof(double)) != cudaSuccess) {
      abf1d_plan_destroy(p);
      return ABF_ERR_OOM;
    }
    p->d_rtab = d_rt;
    if (cudaMemcpy(d_rt, rt.data(), rt.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
      abf1d_plan_destroy(p);
      return ABF_ERR_CUDA;
    }
    v.rtab = d_rt;
  }
  *out = p;
  return ABF_OK;
}

abf_status abf1d_plan_destroy(abf1d_plan p) {
  if (!p) return ABF_ERR_INVALID;
  if (p->d_table) cudaFree(p->d_table);
  if (p->d_status) cudaFree(p->d_status);
  if (p->d_stage) cudaFree(p->d_stage);
  if (p->d_rtab) cudaFree(p->d_rtab);
  delete p;
  return ABF_OK;
}

abf_status abf1d_plan_query(abf1d_plan p, size_t* integrated_bytes, int32_t* left, int32_t* right, int32_t* limbs,
                            int64_t* g_pitch_elems) {
  if (!p) return ABF_ERR_INVALID;
  if (integrated_bytes) *integrated_bytes = p->g_bytes;
  if (left) *left = p->v.left;
  if (right) *right = p->right;
  if (limbs) *limbs = p->v.limbs;
  if (g_pitch_elems) *g_pitch_elems = p->v.Gp;
  return ABF_OK;
}

abf_status abf1d_integrate(abf1d_plan p, const void* d_f, size_t f_pitch, void* d_g, cudaStream_t st) {
  if (!p || !d_f || !d_g) return ABF_ERR_INVALID;
  const int dt = p->desc.in_dtype;
  const size_t esz = dt == ABF_U8 ? 1 : dt == ABF_U16 ? 2 : dt == ABF_F32 ? 4 : 8;
  if (f_pitch < (size_t)p->desc.length * esz || ((uintptr_t)d_g & 15)) return ABF_ERR_INVALID;
  if (p->d_stage) {
    const size_t esz_c = p->stage_wide ? 8 : 4;
    if (abf::run_prefilter(p->pf, p->desc.count, dt, d_f, f_pitch, p->d_stage, p->v.Gp, p->stage_wide, p->d_status,
                           st) != cudaSuccess)
      return ABF_ERR_CUDA;
    return abf::run_row_scan(p->rows, p->d_stage, (size_t)p->v.Gp * esz_c, (uint64_t*)d_g, p->d_status, st) ==
                   cudaSuccess
               ? ABF_OK
               : ABF_ERR_CUDA;
  }
  return abf::run_row_scan(p->rows, d_f, f_pitch, (uint64_t*)d_g, p->d_status, st) == cudaSuccess ? ABF_OK
                                                                                                   : ABF_ERR_CUDA;
}

static abf_status filter1d(abf1d_plan p, const void* d_g, const float* d_a, size_t a_pitch, void* d_s,
                           size_t s_pitch, void* d_num, size_t num_pitch, cudaStream_t st) {
  if (!p || !d_g || !d_a || (!d_s && !d_num)) return ABF_ERR_INVALID;
  if (a_pitch < (size_t)p->desc.length * sizeof(float) || ((uintptr_t)d_g & 15)) return ABF_ERR_INVALID;
  if (d_s && s_pitch < (size_t)p->desc.length * (p->desc.out_dtype == ABF_F64 ? 8 : 4)) return ABF_ERR_INVALID;
  if (d_num && num_pitch < (size_t)p->desc.length * 8 * p->v.limbs) return ABF_ERR_INVALID;
  return abf::run_mesh1d(p->v, (const uint64_t*)d_g, d_a, a_pitch, d_s, s_pitch, (uint64_t*)d_num, num_pitch,
                         p->d_status, st) == cudaSuccess
             ? ABF_OK
             : ABF_ERR_CUDA;
}

abf_status abf1d_filter(abf1d_plan p, const void* d_g, const float* d_a, size_t a_pitch, void* d_s, size_t s_pitch,
                        cudaStream_t st) {
  if (!d_s) return ABF_ERR_INVALID;
  return filter1d(p, d_g, d_a, a_pitch, d_s, s_pitch, nullptr, 0, st);
}

abf_status abf1d_filter_numerator(abf1d_plan p, const void* d_g, const float* d_a, size_t a_pitch, void* d_num,
                                  size_t num_pitch, cudaStream_t st) {
  if (!d_num) return ABF_ERR_INVALID;
  return filter1d(p, d_g, d_a, a_pitch, nullptr, 0, d_num, num_pitch, st);
}

abf_status abf1d_weight_table_host(int32_t n1, int32_t n2, int32_t q_bits, uint64_t* out, size_t out_elems,
                                   size_t* needed_elems, int32_t* K, int32_t* dmin, uint64_t* D) {
  if (n1 < 0 || n1 > 5 || n2 < 0 || n2 > 3 || q_bits < 1 || q_bits > 10) return ABF_ERR_INVALID;
  const int N = n1 + n2 + 1, P = q_bits + 1;
  int dm = 0, k = 0;
  table_shape(N, &dm, &k);
  std::vector<uint64_t> tab;
  unsigned long long Dv = 0;
  try {
    if (!build_table_1d(N, P, k, dm, tab, &Dv)) return ABF_ERR_UNSUPPORTED;
  } catch (const std::bad_alloc&) {
    return ABF_ERR_OOM;
  }
  if (needed_elems) *needed_elems = tab.size();
  if (K) *K = k;
  if (dmin) *dmin = dm;
  if (D) *D = Dv;
  if (out) {
    if (out_elems < tab.size()) return ABF_ERR_INVALID;
    std::copy(tab.begin(), tab.end(), out);
  }
  return ABF_OK;
}

abf_status abf1d_prefilter_host(int32_t n1, int32_t* npoles, double* z, double* A, double* hnorm) {
  if (n1 < 2 || n1 > 5 || !npoles || !z || !A) return ABF_ERR_INVALID;
  PoleSet ps{};
  if (!interp_poles(n1, ps)) return ABF_ERR_UNSUPPORTED;
  *npoles = ps.M;
  for (int p = 0; p < ps.M; ++p) {
    z[p] = ps.z[p];
    A[p] = ps.A[p];
  }
  if (hnorm) *hnorm = ps.hnorm;
  return ABF_OK;
}

abf_status abf1d_last_device_status(abf1d_plan p, int32_t* code) {
  if (!p || !code) return ABF_ERR_INVALID;
  if (cudaDeviceSynchronize() != cudaSuccess) return ABF_ERR_CUDA;
  int32_t val = 0;
  if (cudaMemcpy(&val, p->d_status, sizeof(val), cudaMemcpyDeviceToHost) != cudaSuccess) return ABF_ERR_CUDA;
  if (cudaMemset(p->d_status, 0, sizeof(int32_t)) != cudaSuccess) return ABF_ERR_CUDA;
  *code = val;
  return ABF_OK;
}

}  // extern "C"
