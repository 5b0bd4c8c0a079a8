// Floating-point forms of the filter: per-tile restart windows in pair
// arithmetic (an unevaluated sum hi + lo of two binary64, or of two binary32,
// numbers), with an a-priori error bound checked at every pixel.
//
// The non-adaptive step of Sec. 7 (1) is run not on the whole image but on a
// window around each output tile: the window holds every lattice point the
// tile's mesh reads, so it holds the support of every tile pixel's kernel, and
// filtering f restricted to the window gives the same result at the tile's
// pixels (the filter is linear; the kernel has compact support, Sec. 4).  The
// window keeps the running sums small: their size grows like the window extent
// to the power 4n.  Inside a window the recursions run in the paper's order
// (0, pi/4, pi/2, 3pi/4) with zero input outside the window; the last one
// (3pi/4) is cut at the window's right edge, which only changes g by a
// polynomial of degree < n along each 3pi/4 line, and the mesh's FD along v4
// annihilates that.  Then the mesh of Eq. (final_eqn) runs as in the exact
// form: weights D0 ZP^{*n} (the integer table scaled by 2^-k, D = D0 2^k).
//
// Why pairs.  The mesh cancels the running sums (size G) down to the result
// (size |f| prod c^n), so a relative error e in the sums or weights becomes an
// error of about 2^(4n) G e / prod c^n in s.  For an elongated kernel in a
// window that holds its reads that ratio reaches 1e13 (order 2, steps 1 to
// 150), so single binary64 (e = 2^-53) lands near 1e-3 relative to the value
// range, far from 1e-12.  Pairs give e ~ 2^-104 (binary64) or 2^-46 (binary32).
//
// Pair operations (each written here from its published definition): Knuth's
// TwoSum and Dekker's Fast2Sum give the rounding error of an addition exactly;
// TwoProd via a fused multiply-add gives that of a product; the pair sum and
// product are the double-word algorithms of Joldes, Muller and Popescu (2017),
// relative error below 3u^2 and 5u^2 for unit roundoff u.  Every step uses an
// explicitly rounded intrinsic, so no contraction changes them.
//
// Error bound per pixel (checked, never assumed).  With u the unit roundoff of
// the element type, a running sum over a line of length l has error at most
// l 4u^2 times the sum of magnitudes; 4n passes over lines of at most
// max(ww, wh) give gamma_g = 16 n max(ww, wh) u^2.  The mesh sums at most
// TERMS products per lane, then at most 11 group sums and 5 warp levels:
// gamma_m = 4 (TERMS + 20) u^2; the weights are pairs (2 u^2).  The table rows
// sum to D0 and sum_j |w_j| = 2^(4n), so
//     |S - S_exact| <= 2^(4n) D0 Gabs (gamma_g + gamma_m + 2u^2)
// where Gabs bounds |g| computed from |f|: for a window with f >= 0 it is the
// largest computed sum (times 1 + gamma_g), otherwise |f|max times the
// product over the four directions of binom(l_k + n - 1, n) (each n-fold
// running sum over a line of length l_k grows a bounded sequence by at most
// that factor).  s = S 2^(4Qn) / (D0 prod C^n) in binary64.  A pixel whose
// bound exceeds the form's tolerance (times the plan's value bound) gets NaN
// and sets ABF_DEV_PRECISION.
//
// Tiles: the image is cut into 256 x 256 super-tiles, each split as a quadtree
// down to squares of side T in {8, ..., 256}: a square is split while T exceeds
// its smallest step (in pixels) and T > 8.  So a window is about T + 6n c_max
// wide with T <= c_min, which keeps the window-to-step ratio (and with it G)
// small and the redundant scan work per pixel bounded.
//
// Kernels: block_steps_kernel (smallest and largest step per direction over
// each 8 x 8 block), tile_list_kernel (one thread per super-tile walks its
// quadtree and emits tiles with their windows), tile_filter_kernel (persistent
// CTAs take tiles from a counter; each integrates its window into its own
// scratch slot and filters the tile's pixels).
#include "abf_internal.cuh"

namespace abf {

constexpr int kBlk = 8;           // step-bound block
constexpr int kSuper = 256;       // super-tile
constexpr int kTileThreads = 256; // threads per tile CTA
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kSlotsPerSm = 2;    // tile CTAs (scratch slots) per SM

struct TileRec {
  int x0, y0, T;               // tile origin and side (image coordinates)
  int wx0, wy0, ww, wh;        // window box [wx0, wx0 + ww) x [wy0, wy0 + wh)
};

// ------------------------------------------------------------ pair arithmetic

template <typename T>
struct PairT {
  T hi, lo;
};

__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// s + e = a + b exactly (Knuth).
template <typename T>
__device__ __forceinline__ T two_sum(T a, T b, T& e) {
  const T s = rn_add(a, b);
  const T bb = rn_sub(s, a);
  e = rn_add(rn_sub(a, rn_sub(s, bb)), rn_sub(b, bb));
  return s;
}

// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker).
template <typename T>
__device__ __forceinline__ T fast_two_sum(T a, T b, T& e) {
  const T s = rn_add(a, b);
  e = rn_sub(b, rn_sub(s, a));
  return s;
}

template <typename T>
__device__ __forceinline__ PairT<T> pair_add(PairT<T> x, PairT<T> y) {
  T e1, e2, e3;
  const T s = two_sum(x.hi, y.hi, e1);
  const T t = two_sum(x.lo, y.lo, e2);
  e1 = rn_add(e1, t);
  const T v = fast_two_sum(s, e1, e3);
  e3 = rn_add(e3, e2);
  PairT<T> r;
  r.hi = fast_two_sum(v, e3, r.lo);
  return r;
}

template <typename T>
__device__ __forceinline__ PairT<T> pair_neg(PairT<T> x) {
  return PairT<T>{-x.hi, -x.lo};
}

template <typename T>
__device__ __forceinline__ PairT<T> pair_mul(PairT<T> x, PairT<T> y) {
  const T p = rn_mul(x.hi, y.hi);
  T e = rn_fma(x.hi, y.hi, -p);
  T t = rn_mul(x.hi, y.lo);
  t = rn_fma(x.lo, y.hi, t);
  e = rn_add(e, t);
  PairT<T> r;
  r.hi = fast_two_sum(p, e, r.lo);
  return r;
}

// x times a small integer k (|k| <= 81, exact in T).
template <typename T>
__device__ __forceinline__ PairT<T> pair_scale(PairT<T> x, int k) {
  const T kk = (T)k;
  const T p = rn_mul(x.hi, kk);
  T e = rn_fma(x.hi, kk, -p);
  e = rn_fma(x.lo, kk, e);
  PairT<T> r;
  r.hi = fast_two_sum(p, e, r.lo);
  return r;
}

template <typename T>
__device__ __forceinline__ PairT<T> pair_from(double v) {
  PairT<T> r;
  r.hi = (T)v;
  r.lo = (T)(v - (double)r.hi);
  return r;
}

template <typename T>
__device__ __forceinline__ PairT<T> pair_shfl_xor(PairT<T> x, int o) {
  return PairT<T>{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
}

template <typename T>
__device__ __forceinline__ PairT<T> pair_load(const PairT<T>* p) {
  if constexpr (sizeof(T) == 8) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    return PairT<T>{v.x, v.y};
  } else {
    const float2 v = *reinterpret_cast<const float2*>(p);
    return PairT<T>{v.x, v.y};
  }
}

template <typename T>
__device__ __forceinline__ void pair_store(PairT<T>* p, PairT<T> x) {
  if constexpr (sizeof(T) == 8) *reinterpret_cast<double2*>(p) = make_double2(x.hi, x.lo);
  else *reinterpret_cast<float2*>(p) = make_float2(x.hi, x.lo);
}

// ------------------------------------------------------------ tile geometry

// Smallest and largest integer step per direction over each 8 x 8 block
// (invalid pixels are skipped; an all-invalid block gets min = INT_MAX, max = 0).
__global__ void block_steps_kernel(const PlanView pv, const float4* __restrict__ scales, size_t scale_pitch,
                                   int4* __restrict__ bmin, int4* __restrict__ bmax, int32_t* status) {
  const int bx = blockIdx.x, by = blockIdx.y;
  const int i = threadIdx.x;  // 64 threads: one per pixel of the block
  const int x = bx * kBlk + (i % kBlk), y = by * kBlk + (i / kBlk);
  int4 mn = make_int4(INT_MAX, INT_MAX, INT_MAX, INT_MAX), mx = make_int4(0, 0, 0, 0);
  if (x < pv.W && y < pv.H) {
    int C[4];
    if (pixel_steps(pv, scales, scale_pitch, x, y, C)) {
      mn = make_int4(C[0], C[1], C[2], C[3]);
      mx = mn;
    } else {
      raise_status(status, ABF_DEV_BAD_SCALE);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn.x = min(mn.x, __shfl_xor_sync(0xffffffffu, mn.x, o)); mx.x = max(mx.x, __shfl_xor_sync(0xffffffffu, mx.x, o));
    mn.y = min(mn.y, __shfl_xor_sync(0xffffffffu, mn.y, o)); mx.y = max(mx.y, __shfl_xor_sync(0xffffffffu, mx.y, o));
    mn.z = min(mn.z, __shfl_xor_sync(0xffffffffu, mn.z, o)); mx.z = max(mx.z, __shfl_xor_sync(0xffffffffu, mx.z, o));
    mn.w = min(mn.w, __shfl_xor_sync(0xffffffffu, mn.w, o)); mx.w = max(mx.w, __shfl_xor_sync(0xffffffffu, mx.w, o));
  }
  __shared__ int4 smn[2], smx[2];
  if ((i & 31) == 0) { smn[i >> 5] = mn; smx[i >> 5] = mx; }
  __syncthreads();
  if (i == 0) {
    const int4 a = smn[0], b = smn[1], c = smx[0], d = smx[1];
    bmin[by * gridDim.x + bx] = make_int4(min(a.x, b.x), min(a.y, b.y), min(a.z, b.z), min(a.w, b.w));
    bmax[by * gridDim.x + bx] = make_int4(max(c.x, d.x), max(c.y, d.y), max(c.z, d.z), max(c.w, d.w));
  }
}

// Window margins (left, right, below, above) for steps bounded by m (units 2^-Q):
// a pixel's mesh reads [x - E_x - 2n, x + E_x + n] x [y - E_y - 3n, y + E_y],
// E_x = (n/2)(c1 + c2 + c4), E_y = (n/2)(c2 + c3 + c4).
__device__ __forceinline__ void margins(const PlanView& pv, int4 m, int mg[4]) {
  const int n = pv.n;
  const long long ex = (long long)n * (m.x + m.y + m.w);  // 2 E_x 2^Q
  const long long ey = (long long)n * (m.y + m.z + m.w);
  const long long q2 = 2ll << pv.Q;
  const int Ex = (int)((ex + q2 - 1) / q2), Ey = (int)((ey + q2 - 1) / q2);  // ceil(E)
  mg[0] = Ex + 2 * n + 1;
  mg[1] = Ex + n + 1;
  mg[2] = Ey + 3 * n + 1;
  mg[3] = Ey + 1;
}

__global__ void tile_list_kernel(const PlanView pv, const int4* __restrict__ bmin, const int4* __restrict__ bmax,
                                 int bw, int bh, TileRec* __restrict__ tiles, int* __restrict__ ntiles) {
  const int sidx = blockIdx.x * blockDim.x + threadIdx.x;
  const int sw = (pv.W + kSuper - 1) / kSuper, sh = (pv.H + kSuper - 1) / kSuper;
  if (sidx >= sw * sh) return;
  const int sy = sidx / sw, sx = sidx % sw;
  // depth-first over the quadtree of this super-tile
  int stk[4 * 6 + 4][3];
  int sp = 0;
  stk[sp][0] = sx * kSuper; stk[sp][1] = sy * kSuper; stk[sp][2] = kSuper; ++sp;
  while (sp > 0) {
    --sp;
    const int x0 = stk[sp][0], y0 = stk[sp][1], T = stk[sp][2];
    if (x0 >= pv.W || y0 >= pv.H) continue;
    int cmin = INT_MAX;
    int4 m = make_int4(0, 0, 0, 0);
    for (int by = y0 / kBlk; by < min((y0 + T) / kBlk, bh); ++by)
      for (int bx = x0 / kBlk; bx < min((x0 + T) / kBlk, bw); ++bx) {
        const int4 a = bmin[by * bw + bx], v = bmax[by * bw + bx];
        cmin = min(cmin, min(min(a.x, a.y), min(a.z, a.w)));
        m.x = max(m.x, v.x); m.y = max(m.y, v.y); m.z = max(m.z, v.z); m.w = max(m.w, v.w);
      }
    // split while the side exceeds the smallest step (in pixels)
    if (T > kBlk && (long long)T << pv.Q > (long long)cmin) {
      const int h = T / 2;
      stk[sp][0] = x0; stk[sp][1] = y0; stk[sp][2] = h; ++sp;
      stk[sp][0] = x0 + h; stk[sp][1] = y0; stk[sp][2] = h; ++sp;
      stk[sp][0] = x0; stk[sp][1] = y0 + h; stk[sp][2] = h; ++sp;
      stk[sp][0] = x0 + h; stk[sp][1] = y0 + h; stk[sp][2] = h; ++sp;
      continue;
    }
    int tg[4];
    margins(pv, m, tg);
    TileRec rec;
    rec.x0 = x0; rec.y0 = y0; rec.T = T;
    rec.wx0 = x0 - tg[0];
    rec.wy0 = y0 - tg[2];
    rec.ww = min(T, pv.W - x0) + tg[0] + tg[1];
    rec.wh = min(T, pv.H - y0) + tg[2] + tg[3];
    const int k = atomicAdd(ntiles, 1);
    tiles[k] = rec;
  }
}

template <typename TIn>
__device__ __forceinline__ double load_fd(const void* f, size_t pitch, int x, int y) {
  return (double)reinterpret_cast<const TIn*>(reinterpret_cast<const char*>(f) + (size_t)y * pitch)[x];
}

__device__ __forceinline__ double fetch_f(int dtype, const void* f, size_t pitch, int x, int y) {
  switch (dtype) {
    case ABF_U8: return load_fd<uint8_t>(f, pitch, x, y);
    case ABF_U16: return load_fd<uint16_t>(f, pitch, x, y);
    case ABF_F32: return load_fd<float>(f, pitch, x, y);
    default: return load_fd<double>(f, pitch, x, y);
  }
}

template <int N>
__host__ __device__ constexpr int fd_weight(int t) {
  // w_j = prod_i (-1)^{j_i} binom(N, j_i), tap t = j1 + (N+1) j3 + (N+1)^2 j2 + (N+1)^3 j4
  int w = 1;
  for (int i = 0; i < 4; ++i, t /= (N + 1)) {
    const int j = t % (N + 1);
    const int c = (j == 0 || j == N) ? 1 : N;
    w *= (j & 1) ? -c : c;
  }
  return w;
}

// binom(l + n - 1, n) in binary64 (the growth of an n-fold running sum over l terms).
__device__ __forceinline__ double run_growth(int l, int n) {
  double r = 1.0;
  for (int i = 1; i <= n; ++i) r = r * (double)(l + i - 1) / (double)i;
  return r;
}

template <typename T>
__device__ __forceinline__ double unit_roundoff() {
  return sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;  // 2^-53, 2^-24
}

// Integrate one window (in its scratch slot, row pitch ww) and filter the tile.
template <int N, typename T, typename TOut>
__global__ void __launch_bounds__(kTileThreads, kSlotsPerSm) tile_filter_kernel(
    const PlanView pv, const void* __restrict__ f, size_t f_pitch, const float4* __restrict__ scales,
    size_t scale_pitch, void* __restrict__ s, size_t s_pitch, const TileRec* __restrict__ tiles,
    const int* __restrict__ ntiles, int* __restrict__ counter, PairT<T>* __restrict__ scratch, size_t slot_elems,
    const PairT<T>* __restrict__ wtab, double D0, double tol_abs, int32_t* status) {
  constexpr int R = stencil_count<N>();
  constexpr int TAPS = (N + 1) * (N + 1) * (N + 1) * (N + 1);
  __shared__ int s_dx[R], s_dy[R];
  __shared__ unsigned char s_order[TAPS];
  __shared__ int s_gbeg[12], s_gw[11], s_ng, s_terms;
  __shared__ int4 s_tap[kTileWarps][TAPS];
  __shared__ int s_t;
  __shared__ double s_red[3][kTileWarps];
  __shared__ double s_numerr;  // bound on |S - S_exact| for this tile
  if (threadIdx.x == 0) {
    int c = 0;
    for (int iy = 0; iy < 3 * N; ++iy)
      for (int ix = 0; ix < 3 * N; ++ix)
        if (stencil_keeps<N>(ix, iy)) {
          s_dx[c] = Stencil<N>::kDmin + ix;
          s_dy[c] = Stencil<N>::kDmin + iy;
          ++c;
        }
    // taps grouped by their FD weight (at most 10 distinct values for N <= 3)
    int ng = 0, k = 0, terms = 0;
    for (int t = 0; t < TAPS; ++t) {
      const int w = fd_weight<N>(t);
      bool seen = false;
      for (int g = 0; g < ng; ++g) seen |= s_gw[g] == w;
      if (!seen) s_gw[ng++] = w;
    }
    for (int g = 0; g < ng; ++g) {
      s_gbeg[g] = k;
      for (int t = 0; t < TAPS; ++t)
        if (fd_weight<N>(t) == s_gw[g]) s_order[k++] = (unsigned char)t;
      const int pairs = (k - s_gbeg[g]) * R;
      terms = max(terms, (pairs + 31) / 32);
    }
    s_gbeg[ng] = k;
    s_ng = ng;
    s_terms = terms;
  }
  PairT<T>* gw = scratch + (size_t)blockIdx.x * slot_elems;
  const int nt = *ntiles;
  const int lane = threadIdx.x & 31, wslot = threadIdx.x >> 5;
  const int P = pv.P;
  const int sh = (N % 2 == 0) ? 0 : 1;
  const int one = 1 << pv.Q;
  const int half = (N % 2 == 0) ? 0 : (1 << (P - 1));
  const int mask = (1 << P) - 1;
  const double u = unit_roundoff<T>();
  const double u2 = u * u;

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_t = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= nt) break;
    const TileRec tr = tiles[t];
    const int ww = tr.ww, wh = tr.wh;
    // v1: rows, n running sums each, input = f restricted to the window
    double vmin = 0.0, vabs = 0.0;
    for (int r = threadIdx.x; r < wh; r += blockDim.x) {
      const int y = tr.wy0 + r;
      PairT<T> acc[N];
#pragma unroll
      for (int k = 0; k < N; ++k) acc[k] = PairT<T>{0, 0};
      PairT<T>* row = gw + (size_t)r * ww;
      for (int c = 0; c < ww; ++c) {
        const int x = tr.wx0 + c;
        double fv = 0.0;
        if (y >= 0 && y < pv.H && x >= 0 && x < pv.W) fv = fetch_f(pv.in_dtype, f, f_pitch, x, y);
        vmin = vmin < fv ? vmin : fv;
        vabs = vabs > fabs(fv) ? vabs : fabs(fv);
        PairT<T> v = pair_from<T>(fv);
#pragma unroll
        for (int k = 0; k < N; ++k) {
          acc[k] = pair_add(acc[k], v);
          v = acc[k];
        }
        pair_store(row + c, v);
      }
    }
    // v2 (from (x-1, y-1)), v3 (from (x, y-1)), v4 (from (x+1, y-1)): n times
    // each.  A thread owns whole lines of the direction (sheared columns), so a
    // pass needs no barrier between rows; a line's running sum starts where the
    // line enters the window.  The last pass records the largest |g|.
    double gmax = 0.0;
    __syncthreads();
    for (int dir = 2; dir <= 4; ++dir) {
      const int nlines = (dir == 3) ? ww : ww + wh - 1;
      for (int k = 0; k < N; ++k) {
        const bool last = dir == 4 && k == N - 1;
        for (int l = threadIdx.x; l < nlines; l += blockDim.x) {
          PairT<T> acc{0, 0};
          for (int r = 0; r < wh; ++r) {
            const int c = dir == 2 ? l - (wh - 1) + r : (dir == 3 ? l : l - r);
            if (c < 0 || c >= ww) {
              acc = PairT<T>{0, 0};
              continue;
            }
            PairT<T>* p = gw + (size_t)r * ww + c;
            acc = pair_add(acc, pair_load(p));
            pair_store(p, acc);
            if (last) gmax = fmax(gmax, fabs((double)acc.hi) + fabs((double)acc.lo));
          }
        }
        __syncthreads();
      }
    }
    // the tile's bound on |S - S_exact| (see file header)
    for (int o = 16; o > 0; o >>= 1) {
      vmin = fmin(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
      vabs = fmax(vabs, __shfl_xor_sync(0xffffffffu, vabs, o));
      gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    }
    if (lane == 0) {
      s_red[0][wslot] = vmin;
      s_red[1][wslot] = vabs;
      s_red[2][wslot] = gmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double mn = 0.0, fa = 0.0, gm = 0.0;
      for (int w = 0; w < kTileWarps; ++w) {
        mn = fmin(mn, s_red[0][w]);
        fa = fmax(fa, s_red[1][w]);
        gm = fmax(gm, s_red[2][w]);
      }
      const int lmax = max(ww, wh), lmin = min(ww, wh);
      const double gamma_g = 16.0 * N * (double)lmax * u2;
      const double gamma_m = 4.0 * (double)(s_terms + 20) * u2;
      double gabs;
      if (mn >= 0.0) {
        gabs = gm * (1.0 + 2.0 * gamma_g) * (1.0 + 4.0 * u);
      } else {
        gabs = fa * run_growth(ww, N) * run_growth(wh, N) * run_growth(lmin, N) * run_growth(lmin, N) *
               (1.0 + 64.0 * u);
      }
      s_numerr = (double)(1 << (4 * N)) * D0 * gabs * (gamma_g + gamma_m + 2.0 * u2) * 1.0625;
    }
    __syncthreads();
    const double numerr = s_numerr;
    const int ng = s_ng;
    // mesh for the tile's pixels: warp w takes pixels w, w + WARPS, ... in
    // batches of 32 (lane i reads the scales of the batch's i-th pixel)
    const int tw = min(tr.T, pv.W - tr.x0), th = min(tr.T, pv.H - tr.y0);
    const int npx = tw * th;
    for (int base = wslot * 32; base < npx; base += kTileWarps * 32) {
      const int myp = base + lane;
      const int myx = myp < npx ? tr.x0 + myp % tw : 0;
      const int y = myp < npx ? tr.y0 + myp / tw : 0;
      int C0 = 0, C1 = 0, C2 = 0, C3 = 0, ok = 0;
      if (myp < npx) {
        int C[4];
        if (pixel_steps(pv, scales, scale_pitch, myx, y, C)) {
          C0 = C[0]; C1 = C[1]; C2 = C[2]; C3 = C[3];
          ok = 1;
        } else {
          ok = 3;
        }
      }
      PairT<T> mine{0, 0};
      int4* taps = s_tap[wslot];
      for (int pp = 0; pp < 32; ++pp) {
        if (__shfl_sync(0xffffffffu, ok, pp) != 1) continue;
        const int c0 = __shfl_sync(0xffffffffu, C0, pp), c1 = __shfl_sync(0xffffffffu, C1, pp);
        const int c2 = __shfl_sync(0xffffffffu, C2, pp), c3 = __shfl_sync(0xffffffffu, C3, pp);
        const int tx = (N * (c0 + c1 - c3 - one)) << sh >> 1;
        const int ty = (N * (c1 + c2 + c3 - 3 * one)) << sh >> 1;
        const int xp = __shfl_sync(0xffffffffu, myx, pp), ypp = __shfl_sync(0xffffffffu, y, pp);
        const int y0x = (xp << P) + tx;
        const int y0y = (ypp << P) + ty;
        const int s1 = c0 << sh, s2 = c1 << sh, s3 = c2 << sh, s4 = c3 << sh;
        __syncwarp();
        for (int q = lane; q < TAPS; q += 32) {
          const int tt = s_order[q];
          const int j1 = tt % (N + 1), q1 = tt / (N + 1);
          const int j3 = q1 % (N + 1), q2 = q1 / (N + 1);
          const int j2 = q2 % (N + 1), j4 = q2 / (N + 1);
          const int Yx = y0x - j1 * s1 - j2 * s2 + j4 * s4;
          const int Yy = y0y - j2 * s2 - j3 * s3 - j4 * s4;
          const int px = (Yx + half) >> P;
          const int py = (Yy + half) >> P;
          const int rr = (((Yy + half) & mask) << P) | ((Yx + half) & mask);
          taps[q] = make_int4(px - tr.wx0, py - tr.wy0, rr, 0);
        }
        __syncwarp();
        PairT<T> acc{0, 0};
        for (int g = 0; g < ng; ++g) {
          const int tb = s_gbeg[g], npairs = (s_gbeg[g + 1] - tb) * R;
          PairT<T> part{0, 0};
          for (int idx = lane; idx < npairs; idx += 32) {
            const int tap = tb + idx / R;
            const int cand = idx - (idx / R) * R;
            const int4 ti = taps[tap];
            const int k1 = ti.x + s_dx[cand], k2 = ti.y + s_dy[cand];
            // reads stay inside the window by construction
            const PairT<T> gv = pair_load(gw + (size_t)k2 * ww + k1);
            const PairT<T> wv = pair_load(wtab + (size_t)ti.z * R + cand);
            part = pair_add(part, pair_mul(wv, gv));
          }
          acc = pair_add(acc, pair_scale(part, s_gw[g]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = pair_add(acc, pair_shfl_xor(acc, o));
        if (lane == pp) mine = acc;
      }
      if (myp < npx) {
        TOut* orow = reinterpret_cast<TOut*>(reinterpret_cast<char*>(s) + (size_t)y * s_pitch);
        if (ok == 1) {
          // s = S 2^(4 Q n) / (D0 prod C^n), and the bound on its error
          double den = D0;
          const int Cp[4] = {C0, C1, C2, C3};
          for (int k = 0; k < 4; ++k) {
            const double ck = (double)Cp[k];
            for (int e = 0; e < N; ++e) den *= ck;
          }
          const double sc = ldexp(1.0, 4 * pv.Q * N);
          const double v = ((double)mine.hi + (double)mine.lo) * sc / den;
          const double err = numerr * sc / den + fabs(v) * 1e-15;
          if (err <= tol_abs && isfinite(v)) {
            orow[myx] = (TOut)v;
          } else {
            raise_status(status, ABF_DEV_PRECISION);
            orow[myx] = (TOut)__longlong_as_double(0x7ff8000000000000ll);
          }
        } else {
          raise_status(status, ABF_DEV_BAD_SCALE);
          orow[myx] = (TOut)__longlong_as_double(0x7ff8000000000000ll);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- launcher

// Largest window side: the quadtree stops at T <= max(8, c_min) <= max(8, c_max)
// (T a power of two), and the margins grow with the tile's largest step.
size_t tile_ws_bytes(const PlanView& pv, int pair_bytes, int* slots_out, size_t* slot_elems_out,
                     size_t* off_bmax, size_t* off_tiles, size_t* off_cnt, size_t* off_scratch) {
  const int n = pv.n;
  const double cmax = (double)pv.Cmax / (double)(1 << pv.Q);
  const int E = (int)ceil(1.5 * n * cmax);
  const int mgn = E + 3 * n + 1;
  int Tmax = kSuper;
  while (Tmax > kBlk && (double)Tmax > cmax) Tmax /= 2;
  const int side = Tmax + 2 * mgn;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int slots = (sms > 0 ? sms : 152) * kSlotsPerSm;
  const size_t slot_elems = (size_t)side * side;
  const int bw = (pv.W + kBlk - 1) / kBlk, bh = (pv.H + kBlk - 1) / kBlk;
  const size_t ntmax = (size_t)bw * bh;
  size_t off = 0;
  *off_bmax = off; off += 2 * (((size_t)bw * bh * sizeof(int4) + 255) / 256 * 256);
  *off_tiles = off; off += (ntmax * sizeof(TileRec) + 255) / 256 * 256;
  *off_cnt = off; off += 256;
  *off_scratch = off; off += (size_t)slots * slot_elems * pair_bytes;
  *slots_out = slots;
  *slot_elems_out = slot_elems;
  return off;
}

template <int N, typename T>
static cudaError_t run_tiles_N(const PlanView& pv, const void* f, size_t f_pitch, const void* scales,
                               size_t scale_pitch, void* s, size_t s_pitch, void* ws, const void* wtab, double D0,
                               double tol_abs, int32_t* status, cudaStream_t st) {
  int slots;
  size_t slot_elems, ob, otl, oc, osc;
  tile_ws_bytes(pv, (int)sizeof(PairT<T>), &slots, &slot_elems, &ob, &otl, &oc, &osc);
  char* base = (char*)ws;
  const int bw = (pv.W + kBlk - 1) / kBlk, bh = (pv.H + kBlk - 1) / kBlk;
  int4* bmin = (int4*)(base + ob);
  int4* bmax = bmin + (((size_t)bw * bh * sizeof(int4) + 255) / 256 * 256) / sizeof(int4);
  TileRec* tiles = (TileRec*)(base + otl);
  int* cnt = (int*)(base + oc);     // [0] tile count, [1] work counter
  PairT<T>* scratch = (PairT<T>*)(base + osc);
  cudaError_t e = cudaMemsetAsync(cnt, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  block_steps_kernel<<<dim3(bw, bh), kBlk * kBlk, 0, st>>>(pv, (const float4*)scales, scale_pitch, bmin, bmax, status);
  const int nsuper = ((pv.W + kSuper - 1) / kSuper) * ((pv.H + kSuper - 1) / kSuper);
  tile_list_kernel<<<(nsuper + 63) / 64, 64, 0, st>>>(pv, bmin, bmax, bw, bh, tiles, cnt);
  if (pv.out_dtype == ABF_F64)
    tile_filter_kernel<N, T, double><<<slots, kTileThreads, 0, st>>>(
        pv, f, f_pitch, (const float4*)scales, scale_pitch, s, s_pitch, tiles, cnt, cnt + 1, scratch, slot_elems,
        (const PairT<T>*)wtab, D0, tol_abs, status);
  else
    tile_filter_kernel<N, T, float><<<slots, kTileThreads, 0, st>>>(
        pv, f, f_pitch, (const float4*)scales, scale_pitch, s, s_pitch, tiles, cnt, cnt + 1, scratch, slot_elems,
        (const PairT<T>*)wtab, D0, tol_abs, status);
  return cudaGetLastError();
}

cudaError_t run_tiles(const PlanView& pv, bool f64, const void* f, size_t f_pitch, const void* scales,
                      size_t scale_pitch, void* s, size_t s_pitch, void* ws, const void* wtab, double D0,
                      double tol_abs, int32_t* status, cudaStream_t st) {
  if (f64) {
    switch (pv.n) {
      case 1: return run_tiles_N<1, double>(pv, f, f_pitch, scales, scale_pitch, s, s_pitch, ws, wtab, D0, tol_abs, status, st);
      case 2: return run_tiles_N<2, double>(pv, f, f_pitch, scales, scale_pitch, s, s_pitch, ws, wtab, D0, tol_abs, status, st);
      default: return run_tiles_N<3, double>(pv, f, f_pitch, scales, scale_pitch, s, s_pitch, ws, wtab, D0, tol_abs, status, st);
    }
  }
  // binary32 pairs: order 1 only (the plan refuses higher orders)
  return run_tiles_N<1, float>(pv, f, f_pitch, scales, scale_pitch, s, s_pitch, ws, wtab, D0, tol_abs, status, st);
}

}  // namespace abf
