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
#include <map>
#include <mutex>
#include <utility>

#include "abf_internal.cuh"


namespace abf {

// log2 of the numerator bound for this pixel (see file header), in binary32
// with a margin that covers its rounding (the check only has to be safe).
__device__ __forceinline__ float numerator_log2_bound(const PlanView& pv, const int C[4]) {
  float lp = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) lp += __log2f((float)C[k]) - (float)pv.Q;
  const float q = (float)(1 << pv.Q);
  const float kappa = (1.0f + q / (float)C[0]) * (1.0f + q / (float)C[2]);
  return pv.log2_base + (float)pv.n * lp + __log2f(kappa) + 0.05f;
}

// (-1)^j binom(N, j) for N <= 3: binom is 1 at the ends and N inside.
template <int N>
__device__ __forceinline__ int signed_binom(int j) {
  const int c = (j == 0 || j == N) ? 1 : N;
  return (j & 1) ? -c : c;
}

// Table weight times the FD weight |w_j| (a power of two for n <= 2).
template <int N, typename WT>
__device__ __forceinline__ WT scale_weight(WT w, int aw) {
  if constexpr (N == 1) {
    return w;
  } else if constexpr (N == 2) {
    return w << (__ffs(aw) - 1);
  } else {
    // 128-bit times a small factor (|w_j| <= 81); fits: D 81 < 2^128.
    const uint64_t lo = w.x * (uint64_t)aw;
    const uint64_t hi = __umul64hi(w.x, (uint64_t)aw) + w.y * (uint64_t)aw;
    return make_ulonglong2(lo, hi);
  }
}

template <typename TOut>
__device__ __forceinline__ void store_out(void* s, size_t s_pitch, int x, int y, double v) {
  TOut* row = reinterpret_cast<TOut*>(reinterpret_cast<char*>(s) + (size_t)y * s_pitch);
  row[x] = (TOut)v;
}

// One warp per run of 32 pixels of a row.  Lane i reads the scales of pixel
// x0 + i and rounds them to integer steps; then the warp walks the 32 pixels
// one at a time.  For a pixel, the lanes first tabulate its (n+1)^4 taps
// (lattice point p_j, table row r_j, FD weight w_j) in shared memory; then the
// (tap, neighbour) pairs -- (n+1)^4 taps times the stencil's neighbours -- are
// dealt to the lanes in order, so the lanes of one tap read one contiguous
// table row and one compact patch of g.  For n = 2 the 32 neighbours are
// exactly the 32 lanes: every lane keeps its neighbour, the tap is the same
// for the whole warp, and w_j = +-2^k folds into the table weight as a shift
// with the sign choosing one of two accumulators.  Each lane accumulates
// w_j g[p_j + d] W(r_j - d) modulo 2^(64 L); a warp reduction gives the
// numerator, which lane i keeps for its own pixel and stores at the end.
constexpr int kMeshWarps = 8;      // default rows (warps) per CTA
constexpr int kMeshWarpsMax = 16;  // largest CTA the kernels are compiled for
// Per order: the largest CTA (rows) and the CTAs per SM the register budget is
// set for -- order 3 keeps its wide accumulators in up to 85 registers with
// CTAs of at most 8 rows, orders 1 and 2 fit 64 registers at 16 rows.
__host__ __device__ constexpr int mesh_max_warps(int n) { return n == 3 ? 8 : 16; }
__host__ __device__ constexpr int mesh_min_ctas(int n) { return n == 3 ? 3 : 2; }

// The stencil's neighbours, in the same order as the table rows (one thread).
template <int N>
__device__ __forceinline__ void fill_stencil(int* s_dx, int* s_dy) {
  int c = 0;
  for (int iy = 0; iy < 3 * N; ++iy)
    for (int ix = 0; ix < 3 * N; ++ix)
      if (stencil_keeps<N>(ix, iy)) {
        s_dx[c] = Stencil<N>::kDmin + ix;
        s_dy[c] = Stencil<N>::kDmin + iy;
        ++c;
      }
}

// a <<= k (mod 2^(64 L)), 0 <= k < 64.
template <int L>
__device__ __forceinline__ void wshl(Wide<L>& a, int k) {
  if (k == 0) return;
#pragma unroll
  for (int i = L - 1; i > 0; --i) a.w[i] = (a.w[i] << k) | (a.w[i - 1] >> (64 - k));
  a.w[0] <<= k;
}

// n = 2: the FD weight of vertex j is w_j = (-2)^k, k = #{i : j_i = 1}.  The
// taps are visited grouped by k (group sizes binom(4,k) 2^(4-k) = 16, 32, 24,
// 8, 1), each group summed without its weight and then added with it.
__host__ __device__ constexpr int n2_group_begin(int k) {
  return k <= 0 ? 0 : k == 1 ? 16 : k == 2 ? 48 : k == 3 ? 72 : k == 4 ? 80 : 81;
}

// Tap order for n = 2 (one thread): slot -> natural tap index t = j1 + 3 j3 + 9 j2 + 27 j4.
__device__ __forceinline__ void fill_n2_order(unsigned char* order) {
  int c = 0;
  for (int k = 0; k <= 4; ++k)
    for (int t = 0; t < 81; ++t) {
      int ones = 0;
      for (int u = t, i = 0; i < 4; ++i, u /= 3) ones += (u % 3) == 1;
      if (ones == k) order[c++] = (unsigned char)t;
    }
}

// n = 3: w_j = (-1)^(j1+j2+j3+j4) 3^m, m = #{i : j_i in {1, 2}}.  The taps are
// visited in ten groups, by m and then by the parity of sum j (group size
// binom(4,m) 8 each), each group summed without its weight and then added
// with it.
__host__ __device__ constexpr int n3_group_begin(int g) {
  return g <= 0 ? 0 : g == 1 ? 8 : g == 2 ? 16 : g == 3 ? 48 : g == 4 ? 80 : g == 5 ? 128 : g == 6 ? 176
         : g == 7 ? 208 : g == 8 ? 240 : g == 9 ? 248 : 256;
}

// Tap order for n = 3 (one thread): slot -> natural tap index t = j1 + 4 j3 + 16 j2 + 64 j4.
__device__ __forceinline__ void fill_n3_order(unsigned char* order) {
  int c = 0;
  for (int m = 0; m <= 4; ++m)
    for (int par = 0; par <= 1; ++par)
      for (int t = 0; t < 256; ++t) {
        int mm = 0, sum = 0;
        for (int u = t, i = 0; i < 4; ++i, u /= 4) {
          mm += (u % 4 == 1 || u % 4 == 2);
          sum += u % 4;
        }
        if (mm == m && (sum & 1) == par) order[c++] = (unsigned char)t;
      }
}

// Folded-table columns for the eight symmetries of the square (n = 3):
// perm[sym 69 + c] = index of S(d_c), S = flip x (bit 0), flip y (bit 1), then
// swap x and y (bit 2).  All threads of the CTA take part.
__device__ __forceinline__ void fill_n3_perm(unsigned char* perm, const int* s_dx, const int* s_dy) {
  constexpr int R = stencil_count<3>(), kD = Stencil<3>::kDmin;
  __shared__ signed char s_idx[81];
  for (int i = threadIdx.x; i < 81; i += blockDim.x) s_idx[i] = -1;
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += blockDim.x) s_idx[(s_dy[c] - kD) * 9 + (s_dx[c] - kD)] = (signed char)c;
  __syncthreads();
  for (int k = threadIdx.x; k < 8 * R; k += blockDim.x) {
    const int sym = k / R, c = k - sym * R;
    int ex = (sym & 1) ? -s_dx[c] : s_dx[c], ey = (sym & 2) ? -s_dy[c] : s_dy[c];
    if (sym & 4) {
      const int t = ex;
      ex = ey;
      ey = t;
    }
    perm[k] = (unsigned char)s_idx[(ey - kD) * 9 + (ex - kD)];
  }
  __syncthreads();
}

// A lane's fixed share of the order-3 stencil: neighbours A = lane, B = 32 +
// lane (two full passes per tap) and C = 64 + lane % 5 (the packed pass that
// covers neighbours 64..68 of four taps with lanes 0..19): their g offsets
// dy Gp + dx, rows dy, and folded-table columns under the eight symmetries
// (byte sym of perm*).
struct N3Lane {
  int offA, offB, offC, dyA, dyB, dyC;
  uint32_t permA[2], permB[2], permC[2];
};

__device__ __forceinline__ int perm_col(const uint32_t (&pk)[2], int sym) {
  const uint32_t w = (sym & 4) ? pk[1] : pk[0];  // a select, not an indexed (local-memory) load
  return (int)((w >> ((sym & 3) * 8)) & 0xffu);
}

__device__ __forceinline__ N3Lane n3_lane(int lane, const int* s_off, const int* s_dy, const unsigned char* s_perm) {
  constexpr int R = 69;
  N3Lane ln;
  const int cA = lane, cB = 32 + lane, cC = 64 + lane % 5;
  ln.offA = s_off[cA]; ln.offB = s_off[cB]; ln.offC = s_off[cC];
  ln.dyA = s_dy[cA]; ln.dyB = s_dy[cB]; ln.dyC = s_dy[cC];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t a = 0, b = 0, c = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int sym = 4 * h + k;
      a |= (uint32_t)s_perm[sym * R + cA] << (8 * k);
      b |= (uint32_t)s_perm[sym * R + cB] << (8 * k);
      c |= (uint32_t)s_perm[sym * R + cC] << (8 * k);
    }
    ln.permA[h] = a; ln.permB[h] = b; ln.permC[h] = c;
  }
  return ln;
}

// One pixel's numerator share for n = 3.  taps[s] = (g offset of the tap's
// lattice point, offset of its row in the folded table, lattice row,
// symmetry).  Every group of taps is taken four at a time: each tap in two
// full passes (neighbours 0..31 and 32..63, lane = neighbour, the tap record
// broadcast), then one packed pass in which lanes 0..19 cover neighbours
// 64..68 of the four taps (276 of 288 lane slots busy).  CHECK drops this
// lane's read where its own row is below 0.
template <int L, bool CHECK>
__device__ __forceinline__ void n3_pixel(Wide<L>& acc, const int4* taps, const uint64_t* __restrict__ g,
                                         const ulonglong2* __restrict__ table, const N3Lane& ln, int lane) {
#pragma unroll 1
  for (int gi = 0; gi < 10; ++gi) {
    const int tb = n3_group_begin(gi), te = n3_group_begin(gi + 1);
    Wide<L> part;
    wzero<L>(part);
#pragma unroll 1
    for (int t0 = tb; t0 < te; t0 += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int4 ti = taps[t0 + u];
        if (!CHECK || ti.z + ln.dyA >= 0) {
          const Wide<L> gv = wload<L>(g + (ptrdiff_t)(ti.x + ln.offA) * L);
          mac_weight<L, ulonglong2>(part, gv, __ldg(table + ti.y + perm_col(ln.permA, ti.w)));
        }
        if (!CHECK || ti.z + ln.dyB >= 0) {
          const Wide<L> gv = wload<L>(g + (ptrdiff_t)(ti.x + ln.offB) * L);
          mac_weight<L, ulonglong2>(part, gv, __ldg(table + ti.y + perm_col(ln.permB, ti.w)));
        }
      }
      if (lane < 20) {
        const int4 ti = taps[t0 + lane / 5];
        if (!CHECK || ti.z + ln.dyC >= 0) {
          const Wide<L> gv = wload<L>(g + (ptrdiff_t)(ti.x + ln.offC) * L);
          mac_weight<L, ulonglong2>(part, gv, __ldg(table + ti.y + perm_col(ln.permC, ti.w)));
        }
      }
    }
    // group weight (-1)^parity 3^m, m = gi / 2
    const int m = gi >> 1;
    const uint64_t w3 = m == 0 ? 1 : m == 1 ? 3 : m == 2 ? 9 : m == 3 ? 27 : 81;
    Wide<L> scaled;
    wzero<L>(scaled);
    wmac<L>(scaled, part, w3);
    if (gi & 1) wsub<L>(acc, scaled);
    else wadd<L>(acc, scaled);
  }
}

// One pixel's numerator share for n = 2 (lane = neighbour): taps[s] holds
// (x: g offset of the tap's lattice point from this lane's base gl, y: table
// offset from this lane's base tl, z: the tap's lattice row).  A tap whose
// whole stencil lies below row 0 points at the table's zero row and at a
// readable patch; CHECK also drops this lane's read where its own row is below 0
// (taps that straddle row 0).
template <int L, bool CHECK>
__device__ __forceinline__ void n2_pixel(Wide<L>& acc, const int4* taps, const uint64_t* gl,
                                         const uint64_t* __restrict__ tl, int dy) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    Wide<L> part;
    wzero<L>(part);
#pragma unroll
    for (int s = n2_group_begin(k); s < n2_group_begin(k + 1); ++s) {
      const int2 ti = *reinterpret_cast<const int2*>(&taps[s]);
      if (CHECK && taps[s].z + dy < 0) continue;
      const Wide<L> gv = wload<L>(gl + (ptrdiff_t)ti.x * L);
      const uint64_t wt = __ldg(tl + ti.y);
      mac_weight<L, uint64_t>(part, gv, wt);
    }
    wshl<L>(part, k);
    if (k & 1) wsub<L>(acc, part);
    else wadd<L>(acc, part);
  }
}

// Bounds checking of one pixel's tabulated taps (the fast paths' records:
// x = g offset row * Gp + box column, y = table offset, z = lattice row): a
// tap whose stencil box would leave the lattice box is pointed at the table's
// zero row (zrow) and at the patch in the box corner, so it reads in bounds
// and adds nothing.  Taps wholly below row 0 already read that way.
template <int N>
__device__ __forceinline__ void dbg_taps(const PlanView& pv, int32_t* status, int4* taps, int ntaps, int zrow,
                                         int lane, int x, int y) {
  constexpr int kDlo = Stencil<N>::kDmin, kDhi = Stencil<N>::kDmin + 3 * N - 1;
  const int gp = (int)pv.Gp;
  __syncwarp();
  for (int slot = lane; slot < ntaps; slot += 32) {
    const int4 t = taps[slot];
    if (t.z + kDhi < 0) continue;  // below row 0: redirected already
    const int cx = t.x - t.z * gp;  // box column of the tap's lattice point
    if (!dbg_tap_ok(pv, status, cx, t.z, kDlo, kDhi, kDhi, x, y))
      taps[slot] = make_int4(-kDlo * gp - kDlo, zrow, -kDlo, 0);
  }
}

// Mesh for the run of 32 pixels (x0 .. x0+31, y) of one image; the whole warp
// calls it.  taps: this warp's (n+1)^4-entry shared tap table; s_dx/s_dy: the
// order-n stencil in shared memory.  FAST (n = 2, 3): taps carry plain g and
// table offsets, and the FD weights are applied per group (n2_pixel,
// n3_pixel); s_order is then the group-sorted tap order, s_off (n = 3) the
// neighbours' g offsets dy Gp + dx, and g offsets must fit 32 bits and the
// box have at least 3n rows.
template <int N, int L, bool FAST = false, bool DBG = false>
__device__ __forceinline__ void mesh_run(const PlanView& pv, const uint64_t* __restrict__ g,
                                         const float4* __restrict__ scales, size_t scale_pitch, void* __restrict__ s,
                                         size_t s_pitch, uint64_t* __restrict__ num, size_t num_pitch,
                                         int32_t* status, int y, int x0, int4* taps, const int* s_dx,
                                         const int* s_dy, const unsigned char* s_order = nullptr,
                                         const int* s_off = nullptr, const unsigned char* s_perm = nullptr) {
  using WT = typename WeightT<N>::T;
  constexpr int R = stencil_count<N>();
  constexpr int TAPS = (N + 1) * (N + 1) * (N + 1) * (N + 1);
  constexpr int PAIRS = TAPS * R;
  constexpr int ITERS = (PAIRS + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int myx = x0 + lane;

  // a5: this lane's pixel -> integer steps, validity, numerator bound
  int C0 = 0, C1 = 0, C2 = 0, C3 = 0, ok = 0;  // ok: 0 outside, 1 good, 2 range, 3 bad scale
  if (myx < pv.W) {
    int C[4];
    if (!pixel_steps(pv, scales, scale_pitch, myx, y, C)) {
      ok = 3;
    } else {
      C0 = C[0]; C1 = C[1]; C2 = C[2]; C3 = C[3];
      ok = (numerator_log2_bound(pv, C) < 64.0f * L - 1.0f) ? 1 : 2;
    }
  }
  const WT* __restrict__ table = reinterpret_cast<const WT*>(pv.table);
  const int P = pv.P;
  const int sh = (N % 2 == 0) ? 0 : 1;  // 2^(P-Q)
  const int one = 1 << pv.Q;
  const int half = (N % 2 == 0) ? 0 : (1 << (P - 1));
  const int mask = (1 << P) - 1;
  const long long rowpitch = pv.Gp;
  const int left = pv.left;

  // for n = 2 a lane keeps one neighbour for every tap; for n = 3 (fast) three
  const int my_dx = (R == 32) ? s_dx[lane] : 0;
  const int my_dy = (R == 32) ? s_dy[lane] : 0;
  N3Lane n3ln{};
  if constexpr (FAST && N == 3) n3ln = n3_lane(lane, s_off, s_dy, s_perm);

  Wide<L> mine;
  wzero<L>(mine);
#pragma unroll 1
  for (int pp = 0; pp < 32; ++pp) {
    if (__shfl_sync(0xffffffffu, ok, pp) != 1) continue;
    const int c0 = __shfl_sync(0xffffffffu, C0, pp), c1 = __shfl_sync(0xffffffffu, C1, pp);
    const int c2 = __shfl_sync(0xffffffffu, C2, pp), c3 = __shfl_sync(0xffffffffu, C3, pp);
    // tau in units of 2^-P: (n/2) sum_k (C_k - 2^Q) v_k 2^(P-Q)
    const int tx = (N * (c0 + c1 - c3 - one)) << sh >> 1;
    const int ty = (N * (c1 + c2 + c3 - 3 * one)) << sh >> 1;
    const int y0x = ((x0 + pp) << P) + tx;
    const int y0y = (y << P) + ty;
    const int s1 = c0 << sh, s2 = c1 << sh, s3 = c2 << sh, s4 = c3 << sh;
    __syncwarp();
    Wide<L> acc;
    wzero<L>(acc);
    if constexpr (FAST && N == 3) {
      constexpr int kDyMin = Stencil<N>::kDmin, kDyMax = Stencil<N>::kDmin + 3 * N - 1;
      const int gp = (int)rowpitch;
      int strad = 0;
      for (int slot = lane; slot < TAPS; slot += 32) {
        const int t = s_order[slot];
        const int j1 = t & 3, j3 = (t >> 2) & 3, j2 = (t >> 4) & 3, j4 = t >> 6;
        const int Yx = y0x - j1 * s1 - j2 * s2 + j4 * s4 + half;
        const int Yy = y0y - j2 * s2 - j3 * s3 - j4 * s4 + half;
        const int px = Yx >> P, py = Yy >> P;
        // centred offset, folded onto 0 <= X <= Y <= half
        const int ax = (Yx & mask) - half, ay = (Yy & mask) - half;
        const int fx = ax < 0, fy = ay < 0;
        const int X0 = fx ? -ax : ax, Y0 = fy ? -ay : ay;
        const int sw = X0 > Y0;
        const int X = sw ? Y0 : X0, Y = sw ? X0 : Y0;
        const bool below = py + kDyMax < 0;
        strad |= (py + kDyMin < 0) && !below;
        const int xf = (below ? -kDyMin : py) * gp + px + left;
        const int frow = below ? (half + 1) * (half + 2) / 2 : (Y * (Y + 1) >> 1) + X;
        taps[slot] = make_int4(xf, frow * R, py, below ? 0 : (fx | (fy << 1) | (sw << 2)));
      }
      if constexpr (DBG) dbg_taps<N>(pv, status, taps, TAPS, (half + 1) * (half + 2) / 2 * R, lane, x0 + pp, y);
      const bool check = __any_sync(0xffffffffu, strad) != 0;
      __syncwarp();
      const ulonglong2* tab = reinterpret_cast<const ulonglong2*>(pv.table_fold);
      if (check) n3_pixel<L, true>(acc, taps, g, tab, n3ln, lane);
      else n3_pixel<L, false>(acc, taps, g, tab, n3ln, lane);
    } else if constexpr (FAST) {
      static_assert(N == 2 && R == 32, "fast path is for n = 2 and n = 3");
      constexpr int kDyMin = Stencil<N>::kDmin, kDyMax = Stencil<N>::kDmin + 3 * N - 1;
      const int gp = (int)rowpitch;
      int strad = 0;
      for (int slot = lane; slot < TAPS; slot += 32) {
        const int t = s_order[slot];
        const int j1 = t % 3, j3 = (t / 3) % 3, j2 = (t / 9) % 3, j4 = t / 27;
        const int Yx = y0x - j1 * s1 - j2 * s2 + j4 * s4;
        const int Yy = y0y - j2 * s2 - j3 * s3 - j4 * s4;
        const int px = Yx >> P, py = Yy >> P;
        const int r = ((Yy & mask) << P) | (Yx & mask);
        const bool below = py + kDyMax < 0;
        strad |= (py + kDyMin < 0) && !below;
        const int xf = (below ? -kDyMin : py) * gp + px + left;
        const int tf = (below ? (1 << (2 * P)) : r) * R;
        taps[slot] = make_int4(xf, tf, py, 0);
      }
      if constexpr (DBG) dbg_taps<N>(pv, status, taps, TAPS, (1 << (2 * P)) * R, lane, x0 + pp, y);
      const bool check = __any_sync(0xffffffffu, strad) != 0;
      __syncwarp();
      const uint64_t* gl = g + ((ptrdiff_t)my_dy * rowpitch + my_dx) * L;
      const uint64_t* tl = reinterpret_cast<const uint64_t*>(pv.table) + lane;
      if (check) n2_pixel<L, true>(acc, taps, gl, tl, my_dy);
      else n2_pixel<L, false>(acc, taps, gl, tl, my_dy);
    } else {
      for (int t = lane; t < TAPS; t += 32) {
        const int j1 = t % (N + 1);
        const int t1 = t / (N + 1);
        const int j3 = t1 % (N + 1);
        const int t2 = t1 / (N + 1);
        const int j2 = t2 % (N + 1);
        const int j4 = t2 / (N + 1);
        const int w = signed_binom<N>(j1) * signed_binom<N>(j2) * signed_binom<N>(j3) * signed_binom<N>(j4);
        // y_j = y0 - j1 c1 v1 - j2 c2 v2 - j3 c3 v3 - j4 c4 v4
        const int Yx = y0x - j1 * s1 - j2 * s2 + j4 * s4;
        const int Yy = y0y - j2 * s2 - j3 * s3 - j4 * s4;
        const int px = (Yx + half) >> P;
        const int py = (Yy + half) >> P;
        const int r = (((Yy + half) & mask) << P) | ((Yx + half) & mask);
        // n = 2: store the shift k of |w| = 2^k; otherwise |w|
        const int aw = w < 0 ? -w : w;
        taps[t] = make_int4(px + left, py, r, ((N == 2) ? (__ffs(aw) - 1) : aw) * (w < 0 ? -1 : 1) - (w < 0 ? 1 : 0));
        // bounds checking: a tap whose reads would leave the box gets a row
        // so far below 0 that none of its reads happen
        if constexpr (DBG) {
          constexpr int kDlo = Stencil<N>::kDmin, kDhi = Stencil<N>::kDmin + 3 * N - 1;
          if (py + kDhi >= 0 && !dbg_tap_ok(pv, status, px + left, py, kDlo, kDhi, kDhi, x0 + pp, y))
            taps[t].y = -(1 << 20);
        }
      }
      __syncwarp();
      Wide<L> accn;
      wzero<L>(accn);
#pragma unroll 4
      for (int it = 0; it < ITERS; ++it) {
        const int pair = it * 32 + lane;
        if (PAIRS % 32 != 0 && pair >= PAIRS) continue;
        const int tap = (R == 32) ? it : pair / R;
        const int cand = (R == 32) ? lane : pair - tap * R;
        const int4 ti = taps[tap];
        const int dx = (R == 32) ? my_dx : s_dx[cand];
        const int dy = (R == 32) ? my_dy : s_dy[cand];
        const int k2 = ti.y + dy;
        if (k2 < 0) continue;  // rows below the image: g = 0
        const bool neg = ti.w < 0;
        const int code = neg ? -(ti.w + 1) : ti.w;  // shift (n = 2) or |w_j|
        const WT wt = __ldg(table + (size_t)ti.z * R + cand);
        const Wide<L> gv = wload<L>(g + ((size_t)k2 * rowpitch + (size_t)(ti.x + dx)) * L);
        if constexpr (N == 2) {
          const WT ws = wt << code;
          if (neg) mac_weight<L, WT>(accn, gv, ws);
          else mac_weight<L, WT>(acc, gv, ws);
        } else {
          mac_weight<L, WT>(acc, neg ? wneg<L>(gv) : gv, scale_weight<N, WT>(wt, code));
        }
      }
      if constexpr (N == 2) wsub<L>(acc, accn);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Wide<L> other;
#pragma unroll
      for (int i = 0; i < L; ++i) other.w[i] = __shfl_xor_sync(0xffffffffu, acc.w[i], o);
      wadd<L>(acc, other);
    }
    if (lane == pp) mine = acc;
  }

  if (myx >= pv.W) return;
  const bool f64 = pv.out_dtype == ABF_F64;
  if (ok != 1) {
    raise_status(status, ok == 3 ? ABF_DEV_BAD_SCALE : ABF_DEV_RANGE);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    if (s) {
      if (f64) store_out<double>(s, s_pitch, myx, y, nan);
      else store_out<float>(s, s_pitch, myx, y, nan);
    }
    return;
  }
  if (num) {
    uint64_t* q = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(num) + (size_t)y * num_pitch) + (size_t)myx * L;
#pragma unroll
    for (int i = 0; i < L; ++i) q[i] = mine.w[i];
  }
  if (s) {
    // s = S 2^(4Qn - F) / (D prod C^n)
    double den = pv.Dd;
    const int C[4] = {C0, C1, C2, C3};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double ck = (double)C[k];
      double p = 1.0;
#pragma unroll
      for (int e = 0; e < N; ++e) p *= ck;
      den *= p;
    }
    const double v = ldexp(wto_double<L>(mine), 4 * pv.Q * N - pv.F) / den;
    if (f64) store_out<double>(s, s_pitch, myx, y, v);
    else store_out<float>(s, s_pitch, myx, y, v);
  }
}

// One warp per run of 32 pixels of a row.  Lane i reads the scales of pixel
// x0 + i and rounds them to integer steps; then the warp walks the 32 pixels
// one at a time.  For a pixel, the lanes first tabulate its (n+1)^4 taps
// (lattice point p_j, table row r_j, FD weight w_j) in shared memory; then the
// (tap, neighbour) pairs -- (n+1)^4 taps times the stencil's neighbours -- are
// dealt to the lanes in order, so the lanes of one tap read one contiguous
// table row and one compact patch of g.  For n = 2 the 32 neighbours are
// exactly the 32 lanes: every lane keeps its neighbour, the tap is the same
// for the whole warp, and w_j = +-2^k folds into the table weight as a shift
// with the sign choosing one of two accumulators.  Each lane accumulates
// w_j g[p_j + d] W(r_j - d) modulo 2^(64 L); a warp reduction gives the
// numerator, which lane i keeps for its own pixel and stores at the end.
// A CTA takes the 32-column runs of blockDim.x / 32 consecutive rows (a
// launch parameter, 4 to 16, chosen by the plan's autotuner): neighbouring
// rows have nearby taps, so their g patches are shared in L1.  Each warp's tap
// table lives in dynamic shared memory.
template <int N, int L, bool FAST, bool DBG = false>
__device__ __forceinline__ void mesh_exact_body(const PlanView& pv, const uint64_t* __restrict__ g,
                                                const float4* __restrict__ scales, size_t scale_pitch,
                                                void* __restrict__ s, size_t s_pitch, uint64_t* __restrict__ num,
                                                size_t num_pitch, int32_t* status) {
  constexpr int R = stencil_count<N>();
  constexpr int TAPS = (N + 1) * (N + 1) * (N + 1) * (N + 1);
  __shared__ int s_dx[R], s_dy[R], s_off[R];
  __shared__ unsigned char s_order[TAPS], s_perm[8 * R];
  extern __shared__ int4 s_tap[];
  if (threadIdx.x == 0) {
    fill_stencil<N>(s_dx, s_dy);
    if constexpr (FAST && N == 2) fill_n2_order(s_order);
    if constexpr (FAST && N == 3) fill_n3_order(s_order);
  }
  __syncthreads();
  if (threadIdx.x < R) s_off[threadIdx.x] = s_dy[threadIdx.x] * (int)pv.Gp + s_dx[threadIdx.x];
  if constexpr (FAST && N == 3) fill_n3_perm(s_perm, s_dx, s_dy);
  __syncthreads();
  const int rows = blockDim.x >> 5;
  const int segs = (pv.W + 31) >> 5;
  const int band = blockIdx.x / segs;
  const int y = band * rows + (threadIdx.x >> 5);
  if (y >= pv.H) return;
  const int x0 = (blockIdx.x - band * segs) * 32;
  mesh_run<N, L, FAST, DBG>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, y, x0,
                       s_tap + (threadIdx.x >> 5) * TAPS, s_dx, s_dy, s_order, s_off, s_perm);
}

// Orders 1, 2: CTAs of up to 16 rows, the compiler's register choice for
// 512-thread blocks.  Order 3: up to 8 rows, three CTAs per SM (85 registers
// for its wide accumulators).
// DBG: the bounds-checked variant (plans with ABF_FLAG_DEBUG_BOUNDS).
template <int N, int L, bool FAST, bool DBG>
__global__ void __launch_bounds__(32 * kMeshWarpsMax) mesh_exact_kernel(
    const PlanView pv, const uint64_t* __restrict__ g, const float4* __restrict__ scales, size_t scale_pitch,
    void* __restrict__ s, size_t s_pitch, uint64_t* __restrict__ num, size_t num_pitch, int32_t* status) {
  mesh_exact_body<N, L, FAST, DBG>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status);
}

template <int L, bool FAST, bool DBG>
__global__ void __launch_bounds__(32 * mesh_max_warps(3), mesh_min_ctas(3)) mesh_exact_kernel3(
    const PlanView pv, const uint64_t* __restrict__ g, const float4* __restrict__ scales, size_t scale_pitch,
    void* __restrict__ s, size_t s_pitch, uint64_t* __restrict__ num, size_t num_pitch, int32_t* status) {
  mesh_exact_body<3, L, FAST, DBG>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status);
}

// ------------------------------------------------------------------- batches
// Many images (each its own plan: size, order n, limbs) in one persistent
// launch per (order n, limbs, fast path).  The images' units (rows x 32 columns) are
// numbered consecutively, the most expensive images first; every CTA
// repeatedly takes the next unit from a global counter and filters it with its
// image's plan, so images of uneven size share the GPU without a tail of idle
// SMs.
constexpr int kMaxBatch = 96;

struct BatchJob {
  PlanView pv;
  const uint64_t* g;
  const float4* scales;
  size_t scale_pitch;
  void* s;
  size_t s_pitch;
  int32_t* status;
  long long units_begin;  // first global unit index of this image
  int segs;               // 32-column runs per row
};

struct BatchJobs {
  int njobs;
  long long total_units;
  BatchJob job[kMaxBatch];
};

template <int N, int L, bool FAST>
__device__ __forceinline__ void batch_dispatch_L(const BatchJob& jb, int y, int x0, int4* taps, const int* sdx,
                                                 const int* sdy, const unsigned char* order, const int* soff,
                                                 const unsigned char* perm) {
  mesh_run<N, L, FAST>(jb.pv, jb.g, jb.scales, jb.scale_pitch, jb.s, jb.s_pitch, nullptr, 0, jb.status, y, x0, taps,
                       sdx, sdy, order, soff, perm);
}

// Work items are single warps' runs: 32 columns of one row of one image.
// Every warp takes its next item from a global counter on its own, so a warp
// that finishes early starts its next run at once (no CTA-wide barrier between
// items).  Items are numbered per image band by band (a band = `rows` rows),
// within a band strip by strip, within a strip row by row: the warps of a CTA,
// taking consecutive items, work on nearby rows of one 32-column strip, whose g
// patches meet in L1 as in the single-image launch.  One kernel per order n,
// so that each gets its own register budget; the images of one launch share n
// and limbs and differ in size.
template <int N, int L, bool FAST>
__device__ __forceinline__ void mesh_batch_body(const BatchJobs& jobs, unsigned long long* counter, int rows) {
  constexpr int R = stencil_count<N>();
  constexpr int TAPS = (N + 1) * (N + 1) * (N + 1) * (N + 1);
  __shared__ int s_dx[R], s_dy[R];
  __shared__ int s_offw[(FAST && N == 3) ? kMeshWarpsMax : 1][R];
  __shared__ unsigned char s_order[TAPS], s_perm[8 * R];
  extern __shared__ int4 s_tap[];
  if (threadIdx.x == 0) {
    fill_stencil<N>(s_dx, s_dy);
    if constexpr (FAST && N == 2) fill_n2_order(s_order);
    if constexpr (FAST && N == 3) fill_n3_order(s_order);
  }
  __syncthreads();
  if constexpr (FAST && N == 3) fill_n3_perm(s_perm, s_dx, s_dy);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int4* taps = s_tap + warp * TAPS;
  int* s_off = s_offw[(FAST && N == 3) ? warp : 0];
  int last_job = -1;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(counter, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if ((long long)item >= jobs.total_units) break;
    int lo = 0, hi = jobs.njobs - 1;  // last job with units_begin <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs.job[mid].units_begin <= (long long)item) lo = mid;
      else hi = mid - 1;
    }
    const BatchJob& jb = jobs.job[lo];
    if (FAST && N == 3 && lo != last_job) {
      __syncwarp();
      for (int c = lane; c < R; c += 32) s_off[c] = s_dy[c] * (int)jb.pv.Gp + s_dx[c];
      __syncwarp();
      last_job = lo;
    }
    const long long u = (long long)item - jb.units_begin;
    const long long per_band = (long long)jb.segs * rows;
    const int band = (int)(u / per_band);
    const int rem = (int)(u - (long long)band * per_band);
    const int strip = rem / rows;
    const int y = band * rows + (rem - strip * rows);
    if (y >= jb.pv.H) continue;
    batch_dispatch_L<N, L, FAST>(jb, y, strip * 32, taps, s_dx, s_dy, s_order, s_off, s_perm);
  }
}

template <int N, int L, bool FAST>
__global__ void __launch_bounds__(32 * kMeshWarpsMax) mesh_batch_kernel(const __grid_constant__ BatchJobs jobs,
                                                                        unsigned long long* counter, int rows) {
  mesh_batch_body<N, L, FAST>(jobs, counter, rows);
}

template <int L, bool FAST>
__global__ void __launch_bounds__(32 * mesh_max_warps(3), mesh_min_ctas(3)) mesh_batch_kernel3(
    const __grid_constant__ BatchJobs jobs, unsigned long long* counter, int rows) {
  mesh_batch_body<3, L, FAST>(jobs, counter, rows);
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

// The fast paths (n = 2, 3) address g with 32-bit element offsets (rows
// -3n/2 .. Gh + 3n/2 of pitch Gp) and park taps below the image on rows
// 0 .. 3n-1 of the box.
static bool mesh_fast_ok(const PlanView& pv) {
  return pv.n >= 2 && pv.Gh >= 3 * pv.n && ((long long)pv.Gh + 8) * pv.Gp < (1ll << 31) &&
         (pv.n != 3 || pv.table_fold != nullptr);
}

// Dynamic shared memory of a launch with `warps` rows per CTA: one tap table
// per warp; above 48 KB the kernel must opt in.  The shared-memory carveout is
// also set to what the CTAs that the register file admits per SM need, so that
// the rest of the unified L1/shared storage stays L1 for the g patches and the
// table rows.  The carveout is a property of the kernel, not of a launch: it is
// set again whenever the rows per CTA of the next launch need another one.
template <typename K>
static cudaError_t tap_smem(K kernel, int taps, int warps, size_t* bytes) {
  *bytes = (size_t)warps * taps * sizeof(int4);
  cudaError_t e = cudaSuccess;
  if (*bytes > 48 * 1024) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*bytes);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> pct_of;  // (kernel, rows per CTA) -> carveout percent
  static std::map<const void*, int> set_to;                  // kernel -> carveout last set
  std::lock_guard<std::mutex> lk(mu);
  const std::pair<const void*, int> key((const void*)kernel, warps);
  auto it = pct_of.find(key);
  if (it == pct_of.end()) {
    int pct = -1;
    cudaFuncAttributes fa{};
    int dev = 0, smem_sm = 0;
    if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        fa.numRegs > 0 && smem_sm > 0) {
      const int threads = 32 * warps;
      int ctas = 65536 / (fa.numRegs * threads);
      if (ctas < 1) ctas = 1;
      const size_t need = (size_t)ctas * (fa.sharedSizeBytes + *bytes + 1024);
      pct = (int)((need * 100 + smem_sm - 1) / smem_sm);
      if (pct > 100) pct = 100;
    }
    cudaGetLastError();
    it = pct_of.emplace(key, pct).first;
  }
  if (it->second >= 0) {
    auto s = set_to.find(key.first);
    if (s == set_to.end() || s->second != it->second) {
      if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, it->second) == cudaSuccess)
        set_to[key.first] = it->second;
      cudaGetLastError();
    }
  }
  return cudaSuccess;
}

template <int N, int L>
static cudaError_t launch_mesh_NL(const PlanView& pv, const uint64_t* g, const void* scales, size_t scale_pitch,
                                  void* s, size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status,
                                  int warps, cudaStream_t st) {
  constexpr int TAPS = (N + 1) * (N + 1) * (N + 1) * (N + 1);
  if (warps > mesh_max_warps(N)) warps = mesh_max_warps(N);
  const long long grid = (long long)((pv.W + 31) / 32) * ((pv.H + warps - 1) / warps);
  const int block = 32 * warps;
  const bool fast = N >= 2 && mesh_fast_ok(pv);
  auto go = [&](auto kernel) -> cudaError_t {
    size_t smem = 0;
    cudaError_t e = tap_smem(kernel, TAPS, warps, &smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, block, smem, st>>>(pv, g, (const float4*)scales, scale_pitch, s, s_pitch, num, num_pitch, status);
    return cudaGetLastError();
  };
  if (pv.dbg) {
    if constexpr (N == 3) return fast ? go(mesh_exact_kernel3<L, true, true>) : go(mesh_exact_kernel3<L, false, true>);
    else if constexpr (N == 2)
      return fast ? go(mesh_exact_kernel<N, L, true, true>) : go(mesh_exact_kernel<N, L, false, true>);
    else return go(mesh_exact_kernel<N, L, false, true>);
  }
  if constexpr (N == 3) return fast ? go(mesh_exact_kernel3<L, true, false>) : go(mesh_exact_kernel3<L, false, false>);
  else if constexpr (N == 2)
    return fast ? go(mesh_exact_kernel<N, L, true, false>) : go(mesh_exact_kernel<N, L, false, false>);
  else return go(mesh_exact_kernel<N, L, false, false>);
}

template <int N>
static cudaError_t launch_mesh_N(const PlanView& pv, const uint64_t* g, const void* scales, size_t scale_pitch,
                                 void* s, size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status,
                                 int warps, cudaStream_t st) {
  switch (pv.limbs) {
    case 1: return launch_mesh_NL<N, 1>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, warps, st);
    case 2: return launch_mesh_NL<N, 2>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, warps, st);
    case 3: return launch_mesh_NL<N, 3>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, warps, st);
    default: return launch_mesh_NL<N, 4>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, warps, st);
  }
}

// warps: rows per CTA (4..16; out of range falls back to the default).
cudaError_t run_mesh_exact(const PlanView& pv, const uint64_t* g, const void* scales, size_t scale_pitch, void* s,
                           size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status, int warps,
                           cudaStream_t st) {
  if (warps < 1 || warps > kMeshWarpsMax) warps = kMeshWarps;
  switch (pv.n) {
    case 1: return launch_mesh_N<1>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, warps, st);
    case 2: return launch_mesh_N<2>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, warps, st);
    default: return launch_mesh_N<3>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, warps, st);
  }
}

// Host side of the batched launch: order the images by cost (order n, then
// pixels), number their runs, and launch persistent CTAs over them.
int batch_max_jobs() { return kMaxBatch; }

template <int N, int L, bool FAST>
static cudaError_t launch_batch_NL(const BatchJobs& jobs, unsigned long long* counter, int warps,
                                   cudaStream_t st) {
  constexpr int TAPS = (N + 1) * (N + 1) * (N + 1) * (N + 1);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  auto go = [&](auto kernel) -> cudaError_t {
    size_t smem = 0;
    cudaError_t e2 = tap_smem(kernel, TAPS, warps, &smem);
    if (e2 != cudaSuccess) return e2;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * warps, smem);
    if (per_sm < 1) per_sm = 1;
    kernel<<<sms * per_sm, 32 * warps, smem, st>>>(jobs, counter, warps);
    return cudaGetLastError();
  };
  if constexpr (N == 3) return go(mesh_batch_kernel3<L, FAST>);
  else return go(mesh_batch_kernel<N, L, FAST>);
}

template <int N, bool FAST>
static cudaError_t launch_batch_N(int L, const BatchJobs& jobs, unsigned long long* counter, int warps,
                                  cudaStream_t st) {
  switch (L) {
    case 1: return launch_batch_NL<N, 1, FAST>(jobs, counter, warps, st);
    case 2: return launch_batch_NL<N, 2, FAST>(jobs, counter, warps, st);
    case 3: return launch_batch_NL<N, 3, FAST>(jobs, counter, warps, st);
    default: return launch_batch_NL<N, 4, FAST>(jobs, counter, warps, st);
  }
}

// One persistent launch per (order n, limbs, fast path or not) present, most
// expensive first; counter: 32 64-bit counters (one per launch), device memory.
cudaError_t run_mesh_batch(const BatchIn* in, int njobs, unsigned long long* counter, int warps, cudaStream_t st) {
  if (warps < 1 || warps > kMeshWarpsMax) warps = kMeshWarps;
  auto cost = [&](int i) { return (double)in[i].pv.W * in[i].pv.H; };
  int launch = 0;
  for (int n = 3; n >= 1; --n) {
    const int wn = warps < mesh_max_warps(n) ? warps : mesh_max_warps(n);  // rows per unit
    for (int L = 4; L >= 1; --L) {
      for (int fast = 1; fast >= 0; --fast) {
        if (fast && n == 1) continue;
        int order[kMaxBatch];
        int m = 0;
        for (int i = 0; i < njobs; ++i)
          if (in[i].pv.n == n && in[i].pv.limbs == L && (mesh_fast_ok(in[i].pv) ? 1 : 0) == fast) order[m++] = i;
        if (m == 0) continue;
        for (int i = 1; i < m; ++i)
          for (int j = i; j > 0 && cost(order[j]) > cost(order[j - 1]); --j) {
            const int t = order[j];
            order[j] = order[j - 1];
            order[j - 1] = t;
          }
        BatchJobs jobs;
        jobs.njobs = m;
        long long units = 0;
        for (int k = 0; k < m; ++k) {
          const BatchIn& b = in[order[k]];
          BatchJob& jb = jobs.job[k];
          jb.pv = b.pv;
          jb.g = b.g;
          jb.scales = (const float4*)b.scales;
          jb.scale_pitch = b.scale_pitch;
          jb.s = b.s;
          jb.s_pitch = b.s_pitch;
          jb.status = b.status;
          jb.segs = (b.pv.W + 31) / 32;
          jb.units_begin = units;
          units += (long long)jb.segs * ((b.pv.H + wn - 1) / wn) * wn;  // one item per row run
        }
        jobs.total_units = units;
        unsigned long long* ctr = counter + launch++;
        cudaError_t e;
        if (n == 1) e = launch_batch_N<1, false>(L, jobs, ctr, wn, st);
        else if (n == 2) e = fast ? launch_batch_N<2, true>(L, jobs, ctr, wn, st)
                                  : launch_batch_N<2, false>(L, jobs, ctr, wn, st);
        else e = fast ? launch_batch_N<3, true>(L, jobs, ctr, wn, st)
                      : launch_batch_N<3, false>(L, jobs, ctr, wn, st);
        if (e != cudaSuccess) return e;
      }
    }
  }
  return cudaSuccess;
}

cudaError_t run_prepare_scales(const PlanView& pv, const void* scales, size_t scale_pitch, void* C, size_t C_pitch,
                               int32_t* status, cudaStream_t st) {
  dim3 block(32, 4);
  dim3 grid((pv.W + 31) / 32, (pv.H + 3) / 4);
  prepare_scales_kernel<<<grid, block, 0, st>>>(pv, (const float4*)scales, scale_pitch, (int4*)C, C_pitch, status);
  return cudaGetLastError();
}

}  // namespace abf
