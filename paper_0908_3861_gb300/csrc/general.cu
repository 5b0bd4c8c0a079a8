// Generalised plans: the directional order N = 2 and the B-spline model phi.
//
// Sec. 4 Eq. (def) builds beta^N_a from the directions theta_k = (k-1) pi/N;
// the RS filters of Eq. (RS_filter) exist on the lattice only when
// b cos theta and b sin theta are integers, which among N >= 2 holds for
// N = 4 (Sec. 7, the plain plans) and N = 2: theta = 0, pi/2, b = (1, 1), the
// tensor box splines (Sec. 4: rect = beta^2_(1,1)).  N = 2 uses the directions
// v1 and v3 alone: running sums and FD only along them.
//
// Sec. 6 writes the image as f(x) = sum_k c[k] phi(x - k), c = f * (b^n)^-1;
// Eq. (NA) without interpolation runs the running sums on c and Eq. (mask)
// interpolates with phi * beta^N_b.  Here phi = beta^{E-1}(x1) beta^{E-1}(x2),
// E unit boxes per axis (a reading: Sec. 6 leaves phi open), so the
// interpolation kernel is the box spline with the lattice directions v_k taken
// r_k + (E along v1 and v3) times.  For E >= 3 (degree >= 2) c is irrational:
// c_q = rint(c 2^F) is computed by the separable prefilter (the 1-D filter's
// recursions along rows, unrounded, then along columns, rounded) on a frame
// that extends T samples beyond every image edge, and the method runs exactly
// on c_q.
//
// Every tap lies on the 2^-(Q+1) grid (P = Q + 1: tau = (1/2) sum_k r_k (c_k -
// 1) v_k and the kernel's centre are half-integers at most), where D M is an
// integer (D = D0 2^((sum m - 2) P), the refinement equation); the table holds
// one row per fractional offset r in [0, 1)^2 (p = floor(y)) with the
// neighbours d that carry a weight.  The numerator S = D sum_j w_j g_I(y_j) is
// formed modulo 2^(64 L) as in the plain form, and
// s = S 2^(Q sum r - F) / (D prod_k C_k^{r_k}).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "abf_internal.cuh"

namespace abf {
cudaError_t run_integrate(const PlanView& pv, const void* f, size_t f_pitch, uint64_t* g, void* ws,
                          uint32_t* epoch, int32_t* status, cudaStream_t st);
size_t line_ws_bytes(int Gw, int Gh, int L, int n, int* nbands_out, int* nlines_out);

constexpr int kGenMaxR = 256;    // neighbours per table row
constexpr int kGenMaxTaps = 81;  // prod_k (r_k + 1)
constexpr int kGenWarps = 8;     // rows per CTA

// ------------------------------------------------------------- mesh kernels

// The taps j = (j1..j4) of a plan ordered by their FD weight
// w_j = prod_k (-1)^{j_k} binom(r_k, j_k) (Eq. (RS_filter)), one group per
// distinct weight, each tap's j packed two bits per direction (r_k <= 3).
// Built on the host with the plan; a CTA copies it into shared memory.
struct GenTaps {
  int taps, ng;
  int gbeg[12], gw[11];
  unsigned char order[84];
};
static_assert(sizeof(GenTaps) % 4 == 0 && kGenMaxTaps <= 84, "GenTaps is copied as 32-bit words");

struct GenShared {
  GenTaps t;
  int2 st[kGenMaxR];
};

__device__ __forceinline__ void gen_setup(const PlanView& pv, GenShared& sh) {
  const int* src = reinterpret_cast<const int*>(pv.gtaps);
  int* dst = reinterpret_cast<int*>(&sh.t);
  for (int i = threadIdx.x; i < (int)(sizeof(GenTaps) / 4); i += blockDim.x) dst[i] = src[i];
  for (int i = threadIdx.x; i < pv.R; i += blockDim.x) sh.st[i] = pv.stencil[i];
}

// This lane's pixel -> integer steps C_k and a verdict: 0 outside the image,
// 1 good, 2 numerator bound beyond 64 L - 1 bits, 3 bad scale.
template <int L>
__device__ __forceinline__ int gen_lane_steps(const PlanView& pv, const float4* scales, size_t scale_pitch, int x, int y,
                                              int C[4]) {
  C[0] = C[1] = C[2] = C[3] = 0;
  if (x >= pv.W) return 0;
  if (!pixel_steps(pv, scales, scale_pitch, x, y, C)) return 3;
  float lb = pv.log2_base;
  for (int k = 0; k < 4; ++k) lb += (float)pv.r[k] * (__log2f((float)C[k]) - (float)pv.Q);
  if (pv.E == 0) {
    const float q = (float)(1 << pv.Q);
    lb += __log2f((1.0f + q / (float)C[0]) * (1.0f + q / (float)C[2]));
  }
  return (lb + 0.05f < 64.0f * L - 1.0f) ? 1 : 2;
}

// Stores the numerator and s = S 2^(Q sum r - F) / (D prod_k C_k^{r_k}) of the
// lane's pixel (NaN and a device status for a refused pixel).
template <int L>
__device__ __forceinline__ void gen_store(const PlanView& pv, void* s, size_t s_pitch, uint64_t* num, size_t num_pitch,
                                          int32_t* status, int x, int y, int ok, const int C[4], const Wide<L>& S) {
  if (x >= pv.W) return;
  const bool f64 = pv.out_dtype == ABF_F64;
  char* row = s ? reinterpret_cast<char*>(s) + (size_t)y * s_pitch : nullptr;
  if (ok != 1) {
    raise_status(status, ok == 3 ? ABF_DEV_BAD_SCALE : ABF_DEV_RANGE);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    if (row) {
      if (f64) reinterpret_cast<double*>(row)[x] = nan;
      else reinterpret_cast<float*>(row)[x] = (float)nan;
    }
    return;
  }
  if (num) {
    uint64_t* q = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(num) + (size_t)y * num_pitch) + (size_t)x * L;
#pragma unroll
    for (int i = 0; i < L; ++i) q[i] = S.w[i];
  }
  if (row) {
    // s = S (2^(Q sum r - F) / D) / prod_k C_k^{r_k}; the product in 64-bit
    // integers where it fits (one conversion instead of a binary64 product)
    double den;
    if (pv.den_int) {
      uint64_t p = 1;
      for (int k = 0; k < 4; ++k)
        for (int e = 0; e < pv.r[k]; ++e) p *= (uint64_t)C[k];
      den = (double)p;
    } else {
      den = 1.0;
      for (int k = 0; k < 4; ++k)
        for (int e = 0; e < pv.r[k]; ++e) den *= (double)C[k];
    }
    const double v = (wto_double<L>(S) * pv.out_scale) / den;
    if (f64) reinterpret_cast<double*>(row)[x] = v;
    else reinterpret_cast<float*>(row)[x] = (float)v;
  }
}

// acc += w part for the FD weight w of a tap group.
template <int L>
__device__ __forceinline__ void gen_apply_weight(Wide<L>& acc, const Wide<L>& part, int w) {
  Wide<L> sc;
  wzero<L>(sc);
  wmac<L>(sc, part, (uint64_t)(w < 0 ? -w : w));
  if (w < 0) wsub<L>(acc, sc);
  else wadd<L>(acc, sc);
}

// Wide stencils (R > 64 neighbours): one warp per run of 32 pixels of a row,
// as the plain form's generic path.  Lane i reads pixel x0 + i's steps; for
// each pixel of the run the lanes tabulate its taps (grouped by FD weight) in
// shared memory and then deal the (tap, neighbour) pairs of each group among
// themselves.
template <int L, typename WT, bool DBG>
__global__ void __launch_bounds__(32 * kGenWarps) mesh_gen_kernel(
    const PlanView pv, const uint64_t* __restrict__ g, const float4* __restrict__ scales, size_t scale_pitch,
    void* __restrict__ s, size_t s_pitch, uint64_t* __restrict__ num, size_t num_pitch, int32_t* status) {
  __shared__ GenShared sh;
  __shared__ int4 s_tap[kGenWarps][kGenMaxTaps];
  gen_setup(pv, sh);
  __syncthreads();
  const int R = pv.R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int y = blockIdx.y * kGenWarps + warp;
  if (y >= pv.H) return;
  const int x0 = blockIdx.x * 32;
  const int myx = x0 + lane;
  const int Q = pv.Q, P = pv.P, one = 1 << Q, mask = (1 << P) - 1;
  const int r0 = pv.r[0], r1 = pv.r[1], r3 = pv.r[3], r2 = pv.r[2];
  int C[4];
  const int ok = gen_lane_steps<L>(pv, scales, scale_pitch, myx, y, C);
  const WT* __restrict__ table = reinterpret_cast<const WT*>(pv.table);
  const int taps = sh.t.taps, ng = sh.t.ng;
  int4* tp = s_tap[warp];
  Wide<L> mine;
  wzero<L>(mine);
  for (int pp = 0; pp < 32; ++pp) {
    if (__shfl_sync(0xffffffffu, ok, pp) != 1) continue;
    const int c0 = __shfl_sync(0xffffffffu, C[0], pp), c1 = __shfl_sync(0xffffffffu, C[1], pp);
    const int c2 = __shfl_sync(0xffffffffu, C[2], pp), c3 = __shfl_sync(0xffffffffu, C[3], pp);
    // tau 2^P = sum_k r_k (C_k - 2^Q) v_k; c_k 2^P = 2 C_k
    const int tx = r0 * (c0 - one) + r1 * (c1 - one) - r3 * (c3 - one);
    const int ty = r1 * (c1 - one) + r2 * (c2 - one) + r3 * (c3 - one);
    const int Y0x = ((x0 + pp + pv.ox) << P) + tx;
    const int Y0y = ((y + pv.oy) << P) + ty;
    __syncwarp();
    for (int slot = lane; slot < taps; slot += 32) {
      const int u = sh.t.order[slot];
      const int j1 = u & 3, j2 = (u >> 2) & 3, j3 = (u >> 4) & 3, j4 = u >> 6;
      const int Yx = Y0x - 2 * (j1 * c0 + j2 * c1 - j4 * c3);
      const int Yy = Y0y - 2 * (j2 * c1 + j3 * c2 + j4 * c3);
      tp[slot] = make_int4((Yx >> P) + pv.left, Yy >> P, ((Yy & mask) << P) | (Yx & mask), 0);
    }
    __syncwarp();
    Wide<L> acc;
    wzero<L>(acc);
    for (int gi = 0; gi < ng; ++gi) {
      const int tb = sh.t.gbeg[gi], npairs = (sh.t.gbeg[gi + 1] - tb) * R;
      Wide<L> part;
      wzero<L>(part);
      for (int idx = lane; idx < npairs; idx += 32) {
        const int q = idx / R;
        const int cand = idx - q * R;
        const int4 ti = tp[tb + q];
        const int2 d = sh.st[cand];
        const int k2 = ti.y + d.y;
        if (k2 < 0) continue;  // rows below the box: g = 0
        if (DBG && !dbg_tap_ok(pv, status, ti.x, ti.y, d.x, d.x, d.y, x0 + pp, y)) continue;
        const Wide<L> gv = wload<L>(g + ((size_t)k2 * (size_t)pv.Gp + (size_t)(ti.x + d.x)) * L);
        mac_weight<L, WT>(part, gv, __ldg(table + (size_t)ti.z * R + cand));
      }
      gen_apply_weight<L>(acc, part, sh.t.gw[gi]);
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
  gen_store<L>(pv, s, s_pitch, num, num_pitch, status, myx, y, ok, C, mine);
}

// Bounds checking for one lane and pixel: the taps y0 - sum_k j_k c_k v_k,
// 0 <= j_k <= r_k, span columns from the all-v1-and-v2 corner to the all-v4
// corner and rows up to y0 itself; with the lane's neighbour d added, that
// span must lie in the lattice box (rows below 0 are never read).
__device__ __forceinline__ bool gen_dbg_lane(const PlanView& pv, int32_t* status, int Y0x, int Y0y, int c0, int c1,
                                             int c2, int c3, int2 d, int P, int x, int y) {
  (void)c2;
  const int xlo = ((Y0x - 2 * (pv.r[0] * c0 + pv.r[1] * c1)) >> P) + pv.left;
  const int xhi = ((Y0x + 2 * pv.r[3] * c3) >> P) + pv.left;
  return dbg_tap_ok(pv, status, xlo, Y0y >> P, d.x, d.x + (xhi - xlo), d.y, x, y);
}

// One pixel's share of a lane for N = 2, r = (NN, 0, NN, 0): the (NN + 1)^2
// taps y_j = y0 - j1 c1 v1 - j3 c3 v3 in unrolled loops (positions stepped, no
// tap table), each tap's product accumulated by its FD weight class: |w_j| =
// NN^i with i = #{j1, j3 strictly inside 0..NN} (binom(NN, 1) = binom(NN,
// NN - 1) = NN), the sign (-1)^(j1 + j3); the classes are combined at the end.
template <int L, typename WT, int NN>
__device__ __forceinline__ void gen2_pixel(Wide<L>& acc, const PlanView& pv, const uint64_t* __restrict__ g,
                                           const WT* __restrict__ table, int R, int gl, int2 d, int Y0x, int Y0y,
                                           int c0, int c2, int P, int mask) {
  constexpr int K = NN >= 2 ? 3 : 1;
  Wide<L> ap[K], an[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    wzero<L>(ap[i]);
    wzero<L>(an[i]);
  }
  const int xoff = pv.left + d.x;
#pragma unroll
  for (int j3 = 0; j3 <= NN; ++j3) {
    const int Yy = Y0y - 2 * j3 * c2;
    const int k2 = (Yy >> P) + d.y;
    if (k2 < 0) continue;  // taps below the box: g = 0
    const uint64_t* grow = g + (size_t)k2 * (size_t)pv.Gp * L;
    const WT* trow = table + (size_t)((Yy & mask) << P) * R + gl;
#pragma unroll
    for (int j1 = 0; j1 <= NN; ++j1) {
      const int Yx = Y0x - 2 * j1 * c0;
      const Wide<L> gv = wload<L>(grow + (size_t)((Yx >> P) + xoff) * L);
      const WT wt = __ldg(trow + (size_t)(Yx & mask) * R);
      const int cls = (j1 > 0 && j1 < NN ? 1 : 0) + (j3 > 0 && j3 < NN ? 1 : 0);
      if ((j1 + j3) & 1) mac_weight<L, WT>(an[cls], gv, wt);
      else mac_weight<L, WT>(ap[cls], gv, wt);
    }
  }
  uint64_t m = 1;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    wsub<L>(ap[i], an[i]);
    wmac<L>(acc, ap[i], m);
    m *= (uint64_t)NN;
  }
}

// Stencils of up to 64 neighbours (e.g. the 2 x 2 of N = 2, n = 2): the warp
// owns a run of 32 pixels of a row and works in groups of G lanes, one pixel
// per group, 32 / G neighbouring pixels at once; lane k of a group takes
// neighbour k (and k + 32 when R > 32) of every tap (its table weight is word k of the tap's
// row, so a group reads one contiguous row piece), computes the tap positions
// itself (no shared tap table) and the group sums its lanes by butterfly.
// After each round the group leaders hand the numerators to the lanes that
// own those pixels.
template <int L, typename WT, int G, int NN, int CANDS, bool DBG>
__global__ void __launch_bounds__(32 * kGenWarps) mesh_gen_group_kernel(
    const PlanView pv, const uint64_t* __restrict__ g, const float4* __restrict__ scales, size_t scale_pitch,
    void* __restrict__ s, size_t s_pitch, uint64_t* __restrict__ num, size_t num_pitch, int32_t* status) {
  static_assert(G == 4 || G == 16 || G == 32, "group of 4, 16 or 32 lanes");
  static_assert(CANDS == 1 || (CANDS == 2 && G == 32 && NN == 0), "two neighbours per lane: whole-warp groups");
  constexpr int PPR = 32 / G;  // pixels per round
  __shared__ GenShared sh;
  gen_setup(pv, sh);
  __syncthreads();
  const int R = pv.R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int y = blockIdx.y * kGenWarps + warp;
  if (y >= pv.H) return;
  const int x0 = blockIdx.x * 32;
  const int myx = x0 + lane;
  const int Q = pv.Q, P = pv.P, one = 1 << Q, mask = (1 << P) - 1;
  const int r0 = pv.r[0], r1 = pv.r[1], r3 = pv.r[3], r2 = pv.r[2];
  int C[4];
  const int ok = gen_lane_steps<L>(pv, scales, scale_pitch, myx, y, C);
  const WT* __restrict__ table = reinterpret_cast<const WT*>(pv.table);
  const int ng = sh.t.ng;
  const int grp = lane / G, gl = lane % G;
  const bool has_d = gl < R;
  const int2 d = has_d ? sh.st[gl] : make_int2(0, 0);
  const bool has_d2 = CANDS == 2 && gl + G < R;  // a second neighbour (R > 32)
  const int2 d2 = has_d2 ? sh.st[gl + G] : make_int2(0, 0);
  const long long Gp = pv.Gp;
  Wide<L> mine;
  wzero<L>(mine);
  for (int q = 0; q < G; ++q) {
    const int pp = q * PPR + grp;
    const int okp = __shfl_sync(0xffffffffu, ok, pp);
    const int c0 = __shfl_sync(0xffffffffu, C[0], pp), c1 = __shfl_sync(0xffffffffu, C[1], pp);
    const int c2 = __shfl_sync(0xffffffffu, C[2], pp), c3 = __shfl_sync(0xffffffffu, C[3], pp);
    Wide<L> acc;
    wzero<L>(acc);
    if (okp == 1 && has_d) {
      const int tx = r0 * (c0 - one) + r1 * (c1 - one) - r3 * (c3 - one);
      const int ty = r1 * (c1 - one) + r2 * (c2 - one) + r3 * (c3 - one);
      const int Y0x = ((x0 + pp + pv.ox) << P) + tx;
      const int Y0y = ((y + pv.oy) << P) + ty;
      // bounds checking: this lane's reads of the pixel (all taps, its
      // neighbours) must stay in the box, else the lane reads nothing for it
      const bool skip =
          DBG && (!gen_dbg_lane(pv, status, Y0x, Y0y, c0, c1, c2, c3, d, P, x0 + pp, y) ||
                     (CANDS == 2 && has_d2 && !gen_dbg_lane(pv, status, Y0x, Y0y, c0, c1, c2, c3, d2, P, x0 + pp, y)));
      if (skip) {
      } else if constexpr (NN > 0) {
        gen2_pixel<L, WT, NN>(acc, pv, g, table, R, gl, d, Y0x, Y0y, c0, c2, P, mask);
      } else {
      for (int gi = 0; gi < ng; ++gi) {
        Wide<L> part;
        wzero<L>(part);
        const int te = sh.t.gbeg[gi + 1];
        for (int slot = sh.t.gbeg[gi]; slot < te; ++slot) {
          const int u = sh.t.order[slot];
          const int j1 = u & 3, j2 = (u >> 2) & 3, j3 = (u >> 4) & 3, j4 = u >> 6;
          const int Yx = Y0x - 2 * (j1 * c0 + j2 * c1 - j4 * c3);
          const int Yy = Y0y - 2 * (j2 * c1 + j3 * c2 + j4 * c3);
          const int py = Yy >> P, px = (Yx >> P) + pv.left;
          const WT* trow = table + (size_t)(((Yy & mask) << P) | (Yx & mask)) * R;
          const int k2 = py + d.y;
          if (k2 >= 0) {  // rows below the box: g = 0
            const Wide<L> gv = wload<L>(g + ((size_t)k2 * Gp + (size_t)(px + d.x)) * L);
            mac_weight<L, WT>(part, gv, __ldg(trow + gl));
          }
          if constexpr (CANDS == 2) {
            const int k2b = py + d2.y;
            if (has_d2 && k2b >= 0) {
              const Wide<L> gv = wload<L>(g + ((size_t)k2b * Gp + (size_t)(px + d2.x)) * L);
              mac_weight<L, WT>(part, gv, __ldg(trow + gl + G));
            }
          }
        }
        gen_apply_weight<L>(acc, part, sh.t.gw[gi]);
      }
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      Wide<L> other;
#pragma unroll
      for (int i = 0; i < L; ++i) other.w[i] = __shfl_xor_sync(0xffffffffu, acc.w[i], o);
      wadd<L>(acc, other);
    }
    // lane l's pixel was this round's if l / PPR == q, summed by group l % PPR
    Wide<L> t;
#pragma unroll
    for (int i = 0; i < L; ++i) t.w[i] = __shfl_sync(0xffffffffu, acc.w[i], (lane % PPR) * G);
    if (lane / PPR == q) mine = t;
  }
  gen_store<L>(pv, s, s_pitch, num, num_pitch, status, myx, y, ok, C, mine);
}

// Lanes per pixel for a table of R neighbours: a group of 4 (the 2 x 2 stencil
// of N = 2, n = 2), 16 (3 x 3 and 4 x 4) or the whole warp (up to 32 lanes with
// one neighbour each, up to 64 with two), else 0 (the pair-dealt warp kernel).
static int gen_group_lanes(int R) { return R <= 4 ? 4 : R <= 16 ? 16 : R <= 64 ? 32 : 0; }

template <int L, typename WT, int NN, bool DBG>
static void launch_gen_group(int G, dim3 grid, const PlanView& pv, const uint64_t* g, const float4* sc,
                             size_t scale_pitch, void* s, size_t s_pitch, uint64_t* num, size_t num_pitch,
                             int32_t* status, cudaStream_t st) {
  if (G == 4)
    mesh_gen_group_kernel<L, WT, 4, NN, 1, DBG><<<grid, 32 * kGenWarps, 0, st>>>(pv, g, sc, scale_pitch, s, s_pitch,
                                                                                num, num_pitch, status);
  else if (G == 16)
    mesh_gen_group_kernel<L, WT, 16, NN, 1, DBG><<<grid, 32 * kGenWarps, 0, st>>>(pv, g, sc, scale_pitch, s, s_pitch,
                                                                                 num, num_pitch, status);
  else if (NN > 0 || pv.R <= 32)
    mesh_gen_group_kernel<L, WT, 32, NN, 1, DBG><<<grid, 32 * kGenWarps, 0, st>>>(pv, g, sc, scale_pitch, s, s_pitch,
                                                                                 num, num_pitch, status);
  else if constexpr (NN == 0)
    mesh_gen_group_kernel<L, WT, 32, 0, 2, DBG><<<grid, 32 * kGenWarps, 0, st>>>(pv, g, sc, scale_pitch, s, s_pitch,
                                                                                num, num_pitch, status);
}

// N = 2 (r = (n, 0, n, 0)) with up to 32 neighbours, 8-byte weights and at most
// two limbs takes the unrolled tap loops of gen2_pixel; other plans with up to
// 64 neighbours the run-time tap groups (two neighbours per lane above 32);
// wider stencils the pair-dealt warp kernel.
template <int L, typename WT, bool DBG>
static void launch_gen_WT(const PlanView& pv, const uint64_t* g, const void* scales, size_t scale_pitch, void* s,
                          size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status, cudaStream_t st) {
  dim3 grid((unsigned)((pv.W + 31) / 32), (unsigned)((pv.H + kGenWarps - 1) / kGenWarps));
  const float4* sc = (const float4*)scales;
  const int G = gen_group_lanes(pv.R);
  if (G == 0) {
    mesh_gen_kernel<L, WT, DBG><<<grid, 32 * kGenWarps, 0, st>>>(pv, g, sc, scale_pitch, s, s_pitch, num, num_pitch,
                                                                status);
    return;
  }
  const bool n2 = pv.r[1] == 0 && pv.r[3] == 0 && pv.r[0] == pv.r[2] && pv.r[0] >= 1 && pv.r[0] <= 3 && pv.R <= 32;
  if constexpr (L <= 2 && sizeof(WT) == 8) {
    if (n2) {
      if (pv.r[0] == 1) launch_gen_group<L, WT, 1, DBG>(G, grid, pv, g, sc, scale_pitch, s, s_pitch, num, num_pitch, status, st);
      else if (pv.r[0] == 2) launch_gen_group<L, WT, 2, DBG>(G, grid, pv, g, sc, scale_pitch, s, s_pitch, num, num_pitch, status, st);
      else launch_gen_group<L, WT, 3, DBG>(G, grid, pv, g, sc, scale_pitch, s, s_pitch, num, num_pitch, status, st);
      return;
    }
  }
  launch_gen_group<L, WT, 0, DBG>(G, grid, pv, g, sc, scale_pitch, s, s_pitch, num, num_pitch, status, st);
}

template <int L>
static cudaError_t launch_gen_L(const PlanView& pv, const uint64_t* g, const void* scales, size_t scale_pitch, void* s,
                                size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status, cudaStream_t st) {
  const bool w16 = pv.table_bytes_per_w == 16;
  if (pv.dbg) {
    if (w16) launch_gen_WT<L, ulonglong2, true>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
    else launch_gen_WT<L, uint64_t, true>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
  } else {
    if (w16) launch_gen_WT<L, ulonglong2, false>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
    else launch_gen_WT<L, uint64_t, false>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
  }
  return cudaGetLastError();
}

cudaError_t run_mesh_general(const PlanView& pv, const uint64_t* g, const void* scales, size_t scale_pitch, void* s,
                             size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status, cudaStream_t st) {
  switch (pv.limbs) {
    case 1: return launch_gen_L<1>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
    case 2: return launch_gen_L<2>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
    case 3: return launch_gen_L<3>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
    default: return launch_gen_L<4>(pv, g, scales, scale_pitch, s, s_pitch, num, num_pitch, status, st);
  }
}

// ------------------------------------------------- prefilter, column pass

// The second pass of the separable prefilter: along every column of the row
// pass' output x (c_row 2^(F + G - 4), rows 0 .. H-1, zero above and below),
// the causal and anti-causal recursions of each pole run over the whole
// extended column, rows -T .. H+T-1; c 2^(F + G - 8) = sum_p A_p (y+ - x + y-)
// is rounded to c_q = rint(c 2^F), ties to even.  One thread per column (the
// warp's loads and stores are consecutive columns); the causal sums wait in
// yf (npoles planes of (H + 2T) x W elements).
__global__ void prefilter_cols_kernel(const PrefilterView v, int H, int T, int W, const long long* __restrict__ x,
                                      long long x_pitch, long long* __restrict__ yf, long long* __restrict__ c,
                                      long long c_pitch) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= W) return;
  const int He = H + 2 * T;
  const size_t plane = (size_t)He * W;
  auto xin = [&](int ye) -> long long {
    const int y = ye - T;
    return (y >= 0 && y < H) ? x[(size_t)y * x_pitch + col] : 0ll;
  };
  for (int p = 0; p < v.npoles; ++p) {
    long long y1 = 0;
    const long long Z = v.Z[p];
    for (int ye = 0; ye < He; ++ye) {
      y1 = xin(ye) + __mul64hi(y1, Z);
      yf[p * plane + (size_t)ye * W + col] = y1;
    }
  }
  long long yb[kPfMaxPoles] = {0, 0};
  const int sh = v.G - 8;
  const long long half = 1ll << (sh - 1);
  for (int ye = He - 1; ye >= 0; --ye) {
    const long long xv = xin(ye);
    long long acc = 0;
    for (int p = 0; p < v.npoles; ++p) {
      yb[p] = xv + __mul64hi(yb[p], v.Z[p]);
      acc += __mul64hi(yf[p * plane + (size_t)ye * W + col] - xv, v.A[p]) + __mul64hi(yb[p], v.A[p]);
    }
    long long q = acc >> sh;  // floor
    const long long rem = acc - q * (1ll << sh);
    if (rem > half || (rem == half && (q & 1))) ++q;
    c[(size_t)ye * c_pitch + col] = q;
  }
}

}  // namespace abf

// ---------------------------------------------------------------- host side

using u128 = unsigned __int128;

namespace {

struct GenTable {
  std::vector<uint8_t> bytes;  // (2^P)^2 rows x R weights, little-endian
  std::vector<int2> stencil;   // the R neighbours (dx, dy)
  u128 D = 0;
  int wbytes = 0;
};

u128 gcd_u128(u128 a, u128 b) {
  while (b) {
    const u128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// The box spline M with the lattice directions v1..v4 taken m_k times: its
// values at the integer points (the eigenvector of the refinement equation
// restricted to them, found in floating point, snapped to a rational with
// denominator 2 (N-2)! 2^t and verified exactly), refined to the 2^-P grid
// (M(y) = 2^(2-N) sum_k a_k M(2y - k), a = the coefficients of
// prod_k (1 + z^{v_k})^{m_k}), then one row per fractional offset.
bool build_gen_table(const int m[4], int P, GenTable& out) {
  const int V[4][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 1}};
  const int N = m[0] + m[1] + m[2] + m[3];
  const int x0 = -m[3], x1 = m[0] + m[1], y1 = m[1] + m[2] + m[3];
  const int mw = x1 - x0 + 1, mh = y1 + 1;
  std::vector<int64_t> a((size_t)mw * mh, 0);
  a[(size_t)(0 - x0)] = 1;
  for (int k = 0; k < 4; ++k)
    for (int rep = 0; rep < m[k]; ++rep) {
      std::vector<int64_t> b = a;
      for (int y = 0; y < mh; ++y)
        for (int xi = 0; xi < mw; ++xi) {
          const int64_t v = a[(size_t)y * mw + xi];
          if (!v) continue;
          const int nx = xi + V[k][0], ny = y + V[k][1];
          if (nx < 0 || nx >= mw || ny >= mh) return false;
          b[(size_t)ny * mw + nx] += v;
        }
      a.swap(b);
    }
  auto mask_at = [&](int kx, int ky) -> int64_t {
    const int xi = kx - x0;
    if (xi < 0 || xi >= mw || ky < 0 || ky >= mh) return 0;
    return a[(size_t)ky * mw + xi];
  };
  const int npts = mw * mh;
  std::vector<long double> v(npts, 1.0L / npts), nv(npts);
  for (int it = 0; it < 600; ++it) {
    long double sum = 0;
    for (int p = 0; p < npts; ++p) {
      const int px = p % mw + x0, py = p / mw;
      long double acc = 0;
      for (int q = 0; q < npts; ++q) {
        const int64_t c = mask_at(2 * px - (q % mw + x0), 2 * py - q / mw);
        if (c) acc += (long double)c * v[q];
      }
      nv[p] = acc;
      sum += acc;
    }
    for (int p = 0; p < npts; ++p) v[p] = nv[p] / sum;
  }
  u128 Dc = 2;
  for (int i = 2; i <= N - 2; ++i) Dc *= (u128)i;
  std::vector<u128> Vq(npts);
  bool ok = false;
  for (int attempt = 0; attempt < 8 && !ok; ++attempt, Dc *= 2) {
    ok = true;
    u128 sum = 0;
    for (int p = 0; p < npts; ++p) {
      const long double xv = v[p] * (long double)Dc;
      const long double r = std::floor(xv + 0.5L);
      if (std::fabs((double)(xv - r)) > 1e-3 || r < 0) { ok = false; break; }
      Vq[p] = (u128)r;
      sum += Vq[p];
    }
    if (!ok || sum != Dc) { ok = false; continue; }
    const u128 scale = (u128)1 << (N - 2);
    for (int p = 0; p < npts && ok; ++p) {
      const int px = p % mw + x0, py = p / mw;
      u128 acc = 0;
      for (int q = 0; q < npts; ++q) {
        const int64_t c = mask_at(2 * px - (q % mw + x0), 2 * py - q / mw);
        if (c) acc += (u128)c * Vq[q];
      }
      if (acc != scale * Vq[p]) ok = false;
    }
  }
  if (!ok) return false;
  u128 gg = 0;
  for (int p = 0; p < npts; ++p) gg = gcd_u128(gg, Vq[p]);
  if (gg == 0) return false;
  Dc /= 2;  // the loop doubled it once more after success
  const u128 D0 = Dc / gg;
  for (int p = 0; p < npts; ++p) Vq[p] /= gg;
  int d0bits = 0;
  for (u128 t = D0; t; t >>= 1) ++d0bits;
  if (d0bits + (N - 2) * P > 126) return false;  // D < 2^126: one 128-bit weight word
  // refinement cascade: level l point (i, j) <-> (x0 + i 2^-l, j 2^-l)
  std::vector<u128> cur(Vq), nxt;
  int sx = mw, sy = mh;
  std::vector<std::tuple<int, int, int64_t>> mk;
  for (int ky = 0; ky < mh; ++ky)
    for (int kx = x0; kx <= x1; ++kx)
      if (mask_at(kx, ky)) mk.emplace_back(kx, ky, mask_at(kx, ky));
  for (int l = 1; l <= P; ++l) {
    const int nsx = (mw - 1) * (1 << l) + 1, nsy = (mh - 1) * (1 << l) + 1;
    nxt.assign((size_t)nsx * nsy, 0);
    const int h = 1 << (l - 1);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nsy; ++j)
      for (int i = 0; i < nsx; ++i) {
        u128 acc = 0;
        for (const auto& t : mk) {
          const int ip = i + (x0 - std::get<0>(t)) * h;
          const int jp = j - std::get<1>(t) * h;
          if (ip < 0 || ip >= sx || jp < 0 || jp >= sy) continue;
          acc += (u128)std::get<2>(t) * cur[(size_t)jp * sx + ip];
        }
        nxt[(size_t)j * nsx + i] = acc;
      }
    cur.swap(nxt);
    sx = nsx;
    sy = nsy;
  }
  const u128 D = D0 << ((N - 2) * P);
  const int one = 1 << P;
  // centre of the uncentred kernel, units 2^-P
  const long CX = (long)(m[0] + m[1] - m[3]) * (one / 2), CY = (long)(m[1] + m[2] + m[3]) * (one / 2);
  auto weight = [&](int rx, int ry, int dx, int dy) -> u128 {
    const long X = (long)rx - (long)dx * one + CX, Y = (long)ry - (long)dy * one + CY;
    const long i = X - (long)x0 * one, j = Y;
    if (i < 0 || i >= sx || j < 0 || j >= sy) return 0;
    return cur[(size_t)j * sx + i];
  };
  // candidate neighbours: the centred support lies in |x| <= (x1 - x0)/2, |y| <= y1/2
  const int hx = (x1 - x0) / 2 + 2, hy = y1 / 2 + 2;
  std::vector<int2> cand;
  for (int dy = -hy; dy <= hy; ++dy)
    for (int dx = -hx; dx <= hx; ++dx) {
      bool any = false;
      for (int ry = 0; ry < one && !any; ++ry)
        for (int rx = 0; rx < one && !any; ++rx) any = weight(rx, ry, dx, dy) != 0;
      if (any) cand.push_back(make_int2(dx, dy));
    }
  const int R = (int)cand.size();
  if (R < 1 || R > abf::kGenMaxR) return false;
  const int wb = D < ((u128)1 << 64) ? 8 : 16;
  const size_t rows = (size_t)one * one;
  out.bytes.assign(rows * R * wb, 0);
  bool sums_ok = true;
#pragma omp parallel for schedule(static) reduction(&& : sums_ok)
  for (int ry = 0; ry < one; ++ry)
    for (int rx = 0; rx < one; ++rx) {
      u128 rowsum = 0;
      for (int c = 0; c < R; ++c) {
        const u128 w = weight(rx, ry, cand[c].x, cand[c].y);
        rowsum += w;
        uint8_t* dst = &out.bytes[(((size_t)ry * one + rx) * R + c) * wb];
        for (int b = 0; b < wb; ++b) dst[b] = (uint8_t)(w >> (8 * b));
      }
      if (rowsum != D) sums_ok = false;  // unit lattice sum: the kernel holds unit v1 and v3
    }
  if (!sums_ok) return false;
  out.stencil = cand;
  out.D = D;
  out.wbytes = wb;
  return true;
}

struct GenDevTable {
  void* ptr = nullptr;
  int2* stencil = nullptr;
  int R = 0, wbytes = 0;
  u128 D = 0;
};

std::mutex g_gen_mu;
std::map<std::tuple<int, int, int, int, int, int>, GenDevTable> g_gen_tables;  // (device, m1..m4, P); until exit

abf_status get_gen_table(int device, const int m[4], int P, GenDevTable* out) {
  std::lock_guard<std::mutex> lk(g_gen_mu);
  const auto key = std::make_tuple(device, m[0], m[1], m[2], m[3], P);
  auto it = g_gen_tables.find(key);
  if (it != g_gen_tables.end()) {
    *out = it->second;
    return ABF_OK;
  }
  GenTable ht;
  try {
    if (!build_gen_table(m, P, ht)) return ABF_ERR_UNSUPPORTED;
  } catch (const std::bad_alloc&) {
    return ABF_ERR_OOM;
  }
  GenDevTable dt;
  dt.R = (int)ht.stencil.size();
  dt.wbytes = ht.wbytes;
  dt.D = ht.D;
  if (cudaMalloc(&dt.ptr, ht.bytes.size()) != cudaSuccess) return ABF_ERR_OOM;
  if (cudaMalloc((void**)&dt.stencil, ht.stencil.size() * sizeof(int2)) != cudaSuccess) {
    cudaFree(dt.ptr);
    return ABF_ERR_OOM;
  }
  if (cudaMemcpy(dt.ptr, ht.bytes.data(), ht.bytes.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dt.stencil, ht.stencil.data(), ht.stencil.size() * sizeof(int2), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    cudaFree(dt.ptr);
    cudaFree(dt.stencil);
    return ABF_ERR_CUDA;
  }
  g_gen_tables[key] = dt;
  *out = dt;
  return ABF_OK;
}

double u128_d(u128 v) { return (double)(uint64_t)(v >> 64) * 18446744073709551616.0 + (double)(uint64_t)v; }

// The taps of direction counts r grouped by FD weight (groups in order of
// first appearance, taps in index order within a group).
void build_gen_taps(const int r[4], abf::GenTaps& gt) {
  const int taps = (r[0] + 1) * (r[1] + 1) * (r[2] + 1) * (r[3] + 1);
  std::vector<int> wt((size_t)taps), jj((size_t)taps);
  for (int t = 0; t < taps; ++t) {
    int u = t, w = 1, packed = 0;
    for (int k = 0; k < 4; ++k) {
      const int rk = r[k], j = u % (rk + 1);
      u /= rk + 1;
      int b = 1;  // binom(rk, j)
      for (int i = 0; i < j; ++i) b = b * (rk - i) / (i + 1);
      w *= (j & 1) ? -b : b;
      packed |= j << (2 * k);
    }
    wt[(size_t)t] = w;
    jj[(size_t)t] = packed;
  }
  int ng = 0, c = 0;
  for (int t = 0; t < taps; ++t) {
    bool seen = false;
    for (int q = 0; q < ng; ++q) seen |= gt.gw[q] == wt[(size_t)t];
    if (!seen) gt.gw[ng++] = wt[(size_t)t];
  }
  for (int q = 0; q < ng; ++q) {
    gt.gbeg[q] = c;
    for (int t = 0; t < taps; ++t)
      if (wt[(size_t)t] == gt.gw[q]) gt.order[c++] = (unsigned char)jj[(size_t)t];
  }
  gt.gbeg[ng] = c;
  gt.ng = ng;
  gt.taps = taps;
}

}  // namespace

namespace abf {

// Plan for N = 2 or a model (abf_plan_create hands these over); the
// descriptor has been validated as for the plain plans.
abf_status create_general_plan(const abf_desc* d, abf_plan p) {
  const int n = d->order_n, N = d->directions == 2 ? 2 : 4, E = d->model_boxes;
  if (E < 0 || E > 6) return ABF_ERR_INVALID;
  if (N == 2 && E == 0 && n < 2) return ABF_ERR_UNSUPPORTED;  // rect: a discontinuous kernel
  if (N == 2 && d->scale_kind == ABF_SCALES_ELLIPSE) return ABF_ERR_INVALID;
  const int Q = d->q_bits, P = Q + 1;
  if (Q > 7) return ABF_ERR_UNSUPPORTED;   // table of (2^(Q+1))^2 rows
  int r[4] = {n, N == 4 ? n : 0, n, N == 4 ? n : 0};
  int m[4] = {r[0] + E, r[1], r[2] + E, r[3]};
  const int dev = p->device;
  GenDevTable tab;
  abf_status s = get_gen_table(dev, m, P, &tab);
  if (s != ABF_OK) return s;
  const double qd = std::ldexp(1.0, Q);
  const int Cmax = (int)std::lrint(d->max_scale * qd);
  const double min_scale = d->min_scale > 0 ? d->min_scale : 1.0;
  int Cmin = (int)std::ceil(min_scale * qd - 1e-9);
  if (Cmin < 1) Cmin = 1;
  double vb = d->value_bound;
  if (!(vb > 0)) vb = d->in_dtype == ABF_U8 ? 255.0 : (d->in_dtype == ABF_U16 ? 65535.0 : 0.0);
  if (!(vb > 0)) return ABF_ERR_INVALID;
  // model coefficients and their bound
  const double xmax = std::ldexp(vb, d->in_frac_bits);
  PrefilterView pf{};
  double hnorm = 1.0, cbound = vb;
  int T = 0;
  const int n1 = E - 1;
  if (E >= 3) {
    s = prefilter2d_setup(n1, xmax, &pf, &hnorm, &T);
    if (s != ABF_OK) return s;
    cbound = hnorm * hnorm * vb + std::ldexp(1.0, -d->in_frac_bits);
  }
  // limbs: |S| <= D prod_k c_k^{r_k} |c|max 2^F (unit lattice sum with a model;
  // (1 + 1/c1)(1 + 1/c3) for phi = delta)
  const double cmax = (double)Cmax / qd, cmin = (double)Cmin / qd;
  double lp = 0.0;
  for (int k = 0; k < 4; ++k) lp += r[k] * std::log2(cmax);
  if (d->max_scale_product > 0 && N == 4) lp = n * std::log2(d->max_scale_product);
  const double lb = std::log2(u128_d(tab.D)) + lp + std::log2(cbound) + d->in_frac_bits +
                    (E == 0 ? 2.0 * std::log2(1.0 + 1.0 / cmin) : 0.0) + 1e-6;
  const int L = (int)std::floor((lb + 1.0) / 64.0) + 1;
  if (L > kMaxLimbs) return ABF_ERR_RANGE;
  // lattice box: taps within sum_k r_k (cmax + 1) |v_k| of the pixel, plus the stencil
  double ex = 0.0, ey = 0.0;
  const int V[4][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 1}};
  for (int k = 0; k < 4; ++k) {
    ex += r[k] * (cmax + 1.0) * std::abs(V[k][0]);
    ey += r[k] * (cmax + 1.0) * std::abs(V[k][1]);
  }
  int dminx = 0, dmaxx = 0, dminy = 0, dmaxy = 0;
  {
    std::vector<int2> st((size_t)tab.R);
    if (cudaMemcpy(st.data(), tab.stencil, st.size() * sizeof(int2), cudaMemcpyDeviceToHost) != cudaSuccess)
      return ABF_ERR_CUDA;
    for (const int2& q : st) {
      dminx = std::min(dminx, q.x); dmaxx = std::max(dmaxx, q.x);
      dminy = std::min(dminy, q.y); dmaxy = std::max(dmaxy, q.y);
    }
  }
  const int Wi = d->width + 2 * T, Hi = d->height + 2 * T;
  PlanView& pv = p->pv;
  pv = PlanView{};
  pv.W = d->width; pv.H = d->height; pv.n = n; pv.Q = Q; pv.P = P; pv.F = d->in_frac_bits;
  pv.left = (int)std::ceil(ex) - dminx + 2;
  pv.right = (int)std::ceil(ex) + dmaxx + 2;
  pv.above = (int)std::ceil(ey) + dmaxy + 2;
  pv.Gw = Wi + pv.left + pv.right;
  pv.Gh = Hi + pv.above;
  pv.Gp = ((long long)pv.Gw + 3) / 4 * 4;
  if ((long long)(pv.Gh + 8) * pv.Gp >= (1ll << 40)) return ABF_ERR_INVALID;
  pv.Cmax = Cmax; pv.Cmin = Cmin;
  pv.scale_kind = d->scale_kind; pv.in_dtype = d->in_dtype; pv.out_dtype = d->out_dtype;
  pv.limbs = L;
  pv.value_bound = vb;
  pv.log2D = std::log2(u128_d(tab.D));
  pv.log2_base = (float)(pv.log2D + std::log2(cbound) + d->in_frac_bits);
  pv.Dd = u128_d(tab.D);
  pv.out_scale = std::ldexp(1.0 / pv.Dd, Q * (r[0] + r[1] + r[2] + r[3]) - d->in_frac_bits);
  pv.den_int = (r[0] + r[1] + r[2] + r[3]) * std::log2((double)Cmax + 1.0) < 63.0 ? 1 : 0;
  pv.table_bytes_per_w = tab.wbytes;
  pv.table = tab.ptr;
  pv.table_fold = nullptr;
  for (int k = 0; k < 4; ++k) pv.r[k] = r[k];
  pv.E = E;
  pv.R = tab.R;
  pv.stencil = tab.stencil;
  pv.ox = T;
  pv.oy = T;
  p->D = tab.D;
  // the running sums' view: the image (E < 3) or the staged c_q frame
  PlanView& sv = p->sv;
  sv = pv;
  sv.W = Wi;
  sv.H = Hi;
  sv.F = d->in_frac_bits;
  if (E >= 3) {
    sv.in_dtype = kStageI64;
    pf.length = d->width;
    pf.Gw = Wi;
    pf.left = T;
    pf.scale = std::ldexp(1.0, d->in_frac_bits);
    const double bd = std::floor(xmax);
    pf.bound = bd < 4.0e18 ? (long long)bd : 4000000000000000000ll;
    PrefilterView* hp = new (std::nothrow) PrefilterView(pf);
    if (!hp) return ABF_ERR_OOM;
    p->pf = hp;
    const size_t stage = (size_t)Wi * Hi * 8;
    const size_t inter = (size_t)Wi * d->height * 8;
    const size_t yf = (size_t)pf.npoles * Wi * Hi * 8;
    p->pf_tmp_bytes = inter + yf;
    if (cudaMalloc(&p->d_stage, stage) != cudaSuccess) return ABF_ERR_OOM;
    if (cudaMalloc(&p->d_pf_tmp, p->pf_tmp_bytes) != cudaSuccess) return ABF_ERR_OOM;
  }
  {
    GenTaps gt{};
    build_gen_taps(r, gt);
    if (cudaMalloc(&p->d_gtaps, sizeof(GenTaps)) != cudaSuccess) return ABF_ERR_OOM;
    if (cudaMemcpy(p->d_gtaps, &gt, sizeof(GenTaps), cudaMemcpyHostToDevice) != cudaSuccess) return ABF_ERR_CUDA;
    pv.gtaps = p->d_gtaps;
  }
  p->general = true;
  p->g_bytes = (size_t)pv.Gp * (size_t)pv.Gh * (size_t)L * 8;
  p->ws_bytes = line_ws_bytes(pv.Gw, pv.Gh, L, n, nullptr, nullptr);
  return ABF_OK;
}

void destroy_general_plan(abf_plan p) {
  if (p->d_gtaps) cudaFree(p->d_gtaps);
  p->d_gtaps = nullptr;
  if (p->d_stage) cudaFree(p->d_stage);
  if (p->d_pf_tmp) cudaFree(p->d_pf_tmp);
  delete (PrefilterView*)p->pf;
  p->d_stage = p->d_pf_tmp = nullptr;
  p->pf = nullptr;
}

// Non-adaptive step of a generalised plan: the model's prefilter when it has
// one (rows, then columns into the staged c_q frame), then the running sums
// of the running sums' view.
cudaError_t run_integrate_general(abf_plan p, const void* f, size_t f_pitch, uint64_t* g, void* ws, uint32_t* epoch,
                                  int32_t* status, cudaStream_t st) {
  if (p->pv.E >= 3) {
    const PrefilterView& pf = *(const PrefilterView*)p->pf;
    const int W = p->pv.W, H = p->pv.H, T = p->pv.ox, Wi = p->sv.W;
    long long* inter = (long long*)p->d_pf_tmp;
    long long* yf = inter + (size_t)Wi * H;
    cudaError_t e = run_prefilter_rows_raw(pf, H, p->desc.in_dtype, f, f_pitch, inter, Wi, status, st);
    if (e != cudaSuccess) return e;
    (void)W;
    prefilter_cols_kernel<<<(Wi + 127) / 128, 128, 0, st>>>(pf, H, T, Wi, inter, Wi, yf, (long long*)p->d_stage, Wi);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return run_integrate(p->sv, p->d_stage, (size_t)Wi * 8, g, ws, epoch, status, st);
  }
  return run_integrate(p->sv, f, f_pitch, g, ws, epoch, status, st);
}

// Host-only: the generalised interpolation table (for checks against the
// oracle without a device).
bool general_table_host(const int m[4], int P, std::vector<uint8_t>& bytes, std::vector<int2>& stencil, u128* D,
                        int* wbytes) {
  GenTable t;
  if (!build_gen_table(m, P, t)) return false;
  bytes.swap(t.bytes);
  stencil.swap(t.stencil);
  *D = t.D;
  *wbytes = t.wbytes;
  return true;
}

}  // namespace abf
