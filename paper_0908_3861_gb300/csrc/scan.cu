// Non-adaptive step of Sec. 7 (1), Eq. (RS): the four running-sum recursions
//   F0[k1,k2] = f[k1,k2]  + F0[k1-1,k2]        direction v1 = (1,0)
//   Fq[k1,k2] = F0[k1,k2] + Fq[k1-1,k2-1]      direction v2 = (1,1)
//   Fh[k1,k2] = Fq[k1,k2] + Fh[k1,k2-1]        direction v3 = (0,1)
//   g [k1,k2] = Fh[k1,k2] + g [k1+1,k2-1]      direction v4 = (-1,1)
// with unit weights (the paper's sqrt2 factors sit in the normaliser), each
// applied n times, in wrap-around integers modulo 2^(64 L).
//
// Lattice box: columns [-left, W + right), rows [0, H + above).  Rows below the
// image are identically zero and not stored.  v1, v2, v3 are exact on the box
// (their backward rays leave it where the input is zero).  v4 runs last; a
// backward 3pi/4 ray that leaves through the right edge misses values, and the
// miss is a polynomial of degree < n along that 3pi/4 line (the exit point moves
// linearly along the line), which the FD of the mesh along v4 annihilates.
//
// Kernels:
//   row_scan   : rows of up to 8192 cells: one warp per row in one pass;
//                longer rows (the 1-D filter's signals): one CTA per row, its
//                warps on contiguous segments, segment states composed through
//                shared memory (affine carries).  Input conversion (a0) fused
//                (the 1-D filter's prefiltered models pass integer
//                coefficients staged by its prefilter instead), all n folds of
//                v1 together (lane-local scans + warp shuffles, a running
//                state per fold).
//   line_scan  : v2 / v3 / v4, one thread per line and row segment (sheared so
//                that a warp reads consecutive addresses), lines cut into bands
//                of kBand rows; bands are chained by decoupled look-back on
//                per-line flags, with a bounded wait that raises
//                ABF_DEV_TIMEOUT instead of hanging.
#include <mutex>
#include <type_traits>

#include "abf_internal.cuh"

namespace abf {

// ------------------------------------------------------------------ rows (v1)

template <typename T>
__device__ __forceinline__ double as_double(T v) { return (double)v; }

template <int L>
__device__ __forceinline__ Wide<L> shfl_up_wide(const Wide<L>& v, int d) {
  Wide<L> r;
#pragma unroll
  for (int i = 0; i < L; ++i) r.w[i] = __shfl_up_sync(0xffffffffu, v.w[i], d);
  return r;
}

template <int L>
__device__ __forceinline__ Wide<L> shfl_wide(const Wide<L>& v, int src) {
  Wide<L> r;
#pragma unroll
  for (int i = 0; i < L; ++i) r.w[i] = __shfl_sync(0xffffffffu, v.w[i], src);
  return r;
}

// Inclusive scan of one value per lane across the warp.
template <int L>
__device__ __forceinline__ Wide<L> warp_inclusive(Wide<L> v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    Wide<L> o = shfl_up_wide<L>(v, d);
    if (lane >= d) waddc<L>(v, o);
  }
  return v;
}

constexpr int kRowVec = 4;     // elements per lane per chunk
constexpr int kRowWarps = 8;   // warps per row (one CTA per row)

// acc_k += sum_{j <= k} binom(t + k - j - 1, k - j) c_j: the zero-input
// evolution of the cascaded-sum state c over t samples, added to acc.
template <int L, int NF>
__device__ __forceinline__ void transport_add(Wide<L>* acc, const Wide<L>* c, long long t) {
  const uint64_t b1 = (uint64_t)t, b2 = (uint64_t)(t * (t + 1) / 2), b3 = (uint64_t)(t * (t + 1) / 2 * (t + 2) / 3);
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    waddc<L>(acc[k], c[k]);
    if (k >= 1) wmac<L>(acc[k], c[k - 1], b1);
    if (k >= 2) wmac<L>(acc[k], c[k - 2], b2);
    if (k >= 3) wmac<L>(acc[k], c[k - 3], b3);
  }
}

// One chunk of 32 x kRowVec samples: load (a0 fused), NF cascaded scans with
// the running state carry[] (carry[k] = fold k's sum so far), optional store
// through the warp's shared-memory tile (lane i holds samples 4i..4i+3; the
// store writes 32 consecutive samples per instruction).
// The raw input of one chunk (zeros outside the image), fetched ahead of its
// scan so that the next chunk's loads are in flight during this one's.
template <typename TIn>
__device__ __forceinline__ void row_fetch(const PlanView& pv, const TIn* frow, int x0, int lane, TIn (&raw)[kRowVec]) {
#pragma unroll
  for (int e = 0; e < kRowVec; ++e) {
    const int xi = x0 + lane * kRowVec + e;  // box column
    const int x = xi - pv.left;              // image column
    raw[e] = (frow && x >= 0 && x < pv.W && xi < pv.Gw) ? frow[x] : (TIn)0;
  }
}

template <int L, typename TIn, int NF, bool STORE>
__device__ __forceinline__ void row_chunk(const PlanView& pv, const TIn (&raw)[kRowVec], uint64_t* grow, int x0,
                                          int lane, double scale, long long bound, int32_t* status, Wide<L>* carry,
                                          Wide<L>* tile) {
  Wide<L> v[kRowVec];
#pragma unroll
  for (int e = 0; e < kRowVec; ++e) v[e] = wfrom_i64<L>(convert_f<TIn>(raw[e], scale, bound, status));
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    // lane-local inclusive scan
#pragma unroll
    for (int e = 1; e < kRowVec; ++e) waddc<L>(v[e], v[e - 1]);
    Wide<L> tot = v[kRowVec - 1];
    Wide<L> incl = warp_inclusive<L>(tot, lane);
    Wide<L> excl = shfl_up_wide<L>(incl, 1);
    if (lane == 0) wzero<L>(excl);
    waddc<L>(excl, carry[k]);
#pragma unroll
    for (int e = 0; e < kRowVec; ++e) waddc<L>(v[e], excl);
    Wide<L> last = shfl_wide<L>(incl, 31);
    waddc<L>(carry[k], last);
  }
  if constexpr (STORE) {
#pragma unroll
    for (int e = 0; e < kRowVec; ++e) tile[lane * kRowVec + e] = v[e];
    __syncwarp();
#pragma unroll
    for (int e = 0; e < kRowVec; ++e) {
      const int xi = x0 + e * 32 + lane;
      if (xi < pv.Gw) wstore<L>(grow + (size_t)xi * L, tile[e * 32 + lane]);
    }
    __syncwarp();
  }
}

// One CTA per row, kRowWarps warps each taking a contiguous segment of whole
// chunks.  Phase 1: every warp scans its segment from a zero state and keeps
// the final state (its aggregate).  Then warp w's incoming state is composed
// from the aggregates of warps 0..w-1 by the zero-input evolution (the
// cascaded sums are affine in the incoming state).  Phase 2: every warp
// rescans its segment from its incoming state and stores g.  f is read
// twice; g is written once.
template <int L, typename TIn, int NF>
__device__ __forceinline__ void row_scan_body(const PlanView& pv, const TIn* __restrict__ f, size_t f_pitch,
                                              uint64_t* __restrict__ g, int32_t* status, int y) {
  __shared__ Wide<L> s_agg[kRowWarps][NF];
  __shared__ Wide<L> s_tile[kRowWarps][32 * kRowVec];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double scale = ldexp(1.0, pv.F);
  const double bd = floor(pv.value_bound * scale);
  const long long bound = bd < 4.0e18 ? (long long)bd : 4000000000000000000ll;
  const TIn* frow = (y < pv.H) ? reinterpret_cast<const TIn*>(reinterpret_cast<const char*>(f) + (size_t)y * f_pitch)
                               : nullptr;
  uint64_t* grow = g + (size_t)y * (size_t)pv.Gp * L;
  constexpr int chunk = 32 * kRowVec;
  const int nchunks = (pv.Gw + chunk - 1) / chunk;
  const int per = (nchunks + kRowWarps - 1) / kRowWarps;
  const int c0 = min(nchunks, warp * per), c1 = min(nchunks, c0 + per);
  Wide<L> carry[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) wzero<L>(carry[k]);
  TIn raw[kRowVec], nxt[kRowVec];
  if (c0 < c1) row_fetch<TIn>(pv, frow, c0 * chunk, lane, nxt);
  for (int c = c0; c < c1; ++c) {
#pragma unroll
    for (int e = 0; e < kRowVec; ++e) raw[e] = nxt[e];
    if (c + 1 < c1) row_fetch<TIn>(pv, frow, (c + 1) * chunk, lane, nxt);
    row_chunk<L, TIn, NF, false>(pv, raw, grow, c * chunk, lane, scale, bound, status, carry, nullptr);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NF; ++k) s_agg[warp][k] = carry[k];
  }
  __syncthreads();
  // incoming state: state_{w+1} = T_len(state_w) + agg_w; every segment
  // before this warp's is full (per chunks)
  Wide<L> st[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) wzero<L>(st[k]);
  for (int w = 0; w < warp; ++w) {
    Wide<L> nx[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) nx[k] = s_agg[w][k];
    transport_add<L, NF>(nx, st, (long long)per * chunk);
#pragma unroll
    for (int k = 0; k < NF; ++k) st[k] = nx[k];
  }
  if (c0 < c1) row_fetch<TIn>(pv, frow, c0 * chunk, lane, nxt);
  for (int c = c0; c < c1; ++c) {
#pragma unroll
    for (int e = 0; e < kRowVec; ++e) raw[e] = nxt[e];
    if (c + 1 < c1) row_fetch<TIn>(pv, frow, (c + 1) * chunk, lane, nxt);
    row_chunk<L, TIn, NF, true>(pv, raw, grow, c * chunk, lane, scale, bound, status, st, s_tile[warp]);
  }
}

template <int L, typename TIn, int NF>
__global__ void __launch_bounds__(32 * kRowWarps) row_scan_kernel(const PlanView pv, const TIn* __restrict__ f,
                                                                  size_t f_pitch, uint64_t* __restrict__ g,
                                                                  int32_t* status) {
  row_scan_body<L, TIn, NF>(pv, f, f_pitch, g, status, blockIdx.x);
}

// Rows of up to this many cells are scanned by one warp each, in one pass
// (the serial chain of a row is then at most 64 chunks).  There are only as
// many warps as rows, so small CTAs spread them evenly over the SMs.
constexpr int kRowWarpMaxCells = 8192;
constexpr int kRowsPerCta = 2;

// One warp per row, one pass: the chunks in order, the running states carried
// from chunk to chunk, the raw input fetched two chunks ahead.  f is read once
// and g written once; a CTA holds kRowsPerCta rows.
template <int L, typename TIn, int NF>
__device__ __forceinline__ void row_scan_warp_body(const PlanView& pv, const TIn* __restrict__ f, size_t f_pitch,
                                                   uint64_t* __restrict__ g, int32_t* status, int y, Wide<L>* tile) {
  const int lane = threadIdx.x & 31;
  const double scale = ldexp(1.0, pv.F);
  const double bd = floor(pv.value_bound * scale);
  const long long bound = bd < 4.0e18 ? (long long)bd : 4000000000000000000ll;
  const TIn* frow = (y < pv.H) ? reinterpret_cast<const TIn*>(reinterpret_cast<const char*>(f) + (size_t)y * f_pitch)
                               : nullptr;
  uint64_t* grow = g + (size_t)y * (size_t)pv.Gp * L;
  constexpr int chunk = 32 * kRowVec;
  const int nchunks = (pv.Gw + chunk - 1) / chunk;
  Wide<L> carry[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) wzero<L>(carry[k]);
  TIn b0[kRowVec], b1[kRowVec], b2[kRowVec];
  row_fetch<TIn>(pv, frow, 0, lane, b0);
  if (nchunks > 1) row_fetch<TIn>(pv, frow, chunk, lane, b1);
  for (int c = 0; c < nchunks; ++c) {
    if (c + 2 < nchunks) row_fetch<TIn>(pv, frow, (c + 2) * chunk, lane, b2);
    row_chunk<L, TIn, NF, true>(pv, b0, grow, c * chunk, lane, scale, bound, status, carry, tile);
#pragma unroll
    for (int e = 0; e < kRowVec; ++e) {
      b0[e] = b1[e];
      b1[e] = b2[e];
    }
  }
}

template <int L, typename TIn, int NF>
__global__ void __launch_bounds__(32 * kRowsPerCta) row_scan_warp_kernel(const PlanView pv, const TIn* __restrict__ f,
                                                                         size_t f_pitch, uint64_t* __restrict__ g,
                                                                         int32_t* status) {
  __shared__ Wide<L> s_tile[kRowsPerCta][32 * kRowVec];
  const int warp = threadIdx.x >> 5;
  const int y = blockIdx.x * kRowsPerCta + warp;
  if (y >= pv.Gh) return;
  row_scan_warp_body<L, TIn, NF>(pv, f, f_pitch, g, status, y, s_tile[warp]);
}

// ---------------------------------------------------------- lines (v2, v3, v4)
// One pass per direction carries all n cascaded running sums: per line a state
// (s_1..s_n), updated per element x as s_1 += x, s_2 += s_1, ..., out = s_n.
// A band of R rows maps an incoming state c to T_R(c) + A, where A is the
// band's own result from a zero state and T_t is the zero-input evolution over
// t steps, T_t(c)_k = sum_{j<=k} c_j binom(t + k - j - 1, k - j).  Look-back
// therefore sums T_{dR}(A) over the d-th band below until a band that has
// published its inclusive state P, which enters as T_{dR}(P).

constexpr int kBand = 64;         // rows per band (fewer bands: a shorter look-back chain)
constexpr int kSplit = 4;         // row segments per band, one thread per line and segment
constexpr int kSeg = kBand / kSplit;
// Lines per CTA: the band is staged in shared memory, kBand x lines x L limbs
// (32 KB at most, so that several CTAs per SM keep their copies in flight
// while others wait in the look-back).
template <int L>
__host__ __device__ constexpr int lines_per_cta() { return L <= 2 ? 32 : 16; }
template <int L>
__host__ __device__ constexpr int line_threads() { return lines_per_cta<L>() * kSplit; }
template <int L>
__host__ __device__ constexpr int band_smem_bytes() { return kBand * lines_per_cta<L>() * L * 8; }
constexpr uint32_t kFlagAgg = 1, kFlagPrefix = 2;
constexpr long long kSpinLimit = 1ll << 20;  // polls, 100 ns apart: about a second

struct LineWs {
  uint32_t* flags;    // [nbands][nlines]
  uint64_t* agg;      // [nbands][nlines][NF][L]
  uint64_t* pref;     // [nbands][nlines][NF][L]
  uint32_t* ticket;   // one counter, zeroed before each launch
  int nbands, nlines, ngroups;
};

// DIR: 2 -> v2 = (1,1) (box column xi = l - (Gh-1) + y), 3 -> v3 (xi = l),
//      4 -> v4 = (-1,1) (xi = l - y).
template <int DIR>
__device__ __forceinline__ int line_col(int l, int y, int Gh) {
  if constexpr (DIR == 2) return l - (Gh - 1) + y;
  else if constexpr (DIR == 3) return l;
  else return l - y;
}

template <int L, int NF>
struct LineState {
  Wide<L> s[NF];
};

template <int L, int NF>
__device__ __forceinline__ void st_zero(LineState<L, NF>& a) {
#pragma unroll
  for (int k = 0; k < NF; ++k) wzero<L>(a.s[k]);
}

template <int L, int NF>
__device__ __forceinline__ void st_step(LineState<L, NF>& a, const Wide<L>& x) {
  waddc<L>(a.s[0], x);
#pragma unroll
  for (int k = 1; k < NF; ++k) waddc<L>(a.s[k], a.s[k - 1]);
}

// acc += T_t(c): the zero-input evolution of state c over t steps.
template <int L, int NF>
__device__ __forceinline__ void st_add_transported(LineState<L, NF>& acc, const LineState<L, NF>& c, long long t) {
  waddc<L>(acc.s[0], c.s[0]);
  if constexpr (NF >= 2) {
    waddc<L>(acc.s[1], c.s[1]);
    wmac<L>(acc.s[1], c.s[0], (uint64_t)t);
  }
  if constexpr (NF >= 3) {
    waddc<L>(acc.s[2], c.s[2]);
    wmac<L>(acc.s[2], c.s[1], (uint64_t)t);
    wmac<L>(acc.s[2], c.s[0], (uint64_t)(t * (t + 1) / 2));
  }
}

template <int L, int NF>
__device__ __forceinline__ LineState<L, NF> st_load(const uint64_t* p) {
  LineState<L, NF> r;
#pragma unroll
  for (int k = 0; k < NF; ++k) r.s[k] = wload<L>(p + k * L);
  return r;
}

template <int L, int NF>
__device__ __forceinline__ void st_store(uint64_t* p, const LineState<L, NF>& a) {
#pragma unroll
  for (int k = 0; k < NF; ++k) wstore<L>(p + k * L, a.s[k]);
}

// Copy L limbs (8 * L bytes) from global to shared memory asynchronously, or
// zeros when !ok (a zero-byte source read; the address stays a valid one).
template <int L>
__device__ __forceinline__ void cp_async_elem(uint64_t* dst, const uint64_t* src, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (L % 2 == 0) {
#pragma unroll
    for (int i = 0; i < L / 2; ++i)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d + 16 * i),
                   "l"(__cvta_generic_to_global(src + 2 * i)), "r"(ok ? 16 : 0) : "memory");
  } else {
#pragma unroll
    for (int i = 0; i < L; ++i)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d + 8 * i),
                   "l"(__cvta_generic_to_global(src + i)), "r"(ok ? 8 : 0) : "memory");
  }
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One CTA = one band of kBand rows x lines_per_cta<L>() consecutive lines, one
// thread per line and row segment (kSplit segments of kSeg rows).  Each thread
// copies its segment of its line into shared memory (cp.async, the copies of
// all rows in flight together) and sums it from a zero state; the segment
// aggregates compose into the band aggregate (T_kSeg transports), the
// segment-0 threads run the decoupled look-back for the band and hand every
// segment its incoming state, and each thread rescans its staged segment into
// g: one read and one write of g per pass, with the serial work of a band cut
// into kSplit pieces that run side by side.
template <int L, int DIR, int NF>
__device__ __forceinline__ void line_scan_body(const PlanView& pv, uint64_t* __restrict__ g, const LineWs& ws,
                                               uint32_t epoch, int32_t* status, int band, int grp) {
  constexpr int LPC = lines_per_cta<L>();
  constexpr int SW = NF * L;                          // words of one state
  extern __shared__ __align__(16) uint64_t s_band[];  // [kBand][LPC][L]
  __shared__ __align__(16) uint64_t s_seg[kSplit * LPC * SW];  // [kSplit][LPC] states (16-byte vector accesses)
  const int ln = threadIdx.x % LPC, seg = threadIdx.x / LPC;
  const int l = grp * LPC + ln;
  const bool line_ok = l < ws.nlines;
  const int y0 = band * kBand + seg * kSeg;
  uint64_t* mine = s_band + ((size_t)seg * kSeg * LPC + ln) * L;
  uint64_t* my_state = s_seg + ((size_t)seg * LPC + ln) * SW;

  // stage the segment (zeros outside the box)
#pragma unroll 8
  for (int i = 0; i < kSeg; ++i) {
    const int y = y0 + i;
    const int xi = line_col<DIR>(l, y, pv.Gh);
    const bool ok = line_ok && y < pv.Gh && xi >= 0 && xi < pv.Gw;
    const uint64_t* src = ok ? g + ((size_t)y * (size_t)pv.Gp + (size_t)xi) * L : g;
    cp_async_elem<L>(mine + (size_t)i * LPC * L, src, ok);
  }
  cp_async_wait_all();

  // segment aggregate from a zero state
  LineState<L, NF> agg;
  st_zero<L, NF>(agg);
#pragma unroll 8
  for (int i = 0; i < kSeg; ++i) st_step<L, NF>(agg, wload<L>(mine + (size_t)i * LPC * L));
  st_store<L, NF>(my_state, agg);
  __syncthreads();

  if (seg == 0) {
    // band aggregate: A <- T_kSeg(A) + (next segment's aggregate)
    LineState<L, NF> A = agg;
    for (int q = 1; q < kSplit; ++q) {
      LineState<L, NF> nx = st_load<L, NF>(s_seg + ((size_t)q * LPC + ln) * SW);
      st_add_transported<L, NF>(nx, A, kSeg);
      A = nx;
    }
    // decoupled look-back over the bands below (same line)
    LineState<L, NF> carry;
    st_zero<L, NF>(carry);
    const size_t slot = (size_t)band * ws.nlines + (line_ok ? l : 0);
    if (line_ok) {
      if (band > 0) {
        st_store<L, NF>(ws.agg + slot * NF * L, A);
        st_release(ws.flags + slot, (epoch << 2) | kFlagAgg);  // release: the aggregate is visible first
        // Up to kLook predecessor flags are read per round trip (relaxed loads,
        // then one acquire fence before the values they publish are read): the
        // walk back to the nearest published prefix takes a quarter of the trips.
        constexpr int kLook = 4;
        int bb = band - 1;
        long long dist = 0;  // rows between the end of band bb and the start of this band
        long long spins = 0;
        while (bb >= 0) {
          uint32_t fl[kLook];
#pragma unroll
          for (int q = 0; q < kLook; ++q)
            fl[q] = bb - q >= 0 ? ld_relaxed(ws.flags + (size_t)(bb - q) * ws.nlines + l) : 0u;
          int ready = 0;
          bool prefix = false;
#pragma unroll
          for (int q = 0; q < kLook; ++q) {
            if (ready != q || bb - q < 0) break;
            if ((fl[q] >> 2) != epoch || (fl[q] & 3u) == 0u) break;
            ++ready;
            if ((fl[q] & 3u) == kFlagPrefix) {
              prefix = true;
              break;
            }
          }
          if (ready == 0) {
            if (++spins > kSpinLimit) {
              raise_status(status, ABF_DEV_TIMEOUT);
              break;
            }
            __nanosleep(100);  // back off: waiting CTAs should not crowd the flags' L2 lines
            continue;
          }
          fence_acquire();
          for (int q = 0; q < ready; ++q) {
            const size_t s2 = (size_t)(bb - q) * ws.nlines + l;
            if (prefix && q == ready - 1) {
              st_add_transported<L, NF>(carry, st_load<L, NF>(ws.pref + s2 * NF * L), dist);
            } else {
              st_add_transported<L, NF>(carry, st_load<L, NF>(ws.agg + s2 * NF * L), dist);
              dist += kBand;
            }
          }
          if (prefix) break;
          bb -= ready;
        }
      }
      LineState<L, NF> incl = A;
      st_add_transported<L, NF>(incl, carry, kBand);
      st_store<L, NF>(ws.pref + slot * NF * L, incl);
      st_release(ws.flags + slot, (epoch << 2) | kFlagPrefix);
    }
    // incoming state of every segment: in_0 = carry, in_q = T_kSeg(in_{q-1}) + agg_{q-1}
    LineState<L, NF> in = carry;
    for (int q = 0; q < kSplit; ++q) {
      uint64_t* sq = s_seg + ((size_t)q * LPC + ln) * SW;
      LineState<L, NF> nx = st_load<L, NF>(sq);
      st_store<L, NF>(sq, in);
      st_add_transported<L, NF>(nx, in, kSeg);
      in = nx;
    }
  }
  __syncthreads();

  // rescan the staged segment from its incoming state and write g
  LineState<L, NF> st = st_load<L, NF>(my_state);
#pragma unroll 8
  for (int i = 0; i < kSeg; ++i) {
    const int y = y0 + i;
    const int xi = line_col<DIR>(l, y, pv.Gh);
    const bool ok = line_ok && y < pv.Gh && xi >= 0 && xi < pv.Gw;
    st_step<L, NF>(st, wload<L>(mine + (size_t)i * LPC * L));
    if (ok) wstore<L>(g + ((size_t)y * (size_t)pv.Gp + (size_t)xi) * L, st.s[NF - 1]);
  }
}

// Bands are taken in ticket order, so every band a look-back waits on belongs
// to a CTA that started earlier.
template <int L, int DIR, int NF>
__global__ void __launch_bounds__(line_threads<L>()) line_scan_kernel(const PlanView pv, uint64_t* __restrict__ g,
                                                                       LineWs ws, uint32_t epoch,
                                                                       int32_t* status) {
  __shared__ uint32_t s_ticket;
  if (threadIdx.x == 0) s_ticket = atomicAdd(ws.ticket, 1u);
  __syncthreads();
  const uint32_t t = s_ticket;
  const int band = (int)(t / (uint32_t)ws.ngroups);
  const int grp = (int)(t % (uint32_t)ws.ngroups);
  if (band >= ws.nbands) return;
  line_scan_body<L, DIR, NF>(pv, g, ws, epoch, status, band, grp);
}

// ----------------------------------------------------------------- launchers

// The row pass: r1 running sums along v1 (the 1-D filter's plans keep r1 = n,
// the number of cascaded sums of its rows).
template <int L, typename TIn>
static cudaError_t launch_rows(const PlanView& pv, const void* f, size_t f_pitch, uint64_t* g,
                               int32_t* status, cudaStream_t st) {
  const int threads = 32 * kRowWarps;
  const TIn* fin = (const TIn*)f;
  const int nf = pv.r[0];
  if (pv.Gw <= kRowWarpMaxCells) {  // a warp per row
    const int blocks = (pv.Gh + kRowsPerCta - 1) / kRowsPerCta;
    const int wt = 32 * kRowsPerCta;
    if (nf == 1) row_scan_warp_kernel<L, TIn, 1><<<blocks, wt, 0, st>>>(pv, fin, f_pitch, g, status);
    else if (nf == 2) row_scan_warp_kernel<L, TIn, 2><<<blocks, wt, 0, st>>>(pv, fin, f_pitch, g, status);
    else if (nf == 3) row_scan_warp_kernel<L, TIn, 3><<<blocks, wt, 0, st>>>(pv, fin, f_pitch, g, status);
    else row_scan_warp_kernel<L, TIn, 4><<<blocks, wt, 0, st>>>(pv, fin, f_pitch, g, status);
    return cudaGetLastError();
  }
  const int blocks = pv.Gh;  // one CTA per row
  if (nf == 1) row_scan_kernel<L, TIn, 1><<<blocks, threads, 0, st>>>(pv, fin, f_pitch, g, status);
  else if (nf == 2) row_scan_kernel<L, TIn, 2><<<blocks, threads, 0, st>>>(pv, fin, f_pitch, g, status);
  else if (nf == 3) row_scan_kernel<L, TIn, 3><<<blocks, threads, 0, st>>>(pv, fin, f_pitch, g, status);
  else row_scan_kernel<L, TIn, 4><<<blocks, threads, 0, st>>>(pv, fin, f_pitch, g, status);
  return cudaGetLastError();
}

// The row pass alone (pv.r[0] cascaded sums, 1..4, along rows of the box), for
// the 1-D filter: rows are signals, W the signal length, left = 0.
template <int L>
static cudaError_t rows_L(const PlanView& pv, const void* f, size_t f_pitch, uint64_t* g, int32_t* status,
                          cudaStream_t st) {
  switch (pv.in_dtype) {
    case kStageI32: return launch_rows<L, int32_t>(pv, f, f_pitch, g, status, st);
    case kStageI64: return launch_rows<L, long long>(pv, f, f_pitch, g, status, st);
    case ABF_U8: return launch_rows<L, uint8_t>(pv, f, f_pitch, g, status, st);
    case ABF_U16: return launch_rows<L, uint16_t>(pv, f, f_pitch, g, status, st);
    case ABF_F32: return launch_rows<L, float>(pv, f, f_pitch, g, status, st);
    default: return launch_rows<L, double>(pv, f, f_pitch, g, status, st);
  }
}

cudaError_t run_row_scan(const PlanView& pv, const void* f, size_t f_pitch, uint64_t* g, int32_t* status,
                         cudaStream_t st) {
  switch (pv.limbs) {
    case 1: return rows_L<1>(pv, f, f_pitch, g, status, st);
    case 2: return rows_L<2>(pv, f, f_pitch, g, status, st);
    case 3: return rows_L<3>(pv, f, f_pitch, g, status, st);
    default: return rows_L<4>(pv, f, f_pitch, g, status, st);
  }
}

__global__ void set_ticket_kernel(uint32_t* ticket, uint32_t value) { *ticket = value; }

// first_ticket > 0 skips the first tickets (test hook: their bands never run).
template <int L, int DIR, int NF>
static cudaError_t launch_lines(const PlanView& pv, uint64_t* g, const LineWs& ws, uint32_t epoch,
                                int32_t* status, cudaStream_t st, uint32_t first_ticket = 0) {
  cudaError_t e;
  if (first_ticket == 0) {
    e = cudaMemsetAsync(ws.ticket, 0, sizeof(uint32_t), st);
  } else {
    set_ticket_kernel<<<1, 1, 0, st>>>(ws.ticket, first_ticket);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  const int ctas = ws.nbands * ws.ngroups;
  constexpr int smem = band_smem_bytes<L>();
  // the shared-memory limit of this instantiation, set once per device before its first launch
  static bool attr[64] = {};
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    e = cudaFuncSetAttribute(line_scan_kernel<L, DIR, NF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  line_scan_kernel<L, DIR, NF><<<ctas, line_threads<L>(), smem, st>>>(pv, g, ws, epoch, status);
  return cudaGetLastError();
}

// Workspace needed by the line scans for a plan (bytes): flags plus an
// n-component aggregate and prefix of L limbs per (band, line).
size_t line_ws_bytes(int Gw, int Gh, int L, int n, int* nbands_out, int* nlines_out) {
  const int nbands = (Gh + kBand - 1) / kBand;
  const int nlines = Gw + Gh;  // enough for every direction
  if (nbands_out) *nbands_out = nbands;
  if (nlines_out) *nlines_out = nlines;
  const size_t cells = (size_t)nbands * (size_t)nlines;
  size_t bytes = 256;                         // ticket
  bytes += ((cells * 4 + 255) / 256) * 256;   // flags
  bytes += cells * 8 * L * n * 2;             // agg + pref
  return bytes;
}

// Bytes at the start of a line-scan workspace that must read as zero before
// the first scan of a call: the ticket counter and the look-back flags.  A
// workspace holds arbitrary bytes when it arrives (a fresh allocation may
// reuse memory of any earlier buffer), and a stale word can look like a valid
// flag, so every call clears them; later passes of the same call tell their
// flags apart by epoch.
size_t line_ws_zero_bytes(int Gw, int Gh) {
  const size_t cells = (size_t)((Gh + kBand - 1) / kBand) * (size_t)(Gw + Gh);
  return 256 + ((cells * 4 + 255) / 256) * 256;
}

template <int L>
static LineWs carve(void* ws, int Gw, int Gh, int n, int DIR) {
  LineWs w;
  int nbands, nlines_all;
  line_ws_bytes(Gw, Gh, L, n, &nbands, &nlines_all);
  char* p = (char*)ws;
  w.ticket = (uint32_t*)p;
  p += 256;
  const size_t cells = (size_t)nbands * (size_t)nlines_all;
  w.flags = (uint32_t*)p;
  p += ((cells * 4 + 255) / 256) * 256;
  w.agg = (uint64_t*)p;
  p += cells * 8 * L * n;
  w.pref = (uint64_t*)p;
  w.nbands = nbands;
  w.nlines = nlines_all;  // slot stride, the same for every direction
  w.ngroups = ((DIR == 3 ? Gw : Gw + Gh - 1) + lines_per_cta<L>() - 1) / lines_per_cta<L>();
  return w;
}

template <int L, int NF>
static cudaError_t line_dir_NF(int dir, const PlanView& pv, uint64_t* g, void* ws, uint32_t ep, int32_t* status,
                               cudaStream_t st) {
  const LineWs w = carve<L>(ws, pv.Gw, pv.Gh, NF, dir);
  if (dir == 2) return launch_lines<L, 2, NF>(pv, g, w, ep, status, st);
  if (dir == 3) return launch_lines<L, 3, NF>(pv, g, w, ep, status, st);
  return launch_lines<L, 4, NF>(pv, g, w, ep, status, st);
}

// v2, v3, v4 in the paper's order, r_k cascaded sums each (none where r_k = 0).
template <int L>
static cudaError_t lines_all(const PlanView& pv, uint64_t* g, void* ws, uint32_t* epoch, int32_t* status,
                             cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int dir = 2; dir <= 4 && e == cudaSuccess; ++dir) {
    const int nf = pv.r[dir - 1];
    if (nf == 0) continue;
    const uint32_t ep = (*epoch = (*epoch + 1) & 0x3fffffffu);
    if (nf == 1) e = line_dir_NF<L, 1>(dir, pv, g, ws, ep, status, st);
    else if (nf == 2) e = line_dir_NF<L, 2>(dir, pv, g, ws, ep, status, st);
    else e = line_dir_NF<L, 3>(dir, pv, g, ws, ep, status, st);
  }
  return e;
}

template <int L>
static cudaError_t integrate_L(const PlanView& pv, const void* f, size_t f_pitch, uint64_t* g, void* ws,
                               uint32_t* epoch, int32_t* status, cudaStream_t st) {
  cudaError_t e;
  switch (pv.in_dtype) {
    case ABF_U8: e = launch_rows<L, uint8_t>(pv, f, f_pitch, g, status, st); break;
    case ABF_U16: e = launch_rows<L, uint16_t>(pv, f, f_pitch, g, status, st); break;
    case ABF_F32: e = launch_rows<L, float>(pv, f, f_pitch, g, status, st); break;
    case kStageI64: e = launch_rows<L, long long>(pv, f, f_pitch, g, status, st); break;
    default: e = launch_rows<L, double>(pv, f, f_pitch, g, status, st); break;
  }
  if (e != cudaSuccess) return e;
  return lines_all<L>(pv, g, ws, epoch, status, st);
}

// Test hook for the bounded look-back wait: one v3 pass whose band-0 CTAs
// never run, so band 1 waits on flags nothing sets, gives up after its bounded
// spin (ABF_DEV_TIMEOUT) and the pass completes.  g is left undefined.
template <int L, int NF>
static cudaError_t starved_NF(const PlanView& pv, uint64_t* g, void* ws, uint32_t* epoch, int32_t* status,
                              cudaStream_t st) {
  const uint32_t ep = (*epoch = (*epoch + 1) & 0x3fffffffu);
  const LineWs w = carve<L>(ws, pv.Gw, pv.Gh, NF, 3);
  return launch_lines<L, 3, NF>(pv, g, w, ep, status, st, (uint32_t)w.ngroups);
}

template <int L>
static cudaError_t starved_L(const PlanView& pv, uint64_t* g, void* ws, uint32_t* epoch, int32_t* status,
                             cudaStream_t st) {
  switch (pv.n) {
    case 1: return starved_NF<L, 1>(pv, g, ws, epoch, status, st);
    case 2: return starved_NF<L, 2>(pv, g, ws, epoch, status, st);
    default: return starved_NF<L, 3>(pv, g, ws, epoch, status, st);
  }
}

cudaError_t run_lookback_starved(const PlanView& pv, uint64_t* g, void* ws, uint32_t* epoch, int32_t* status,
                                 cudaStream_t st) {
  const cudaError_t e = cudaMemsetAsync(ws, 0, line_ws_zero_bytes(pv.Gw, pv.Gh), st);
  if (e != cudaSuccess) return e;
  switch (pv.limbs) {
    case 1: return starved_L<1>(pv, g, ws, epoch, status, st);
    case 2: return starved_L<2>(pv, g, ws, epoch, status, st);
    case 3: return starved_L<3>(pv, g, ws, epoch, status, st);
    default: return starved_L<4>(pv, g, ws, epoch, status, st);
  }
}

// The scans alone, on a workspace whose ticket and flags already read as zero.
static cudaError_t integrate_cleared(const PlanView& pv, const void* f, size_t f_pitch, uint64_t* g, void* ws,
                                     uint32_t* epoch, int32_t* status, cudaStream_t st) {
  switch (pv.limbs) {
    case 1: return integrate_L<1>(pv, f, f_pitch, g, ws, epoch, status, st);
    case 2: return integrate_L<2>(pv, f, f_pitch, g, ws, epoch, status, st);
    case 3: return integrate_L<3>(pv, f, f_pitch, g, ws, epoch, status, st);
    default: return integrate_L<4>(pv, f, f_pitch, g, ws, epoch, status, st);
  }
}

cudaError_t run_integrate(const PlanView& pv, const void* f, size_t f_pitch, uint64_t* g, void* ws,
                          uint32_t* epoch, int32_t* status, cudaStream_t st) {
  const cudaError_t e = cudaMemsetAsync(ws, 0, line_ws_zero_bytes(pv.Gw, pv.Gh), st);
  if (e != cudaSuccess) return e;
  return integrate_cleared(pv, f, f_pitch, g, ws, epoch, status, st);
}

// ----------------------------------------------------------------- batches
// The non-adaptive step of many images in one launch per pass: the images
// of one (limbs, order, input type) group share a row-pass launch (one CTA per
// row of any image) and one launch per line direction (every CTA takes a
// ticket; tickets run image by image and, within an image, band by band, so a
// look-back only waits on bands of its own image that hold earlier tickets).
// Each image keeps its own look-back workspace; all of them are cleared by one
// launch at the start.
constexpr int kMaxIntBatch = 96;

struct IntIn {
  PlanView pv;
  const void* f;
  size_t f_pitch;
  uint64_t* g;
  void* ws;
  int32_t* status;
};

struct IntJob {
  PlanView pv;
  const void* f;
  size_t f_pitch;
  uint64_t* g;
  LineWs ws;
  int32_t* status;
  long long first;  // first row (row pass) or ticket (line pass) of this image
};

struct IntJobs {
  int njobs;
  long long total;
  IntJob job[kMaxIntBatch];
};
static_assert(sizeof(IntJobs) <= 32000, "kernel parameter space");

struct ClearJobs {
  int n;
  uint4* ptr[kMaxIntBatch + 1];
  unsigned int words[kMaxIntBatch + 1];  // 16-byte words to clear
};

__global__ void clear_batch_kernel(const __grid_constant__ ClearJobs cj) {
  const int j = blockIdx.y;
  if (j >= cj.n) return;
  uint4* p = cj.ptr[j];
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < cj.words[j]; i += gridDim.x * blockDim.x)
    p[i] = make_uint4(0, 0, 0, 0);
}

__device__ __forceinline__ int find_int_job(const IntJobs& jobs, long long item) {
  int lo = 0, hi = jobs.njobs - 1;  // last job with first <= item
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs.job[mid].first <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int L, typename TIn, int NF>
__global__ void __launch_bounds__(32 * kRowWarps) row_scan_batch_kernel(const __grid_constant__ IntJobs jobs) {
  const long long b = blockIdx.x;
  const IntJob& jb = jobs.job[find_int_job(jobs, b)];
  row_scan_body<L, TIn, NF>(jb.pv, (const TIn*)jb.f, jb.f_pitch, jb.g, jb.status, (int)(b - jb.first));
}

// The same over the rows of all jobs with a warp per row (every job's rows
// short enough).
template <int L, typename TIn, int NF>
__global__ void __launch_bounds__(32 * kRowsPerCta) row_scan_batch_warp_kernel(const __grid_constant__ IntJobs jobs) {
  __shared__ Wide<L> s_tile[kRowsPerCta][32 * kRowVec];
  const int warp = threadIdx.x >> 5;
  const long long b = (long long)blockIdx.x * kRowsPerCta + warp;
  if (b >= jobs.total) return;
  const IntJob& jb = jobs.job[find_int_job(jobs, b)];
  row_scan_warp_body<L, TIn, NF>(jb.pv, (const TIn*)jb.f, jb.f_pitch, jb.g, jb.status, (int)(b - jb.first),
                                 s_tile[warp]);
}

template <int L, int DIR, int NF>
__global__ void __launch_bounds__(line_threads<L>()) line_scan_batch_kernel(const __grid_constant__ IntJobs jobs,
                                                                             uint32_t* ticket, uint32_t epoch) {
  __shared__ uint32_t s_ticket;
  if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1u);
  __syncthreads();
  const long long t = s_ticket;
  if (t >= jobs.total) return;
  const IntJob& jb = jobs.job[find_int_job(jobs, t)];
  const long long u = t - jb.first;
  const int band = (int)(u / jb.ws.ngroups), grp = (int)(u % jb.ws.ngroups);
  line_scan_body<L, DIR, NF>(jb.pv, jb.g, jb.ws, epoch, jb.status, band, grp);
}

template <int L, int DIR, int NF>
static cudaError_t launch_lines_batch(const IntIn* in, const int* idx, int m, uint32_t* ticket, uint32_t epoch,
                                      cudaStream_t st) {
  IntJobs jobs;
  jobs.njobs = m;
  long long t = 0;
  for (int k = 0; k < m; ++k) {
    const IntIn& b = in[idx[k]];
    IntJob& jb = jobs.job[k];
    jb.pv = b.pv;
    jb.f = b.f;
    jb.f_pitch = b.f_pitch;
    jb.g = b.g;
    jb.ws = carve<L>(b.ws, b.pv.Gw, b.pv.Gh, NF, DIR);
    jb.status = b.status;
    jb.first = t;
    t += (long long)jb.ws.nbands * jb.ws.ngroups;
  }
  jobs.total = t;
  if (t >= (1ll << 31)) return cudaErrorInvalidValue;
  constexpr int smem = band_smem_bytes<L>();
  static bool attr[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    e = cudaFuncSetAttribute(line_scan_batch_kernel<L, DIR, NF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  line_scan_batch_kernel<L, DIR, NF><<<(unsigned)t, line_threads<L>(), smem, st>>>(jobs, ticket, epoch);
  return cudaGetLastError();
}

template <int L, typename TIn, int NF>
static cudaError_t integrate_group(const IntIn* in, const int* idx, int m, uint32_t* tickets, uint32_t epoch0,
                                   cudaStream_t st) {
  IntJobs jobs;
  jobs.njobs = m;
  long long rows = 0;
  bool short_rows = true;
  for (int k = 0; k < m; ++k) {
    const IntIn& b = in[idx[k]];
    IntJob& jb = jobs.job[k];
    jb.pv = b.pv;
    jb.f = b.f;
    jb.f_pitch = b.f_pitch;
    jb.g = b.g;
    jb.status = b.status;
    jb.first = rows;
    rows += b.pv.Gh;
    short_rows = short_rows && b.pv.Gw <= kRowWarpMaxCells;
  }
  jobs.total = rows;
  if (rows >= (1ll << 31)) return cudaErrorInvalidValue;
  if (short_rows)
    row_scan_batch_warp_kernel<L, TIn, NF><<<(unsigned)((rows + kRowsPerCta - 1) / kRowsPerCta), 32 * kRowsPerCta, 0,
                                              st>>>(jobs);
  else
    row_scan_batch_kernel<L, TIn, NF><<<(unsigned)rows, 32 * kRowWarps, 0, st>>>(jobs);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_lines_batch<L, 2, NF>(in, idx, m, tickets + 0, epoch0 + 1, st);
  if (e == cudaSuccess) e = launch_lines_batch<L, 3, NF>(in, idx, m, tickets + 1, epoch0 + 2, st);
  if (e == cudaSuccess) e = launch_lines_batch<L, 4, NF>(in, idx, m, tickets + 2, epoch0 + 3, st);
  return e;
}

template <int L, typename TIn>
static cudaError_t integrate_group_n(int n, const IntIn* in, const int* idx, int m, uint32_t* tickets,
                                     uint32_t epoch0, cudaStream_t st) {
  if (n == 1) return integrate_group<L, TIn, 1>(in, idx, m, tickets, epoch0, st);
  if (n == 2) return integrate_group<L, TIn, 2>(in, idx, m, tickets, epoch0, st);
  return integrate_group<L, TIn, 3>(in, idx, m, tickets, epoch0, st);
}

template <int L>
static cudaError_t integrate_group_L(int n, int dtype, const IntIn* in, const int* idx, int m, uint32_t* tickets,
                                     uint32_t epoch0, cudaStream_t st) {
  switch (dtype) {
    case ABF_U8: return integrate_group_n<L, uint8_t>(n, in, idx, m, tickets, epoch0, st);
    case ABF_U16: return integrate_group_n<L, uint16_t>(n, in, idx, m, tickets, epoch0, st);
    case ABF_F32: return integrate_group_n<L, float>(n, in, idx, m, tickets, epoch0, st);
    default: return integrate_group_n<L, double>(n, in, idx, m, tickets, epoch0, st);
  }
}

int integrate_batch_max_jobs() { return kMaxIntBatch; }

// njobs <= kMaxIntBatch; ws: 256 bytes of device memory (ticket counters, one per
// pass, cleared here); epoch0: the first of 3 x (number of groups) epochs
// reserved for this call.
cudaError_t run_integrate_batch(const IntIn* in, int njobs, uint32_t* ws, uint32_t epoch0, cudaStream_t st) {
  if (njobs < 1 || njobs > kMaxIntBatch) return cudaErrorInvalidValue;
  ClearJobs cj;
  cj.n = njobs + 1;
  unsigned int most = 16;
  for (int i = 0; i < njobs; ++i) {
    cj.ptr[i] = (uint4*)in[i].ws;
    cj.words[i] = (unsigned int)(line_ws_zero_bytes(in[i].pv.Gw, in[i].pv.Gh) / 16);
    most = most > cj.words[i] ? most : cj.words[i];
  }
  cj.ptr[njobs] = (uint4*)ws;
  cj.words[njobs] = 16;
  const unsigned gx = (most + 255) / 256 < 64 ? (most + 255) / 256 : 64;
  clear_batch_kernel<<<dim3(gx, njobs + 1), 256, 0, st>>>(cj);
  cudaError_t e = cudaGetLastError();
  int done[kMaxIntBatch] = {};
  int group = 0;
  for (int i = 0; i < njobs && e == cudaSuccess; ++i) {
    if (done[i]) continue;
    int idx[kMaxIntBatch], m = 0;
    for (int k = i; k < njobs; ++k)
      if (!done[k] && in[k].pv.limbs == in[i].pv.limbs && in[k].pv.n == in[i].pv.n &&
          in[k].pv.in_dtype == in[i].pv.in_dtype) {
        idx[m++] = k;
        done[k] = 1;
      }
    if (group >= 20) return cudaErrorInvalidValue;  // 3 counters per group in 64
    uint32_t* tickets = ws + 3 * group;
    const uint32_t ep = epoch0 + 3 * (uint32_t)group;
    ++group;
    switch (in[i].pv.limbs) {
      case 1: e = integrate_group_L<1>(in[i].pv.n, in[i].pv.in_dtype, in, idx, m, tickets, ep, st); break;
      case 2: e = integrate_group_L<2>(in[i].pv.n, in[i].pv.in_dtype, in, idx, m, tickets, ep, st); break;
      case 3: e = integrate_group_L<3>(in[i].pv.n, in[i].pv.in_dtype, in, idx, m, tickets, ep, st); break;
      default: e = integrate_group_L<4>(in[i].pv.n, in[i].pv.in_dtype, in, idx, m, tickets, ep, st); break;
    }
  }
  return e;
}

// ------------------------------------------------------ fixed-scratch variant
// Scratch for abf_integrate_noalloc: callers that cannot allocate device
// memory get the line scans' look-back workspace from this fixed array instead
// of a buffer of their own.  It lives in the library's device image, so every
// GPU that loads the library holds it until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices] = {};

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

// Device address of the fixed scratch on the current device.  In host code the
// array's name only stands for it, so the address is looked up once per device
// (with that device current) and remembered.
static cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

// The same scans as run_integrate, on the fixed scratch (which clears the
// ticket and the flags first: the array keeps whatever the previous call left).
cudaError_t run_integrate_noalloc(const PlanView& pv, const void* f, size_t f_pitch, uint64_t* g, uint32_t* epoch,
                                  int32_t* status, cudaStream_t st) {
  void* ws = nullptr;
  const cudaError_t e = noalloc_scratch(&ws);
  if (e != cudaSuccess) return e;
  return run_integrate(pv, f, f_pitch, g, ws, epoch, status, st);
}

}  // namespace abf
