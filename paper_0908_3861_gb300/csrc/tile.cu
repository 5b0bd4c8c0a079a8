// Floating-point forms of the filter: per-tile restart windows (binary64 or
// binary32).
//
// The non-adaptive step of Sec. 7 (1) is run not on the whole image but on a
// window around each output tile: the window holds every lattice point the
// tile's mesh reads, so it holds the support of every tile pixel's kernel, and
// filtering f restricted to the window gives the same result at the tile's
// pixels (the filter is linear; the kernel has compact support, Sec. 4).  The
// window keeps the running sums small enough for floating point: their size
// grows like the window extent to the power 4n.  Inside a window the
// recursions run in the paper's order (0, pi/4, pi/2, 3pi/4) with zero input
// outside the window; the last one (3pi/4) is cut at the window's right edge,
// which only changes g by a polynomial of degree < n along each 3pi/4 line, and
// the mesh's FD along v4 annihilates that.  Then the mesh of Eq. (final_eqn)
// runs exactly as in the exact form, in floating point: weights D ZP^{*n} / D.
//
// Tiles: the image is cut into 256 x 256 super-tiles, each split as a quadtree
// down to squares of side T in {8, ..., 256}: a square is split while T exceeds
// its smallest step (in pixels) and T > 8.  So a window is about T + 6n c_max
// wide with T <= c_min: the ratio window / step stays near 7 (keeping the
// running sums, and so the rounding amplification, small), and with T near
// the step the redundant scan work per pixel stays bounded too.
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
constexpr int kSlotsPerSm = 4;    // tile CTAs (scratch slots) per SM
template <int N>
__host__ __device__ constexpr int tile_threads() { return kTileThreads; }

struct TileRec {
  int x0, y0, T;               // tile origin and side (image coordinates)
  int wx0, wy0, ww, wh;        // window box [wx0, wx0 + ww) x [wy0, wy0 + wh)
};


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
__device__ __forceinline__ int signed_binom_t(int j) {
  const int c = (j == 0 || j == N) ? 1 : N;
  return (j & 1) ? -c : c;
}

// Integrate one window (in its scratch slot, row pitch ww) and filter the tile.
template <int N, typename Real, typename TOut>
__global__ void __launch_bounds__(tile_threads<N>()) tile_filter_kernel(
    const PlanView pv, const void* __restrict__ f, size_t f_pitch, const float4* __restrict__ scales,
    size_t scale_pitch, void* __restrict__ s, size_t s_pitch, const TileRec* __restrict__ tiles,
    const int* __restrict__ ntiles, int* __restrict__ counter, Real* __restrict__ scratch, size_t slot_elems,
    const Real* __restrict__ wtab, int32_t* status) {
  constexpr int R = stencil_count<N>();
  constexpr int TAPS = (N + 1) * (N + 1) * (N + 1) * (N + 1);
  constexpr int PAIRS = TAPS * R;
  constexpr int ITERS = (PAIRS + 31) / 32;
  constexpr int WARPS = tile_threads<N>() / 32;
  __shared__ int s_dx[R], s_dy[R];
  __shared__ int4 s_tap[WARPS][TAPS];
  __shared__ int s_t;
  if (threadIdx.x == 0) {
    int c = 0;
    for (int iy = 0; iy < 3 * N; ++iy)
      for (int ix = 0; ix < 3 * N; ++ix)
        if (stencil_keeps<N>(ix, iy)) {
          s_dx[c] = Stencil<N>::kDmin + ix;
          s_dy[c] = Stencil<N>::kDmin + iy;
          ++c;
        }
  }
  Real* gw = scratch + (size_t)blockIdx.x * slot_elems;
  const int nt = *ntiles;
  const int lane = threadIdx.x & 31, wslot = threadIdx.x >> 5;
  const int P = pv.P;
  const int sh = (N % 2 == 0) ? 0 : 1;
  const int one = 1 << pv.Q;
  const int half = (N % 2 == 0) ? 0 : (1 << (P - 1));
  const int mask = (1 << P) - 1;
  const Real fscale = (Real)1.0;

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_t = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= nt) break;
    const TileRec tr = tiles[t];
    const int ww = tr.ww, wh = tr.wh;
    // v1: rows, n running sums each, input = f restricted to the window
    for (int r = threadIdx.x; r < wh; r += blockDim.x) {
      const int y = tr.wy0 + r;
      Real acc[N];
#pragma unroll
      for (int k = 0; k < N; ++k) acc[k] = 0;
      Real* row = gw + (size_t)r * ww;
      for (int c = 0; c < ww; ++c) {
        const int x = tr.wx0 + c;
        Real v = 0;
        if (y >= 0 && y < pv.H && x >= 0 && x < pv.W) v = (Real)fetch_f(pv.in_dtype, f, f_pitch, x, y) * fscale;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          acc[k] += v;
          v = acc[k];
        }
        row[c] = v;
      }
    }
    __syncthreads();
    // v2 (from (x-1, y-1)), v3 (from (x, y-1)), v4 (from (x+1, y-1)): n times
    // each.  A thread owns whole lines of the direction (sheared columns), so a
    // pass needs no barrier between rows; a line's running sum starts where the
    // line enters the window.
    for (int dir = 2; dir <= 4; ++dir) {
      const int nlines = (dir == 3) ? ww : ww + wh - 1;
      for (int k = 0; k < N; ++k) {
        for (int l = threadIdx.x; l < nlines; l += blockDim.x) {
          Real acc = 0;
          for (int r = 0; r < wh; ++r) {
            const int c = dir == 2 ? l - (wh - 1) + r : (dir == 3 ? l : l - r);
            if (c < 0 || c >= ww) {
              acc = 0;
              continue;
            }
            Real* p = gw + (size_t)r * ww + c;
            acc += *p;
            *p = acc;
          }
        }
        __syncthreads();
      }
    }
    // mesh for the tile's pixels: warp w takes pixels w, w + WARPS, ... in
    // batches of 32 (lane i reads the scales of the batch's i-th pixel)
    const int tw = min(tr.T, pv.W - tr.x0), th = min(tr.T, pv.H - tr.y0);
    const int npx = tw * th;
    for (int base = wslot * 32; base < npx; base += WARPS * 32) {
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
      Real mine = 0;
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
          const int j1 = q % (N + 1), q1 = q / (N + 1);
          const int j3 = q1 % (N + 1), q2 = q1 / (N + 1);
          const int j2 = q2 % (N + 1), j4 = q2 / (N + 1);
          const int w = signed_binom_t<N>(j1) * signed_binom_t<N>(j2) * signed_binom_t<N>(j3) * signed_binom_t<N>(j4);
          const int Yx = y0x - j1 * s1 - j2 * s2 + j4 * s4;
          const int Yy = y0y - j2 * s2 - j3 * s3 - j4 * s4;
          const int px = (Yx + half) >> P;
          const int py = (Yy + half) >> P;
          const int r = (((Yy + half) & mask) << P) | ((Yx + half) & mask);
          taps[q] = make_int4(px - tr.wx0, py - tr.wy0, r, w);
        }
        __syncwarp();
        Real acc = 0;
        Real ak[5] = {0, 0, 0, 0, 0};  // n = 2: accumulators for |w_j| = 1, 2, 4, 8, 16
#pragma unroll 8
        for (int it = 0; it < ITERS; ++it) {
          const int pair = it * 32 + lane;
          if (PAIRS % 32 != 0 && pair >= PAIRS) continue;
          const int tap = (R == 32) ? it : pair / R;
          const int cand = (R == 32) ? lane : pair - tap * R;
          const int4 ti = taps[tap];
          const int k1 = ti.x + s_dx[cand], k2 = ti.y + s_dy[cand];
          // reads stay inside the window by construction
          const Real gv = gw[(size_t)k2 * ww + k1];
          const Real wv = wtab[(size_t)ti.z * R + cand];
          if constexpr (N == 1) {
            acc = fma(ti.w < 0 ? -wv : wv, gv, acc);
          } else if constexpr (N == 2) {
            const Real sw = ti.w < 0 ? -wv : wv;
            switch (__ffs(ti.w < 0 ? -ti.w : ti.w) - 1) {  // uniform across the warp for n = 2
              case 0: ak[0] = fma(sw, gv, ak[0]); break;
              case 1: ak[1] = fma(sw, gv, ak[1]); break;
              case 2: ak[2] = fma(sw, gv, ak[2]); break;
              case 3: ak[3] = fma(sw, gv, ak[3]); break;
              default: ak[4] = fma(sw, gv, ak[4]); break;
            }
          } else {
            acc = fma((Real)ti.w * wv, gv, acc);
          }
        }
        if constexpr (N == 2) acc = ak[0] + (Real)2 * ak[1] + (Real)4 * ak[2] + (Real)8 * ak[3] + (Real)16 * ak[4];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == pp) {
          double den = 1.0;
          const int Cp[4] = {c0, c1, c2, c3};
          for (int k2i = 0; k2i < 4; ++k2i) {
            double ck = ldexp((double)Cp[k2i], -pv.Q), pw = 1.0;
            for (int e = 0; e < N; ++e) pw *= ck;
            den *= pw;
          }
          mine = (Real)((double)acc / den);
        }
      }
      if (myp < npx) {
        TOut* orow = reinterpret_cast<TOut*>(reinterpret_cast<char*>(s) + (size_t)y * s_pitch);
        if (ok == 1) {
          orow[myx] = (TOut)mine;
        } else {
          raise_status(status, ABF_DEV_BAD_SCALE);
          orow[myx] = (TOut)__longlong_as_double(0x7ff8000000000000ll);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- launcher

size_t tile_ws_bytes(const PlanView& pv, int real_bytes, int* slots_out, size_t* slot_elems_out,
                     size_t* off_bmax, size_t* off_tiles, size_t* off_cnt, size_t* off_scratch) {
  const int n = pv.n;
  const double cmax = (double)pv.Cmax / (double)(1 << pv.Q);
  const int E = (int)ceil(1.5 * n * cmax);
  const int mgn = E + 3 * n + 1;
  const int side = kSuper + 2 * mgn;  // largest window side (T <= 256)
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
  *off_scratch = off; off += (size_t)slots * slot_elems * real_bytes;
  *slots_out = slots;
  *slot_elems_out = slot_elems;
  return off;
}

template <int N, typename Real>
static cudaError_t run_tiles_N(const PlanView& pv, const void* f, size_t f_pitch, const void* scales,
                               size_t scale_pitch, void* s, size_t s_pitch, void* ws, const void* wtab,
                               int32_t* status, cudaStream_t st) {
  int slots;
  size_t slot_elems, ob, otl, oc, osc;
  tile_ws_bytes(pv, sizeof(Real), &slots, &slot_elems, &ob, &otl, &oc, &osc);
  char* base = (char*)ws;
  const int bw = (pv.W + kBlk - 1) / kBlk, bh = (pv.H + kBlk - 1) / kBlk;
  int4* bmin = (int4*)(base + ob);
  int4* bmax = bmin + (((size_t)bw * bh * sizeof(int4) + 255) / 256 * 256) / sizeof(int4);
  TileRec* tiles = (TileRec*)(base + otl);
  int* cnt = (int*)(base + oc);     // [0] tile count, [1] work counter
  Real* scratch = (Real*)(base + osc);
  cudaError_t e = cudaMemsetAsync(cnt, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  block_steps_kernel<<<dim3(bw, bh), kBlk * kBlk, 0, st>>>(pv, (const float4*)scales, scale_pitch, bmin, bmax, status);
  const int nsuper = ((pv.W + kSuper - 1) / kSuper) * ((pv.H + kSuper - 1) / kSuper);
  tile_list_kernel<<<(nsuper + 63) / 64, 64, 0, st>>>(pv, bmin, bmax, bw, bh, tiles, cnt);
  if (pv.out_dtype == ABF_F64)
    tile_filter_kernel<N, Real, double><<<slots, tile_threads<N>(), 0, st>>>(
        pv, f, f_pitch, (const float4*)scales, scale_pitch, s, s_pitch, tiles, cnt, cnt + 1, scratch, slot_elems,
        (const Real*)wtab, status);
  else
    tile_filter_kernel<N, Real, float><<<slots, tile_threads<N>(), 0, st>>>(
        pv, f, f_pitch, (const float4*)scales, scale_pitch, s, s_pitch, tiles, cnt, cnt + 1, scratch, slot_elems,
        (const Real*)wtab, status);
  return cudaGetLastError();
}

cudaError_t run_tiles(const PlanView& pv, bool f64, const void* f, size_t f_pitch, const void* scales,
                      size_t scale_pitch, void* s, size_t s_pitch, void* ws, const void* wtab, int32_t* status,
                      cudaStream_t st) {
  if (f64) {
    switch (pv.n) {
      case 1: return run_tiles_N<1, double>(pv, f, f_pitch, scales, scale_pitch, s, s_pitch, ws, wtab, status, st);
      case 2: return run_tiles_N<2, double>(pv, f, f_pitch, scales, scale_pitch, s, s_pitch, ws, wtab, status, st);
      default: return run_tiles_N<3, double>(pv, f, f_pitch, scales, scale_pitch, s, s_pitch, ws, wtab, status, st);
    }
  }
  switch (pv.n) {
    case 1: return run_tiles_N<1, float>(pv, f, f_pitch, scales, scale_pitch, s, s_pitch, ws, wtab, status, st);
    case 2: return run_tiles_N<2, float>(pv, f, f_pitch, scales, scale_pitch, s, s_pitch, ws, wtab, status, st);
    default: return run_tiles_N<3, float>(pv, f, f_pitch, scales, scale_pitch, s, s_pitch, ws, wtab, status, st);
  }
}

}  // namespace abf
