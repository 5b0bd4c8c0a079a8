// Host side of libabf: plans, the exact ZP^{*n} weight tables, and the C ABI.
//
// Weight table.  The interpolation kernel of Eq. (final_eqn) is the ZP element
// of Sec. 7 (the four-direction box spline with unit lattice directions
// v1..v4), n-fold self-convolved at order n: a box spline M with N = 4n
// directions.  Its values on the 2^-P grid are computed exactly, in integers, by
// the refinement equation of box splines,
//     M(y) = 2^(2-N) sum_k a_k M(2y - k),   sum_k a_k z^k = prod_xi (1 + z^xi),
// starting from its values at the integer points (the eigenvector of the same
// equation restricted to the integers, found in floating point, snapped to a
// rational with a factorial denominator and then verified exactly).  Each
// halving of the grid multiplies the common denominator by 2^(N-2), so
// D = D0 2^((4n-2) P) makes every table entry an integer (D0: the least common
// denominator of the integer-point values).  Every row (the 3n x 3n neighbours
// of one fractional offset) sums to D exactly (partition of unity); the
// generator checks that too.
#include <algorithm>
#include <cctype>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "abf_internal.cuh"

// ------------------------------------------------------- fault injection

namespace {
std::atomic<int> g_fault[4];
std::once_flag g_fault_env;

// ABF_FAULT = kind[:count][,kind[:count]...]
void fault_env() {
  const char* e = std::getenv("ABF_FAULT");
  if (!e) return;
  std::string v(e);
  size_t pos = 0;
  while (pos <= v.size()) {
    size_t end = v.find(',', pos);
    if (end == std::string::npos) end = v.size();
    std::string item = v.substr(pos, end - pos);
    int count = 1;
    const size_t colon = item.find(':');
    if (colon != std::string::npos) {
      count = std::atoi(item.c_str() + colon + 1);
      item = item.substr(0, colon);
    }
    int kind = item == "alloc" ? ABF_FAULT_ALLOC : item == "queue_stall" ? ABF_FAULT_QUEUE_STALL
                                                : item == "bad_desc" ? ABF_FAULT_BAD_DESC : 0;
    if (kind && count >= 0) g_fault[kind].store(count);
    pos = end + 1;
  }
}
}  // namespace

namespace abf {
bool fault_take(int kind) {
  std::call_once(g_fault_env, fault_env);
  int v = g_fault[kind].load();
  while (v > 0)
    if (g_fault[kind].compare_exchange_weak(v, v - 1)) return true;
  return false;
}
bool fault_active(int kind) {
  std::call_once(g_fault_env, fault_env);
  return g_fault[kind].load() > 0;
}
}  // namespace abf


namespace abf {
cudaError_t run_integrate(const PlanView& pv, const void* f, size_t f_pitch, uint64_t* g, void* ws,
                          uint32_t* epoch, int32_t* status, cudaStream_t st);
size_t line_ws_bytes(int Gw, int Gh, int L, int n, int* nbands_out, int* nlines_out);
cudaError_t run_mesh_exact(const PlanView& pv, const uint64_t* g, const void* scales, size_t scale_pitch, void* s,
                           size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status, int warps,
                           cudaStream_t st);
cudaError_t run_prepare_scales(const PlanView& pv, const void* scales, size_t scale_pitch, void* C, size_t C_pitch,
                               int32_t* status, cudaStream_t st);
cudaError_t run_measure_scales(const PlanView& pv, const void* scales, size_t scale_pitch,
                               unsigned long long* out2, int32_t* status, cudaStream_t st);
size_t noalloc_scratch_bytes();
int batch_max_jobs();
cudaError_t run_lookback_starved(const PlanView& pv, uint64_t* g, void* ws, uint32_t* epoch, int32_t* status,
                                 cudaStream_t st);
cudaError_t run_mesh_batch(const BatchIn* in, int njobs, unsigned long long* counter, int warps, cudaStream_t st);
size_t tile_ws_bytes(const PlanView& pv, int real_bytes, int* slots_out, size_t* slot_elems_out, size_t* off_bmax,
                     size_t* off_tiles, size_t* off_cnt, size_t* off_scratch);
cudaError_t run_tiles(const PlanView& pv, bool f64, const void* f, size_t f_pitch, const void* scales,
                      size_t scale_pitch, void* s, size_t s_pitch, void* ws, const void* wtab, double D0,
                      double tol_abs, int32_t* status, cudaStream_t st);
cudaError_t run_integrate_noalloc(const PlanView& pv, const void* f, size_t f_pitch, uint64_t* g, uint32_t* epoch,
                                  int32_t* status, cudaStream_t st);
struct IntIn {
  PlanView pv;
  const void* f;
  size_t f_pitch;
  uint64_t* g;
  void* ws;
  int32_t* status;
};
int integrate_batch_max_jobs();
abf_status create_general_plan(const abf_desc* d, abf_plan p);
void destroy_general_plan(abf_plan p);
cudaError_t run_integrate_general(abf_plan p, const void* f, size_t f_pitch, uint64_t* g, void* ws, uint32_t* epoch,
                                  int32_t* status, cudaStream_t st);
cudaError_t run_mesh_general(const PlanView& pv, const uint64_t* g, const void* scales, size_t scale_pitch, void* s,
                             size_t s_pitch, uint64_t* num, size_t num_pitch, int32_t* status, cudaStream_t st);
bool general_table_host(const int m[4], int P, std::vector<uint8_t>& bytes, std::vector<int2>& stencil,
                        unsigned __int128* D, int* wbytes);
cudaError_t run_integrate_batch(const IntIn* in, int njobs, uint32_t* ws, uint32_t epoch0, cudaStream_t st);
}  // namespace abf

using u128 = unsigned __int128;

namespace {

// ------------------------------------------------------------- weight tables

struct HostTable {
  std::vector<uint8_t> bytes;  // (2^P)^2 rows x row_len weights, little-endian
  u128 D = 0;
  int wbytes = 0;
  int row_len = 0;
  std::string err;
};

u128 gcd128(u128 a, u128 b) {
  while (b) {
    u128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

bool build_table(int n, int P, HostTable& out) {
  const int N = 4 * n;
  const int V[4][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 1}};
  // Mask prod_k (1 + z^{v_k})^n on x in [-n, 2n], y in [0, 3n].
  const int mw = 3 * n + 1, mh = 3 * n + 1, mx0 = -n;
  std::vector<int64_t> a(mw * mh, 0);
  a[(0 - mx0) + 0 * mw] = 1;
  for (int k = 0; k < 4; ++k)
    for (int r = 0; r < n; ++r) {
      std::vector<int64_t> b = a;
      for (int y = 0; y < mh; ++y)
        for (int xi = 0; xi < mw; ++xi) {
          const int64_t v = a[xi + y * mw];
          if (!v) continue;
          const int nx = xi + V[k][0], ny = y + V[k][1];
          if (nx < 0 || nx >= mw || ny < 0 || ny >= mh) { out.err = "mask out of range"; return false; }
          b[nx + ny * mw] += v;
        }
      a.swap(b);
    }
  auto mask_at = [&](int kx, int ky) -> int64_t {
    const int xi = kx - mx0;
    if (xi < 0 || xi >= mw || ky < 0 || ky >= mh) return 0;
    return a[xi + ky * mw];
  };
  // Integer-point values: v_p = 2^(2-N) sum_q a_{2p-q} v_q on the support points.
  const int npts = mw * mh;
  std::vector<long double> v(npts, 1.0L / npts), nv(npts);
  for (int it = 0; it < 400; ++it) {
    long double s = 0;
    for (int p = 0; p < npts; ++p) {
      const int px = p % mw + mx0, py = p / mw;
      long double acc = 0;
      for (int q = 0; q < npts; ++q) {
        const int64_t c = mask_at(2 * px - (q % mw + mx0), 2 * py - q / mw);
        if (c) acc += (long double)c * v[q];
      }
      nv[p] = acc;
      s += acc;
    }
    for (int p = 0; p < npts; ++p) v[p] = nv[p] / s;
  }
  // Snap to the denominator 2 (N-2)! and verify exactly.
  u128 Dc = 2;
  for (int i = 2; i <= N - 2; ++i) Dc *= (u128)i;
  std::vector<u128> Vq(npts);
  bool ok = false;
  for (int attempt = 0; attempt < 8 && !ok; ++attempt, Dc *= 2) {
    ok = true;
    u128 sum = 0;
    for (int p = 0; p < npts; ++p) {
      const long double x = v[p] * (long double)Dc;
      const long double r = std::floor(x + 0.5L);
      if (std::fabs((double)(x - r)) > 1e-3 || r < 0) { ok = false; break; }
      Vq[p] = (u128)r;
      sum += Vq[p];
    }
    if (!ok || sum != Dc) { ok = false; continue; }
    const u128 scale = (u128)1 << (N - 2);
    for (int p = 0; p < npts && ok; ++p) {
      const int px = p % mw + mx0, py = p / mw;
      u128 acc = 0;
      for (int q = 0; q < npts; ++q) {
        const int64_t c = mask_at(2 * px - (q % mw + mx0), 2 * py - q / mw);
        if (c) acc += (u128)c * Vq[q];
      }
      if (acc != scale * Vq[p]) ok = false;
    }
    if (ok) break;
  }
  if (!ok) { out.err = "integer-point values of ZP^n failed the exact check"; return false; }
  u128 g = Dc;
  for (int p = 0; p < npts; ++p) g = gcd128(g, Vq[p]);
  const u128 D0 = Dc / g;
  for (int p = 0; p < npts; ++p) Vq[p] /= g;

  // Refinement cascade to the 2^-P grid: level l has (3n 2^l + 1)^2 points,
  // index (i, j) <-> (x, y) = (-n + i 2^-l, j 2^-l).
  std::vector<u128> cur(Vq), nxt;
  int side = 3 * n + 1;
  std::vector<std::tuple<int, int, int64_t>> mk;
  for (int ky = 0; ky < mh; ++ky)
    for (int kx = mx0; kx < mx0 + mw; ++kx)
      if (mask_at(kx, ky)) mk.emplace_back(kx, ky, mask_at(kx, ky));
  for (int l = 1; l <= P; ++l) {
    const int nside = 3 * n * (1 << l) + 1;
    nxt.assign((size_t)nside * nside, 0);
    const int h = 1 << (l - 1);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nside; ++j) {
      for (int i = 0; i < nside; ++i) {
        u128 acc = 0;
        for (const auto& t : mk) {
          const int ip = i - (n + std::get<0>(t)) * h;
          const int jp = j - std::get<1>(t) * h;
          if (ip < 0 || ip >= side || jp < 0 || jp >= side) continue;
          acc += (u128)std::get<2>(t) * cur[(size_t)jp * side + ip];
        }
        nxt[(size_t)j * nside + i] = acc;
      }
    }
    cur.swap(nxt);
    side = nside;
  }
  const u128 D = D0 << ((N - 2) * P);
  // Centred table rows: row (ry, rx) holds D ZP^{*n}(r - d) for the stencil's
  // neighbours d, in the stencil's order.
  int scount = 0, sdx[81] = {0}, sdy[81] = {0};
  if (n == 1) { constexpr abf::Stencil<1> s{}; scount = s.count; for (int i = 0; i < s.count; ++i) { sdx[i] = s.dx[i]; sdy[i] = s.dy[i]; } }
  if (n == 2) { constexpr abf::Stencil<2> s{}; scount = s.count; for (int i = 0; i < s.count; ++i) { sdx[i] = s.dx[i]; sdy[i] = s.dy[i]; } }
  if (n == 3) { constexpr abf::Stencil<3> s{}; scount = s.count; for (int i = 0; i < s.count; ++i) { sdx[i] = s.dx[i]; sdy[i] = s.dy[i]; } }
  const int one = 1 << P;
  const int half = (n % 2 == 0) ? 0 : one / 2;
  const int wb = (n == 1) ? 4 : (n == 2 ? 8 : 16);
  if (n == 1 && D >= ((u128)1 << 32)) { out.err = "D too large for 32-bit weights"; return false; }
  if (n == 2 && D >= ((u128)1 << 60)) { out.err = "D too large for 64-bit weights"; return false; }
  if (n == 3 && D >= ((u128)1 << 121)) { out.err = "D too large for 128-bit weights"; return false; }
  const size_t rows = (size_t)one * one;
  out.bytes.assign(rows * scount * wb, 0);
  out.row_len = scount;
  bool sums_ok = true;
#pragma omp parallel for schedule(static) reduction(&& : sums_ok)
  for (int ry = 0; ry < one; ++ry) {
    for (int rx = 0; rx < one; ++rx) {
      u128 rowsum = 0;
      for (int c = 0; c < scount; ++c) {
        // uncentred point (r - d) + n (1/2, 3/2), in units of 2^-P
        const long X = (long)rx - half - (long)sdx[c] * one + (long)n * one / 2;
        const long Y = (long)ry - half - (long)sdy[c] * one + (long)3 * n * one / 2;
        const long i = X + (long)n * one, j = Y;
        u128 w = 0;
        if (i >= 0 && i < side && j >= 0 && j < side) w = cur[(size_t)j * side + i];
        rowsum += w;
        uint8_t* dst = &out.bytes[(((size_t)ry * one + rx) * scount + c) * wb];
        for (int b = 0; b < wb; ++b) dst[b] = (uint8_t)(w >> (8 * b));
      }
      if (rowsum != D) sums_ok = false;   // also proves the dropped neighbours are zero
    }
  }
  if (!sums_ok) { out.err = "ZP^n weight rows do not sum to D"; return false; }
  out.D = D;
  out.wbytes = wb;
  return true;
}

// Order-3 table folded by the symmetries of the square.  ZP^{*n} is invariant
// under x -> -x, y -> -y and x <-> y, so D ZP^{*n}(r - d) = F[S(r)][S(d)] for
// the symmetry S that takes the centred offset r = (Rx, Ry) 2^-P, Rx, Ry in
// [-2^(P-1), 2^(P-1)), to 0 <= X <= Y <= 2^(P-1) (flip x if Rx < 0, flip y if
// Ry < 0, then swap if X > Y).  F has (h+1)(h+2)/2 rows, h = 2^(P-1): row
// Y (Y+1)/2 + X, columns in stencil order.  Rows with Y = h (r_y = +1/2) are
// not in the full table; they come from the flipped row r_y = -1/2.  Every
// full-table entry is checked against its folded counterpart.
bool fold_table(const HostTable& ht, int n, int P, std::vector<uint8_t>& out) {
  int cnt = 0, cdx[81], cdy[81], idx[9][9];
  for (auto& row : idx)
    for (int& v : row) v = -1;
  if (n != 3) return false;
  {
    constexpr abf::Stencil<3> st{};
    cnt = st.count;
    for (int i = 0; i < cnt; ++i) {
      cdx[i] = st.dx[i];
      cdy[i] = st.dy[i];
      idx[st.dy[i] - st.kDmin][st.dx[i] - st.kDmin] = i;
    }
  }
  const int dmin = abf::Stencil<3>::kDmin;
  auto index_of = [&](int ex, int ey) -> int {
    if (ex < dmin || ex >= dmin + 9 || ey < dmin || ey >= dmin + 9) return -1;
    return idx[ey - dmin][ex - dmin];
  };
  const int one = 1 << P, h = one / 2;
  const size_t wb = (size_t)ht.wbytes, rowb = (size_t)cnt * wb;
  const size_t frows = (size_t)(h + 1) * (h + 2) / 2;
  out.assign(frows * rowb, 0);
  auto full_row = [&](int Rx, int Ry) { return ((size_t)(Ry + h) * one + (Rx + h)) * rowb; };
  bool ok = true;
  for (int Y = 0; Y <= h && ok; ++Y)
    for (int X = 0; X <= Y && ok; ++X) {
      const bool fy = Y == h, fx = X == h;  // preimage (X or -h, Y or -h) in the full table
      const int Rx = fx ? -h : X, Ry = fy ? -h : Y;
      uint8_t* dst = &out[((size_t)Y * (Y + 1) / 2 + X) * rowb];
      for (int e = 0; e < cnt; ++e) {
        const int c = index_of(fx ? -cdx[e] : cdx[e], fy ? -cdy[e] : cdy[e]);
        if (c < 0) { ok = false; break; }
        std::memcpy(dst + e * wb, &ht.bytes[full_row(Rx, Ry) + c * wb], wb);
      }
    }
  if (!ok) return false;
  // check: every full entry equals its folded counterpart
#pragma omp parallel for schedule(static) reduction(&& : ok)
  for (int Ry = -h; Ry < h; ++Ry) {
    for (int Rx = -h; Rx < h; ++Rx) {
      const bool fx = Rx < 0, fy = Ry < 0;
      int X = fx ? -Rx : Rx, Y = fy ? -Ry : Ry;
      const bool sw = X > Y;
      if (sw) std::swap(X, Y);
      const uint8_t* frow = &out[((size_t)Y * (Y + 1) / 2 + X) * rowb];
      for (int c = 0; c < cnt; ++c) {
        int ex = fx ? -cdx[c] : cdx[c], ey = fy ? -cdy[c] : cdy[c];
        if (sw) std::swap(ex, ey);
        const int e = index_of(ex, ey);
        if (e < 0 || std::memcmp(&ht.bytes[full_row(Rx, Ry) + c * wb], frow + e * wb, wb) != 0) ok = false;
      }
    }
  }
  return ok;
}

struct DeviceTable {
  void* ptr = nullptr;
  void* fold = nullptr;  // folded order-3 table (plus a zero row), else null
  u128 D = 0;
  int wbytes = 0;
};

std::mutex g_table_mu;
std::map<std::tuple<int, int, int>, DeviceTable> g_tables;  // (device, n, P); held until exit

abf_status get_table(int device, int n, int P, DeviceTable* out) {
  std::lock_guard<std::mutex> lk(g_table_mu);
  auto key = std::make_tuple(device, n, P);
  auto it = g_tables.find(key);
  if (it != g_tables.end()) {
    *out = it->second;
    return ABF_OK;
  }
  HostTable ht;
  try {
    if (!build_table(n, P, ht)) return ABF_ERR_UNSUPPORTED;
  } catch (const std::bad_alloc&) {
    return ABF_ERR_OOM;
  }
  // One all-zero row follows the 2^(2P) table rows: a tap known to read only
  // zeros of g may point there instead of being tested per lane.
  DeviceTable dt;
  const size_t row_bytes = (size_t)ht.row_len * ht.wbytes;
  if (cudaMalloc(&dt.ptr, ht.bytes.size() + row_bytes) != cudaSuccess) return ABF_ERR_OOM;
  if (cudaMemcpy(dt.ptr, ht.bytes.data(), ht.bytes.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset((char*)dt.ptr + ht.bytes.size(), 0, row_bytes) != cudaSuccess) {
    cudaFree(dt.ptr);
    return ABF_ERR_CUDA;
  }
  if (n == 3) {
    std::vector<uint8_t> fb;
    bool folded = false;
    try {
      folded = fold_table(ht, n, P, fb);
    } catch (const std::bad_alloc&) {
      cudaFree(dt.ptr);
      return ABF_ERR_OOM;
    }
    if (!folded) {
      cudaFree(dt.ptr);
      return ABF_ERR_UNSUPPORTED;
    }
    if (cudaMalloc(&dt.fold, fb.size() + row_bytes) != cudaSuccess) {
      cudaFree(dt.ptr);
      return ABF_ERR_OOM;
    }
    if (cudaMemcpy(dt.fold, fb.data(), fb.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset((char*)dt.fold + fb.size(), 0, row_bytes) != cudaSuccess) {
      cudaFree(dt.ptr);
      cudaFree(dt.fold);
      return ABF_ERR_CUDA;
    }
  }
  dt.D = ht.D;
  dt.wbytes = ht.wbytes;
  g_tables[key] = dt;
  *out = dt;
  return ABF_OK;
}

// Look-back flags carry an epoch so that the passes of one call need no
// clearing between them (the call clears the flags once, at its start).
// Epochs come from one process-wide counter.  Epoch 0 is never issued: it is
// the value of a cleared flag.
std::atomic<uint32_t> g_epoch{0};

uint32_t reserve_epochs(uint32_t count) {
  for (;;) {
    uint32_t base = g_epoch.fetch_add(count) & 0x3fffffffu;
    if (base + count <= 0x3fffffffu) return base;  // the scans use base+1 .. base+count
  }
}

// Pair copies of a weight table for the floating-point forms: entry w (the
// integer D ZP^{*n}) scaled by 2^-k, where D = D0 2^k with k = (4n - 2) P, as
// hi + lo with hi = w rounded to p bits and lo = the rest rounded to p bits
// (p = 53 or 24), both scaled by 2^-k (exact: a power of two).  The scaled
// rows sum to D0.
std::map<std::tuple<int, int, int, int>, std::pair<void*, double>> g_pair_tables;  // (device, n, P, bytes)

// v rounded to p significant bits, ties to even (an integer again).
u128 round_bits(u128 v, int p) {
  int b = 0;
  for (u128 t = v; t; t >>= 1) ++b;
  if (b <= p) return v;
  const int sh = b - p;
  const u128 q = v >> sh, rem = v & (((u128)1 << sh) - 1), half = (u128)1 << (sh - 1);
  u128 r = q;
  if (rem > half || (rem == half && (q & 1))) r += 1;
  return r << sh;
}

abf_status get_pair_table(int device, int n, int P, int real_bytes, void** out, double* D0_out) {
  std::lock_guard<std::mutex> lk(g_table_mu);
  auto key = std::make_tuple(device, n, P, real_bytes);
  auto it = g_pair_tables.find(key);
  if (it != g_pair_tables.end()) {
    *out = it->second.first;
    *D0_out = it->second.second;
    return ABF_OK;
  }
  HostTable ht;
  try {
    if (!build_table(n, P, ht)) return ABF_ERR_UNSUPPORTED;
  } catch (const std::bad_alloc&) {
    return ABF_ERR_OOM;
  }
  const int k = (4 * n - 2) * P;
  const u128 D0 = ht.D >> k;
  if ((D0 << k) != ht.D) return ABF_ERR_UNSUPPORTED;
  const int p = real_bytes == 8 ? 53 : 24;
  const size_t count = ht.bytes.size() / ht.wbytes;
  std::vector<uint8_t> buf(count * 2 * real_bytes);
  for (size_t i = 0; i < count; ++i) {
    u128 w = 0;
    for (int b = 0; b < ht.wbytes; ++b) w |= (u128)ht.bytes[i * ht.wbytes + b] << (8 * b);
    const u128 hi = round_bits(w, p);
    const bool neg = hi > w;
    const u128 lo = round_bits(neg ? hi - w : w - hi, p);
    if (real_bytes == 8) {
      const double h = std::ldexp((double)hi, -k), l = std::ldexp(neg ? -(double)lo : (double)lo, -k);
      std::memcpy(&buf[i * 16], &h, 8);
      std::memcpy(&buf[i * 16 + 8], &l, 8);
    } else {
      const float h = std::ldexp((float)hi, -k), l = std::ldexp(neg ? -(float)lo : (float)lo, -k);
      std::memcpy(&buf[i * 8], &h, 4);
      std::memcpy(&buf[i * 8 + 4], &l, 4);
    }
  }
  void* d = nullptr;
  if (cudaMalloc(&d, buf.size()) != cudaSuccess) return ABF_ERR_OOM;
  if (cudaMemcpy(d, buf.data(), buf.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return ABF_ERR_CUDA;
  }
  const double d0 = (double)(uint64_t)D0;
  g_pair_tables[key] = std::make_pair(d, d0);
  *out = d;
  *D0_out = d0;
  return ABF_OK;
}

double u128_to_double(u128 v) { return (double)(uint64_t)(v >> 64) * 18446744073709551616.0 + (double)(uint64_t)v; }

}  // namespace

// ------------------------------------------------------------------ the plan

static abf_status cuda_status(cudaError_t e) { return e == cudaSuccess ? ABF_OK : ABF_ERR_CUDA; }

abf_status abf::integrate_with_status(abf_plan p, const void* d_f, size_t f_pitch, void* d_g, void* d_ws,
                                      int32_t* d_status, cudaStream_t st) {
  if (!p || !d_f || !d_g || !d_ws || !d_status) return ABF_ERR_INVALID;
  if (p->desc.form != ABF_FORM_EXACT) return ABF_ERR_UNSUPPORTED;
  const size_t esz = p->pv.in_dtype == ABF_U8 ? 1 : p->pv.in_dtype == ABF_U16 ? 2 : p->pv.in_dtype == ABF_F32 ? 4 : 8;
  if (f_pitch < (size_t)p->pv.W * esz) return ABF_ERR_INVALID;
  if (((uintptr_t)d_g & 15) || ((uintptr_t)d_ws & 15)) return ABF_ERR_INVALID;
  uint32_t ep = reserve_epochs(3u * (uint32_t)p->pv.n);
  if (p->general)
    return cuda_status(abf::run_integrate_general(p, d_f, f_pitch, (uint64_t*)d_g, d_ws, &ep, d_status, st));
  return cuda_status(abf::run_integrate(p->pv, d_f, f_pitch, (uint64_t*)d_g, d_ws, &ep, d_status, st));
}

abf_status abf::filter_with_status(abf_plan p, const void* d_g, const void* d_scales, size_t scale_pitch, void* d_s,
                                   size_t s_pitch, int32_t* d_status, cudaStream_t st) {
  if (!p || !d_g || !d_scales || !d_s || !d_status) return ABF_ERR_INVALID;
  if (p->desc.form != ABF_FORM_EXACT) return ABF_ERR_UNSUPPORTED;
  const size_t osz = p->pv.out_dtype == ABF_F64 ? 8 : 4;
  if (scale_pitch < (size_t)p->pv.W * 16 || s_pitch < (size_t)p->pv.W * osz) return ABF_ERR_INVALID;
  if (((uintptr_t)d_scales & 15) || (scale_pitch & 15)) return ABF_ERR_INVALID;
  if (p->general)
    return cuda_status(abf::run_mesh_general(p->pv, (const uint64_t*)d_g, d_scales, scale_pitch, d_s, s_pitch, nullptr,
                                             0, d_status, st));
  return cuda_status(abf::run_mesh_exact(p->pv, (const uint64_t*)d_g, d_scales, scale_pitch, d_s, s_pitch, nullptr, 0,
                                         d_status, p->mesh_warps, st));
}



// The tuning cache (defined with the autotuner below).
static int tune_lookup(const std::string& key, int dflt);
static std::string plan_tune_key(abf_plan p);

extern "C" {

int32_t abf_version(void) { return 1; }

const char* abf_status_str(abf_status s) {
  switch (s) {
    case ABF_OK: return "ok";
    case ABF_ERR_INVALID: return "invalid argument";
    case ABF_ERR_OOM: return "out of memory";
    case ABF_ERR_CUDA: return "CUDA error";
    case ABF_ERR_UNSUPPORTED: return "unsupported";
    case ABF_ERR_RANGE: return "numerator exceeds the limb budget";
    case ABF_ERR_TIMEOUT: return "timeout";
    case ABF_ERR_BUSY: return "busy";
  }
  return "unknown status";
}

abf_status abf_debug_inject_fault(int32_t kind, int32_t count) {
  if (kind < ABF_FAULT_ALLOC || kind > ABF_FAULT_BAD_DESC || count < 0) return ABF_ERR_INVALID;
  std::call_once(g_fault_env, fault_env);
  g_fault[kind].store(count);
  return ABF_OK;
}

// ABF_FLAG_DEBUG_BOUNDS: the word that records the first pixel whose taps
// would read outside the lattice box (the mesh kernels check when pv.dbg is set).
static abf_status attach_debug_word(abf_plan p) {
  if (!(p->desc.flags & ABF_FLAG_DEBUG_BOUNDS)) return ABF_OK;
  if (cudaMalloc(&p->d_dbg, sizeof(unsigned long long)) != cudaSuccess) return ABF_ERR_OOM;
  if (cudaMemset(p->d_dbg, 0, sizeof(unsigned long long)) != cudaSuccess) return ABF_ERR_CUDA;
  p->pv.dbg = (unsigned long long*)p->d_dbg;
  return ABF_OK;
}

abf_status abf_plan_create(const abf_desc* d, abf_plan* out) {
  if (!d || !out) return ABF_ERR_INVALID;
  *out = nullptr;
  if (abf::fault_take(ABF_FAULT_BAD_DESC)) return ABF_ERR_INVALID;
  const int n = d->order_n;
  if (d->width < 1 || d->height < 1 || n < 1 || n > 3) return ABF_ERR_INVALID;
  if (d->in_dtype < ABF_U8 || d->in_dtype > ABF_F64) return ABF_ERR_INVALID;
  if (d->out_dtype != ABF_F32 && d->out_dtype != ABF_F64) return ABF_ERR_INVALID;
  if (d->scale_kind < ABF_SCALES_C4 || d->scale_kind > ABF_SCALES_ELLIPSE) return ABF_ERR_INVALID;
  if (d->q_bits < 1 || d->q_bits > (n == 1 ? 9 : 8)) return ABF_ERR_INVALID;
  if (d->in_frac_bits < 0 || d->in_frac_bits > 40) return ABF_ERR_INVALID;
  if (d->in_dtype <= ABF_U16 && d->in_frac_bits != 0) return ABF_ERR_INVALID;
  if (!(d->max_scale > 0) || !std::isfinite(d->max_scale) || d->max_scale > 4096) return ABF_ERR_INVALID;
  if (d->form < ABF_FORM_EXACT || d->form > ABF_FORM_TILE_F32) return ABF_ERR_INVALID;
  const bool exact = d->form == ABF_FORM_EXACT;
  const int Q = d->q_bits;
  const int P = (n % 2 == 0) ? Q : Q + 1;
  const double qd = std::ldexp(1.0, Q);
  const int Cmax = (int)std::lrint(d->max_scale * qd);
  const double min_scale = d->min_scale > 0 ? d->min_scale : 1.0;
  int Cmin = (int)std::ceil(min_scale * qd - 1e-9);
  if (Cmin < 1) Cmin = 1;
  if (Cmax < 1 || Cmin > Cmax) return ABF_ERR_INVALID;
  double vb = d->value_bound;
  if (!(vb > 0)) {
    if (d->in_dtype == ABF_U8) vb = 255.0;
    else if (d->in_dtype == ABF_U16) vb = 65535.0;
    else return ABF_ERR_INVALID;  // float input: the bound sizes the limbs / the error tolerance
  }
  // binary32 pairs reach 1e-5 (times the value bound) at order 1 only: see abf.h
  if (d->form == ABF_FORM_TILE_F32 && n != 1) return ABF_ERR_UNSUPPORTED;
  if (d->directions != 0 && d->directions != 2 && d->directions != 4) return ABF_ERR_INVALID;
  if (d->model_boxes < 0 || d->model_boxes > 6) return ABF_ERR_INVALID;
  const bool general = d->directions == 2 || d->model_boxes > 0;
  if (general && !exact) return ABF_ERR_UNSUPPORTED;
  if (d->flags & ~ABF_FLAG_DEBUG_BOUNDS) return ABF_ERR_INVALID;
  if ((d->flags & ABF_FLAG_DEBUG_BOUNDS) && !exact) return ABF_ERR_UNSUPPORTED;  // checks are in the exact mesh
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ABF_ERR_CUDA;

  abf_plan p = new (std::nothrow) abf_plan_s();
  if (!p) return ABF_ERR_OOM;
  p->desc = *d;
  p->device = dev;
  if (general) {
    abf_status gs = abf::create_general_plan(d, p);
    if (gs == ABF_OK && (abf::fault_take(ABF_FAULT_ALLOC) || cudaMalloc(&p->d_status, sizeof(int32_t)) != cudaSuccess))
      gs = ABF_ERR_OOM;
    if (gs == ABF_OK && cudaMemset(p->d_status, 0, sizeof(int32_t)) != cudaSuccess) gs = ABF_ERR_CUDA;
    if (gs == ABF_OK) gs = attach_debug_word(p);
    if (gs != ABF_OK) {
      abf::destroy_general_plan(p);
      if (p->d_status) cudaFree(p->d_status);
      if (p->d_dbg) cudaFree(p->d_dbg);
      delete p;
      return gs;
    }
    *out = p;
    return ABF_OK;
  }
  DeviceTable tab;
  abf_status s = get_table(dev, n, P, &tab);
  if (s != ABF_OK) { delete p; return s; }
  p->D = tab.D;

  // Numerator bound -> limbs.
  const double cmax = (double)Cmax / qd;
  const double prod = d->max_scale_product > 0 ? d->max_scale_product : std::pow(cmax, 4.0);
  const double cmin = (double)Cmin / qd;
  const double log2D = std::log2(u128_to_double(tab.D));
  const double lb = log2D + n * std::log2(prod) + std::log2(vb) + d->in_frac_bits +
                    2.0 * std::log2(1.0 + 1.0 / cmin) + 1e-6;
  const int L = exact ? (int)std::floor((lb + 1.0) / 64.0) + 1 : 1;
  if (L > abf::kMaxLimbs) { delete p; return ABF_ERR_RANGE; }

  // Lattice box: reads of a pixel span [m1 - E - 2n, m1 + E + n] x [m2 - E - 3n, m2 + E],
  // E = (n/2)(c_a + c_b + c_c) <= 1.5 n cmax.
  const double E = 1.5 * n * cmax;
  abf::PlanView& pv = p->pv;
  pv.W = d->width; pv.H = d->height; pv.n = n; pv.Q = Q; pv.P = P; pv.F = d->in_frac_bits;
  pv.left = (int)std::ceil(E + 2 * n);
  pv.right = (int)std::ceil(E + n);
  pv.above = (int)std::ceil(E);
  pv.Gw = pv.W + pv.left + pv.right;
  pv.Gh = pv.H + pv.above;
  pv.Gp = ((long long)pv.Gw + 3) / 4 * 4;
  pv.Cmax = Cmax; pv.Cmin = Cmin;
  pv.scale_kind = d->scale_kind; pv.in_dtype = d->in_dtype; pv.out_dtype = d->out_dtype;
  pv.limbs = L;
  pv.value_bound = vb;
  pv.log2D = log2D;
  pv.log2_base = (float)(log2D + std::log2(vb) + d->in_frac_bits);
  pv.Dd = u128_to_double(tab.D);
  pv.table_bytes_per_w = tab.wbytes;
  pv.table = tab.ptr;
  pv.table_fold = tab.fold;
  for (int k = 0; k < 4; ++k) pv.r[k] = n;
  pv.E = 0;
  pv.ox = pv.oy = 0;
  if (exact) {
    p->g_bytes = (size_t)pv.Gp * (size_t)pv.Gh * (size_t)L * 8;
    p->ws_bytes = abf::line_ws_bytes(pv.Gw, pv.Gh, L, n, nullptr, nullptr);
  } else {
    const int rb = d->form == ABF_FORM_PLAIN_F64 ? 8 : 4;
    abf_status rs = get_pair_table(dev, n, P, rb, &p->real_table, &p->D0);
    if (rs != ABF_OK) { delete p; return rs; }
    p->tol_abs = (d->form == ABF_FORM_PLAIN_F64 ? 1e-12 : 1e-5) * vb;
    int slots;
    size_t se, o1, o2, o3, o4;
    p->g_bytes = 0;
    p->ws_bytes = abf::tile_ws_bytes(pv, 2 * rb, &slots, &se, &o1, &o2, &o3, &o4);
  }
  if (abf::fault_take(ABF_FAULT_ALLOC) || cudaMalloc(&p->d_status, sizeof(int32_t)) != cudaSuccess) {
    delete p;
    return ABF_ERR_OOM;
  }
  if (cudaMemset(p->d_status, 0, sizeof(int32_t)) != cudaSuccess) {
    cudaFree(p->d_status);
    delete p;
    return ABF_ERR_CUDA;
  }
  const abf_status ds = attach_debug_word(p);
  if (ds != ABF_OK) {
    cudaFree(p->d_status);
    delete p;
    return ds;
  }
  if (exact) p->mesh_warps = tune_lookup(plan_tune_key(p), p->mesh_warps);  // a tuning kept from earlier runs
  *out = p;
  return ABF_OK;
}

abf_status abf_plan_destroy(abf_plan p) {
  if (!p) return ABF_ERR_INVALID;
  if (p->general) abf::destroy_general_plan(p);
  if (p->d_status) cudaFree(p->d_status);
  if (p->d_dbg) cudaFree(p->d_dbg);
  delete p;
  return ABF_OK;
}

abf_status abf_debug_bounds_violation(abf_plan p, int64_t* pixel) {
  if (!p || !pixel || !p->d_dbg) return ABF_ERR_INVALID;
  unsigned long long v = 0;
  if (cudaMemcpy(&v, p->d_dbg, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return ABF_ERR_CUDA;
  if (cudaMemset(p->d_dbg, 0, sizeof(v)) != cudaSuccess) return ABF_ERR_CUDA;
  *pixel = v ? (int64_t)(v - 1) : -1;
  return ABF_OK;
}

abf_status abf_plan_query(abf_plan p, size_t* integrated_bytes, size_t* workspace_bytes, int32_t* halo_lrbt,
                          int32_t* limbs, int64_t* g_pitch_elems) {
  if (!p) return ABF_ERR_INVALID;
  if (integrated_bytes) *integrated_bytes = p->g_bytes;
  if (workspace_bytes) *workspace_bytes = p->ws_bytes;
  if (halo_lrbt) {
    halo_lrbt[0] = p->pv.left;
    halo_lrbt[1] = p->pv.right;
    halo_lrbt[2] = 0;
    halo_lrbt[3] = p->pv.above;
  }
  if (limbs) *limbs = p->pv.limbs;
  if (g_pitch_elems) *g_pitch_elems = p->pv.Gp;
  return ABF_OK;
}

abf_status abf_plan_denominator(abf_plan p, uint32_t* w4) {
  if (!p || !w4) return ABF_ERR_INVALID;
  for (int i = 0; i < 4; ++i) w4[i] = (uint32_t)(p->D >> (32 * i));
  return ABF_OK;
}

abf_status abf_integrate(abf_plan p, const void* d_f, size_t f_pitch, void* d_g, void* d_ws, cudaStream_t st) {
  if (!p) return ABF_ERR_INVALID;
  return abf::integrate_with_status(p, d_f, f_pitch, d_g, d_ws, p->d_status, st);
}

abf_status abf_debug_starved_lookback(abf_plan p, void* d_g, void* d_ws, cudaStream_t st) {
  if (!p || !d_g || !d_ws) return ABF_ERR_INVALID;
  if (p->desc.form != ABF_FORM_EXACT) return ABF_ERR_UNSUPPORTED;
  if (((uintptr_t)d_g & 15) || ((uintptr_t)d_ws & 15)) return ABF_ERR_INVALID;
  uint32_t ep = reserve_epochs(1u);
  return cuda_status(abf::run_lookback_starved(p->pv, (uint64_t*)d_g, d_ws, &ep, p->d_status, st));
}

abf_status abf_integrate_noalloc(abf_plan p, const void* d_f, size_t f_pitch, void* d_g, cudaStream_t st) {
  if (!p || !d_f || !d_g) return ABF_ERR_INVALID;
  if (p->desc.form != ABF_FORM_EXACT) return ABF_ERR_UNSUPPORTED;
  const size_t esz = p->pv.in_dtype == ABF_U8 ? 1 : p->pv.in_dtype == ABF_U16 ? 2 : p->pv.in_dtype == ABF_F32 ? 4 : 8;
  if (f_pitch < (size_t)p->pv.W * esz) return ABF_ERR_INVALID;
  if ((uintptr_t)d_g & 15) return ABF_ERR_INVALID;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return ABF_ERR_CUDA;
  if (dev != p->device) return ABF_ERR_INVALID;
  if (p->ws_bytes > abf::noalloc_scratch_bytes() || p->general) return ABF_ERR_UNSUPPORTED;
  uint32_t ep = reserve_epochs(3u * (uint32_t)p->pv.n);
  return cuda_status(abf::run_integrate_noalloc(p->pv, d_f, f_pitch, (uint64_t*)d_g, &ep, p->d_status, st));
}

abf_status abf_filter(abf_plan p, const void* d_src, size_t src_pitch, const void* d_scales, size_t scale_pitch,
                      void* d_s, size_t s_pitch, void* d_ws, cudaStream_t st) {
  if (!p || !d_src || !d_scales || !d_s) return ABF_ERR_INVALID;
  const size_t osz = p->pv.out_dtype == ABF_F64 ? 8 : 4;
  if (scale_pitch < (size_t)p->pv.W * 16 || s_pitch < (size_t)p->pv.W * osz) return ABF_ERR_INVALID;
  if (((uintptr_t)d_scales & 15) || (scale_pitch & 15)) return ABF_ERR_INVALID;
  if (p->desc.form != ABF_FORM_EXACT) {
    const size_t esz = p->pv.in_dtype == ABF_U8 ? 1 : p->pv.in_dtype == ABF_U16 ? 2 : p->pv.in_dtype == ABF_F32 ? 4 : 8;
    if (!d_ws || src_pitch < (size_t)p->pv.W * esz) return ABF_ERR_INVALID;
    return cuda_status(abf::run_tiles(p->pv, p->desc.form == ABF_FORM_PLAIN_F64, d_src, src_pitch, d_scales,
                                      scale_pitch, d_s, s_pitch, d_ws, p->real_table, p->D0, p->tol_abs,
                                      p->d_status, st));
  }
  return abf::filter_with_status(p, d_src, d_scales, scale_pitch, d_s, s_pitch, p->d_status, st);
}

abf_status abf_filter_numerator(abf_plan p, const void* d_g, const void* d_scales, size_t scale_pitch, void* d_num,
                                size_t num_pitch, void* d_ws, cudaStream_t st) {
  (void)d_ws;
  if (!p || !d_g || !d_scales || !d_num) return ABF_ERR_INVALID;
  if (p->desc.form != ABF_FORM_EXACT) return ABF_ERR_UNSUPPORTED;
  if (scale_pitch < (size_t)p->pv.W * 16 || num_pitch < (size_t)p->pv.W * 8 * p->pv.limbs) return ABF_ERR_INVALID;
  if (((uintptr_t)d_scales & 15) || (scale_pitch & 15)) return ABF_ERR_INVALID;
  if (p->general)
    return cuda_status(abf::run_mesh_general(p->pv, (const uint64_t*)d_g, d_scales, scale_pitch, nullptr, 0,
                                             (uint64_t*)d_num, num_pitch, p->d_status, st));
  return cuda_status(abf::run_mesh_exact(p->pv, (const uint64_t*)d_g, d_scales, scale_pitch, nullptr, 0,
                                         (uint64_t*)d_num, num_pitch, p->d_status, p->mesh_warps, st));
}

int32_t abf_batch_max_jobs(void) { return abf::batch_max_jobs(); }

}  // extern "C"

// Tuning cache: the rows per CTA chosen for a plan (key "plan:<GPU>:n,L,W,H,Q,
// scale kind") or a batch composition (key "batch:<GPU>:" + the sorted (n,
// limbs, width, height) of its images), process-wide and, when the
// environment variable ABF_TUNE_CACHE names a file, kept there as a flat JSON
// object {"key": rows, ...}: read at the first lookup, rewritten (through a
// temporary file and a rename) after every tuning.  A file that does not parse
// is ignored.
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tuned;
static bool g_tune_loaded = false;

// The current device's name (queried once per device: the property query is slow).
static std::string gpu_name() {
  static std::mutex mu;
  static std::map<int, std::string> names;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::lock_guard<std::mutex> lk(mu);
  auto it = names.find(dev);
  if (it != names.end()) return it->second;
  cudaDeviceProp prop{};
  std::string n = "unknown";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) n = prop.name;
  else cudaGetLastError();
  for (char& c : n)
    if (c == '"' || c == '\\' || c == ':') c = '_';
  names[dev] = n;
  return n;
}

// Parses {"key": int, ...}; false (and nothing taken) on any other content.
static bool parse_tune_json(const std::string& t, std::map<std::string, int>& out) {
  std::map<std::string, int> m;
  size_t i = 0;
  auto ws = [&] { while (i < t.size() && std::isspace((unsigned char)t[i])) ++i; };
  ws();
  if (i >= t.size() || t[i] != '{') return false;
  ++i;
  ws();
  if (i < t.size() && t[i] == '}') { out.swap(m); return true; }
  for (;;) {
    ws();
    if (i >= t.size() || t[i] != '"') return false;
    const size_t k0 = ++i;
    while (i < t.size() && t[i] != '"') ++i;
    if (i >= t.size()) return false;
    const std::string key = t.substr(k0, i - k0);
    ++i;
    ws();
    if (i >= t.size() || t[i] != ':') return false;
    ++i;
    ws();
    const size_t v0 = i;
    while (i < t.size() && std::isdigit((unsigned char)t[i])) ++i;
    if (i == v0 || i - v0 > 6) return false;
    m[key] = std::atoi(t.substr(v0, i - v0).c_str());
    ws();
    if (i < t.size() && t[i] == ',') { ++i; continue; }
    if (i < t.size() && t[i] == '}') break;
    return false;
  }
  out.swap(m);
  return true;
}

// Call with g_tune_mu held.
static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("ABF_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "rb");
  if (!f) return;
  std::string t;
  char buf[4096];
  size_t k;
  while ((k = std::fread(buf, 1, sizeof buf, f)) > 0 && t.size() < (1u << 20)) t.append(buf, k);
  std::fclose(f);
  std::map<std::string, int> m;
  if (parse_tune_json(t, m))
    for (auto& kv : m)
      if (kv.second == 4 || kv.second == 8 || kv.second == 16) g_tuned[kv.first] = kv.second;
}

static void tune_save_locked() {
  const char* path = std::getenv("ABF_TUNE_CACHE");
  if (!path || !*path) return;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return;
  std::fputs("{", f);
  bool first = true;
  for (auto& kv : g_tuned) {
    std::fprintf(f, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
    first = false;
  }
  std::fputs("\n}\n", f);
  const bool ok = std::fclose(f) == 0;
  if (ok) std::rename(tmp.c_str(), path);
  else std::remove(tmp.c_str());
}

static int tune_lookup(const std::string& key, int dflt) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  auto it = g_tuned.find(key);
  return it != g_tuned.end() ? it->second : dflt;
}

static void tune_store(const std::string& key, int rows) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  g_tuned[key] = rows;
  tune_save_locked();
}

static std::string plan_tune_key(abf_plan p) {
  char buf[160];
  std::snprintf(buf, sizeof buf, "plan:%s:%d,%d,%d,%d,%d,%d", gpu_name().c_str(), p->pv.n, p->pv.limbs, p->pv.W,
                p->pv.H, p->pv.Q, p->pv.scale_kind);
  return buf;
}

static abf_status batch_inputs(const abf_job* jobs, int32_t njobs, std::vector<abf::BatchIn>& in, std::string* key) {
  in.resize((size_t)njobs);
  std::vector<std::tuple<int, int, int, int>> sig;
  for (int i = 0; i < njobs; ++i) {
    const abf_job& j = jobs[i];
    abf_plan p = j.plan;
    if (!p || !j.d_g || !j.d_scales || !j.d_s) return ABF_ERR_INVALID;
    if (p->desc.form != ABF_FORM_EXACT || p->general) return ABF_ERR_UNSUPPORTED;
    const size_t osz = p->pv.out_dtype == ABF_F64 ? 8 : 4;
    if (j.scale_pitch < (size_t)p->pv.W * 16 || j.s_pitch < (size_t)p->pv.W * osz) return ABF_ERR_INVALID;
    if (((uintptr_t)j.d_scales & 15) || (j.scale_pitch & 15)) return ABF_ERR_INVALID;
    in[i] = abf::BatchIn{p->pv, (const uint64_t*)j.d_g, j.d_scales, j.scale_pitch, j.d_s, j.s_pitch, p->d_status};
    sig.emplace_back(p->pv.n, p->pv.limbs, p->pv.W, p->pv.H);
  }
  if (key) {
    std::sort(sig.begin(), sig.end());
    *key = "batch:" + gpu_name() + ":";
    for (auto& t : sig) {
      char buf[64];
      std::snprintf(buf, sizeof buf, "%d.%d.%d.%d;", std::get<0>(t), std::get<1>(t), std::get<2>(t), std::get<3>(t));
      *key += buf;
    }
  }
  return ABF_OK;
}

static cudaError_t batch_launch(const std::vector<abf::BatchIn>& in, void* d_ws, int warps, cudaStream_t st) {
  const int chunk = abf::batch_max_jobs();
  const int njobs = (int)in.size();
  for (int b = 0; b < njobs; b += chunk) {
    const int k = std::min(chunk, njobs - b);
    cudaError_t e = abf::run_mesh_batch(in.data() + b, k, (unsigned long long*)d_ws, warps, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The tuner's candidates: rows (warps) per CTA of the mesh.
static const int kTuneWarps[3] = {4, 8, 16};

// Times fn(warps) for every candidate (one untimed run, then one timed run
// with CUDA events on the stream) and returns the fastest; ms[3] gets the
// times (ms).  Synchronises the stream.
template <typename F>
static abf_status tune_warps(F fn, cudaStream_t st, int* best, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return ABF_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ABF_ERR_CUDA;
  }
  abf_status res = ABF_OK;
  float bestms = 0;
  for (int i = 0; i < 3 && res == ABF_OK; ++i) {
    if (fn(kTuneWarps[i]) != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess ||
        fn(kTuneWarps[i]) != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess) {
      res = ABF_ERR_CUDA;
      break;
    }
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    if (ms) ms[i] = t;
    if (i == 0 || t < bestms) {
      bestms = t;
      *best = kTuneWarps[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return res;
}

extern "C" {

abf_status abf_integrate_batch(const abf_integrate_job* jobs, int32_t njobs, void* d_ws, size_t ws_bytes,
                               cudaStream_t st) {
  if (!jobs || njobs < 0 || !d_ws || ws_bytes < 256 || ((uintptr_t)d_ws & 15)) return ABF_ERR_INVALID;
  if (njobs == 0) return ABF_OK;
  std::vector<abf::IntIn> in((size_t)njobs);
  for (int i = 0; i < njobs; ++i) {
    const abf_integrate_job& j = jobs[i];
    abf_plan p = j.plan;
    if (!p || !j.d_f || !j.d_g || !j.d_ws) return ABF_ERR_INVALID;
    if (p->desc.form != ABF_FORM_EXACT || p->general) return ABF_ERR_UNSUPPORTED;
    const size_t esz = p->pv.in_dtype == ABF_U8 ? 1 : p->pv.in_dtype == ABF_U16 ? 2 : p->pv.in_dtype == ABF_F32 ? 4 : 8;
    if (j.f_pitch < (size_t)p->pv.W * esz) return ABF_ERR_INVALID;
    if (((uintptr_t)j.d_g & 15) || ((uintptr_t)j.d_ws & 15)) return ABF_ERR_INVALID;
    in[i] = abf::IntIn{p->pv, j.d_f, j.f_pitch, (uint64_t*)j.d_g, j.d_ws, p->d_status};
  }
  const int chunk = abf::integrate_batch_max_jobs();
  for (int b = 0; b < njobs; b += chunk) {
    const int k = std::min(chunk, njobs - b);
    const uint32_t ep = reserve_epochs(3u * (uint32_t)k);
    if (abf::run_integrate_batch(in.data() + b, k, (uint32_t*)d_ws, ep, st) != cudaSuccess) return ABF_ERR_CUDA;
  }
  return ABF_OK;
}

int32_t abf_integrate_batch_max_jobs(void) { return abf::integrate_batch_max_jobs(); }

abf_status abf_general_table_host(int32_t directions, int32_t n, int32_t model_boxes, int32_t q_bits, void* out,
                                  size_t out_bytes, size_t* needed_bytes, int32_t* wbytes, int32_t* R,
                                  int32_t* stencil_xy, uint32_t* D_words4) {
  if (directions != 2 && directions != 4) return ABF_ERR_INVALID;
  if (n < 1 || n > 3 || model_boxes < 0 || model_boxes > 6 || q_bits < 1 || q_bits > 7) return ABF_ERR_INVALID;
  const int m[4] = {n + model_boxes, directions == 4 ? n : 0, n + model_boxes, directions == 4 ? n : 0};
  std::vector<uint8_t> bytes;
  std::vector<int2> st;
  u128 D = 0;
  int wb = 0;
  try {
    if (!abf::general_table_host(m, q_bits + 1, bytes, st, &D, &wb)) return ABF_ERR_UNSUPPORTED;
  } catch (const std::bad_alloc&) {
    return ABF_ERR_OOM;
  }
  if (needed_bytes) *needed_bytes = bytes.size();
  if (wbytes) *wbytes = wb;
  if (R) *R = (int32_t)st.size();
  if (stencil_xy)
    for (size_t i = 0; i < st.size() && i < 256; ++i) {
      stencil_xy[2 * i] = st[i].x;
      stencil_xy[2 * i + 1] = st[i].y;
    }
  if (D_words4)
    for (int i = 0; i < 4; ++i) D_words4[i] = (uint32_t)(D >> (32 * i));
  if (out) {
    if (out_bytes < bytes.size()) return ABF_ERR_INVALID;
    std::memcpy(out, bytes.data(), bytes.size());
  }
  return ABF_OK;
}

abf_status abf_filter_batch(const abf_job* jobs, int32_t njobs, void* d_ws, size_t ws_bytes, cudaStream_t st) {
  if (!jobs || njobs < 0 || !d_ws || ws_bytes < 256 || ((uintptr_t)d_ws & 15)) return ABF_ERR_INVALID;
  if (njobs == 0) return ABF_OK;
  std::vector<abf::BatchIn> in;
  std::string key;
  abf_status s = batch_inputs(jobs, njobs, in, &key);
  if (s != ABF_OK) return s;
  const int warps = tune_lookup(key, 8);
  return batch_launch(in, d_ws, warps, st) == cudaSuccess ? ABF_OK : ABF_ERR_CUDA;
}

abf_status abf_plan_autotune(abf_plan p, const void* d_g, const void* d_scales, size_t scale_pitch, void* d_s,
                             size_t s_pitch, cudaStream_t st, int32_t* warps_out, float* ms3) {
  if (!p || !d_g || !d_scales || !d_s) return ABF_ERR_INVALID;
  if (p->desc.form != ABF_FORM_EXACT || p->general) return ABF_ERR_UNSUPPORTED;
  const size_t osz = p->pv.out_dtype == ABF_F64 ? 8 : 4;
  if (scale_pitch < (size_t)p->pv.W * 16 || s_pitch < (size_t)p->pv.W * osz) return ABF_ERR_INVALID;
  if (((uintptr_t)d_scales & 15) || (scale_pitch & 15)) return ABF_ERR_INVALID;
  int best = p->mesh_warps;
  abf_status s = tune_warps(
      [&](int w) {
        return abf::run_mesh_exact(p->pv, (const uint64_t*)d_g, d_scales, scale_pitch, d_s, s_pitch, nullptr, 0,
                                   p->d_status, w, st);
      },
      st, &best, ms3);
  if (s != ABF_OK) return s;
  p->mesh_warps = best;
  tune_store(plan_tune_key(p), best);
  if (warps_out) *warps_out = best;
  return ABF_OK;
}

abf_status abf_plan_rows(abf_plan p, int32_t* rows) {
  if (!p || !rows) return ABF_ERR_INVALID;
  *rows = p->mesh_warps;
  return ABF_OK;
}

abf_status abf_batch_autotune(const abf_job* jobs, int32_t njobs, void* d_ws, size_t ws_bytes, cudaStream_t st,
                              int32_t* warps_out, float* ms3) {
  if (!jobs || njobs <= 0 || !d_ws || ws_bytes < 256 || ((uintptr_t)d_ws & 15)) return ABF_ERR_INVALID;
  std::vector<abf::BatchIn> in;
  std::string key;
  abf_status s = batch_inputs(jobs, njobs, in, &key);
  if (s != ABF_OK) return s;
  int best = 8;
  s = tune_warps([&](int w) { return batch_launch(in, d_ws, w, st); }, st, &best, ms3);
  if (s != ABF_OK) return s;
  tune_store(key, best);
  if (warps_out) *warps_out = best;
  return ABF_OK;
}

abf_status abf_prepare_scales(abf_plan p, const void* d_scales, size_t scale_pitch, void* d_C, size_t C_pitch,
                              cudaStream_t st) {
  if (!p || !d_scales || !d_C) return ABF_ERR_INVALID;
  if (scale_pitch < (size_t)p->pv.W * 16 || C_pitch < (size_t)p->pv.W * 16) return ABF_ERR_INVALID;
  if (((uintptr_t)d_scales & 15) || (scale_pitch & 15) || ((uintptr_t)d_C & 15) || (C_pitch & 15))
    return ABF_ERR_INVALID;
  return cuda_status(abf::run_prepare_scales(p->pv, d_scales, scale_pitch, d_C, C_pitch, p->d_status, st));
}

abf_status abf_measure_scales(const abf_desc* d, const void* d_scales, size_t scale_pitch, double* max_step,
                              double* max_product, cudaStream_t st) {
  if (!d || !d_scales || !max_step || !max_product) return ABF_ERR_INVALID;
  if (d->width < 1 || d->height < 1 || d->order_n < 1 || d->order_n > 3) return ABF_ERR_INVALID;
  if (d->scale_kind < ABF_SCALES_C4 || d->scale_kind > ABF_SCALES_ELLIPSE) return ABF_ERR_INVALID;
  if (d->q_bits < 1 || d->q_bits > 9 || !(d->max_scale > 0)) return ABF_ERR_INVALID;
  if (scale_pitch < (size_t)d->width * 16 || (scale_pitch & 15) || ((uintptr_t)d_scales & 15)) return ABF_ERR_INVALID;
  abf::PlanView pv{};
  pv.W = d->width; pv.H = d->height; pv.n = d->order_n; pv.Q = d->q_bits;
  pv.scale_kind = d->scale_kind;
  pv.Cmax = (int)std::lrint(d->max_scale * std::ldexp(1.0, d->q_bits));
  void* buf = nullptr;
  if (cudaMalloc(&buf, 2 * sizeof(unsigned long long) + sizeof(int32_t)) != cudaSuccess) return ABF_ERR_OOM;
  int32_t* stw = (int32_t*)((char*)buf + 2 * sizeof(unsigned long long));
  abf_status rs = ABF_OK;
  unsigned long long h[2] = {0, 0};
  int32_t hs = 0;
  if (cudaMemsetAsync(stw, 0, sizeof(int32_t), st) != cudaSuccess ||
      abf::run_measure_scales(pv, d_scales, scale_pitch, (unsigned long long*)buf, stw, st) != cudaSuccess ||
      cudaMemcpyAsync(h, buf, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&hs, stw, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    rs = ABF_ERR_CUDA;
  cudaFree(buf);
  if (rs != ABF_OK) return rs;
  double a, b;
  std::memcpy(&a, &h[0], 8);
  std::memcpy(&b, &h[1], 8);
  *max_step = a;
  *max_product = b;
  return hs ? ABF_ERR_INVALID : ABF_OK;
}

abf_status abf_weight_table_host(int32_t n, int32_t q_bits, void* out, size_t out_bytes, size_t* needed_bytes,
                                 int32_t* wbytes, uint32_t* D_words4) {
  if (n < 1 || n > 3 || q_bits < 1 || q_bits > (n == 1 ? 9 : 8)) return ABF_ERR_INVALID;
  const int P = (n % 2 == 0) ? q_bits : q_bits + 1;
  HostTable ht;
  try {
    if (!build_table(n, P, ht)) return ABF_ERR_UNSUPPORTED;
  } catch (const std::bad_alloc&) {
    return ABF_ERR_OOM;
  }
  if (needed_bytes) *needed_bytes = ht.bytes.size();
  if (wbytes) *wbytes = ht.wbytes;
  if (D_words4)
    for (int i = 0; i < 4; ++i) D_words4[i] = (uint32_t)(ht.D >> (32 * i));
  if (out) {
    if (out_bytes < ht.bytes.size()) return ABF_ERR_INVALID;
    std::memcpy(out, ht.bytes.data(), ht.bytes.size());
  }
  return ABF_OK;
}

abf_status abf_last_device_status(abf_plan p, int32_t* code) {
  if (!p || !code) return ABF_ERR_INVALID;
  if (cudaDeviceSynchronize() != cudaSuccess) return ABF_ERR_CUDA;
  int32_t v = 0;
  if (cudaMemcpy(&v, p->d_status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return ABF_ERR_CUDA;
  if (cudaMemset(p->d_status, 0, sizeof(int32_t)) != cudaSuccess) return ABF_ERR_CUDA;
  *code = v;
  return ABF_OK;
}

}  // extern "C"
