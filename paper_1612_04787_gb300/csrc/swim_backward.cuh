// Affine-warp window preparation and the adjoint (backward) of the match.
//
// Forward with warps: the moving window of window b is the moving section
// resampled bilinearly at p(i, j) = origin + c + A (i - c, j - c) + t
// (theta = a_yy, a_yx, t_y, a_xy, a_xx, t_x; c = n/2), the reference window is
// gathered (or projected over K sections); both are written to the
// workspace as float32 windows and the streaming kernels run on them.
//
// Backward (gradients of L = sum_b gp_b peak_b + gs_b snr_b with the peak
// index, hence the background set, held fixed -- the argmax has no
// derivative).  The forward is recomputed, saving C and R, then:
//   dL/ds     delta at the peak (peak term) and the SNR Z-score derivative
//             over the background (built on the fly, never stored)
//   dL/dG     = DFT2(dL/ds)                         [rows: BK5, columns: BK6]
//   dL/dC     = e^{i phi} rho^-w [(1-w) Re u - i Im u] / n^2, u = conj(dL/dG) e^{i phi}
//   dL/dw     = -sum_k ln(rho_k) Re(conj(dL/dG_k) G_k)
//   dL/dM     = dL/dC R
//   dL/dm'    = Re(n^2 IDFT2(dL/dM))                [columns: BK6, rows: BK7]
//   dL/dm     = A dL/dm' - A sum(A dL/dm') / sum(A)
//   dL/dtheta = sum_ij dL/dm_ij grad(bilinear)(p_ij) dp_ij/dtheta   [BK8]
// All spectra are Hermitian, so only kx in [0, n/2] is transformed, with the
// real columns kx = 0 and kx = n/2 packed as one complex column.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "swim_stream.cuh"

namespace swift {

// ---------------------------------------------------------------------------
// BP: prepare float32 windows (affine resampling / gather / projection)
// ---------------------------------------------------------------------------
// Warped sample position of window pixel (i, j) in the moving section, as an
// exact integer base (the window centre, origin + n/2) plus a small FP32
// local offset a (i - n/2, j - n/2) + t (|offset| < ~n): its rounding stays
// near 1e-5 px, where adding it to a section coordinate would round to
// ~2e-4 px at 4096 and move samples across pixel lines (where the bilinear
// derivative jumps).  Gives the top-left tap, clamped to the last row or
// column pair, and the fraction from it.
__device__ __forceinline__ void warp_tap(int base, float local, int last_pair, int& t0, float& f) {
  const float fl = floorf(local);
  const int t = base + static_cast<int>(fl);
  t0 = min(t, last_pair);
  f = (local - fl) + static_cast<float>(t - t0);
}

// Whether every sample of the warped moving window lies in the image: the
// four corners of the window, mapped by the affine about its centre (cy, cx),
// within [0, h - 1] x [0, w - 1].  Part of the window guard of the kernels
// that read the warped window (preparation and the affine adjoint).
template <int N>
__device__ __forceinline__ bool warped_inside(const float (&th)[6], int cy, int cx, int h, int w) {
  const float c = 0.5f * N;
  bool ok = true;
#pragma unroll
  for (int corner = 0; corner < 4; ++corner) {
    const float di = (corner & 1 ? N - 1 : 0) - c, dj = (corner & 2 ? N - 1 : 0) - c;
    const float ly = th[0] * di + th[1] * dj + th[2];
    const float lx = th[3] * di + th[4] * dj + th[5];
    ok = ok && ly >= static_cast<float>(-cy) && lx >= static_cast<float>(-cx) && ly <= static_cast<float>(h - 1 - cy) &&
         lx <= static_cast<float>(w - 1 - cx);
  }
  return ok;
}

template <int N, typename TIn>
__global__ void __launch_bounds__(256) prep_kernel(const MatchLaunch L, const BackLaunch K, const BackWork BW,
                                                   long long b0) {
  constexpr int RB = 16;  // rows per CTA
  const long long s = blockIdx.x / (N / RB);
  const int rb = blockIdx.x % (N / RB);
  const long long b = b0 + s;
  const int tid = threadIdx.x;
  const int my = __ldg(L.mov_origin + 2 * b), mx = __ldg(L.mov_origin + 2 * b + 1);
  const int ry = __ldg(L.ref_origin + 2 * b), rx = __ldg(L.ref_origin + 2 * b + 1);
  // level and reference bounds through the shared guard (the moving window's
  // bounds are its warped corners, below)
  const int lv = L.level_idx != nullptr ? __ldg(L.level_idx + b) : L.level;
  const int guard = window_check(N, lv, L.level, ry, rx, 0, 0, L.ref_h, L.ref_w, N, N);
  if (guard == kWindowOtherLevel) {
    if (rb == 0 && tid == 0) BW.pre_status[s] = kStatusSkip;
    return;
  }
  float th[6] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f};
  if (K.affine != nullptr) {
#pragma unroll
    for (int k = 0; k < 6; ++k) th[k] = __ldg(K.affine + 6 * b + k);
  }
  const float c = 0.5f * N;
  const int cy = my + N / 2, cx = mx + N / 2;  // window centre: the integer base of every sample
  // bounds: the reference window, and the four corners of the warped moving window
  const bool ok = guard == SWIFT_WIN_OK && warped_inside<N>(th, cy, cx, L.mov_h, L.mov_w);
  if (rb == 0 && tid == 0) BW.pre_status[s] = ok ? SWIFT_WIN_OK : SWIFT_WIN_OUT_OF_BOUNDS;
  if (!ok) return;
  const TIn* mov = static_cast<const TIn*>(L.mov);
  const TIn* ref = static_cast<const TIn*>(L.ref) + static_cast<long long>(ry) * L.ref_pitch + rx;
  const float inv_k = 1.0f / static_cast<float>(L.ref_count);
  float* mp = BW.mp + s * N * N;
  float* rp = BW.rp + s * N * N;
  if constexpr (sizeof(TIn) == 1) {
    // uint8: thread (row, group) takes PT consecutive pixels of one row.  The
    // reference rows come in aligned 32-bit words (funnel-shifted to the
    // window's byte offset; the word after the last needed byte is not read)
    // and are summed over the sections as 16-bit integer lanes: exact, so
    // the mean equals the float sum of the pixels in any order.
    constexpr int PT = RB * N / 256;  // pixels per thread: n / 16
    constexpr int NW = PT / 4;        // output words of four pixels
    static_assert(PT % 4 == 0 && N / PT == 16, "16 threads per row, whole words");
    const int i = rb * RB + tid / 16, x0 = (tid % 16) * PT;
    uint32_t lo[NW], hi[NW];  // pixel sums: (p0, p1) and (p2, p3) of each word as 16-bit lanes
#pragma unroll
    for (int q = 0; q < NW; ++q) lo[q] = hi[q] = 0u;
    for (int k = 0; k < L.ref_count; ++k) {
      const uintptr_t a = reinterpret_cast<uintptr_t>(ref + k * L.ref_stride + static_cast<long long>(i) * L.ref_pitch + x0);
      const uint32_t* wp = reinterpret_cast<const uint32_t*>(a & ~static_cast<uintptr_t>(3));
      const uint32_t sh = 8u * static_cast<uint32_t>(a & 3);
      uint32_t w[NW + 1];
#pragma unroll
      for (int q = 0; q < NW; ++q) w[q] = __ldg(wp + q);
      w[NW] = sh ? __ldg(wp + NW) : 0u;
#pragma unroll
      for (int q = 0; q < NW; ++q) {
        const uint32_t o = __funnelshift_r(w[q], w[q + 1], sh);
        lo[q] += __byte_perm(o, 0u, 0x4140);
        hi[q] += __byte_perm(o, 0u, 0x4342);
      }
    }
    const float di = i - c;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      float4 r4 = make_float4(static_cast<float>(lo[q] & 0xffffu), static_cast<float>(lo[q] >> 16),
                              static_cast<float>(hi[q] & 0xffffu), static_cast<float>(hi[q] >> 16));
      if (L.ref_count > 1) r4 = make_float4(r4.x * inv_k, r4.y * inv_k, r4.z * inv_k, r4.w * inv_k);
      *reinterpret_cast<float4*>(rp + i * N + x0 + 4 * q) = r4;
      float mv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = x0 + 4 * q + u;
        const float dj = j - c;
        int y0, x0t;
        float fy, fx;
        warp_tap(cy, th[0] * di + th[1] * dj + th[2], L.mov_h - 2, y0, fy);
        warp_tap(cx, th[3] * di + th[4] * dj + th[5], L.mov_w - 2, x0t, fx);
        const TIn* p = mov + static_cast<long long>(y0) * L.mov_pitch + x0t;
        const float s00 = load_px<TIn>(p), s01 = load_px<TIn>(p + 1);
        const float s10 = load_px<TIn>(p + L.mov_pitch), s11 = load_px<TIn>(p + L.mov_pitch + 1);
        mv[u] = (1.f - fy) * ((1.f - fx) * s00 + fx * s01) + fy * ((1.f - fx) * s10 + fx * s11);
      }
      *reinterpret_cast<float4*>(mp + i * N + x0 + 4 * q) = make_float4(mv[0], mv[1], mv[2], mv[3]);
    }
    return;
  }
  for (int e = tid; e < RB * N; e += 256) {
    const int i = rb * RB + e / N, j = e % N;
    // reference (mean of ref_count sections)
    float rv = load_px<TIn>(ref + static_cast<long long>(i) * L.ref_pitch + j);
    for (int k = 1; k < L.ref_count; ++k) rv += load_px<TIn>(ref + k * L.ref_stride + static_cast<long long>(i) * L.ref_pitch + j);
    rp[i * N + j] = L.ref_count > 1 ? rv * inv_k : rv;
    // moving: bilinear sample at the warped position
    const float di = i - c, dj = j - c;
    int y0, x0;
    float fy, fx;
    warp_tap(cy, th[0] * di + th[1] * dj + th[2], L.mov_h - 2, y0, fy);
    warp_tap(cx, th[3] * di + th[4] * dj + th[5], L.mov_w - 2, x0, fx);
    const TIn* p = mov + static_cast<long long>(y0) * L.mov_pitch + x0;
    const float s00 = load_px<TIn>(p), s01 = load_px<TIn>(p + 1);
    const float s10 = load_px<TIn>(p + L.mov_pitch), s11 = load_px<TIn>(p + L.mov_pitch + 1);
    mp[i * N + j] = (1.f - fy) * ((1.f - fx) * s00 + fx * s01) + fy * ((1.f - fx) * s10 + fx * s11);
  }
}

// ---------------------------------------------------------------------------
// BK4: per-window forward statistics kept for the backward
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(32) back_stats_kernel(const MatchLaunch L, const StreamWork W, double* bst) {
  using G = StreamGeom<N>;
  const long long s = blockIdx.x;
  const int lane = threadIdx.x;
  double* o = bst + 8 * s;
  const int st = stat_status(W.stats[s]);
  if (st != SWIFT_WIN_OK) {
    if (lane == 0) o[6] = static_cast<double>(st == kStatusSkip ? kStatusSkip : st);
    return;
  }
  unsigned long long gk = 0ull;
  double ta = 0.0, tc = 0.0;
  for (int k = 0; k < G::NB3; ++k) {
    const unsigned long long* part = W.part + 3 * (s * G::NB3 + k);
    gk = part[0] > gk ? part[0] : gk;
    ta += __longlong_as_double(static_cast<long long>(part[1]));
    tc += __longlong_as_double(static_cast<long long>(part[2]));
  }
  const uint32_t pidx = key_index(gk);
  const int py = static_cast<int>(pidx / N), px = static_cast<int>(pidx % N);
  const float* surf = reinterpret_cast<const float*>(W.zr + s * N * N);
  const int R = static_cast<int>(sqrtf(L.radius2)) + 1;
  double da = 0.0, dc = 0.0, dn = 0.0;
  for (int e = lane; e < (2 * R + 1) * (2 * R + 1); e += 32) {
    const int dy = e / (2 * R + 1) - R, dx = e % (2 * R + 1) - R;
    if (static_cast<float>(dy * dy + dx * dx) <= L.radius2) {
      const double v = surf[((py + dy) & (N - 1)) * N + ((px + dx) & (N - 1))];
      da += v;
      dc += v * v;
      dn += 1.0;
    }
  }
  da = warp_sum_f64(da);
  dc = warp_sum_f64(dc);
  dn = warp_sum_f64(dn);
  if (lane == 0) {
    const double tn = static_cast<double>(N) * N - dn;
    const double mu = (ta - da) / tn;
    double var = (tc - dc) / tn - mu * mu;
    const double sd = var > 0.0 ? sqrt(var) : 0.0;
    const double pk = static_cast<double>(key_value(gk));
    o[0] = mu;
    o[1] = sd;
    o[2] = sd > 0.0 ? (pk - mu) / sd : 0.0;
    o[3] = pk;
    o[4] = py;
    o[5] = px;
    o[6] = sd > 0.0 ? SWIFT_WIN_OK : SWIFT_WIN_FLAT;  // no gradient through a zero-variance background
    o[7] = tn;
  }
}

// ---------------------------------------------------------------------------
// BK5: row DFTs of dL/ds (two real rows y, y + n/2 as one complex row)
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) back_grows_kernel(const MatchLaunch L, const BackLaunch K, const BackWork BW,
                                                          long long b0) {
  using G = StreamGeom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, PB = G::PB, RS = G::RS, T = G::T;
  constexpr int W2 = N / 2 + 1;
  const long long s = blockIdx.x / G::NB3;
  const int pb = blockIdx.x % G::NB3;
  const long long b = b0 + s;
  const int tid = threadIdx.x;
  const double* st = BW.bst + 8 * s;
  if (static_cast<int>(st[6]) != SWIFT_WIN_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* slab = reinterpret_cast<float2*>(smem_raw);  // [PB][RS]
  float2* twid = slab + PB * RS;
  for (int i = tid; i < N; i += T) twid[i] = L.twiddle[i];
  const float mu = static_cast<float>(st[0]), sd = static_cast<float>(st[1]), z = static_cast<float>(st[2]);
  const int py = static_cast<int>(st[4]), px = static_cast<int>(st[5]);
  const float nbg = static_cast<float>(st[7]);
  const float gp = __ldg(K.grad_peak + b), gs = __ldg(K.grad_snr + b);
  const float c_bg = -gs / (nbg * sd), c_dev = -gs * z / (nbg * sd * sd), c_pk = gp + gs / sd;
  const float* surf = reinterpret_cast<const float*>(BW.fw.zr + s * N * N);
  auto grad_s = [&](int y, int x) -> float {
    int dy = abs(y - py);
    dy = min(dy, N - dy);
    int dx = abs(x - px);
    dx = min(dx, N - dx);
    float g = (y == py && x == px) ? c_pk : 0.f;
    if (static_cast<float>(dy * dy + dx * dx) > L.radius2) g += c_bg + c_dev * (surf[y * N + x] - mu);
    return g;
  };
  for (int e = tid; e < PB * N; e += T) {
    const int p = e / N, x = e % N;
    const int y1 = pb * PB + p, y2 = y1 + N / 2;
    slab[p * RS + G::phys(x)] = make_float2(grad_s(y1, x), grad_s(y2, x));
  }
  __syncthreads();
  constexpr int TA = PB * R2, TB = PB * R1;
#pragma unroll
  for (int i = 0; i < (TA + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TA % T != 0 && task >= TA) break;
    const int p = task / R2, j = task % R2;
    float2* row = slab + p * RS;
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = row[G::phys(j + R2 * m)];
    dft<R1, -1>(v);
#pragma unroll
    for (int q = 0; q < R1; ++q) row[G::phys(j + R2 * q)] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < (TB + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TB % T != 0 && task >= TB) break;
    const int p = task / R1, k1 = task % R1;
    float2* row = slab + p * RS;
    float2 v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      const float2 x = row[G::phys(R2 * k1 + n2)];
      v[n2] = n2 == 0 ? x : cmul(x, twid[n2 * R1 + k1]);
    }
    dft<R2, -1>(v);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) row[G::phys(R2 * k1 + k2)] = v[k2];
  }
  __syncthreads();
  // unpack the two rows' half spectra: A = (Q[k] + conj Q[-k]) / 2, B = (Q[k] - conj Q[-k]) / 2i
  float2* gr = BW.gr + s * N * W2;
  for (int e = tid; e < PB * W2; e += T) {
    const int p = e / W2, kx = e % W2;
    const float2* row = slab + p * RS;
    const float2 q = row[G::phys(G::rho(kx))];
    const float2 qn = row[G::phys(G::rho((N - kx) & (N - 1)))];
    const int y1 = pb * PB + p, y2 = y1 + N / 2;
    gr[y1 * W2 + kx] = make_float2(0.5f * (q.x + qn.x), 0.5f * (q.y - qn.y));
    gr[y2 * W2 + kx] = make_float2(0.5f * (q.y + qn.y), -0.5f * (q.x - qn.x));
  }
}

// ---------------------------------------------------------------------------
// BK6: column DFTs of the row spectra -> dL/dG; whitening adjoint -> dL/dM,
//      dL/dw; inverse column DFTs of dL/dM
// ---------------------------------------------------------------------------
template <int N>
struct BackColGeom {
  static constexpr int R1 = StreamGeom<N>::R1, R2 = StreamGeom<N>::R2;
  static constexpr int CB = 256 / R2;            // lines per CTA (line 0 of block 0 packs kx = 0 and n/2)
  static constexpr int NB = (N / 2) / CB;
  static constexpr int LS = CB + 8;
};

template <int N>
__global__ void __launch_bounds__(256) back_gcols_kernel(const MatchLaunch L, const BackWork BW) {
  using G = StreamGeom<N>;
  using BG = BackColGeom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, CB = BG::CB, LS = BG::LS, T = 256;
  constexpr int W2 = N / 2 + 1;
  const long long s = blockIdx.x / BG::NB;
  const int cb = blockIdx.x % BG::NB;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (static_cast<int>(BW.bst[8 * s + 6]) != SWIFT_WIN_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* slab = reinterpret_cast<float2*>(smem_raw);  // [ky][lc]
  float2* dcbuf = slab + N * LS;
  float2* twid = dcbuf + N;
  __shared__ double wred[8];
  for (int i = tid; i < N; i += T) twid[i] = L.twiddle[i];
  const float2* gr = BW.gr + s * N * W2;
  for (int e = tid; e < N * CB; e += T) {
    const int lc = e % CB, y = e / CB;
    const int line = cb * CB + lc;
    float2 v;
    if (line == 0) {
      v = make_float2(gr[y * W2].x, gr[y * W2 + N / 2].x);  // both columns are real
    } else {
      v = gr[y * W2 + line];
    }
    slab[y * LS + lc] = v;
  }
  __syncthreads();
  constexpr int TA = CB * R2, TB = CB * R1;
#pragma unroll
  for (int i = 0; i < (TA + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TA % T != 0 && task >= TA) break;
    const int j = task / CB, lc = task % CB;
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = slab[(j + R2 * m) * LS + lc];
    dft<R1, -1>(v);
#pragma unroll
    for (int q = 0; q < R1; ++q) slab[(j + R2 * q) * LS + lc] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < (TB + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TB % T != 0 && task >= TB) break;
    const int k1 = task / CB, lc = task % CB;
    float2 v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      const float2 x = slab[(R2 * k1 + n2) * LS + lc];
      v[n2] = n2 == 0 ? x : cmul(x, twid[n2 * R1 + k1]);
    }
    dft<R2, -1>(v);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) slab[(R2 * k1 + k2) * LS + lc] = v[k2];
  }
  __syncthreads();
  // per bin: whitening adjoint
  const float w = L.w;
  const float inv_n2 = 1.0f / (static_cast<float>(N) * static_cast<float>(N));
  const float2* crC = BW.cr + s * 2 * N * W2;
  const float2* crR = crC + N * W2;
  float gw = 0.f;
  auto adjoint = [&](int ky, int kx, float2 gG) -> float2 {
    const float2 C = crC[ky * W2 + kx];
    const float rho2 = fmaf(C.x, C.x, C.y * C.y);
    if (!(rho2 > 0.f) || (kx == 0 && ky == 0)) return make_float2(0.f, 0.f);
    const float l2 = 0.5f * log2f(rho2);               // log2 rho
    const float pw = exp2f(-w * l2);                   // rho^-w
    const float inv_rho = exp2f(-l2);
    const float2 e = make_float2(C.x * inv_rho, C.y * inv_rho);
    const float2 u = make_float2(gG.x * e.x + gG.y * e.y, gG.x * e.y - gG.y * e.x);  // conj(gG) e
    const float sc = pw * inv_n2;
    const float ar = (1.f - w) * u.x, ai = -u.y;       // (1-w) Re u - i Im u
    const float2 gC = make_float2(sc * (e.x * ar - e.y * ai), sc * (e.x * ai + e.y * ar));
    // dL/dw term: -ln(rho) Re(conj(gG) G), G = C rho^-w / n^2
    const float reGG = (gG.x * C.x + gG.y * C.y) * sc;
    const float mult = (kx == 0 || kx == N / 2) ? 1.f : 2.f;
    gw -= mult * 0.69314718055994531f * l2 * reGG;
    const float2 R = crR[ky * W2 + kx];
    return cmul(gC, R);                                // dL/dM = dL/dC R
  };
#pragma unroll
  for (int i = 0; i < (TB + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TB % T != 0 && task >= TB) break;
    const int k1 = task / CB, lc = task % CB;
    const int line = cb * CB + lc;
    const bool packed = line == 0;
    float2 v[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int ky = k1 + R1 * k2;
      const float2 x = slab[(R2 * k1 + k2) * LS + lc];
      if (packed) {
        const float2 xn = slab[G::rho((N - ky) & (N - 1)) * LS];
        const float2 g0 = make_float2(0.5f * (x.x + xn.x), 0.5f * (x.y - xn.y));   // kx = 0
        const float2 gn = make_float2(0.5f * (x.y + xn.y), -0.5f * (x.x - xn.x));  // kx = n/2
        const float2 m0 = adjoint(ky, 0, g0), mn = adjoint(ky, N / 2, gn);
        v[k2] = make_float2(m0.x - mn.y, m0.y + mn.x);  // m0 + i mn (both columns real after the inverse)
      } else {
        v[k2] = adjoint(ky, line, x);
      }
    }
    dft<R2, +1>(v);
#pragma unroll
    for (int n2 = 1; n2 < R2; ++n2) v[n2] = cmulc(v[n2], twid[n2 * R1 + k1]);
    if (packed) {
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) dcbuf[R2 * k1 + n2] = v[n2];
    } else {
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) slab[(R2 * k1 + n2) * LS + lc] = v[n2];
    }
  }
  const double gwd = warp_sum_f64(static_cast<double>(gw));
  if (lane == 0) wred[warp] = gwd;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += wred[k];
    BW.gwp[s * BG::NB + cb] = t;
  }
  // inverse pass A' -> dL/dM inverse columns (natural y), stored like H
  float2* hm = BW.fw.h + s * N * (N / 2);
#pragma unroll
  for (int i = 0; i < (TA + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TA % T != 0 && task >= TA) break;
    const int n2 = task / CB, lc = task % CB;
    const int line = cb * CB + lc;
    float2 v[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = line == 0 ? dcbuf[n2 + R2 * k1] : slab[(n2 + R2 * k1) * LS + lc];
    dft<R1, +1>(v);
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) hm[(n2 + R2 * n1) * (N / 2) + line] = v[n1];
  }
}

// ---------------------------------------------------------------------------
// BK7: inverse row DFTs of dL/dM -> dL/dm' (real), taper-weighted block sums
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) back_grows_inv_kernel(const MatchLaunch L, const BackWork BW) {
  using G = StreamGeom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, PB = G::PB, RS = G::RS, T = G::T;
  const long long s = blockIdx.x / G::NB3;
  const int pb = blockIdx.x % G::NB3;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (static_cast<int>(BW.bst[8 * s + 6]) != SWIFT_WIN_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* slab = reinterpret_cast<float2*>(smem_raw);
  float2* twid = slab + PB * RS;
  float* tap = reinterpret_cast<float*>(twid + N);
  __shared__ double wsum[T / 32];
  for (int i = tid; i < N; i += T) {
    twid[i] = L.twiddle[i];
    tap[i] = L.taper[i];
  }
  const float2* hw = BW.fw.h + s * N * (N / 2);
  for (int e = tid; e < PB * (N / 2); e += T) {
    const int p = e / (N / 2), kx = e % (N / 2);
    const int y1 = pb * PB + p, y2 = y1 + N / 2;
    const float2 h1 = hw[y1 * (N / 2) + kx], h2 = hw[y2 * (N / 2) + kx];
    float2* row = slab + p * RS;
    if (kx == 0) {
      row[G::phys(0)] = make_float2(h1.x, h2.x);
      row[G::phys(N / 2)] = make_float2(h1.y, h2.y);
    } else {
      row[G::phys(kx)] = make_float2(h1.x - h2.y, h1.y + h2.x);
      row[G::phys(N - kx)] = make_float2(h1.x + h2.y, h2.x - h1.y);
    }
  }
  __syncthreads();
  constexpr int TA = PB * R2, TB = PB * R1;
#pragma unroll
  for (int i = 0; i < (TA + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TA % T != 0 && task >= TA) break;
    const int p = task / R2, j = task % R2;
    float2* row = slab + p * RS;
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = row[G::phys(j + R2 * m)];
    dft<R1, +1>(v);
#pragma unroll
    for (int q = 0; q < R1; ++q) row[G::phys(j + R2 * q)] = v[q];
  }
  __syncthreads();
  float* gmp = reinterpret_cast<float*>(BW.fw.zr + s * N * N);
  float acc = 0.f;
#pragma unroll
  for (int i = 0; i < (TB + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TB % T != 0 && task >= TB) break;
    const int p = task / R1, k1 = task % R1;
    const float2* row = slab + p * RS;
    float2 v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      const float2 x = row[G::phys(R2 * k1 + n2)];
      v[n2] = n2 == 0 ? x : cmulc(x, twid[n2 * R1 + k1]);
    }
    dft<R2, +1>(v);
    const int y1 = pb * PB + p, y2 = y1 + N / 2;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int x = k1 + R1 * k2;
      gmp[y1 * N + x] = v[k2].x;
      gmp[y2 * N + x] = v[k2].y;
      acc = fmaf(tap[y1] * tap[x], v[k2].x, fmaf(tap[y2] * tap[x], v[k2].y, acc));
    }
  }
  const double d = warp_sum_f64(static_cast<double>(acc));
  if (lane == 0) wsum[warp] = d;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int k = 0; k < T / 32; ++k) t += wsum[k];
    BW.gsum[s * G::NB3 + pb] = t;
  }
}

// ---------------------------------------------------------------------------
// BK8: taper/mean adjoint and the bilinear/affine adjoint -> dL/dtheta
// ---------------------------------------------------------------------------
template <int N, typename TIn>
__global__ void __launch_bounds__(256) back_affine_kernel(const MatchLaunch L, const BackLaunch K, const BackWork BW,
                                                          long long b0) {
  using G = StreamGeom<N>;
  constexpr int NBC = BackColGeom<N>::NB;
  const long long s = blockIdx.x;
  const long long b = b0 + s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ double red[8][6];
  __shared__ float tap[N];
  const int st = static_cast<int>(BW.bst[8 * s + 6]);
  if (st == kStatusSkip || BW.pre_status[s] == kStatusSkip) {
    if (tid == 0) BW.gwin[s] = 0.0;
    return;
  }
  if (st != SWIFT_WIN_OK) {
    if (tid < 6) K.grad_affine[6 * b + tid] = 0.f;
    if (tid == 0) BW.gwin[s] = 0.0;
    return;
  }
  for (int i = tid; i < N; i += 256) tap[i] = L.taper[i];
  double sa = 0.0;
  for (int k = 0; k < G::NB3; ++k) sa += BW.gsum[s * G::NB3 + k];
  const float mean_term = static_cast<float>(sa * L.inv_sum_a);  // sum(A g) / sum(A)
  float th[6] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f};
  if (K.affine != nullptr) {
#pragma unroll
    for (int k = 0; k < 6; ++k) th[k] = __ldg(K.affine + 6 * b + k);
  }
  const int my = __ldg(L.mov_origin + 2 * b), mx = __ldg(L.mov_origin + 2 * b + 1);
  const float c = 0.5f * N;
  const int cy = my + N / 2, cx = mx + N / 2;  // window centre: the integer base of every sample
  {
    // the window guard again, from the launch's own arrays: the samples below
    // are read only for a window of this level whose warped corners lie inside
    const int lv = L.level_idx != nullptr ? __ldg(L.level_idx + b) : L.level;
    if (lv != L.level || !warped_inside<N>(th, cy, cx, L.mov_h, L.mov_w)) {
      if (tid < 6 && lv == L.level) K.grad_affine[6 * b + tid] = 0.f;
      if (tid == 0) BW.gwin[s] = 0.0;
      return;
    }
  }
  const TIn* mov = static_cast<const TIn*>(L.mov);
  const float* gmp = reinterpret_cast<const float*>(BW.fw.zr + s * N * N);
  __syncthreads();
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int e = tid; e < N * N; e += 256) {
    const int i = e / N, j = e % N;
    const float gm = tap[i] * tap[j] * (gmp[e] - mean_term);
    const float di = i - c, dj = j - c;
    int y0, x0;
    float fy, fx;
    warp_tap(cy, th[0] * di + th[1] * dj + th[2], L.mov_h - 2, y0, fy);
    warp_tap(cx, th[3] * di + th[4] * dj + th[5], L.mov_w - 2, x0, fx);
    const TIn* p = mov + static_cast<long long>(y0) * L.mov_pitch + x0;
    const float s00 = load_px<TIn>(p), s01 = load_px<TIn>(p + 1);
    const float s10 = load_px<TIn>(p + L.mov_pitch), s11 = load_px<TIn>(p + L.mov_pitch + 1);
    const float dY = (1.f - fx) * (s10 - s00) + fx * (s11 - s01);
    const float dX = (1.f - fy) * (s01 - s00) + fy * (s11 - s10);
    const float gy = gm * dY, gx = gm * dX;
    acc[0] = fmaf(gy, di, acc[0]);
    acc[1] = fmaf(gy, dj, acc[1]);
    acc[2] += gy;
    acc[3] = fmaf(gx, di, acc[3]);
    acc[4] = fmaf(gx, dj, acc[4]);
    acc[5] += gx;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double v = warp_sum_f64(static_cast<double>(acc[k]));
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (tid < 6) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k][tid];
    K.grad_affine[6 * b + tid] = static_cast<float>(t);
  }
  if (tid == 0) {
    double t = 0.0;
    for (int k = 0; k < NBC; ++k) t += BW.gwp[s * NBC + k];
    BW.gwin[s] = t;
  }
}

// ---------------------------------------------------------------------------
// BK9: deterministic sum of the per-window dL/dw of a slice into the level's
//      accumulator (fixed order: strided per thread, then a fixed tree)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) back_wsum_kernel(const BackWork BW, long long count, double* acc) {
  __shared__ double red[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double t = 0.0;
  for (long long s = tid; s < count; s += 256) t += BW.gwin[s];
  t = warp_sum_f64(t);
  if (lane == 0) red[warp] = t;
  __syncthreads();
  if (tid == 0) {
    double u = 0.0;
    for (int k = 0; k < 8; ++k) u += red[k];
    *acc += u;
  }
}

}  // namespace swift
