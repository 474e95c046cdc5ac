// Streaming forward matching: five kernels of small independent CTAs that
// pass each window's intermediates through a plan-owned workspace.
//
//   K0 stats     one CTA per window: bounds, flat / non-finite checks and the
//                taper-weighted means of both windows
//   K1 rows      (window, row block): apodise z = m' + i r', 1D DFT of each row
//                -> Zr[y][kx]
//   K2 columns   (window, column block closed under kx -> -kx): 1D DFT of the
//                columns, Hermitian unpack of M and R, C = M conj(R),
//                whitening G = C |C|^-w / n^2 (G[0,0] = 0), inverse DFT of the
//                columns kx in [0, n/2] -> H[y][kx] (kx = 0 carries kx = n/2
//                as its imaginary part)
//   K3 inv rows  (window, block of row pairs): rows y and y + n/2 of H form one
//                complex row (Hermitian completion), inverse DFT -> match
//                response s for both rows; block argmax
//   K4 finalize  one CTA per window: global argmax, SNR over the background
//                outside the exclusion disc, subpixel parabola fit, result
//
// Every CTA works alone (no clusters, no cross-CTA waits), so many CTAs share
// an SM and hide each other's latency.  1D transforms use the same in-place
// two-pass radix scheme as the fused kernel (pass A strided, pass B on
// contiguous blocks with twiddles; "rho" digit-reversed order in between).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dft_regs.cuh"
#include "swim_kernel.cuh"
#include "swift_internal.h"

namespace swift {

constexpr int kStatusSkip = kWindowOtherLevel;  // window of another level: no result written here
// flags of a row-block statistics record (the row kernel's STATS mode)
constexpr int kRowDiffM = 1;      // a moving pixel differs from the moving window's first pixel
constexpr int kRowDiffR = 2;      // a reference pixel differs from the reference window's first pixel
constexpr int kRowNonFinite = 4;  // a non-finite float pixel
constexpr int kRowTimeout = 8;    // the block's staged rows never arrived

template <int N>
struct StreamGeom {
  static constexpr int R1 = N == 64 ? 8 : 16;
  static constexpr int R2 = N / R1;        // 8, 8, 16, 32 for n = 64 .. 512
  static constexpr int T = 256;
  static constexpr int RS = N == 512 ? 528 : (N == 256 ? 272 : (N == 128 ? 152 : 72));  // padded row stride
  static constexpr int RB = T / R2;        // K1: rows per CTA
  static constexpr int CB = N == 512 ? 8 : 16;  // K2: kx values (plus partners) per CTA
  static constexpr int NB2 = N / (2 * CB);
  static constexpr int T2 = 2 * CB * R2;   // K2: threads (one pass-A task each)
  // K1 staging row stride (elements): the pad puts the rows that one warp's
  // pass-A loads touch on different shared-memory banks
  template <typename TIn>
  static constexpr int stage_stride() {
    return N + ((sizeof(TIn) == 4 && R2 == 8) ? 8 : 16);
  }
  static constexpr int PB = (T / R2) < (N / 2) ? (T / R2) : (N / 2);  // K3: row pairs per CTA
  static constexpr int NB3 = (N / 2) / PB;
  static_assert(R1 * R2 == N, "radix");
  static_assert(RS >= N + N / R2, "padding");
  static __device__ __forceinline__ int phys(int p) { return p + p / R2; }
  static __device__ __forceinline__ int rho(int k) { return k / R1 + R2 * (k % R1); }
  // K2 column ownership (same scheme as the fused kernel with C = NB2, Q = CB)
  static __device__ __forceinline__ int kx_of(int b, int lc) {
    if (lc < CB) return CB * b + lc;
    if (b == 0 && lc == CB) return N / 2;
    return N - (CB * b + lc - CB);
  }
};


__device__ __forceinline__ int stat_status(const float4& s) { return __float_as_int(s.z); }

// One window's view of a workspace: batch index (origins, level, result) and
// its own statistics word, row spectra Zr, inverse-column output H and K3
// block partials.  The five-kernel schedule takes window s of a slice; the
// persistent schedule takes a ring slot.  Workspace words are read through
// L2 (ld.global.cg): in the persistent schedule another SM may have written
// them since this SM's L1 last saw those lines.
struct WinRef {
  long long b = 0;                     // window index in the batch
  float4* stats = nullptr;             // [1]
  float2* zr = nullptr;                // [n][n]
  float2* h = nullptr;                 // [n][n/2]
  unsigned long long* part = nullptr;  // [NB3][3]
  const int* pre = nullptr;            // status decided before the statistics, or null
  unsigned int* done = nullptr;        // finished inverse-row blocks of the window (finalize in K3), or null
  float* rstat = nullptr;              // [n / RB][8] row-block statistics records: the sums of A m and
                                       // A r as float pairs (hi, lo), the flags (as int bits), unused
};

template <int N>
__device__ __forceinline__ WinRef slice_ref(const MatchLaunch& L, const StreamWork& W, long long s) {
  WinRef R;
  R.b = W.b0 + s;
  R.stats = W.stats + s;
  R.zr = W.zr + s * N * N;
  R.h = W.h + s * N * (N / 2);
  R.part = W.part + 3 * s * StreamGeom<N>::NB3;
  R.pre = L.pre_status != nullptr ? L.pre_status + s : nullptr;
  R.done = W.done != nullptr ? W.done + s : nullptr;
  R.rstat = W.rstat != nullptr ? W.rstat + s * (N / StreamGeom<N>::RB) * 8 : nullptr;
  return R;
}

__device__ __forceinline__ float4 load_stats(const WinRef& R) { return __ldcg(R.stats); }

// ---------------------------------------------------------------------------
// K0: statistics
// ---------------------------------------------------------------------------
template <int N, typename TIn>
__device__ __forceinline__ void stats_stage(const MatchLaunch& L, const WinRef& R) {
  const long long b = R.b;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ float tap[N];
  __shared__ double red[8][2];
  __shared__ float mred[8][4];
  __shared__ int bred[8];
  auto put = [&](int status, float mm, float mr) {
    if (tid == 0) *R.stats = make_float4(mm, mr, __int_as_float(status), 0.f);
  };
  if (R.pre != nullptr && *R.pre != SWIFT_WIN_OK) {
    put(*R.pre, 0.f, 0.f);
    return;
  }
  const int guard = launch_window_check(L, b, N);
  if (guard != SWIFT_WIN_OK) {
    // test hook: report a window of another level as OK without reading it, as
    // a raced or stale workspace could; the row kernels' own guard must skip it
    put(L.stale_ok && guard == kWindowOtherLevel ? SWIFT_WIN_OK : guard, 0.f, 0.f);
    return;
  }
  const TIn* mbase;
  const TIn* rbase;
  long long mpitch, rpitch;
  if (L.patch_mode) {
    mbase = static_cast<const TIn*>(L.mov) + b * L.mov_stride;
    rbase = static_cast<const TIn*>(L.ref) + b * L.ref_stride;
    mpitch = rpitch = N;
  } else {
    const int my = __ldg(L.mov_origin + 2 * b), mx = __ldg(L.mov_origin + 2 * b + 1);
    const int ry = __ldg(L.ref_origin + 2 * b), rx = __ldg(L.ref_origin + 2 * b + 1);
    mbase = static_cast<const TIn*>(L.mov) + static_cast<long long>(my) * L.mov_pitch + mx;
    rbase = static_cast<const TIn*>(L.ref) + static_cast<long long>(ry) * L.ref_pitch + rx;
    mpitch = L.mov_pitch;
    rpitch = L.ref_pitch;
  }
  for (int i = tid; i < N; i += 256) tap[i] = L.taper[i];
  __syncthreads();
  const float inv_k = 1.0f / static_cast<float>(L.ref_count);
  float sm = 0.f, sr = 0.f, mn_m = 3.4e38f, mx_m = -3.4e38f, mn_r = 3.4e38f, mx_r = -3.4e38f;
  int bad = 0;
  auto accum = [&](float a, float mv, float rv) {
    sm = fmaf(a, mv, sm);
    sr = fmaf(a, rv, sr);
    mn_m = fminf(mn_m, mv);
    mx_m = fmaxf(mx_m, mv);
    mn_r = fminf(mn_r, rv);
    mx_r = fmaxf(mx_r, rv);
    if constexpr (sizeof(TIn) == 4) bad |= !(fabsf(mv) <= 3.4e38f) | !(fabsf(rv) <= 3.4e38f);
  };
  // 16-byte vector loads when both windows' rows are 16-byte aligned
  constexpr int VEC = 16 / static_cast<int>(sizeof(TIn));
  const bool vec = L.ref_count == 1 && ((reinterpret_cast<uintptr_t>(mbase) | reinterpret_cast<uintptr_t>(rbase) |
                                         static_cast<uintptr_t>(mpitch * sizeof(TIn)) |
                                         static_cast<uintptr_t>(rpitch * sizeof(TIn))) & 15) == 0;
  if (vec) {
    // batches of BATCH vectors per thread and image, all loads issued before use
    constexpr int PER = N * N / VEC / 256;
    constexpr int BATCH = PER < 8 ? PER : 8;
    static_assert(PER % BATCH == 0, "vector batches");
    // a thread's vectors all start at the same column x0 (256 is a multiple
    // of the N / VEC vectors of a row): its VEC column tapers stay in registers
    static_assert(256 % (N / VEC) == 0, "fixed column per thread");
    const int x0 = (tid % (N / VEC)) * VEC;
    float tx[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) tx[k] = tap[x0 + k];
    // uint8: a window is flat when every pixel equals every other, so each
    // thread ORs together the XOR of its packed words with its first pixel
    // replicated (one logic instruction a word) instead of per-pixel minima
    // and maxima; each vector's tapered sum is a dot product with the column
    // tapers, scaled by the row taper once: sum_x a_y a_x m = a_y (sum_x a_x m)
    uint32_t rep_m = 0u, rep_r = 0u, diff_m = 0u, diff_r = 0u;
    if constexpr (sizeof(TIn) == 1) {
      const int y0 = tid / (N / VEC);
      rep_m = 0x01010101u * __ldg(reinterpret_cast<const unsigned char*>(mbase + y0 * mpitch + x0));
      rep_r = 0x01010101u * __ldg(reinterpret_cast<const unsigned char*>(rbase + y0 * rpitch + x0));
    }
#pragma unroll 1
    for (int i0 = 0; i0 < PER; i0 += BATCH) {
      uint4 mqs[BATCH], rqs[BATCH];
#pragma unroll
      for (int bq = 0; bq < BATCH; ++bq) {
        const int y = (tid + (i0 + bq) * 256) / (N / VEC);
        mqs[bq] = __ldg(reinterpret_cast<const uint4*>(mbase + y * mpitch + x0));
        rqs[bq] = __ldg(reinterpret_cast<const uint4*>(rbase + y * rpitch + x0));
      }
#pragma unroll
      for (int bq = 0; bq < BATCH; ++bq) {
        const int y = (tid + (i0 + bq) * 256) / (N / VEC);
        const uint4 mq = mqs[bq], rq = rqs[bq];
        const float ay = tap[y];
        if constexpr (sizeof(TIn) == 1) {
          const uint32_t mw[4] = {mq.x, mq.y, mq.z, mq.w}, rw[4] = {rq.x, rq.y, rq.z, rq.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            diff_m |= mw[q] ^ rep_m;
            diff_r |= rw[q] ^ rep_r;
          }
          float dm = 0.f, dr = 0.f;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            dm = fmaf(tx[k], static_cast<float>((mw[k >> 2] >> (8 * (k & 3))) & 0xffu), dm);
            dr = fmaf(tx[k], static_cast<float>((rw[k >> 2] >> (8 * (k & 3))) & 0xffu), dr);
          }
          sm = fmaf(ay, dm, sm);
          sr = fmaf(ay, dr, sr);
        } else {
          const float mf[4] = {__uint_as_float(mq.x), __uint_as_float(mq.y), __uint_as_float(mq.z),
                               __uint_as_float(mq.w)};
          const float rf[4] = {__uint_as_float(rq.x), __uint_as_float(rq.y), __uint_as_float(rq.z),
                               __uint_as_float(rq.w)};
#pragma unroll
          for (int k = 0; k < 4; ++k) accum(ay * tx[k], mf[k], rf[k]);
        }
      }
    }
    if constexpr (sizeof(TIn) == 1) {
      // as extremes for the block reduction: the thread's first pixel, and a
      // maximum no byte takes when its pixels differ (flat: global min = max)
      const float f_m = static_cast<float>(rep_m & 0xffu), f_r = static_cast<float>(rep_r & 0xffu);
      mn_m = f_m, mx_m = diff_m ? 256.f : f_m;
      mn_r = f_r, mx_r = diff_r ? 256.f : f_r;
    }
  } else {
    for (int e = tid; e < N * N; e += 256) {  // consecutive threads, consecutive x
      const int y = e / N, x = e % N;
      const TIn* rrow = rbase + y * rpitch;
      const float mv = load_px<TIn>(mbase + y * mpitch + x);
      float rv = load_px<TIn>(rrow + x);
      for (int k = 1; k < L.ref_count; ++k) rv += load_px<TIn>(rrow + k * L.ref_stride + x);
      if (L.ref_count > 1) rv *= inv_k;
      accum(tap[y] * tap[x], mv, rv);
    }
  }
  const double dm = warp_sum_ff(sm), dr = warp_sum_ff(sr);
  float a0 = warp_min_f32(mn_m), a1 = warp_max_f32(mx_m), a2 = warp_min_f32(mn_r), a3 = warp_max_f32(mx_r);
  int bb = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    red[warp][0] = dm;
    red[warp][1] = dr;
    mred[warp][0] = a0;
    mred[warp][1] = a1;
    mred[warp][2] = a2;
    mred[warp][3] = a3;
    bred[warp] = bb;
  }
  __syncthreads();
  if (tid == 0) {
    double tm = 0, tr = 0;
    float e = 3.4e38f, f = -3.4e38f, g = 3.4e38f, h = -3.4e38f;
    int nb = 0;
    for (int v = 0; v < 8; ++v) {
      tm += red[v][0];
      tr += red[v][1];
      e = fminf(e, mred[v][0]);
      f = fmaxf(f, mred[v][1]);
      g = fminf(g, mred[v][2]);
      h = fmaxf(h, mred[v][3]);
      nb |= bred[v];
    }
    const int st = nb ? SWIFT_WIN_NONFINITE : ((e == f || g == h) ? SWIFT_WIN_FLAT : SWIFT_WIN_OK);
    *R.stats = make_float4(static_cast<float>(tm * L.inv_sum_a), static_cast<float>(tr * L.inv_sum_a),
                           __int_as_float(st), 0.f);
  }
}

template <int N, typename TIn>
__global__ void __launch_bounds__(256) stream_stats_kernel(const MatchLaunch L, const StreamWork W) {
  stats_stage<N, TIn>(L, slice_ref<N>(L, W, blockIdx.x));
}

// ---------------------------------------------------------------------------
// K1: row transforms of z = m' + i r'
// ---------------------------------------------------------------------------
// 16 x 16 byte transpose within each half-warp.  On entry lane L (its lane
// index mod 16) holds bytes t = 0..15 of chunk L (byte t in w[t / 4] at bit
// 8 (t % 4)); on exit it holds byte L of every chunk, chunk m as byte m.
// Each of the four stages swaps one bit of the lane index with the same bit
// of the byte index: lanes L and L ^ d trade the half of their bytes whose
// bit differs from their own lane bit (two words per shuffle).
__device__ __forceinline__ void transpose16_u8(uint32_t (&w)[4], int L) {
  {  // lane bit 3 <-> byte bit 3 (word pairs {0,1} / {2,3})
    const bool hi = (L & 8) != 0;
    uint32_t a = hi ? w[0] : w[2], b = hi ? w[1] : w[3];
    a = __shfl_xor_sync(0xffffffffu, a, 8);
    b = __shfl_xor_sync(0xffffffffu, b, 8);
    if (hi) {
      w[0] = a;
      w[1] = b;
    } else {
      w[2] = a;
      w[3] = b;
    }
  }
  {  // lane bit 2 <-> byte bit 2 (words {0,2} / {1,3})
    const bool hi = (L & 4) != 0;
    uint32_t a = hi ? w[0] : w[1], b = hi ? w[2] : w[3];
    a = __shfl_xor_sync(0xffffffffu, a, 4);
    b = __shfl_xor_sync(0xffffffffu, b, 4);
    if (hi) {
      w[0] = a;
      w[2] = b;
    } else {
      w[1] = a;
      w[3] = b;
    }
  }
  {  // lane bit 1 <-> byte bit 1 (16-bit halves of each word)
    const bool hi = (L & 2) != 0;
    const uint32_t give = hi ? 0x5410u : 0x7632u;
    uint32_t a = __byte_perm(w[0], w[1], give), b = __byte_perm(w[2], w[3], give);
    a = __shfl_xor_sync(0xffffffffu, a, 2);
    b = __shfl_xor_sync(0xffffffffu, b, 2);
    const uint32_t s0 = hi ? 0x3254u : 0x5410u, s1 = hi ? 0x3276u : 0x7610u;
    w[0] = __byte_perm(w[0], a, s0);
    w[1] = __byte_perm(w[1], a, s1);
    w[2] = __byte_perm(w[2], b, s0);
    w[3] = __byte_perm(w[3], b, s1);
  }
  {  // lane bit 0 <-> byte bit 0 (odd / even bytes of each word)
    const bool hi = (L & 1) != 0;
    const uint32_t give = hi ? 0x6420u : 0x7531u;
    uint32_t a = __byte_perm(w[0], w[1], give), b = __byte_perm(w[2], w[3], give);
    a = __shfl_xor_sync(0xffffffffu, a, 1);
    b = __shfl_xor_sync(0xffffffffu, b, 1);
    const uint32_t s0 = hi ? 0x3514u : 0x5240u, s1 = hi ? 0x3716u : 0x7260u;
    w[0] = __byte_perm(w[0], a, s0);
    w[1] = __byte_perm(w[1], a, s1);
    w[2] = __byte_perm(w[2], b, s0);
    w[3] = __byte_perm(w[3], b, s1);
  }
}

// Bytes 16 c + o .. 16 c + o + 15 (0 <= o < 16) of a shared-memory row that
// starts on a 16-byte boundary, as four little-endian words: two 16-byte
// loads (one when o = 0, which the window makes uniform over the CTA) and a
// funnel shift by o bytes.  The row holds at least 16 (c + 2) bytes.
__device__ __forceinline__ void tile_bytes16(const unsigned char* row, int c, int o, uint32_t (&w)[4]) {
  const uint4* p = reinterpret_cast<const uint4*>(row) + c;
  const uint4 a = p[0];
  if (o == 0) {
    w[0] = a.x, w[1] = a.y, w[2] = a.z, w[3] = a.w;
    return;
  }
  const uint4 n = p[1];
  const uint32_t u[8] = {a.x, a.y, a.z, a.w, n.x, n.y, n.z, n.w};
  const int k = o >> 2;
  const uint32_t sh = 8u * static_cast<uint32_t>(o & 3);
  uint32_t d[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) d[i] = k == 0 ? u[i] : (k == 1 ? u[i + 1] : (k == 2 ? u[i + 2] : u[i + 3]));
#pragma unroll
  for (int q = 0; q < 4; ++q) w[q] = __funnelshift_r(d[q], d[q + 1], sh);
}

// per-warp partials of a row block's statistics (STATS mode), in shared memory
struct RowBlockSums {
  float s[8][2];
  int f[8];
};
__device__ __forceinline__ RowBlockSums& row_block_sums() {
  __shared__ RowBlockSums rbs;
  return rbs;
}

// STATS (plain forward, n <= 256): no statistics kernel ran.  The block
// checks the window's level and bounds itself (block 0 writes the status word;
// the column-pair kernel sets the final one), transforms the rows of the
// tapered windows A m and A r without their means, and records in R.rstat[rb]
// its sums of A m and A r (float pairs over the block's warps), and flags: bit 0 / 1
// a pixel of the moving / reference rows differs from that window's first
// pixel (so a window is flat when no block sets the bit), bit 2 a non-finite
// float pixel.  The column-pair kernel removes the means in the spectrum.
template <int N, typename TIn, bool STATS = false>
__device__ __forceinline__ void rows_stage(const MatchLaunch& L, const WinRef& R, int rb, const RowMaps* M = nullptr) {
  using G = StreamGeom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, RB = G::RB, RS = G::RS, T = G::T;
  constexpr int KB = (RB * R1 + T - 1) / T;
  constexpr int MS = G::template stage_stride<TIn>();
  constexpr int TS = R1 + 4;  // row stride of the transposed column taper (16-byte rows, no bank conflicts)
  // uint8 windows of 256 x 256: pass A takes its pixels from the thread's own
  // 16-byte loads through a half-warp byte transpose instead of a staged copy
  constexpr bool kShfl = N == 256 && sizeof(TIn) == 1;
  const long long b = R.b;
  const int tid = threadIdx.x;
  float4 st = make_float4(0.f, 0.f, 0.f, 0.f);  // the means (none in STATS mode)
  if constexpr (STATS) {
    const int guard = launch_window_check(L, b, N);
    if (rb == 0 && tid == 0) *R.stats = make_float4(0.f, 0.f, __int_as_float(guard), 0.f);
    if (guard != SWIFT_WIN_OK) return;
  } else {
    st = load_stats(R);
    if (stat_status(st) != SWIFT_WIN_OK) return;
    // the window's level and bounds, from the launch's own arrays: a status
    // word left by another call never makes this kernel read
    const int guard = launch_window_check(L, b, N);
    if (guard != SWIFT_WIN_OK) {
      if (tid == 0) *R.stats = make_float4(0.f, 0.f, __int_as_float(guard), 0.f);
      return;
    }
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* slab = reinterpret_cast<float2*>(smem_raw);  // [RB][RS]
  float2* twid = slab + RB * RS;
  float* tap = reinterpret_cast<float*>(twid + N);
  float* tapT = tap + N;  // [R2][TS]: tapT[j][m] = tap[j + R2 m]
  // raw rows: uint8/float32 moving and reference; the reference of a K-section
  // model (or unaligned rows) is staged as float in rfstage, which aliases the slab
  TIn* mstage = reinterpret_cast<TIn*>(tapT + R2 * TS);  // [RB][MS]
  TIn* rstage = mstage + RB * MS;
  float* rfstage = reinterpret_cast<float*>(slab);
  // the plan's tables are requested first (into registers, stored below)
  constexpr int NT = (N + T - 1) / T;
  float2 twr[NT];
  float tpr[NT];
#pragma unroll
  for (int q = 0; q < NT; ++q) {
    const int i = tid + q * T;
    if (N % T == 0 || i < N) {
      twr[q] = L.twiddle[i];
      tpr[q] = L.taper[i];
    }
  }
  const TIn* mbase;
  const TIn* rbase;
  long long mpitch, rpitch;
  int my = 0, mx = 0, ry = 0, rx = 0;
  if (L.patch_mode) {
    mbase = static_cast<const TIn*>(L.mov) + b * L.mov_stride;
    rbase = static_cast<const TIn*>(L.ref) + b * L.ref_stride;
    mpitch = rpitch = N;
  } else {
    my = __ldg(L.mov_origin + 2 * b);
    mx = __ldg(L.mov_origin + 2 * b + 1);
    ry = __ldg(L.ref_origin + 2 * b);
    rx = __ldg(L.ref_origin + 2 * b + 1);
    mbase = static_cast<const TIn*>(L.mov) + static_cast<long long>(my) * L.mov_pitch + mx;
    rbase = static_cast<const TIn*>(L.ref) + static_cast<long long>(ry) * L.ref_pitch + rx;
    mpitch = L.mov_pitch;
    rpitch = L.ref_pitch;
  }
  // uint8 section rows through the tensor maps (RowMaps): the tiles start at
  // the staging area's first 128-byte boundary (rows_smem leaves the slack);
  // one thread issues both box copies before the tables are stored, so the
  // copies run under the table stores
  __shared__ __align__(8) unsigned long long stage_bar;
  const uint32_t mbar = smem_addr(&stage_bar);
  bool tma = false;
  TIn* mtile = mstage;
  if constexpr (sizeof(TIn) == 1) {
    tma = M != nullptr && M->on && (M->all || ((mx | rx) & 15) != 0);
    const uint32_t a = smem_addr(mstage);
    mtile = mstage + (((a + 127u) & ~127u) - a);
  }
  TIn* rtile = mtile + RB * MS;
  if constexpr (sizeof(TIn) == 1) {
    static_assert(MS == N + 16, "tile rows of n / 16 + 1 chunks of 16 bytes");
    if (tma && tid == 0) {
      mbar_init(mbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(mbar, 2 * RB * MS + L.stall_tx);
      tma_load_3d(smem_addr(mtile), &M->mov, 0, mx >> 4, my + rb * RB, mbar);
      tma_load_3d(smem_addr(rtile), &M->ref, 0, rx >> 4, ry + rb * RB, mbar);
    }
  }
#pragma unroll
  for (int q = 0; q < NT; ++q) {
    const int i = tid + q * T;
    if (N % T == 0 || i < N) {
      twid[i] = twr[q];
      tap[i] = tpr[q];
      tapT[(i % R2) * TS + i / R2] = tpr[q];
    }
  }
  // a staging copy that did not arrive (bounded wait): the window is marked
  // SWIFT_WIN_TIMEOUT after one more wait for the copies in flight
  auto staging_timeout = [&]() {
    if (tid == 0) {
      mbar_wait_bounded(mbar, 0);
      *R.stats = make_float4(0.f, 0.f, __int_as_float(SWIFT_WIN_TIMEOUT), 0.f);
      if constexpr (STATS) {
        // block 0 may write OK after this: the record carries the timeout
        float* rec = R.rstat + 8 * rb;
        rec[0] = rec[1] = rec[2] = rec[3] = 0.f;
        rec[4] = __int_as_float(kRowTimeout);
      }
    }
  };
  // STATS: the windows' first pixels (the reference's as the staged rows
  // average a K-section model), which the block's pixels are compared with
  float p0m = 0.f, p0r = 0.f;
  if constexpr (STATS) {
    p0m = load_px<TIn>(mbase);
    float r0 = load_px<TIn>(rbase);
    if (L.ref_count > 1) {
      for (int k = 1; k < L.ref_count; ++k) r0 += load_px<TIn>(rbase + k * L.ref_stride);
      r0 *= 1.0f / static_cast<float>(L.ref_count);
    }
    p0r = r0;
  }
  mbase += static_cast<long long>(rb * RB) * mpitch;
  rbase += static_cast<long long>(rb * RB) * rpitch;
  // stage the block's RB rows of both windows when they are 16-byte aligned:
  // uint8 rows (256 B at n = 256) by 16-byte vector loads; float rows (1 KB)
  // by bulk asynchronous copies (cp.async.bulk issued by one thread,
  // completion counted on an mbarrier), which measured faster for them and
  // slower for the short uint8 rows.  The copy wait is bounded (about 2 s): a
  // block whose copies did not arrive marks its window SWIFT_WIN_TIMEOUT,
  // waits once more for the copies in flight and leaves.
  const bool vec = L.ref_count == 1 && ((reinterpret_cast<uintptr_t>(mbase) | reinterpret_cast<uintptr_t>(rbase) |
                                         static_cast<uintptr_t>(mpitch * sizeof(TIn)) |
                                         static_cast<uintptr_t>(rpitch * sizeof(TIn))) & 15) == 0;
  uint32_t wm[4] = {0u, 0u, 0u, 0u}, wr[4] = {0u, 0u, 0u, 0u};  // kShfl: bytes 16 L .. 16 L + 15 of a row
  if (tma) {
    __syncthreads();  // the barrier is initialised before anyone waits on it
    const bool arrived = mbar_wait_bounded(mbar, 0);
    if (__syncthreads_or(!arrived)) {
      staging_timeout();
      return;
    }
    if constexpr (kShfl) {
      const int r = tid / 16, c = tid % 16;
      tile_bytes16(mtile + r * MS, c, mx & 15, wm);
      tile_bytes16(rtile + r * MS, c, rx & 15, wr);
    }
  } else if (vec) {
    if constexpr (kShfl) {
      static_assert(RB * N / 16 == T && R2 == 16, "one 16-byte vector per thread and window");
      const int r = tid / 16, x0 = (tid % 16) * 16;
      const uint4 a = __ldg(reinterpret_cast<const uint4*>(mbase + r * mpitch + x0));
      const uint4 c = __ldg(reinterpret_cast<const uint4*>(rbase + r * rpitch + x0));
      wm[0] = a.x, wm[1] = a.y, wm[2] = a.z, wm[3] = a.w;
      wr[0] = c.x, wr[1] = c.y, wr[2] = c.z, wr[3] = c.w;
    } else if constexpr (sizeof(TIn) == 4) {
      constexpr uint32_t kRowBytes = N * sizeof(TIn);
      static_assert(kRowBytes % 16 == 0 && (MS * sizeof(TIn)) % 16 == 0, "bulk copy granularity");
      if (tid == 0) {
        mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(mbar, 2 * RB * kRowBytes + L.stall_tx);
        for (int r = 0; r < RB; ++r) {
          bulk_g2s(smem_addr(mstage + r * MS), mbase + r * mpitch, kRowBytes, mbar);
          bulk_g2s(smem_addr(rstage + r * MS), rbase + r * rpitch, kRowBytes, mbar);
        }
      }
      __syncthreads();  // the barrier is initialised before anyone waits on it
      const bool arrived = mbar_wait_bounded(mbar, 0);
      if (__syncthreads_or(!arrived)) {
        staging_timeout();
        return;
      }
    } else {
      constexpr int VEC = 16 / static_cast<int>(sizeof(TIn));
      constexpr int NV = RB * N / VEC;  // vectors per image
      uint4 q[2 * ((NV + T - 1) / T)];
#pragma unroll
      for (int i = 0; i < (NV + T - 1) / T; ++i) {
        const int e = tid + i * T;
        if (NV % T == 0 || e < NV) {
          const int r = e / (N / VEC), x0 = (e % (N / VEC)) * VEC;
          q[2 * i] = __ldg(reinterpret_cast<const uint4*>(mbase + r * mpitch + x0));
          q[2 * i + 1] = __ldg(reinterpret_cast<const uint4*>(rbase + r * rpitch + x0));
        }
      }
#pragma unroll
      for (int i = 0; i < (NV + T - 1) / T; ++i) {
        const int e = tid + i * T;
        if (NV % T == 0 || e < NV) {
          const int o = (e / (N / VEC)) * MS + (e % (N / VEC)) * VEC;
          *reinterpret_cast<uint4*>(mstage + o) = q[2 * i];
          *reinterpret_cast<uint4*>(rstage + o) = q[2 * i + 1];
        }
      }
    }
  } else {
    const float inv_k = 1.0f / static_cast<float>(L.ref_count);
    for (int e = tid; e < RB * N; e += T) {
      const int r = e / N, x = e % N;
      mstage[r * MS + x] = __ldg(mbase + r * mpitch + x);
      float rv = load_px<TIn>(rbase + r * rpitch + x);
      if (L.ref_count > 1) {
        for (int k = 1; k < L.ref_count; ++k) rv += load_px<TIn>(rbase + k * L.ref_stride + r * rpitch + x);
        rv *= inv_k;
      }
      rfstage[r * MS + x] = rv;
    }
  }
  if (!tma) __syncthreads();  // (the tensor-map tiles: each thread saw the copies arrive)
  // the rows as uint8 / float32 values: in registers (kShfl), else staged
  const bool regs = vec || tma;
  const TIn* ms = mstage;
  const TIn* rs = rstage;
  if constexpr (sizeof(TIn) == 1) {
    if (tma) {
      ms = mtile + (mx & 15);
      rs = rtile + (rx & 15);
    }
  }
  // pass A: thread (line, j) takes x = j + R2 m of row rb*RB + line
  const int line = tid / R2, j = tid % R2;
  const int y = rb * RB + line;
  float mv[R1], rv[R1];
  int rflags = 0;  // STATS: this thread's record flags
  if constexpr (STATS && kShfl) {
    if (regs) {
      // the thread's 16 bytes of each row against the first pixel replicated
      const uint32_t rm = 0x01010101u * static_cast<uint32_t>(p0m), rr = 0x01010101u * static_cast<uint32_t>(p0r);
      uint32_t dm = 0u, dr = 0u;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        dm |= wm[q] ^ rm;
        dr |= wr[q] ^ rr;
      }
      rflags = (dm ? kRowDiffM : 0) | (dr ? kRowDiffR : 0);
    }
  }
  if (kShfl && regs) {
    // lane j of the half-warp of row `line` receives x = j + 16 m, m = 0..15
    transpose16_u8(wm, j);
    transpose16_u8(wr, j);
#pragma unroll
    for (int m = 0; m < R1; ++m) {
      mv[m] = static_cast<float>((wm[m >> 2] >> (8 * (m & 3))) & 0xffu);
      rv[m] = static_cast<float>((wr[m >> 2] >> (8 * (m & 3))) & 0xffu);
    }
  } else {
#pragma unroll
    for (int m = 0; m < R1; ++m) {
      const int e = line * MS + j + R2 * m;
      mv[m] = static_cast<float>(ms[e]);
      rv[m] = regs ? static_cast<float>(rs[e]) : rfstage[e];
    }
  }
  if constexpr (STATS) {
    if (!(kShfl && regs)) {
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        rflags |= (mv[m] != p0m ? kRowDiffM : 0) | (rv[m] != p0r ? kRowDiffR : 0);
        if constexpr (sizeof(TIn) == 4) {
          rflags |= (!(fabsf(mv[m]) <= 3.4e38f) || !(fabsf(rv[m]) <= 3.4e38f)) ? kRowNonFinite : 0;
        }
      }
    }
  }
  if (!regs) __syncthreads();  // rfstage aliases the slab written below
  {
    const float ay = tap[y];
    float tx[R1];
#pragma unroll
    for (int q = 0; q < R1 / 4; ++q) {
      const float4 t4 = reinterpret_cast<const float4*>(tapT + j * TS)[q];
      tx[4 * q] = t4.x, tx[4 * q + 1] = t4.y, tx[4 * q + 2] = t4.z, tx[4 * q + 3] = t4.w;
    }
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) {
      const float a = ay * tx[m];
      if constexpr (STATS) {
        v[m] = make_float2(a * mv[m], a * rv[m]);
      } else {
        v[m] = make_float2(a * (mv[m] - st.x), a * (rv[m] - st.y));
      }
    }
    if constexpr (STATS) {
      // the block's sums of A m and A r: FP32 within a warp (positive terms
      // for uint8 windows), FP64 over the warps after the barrier below
      float sm = 0.f, sr = 0.f;
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        sm += v[m].x;
        sr += v[m].y;
      }
      sm = warp_sum_f32(sm);
      sr = warp_sum_f32(sr);
      const int f = static_cast<int>(__reduce_or_sync(0xffffffffu, static_cast<unsigned>(rflags)));
      if ((tid & 31) == 0) {
        RowBlockSums& S = row_block_sums();
        S.s[tid >> 5][0] = sm;
        S.s[tid >> 5][1] = sr;
        S.f[tid >> 5] = f;
      }
    }
    dft<R1, -1>(v);
    float2* row = slab + line * RS;
#pragma unroll
    for (int q = 0; q < R1; ++q) row[G::phys(j + R2 * q)] = v[q];
  }
  __syncthreads();
  if constexpr (STATS) {
    if (tid < 32) {
      // warp 0: the warps' partials summed as float pairs (no FP64 on this
      // GPU's slow unit), one 32-byte record
      const RowBlockSums& S = row_block_sums();
      const int lane = tid;
      float hm = lane < T / 32 ? S.s[lane][0] : 0.f, lm = 0.f;
      float hr = lane < T / 32 ? S.s[lane][1] : 0.f, lr = 0.f;
      warp_sum_ff2(hm, lm);
      warp_sum_ff2(hr, lr);
      const int fl = static_cast<int>(__reduce_or_sync(0xffffffffu, lane < T / 32 ? static_cast<unsigned>(S.f[lane]) : 0u));
      if (lane == 0) {
        float* rec = R.rstat + 8 * rb;
        *reinterpret_cast<float4*>(rec) = make_float4(hm, lm, hr, lr);
        rec[4] = __int_as_float(fl);
      }
    }
  }
  // pass B: thread (line, k1) -> X[k1 + R1 k2], written to Zr[y][kx]
#pragma unroll
  for (int i = 0; i < KB; ++i) {
    const int task = tid + i * T;
    if ((RB * R1) % T != 0 && task >= RB * R1) break;  // n = 512: 128 tasks for 256 threads
    const int ln = task / R1, k1 = task % R1;
    const float2* row = slab + ln * RS;
    float2 v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      const float2 x = row[G::phys(R2 * k1 + n2)];
      v[n2] = n2 == 0 ? x : cmul(x, twid[n2 * R1 + k1]);
    }
    dft<R2, -1>(v);
    float2* zrow = R.zr + (rb * RB + ln) * N;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) zrow[k1 + R1 * k2] = v[k2];
  }
}

template <int N, typename TIn, bool STATS = false>
__global__ void __launch_bounds__(256, N == 512 ? 1 : 4)
    stream_rows_kernel(const MatchLaunch L, const StreamWork W, const __grid_constant__ RowMaps M) {
  constexpr int NRB = N / StreamGeom<N>::RB;
  rows_stage<N, TIn, STATS>(L, slice_ref<N>(L, W, blockIdx.x / NRB), blockIdx.x % NRB, &M);
}

// ---------------------------------------------------------------------------
// K2: column transforms, unpack, whitening, inverse column transforms
// ---------------------------------------------------------------------------
// SAVE: also store C = M conj(R) and R for kx in [0, n/2] (all ky) to `cr`
// ([2][n][n/2+1]) for the backward pass.
template <int N, bool SAVE = false>
__global__ void __launch_bounds__(StreamGeom<N>::T2) stream_cols_kernel(const MatchLaunch L, const StreamWork W,
                                                                        float2* cr = nullptr) {
  using G = StreamGeom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, CB = G::CB, T = G::T2;
  constexpr int LINES = 2 * CB;
  constexpr int LS = LINES + 8;  // padded row stride of the column slab
  const long long s = blockIdx.x / G::NB2;
  const int cb = blockIdx.x % G::NB2;
  const int tid = threadIdx.x;
  if (stat_status(W.stats[s]) != SWIFT_WIN_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* slab = reinterpret_cast<float2*>(smem_raw);  // [ky][lc], row stride LS
  // twiddles transposed, [k1][n2] with rows of R2 + 2 (16-byte multiples, two
  // CTA-uniform rows per warp on different banks): a thread of passes B / B'
  // reads its R2 twiddles as R2 / 2 16-byte pairs
  constexpr int TW = R2 + 2;
  float2* twT = slab + N * LS;
  for (int i = tid; i < N; i += T) twT[(i % R1) * TW + i / R1] = L.twiddle[i];
  // column pass A (rows j + R2 m) straight from Zr: consecutive threads take
  // consecutive lines, i.e. contiguous kx runs of a row (coalesced)
  const float2* zr = W.zr + s * N * N;
  constexpr int TA = LINES * R2, TB = LINES * R1;
#pragma unroll
  for (int i = 0; i < (TA + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TA % T != 0 && task >= TA) break;
    const int j = task / LINES, lc = task % LINES;
    const int kx = G::kx_of(cb, lc);
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = __ldcs(zr + (j + R2 * m) * N + kx);
    dft<R1, -1>(v);
#pragma unroll
    for (int q = 0; q < R1; ++q) slab[(j + R2 * q) * LS + lc] = v[q];
  }
  __syncthreads();
  // column pass B (rows R2 k1 + n2), in place: rho order
#pragma unroll
  for (int i = 0; i < (TB + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TB % T != 0 && task >= TB) break;
    const int k1 = task / LINES, lc = task % LINES;
    float2 v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) v[n2] = slab[(R2 * k1 + n2) * LS + lc];
    const float4* tw4 = reinterpret_cast<const float4*>(twT + k1 * TW);
#pragma unroll
    for (int q = 0; q < R2 / 2; ++q) {
      const float4 t = tw4[q];
      if (q > 0) v[2 * q] = cmul(v[2 * q], make_float2(t.x, t.y));
      v[2 * q + 1] = cmul(v[2 * q + 1], make_float2(t.z, t.w));
    }
    dft<R2, -1>(v);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) slab[(R2 * k1 + k2) * LS + lc] = v[k2];
  }
  __syncthreads();
  // unpack + whiten on lines lc < CB (kx = CB*cb + lc), all threads: slab row
  // p = R2 k1 + k2 holds ky = k1 + R1 k2; the partner Z[-ky][-kx] sits in line
  // lc + CB (line 0 of block 0 is its own partner and carries kx = n/2 in
  // line CB).  G is written in place after every read is done.
  const float half_w = -0.5f * L.w;
  const float inv_n2 = 1.0f / (static_cast<float>(N) * static_cast<float>(N));
  constexpr int EW = N * CB / T;  // elements per thread
  static_assert(EW * T == N * CB, "whitening split");
  float2 gv[EW];
#pragma unroll
  for (int i = 0; i < EW; ++i) {
    const int e = tid + i * T;
    const int p = e / CB, lc = e % CB;
    const int ky = p / R2 + R1 * (p % R2);
    const int nky = (N - ky) & (N - 1);
    const bool dc_col = (cb == 0 && lc == 0);
    const int plc = dc_col ? 0 : lc + CB;
    const float2 a = slab[p * LS + lc];
    const float2 bb = slab[G::rho(nky) * LS + plc];
    const float2 c = make_float2(0.5f * fmaf(a.x, bb.y, a.y * bb.x),
                                 0.25f * ((a.x * a.x + a.y * a.y) - (bb.x * bb.x + bb.y * bb.y)));
    const float mag2 = fmaf(c.x, c.x, c.y * c.y);
    const float sc = whiten_factor(mag2, half_w) * inv_n2;
    float2 g = make_float2(c.x * sc, c.y * sc);
    if constexpr (SAVE) {
      // R = (A - conj(B)) / 2i
      const size_t o = (static_cast<size_t>(s) * 2 * N + ky) * (N / 2 + 1) + (CB * cb + lc);
      cr[o] = c;
      cr[o + static_cast<size_t>(N) * (N / 2 + 1)] = make_float2(0.5f * (a.y + bb.y), -0.5f * (a.x - bb.x));
    }
    if (dc_col) {
      const float2 a2 = slab[p * LS + CB];
      const float2 b2 = slab[G::rho(nky) * LS + CB];
      const float2 c2 = make_float2(0.5f * fmaf(a2.x, b2.y, a2.y * b2.x),
                                    0.25f * ((a2.x * a2.x + a2.y * a2.y) - (b2.x * b2.x + b2.y * b2.y)));
      if constexpr (SAVE) {
        const size_t o = (static_cast<size_t>(s) * 2 * N + ky) * (N / 2 + 1) + N / 2;
        cr[o] = c2;
        cr[o + static_cast<size_t>(N) * (N / 2 + 1)] = make_float2(0.5f * (a2.y + b2.y), -0.5f * (a2.x - b2.x));
      }
      const float mq = fmaf(c2.x, c2.x, c2.y * c2.y);
      const float sq = whiten_factor(mq, half_w) * inv_n2;
      if (ky == 0) g = make_float2(0.f, 0.f);  // G[0,0] = 0
      g = make_float2(g.x - c2.y * sq, g.y + c2.x * sq);
    }
    gv[i] = g;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < EW; ++i) {
    const int e = tid + i * T;
    slab[(e / CB) * LS + e % CB] = gv[i];
  }
  __syncthreads();
  // inverse pass B' on lines lc < CB, in place
  constexpr int TBh = CB * R1, TAh = CB * R2;
#pragma unroll
  for (int i = 0; i < (TBh + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TBh % T != 0 && task >= TBh) break;
    const int k1 = task / CB, lc = task % CB;
    float2 v[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k2] = slab[(R2 * k1 + k2) * LS + lc];
    dft<R2, +1>(v);
    const float4* tw4 = reinterpret_cast<const float4*>(twT + k1 * TW);
#pragma unroll
    for (int q = 0; q < R2 / 2; ++q) {
      const float4 t = tw4[q];
      if (q > 0) v[2 * q] = cmulc(v[2 * q], make_float2(t.x, t.y));
      v[2 * q + 1] = cmulc(v[2 * q + 1], make_float2(t.z, t.w));
    }
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) slab[(R2 * k1 + n2) * LS + lc] = v[n2];
  }
  __syncthreads();
  // inverse pass A' -> H[y = n2 + R2 n1][kx]
  float2* hw = W.h + s * N * (N / 2);
#pragma unroll
  for (int i = 0; i < (TAh + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TAh % T != 0 && task >= TAh) break;
    const int n2 = task / CB, lc = task % CB;
    float2 v[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = slab[(n2 + R2 * k1) * LS + lc];
    dft<R1, +1>(v);
    const int kx = CB * cb + lc;  // 0 for the packed (DC, Nyquist) column
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) hw[(n2 + R2 * n1) * (N / 2) + kx] = v[n1];
  }
}

// ---------------------------------------------------------------------------
// K2 (plain forward, n = 64, 128, 256): column pairs with the Hermitian unpack
// at load time
// ---------------------------------------------------------------------------
// A CTA owns CB values kx in [CB cb, CB cb + CB) of the half spectrum and reads
// the row spectra of kx and of its partner n - kx.  Per row y the two real
// windows' row spectra separate pointwise,
//     a = Z[y][kx] + conj(Z[y][n - kx]) = 2 M_row[y][kx]
//     b = Z[y][kx] - conj(Z[y][n - kx]) = 2i R_row[y][kx],
// so one thread transforms the columns of a and b together, and after the
// second radix pass holds M and R (times 2 and 2i) at the same bins
// ky = k1 + R1 k2.  The cross power C = M conj(R) = i a conj(b) / 4, the
// whitening and the first inverse pass then run in that thread's registers:
// no partner exchange, and two barriers per CTA.  The 1/4 and 1/n^2 factors
// ride in the whitening exponent: C |C|^-w / n^2 = C4 |C4|^-w 4^(w-1) / n^2
// with C4 = i a conj(b).
//
// kx = 0 and kx = n/2 (both their own partners, both real columns after the
// row transform) share the task lc = 0 of block 0: a = 2 (Re Z[y][0] + i Re
// Z[y][n/2]), b = 2i (Im Z[y][0] + i Im Z[y][n/2]).  After the column
// transform those tasks separate the two columns through the bins -ky (held by
// the task k1' = -k1 mod R1), exchanged in shared memory, and whiten both; the
// inverse input is G[.][0] + i G[.][n/2], whose inverse column transform is
// H[y][0] + i H[y][n/2] (both real), the packed layout the inverse-row kernel
// reads.
template <int N>
struct PairGeom {
  using G = StreamGeom<N>;
  static constexpr int R1 = G::R1, R2 = G::R2;
  static constexpr int CB = N == 256 ? 16 : 32;  // kx per CTA
  static constexpr int NB = (N / 2) / CB;        // CTAs per window
  static constexpr int T = 256;
  static constexpr int TA = CB * R2;  // pass A / A' tasks (line j or n2, column lc)
  static constexpr int TB = CB * R1;  // pass B / B' tasks (k1, lc)
  static constexpr int TW = R2 + 2;   // row stride of the transposed twiddle table (float2)
  static_assert(TA % T == 0 && TB % T == 0, "whole task rounds");
  static_assert(N / 2 % CB == 0, "column blocks");
};

__device__ __forceinline__ float whiten_scaled(float mag2, float half_w, float lscale) {
  // |C4|^-w times 2^lscale (lg2 / ex2 hardware approximations; the input of
  // lg2 is scaled by 2^64 below 2^-100, so neither instruction meets a
  // subnormal)
  if (!(mag2 > 0.f)) return 0.f;
  const bool tiny = mag2 < 0x1p-100f;
  float lg, f;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(tiny ? mag2 * 0x1p64f : mag2));
  if (tiny) lg -= 64.f;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"(fmaf(half_w, lg, lscale)));
  return f;
}

// CORRECT (after a STATS row kernel): the window's means and status come from
// the row blocks' records, and the means are removed in the spectrum: the
// transform of A (x - mu) is that of A x minus mu Ahat(ky) Ahat(kx), Ahat the
// (real) DFT of the symmetric 1D taper (L.ahat).  A flat, non-finite or timed
// out window gets its status word here and is left.
template <int N, bool CORRECT = false>
__device__ __forceinline__ void cpair_stage(const MatchLaunch& L, const WinRef& R, int cb) {
  using P = PairGeom<N>;
  constexpr int R1 = P::R1, R2 = P::R2, CB = P::CB, T = P::T, TW = P::TW;
  constexpr int RB = P::TB / T;  // pass B rounds per thread
  constexpr int NRB = N / StreamGeom<N>::RB;  // row blocks of a window
  const int tid = threadIdx.x;
  if (stat_status(load_stats(R)) != SWIFT_WIN_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* slab = reinterpret_cast<float4*>(smem_raw);  // [N][CB]: (a, b) after pass A
  float2* slab2 = reinterpret_cast<float2*>(smem_raw);  // [N][CB]: G after pass B' (reuses slab)
  float4* xbuf = slab + N * CB;                          // [R1][R2]: block 0, lc = 0
  float2* twT = reinterpret_cast<float2*>(xbuf + N);     // [R1][TW]: W_n^(k1 n2)
  float* ahat = reinterpret_cast<float*>(twT + R1 * TW);  // [N] (CORRECT)
  __shared__ float c_mu[2];
  __shared__ int c_status;
  for (int i = tid; i < N; i += T) twT[(i % R1) * TW + i / R1] = L.twiddle[i];
  // CORRECT: the row-block records are requested first (warp 0, one record a
  // lane) and combined during pass A, behind its column loads
  float4 rec_s = make_float4(0.f, 0.f, 0.f, 0.f);  // (hi, lo) of the sums of A m and A r
  unsigned rec_f = 0u;
  if constexpr (CORRECT) {
    static_assert(NRB <= 32, "one record per lane");
    if (tid < NRB) {
      const float* rec = R.rstat + 8 * tid;
      rec_s = __ldcg(reinterpret_cast<const float4*>(rec));
      rec_f = static_cast<unsigned>(__float_as_int(__ldcg(rec + 4)));
    }
    for (int i = tid; i < N; i += T) ahat[i] = L.ahat[i];
  }
  // pass A: task (j, lc) takes rows y = j + R2 m of columns kx and n - kx
  const float2* zr = R.zr;
#pragma unroll
  for (int r = 0; r < P::TA / T; ++r) {
    const int task = tid + r * T;
    const int j = task / CB, lc = task % CB;
    const int kx = CB * cb + lc;
    const bool packed = kx == 0;  // columns 0 and n/2
    const int kn = packed ? N / 2 : N - kx;
    float2 a[R1], b[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) {
      const float2 zk = __ldcg(zr + (j + R2 * m) * N + kx);
      const float2 zn = __ldcg(zr + (j + R2 * m) * N + kn);
      if (packed) {
        a[m] = make_float2(2.f * zk.x, 2.f * zn.x);
        b[m] = make_float2(-2.f * zn.y, 2.f * zk.y);
      } else {
        a[m] = make_float2(zk.x + zn.x, zk.y - zn.y);
        b[m] = make_float2(zk.x - zn.x, zk.y + zn.y);
      }
    }
    if constexpr (CORRECT) {
      if (r == 0 && tid < 32) {
        // warp 0, while its column loads are in flight: the window's
        // row-block records as float-pair sums (lanes without a record hold
        // zeros), flags ORed
        float hm = rec_s.x, lm = rec_s.y, hr = rec_s.z, lr = rec_s.w;
        warp_sum_ff2(hm, lm);
        warp_sum_ff2(hr, lr);
        const unsigned fl = __reduce_or_sync(0xffffffffu, rec_f);
        if (tid == 0) {
          c_status = (fl & kRowTimeout) ? SWIFT_WIN_TIMEOUT
                     : (fl & kRowNonFinite) ? SWIFT_WIN_NONFINITE
                     : ((fl & (kRowDiffM | kRowDiffR)) != (kRowDiffM | kRowDiffR)) ? SWIFT_WIN_FLAT
                                                                                    : SWIFT_WIN_OK;
          // mean = (hi + lo) / sum A, the pair rounded once
          const float inv = static_cast<float>(L.inv_sum_a);
          c_mu[0] = fmaf(hm, inv, lm * inv);
          c_mu[1] = fmaf(hr, inv, lr * inv);
        }
      }
    }
    dft<R1, -1>(a);
    dft<R1, -1>(b);
#pragma unroll
    for (int q = 0; q < R1; ++q) slab[(j + R2 * q) * CB + lc] = make_float4(a[q].x, a[q].y, b[q].x, b[q].y);
  }
  __syncthreads();
  if constexpr (CORRECT) {
    if (c_status != SWIFT_WIN_OK) {
      if (cb == 0 && tid == 0) *R.stats = make_float4(0.f, 0.f, __int_as_float(c_status), 0.f);
      return;
    }
  }
  const float half_w = -0.5f * L.w;
  // 2^lscale = 4^(w-1) / n^2
  const float lscale = 2.f * L.w - 2.f - 2.f * static_cast<float>(__ffs(N) - 1);
  // pass B (twiddles, DFT over n2), cross power, whitening and inverse pass B'
  // (DFT over k2, conjugate twiddles), all on the task's R2 bins; the results
  // stay in registers until every task has read the slab
  float2 g[RB][R2];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    const int task = tid + r * T;
    const int k1 = task / CB, lc = task % CB;
    const float4* tw4 = reinterpret_cast<const float4*>(twT + k1 * TW);
    float2 a[R2], b[R2];
#pragma unroll
    for (int q = 0; q < R2 / 2; ++q) {
      const float4 t = tw4[q];
      const float4 u = slab[(R2 * k1 + 2 * q) * CB + lc], v = slab[(R2 * k1 + 2 * q + 1) * CB + lc];
      a[2 * q] = make_float2(u.x, u.y);
      b[2 * q] = make_float2(u.z, u.w);
      if (q > 0) {
        a[2 * q] = cmul(a[2 * q], make_float2(t.x, t.y));
        b[2 * q] = cmul(b[2 * q], make_float2(t.x, t.y));
      }
      a[2 * q + 1] = cmul(make_float2(v.x, v.y), make_float2(t.z, t.w));
      b[2 * q + 1] = cmul(make_float2(v.z, v.w), make_float2(t.z, t.w));
    }
    dft<R2, -1>(a);
    dft<R2, -1>(b);
    if constexpr (CORRECT) {
      // a = 2 M, b = 2i R at ky = k1 + R1 k2: subtract 2 mu Ahat(ky) Ahat(kx)
      const int kx = CB * cb + lc;
      if (kx == 0) {
        // packed columns: a = 2 (M0 + i Mh), b = 2i R0 - 2 Rh (kx = 0 and n/2)
        const float am0 = 2.f * c_mu[0] * ahat[0], amh = 2.f * c_mu[0] * ahat[N / 2];
        const float ar0 = 2.f * c_mu[1] * ahat[0], arh = 2.f * c_mu[1] * ahat[N / 2];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const float ay = ahat[k1 + R1 * k2];
          a[k2].x = fmaf(-am0, ay, a[k2].x);
          a[k2].y = fmaf(-amh, ay, a[k2].y);
          b[k2].y = fmaf(-ar0, ay, b[k2].y);
          b[k2].x = fmaf(arh, ay, b[k2].x);
        }
      } else {
        const float ax = ahat[kx];
        if (ax != 0.f) {  // the Hann and untapered transforms vanish off a few bins
          const float am = 2.f * c_mu[0] * ax, ar = 2.f * c_mu[1] * ax;
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) {
            const float ay = ahat[k1 + R1 * k2];
            a[k2].x = fmaf(-am, ay, a[k2].x);
            b[k2].y = fmaf(-ar, ay, b[k2].y);
          }
        }
      }
    }
    if (cb == 0 && lc == 0) {
      // columns 0 and n/2: separated after the barrier below
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) xbuf[k1 * R2 + k2] = make_float4(a[k2].x, a[k2].y, b[k2].x, b[k2].y);
      continue;
    }
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      // C4 = i a conj(b)
      const float cr = fmaf(a[k2].x, b[k2].y, -a[k2].y * b[k2].x);
      const float ci = fmaf(a[k2].x, b[k2].x, a[k2].y * b[k2].y);
      const float f = whiten_scaled(fmaf(cr, cr, ci * ci), half_w, lscale);
      a[k2] = make_float2(cr * f, ci * f);
    }
    dft<R2, +1>(a);
#pragma unroll
    for (int q = 0; q < R2 / 2; ++q) {
      const float4 t = tw4[q];
      g[r][2 * q] = q == 0 ? a[0] : cmulc(a[2 * q], make_float2(t.x, t.y));
      g[r][2 * q + 1] = cmulc(a[2 * q + 1], make_float2(t.z, t.w));
    }
  }
  __syncthreads();  // the slab is read; G goes into the same space
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    const int task = tid + r * T;
    const int k1 = task / CB, lc = task % CB;
    if (cb == 0 && lc == 0) continue;
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) slab2[(R2 * k1 + n2) * CB + lc] = g[r][n2];
  }
  if (cb == 0 && tid < R1) {
    const int k1 = tid, k1p = (R1 - k1) % R1;
    float2 gp[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      // bin -ky of ky = k1 + R1 k2
      const int k2p = k1 == 0 ? (R2 - k2) % R2 : R2 - 1 - k2;
      const float4 u = xbuf[k1 * R2 + k2], v = xbuf[k1p * R2 + k2p];
      // a = 2 (M0 + i Mh), b = 2i (R0 + i Rh), with M0, Mh, R0, Rh the
      // column spectra of kx = 0 and n/2 (Hermitian in ky)
      const float2 m0 = make_float2(0.25f * (u.x + v.x), 0.25f * (u.y - v.y));
      const float2 mh = make_float2(0.25f * (u.y + v.y), -0.25f * (u.x - v.x));
      // q = b / 2i
      const float2 q = make_float2(0.5f * u.w, -0.5f * u.z), qp = make_float2(0.5f * v.w, -0.5f * v.z);
      const float2 r0 = make_float2(0.5f * (q.x + qp.x), 0.5f * (q.y - qp.y));
      const float2 rh = make_float2(0.5f * (q.y + qp.y), -0.5f * (q.x - qp.x));
      // C4 = 4 M conj(R) of each column
      const float2 c0 = cmulc(m0, r0), ch = cmulc(mh, rh);
      const float2 c40 = make_float2(4.f * c0.x, 4.f * c0.y), c4h = make_float2(4.f * ch.x, 4.f * ch.y);
      const float f0 = (k1 == 0 && k2 == 0) ? 0.f : whiten_scaled(fmaf(c40.x, c40.x, c40.y * c40.y), half_w, lscale);
      const float fh = whiten_scaled(fmaf(c4h.x, c4h.x, c4h.y * c4h.y), half_w, lscale);
      // G[.][0] + i G[.][n/2]
      gp[k2] = make_float2(c40.x * f0 - c4h.y * fh, c40.y * f0 + c4h.x * fh);
    }
    dft<R2, +1>(gp);
    const float4* tw4 = reinterpret_cast<const float4*>(twT + k1 * TW);
#pragma unroll
    for (int q = 0; q < R2 / 2; ++q) {
      const float4 t = tw4[q];
      if (q > 0) gp[2 * q] = cmulc(gp[2 * q], make_float2(t.x, t.y));
      gp[2 * q + 1] = cmulc(gp[2 * q + 1], make_float2(t.z, t.w));
    }
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) slab2[(R2 * k1 + n2) * CB] = gp[n2];
  }
  __syncthreads();
  // inverse pass A' -> H[y = n2 + R2 n1][kx]
  float2* hw = R.h;
#pragma unroll
  for (int r = 0; r < P::TA / T; ++r) {
    const int task = tid + r * T;
    const int n2 = task / CB, lc = task % CB;
    float2 v[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = slab2[(n2 + R2 * k1) * CB + lc];
    dft<R1, +1>(v);
    const int kx = CB * cb + lc;
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) hw[(n2 + R2 * n1) * (N / 2) + kx] = v[n1];
  }
}

template <int N, bool CORRECT = false>
__global__ void __launch_bounds__(256, 2) stream_cpair_kernel(const MatchLaunch L, const StreamWork W) {
  cpair_stage<N, CORRECT>(L, slice_ref<N>(L, W, blockIdx.x / PairGeom<N>::NB), blockIdx.x % PairGeom<N>::NB);
}

// ---------------------------------------------------------------------------
// K3: inverse row transforms of row pairs (y, y + N/2), block argmax
// ---------------------------------------------------------------------------
// The row-pair steps are shared with K4, which recomputes the few rows around
// the peak with the same instructions (so its values equal K3's bit for bit).
//
// irow_assemble: slab row p (< np) gets P = H[y1] + i H[y1 + n/2], the packed
// pair of half rows completed by Hermitian symmetry, y1 = y1_of(p) < n/2.
template <int N, int PB, int T, typename Y1>
__device__ __forceinline__ void irow_assemble(const float2* __restrict__ hw, float2* slab, int np, Y1 y1_of,
                                              int tid) {
  using G = StreamGeom<N>;
  constexpr int RS = G::RS;
  constexpr int K = PB * (N / 2) / T;
  static_assert(K * T == PB * (N / 2), "assembly split");
  float2 h1[K], h2[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int e = tid + i * T;
    const int p = e / (N / 2), kx = e % (N / 2);
    if (p < np) {
      const int y1 = y1_of(p), y2 = y1 + N / 2;
      h1[i] = __ldcg(hw + y1 * (N / 2) + kx);
      h2[i] = __ldcg(hw + y2 * (N / 2) + kx);
    }
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int e = tid + i * T;
    const int p = e / (N / 2), kx = e % (N / 2);
    if (p >= np) continue;
    float2* row = slab + p * RS;
    if (kx == 0) {
      row[G::phys(0)] = make_float2(h1[i].x, h2[i].x);
      row[G::phys(N / 2)] = make_float2(h1[i].y, h2[i].y);
    } else {
      row[G::phys(kx)] = make_float2(h1[i].x - h2[i].y, h1[i].y + h2[i].x);
      row[G::phys(N - kx)] = make_float2(h1[i].x + h2[i].y, h2[i].x - h1[i].y);
    }
  }
}

// irow_passA: first inverse radix pass (DFT over m of x = j + R2 m), in place
template <int N, int PB, int T>
__device__ __forceinline__ void irow_passA(float2* slab, int np, int tid) {
  using G = StreamGeom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, RS = G::RS;
  constexpr int TA = PB * R2;
#pragma unroll
  for (int i = 0; i < (TA + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TA % T != 0 && task >= TA) break;
    const int p = task / R2, j = task % R2;
    if (p >= np) continue;
    float2* row = slab + p * RS;
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = row[G::phys(j + R2 * m)];
    dft<R1, +1>(v);
#pragma unroll
    for (int q = 0; q < R1; ++q) row[G::phys(j + R2 * q)] = v[q];
  }
}

// irow_passB: second inverse radix pass of one packed row for residue k1:
// v[k2] = s[y1][x] + i s[y2][x] at x = k1 + R1 k2
template <int N>
__device__ __forceinline__ void irow_passB(const float2* row, const float2* twid, int k1,
                                           float2 (&v)[StreamGeom<N>::R2]) {
  using G = StreamGeom<N>;
  constexpr int R1 = G::R1, R2 = G::R2;
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    const float2 x = row[G::phys(R2 * k1 + n2)];
    v[n2] = n2 == 0 ? x : cmulc(x, twid[n2 * R1 + k1]);
  }
  dft<R2, +1>(v);
}

// WRITE_S: also store the match response s ([n][n] float32 in the Zr space),
// which the backward pass and the tensor-core schedule read; the plain forward
// keeps only the block argmax keys and sums.
template <int N>
__device__ __forceinline__ void disc_stage(const MatchLaunch& L, const WinRef& R);

// With R.done (n <= 256, exclusion radius below 8 px, plain forward), the
// block that finishes a window's inverse rows last also finalizes it (peak,
// SNR, subpixel: disc_stage), so the finalize costs no launch and its latency
// hides behind other windows' blocks; the block pb = 0 writes the record of a
// window whose status is not OK.
template <int N, bool WRITE_S>
__device__ __forceinline__ void irows_stage(const MatchLaunch& L, const WinRef& R, int pb) {
  using G = StreamGeom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, PB = G::PB, RS = G::RS, T = G::T;
  constexpr bool kFold = !WRITE_S && N <= 256;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    const int st = stat_status(load_stats(R));
    if (st != SWIFT_WIN_OK) {
      if (kFold && R.done != nullptr && pb == 0 && tid == 0 && st != kStatusSkip) {
        swift_result r = {0, 0, 0.f, 0.f, 0.f, 0.f, st, 0};
        L.out[R.b] = r;
      }
      return;
    }
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* slab = reinterpret_cast<float2*>(smem_raw);  // [PB][RS]
  float2* twid = slab + PB * RS;
  __shared__ unsigned long long wkey[T / 32];
  __shared__ float4 wsum[T / 32];  // per warp: the float pairs (hi, lo) of the sums of s and s^2
  for (int i = tid; i < N; i += T) twid[i] = L.twiddle[i];
  const float2* hw = R.h;
  irow_assemble<N, PB, T>(hw, slab, PB, [&](int p) { return pb * PB + p; }, tid);
  __syncthreads();
  irow_passA<N, PB, T>(slab, PB, tid);
  __syncthreads();
  float* surf = reinterpret_cast<float*>(R.zr);  // [N][N] response
  // running maxima of the y1 rows and of the y2 rows: each thread meets either
  // set in increasing row-major index, so a strict '>' keeps the smallest
  // index among equal values; one argmax key per set at the end
  // (initial index: the thread's first pixel of each set)
  constexpr int TB = PB * R1;
  float bva = -INFINITY, bvb = -INFINITY;
  uint32_t bia = static_cast<uint32_t>((pb * PB + tid / R1) * N + tid % R1), bib = bia + (N / 2) * N;
  float s1 = 0.f, s2 = 0.f;  // sums of s and s^2 over every pixel of the block
#pragma unroll
  for (int i = 0; i < (TB + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if (TB % T != 0 && task >= TB) break;
    const int p = task / R1, k1 = task % R1;
    float2 v[R2];
    irow_passB<N>(slab + p * RS, twid, k1, v);
    const int y1 = pb * PB + p, y2 = y1 + N / 2;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int x = k1 + R1 * k2;
      if constexpr (WRITE_S) {
        surf[y1 * N + x] = v[k2].x;
        surf[y2 * N + x] = v[k2].y;
      }
      s1 += v[k2].x + v[k2].y;
      s2 = fmaf(v[k2].x, v[k2].x, fmaf(v[k2].y, v[k2].y, s2));
      if (v[k2].x > bva) {
        bva = v[k2].x;
        bia = static_cast<uint32_t>(y1 * N + x);
      }
      if (v[k2].y > bvb) {
        bvb = v[k2].y;
        bib = static_cast<uint32_t>(y2 * N + x);
      }
    }
  }
  unsigned long long best = 0ull;
  if (TB % T == 0 || tid < TB) {  // n = 512: threads without a task hold no pixel
    const unsigned long long ka = argmax_key(bva, bia), kb = argmax_key(bvb, bib);
    best = ka > kb ? ka : kb;
  }
  best = warp_max_u64(best);
  // the block's sums as float pairs (FP32 additions with their errors kept),
  // over the lanes and then over the warps; one FP64 addition per total
  float h1 = s1, l1 = 0.f, h2 = s2, l2 = 0.f;
  warp_sum_ff2(h1, l1);
  warp_sum_ff2(h2, l2);
  if (lane == 0) {
    wkey[warp] = best;
    wsum[warp] = make_float4(h1, l1, h2, l2);
  }
  __syncthreads();
  if (warp == 0) {
    const unsigned long long k = warp_max_u64(lane < T / 32 ? wkey[lane] : 0ull);
    const float4 q = lane < T / 32 ? wsum[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    float a1 = q.x, e1 = q.y, a2 = q.z, e2 = q.w;
    warp_sum_ff2(a1, e1);
    warp_sum_ff2(a2, e2);
    if (lane == 0) {
      const double t1 = static_cast<double>(a1) + static_cast<double>(e1);
      const double t2 = static_cast<double>(a2) + static_cast<double>(e2);
      unsigned long long* part = R.part + 3 * pb;
      part[0] = k;
      part[1] = static_cast<unsigned long long>(__double_as_longlong(t1));
      part[2] = static_cast<unsigned long long>(__double_as_longlong(t2));
    }
  }
  if constexpr (kFold) {
    if (R.done != nullptr) {
      __shared__ int s_last;
      // (thread 0 wrote this block's partial itself: its fence below orders
      // the partial before its ticket)
      if (tid == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(R.done, 1u);
        s_last = prev == static_cast<unsigned int>(G::NB3 - 1);
        if (s_last) {
          __threadfence();  // the other blocks' partials are visible to this block
          *R.done = 0u;     // ready for the next call
        }
      }
      __syncthreads();
      if (s_last) disc_stage<N>(L, R);
    }
  }
}

template <int N, bool WRITE_S = true>
__global__ void __launch_bounds__(256, 5) stream_irows_kernel(const MatchLaunch L, const StreamWork W) {
  irows_stage<N, WRITE_S>(L, slice_ref<N>(L, W, blockIdx.x / StreamGeom<N>::NB3), blockIdx.x % StreamGeom<N>::NB3);
}

// Finalize of one window by the last of its inverse-row blocks (256
// threads, exclusion radius below 8 px): the global argmax and totals from
// the blocks' partials, the rows py - R .. py + R recomputed with the
// inverse-row steps (the values equal the blocks' own bit for bit), the
// (2R + 1)^2 values around the peak kept in shared memory, the disc sums in
// FP64 and the record.
template <int N>
__device__ __forceinline__ void disc_stage(const MatchLaunch& L, const WinRef& R) {
  using G = StreamGeom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, RS = G::RS, T = 256, PB = 16;
  constexpr int TB = PB * R1;
  constexpr int RMAX = 7;
  constexpr int DW = 2 * RMAX + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* slab = reinterpret_cast<float2*>(smem_raw);  // [PB][RS]
  float2* twid = slab + PB * RS;
  __shared__ unsigned long long d_key;
  __shared__ double d_tot[2];
  __shared__ float d_val[DW][DW];  // s around the peak, [dy + R][dx + R]
  __syncthreads();  // the block's own inverse rows are done with the shared memory
  for (int i = tid; i < N; i += T) twid[i] = L.twiddle[i];
  if (warp == 0) {
    unsigned long long gk = 0ull;
    double ta = 0.0, tc = 0.0;
    for (int k = lane; k < G::NB3; k += 32) {
      const unsigned long long* part = R.part + 3 * k;
      const unsigned long long v = __ldcg(part);
      gk = v > gk ? v : gk;
      ta += __longlong_as_double(static_cast<long long>(__ldcg(part + 1)));
      tc += __longlong_as_double(static_cast<long long>(__ldcg(part + 2)));
    }
    gk = warp_max_u64(gk);
    ta = warp_sum_f64(ta);
    tc = warp_sum_f64(tc);
    if (lane == 0) {
      d_key = gk;
      d_tot[0] = ta;
      d_tot[1] = tc;
    }
  }
  __syncthreads();
  const unsigned long long gk = d_key;
  const uint32_t pidx = key_index(gk);
  const int py = static_cast<int>(pidx / N), px = static_cast<int>(pidx % N);
  int rr = static_cast<int>(sqrtf(L.radius2));
  while ((rr + 1) * (rr + 1) <= static_cast<int>(L.radius2)) ++rr;
  while (rr * rr > static_cast<int>(L.radius2)) --rr;
  rr = rr < 1 ? 1 : rr;  // at most RMAX: the host folds the finalize only for r2 < 64
  const int np = 2 * rr + 1;  // row pairs holding the rows py - rr .. py + rr
  const int p0 = (py - rr) & (N / 2 - 1);
  irow_assemble<N, PB, T>(R.h, slab, np, [&](int p) { return (p0 + p) & (N / 2 - 1); }, tid);
  __syncthreads();
  irow_passA<N, PB, T>(slab, np, tid);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < (TB + T - 1) / T; ++i) {
    const int task = tid + i * T;
    if ((TB % T != 0 && task >= TB) || task / R1 >= np) continue;
    const int p = task / R1, k1 = task % R1;
    float2 v[R2];
    irow_passB<N>(slab + p * RS, twid, k1, v);
    const int y1 = (p0 + p) & (N / 2 - 1);
    const int dy1 = ((y1 - py + N / 2) & (N - 1)) - N / 2, dy2 = ((y1 + N / 2 - py + N / 2) & (N - 1)) - N / 2;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int dx = ((k1 + R1 * k2 - px + N / 2) & (N - 1)) - N / 2;
      if (dx >= -rr && dx <= rr) {
        if (dy1 >= -rr && dy1 <= rr) d_val[dy1 + RMAX][dx + RMAX] = v[k2].x;
        if (dy2 >= -rr && dy2 <= rr) d_val[dy2 + RMAX][dx + RMAX] = v[k2].y;
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    double da = 0.0, dc = 0.0, dn = 0.0;
    for (int e = lane; e < np * np; e += 32) {
      const int dy = e / np - rr, dx = e % np - rr;
      if (dy * dy + dx * dx <= static_cast<int>(L.radius2)) {
        const double d = d_val[dy + RMAX][dx + RMAX];
        da += d;
        dc += d * d;
        dn += 1.0;
      }
    }
    da = warp_sum_f64(da);
    dc = warp_sum_f64(dc);
    dn = warp_sum_f64(dn);
    if (lane == 0) {
      const float nb[4] = {d_val[RMAX - 1][RMAX], d_val[RMAX + 1][RMAX], d_val[RMAX][RMAX - 1], d_val[RMAX][RMAX + 1]};
      L.out[R.b] = window_result(N, py, px, key_value(gk), d_tot[0] - da, d_tot[1] - dc,
                                 static_cast<double>(N) * N - dn, nb);
    }
  }
}

// ---------------------------------------------------------------------------
// K4: peak, SNR, subpixel, result
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) stream_final_kernel(const MatchLaunch L, const StreamWork W) {
  using G = StreamGeom<N>;
  const long long s = blockIdx.x;
  const long long b = W.b0 + s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int st = stat_status(W.stats[s]);
  if (st == kStatusSkip) return;
  swift_result* out = L.out + b;
  if (st != SWIFT_WIN_OK) {
    if (tid == 0) {
      swift_result r = {0, 0, 0.f, 0.f, 0.f, 0.f, st, 0};
      *out = r;
    }
    return;
  }
  // one warp per window: totals from the block partials of K3, minus the
  // pixels inside the exclusion disc (read back from the response), in FP64
  if (warp != 0) return;
  unsigned long long gk = 0ull;
  double ta = 0.0, tc = 0.0;
#pragma unroll
  for (int k = 0; k < G::NB3; ++k) {
    const unsigned long long* part = W.part + 3 * (s * G::NB3 + k);
    const unsigned long long v = part[0];
    gk = v > gk ? v : gk;
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
    const float nb[4] = {surf[((py + N - 1) & (N - 1)) * N + px], surf[((py + 1) & (N - 1)) * N + px],
                         surf[py * N + ((px + N - 1) & (N - 1))], surf[py * N + ((px + 1) & (N - 1))]};
    *out = window_result(N, py, px, key_value(gk), ta - da, tc - dc, static_cast<double>(N) * N - dn, nb);
  }
}

// ---------------------------------------------------------------------------
// K4 (plain forward): peak, SNR and subpixel fit without a stored response
// ---------------------------------------------------------------------------
// K3 keeps only block argmax keys and the sums of s and s^2.  The exclusion
// disc (radius r) and the parabola need s on the rows within R = floor(r) + 1
// of the peak; this kernel recomputes those rows from H with K3's own row-pair
// steps (the values equal K3's bit for bit, so total minus disc is exact up to
// the FP64 sums) -- a pruned inverse: about 2R + 1 of the n/2 row pairs
// instead of a full n x n response written and read back.
// T threads per window, PB row pairs per chunk (T / 16)
template <int N, int T>
__device__ __forceinline__ void peak_stage(const MatchLaunch& L, const WinRef& R) {
  using G = StreamGeom<N>;
  constexpr int R1 = G::R1, R2 = G::R2, RS = G::RS;
  constexpr int PB = T / 16;
  constexpr int TB = PB * R1;
  const long long b = R.b;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int st = stat_status(load_stats(R));
  if (st == kStatusSkip) return;
  swift_result* out = L.out + b;
  if (st != SWIFT_WIN_OK) {
    if (tid == 0) {
      swift_result r = {0, 0, 0.f, 0.f, 0.f, 0.f, st, 0};
      *out = r;
    }
    return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* slab = reinterpret_cast<float2*>(smem_raw);  // [PB][RS]
  float2* twid = slab + PB * RS;
  __shared__ unsigned long long s_key;
  __shared__ double s_tot[2];
  __shared__ double s_red[T / 32][3];
  __shared__ float s_nb[4];  // s at (py - 1, px), (py + 1, px), (py, px - 1), (py, px + 1)
  for (int i = tid; i < N; i += T) twid[i] = L.twiddle[i];
  if (warp == 0) {
    // global argmax and totals from the block partials of K3
    unsigned long long gk = 0ull;
    double ta = 0.0, tc = 0.0;
    for (int k = lane; k < G::NB3; k += 32) {
      const unsigned long long* part = R.part + 3 * k;
      const unsigned long long v = __ldcg(part);
      gk = v > gk ? v : gk;
      ta += __longlong_as_double(static_cast<long long>(__ldcg(part + 1)));
      tc += __longlong_as_double(static_cast<long long>(__ldcg(part + 2)));
    }
    gk = warp_max_u64(gk);
    ta = warp_sum_f64(ta);
    tc = warp_sum_f64(tc);
    if (lane == 0) {
      s_key = gk;
      s_tot[0] = ta;
      s_tot[1] = tc;
    }
  }
  __syncthreads();
  const unsigned long long gk = s_key;
  const uint32_t pidx = key_index(gk);
  const int py = static_cast<int>(pidx / N), px = static_cast<int>(pidx % N);
  // rows within rr of the peak: the disc (dy^2 + dx^2 <= r2, so |dy| <=
  // floor(sqrt(r2))) and the parabola's neighbours (|dy| <= 1)
  int rr = static_cast<int>(sqrtf(L.radius2));
  while ((rr + 1) * (rr + 1) <= static_cast<int>(L.radius2)) ++rr;
  while (rr * rr > static_cast<int>(L.radius2)) --rr;
  rr = rr < 1 ? 1 : rr;
  // row pairs (y, y + n/2) holding the rows py - rr .. py + rr: consecutive pair indices
  const int npairs = 2 * rr + 1 < N / 2 ? 2 * rr + 1 : N / 2;
  const int p0 = (py - rr) & (N / 2 - 1);
  const float2* hw = R.h;
  double da = 0.0, dc = 0.0, dn = 0.0;
  for (int c0 = 0; c0 < npairs; c0 += PB) {
    const int np = npairs - c0 < PB ? npairs - c0 : PB;
    irow_assemble<N, PB, T>(hw, slab, np, [&](int p) { return (p0 + c0 + p) & (N / 2 - 1); }, tid);
    __syncthreads();
    irow_passA<N, PB, T>(slab, np, tid);
    __syncthreads();
    // pass B into registers, then the outputs back into the slab in natural
    // order (slab row p, position phys(x): s[y1][x] + i s[y1 + n/2][x])
    constexpr int KB = (TB + T - 1) / T;
    float2 v[KB][R2];
#pragma unroll
    for (int i = 0; i < KB; ++i) {
      const int task = tid + i * T;
      if ((TB % T != 0 && task >= TB) || task / R1 >= np) continue;
      irow_passB<N>(slab + (task / R1) * RS, twid, task % R1, v[i]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < KB; ++i) {
      const int task = tid + i * T;
      if ((TB % T != 0 && task >= TB) || task / R1 >= np) continue;
      float2* row = slab + (task / R1) * RS;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) row[G::phys(task % R1 + R1 * k2)] = v[i][k2];
    }
    __syncthreads();
    // disc pixels of this chunk's rows (FP64 sums) and the peak's neighbours
    if (warp == 0) {
      const int D = 2 * rr + 1;
      for (int e = lane; e < D * D; e += 32) {
        const int dy = e / D - rr, dx = e % D - rr;
        const int y = (py + dy) & (N - 1), x = (px + dx) & (N - 1);
        const int slot = ((y & (N / 2 - 1)) - p0 - c0) & (N / 2 - 1);
        if (slot >= np) continue;  // a row of another chunk
        const float2 pv = slab[slot * RS + G::phys(x)];
        const float val = y >= N / 2 ? pv.y : pv.x;
        if (dy * dy + dx * dx <= static_cast<int>(L.radius2)) {
          const double d = val;
          da += d;
          dc += d * d;
          dn += 1.0;
        }
        if (dx == 0 && (dy == -1 || dy == 1)) s_nb[dy < 0 ? 0 : 1] = val;
        if (dy == 0 && (dx == -1 || dx == 1)) s_nb[dx < 0 ? 2 : 3] = val;
      }
    }
    __syncthreads();  // the slab is reused by the next chunk
  }
  da = warp_sum_f64(da);
  dc = warp_sum_f64(dc);
  dn = warp_sum_f64(dn);
  if (lane == 0) {
    s_red[warp][0] = da;
    s_red[warp][1] = dc;
    s_red[warp][2] = dn;
  }
  __syncthreads();
  if (tid == 0) {
    for (int k = 1; k < T / 32; ++k) {
      da += s_red[k][0];
      dc += s_red[k][1];
      dn += s_red[k][2];
    }
    *out = window_result(N, py, px, key_value(gk), s_tot[0] - da, s_tot[1] - dc, static_cast<double>(N) * N - dn,
                         s_nb);
  }
}

template <int N>
struct PeakGeom {
  static constexpr int T = 128;  // threads per window (standalone kernel)
  static constexpr int PB = T / 16;
};

template <int N>
__global__ void __launch_bounds__(128, 5) stream_peak_kernel(const MatchLaunch L, const StreamWork W) {
  peak_stage<N, PeakGeom<N>::T>(L, slice_ref<N>(L, W, blockIdx.x));
}

// ---------------------------------------------------------------------------
// dynamic shared-memory sizes of the streaming kernels
// ---------------------------------------------------------------------------
template <int N, typename TIn>
constexpr size_t rows_smem() {
  using G = StreamGeom<N>;
  // (uint8: 128 bytes of slack that align the tensor-map tiles)
  return sizeof(float2) * (G::RB * G::RS + N) + sizeof(float) * (N + G::R2 * (G::R1 + 4)) +
         2 * sizeof(TIn) * G::RB * G::template stage_stride<TIn>() + (sizeof(TIn) == 1 ? 128 : 0);
}
template <int N>
constexpr size_t cols_smem() {
  using G = StreamGeom<N>;
  return sizeof(float2) * (N * (2 * G::CB + 8) + G::R1 * (G::R2 + 2));
}
template <int N>
constexpr size_t cpair_smem() {
  using P = PairGeom<N>;
  return sizeof(float4) * N * P::CB + sizeof(float4) * N + sizeof(float2) * P::R1 * P::TW + sizeof(float) * N;
}
template <int N>
constexpr size_t peak_smem() {
  return sizeof(float2) * (PeakGeom<N>::PB * StreamGeom<N>::RS + N);
}
template <int N>
constexpr size_t irows_smem() {
  using G = StreamGeom<N>;
  return sizeof(float2) * (G::PB * G::RS + N);
}

// dynamic shared-memory opt-in, once per device and kernel
template <typename K>
inline cudaError_t smem_optin(K kern, size_t bytes, unsigned& done_mask, int dev) {
  if (dev < 32 && (done_mask & (1u << dev))) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e == cudaSuccess && dev < 32) done_mask |= 1u << dev;
  return e;
}

}  // namespace swift
