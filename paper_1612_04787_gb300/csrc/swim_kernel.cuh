// Fused forward matching kernel: one window pair at a time per cluster of C
// CTAs; persistent clusters walk the batch with a static stride.
//
// Per window pair (Sec. III, the swim step):
//   gather -> weighted-mean removal + cosine taper -> z = m' + i r'
//   -> 2D DFT of z (rows, then columns) -> unpack M, R from Z (Hermitian
//   split) -> C = M conj(R) -> G = C |C|^-w / n^2, G[0,0] = 0
//   -> inverse 2D DFT of the Hermitian G (columns for kx <= n/2 only, then
//   rows two at a time as one complex transform) -> real match response s
//   -> peak (argmax, smallest index on ties) -> SNR against the background
//   outside the exclusion disc -> separable parabola subpixel fit.
//
// Data layout.  The n x n complex field is split across the C CTAs of a
// cluster.  In the row phase CTA r owns rows [r n/C, (r+1) n/C); in the
// column phase it owns n/C columns closed under kx -> -kx, so the Hermitian
// unpack stays inside the CTA.  The two redistributions go through
// distributed shared memory: every thread holds its share in registers, the
// cluster synchronises, the values are stored straight into the owner CTA's
// shared memory (st.shared::cluster), and a second cluster barrier publishes
// them.  With C = 1 the same code runs inside one CTA.
//
// 1D transforms.  A length-n line (n = R1 R2) is transformed by two radix
// passes that are in place per thread, so no thread overwrites what another
// still has to read and a pass needs no barrier between its loads and stores:
//   pass A: thread j loads positions j + R2 m (m < R1), DFT_R1, stores back;
//   pass B: thread k1 loads the contiguous block R2 k1 + n2 (n2 < R2),
//           multiplies by W_n^{n2 k1}, DFT_R2.
// The result X[k1 + R1 k2] then sits at position k2 + R2 k1 ("digit-reversed"
// order rho); the inverse column transform consumes that order directly (its
// passes run in the opposite order), and the row/column redistributions
// scatter to natural order for free.  Row lines are padded by one element
// every R2 so the strided accesses are free of bank conflicts.
//
// uint8 section windows are staged by the bulk-copy engine (cp.async.bulk,
// one copy per row, completion counted on an mbarrier): the next window's
// rows are fetched while the current window is transformed.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dft_regs.cuh"
#include "swift_internal.h"

namespace swift {

template <int N, int C>
struct Geometry;
template <>
struct Geometry<64, 1> {
  static constexpr int T = 512, R1 = 8, R2 = 8, RS = 72, MINB = 2;
};
template <>
struct Geometry<128, 2> {
  static constexpr int T = 512, R1 = 16, R2 = 8, RS = 152, MINB = 2;
};
template <>
struct Geometry<256, 8> {
  static constexpr int T = 512, R1 = 16, R2 = 16, RS = 272, MINB = 2;
};

template <int N, int C>
struct Plan2D {
  using G = Geometry<N, C>;
  static constexpr int T = G::T, R1 = G::R1, R2 = G::R2, RS = G::RS;
  static constexpr int ROWS = N / C;      // lines owned per CTA in each phase
  static constexpr int Q = N / (2 * C);  // kx in [Q r, Q r + Q) plus their partners
  static constexpr int HALF = ROWS / 2;  // packed inverse rows per CTA
  static constexpr int SPAN = N + 16;    // staged bytes per row (16-byte aligned span)
  static_assert(R1 * R2 == N, "radix split");
  static_assert(RS >= N + N / R2, "row padding");
  static_assert(HALF % R2 == 0, "row pairing must stay inside one thread");
  // task counts of each pass and the per-thread slot counts
  static constexpr int TA = ROWS * R2;   // pass A tasks over a full slab (R1 points each)
  static constexpr int TB = ROWS * R1;   // pass B tasks over a full slab (R2 points each)
  static constexpr int TAh = HALF * R2;  // over half a slab
  static constexpr int TBh = HALF * R1;
  static constexpr int KA = (TA + T - 1) / T, KB = (TB + T - 1) / T;
  static constexpr int KAh = (TAh + T - 1) / T, KBh = (TBh + T - 1) / T;
  // shared memory (complex elements)
  static constexpr int ROW_SLAB = ROWS * RS;
  static constexpr int COL_SLAB = N * ROWS;
  static constexpr int SLAB = ROW_SLAB > COL_SLAB ? ROW_SLAB : COL_SLAB;
  static __device__ __forceinline__ int phys(int p) { return p + p / R2; }
  // digit-reversed position of frequency k
  static __device__ __forceinline__ int rho(int k) { return k / R1 + R2 * (k % R1); }
  // column ownership: (rank, local column) -> kx, and kx -> (rank, local column)
  static __device__ __forceinline__ int kx_of(int r, int lc) {
    if (lc < Q) return Q * r + lc;
    if (r == 0 && lc == Q) return N / 2;
    return N - (Q * r + lc - Q);
  }
  static __device__ __forceinline__ void owner_of(int kx, int& r, int& lc) {
    if (kx < N / 2) {
      r = kx / Q;
      lc = kx % Q;
    } else if (kx == N / 2) {
      r = 0;
      lc = Q;
    } else {
      int k2 = N - kx;
      r = k2 / Q;
      lc = Q + k2 % Q;
    }
  }
};

// ---------------------------------------------------------------------------
// cluster helpers (C == 1: plain shared memory and __syncthreads)
// ---------------------------------------------------------------------------
template <int C>
__device__ __forceinline__ unsigned cluster_rank() {
  if constexpr (C == 1) {
    return 0;
  } else {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
  }
}

template <int C>
__device__ __forceinline__ void cluster_barrier() {
  if constexpr (C == 1) {
    __syncthreads();
  } else {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  }
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared::cluster address of the same offset in CTA `rank`
template <int C>
__device__ __forceinline__ uint32_t map_rank(uint32_t local, unsigned rank) {
  if constexpr (C == 1) {
    return local;
  } else {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
  }
}

template <int C>
__device__ __forceinline__ void st_cl(uint32_t addr, float2 v) {
  if constexpr (C == 1) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
  } else {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
  }
}
template <int C>
__device__ __forceinline__ void st_cl_f32(uint32_t addr, float v) {
  if constexpr (C == 1) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
  } else {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
  }
}
template <int C>
__device__ __forceinline__ void st_cl_f64(uint32_t addr, double v) {
  if constexpr (C == 1) {
    asm volatile("st.shared.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
  } else {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
  }
}
template <int C>
__device__ __forceinline__ void st_cl_u64(uint32_t addr, unsigned long long v) {
  if constexpr (C == 1) {
    asm volatile("st.shared.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
  } else {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
  }
}

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (the staged uint8 window loads)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on an mbarrier phase: gives up after ~2 s of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
  if (mbar_try_wait(mbar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (;;) {
    if (mbar_try_wait(mbar, parity)) return true;
    if (globaltimer() - t0 > 2000000000ull) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}
// Tiled tensor copy of the box at (c0, c1, c2) of a 3D tensor map (the map a
// __grid_constant__ kernel argument) into shared memory at `dst` (128-byte
// aligned), its bytes counted on the mbarrier; boxes reaching past the
// tensor's extent read zeros there.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* map, int c0, int c1, int c2, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
      : "memory");
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
// Whitening factor |C|^-w from |C|^2 (Sec. II): 2^(-w/2 log2 |C|^2), 0 where
// |C| = 0.  The base-2 logarithm and exponential are the hardware
// approximations (PTX lg2.approx / ex2.approx, a few ulp); their
// subnormal-flushing forms are safe because inputs below 2^-100 are first
// scaled by 2^64 (exact) and the exponent stays within [-64, 75], so neither
// instruction sees or makes a subnormal.
__device__ __forceinline__ float whiten_factor(float mag2, float half_w) {
  if (!(mag2 > 0.f)) return 0.f;
  const bool tiny = mag2 < 0x1p-100f;
  float lg, f;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(tiny ? mag2 * 0x1p64f : mag2));
  if (tiny) lg -= 64.f;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"(half_w * lg));
  return f;
}

// ---------------------------------------------------------------------------
// (value, index) ordering for the argmax: larger value wins, then smaller
// index.  High 32 bits: order-preserving encoding of the float; low: ~index.
__device__ __forceinline__ unsigned long long argmax_key(float v, uint32_t idx) {
  uint32_t b = __float_as_uint(v);
  b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  return (static_cast<unsigned long long>(b) << 32) | static_cast<unsigned long long>(~idx);
}
__device__ __forceinline__ float key_value(unsigned long long k) {
  uint32_t b = static_cast<uint32_t>(k >> 32);
  b = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
  return __uint_as_float(b);
}
__device__ __forceinline__ uint32_t key_index(unsigned long long k) { return ~static_cast<uint32_t>(k); }

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Warp sum of FP32 values carried as an unevaluated float pair (hi + lo, the
// error of every addition kept by Knuth's TwoSum), returned as a double: about
// 48 significant bits from FP32 additions only.  This GPU's FP64 unit issues
// a warp instruction every few dozen cycles, so an FP64 butterfly makes the
// per-warp block sums of the streaming kernels wait on it.  Every lane ends
// with the same pair: TwoSum's (s, e) is exact and symmetric in its operands.
__device__ __forceinline__ void warp_sum_ff2(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, o), olo = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = __fadd_rn(hi, ohi);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(ohi, bb));
    const float t = __fadd_rn(e, __fadd_rn(lo, olo));
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
  }
}
__device__ __forceinline__ double warp_sum_ff(float v) {
  float hi = v, lo = 0.f;
  warp_sum_ff2(hi, lo);
  return static_cast<double>(hi) + static_cast<double>(lo);
}
__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_min_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// the record of one window (Sec. III): the peak, its SNR against the
// background outside the exclusion disc, the parabola subpixel fit
// ---------------------------------------------------------------------------
// Peak (py, px, value pk); ta, tc, tn: the sum of s, the sum of s^2 and the
// number of background pixels (FP64 sums); nb: the wrapped neighbours
// s(py-1, px), s(py+1, px), s(py, px-1), s(py, px+1).  SNR = (pk - mu) / sigma
// (population sigma; +inf when sigma = 0 and the peak is above the mean), a
// separable 3-point parabola per axis clamped to [-1/2, 1/2] (0 when not
// concave), shifts in [-n/2, n/2).  The background mean and
// variance are formed in FP64; the ratios that follow need no FP64 (their
// results are stored as FP32): this GPU's FP64 divide and square root are
// long chains on a slow unit, on the critical path of every window.
//   1 / tn: the FP32 reciprocal (correctly rounded; tn is an integer below
//     2^24) refined by one Newton-Raphson step x + x (1 - tn x), about 46 bits;
//   SNR = (peak - mean) / sqrt(var): FP32 reciprocal square root of the FP64
//     variance (a variance below the FP32 normal range takes the FP64 route);
//   parabola: numerator and denominator exact in FP64 (sums of three FP32
//     values), their ratio in FP32.
__device__ __forceinline__ swift_result window_result(int n, int py, int px, float pkf, double ta, double tc,
                                                      double tn, const float* nb) {
  const double x0 = static_cast<double>(__frcp_rn(static_cast<float>(tn)));
  const double inv = fma(x0, fma(-tn, x0, 1.0), x0);
  const double mu = ta * inv;
  const double var = fma(tc, inv, -mu * mu);
  const double pk = static_cast<double>(pkf);
  float snr;
  if (var > 0.0) {
    const float vf = static_cast<float>(var);
    if (vf >= 1.17549435e-38f) {
      snr = static_cast<float>(pk - mu) * rsqrtf(vf);
    } else {
      snr = static_cast<float>((pk - mu) / sqrt(var));
    }
  } else {
    snr = pk > mu ? __int_as_float(0x7f800000) : 0.f;
  }
  auto parab = [](float sm, float s0, float sp) -> float {
    const double den = static_cast<double>(sm) - 2.0 * static_cast<double>(s0) + static_cast<double>(sp);
    if (!(den < 0.0)) return 0.f;
    const float d = 0.5f * static_cast<float>(static_cast<double>(sm) - static_cast<double>(sp)) /
                    static_cast<float>(den);
    return d < -0.5f ? -0.5f : (d > 0.5f ? 0.5f : d);
  };
  const float fy = parab(nb[0], pkf, nb[1]);
  const float fx = parab(nb[2], pkf, nb[3]);
  const int dy = py < n / 2 ? py : py - n;
  const int dx = px < n / 2 ? px : px - n;
  swift_result r;
  r.dy = dy;
  r.dx = dx;
  r.sy = static_cast<float>(dy) + fy;
  r.sx = static_cast<float>(dx) + fx;
  r.snr = snr;
  r.peak = pkf;
  r.status = SWIFT_WIN_OK;
  r.reserved = 0;
  return r;
}

// ---------------------------------------------------------------------------
// shared-memory scratch besides the slab
// ---------------------------------------------------------------------------
constexpr int kMaxC = 8;
struct WinInfo {
  long long w;             // window index (>= n_windows: no more work)
  int my, mx, ry, rx;      // origins (section mode)
  int ok;                  // inside both images
};
struct __align__(16) Scratch {
  WinInfo win[2];
  unsigned long long mbar;  // staged-load barrier
  float wsum[32][2];
  float wmin[32][2], wmax[32][2];
  int wbad[32];
  unsigned long long wkey[32];
  float wbg[32][4];  // per warp: sum s (hi, lo), sum s^2 (hi, lo)
  int wcnt[32];
  // cluster all-gather slots: written by every CTA into every CTA
  double csum[kMaxC][2];
  float cmin[kMaxC][2], cmax[kMaxC][2];
  unsigned long long cbad[kMaxC];
  unsigned long long ckey[kMaxC];
  double cbg[kMaxC][3];
  float nb[4];  // peak neighbours for the subpixel fit (rank 0): y-1, y+1, x-1, x+1
  int broken;   // a staged load timed out
};

template <typename TIn>
__device__ __forceinline__ float load_px(const TIn* p) {
  if constexpr (sizeof(TIn) == 1) {
    return static_cast<float>(__ldg(reinterpret_cast<const unsigned char*>(p)));
  } else {
    return __ldg(reinterpret_cast<const float*>(p));
  }
}

// window_check for window b of launch L, from its level and origin arrays
// (patch mode: the level only)
__device__ __forceinline__ int launch_window_check(const MatchLaunch& L, long long b, int n) {
  const int lv = L.level_idx != nullptr ? __ldg(L.level_idx + b) : L.level;
  if (L.patch_mode) return window_check(n, lv, L.level, 0, 0, 0, 0, n, n, n, n);
  return window_check(n, lv, L.level, __ldg(L.ref_origin + 2 * b), __ldg(L.ref_origin + 2 * b + 1),
                      __ldg(L.mov_origin + 2 * b), __ldg(L.mov_origin + 2 * b + 1), L.ref_h, L.ref_w, L.mov_h,
                      L.mov_w);
}

template <int N, int C, bool BULK>
constexpr size_t forward_smem_bytes() {
  using P = Plan2D<N, C>;
  return sizeof(float2) * (P::SLAB + 2 * N) + sizeof(float) * N + (BULK ? 2 * P::ROWS * P::SPAN : 0) +
         sizeof(Scratch);
}

// ---------------------------------------------------------------------------
// the fused forward kernel
// ---------------------------------------------------------------------------
template <int N, int C, typename TIn, bool BULK>
__global__ void __launch_bounds__(Plan2D<N, C>::T, Geometry<N, C>::MINB) swim_forward_kernel(const MatchLaunch L) {
  using P = Plan2D<N, C>;
  constexpr int T = P::T, R1 = P::R1, R2 = P::R2, ROWS = P::ROWS, Q = P::Q, RS = P::RS, HALF = P::HALF;
  constexpr int NW = T / 32;
  static_assert(!BULK || sizeof(TIn) == 1, "bulk staging is for uint8 windows");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* slab = reinterpret_cast<float2*>(smem_raw);
  float2* dcbuf = slab + P::SLAB;                  // inverse column kx = 0 (packed with n/2)
  float2* twid = dcbuf + N;                        // [R2][R1] W_N^{n2 k1}
  float* taper = reinterpret_cast<float*>(twid + N);
  unsigned char* stage = reinterpret_cast<unsigned char*>(taper + N);  // [2][ROWS][SPAN]
  Scratch* sc = reinterpret_cast<Scratch*>(stage + (BULK ? 2 * ROWS * P::SPAN : 0));

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const unsigned rank = cluster_rank<C>();
  const long long cid = static_cast<long long>(blockIdx.x) / C;
  const long long G = static_cast<long long>(gridDim.x) / C;
  const long long B = L.n_windows;
  const uint32_t mbar = smem_addr(&sc->mbar);

  for (int i = tid; i < N; i += T) {
    twid[i] = L.twiddle[i];
    taper[i] = L.taper[i];
  }

  // Window descriptors live in shared memory, double-buffered: lane 0 of
  // warp 0 finds the next window of this cluster's stride set (skipping other
  // levels), reads its origins once and checks its bounds.
  auto fetch_info = [&](int slot, long long w) {
    while (w < B && L.level_idx != nullptr && __ldg(L.level_idx + w) != L.level) w += G;
    WinInfo wi;
    wi.w = w;
    wi.my = wi.mx = wi.ry = wi.rx = 0;
    wi.ok = 1;
    if (w < B && !L.patch_mode) {
      wi.my = __ldg(L.mov_origin + 2 * w);
      wi.mx = __ldg(L.mov_origin + 2 * w + 1);
      wi.ry = __ldg(L.ref_origin + 2 * w);
      wi.rx = __ldg(L.ref_origin + 2 * w + 1);
      wi.ok = window_check(N, L.level, L.level, wi.ry, wi.rx, wi.my, wi.mx, L.ref_h, L.ref_w, L.mov_h, L.mov_w) ==
              SWIFT_WIN_OK;
    }
    sc->win[slot] = wi;
  };
  // bulk-stage this CTA's ROWS rows of both windows (called by warp 0)
  auto prefetch = [&](const WinInfo& wi) {
    if constexpr (BULK) {
      const int ms = wi.mx & ~15, rs = wi.rx & ~15;
      const uint32_t mbytes = static_cast<uint32_t>(((wi.mx + N + 15) & ~15) - ms);
      const uint32_t rbytes = static_cast<uint32_t>(((wi.rx + N + 15) & ~15) - rs);
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(mbar, static_cast<uint32_t>(ROWS) * (mbytes + rbytes));
      }
      __syncwarp();
      const unsigned char* mb = static_cast<const unsigned char*>(L.mov) +
                                static_cast<long long>(wi.my + rank * ROWS) * L.mov_pitch + ms;
      const unsigned char* rb = static_cast<const unsigned char*>(L.ref) +
                                static_cast<long long>(wi.ry + rank * ROWS) * L.ref_pitch + rs;
      const uint32_t s0 = smem_addr(stage);
      for (int r = lane; r < ROWS; r += 32) {
        bulk_g2s(s0 + r * P::SPAN, mb + static_cast<long long>(r) * L.mov_pitch, mbytes, mbar);
        bulk_g2s(s0 + (ROWS + r) * P::SPAN, rb + static_cast<long long>(r) * L.ref_pitch, rbytes, mbar);
      }
    }
  };

  const float inv_k = 1.0f / static_cast<float>(L.ref_count);
  // raw pixels of one window straight from global memory into the thread's
  // pass-A registers (no staging)
  float mraw[P::KA][R1], rraw[P::KA][R1];
  auto load_direct = [&](const WinInfo& wi) {
    const TIn* mbase;
    const TIn* rbase;
    long long mpitch, rpitch;
    if (L.patch_mode) {
      mbase = static_cast<const TIn*>(L.mov) + wi.w * L.mov_stride;
      rbase = static_cast<const TIn*>(L.ref) + wi.w * L.ref_stride;
      mpitch = rpitch = N;
    } else {
      mbase = static_cast<const TIn*>(L.mov) + static_cast<long long>(wi.my) * L.mov_pitch + wi.mx;
      rbase = static_cast<const TIn*>(L.ref) + static_cast<long long>(wi.ry) * L.ref_pitch + wi.rx;
      mpitch = L.mov_pitch;
      rpitch = L.ref_pitch;
    }
#pragma unroll
    for (int i = 0; i < P::KA; ++i) {
      const int task = tid + i * T;
      const int line = task / R2, j = task % R2;
      const int y = rank * ROWS + line;
      const TIn* mrow = mbase + y * mpitch + j;
      const TIn* rrow = rbase + y * rpitch + j;
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        mraw[i][m] = load_px<TIn>(mrow + R2 * m);
        float rv = load_px<TIn>(rrow + R2 * m);
        for (int k = 1; k < L.ref_count; ++k) rv += load_px<TIn>(rrow + k * L.ref_stride + R2 * m);
        rraw[i][m] = L.ref_count > 1 ? rv * inv_k : rv;
      }
    }
  };
  // patch stacks of one level (64 x 64: the single-window latency case; the
  // larger kernels would keep their pixel registers live across windows): the
  // first window needs no descriptor, so its pixels are requested together
  // with the tables (one memory latency instead of two before the first
  // transform)
  bool preloaded = false;
  if constexpr (!BULK && N == 64) {
    if (L.patch_mode && L.level_idx == nullptr && cid < B) {
      WinInfo w0;
      w0.w = cid;
      w0.my = w0.mx = w0.ry = w0.rx = 0;
      w0.ok = 1;
      load_direct(w0);
      preloaded = true;
    }
  }
  // the first descriptor's loads overlap the table loads above
  if (tid == 0) {
    sc->broken = 0;
    if constexpr (BULK) {
      mbar_init(mbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fetch_info(0, cid);
  }
  __syncthreads();
  int cur = 0;
  if (BULK && warp == 0) {
    const WinInfo wi = sc->win[0];
    if (wi.w < B && wi.ok) prefetch(wi);
  }
  uint32_t parity = 0;
  const float half_w = -0.5f * L.w;
  const float inv_n2 = 1.0f / (static_cast<float>(N) * static_cast<float>(N));

  for (;;) {
    const WinInfo wi = sc->win[cur];
    if (wi.w >= B) break;
    swift_result* out = L.out + wi.w;
    if (!wi.ok) {  // uniform across the cluster
      if (rank == 0 && tid == 0) {
        swift_result r = {0, 0, 0.f, 0.f, 0.f, 0.f, SWIFT_WIN_OUT_OF_BOUNDS, 0};
        *out = r;
      }
      if (tid == 0) fetch_info(cur ^ 1, wi.w + G);
      __syncthreads();
      cur ^= 1;
      if (BULK && warp == 0) {
        const WinInfo nx = sc->win[cur];
        if (nx.w < B && nx.ok) prefetch(nx);
      }
      continue;
    }

    // ---- load raw pixels for row pass A; window statistics ----------------
    // task (line, j): elements x = j + R2 m, m < R1, of row rank*ROWS + line
    float s_m = 0.f, s_r = 0.f;
    float mn_m = 3.4e38f, mx_m = -3.4e38f, mn_r = 3.4e38f, mx_r = -3.4e38f;
    int bad = 0;
    if constexpr (BULK) {
      if (!mbar_wait_bounded(mbar, parity)) sc->broken = 1;
      parity ^= 1u;
      const int mo = wi.mx & 15, ro = wi.rx & 15;
#pragma unroll
      for (int i = 0; i < P::KA; ++i) {
        const int task = tid + i * T;
        const int line = task / R2, j = task % R2;
        const unsigned char* ms = stage + line * P::SPAN + mo + j;
        const unsigned char* rs = stage + (ROWS + line) * P::SPAN + ro + j;
#pragma unroll
        for (int m = 0; m < R1; ++m) {
          mraw[i][m] = static_cast<float>(ms[R2 * m]);
          rraw[i][m] = static_cast<float>(rs[R2 * m]);
        }
      }
    } else {
      if (!preloaded) load_direct(wi);
      preloaded = false;
    }
#pragma unroll
    for (int i = 0; i < P::KA; ++i) {
      const int task = tid + i * T;
      const int line = task / R2, j = task % R2;
      const float ay = taper[rank * ROWS + line];
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        const float a = ay * taper[j + R2 * m];
        s_m = fmaf(a, mraw[i][m], s_m);
        s_r = fmaf(a, rraw[i][m], s_r);
        mn_m = fminf(mn_m, mraw[i][m]);
        mx_m = fmaxf(mx_m, mraw[i][m]);
        mn_r = fminf(mn_r, rraw[i][m]);
        mx_r = fmaxf(mx_r, rraw[i][m]);
        if constexpr (sizeof(TIn) == 4) {
          bad |= !(fabsf(mraw[i][m]) <= 3.4e38f) | !(fabsf(rraw[i][m]) <= 3.4e38f);
        }
      }
    }
    {
      float a = warp_sum_f32(s_m), c = warp_sum_f32(s_r);
      float e = warp_min_f32(mn_m), f = warp_max_f32(mx_m), g = warp_min_f32(mn_r), h = warp_max_f32(mx_r);
      int bb = __any_sync(0xffffffffu, bad);
      if (lane == 0) {
        sc->wsum[warp][0] = a;
        sc->wsum[warp][1] = c;
        sc->wmin[warp][0] = e;
        sc->wmax[warp][0] = f;
        sc->wmin[warp][1] = g;
        sc->wmax[warp][1] = h;
        sc->wbad[warp] = bb;
      }
    }
    __syncthreads();  // also: the staged rows have been read by everyone
    if (warp == 0) {
      // next window: descriptor, then its staged rows
      if (lane == 0) fetch_info(cur ^ 1, wi.w + G);
      __syncwarp();
      if (BULK) {
        const WinInfo nx = sc->win[cur ^ 1];
        if (nx.w < B && nx.ok) prefetch(nx);
      }
    } else if (warp == 1) {
      // block statistics, all-gathered into every CTA of the cluster
      const double a = warp_sum_ff(lane < NW ? sc->wsum[lane][0] : 0.f);
      const double c = warp_sum_ff(lane < NW ? sc->wsum[lane][1] : 0.f);
      float e = lane < NW ? sc->wmin[lane][0] : 3.4e38f, f = lane < NW ? sc->wmax[lane][0] : -3.4e38f;
      float g = lane < NW ? sc->wmin[lane][1] : 3.4e38f, h = lane < NW ? sc->wmax[lane][1] : -3.4e38f;
      int bb = (lane < NW ? sc->wbad[lane] : 0) | sc->broken;
      e = warp_min_f32(e);
      f = warp_max_f32(f);
      g = warp_min_f32(g);
      h = warp_max_f32(h);
      bb = __any_sync(0xffffffffu, bb);
      if (lane < C) {
        const unsigned r = lane;
        st_cl_f64<C>(map_rank<C>(smem_addr(&sc->csum[rank][0]), r), a);
        st_cl_f64<C>(map_rank<C>(smem_addr(&sc->csum[rank][1]), r), c);
        st_cl_u64<C>(map_rank<C>(smem_addr(&sc->cmin[rank][0]), r),
                     (static_cast<unsigned long long>(__float_as_uint(g)) << 32) | __float_as_uint(e));
        st_cl_u64<C>(map_rank<C>(smem_addr(&sc->cmax[rank][0]), r),
                     (static_cast<unsigned long long>(__float_as_uint(h)) << 32) | __float_as_uint(f));
        st_cl_u64<C>(map_rank<C>(smem_addr(&sc->cbad[rank]), r), static_cast<unsigned long long>(bb ? 1 : 0));
      }
    }
    cluster_barrier<C>();
    float mu_m, mu_r;
    int wstatus;
    {
      double a = 0, c = 0;
      float e = 3.4e38f, f = -3.4e38f, g = 3.4e38f, h = -3.4e38f;
      unsigned long long bb = 0;
#pragma unroll
      for (int r = 0; r < C; ++r) {
        a += sc->csum[r][0];
        c += sc->csum[r][1];
        e = fminf(e, sc->cmin[r][0]);
        g = fminf(g, sc->cmin[r][1]);
        f = fmaxf(f, sc->cmax[r][0]);
        h = fmaxf(h, sc->cmax[r][1]);
        bb |= sc->cbad[r];
      }
      wstatus = (bb & 1) ? (sizeof(TIn) == 4 ? SWIFT_WIN_NONFINITE : SWIFT_WIN_TIMEOUT)
                         : ((e == f || g == h) ? SWIFT_WIN_FLAT : SWIFT_WIN_OK);
      if (sizeof(TIn) == 4 && sc->broken) wstatus = SWIFT_WIN_TIMEOUT;
      mu_m = static_cast<float>(a * L.inv_sum_a);
      mu_r = static_cast<float>(c * L.inv_sum_a);
    }
    if (wstatus != SWIFT_WIN_OK) {
      if (rank == 0 && tid == 0) {
        swift_result r = {0, 0, 0.f, 0.f, 0.f, 0.f, wstatus, 0};
        *out = r;
      }
      cluster_barrier<C>();  // the all-gather slots are rewritten by the next window
      cur ^= 1;
      continue;
    }

    // ---- row pass A: apodise, DFT_R1 over x = j + R2 m, store in place -----
#pragma unroll
    for (int i = 0; i < P::KA; ++i) {
      const int task = tid + i * T;
      const int line = task / R2, j = task % R2;
      const float ay = taper[rank * ROWS + line];
      float2 v[R1];
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        const float a = ay * taper[j + R2 * m];
        v[m] = make_float2(a * (mraw[i][m] - mu_m), a * (rraw[i][m] - mu_r));
      }
      dft<R1, -1>(v);
      float2* row = slab + line * RS;
#pragma unroll
      for (int q = 0; q < R1; ++q) row[P::phys(j + R2 * q)] = v[q];
    }
    // with R1 = R2 pass B reads only what the same warp's lanes wrote in pass A
    if constexpr (R1 == R2) {
      __syncwarp();
    } else {
      __syncthreads();
    }

    // ---- row pass B: block R2 k1 + n2, twiddle, DFT_R2, push to columns ----
    {
      float2 h[P::KB][R2];
#pragma unroll
      for (int i = 0; i < P::KB; ++i) {
        const int task = tid + i * T;
        const int line = task / R1, k1 = task % R1;
        const float2* row = slab + line * RS;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
          float2 x = row[P::phys(R2 * k1 + n2)];
          h[i][n2] = n2 == 0 ? x : cmul(x, twid[n2 * R1 + k1]);
        }
        dft<R2, -1>(h[i]);
      }
      cluster_barrier<C>();  // every CTA finished reading its row slab
      const uint32_t base = smem_addr(slab);
#pragma unroll
      for (int i = 0; i < P::KB; ++i) {
        const int task = tid + i * T;
        const int line = task / R1, k1 = task % R1;
        const int y = rank * ROWS + line;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const int kx = k1 + R1 * k2;
          int orank, lc;
          P::owner_of(kx, orank, lc);
          st_cl<C>(map_rank<C>(base + static_cast<uint32_t>((y * ROWS + lc) * sizeof(float2)), orank), h[i][k2]);
        }
      }
      cluster_barrier<C>();  // column slabs complete
    }

    // ---- column pass A (rows j + R2 m), in place ----------------------------
#pragma unroll
    for (int i = 0; i < P::KA; ++i) {
      const int task = tid + i * T;
      const int j = task / ROWS, lc = task % ROWS;
      float2 v[R1];
#pragma unroll
      for (int m = 0; m < R1; ++m) v[m] = slab[(j + R2 * m) * ROWS + lc];
      dft<R1, -1>(v);
#pragma unroll
      for (int q = 0; q < R1; ++q) slab[(j + R2 * q) * ROWS + lc] = v[q];
    }
    __syncthreads();

    // ---- column pass B (rows R2 k1 + n2), in place: Z in rho order ----------
#pragma unroll
    for (int i = 0; i < P::KB; ++i) {
      const int task = tid + i * T;
      const int k1 = task / ROWS, lc = task % ROWS;
      float2 v[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) {
        float2 x = slab[(R2 * k1 + n2) * ROWS + lc];
        v[n2] = n2 == 0 ? x : cmul(x, twid[n2 * R1 + k1]);
      }
      dft<R2, -1>(v);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) slab[(R2 * k1 + k2) * ROWS + lc] = v[k2];
    }
    __syncthreads();

    // ---- unpack + whiten + inverse column pass B' ---------------------------
    // thread (k1, lc < Q) owns the block of ky = k1 + R1 k2 (rows R2 k1 + k2).
    // Z = DFT(m' + i r'); with A = Z[k], B = Z[-k]:
    //   C = M conj(R) = ( Im(A B) / 2 , (|A|^2 - |B|^2) / 4 )
#pragma unroll
    for (int i = 0; i < P::KBh; ++i) {
      const int task = tid + i * T;
      if (P::TBh % T != 0 && task >= P::TBh) break;
      const int k1 = task / Q, lc = task % Q;
      const bool dc_col = (rank == 0 && lc == 0);
      const int plc = dc_col ? 0 : lc + Q;
      float2 v[R2];
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const int ky = k1 + R1 * k2;
        const int nky = (N - ky) & (N - 1);
        const float2 a = slab[(R2 * k1 + k2) * ROWS + lc];
        const float2 b = slab[P::rho(nky) * ROWS + plc];
        const float2 c = make_float2(0.5f * fmaf(a.x, b.y, a.y * b.x),
                                     0.25f * ((a.x * a.x + a.y * a.y) - (b.x * b.x + b.y * b.y)));
        const float mag2 = fmaf(c.x, c.x, c.y * c.y);
        const float s = whiten_factor(mag2, half_w) * inv_n2;
        float2 g = make_float2(c.x * s, c.y * s);
        if (dc_col) {
          // the Nyquist column kx = n/2 rides along as the imaginary part: both
          // columns are real after the inverse column transform
          const float2 a2 = slab[(R2 * k1 + k2) * ROWS + Q];
          const float2 b2 = slab[P::rho(nky) * ROWS + Q];
          const float2 c2 = make_float2(0.5f * fmaf(a2.x, b2.y, a2.y * b2.x),
                                        0.25f * ((a2.x * a2.x + a2.y * a2.y) - (b2.x * b2.x + b2.y * b2.y)));
          const float mq = fmaf(c2.x, c2.x, c2.y * c2.y);
          const float sq = whiten_factor(mq, half_w) * inv_n2;
          if (ky == 0) g = make_float2(0.f, 0.f);  // G[0,0] = 0
          g = make_float2(g.x - c2.y * sq, g.y + c2.x * sq);
        }
        v[k2] = g;
      }
      dft<R2, +1>(v);
#pragma unroll
      for (int n2 = 1; n2 < R2; ++n2) v[n2] = cmulc(v[n2], twid[n2 * R1 + k1]);
      if (dc_col) {
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) dcbuf[R2 * k1 + n2] = v[n2];
      } else {
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) slab[(R2 * k1 + n2) * ROWS + lc] = v[n2];
      }
    }
    __syncthreads();

    // ---- inverse column pass A' (rows n2 + R2 k1), push packed row pairs -----
    {
      float2 h[P::KAh][R1];
#pragma unroll
      for (int i = 0; i < P::KAh; ++i) {
        const int task = tid + i * T;
        const int n2 = task / Q, lc = task % Q;
        const bool valid = (P::TAh % T == 0) || task < P::TAh;
        const bool dc_col = (rank == 0 && lc == 0);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
          h[i][k1] = valid ? (dc_col ? dcbuf[n2 + R2 * k1] : slab[(n2 + R2 * k1) * ROWS + lc])
                           : make_float2(0.f, 0.f);
        }
        dft<R1, +1>(h[i]);  // h[i][n1] = H[y = n2 + R2 n1]
      }
      cluster_barrier<C>();  // every CTA finished reading its column slab
      const uint32_t base = smem_addr(slab);
      constexpr int NP = HALF / R2;  // n1 offset between the rows of a pair
#pragma unroll
      for (int i = 0; i < P::KAh; ++i) {
        const int task = tid + i * T;
        if (P::TAh % T != 0 && task >= P::TAh) break;
        const int n2 = task / Q, lc = task % Q;
        const int kx = P::kx_of(rank, lc);
        const bool dc_col = (rank == 0 && lc == 0);
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
          if ((n1 % (ROWS / R2)) >= NP) continue;  // n1 is the first row of a pair
          const int y1 = n2 + R2 * n1;
          const int orank = y1 / ROWS, p = y1 % ROWS;
          const uint32_t addr = map_rank<C>(base + static_cast<uint32_t>(p * RS * sizeof(float2)), orank);
          const float2 h1 = h[i][n1], h2 = h[i][n1 + NP];
          if (dc_col) {
            st_cl<C>(addr + P::phys(0) * sizeof(float2), make_float2(h1.x, h2.x));
            st_cl<C>(addr + P::phys(N / 2) * sizeof(float2), make_float2(h1.y, h2.y));
          } else {
            st_cl<C>(addr + P::phys(kx) * sizeof(float2), make_float2(h1.x - h2.y, h1.y + h2.x));
            st_cl<C>(addr + P::phys(N - kx) * sizeof(float2), make_float2(h1.x + h2.y, h2.x - h1.y));
          }
        }
      }
      cluster_barrier<C>();  // packed rows complete
    }

    // ---- inverse row pass A on packed rows, in place -------------------------
#pragma unroll
    for (int i = 0; i < P::KAh; ++i) {
      const int task = tid + i * T;
      if (P::TAh % T != 0 && task >= P::TAh) break;
      const int line = task / R2, j = task % R2;
      float2* row = slab + line * RS;
      float2 v[R1];
#pragma unroll
      for (int m = 0; m < R1; ++m) v[m] = row[P::phys(j + R2 * m)];
      dft<R1, +1>(v);
#pragma unroll
      for (int q = 0; q < R1; ++q) row[P::phys(j + R2 * q)] = v[q];
    }
    if constexpr (R1 == R2) {  // the same lanes' packed row, as in the forward rows
      __syncwarp();
    } else {
      __syncthreads();
    }

    // ---- inverse row pass B -> surface (kept in place), argmax ---------------
    // the surface stays in place (re: row y1, im: row y2 of each packed line);
    // the SNR pass below reads it back instead of holding it across barriers
    // running maxima of the y1 rows and of the y2 rows: each thread meets
    // either set in increasing row-major index, so a strict '>' keeps the
    // smallest index among equal values (initial index: the thread's first
    // pixel of each set); one argmax key per set at the end
    float bva = -INFINITY, bvb = -INFINITY;
    uint32_t bia = static_cast<uint32_t>((rank * ROWS + tid / R1) * N + tid % R1), bib = bia + HALF * N;
#pragma unroll
    for (int i = 0; i < P::KBh; ++i) {
      const int task = tid + i * T;
      const bool valid = (P::TBh % T == 0) || task < P::TBh;
      const int line = task / R1, k1 = task % R1;
      if (valid) {
        float2* row = slab + line * RS;
        float2 sv[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
          float2 x = row[P::phys(R2 * k1 + n2)];
          sv[n2] = n2 == 0 ? x : cmulc(x, twid[n2 * R1 + k1]);
        }
        dft<R2, +1>(sv);  // sv[k2] = s at x = k1 + R1 k2
        const int y1 = rank * ROWS + line, y2 = y1 + HALF;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          row[P::phys(R2 * k1 + k2)] = sv[k2];
          const int x = k1 + R1 * k2;
          if (sv[k2].x > bva) {
            bva = sv[k2].x;
            bia = static_cast<uint32_t>(y1 * N + x);
          }
          if (sv[k2].y > bvb) {
            bvb = sv[k2].y;
            bib = static_cast<uint32_t>(y2 * N + x);
          }
        }
      }
    }
    unsigned long long best = 0ull;
    if ((P::TBh % T == 0) || tid < P::TBh) {  // threads without a task hold no pixel
      const unsigned long long ka = argmax_key(bva, bia), kb = argmax_key(bvb, bib);
      best = ka > kb ? ka : kb;
    }
    best = warp_max_u64(best);
    if (lane == 0) sc->wkey[warp] = best;
    __syncthreads();
    if (warp == 0) {
      unsigned long long bk = warp_max_u64(lane < NW ? sc->wkey[lane] : 0ull);
      if (lane < C) st_cl_u64<C>(map_rank<C>(smem_addr(&sc->ckey[rank]), lane), bk);
    }
    cluster_barrier<C>();
    unsigned long long gk = 0ull;
#pragma unroll
    for (int r = 0; r < C; ++r) gk = sc->ckey[r] > gk ? sc->ckey[r] : gk;
    const uint32_t pidx = key_index(gk);
    const int py = static_cast<int>(pidx / N), px = static_cast<int>(pidx % N);

    // ---- SNR background partials (outside the exclusion disc) ---------------
    {
      float s1 = 0.f, s2 = 0.f;
      int cnt = 0;
#pragma unroll
      for (int i = 0; i < P::KBh; ++i) {
        const int task = tid + i * T;
        const bool valid = (P::TBh % T == 0) || task < P::TBh;
        const int line = task / R1, k1 = task % R1;
        if (valid) {
          int dya = abs(static_cast<int>(rank * ROWS + line) - py);
          dya = min(dya, N - dya);
          int dyb = abs(static_cast<int>(rank * ROWS + line + HALF) - py);
          dyb = min(dyb, N - dyb);
          const float2* row = slab + line * RS;
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) {
            const int x = k1 + R1 * k2;
            int dx = abs(x - px);
            dx = min(dx, N - dx);
            const float2 sab = row[P::phys(R2 * k1 + k2)];
            const float sa = sab.x, sb = sab.y;
            if (static_cast<float>(dya * dya + dx * dx) > L.radius2) {
              s1 += sa;
              s2 = fmaf(sa, sa, s2);
              ++cnt;
            }
            if (static_cast<float>(dyb * dyb + dx * dx) > L.radius2) {
              s1 += sb;
              s2 = fmaf(sb, sb, s2);
              ++cnt;
            }
          }
        }
      }
      // float-pair warp sums (FP32 instructions only), integer counts
      float a1 = s1, e1 = 0.f, a2 = s2, e2 = 0.f;
      warp_sum_ff2(a1, e1);
      warp_sum_ff2(a2, e2);
      const int nw = __reduce_add_sync(0xffffffffu, cnt);
      if (lane == 0) {
        sc->wbg[warp][0] = a1;
        sc->wbg[warp][1] = e1;
        sc->wbg[warp][2] = a2;
        sc->wbg[warp][3] = e2;
        sc->wcnt[warp] = nw;
      }
    }
    __syncthreads();
    if (warp == 0) {
      float a1 = lane < NW ? sc->wbg[lane][0] : 0.f, e1 = lane < NW ? sc->wbg[lane][1] : 0.f;
      float a2 = lane < NW ? sc->wbg[lane][2] : 0.f, e2 = lane < NW ? sc->wbg[lane][3] : 0.f;
      warp_sum_ff2(a1, e1);
      warp_sum_ff2(a2, e2);
      const int nc = __reduce_add_sync(0xffffffffu, lane < NW ? sc->wcnt[lane] : 0);
      const double a = static_cast<double>(a1) + static_cast<double>(e1);
      const double c = static_cast<double>(a2) + static_cast<double>(e2);
      const double n = static_cast<double>(nc);
      if (lane == 0) {
        const uint32_t dst = map_rank<C>(smem_addr(&sc->cbg[rank][0]), 0);
        st_cl_f64<C>(dst, a);
        st_cl_f64<C>(dst + 8, c);
        st_cl_f64<C>(dst + 16, n);
      }
      // peak neighbours held by this CTA go to rank 0 (lanes 0..3: y-1, y+1, x-1, x+1)
      if (lane < 4) {
        const int yk = lane == 0 ? ((py + N - 1) & (N - 1)) : (lane == 1 ? ((py + 1) & (N - 1)) : py);
        const int xk = lane == 2 ? ((px + N - 1) & (N - 1)) : (lane == 3 ? ((px + 1) & (N - 1)) : px);
        if (yk / ROWS == static_cast<int>(rank)) {
          const int yl = yk % ROWS;
          const float2 e = slab[(yl % HALF) * RS + P::phys(P::rho(xk))];
          st_cl_f32<C>(map_rank<C>(smem_addr(&sc->nb[lane]), 0), yl < HALF ? e.x : e.y);
        }
      }
    }
    cluster_barrier<C>();
    if (rank == 0 && tid == 0) {
      double a = 0, c = 0, n = 0;
      for (int r = 0; r < C; ++r) {
        a += sc->cbg[r][0];
        c += sc->cbg[r][1];
        n += sc->cbg[r][2];
      }
      swift_result r = window_result(N, py, px, key_value(gk), a, c, n, sc->nb);
      if (sc->broken) r.status = SWIFT_WIN_TIMEOUT;
      *out = r;
    }
    cur ^= 1;
  }
  if constexpr (BULK) {
    // a staged load that timed out may still be in flight: wait for it (bounded)
    if (sc->broken) mbar_wait_bounded(mbar, parity);
  }
}

}  // namespace swift
