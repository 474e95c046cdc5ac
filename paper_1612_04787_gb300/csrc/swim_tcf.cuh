// Tensor-core precision variant: every 1D transform is a 256- or 128-point
// DFT computed by one warp with the four-step factorisation n = 16 * Q
// (Q = 16 or 8):
//
//   x[Q n1 + n2]  --(16-point DFT over n1: tensor-core product F16 . x)-->
//   Y[k1][n2]     --(twiddle W_n^{k1 n2}, FP32)-->
//   Y'[k1][n2]    --(Q-point DFT over n2: tensor-core product Y' . F_Q)-->
//   X[k1 + 16 k2]
//
// Both products are mma.sync m16n8k16 with complex numbers written as real
// 2x2 blocks ([[Re, -Im], [Im, Re]]), BF16 or FP16 operands and FP32
// accumulation.  Each FP32 operand x is split into hi = round16(x) and
// lo = round16(x - hi) and a product is accumulated as lo*hi + hi*lo + hi*hi
// (lo*lo lies below FP32 rounding of the sum).  The accumulator fragment of
// the first product has exactly the register layout of the A operand of the
// second, so a transform never leaves the registers; the DFT-matrix operand
// of the second product is the transpose of the first's and reuses its
// fragments.  The inverse transform is conj(DFT(conj(x))).
//
// FP16 has a narrow exponent range: each transform first finds the largest
// magnitude of its input (warp reduction) and scales the input by the power
// of two that puts it in [2^14, 2^15); the 16-point stage's output is scaled
// by 1/16 before it is split again; the epilogue removes both exactly.  BF16
// shares FP32's exponent range and is not scaled.
//
// The streaming schedule around the transforms (Sec. III steps):
//   K0 stats     the FP32 path's statistics kernel (bounds, flat/non-finite,
//                taper-weighted means)
//   T1 rows      apodise z = m' + i r' row by row, row DFT, transpose through
//                shared memory -> Zt[kx][y]
//   T2 columns   one warp per column pair (kx, n - kx): two column DFTs,
//                Hermitian unpack of M and R, C = M conj(R), whitening,
//                inverse column DFT -> Ht[kx][y] (kx = 0 carries kx = n/2 as
//                its imaginary part)
//   T3 inv rows  rows y and y + n/2 as one complex row (Hermitian completion),
//                inverse row DFT -> response s; argmax and FP64 block sums
//   K4 finalize  the FP32 path's SNR / subpixel kernel
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "swim_stream.cuh"

namespace swift {

// resident CTAs per SM each kernel is compiled for (its register cap),
// measured per kernel: the 256-point row kernel runs faster unspilled at 2,
// everything else at 3
template <int N, bool ROWS>
constexpr int tcf_minb() {
  return (N == 256 && ROWS) ? 2 : 3;
}

constexpr int kTcfFragRegs = 40;  // per lane: F16 A fragments hi (16) + lo (16), F8 B fragments hi (4) + lo (4)

template <int N>
struct TcfGeom {
  static constexpr int Q = N / 16;     // second factor
  static constexpr int NT1 = Q / 8;    // n-tiles of the first product (n2 = g + 8 j)
  static constexpr int S = 4 * NT1;    // complex values per lane
  static constexpr int NT3 = Q / 4;    // n-tiles of the second product
  static constexpr int KS3 = Q / 8;    // k-steps of the second product
  static_assert(N == 128 || N == 256, "tensor-core DFT sizes");
};

// lane (g, t) = (lane / 4, lane % 4).  Input slot c + 4 j holds
// x[Q n1 + n2] with n1 = 2t + {0, 1, 8, 9}[c], n2 = g + 8 j; output slot
// q + 4 j (q = 2 h + e) holds X[k1 + 16 k2] with k1 = g + 8 h, k2 = 8 j + 2 t + e.
template <int N>
__device__ __forceinline__ int tcf_in_index(int lane, int slot) {
  const int g = lane >> 2, t = lane & 3, c = slot & 3, j = slot >> 2;
  return TcfGeom<N>::Q * (2 * t + (c & 1) + 8 * (c >> 1)) + g + 8 * j;
}
template <int N>
__device__ __forceinline__ int tcf_out_index(int lane, int slot) {
  const int g = lane >> 2, t = lane & 3, q = slot & 3, j = slot >> 2;
  return (g + 8 * (q >> 1)) + 16 * (8 * j + 2 * t + (q & 1));
}

// 4-bit XOR swizzle for shared-memory tiles indexed by a transform index k:
// within one warp access the lanes' (g mod 4, t) give 16 distinct values
__device__ __forceinline__ int tcf_swz(int k) { return (k & 3) | ((((k >> 5) ^ (k >> 4)) & 3) << 2); }
// bijective position of element k of a length-n vector in shared memory
__device__ __forceinline__ int tcf_vpos(int k) { return k ^ ((((k >> 5) ^ (k >> 4)) & 3) << 2); }

template <bool FP16>
__device__ __forceinline__ void tcf_split(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  if constexpr (FP16) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}

template <bool FP16>
__device__ __forceinline__ void tcf_mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                        uint32_t b0, uint32_t b1) {
  if constexpr (FP16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
}

// One warp's n-point DFT engine.  The constant fragments live in shared
// memory (copied once per CTA, [10][32] uint4: lane-contiguous, so a warp's
// 16-byte reads are conflict-free) and the twiddles are read through L1;
// registers hold only the data.
constexpr int kTcfFragVecs = kTcfFragRegs / 4;  // uint4 per lane

// copy the per-lane fragments of global layout [32][40] to shared [10][32] uint4
__device__ __forceinline__ void tcf_stage_frags(const uint32_t* frag, uint4* sfrag, int tid, int nthreads) {
  for (int e = tid; e < 32 * kTcfFragVecs; e += nthreads) {
    const int lane = e / kTcfFragVecs, v = e % kTcfFragVecs;
    sfrag[v * 32 + lane] = __ldg(reinterpret_cast<const uint4*>(frag + lane * kTcfFragRegs) + v);
  }
}

template <int N, bool FP16>
struct WarpDft {
  using G = TcfGeom<N>;
  const uint4* sf;   // shared [10][32]: 0-3 F16 hi (index 2 mt + ks), 4-7 F16 lo, 8 F8 hi, 9 F8 lo
  const float2* tw;  // global twiddle table W_n^m
  int lane;

  __device__ __forceinline__ void load(const TcfLaunch& T, const uint4* sfrag, int ln) {
    sf = sfrag;
    tw = T.tw;
    lane = ln;
  }
  __device__ __forceinline__ uint4 frag(int v) const { return sf[v * 32 + lane]; }

  // In place: x holds the input slots on entry and the output slots on exit.
  // DIR = -1: forward exp(-2 pi i k x / n); DIR = +1: unnormalised inverse.
  template <int DIR>
  __device__ __forceinline__ void run(float2 (&x)[G::S]) const {
    constexpr float cj = DIR > 0 ? -1.0f : 1.0f;
    float sc = 1.0f, inv = 1.0f;
    if constexpr (FP16) {
      float m = 0.f;
#pragma unroll
      for (int s = 0; s < G::S; ++s) m = fmaxf(m, fmaxf(fabsf(x[s].x), fabsf(x[s].y)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (m > 0.f && m <= 3.4e38f) {
        const int e = ((__float_as_int(m) >> 23) & 0xff) - 127;
        const int p = max(-100, min(100, 14 - e));
        sc = __int_as_float((p + 127) << 23);
        inv = __int_as_float((4 - p + 127) << 23);  // 16 / sc
      }
    }
    // first product: D1[(mt, k1)][n2] = sum_(ks, n1) F16big[(mt, k1)][(ks, n1)] x[(ks, n1)][n2]
    // (the data operand is split once per (j, ks); each constant fragment is
    // read from shared memory once per transform)
    uint32_t bsp[G::NT1][2][4];  // hi0, hi1, lo0, lo1
#pragma unroll
    for (int j = 0; j < G::NT1; ++j)
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        float v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = (ks == 0 ? x[c + 4 * j].x : cj * x[c + 4 * j].y) * sc;
        tcf_split<FP16>(v[0], v[1], bsp[j][ks][0], bsp[j][ks][2]);
        tcf_split<FP16>(v[2], v[3], bsp[j][ks][1], bsp[j][ks][3]);
      }
    float d1[2][G::NT1][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int j = 0; j < G::NT1; ++j) d1[mt][j][0] = d1[mt][j][1] = d1[mt][j][2] = d1[mt][j][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const uint4 ah = frag(2 * mt + ks), al = frag(4 + 2 * mt + ks);
#pragma unroll
        for (int j = 0; j < G::NT1; ++j) {
          tcf_mma<FP16>(d1[mt][j], al.x, al.y, al.z, al.w, bsp[j][ks][0], bsp[j][ks][1]);
          tcf_mma<FP16>(d1[mt][j], ah.x, ah.y, ah.z, ah.w, bsp[j][ks][2], bsp[j][ks][3]);
          tcf_mma<FP16>(d1[mt][j], ah.x, ah.y, ah.z, ah.w, bsp[j][ks][0], bsp[j][ks][1]);
        }
      }
    // twiddles (and the FP16 stage scale)
    constexpr float s16 = FP16 ? 0.0625f : 1.0f;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < G::NT1; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float yr = d1[0][j][q] * s16, yi = d1[1][j][q] * s16;
        const int k1 = g + 8 * (q >> 1), n2 = 8 * j + 2 * t + (q & 1);
        const float2 w = __ldg(tw + ((k1 * n2) & (N - 1)));
        d1[0][j][q] = fmaf(yr, w.x, -yi * w.y);
        d1[1][j][q] = fmaf(yr, w.y, yi * w.x);
      }
    // second product: X[k1][(c', k2)] = sum_(c, n2) Y'[k1][(c, n2)] FQbig[(c, n2)][(c', k2)]
    float d3[G::NT3][4];
#pragma unroll
    for (int n = 0; n < G::NT3; ++n) d3[n][0] = d3[n][1] = d3[n][2] = d3[n][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < G::KS3; ++ks) {
      uint32_t ah[4], al[4];
      if constexpr (G::Q == 16) {  // k-step ks covers part ks (re / im) of n2 = 0..15
        tcf_split<FP16>(d1[ks][0][0], d1[ks][0][1], ah[0], al[0]);
        tcf_split<FP16>(d1[ks][0][2], d1[ks][0][3], ah[1], al[1]);
        tcf_split<FP16>(d1[ks][1][0], d1[ks][1][1], ah[2], al[2]);
        tcf_split<FP16>(d1[ks][1][2], d1[ks][1][3], ah[3], al[3]);
      } else {  // one k-step: re n2 = 0..7, then im n2 = 0..7
        tcf_split<FP16>(d1[0][0][0], d1[0][0][1], ah[0], al[0]);
        tcf_split<FP16>(d1[0][0][2], d1[0][0][3], ah[1], al[1]);
        tcf_split<FP16>(d1[1][0][0], d1[1][0][1], ah[2], al[2]);
        tcf_split<FP16>(d1[1][0][2], d1[1][0][3], ah[3], al[3]);
      }
      // B fragments: F16big^T (Q = 16; fragment (ks, n = 2 mt + h) = A fragment
      // (mt, ks) registers h, 2 + h) or F8big; each read once per k-step
      uint4 fh[(G::NT3 + 1) / 2], fl[(G::NT3 + 1) / 2];
#pragma unroll
      for (int p = 0; p < (G::NT3 + 1) / 2; ++p) {
        fh[p] = G::Q == 16 ? frag(2 * p + ks) : frag(8);
        fl[p] = G::Q == 16 ? frag(4 + 2 * p + ks) : frag(9);
      }
#pragma unroll
      for (int n = 0; n < G::NT3; ++n) {
        uint32_t bh0, bh1, bl0, bl1;
        if constexpr (G::Q == 16) {
          const uint4 h4 = fh[n >> 1], l4 = fl[n >> 1];
          bh0 = (n & 1) ? h4.y : h4.x;
          bh1 = (n & 1) ? h4.w : h4.z;
          bl0 = (n & 1) ? l4.y : l4.x;
          bl1 = (n & 1) ? l4.w : l4.z;
        } else {
          const uint4 gh = fh[0], gl = fl[0];
          bh0 = n ? gh.z : gh.x;
          bh1 = n ? gh.w : gh.y;
          bl0 = n ? gl.z : gl.x;
          bl1 = n ? gl.w : gl.y;
        }
        tcf_mma<FP16>(d3[n], al[0], al[1], al[2], al[3], bh0, bh1);
        tcf_mma<FP16>(d3[n], ah[0], ah[1], ah[2], ah[3], bl0, bl1);
        tcf_mma<FP16>(d3[n], ah[0], ah[1], ah[2], ah[3], bh0, bh1);
      }
    }
#pragma unroll
    for (int j = 0; j < G::NT1; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q + 4 * j] = make_float2(d3[j][q] * inv, cj * d3[j + G::NT1][q] * inv);
  }
};

// ---------------------------------------------------------------------------
// T1: rows.  CTA = 8 warps x 2 rows.  The CTA's 16 rows of both windows are
// staged in shared memory first (16-byte vector loads when aligned; the
// reference of a K-section model is averaged into a float stage), then each
// warp transforms its rows; the spectra leave through a shared-memory
// transpose as Zt[s][kx][y].
// ---------------------------------------------------------------------------
constexpr int kTcfRowsPerCta = 16;

// position of pixel x in a staged float row: XOR on bits 3-4 by bits 5-6 so
// that the four lane groups of a DFT input read (x = 32 t + ...) hit
// different banks; 4-aligned groups stay contiguous
template <typename TIn>
__device__ __forceinline__ int tcf_stage_pos(int x) {
  if constexpr (sizeof(TIn) == 1) return x;
  return x ^ (((x >> 5) & 3) << 3);
}

template <int N, typename TIn>
constexpr size_t tcf_rows_smem() {
  constexpr int RT = kTcfRowsPerCta;
  return sizeof(float2) * N * RT + sizeof(float) * N + sizeof(TIn) * RT * N + sizeof(float) * RT * N;
}

template <int N, bool FP16, typename TIn>
__global__ void __launch_bounds__(256, tcf_minb<N, true>()) tcf_rows_kernel(const MatchLaunch L, const StreamWork W, const TcfLaunch T) {
  using G = TcfGeom<N>;
  constexpr int RT = kTcfRowsPerCta;
  const long long s = blockIdx.x / (N / RT);
  const int rb = blockIdx.x % (N / RT);
  const long long b = W.b0 + s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float4 st = W.stats[s];
  if (stat_status(st) != SWIFT_WIN_OK) return;
  {
    const int guard = launch_window_check(L, b, N);  // level and bounds from the launch's arrays
    if (guard != SWIFT_WIN_OK) {
      if (tid == 0) W.stats[s] = make_float4(0.f, 0.f, __int_as_float(guard), 0.f);
      return;
    }
  }
  extern __shared__ __align__(16) unsigned char tcf_smem[];
  float2* tile = reinterpret_cast<float2*>(tcf_smem);  // [N][RT], swizzled columns
  float* tap = reinterpret_cast<float*>(tile + N * RT);
  TIn* mstage = reinterpret_cast<TIn*>(tap + N);       // [RT][N]
  float* rstage = reinterpret_cast<float*>(mstage + RT * N);  // [RT][N] (float reference)
  TIn* rstage_t = reinterpret_cast<TIn*>(rstage);             // [RT][N] (reference as TIn)
  for (int i = tid; i < N; i += 256) tap[i] = L.taper[i];
  const TIn* mbase;
  const TIn* rbase;
  long long mpitch, rpitch;
  if (L.patch_mode) {
    mbase = static_cast<const TIn*>(L.mov) + b * L.mov_stride;
    rbase = static_cast<const TIn*>(L.ref) + b * L.ref_stride;
    mpitch = rpitch = N;
  } else {
    mbase = static_cast<const TIn*>(L.mov) + static_cast<long long>(__ldg(L.mov_origin + 2 * b)) * L.mov_pitch +
            __ldg(L.mov_origin + 2 * b + 1);
    rbase = static_cast<const TIn*>(L.ref) + static_cast<long long>(__ldg(L.ref_origin + 2 * b)) * L.ref_pitch +
            __ldg(L.ref_origin + 2 * b + 1);
    mpitch = L.mov_pitch;
    rpitch = L.ref_pitch;
  }
  mbase += static_cast<long long>(rb * RT) * mpitch;
  rbase += static_cast<long long>(rb * RT) * rpitch;
  constexpr int VEC = 16 / static_cast<int>(sizeof(TIn));
  const bool vec = L.ref_count == 1 && ((reinterpret_cast<uintptr_t>(mbase) | reinterpret_cast<uintptr_t>(rbase) |
                                         static_cast<uintptr_t>(mpitch * sizeof(TIn)) |
                                         static_cast<uintptr_t>(rpitch * sizeof(TIn))) & 15) == 0;
  if (vec) {
    constexpr int NV = RT * N / VEC;
    constexpr int IT = (NV + 255) / 256;
    uint4 q[2 * IT];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      const int e = tid + 256 * i;
      if (NV % 256 == 0 || e < NV) {
        const int r = e / (N / VEC), x0 = (e % (N / VEC)) * VEC;
        q[2 * i] = __ldg(reinterpret_cast<const uint4*>(mbase + r * mpitch + x0));
        q[2 * i + 1] = __ldg(reinterpret_cast<const uint4*>(rbase + r * rpitch + x0));
      }
    }
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      const int e = tid + 256 * i;
      if (NV % 256 == 0 || e < NV) {
        const int r = e / (N / VEC), x0 = (e % (N / VEC)) * VEC;
        const int p = r * N + tcf_stage_pos<TIn>(x0);
        *reinterpret_cast<uint4*>(mstage + p) = q[2 * i];
        *reinterpret_cast<uint4*>(rstage_t + p) = q[2 * i + 1];
      }
    }
  } else {
    const float inv_k = 1.0f / static_cast<float>(L.ref_count);
    for (int e = tid; e < RT * N; e += 256) {
      const int r = e / N, x = e % N;
      mstage[r * N + tcf_stage_pos<TIn>(x)] = __ldg(mbase + r * mpitch + x);
      float rv = load_px<TIn>(rbase + r * rpitch + x);
      if (L.ref_count > 1) {
        for (int k = 1; k < L.ref_count; ++k) rv += load_px<TIn>(rbase + k * L.ref_stride + r * rpitch + x);
        rv *= inv_k;
      }
      rstage[r * N + tcf_stage_pos<float>(x)] = rv;
    }
  }
  __shared__ uint4 sfrag[kTcfFragVecs * 32];
  tcf_stage_frags(T.frag, sfrag, tid, 256);
  WarpDft<N, FP16> dft;
  dft.load(T, sfrag, lane);
  __syncthreads();
#pragma unroll 1
  for (int r = 0; r < 2; ++r) {
    const int yl = 2 * warp + r;
    const float ay = tap[rb * RT + yl];
    float2 x[G::S];
#pragma unroll
    for (int sl = 0; sl < G::S; ++sl) {
      const int xi = tcf_in_index<N>(lane, sl);
      const float mv = static_cast<float>(mstage[yl * N + tcf_stage_pos<TIn>(xi)]);
      const float rv = vec ? static_cast<float>(rstage_t[yl * N + tcf_stage_pos<TIn>(xi)])
                           : rstage[yl * N + tcf_stage_pos<float>(xi)];
      const float a = ay * tap[xi];
      x[sl] = make_float2(a * (mv - st.x), a * (rv - st.y));
    }
    dft.template run<-1>(x);
#pragma unroll
    for (int sl = 0; sl < G::S; ++sl) {
      const int k = tcf_out_index<N>(lane, sl);
      tile[k * RT + (yl ^ tcf_swz(k))] = x[sl];
    }
  }
  __syncthreads();
  float2* zt = W.zr + static_cast<long long>(s) * N * N + rb * RT;
#pragma unroll 4
  for (int e = tid; e < N * RT; e += 256) {
    const int k = e / RT, yl = e % RT;
    __stcg(zt + static_cast<long long>(k) * N + yl, tile[k * RT + (yl ^ tcf_swz(k))]);
  }
}

// ---------------------------------------------------------------------------
// T2: columns.  One warp per column pair (kx, n - kx); kx = 0 pairs with n/2.
// ---------------------------------------------------------------------------
template <int N, bool FP16>
__global__ void __launch_bounds__(256, tcf_minb<N, false>()) tcf_cols_kernel(const MatchLaunch L, const StreamWork W, const TcfLaunch T) {
  using G = TcfGeom<N>;
  const long long s = blockIdx.x / (N / 16);
  const int cb = blockIdx.x % (N / 16);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (stat_status(W.stats[s]) != SWIFT_WIN_OK) return;
  __shared__ __align__(16) float2 vec[8][2][N];
  __shared__ uint4 sfrag[kTcfFragVecs * 32];
  tcf_stage_frags(T.frag, sfrag, tid, 256);
  WarpDft<N, FP16> dft;
  dft.load(T, sfrag, lane);
  const int kx = cb * 8 + warp;  // in [0, n/2)
  const int ka = kx, kb = kx == 0 ? N / 2 : N - kx;
  const float2* zt = W.zr + static_cast<long long>(s) * N * N;
  float2* va = vec[warp][0];
  float2* vb = vec[warp][1];
  // forward column transforms of columns ka and kb
  __syncthreads();  // fragments staged
#pragma unroll 1
  for (int c = 0; c < 2; ++c) {
    const int kc = c == 0 ? ka : kb;
    float2* v = c == 0 ? va : vb;
    float2 x[G::S];
#pragma unroll
    for (int sl = 0; sl < G::S; ++sl) x[sl] = __ldcs(zt + static_cast<long long>(kc) * N + tcf_in_index<N>(lane, sl));
    dft.template run<-1>(x);
#pragma unroll
    for (int sl = 0; sl < G::S; ++sl) v[tcf_vpos(tcf_out_index<N>(lane, sl))] = x[sl];
  }
  __syncwarp();
  // unpack C = M conj(R) = (Im(a b) / 2, (|a|^2 - |b|^2) / 4), a = Z[k], b = Z[-k]; whitening
  const float half_w = -0.5f * L.w;
  const float inv_n2 = 1.0f / (static_cast<float>(N) * static_cast<float>(N));
  auto whiten = [&](float2 a, float2 bb, bool dc) -> float2 {
    const float2 c = make_float2(0.5f * fmaf(a.x, bb.y, a.y * bb.x),
                                 0.25f * ((a.x * a.x + a.y * a.y) - (bb.x * bb.x + bb.y * bb.y)));
    const float mag2 = fmaf(c.x, c.x, c.y * c.y);
    float sc = whiten_factor(mag2, half_w) * inv_n2;
    if (dc) sc = 0.f;  // G[0][0] = 0
    return make_float2(c.x * sc, c.y * sc);
  };
  float2 x[G::S];
#pragma unroll
  for (int sl = 0; sl < G::S; ++sl) {
    const int ky = tcf_in_index<N>(lane, sl);
    const int my = (N - ky) & (N - 1);
    if (kx != 0) {
      x[sl] = whiten(va[tcf_vpos(ky)], vb[tcf_vpos(my)], false);
    } else {  // real columns 0 and n/2 packed: G0 + i G_{n/2}
      const float2 g0 = whiten(va[tcf_vpos(ky)], va[tcf_vpos(my)], ky == 0);
      const float2 g1 = whiten(vb[tcf_vpos(ky)], vb[tcf_vpos(my)], false);
      x[sl] = make_float2(g0.x - g1.y, g0.y + g1.x);
    }
  }
  dft.template run<1>(x);
  float2* ht = W.h + (static_cast<long long>(s) * (N / 2) + kx) * N;
#pragma unroll
  for (int sl = 0; sl < G::S; ++sl) __stcg(ht + tcf_out_index<N>(lane, sl), x[sl]);
}

// ---------------------------------------------------------------------------
// T3: inverse rows.  CTA = 8 warps, PB row pairs (y, y + n/2); block argmax
// and FP64 sums in the streaming finalize kernel's partial layout.
// ---------------------------------------------------------------------------
template <int N, bool FP16>
__global__ void __launch_bounds__(256, tcf_minb<N, false>()) tcf_irows_kernel(const MatchLaunch L, const StreamWork W, const TcfLaunch T) {
  using G = TcfGeom<N>;
  constexpr int PB = StreamGeom<N>::PB, NB3 = StreamGeom<N>::NB3;
  constexpr int CW = 2 * PB;  // tile columns: y0 + [0, PB) and y0 + n/2 + [0, PB)
  constexpr int PPW = PB / 8;
  static_assert(PB % 8 == 0 && NB3 * PB == N / 2, "row pairs");
  const long long s = blockIdx.x / NB3;
  const int blk = blockIdx.x % NB3;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (stat_status(W.stats[s]) != SWIFT_WIN_OK) return;
  __shared__ __align__(16) float2 tile[(N / 2) * CW];
  __shared__ unsigned long long wk[8];
  __shared__ double ws[8][2];
  __shared__ uint4 sfrag[kTcfFragVecs * 32];
  tcf_stage_frags(T.frag, sfrag, tid, 256);
  WarpDft<N, FP16> dft;
  dft.load(T, sfrag, lane);
  const int y0 = blk * PB;
  const float2* ht = W.h + static_cast<long long>(s) * (N / 2) * N;
#pragma unroll 4
  for (int e = tid; e < (N / 2) * CW; e += 256) {
    const int kx = e / CW, c = e % CW;
    const int y = c < PB ? y0 + c : y0 + N / 2 + (c - PB);
    tile[kx * CW + (c ^ tcf_swz(kx))] = __ldcs(ht + static_cast<long long>(kx) * N + y);
  }
  __syncthreads();
  float* surf = reinterpret_cast<float*>(W.zr + static_cast<long long>(s) * N * N);
  unsigned long long best = 0ull;
  float s1 = 0.f, s2 = 0.f;
#pragma unroll 1
  for (int p = 0; p < PPW; ++p) {
    const int pr = warp * PPW + p;
    const int ca = pr, cbb = PB + pr;
    const int y = y0 + pr, y2 = y + N / 2;
    float2 x[G::S];
#pragma unroll
    for (int sl = 0; sl < G::S; ++sl) {
      const int k = tcf_in_index<N>(lane, sl);
      float2 v;
      if (k == 0 || k == N / 2) {
        const float2 u = tile[ca ^ tcf_swz(0)], w = tile[cbb ^ tcf_swz(0)];
        v = k == 0 ? make_float2(u.x, w.x) : make_float2(u.y, w.y);
      } else if (k < N / 2) {  // P = H_y + i H_y2
        const float2 u = tile[k * CW + (ca ^ tcf_swz(k))], w = tile[k * CW + (cbb ^ tcf_swz(k))];
        v = make_float2(u.x - w.y, u.y + w.x);
      } else {  // Hermitian completion: H_y[k] = conj(H_y[n - k])
        const int m = N - k;
        const float2 u = tile[m * CW + (ca ^ tcf_swz(m))], w = tile[m * CW + (cbb ^ tcf_swz(m))];
        v = make_float2(u.x + w.y, w.x - u.y);
      }
      x[sl] = v;
    }
    dft.template run<1>(x);
#pragma unroll
    for (int sl = 0; sl < G::S; ++sl) {
      const int xo = tcf_out_index<N>(lane, sl);
      const float va = x[sl].x, vb = x[sl].y;
      const unsigned long long ka = argmax_key(va, static_cast<uint32_t>(y * N + xo));
      const unsigned long long kb = argmax_key(vb, static_cast<uint32_t>(y2 * N + xo));
      best = ka > best ? ka : best;
      best = kb > best ? kb : best;
      s1 += va + vb;
      s2 = fmaf(va, va, fmaf(vb, vb, s2));
      surf[y * N + xo] = va;
      surf[y2 * N + xo] = vb;
    }
  }
  best = warp_max_u64(best);
  const double d1 = warp_sum_f64(static_cast<double>(s1)), d2 = warp_sum_f64(static_cast<double>(s2));
  if (lane == 0) {
    wk[warp] = best;
    ws[warp][0] = d1;
    ws[warp][1] = d2;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long k = 0ull;
    double a = 0.0, c = 0.0;
    for (int v = 0; v < 8; ++v) {
      k = wk[v] > k ? wk[v] : k;
      a += ws[v][0];
      c += ws[v][1];
    }
    unsigned long long* part = W.part + 3 * (s * NB3 + blk);
    part[0] = k;
    part[1] = static_cast<unsigned long long>(__double_as_longlong(a));
    part[2] = static_cast<unsigned long long>(__double_as_longlong(c));
  }
}

}  // namespace swift
