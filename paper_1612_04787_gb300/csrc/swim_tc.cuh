// Tensor-core precision variant: every 1D transform of the match as a batched
// DFT-matrix GEMM on the tensor cores (mma.sync m16n8k16, BF16 or FP16
// operands, FP32 accumulation), with split-precision compensation: each FP32
// operand x is split into hi = round(x) and lo = round(x - hi), and a product
// is accumulated as hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32
// rounding of the result).
//
// Complex data is kept planar ([re plane][im plane]) so each transform is a
// plain real GEMM with a 2n x 2n block DFT matrix:
//   rows     Zr[(c', y)][kx] = sum_{c, x} z[c][y][x] Wr[(c, x)][(c', kx)]
//   columns  Z[(c', ky)][x]  = sum_{c, y} Wc[(c', ky)][(c, y)] Zr[c][y][x]
//   (the inverse transforms use the conjugate matrices; the last one keeps
//   only the real part, n output columns)
// with Wr[(re, x)][(re, kx)] = cos, Wr[(im, x)][(re, kx)] = -s, ... for the
// forward e^{-2 pi i k x / n} (s = sin 2 pi k x / n).  Statistics, peak, SNR
// and subpixel fit reuse the streaming kernels (FP64 accumulation).
//
// FP16 has a narrow exponent range, so in that mode each CTA first finds the
// largest magnitude of its slab of the data operand (the matrix entries are
// bounded by 1) and scales the slab by the power of two that puts it in
// [2^14, 2^15); the epilogue removes the scale exactly.  BF16 shares FP32's
// exponent range and is not scaled.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "swim_stream.cuh"

namespace swift {

enum TcMat : int { TC_WR = 0, TC_WC = 1, TC_WRI = 2, TC_WCI = 3 };

// ---------------------------------------------------------------------------
// split an FP32 pair into (hi, lo) pairs of 16-bit floats, packed in .b32
// ---------------------------------------------------------------------------
template <bool FP16>
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
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
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  if constexpr (FP16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
}

// ---------------------------------------------------------------------------
// The batched GEMM.  CTA tile 64 x 64 outputs, 4 warps of 32 x 32, K step 32.
// MODE selects the operands of each transform (see the header comment):
//   0 rows:    A = apodised window z (M = n rows y, K = 2n (c, x)), B = Wr (2n x 2n)
//   1 columns: A = Wc (2n x 2n), B = data (K = 2n rows (c, y), N = n columns x)
//   2 inverse columns: as 1 with Wc* ([WCI])
//   3 inverse rows:    A = data (M = n rows y, K = 2n (c, kx)), B = Wri (2n x n), real part only
// ---------------------------------------------------------------------------

template <int N, int MODE, bool FP16, typename TIn>
__global__ void __launch_bounds__(128) tc_gemm_kernel(const MatchLaunch L, const TcLaunch T) {
  constexpr int K = 2 * N;
  constexpr int M = (MODE == 1 || MODE == 2) ? 2 * N : N;
  constexpr int NO = (MODE == 0) ? 2 * N : N;
  constexpr int TM = M / 64, TN = NO / 64;
  constexpr int BK = 32;
  const long long s = blockIdx.x / (TM * TN);
  const int tile = blockIdx.x % (TM * TN);
  const int m0 = (tile / TN) * 64, n0 = (tile % TN) * 64;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const float4 st = T.stats[s];
  if (stat_status(st) != SWIFT_WIN_OK) return;
  __shared__ float As[64][BK + 2];  // [m][k]
  __shared__ float Bs[64][BK + 2];  // [n][k] (transposed: k contiguous)
  __shared__ float tap[N];
  const long long b = T.b0 + s;  // window of the batch
  const float* mats = T.mats;
  const float* W = mats + static_cast<size_t>(MODE == 0 ? TC_WR : (MODE == 1 ? TC_WC : (MODE == 2 ? TC_WCI : TC_WRI))) * K * K;
  // forward columns and inverse columns read x0; inverse rows read x1
  const float* in = (MODE == 1 || MODE == 2) ? T.x0 + s * 2 * N * N : T.x1 + s * 2 * N * N;
  if (MODE == 0) {
    for (int i = tid; i < N; i += 128) tap[i] = L.taper[i];
  }
  // raw window of MODE 0
  const TIn* mbase = nullptr;
  const TIn* rbase = nullptr;
  long long mpitch = N, rpitch = N;
  if constexpr (MODE == 0) {
    const long long wb = b;
    if (L.patch_mode) {
      mbase = static_cast<const TIn*>(L.mov) + wb * L.mov_stride;
      rbase = static_cast<const TIn*>(L.ref) + wb * L.ref_stride;
    } else {
      mbase = static_cast<const TIn*>(L.mov) + static_cast<long long>(__ldg(L.mov_origin + 2 * wb)) * L.mov_pitch +
              __ldg(L.mov_origin + 2 * wb + 1);
      rbase = static_cast<const TIn*>(L.ref) + static_cast<long long>(__ldg(L.ref_origin + 2 * wb)) * L.ref_pitch +
              __ldg(L.ref_origin + 2 * wb + 1);
      mpitch = L.mov_pitch;
      rpitch = L.ref_pitch;
    }
  }
  const float inv_k = 1.0f / static_cast<float>(L.ref_count);
  // apodised pixel of channel c (0 moving, 1 reference), reference projected
  // over ref_count sections
  auto apod = [&](int c, int y, int x) -> float {
    float raw;
    if (c == 0) {
      raw = load_px<TIn>(mbase + y * mpitch + x);
    } else {
      raw = load_px<TIn>(rbase + y * rpitch + x);
      if (L.ref_count > 1) {
        for (int k = 1; k < L.ref_count; ++k) raw += load_px<TIn>(rbase + k * L.ref_stride + y * rpitch + x);
        raw *= inv_k;
      }
    }
    return tap[y] * tap[x] * (raw - (c == 0 ? st.x : st.y));
  };
  __syncthreads();
  float in_scale = 1.0f;
  if constexpr (FP16) {
    __shared__ float red[4];
    float mx = 0.f;
    if constexpr (MODE == 0 && sizeof(TIn) == 1) {
      mx = 255.f;  // |a(y) a(x) (p - mu)| <= 255 for 8-bit pixels
    } else if constexpr (MODE == 0) {
      for (int e = tid; e < 64 * K; e += 128) mx = fmaxf(mx, fabsf(apod((e % K) / N, m0 + e / K, e % N)));
    } else if constexpr (MODE == 3) {
      for (int e = tid; e < 64 * K; e += 128) {
        const int gm = m0 + e / K, gk = e % K;
        mx = fmaxf(mx, fabsf(in[((gk / N) * N + gm) * N + gk % N]));
      }
    } else {
      for (int e = tid; e < 64 * K; e += 128) mx = fmaxf(mx, fabsf(in[static_cast<size_t>(e / 64) * N + n0 + e % 64]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
    if (mx > 0.f && mx <= 3.4e38f) {
      const int e = ((__float_as_int(mx) >> 23) & 0xff) - 127;  // floor(log2 mx) for normal mx
      const int p = max(-126, min(127, 14 - e));
      in_scale = __int_as_float((p + 127) << 23);
    }
  }
  float acc[2][4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
    // stage A (64 x BK) and B (BK x 64 -> Bs[n][k]) as FP32
    for (int e = tid; e < 64 * BK; e += 128) {
      const int mm = e / BK, kk = e % BK;
      const int gm = m0 + mm, gk = k0 + kk;
      float v;
      if constexpr (MODE == 0) {
        v = apod(gk / N, gm, gk % N) * in_scale;  // A[y][(c, x)] = a(y) a(x) (raw_c[y][x] - mu_c)
      } else if constexpr (MODE == 3) {
        const int c = gk / N, kx = gk % N;  // A[y][(c, kx)] = in[c][y][kx]
        v = in[(c * N + gm) * N + kx] * in_scale;
      } else {
        v = W[static_cast<size_t>(gm) * K + gk];
      }
      As[mm][kk] = v;
    }
    for (int e = tid; e < 64 * BK; e += 128) {
      const int nn = e % 64, kk = e / 64;
      const int gn = n0 + nn, gk = k0 + kk;
      float v;
      if constexpr (MODE == 1 || MODE == 2) {
        v = in[static_cast<size_t>(gk) * N + gn] * in_scale;  // B[(c, y)][x] = in[c][y][x]
      } else {
        v = W[static_cast<size_t>(gk) * (MODE == 3 ? N : K) + gn];
      }
      Bs[nn][kk] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + g;
        split2<FP16>(As[r][ks + 2 * t], As[r][ks + 2 * t + 1], ah[i][0], al[i][0]);
        split2<FP16>(As[r + 8][ks + 2 * t], As[r + 8][ks + 2 * t + 1], ah[i][1], al[i][1]);
        split2<FP16>(As[r][ks + 2 * t + 8], As[r][ks + 2 * t + 9], ah[i][2], al[i][2]);
        split2<FP16>(As[r + 8][ks + 2 * t + 8], As[r + 8][ks + 2 * t + 9], ah[i][3], al[i][3]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cidx = wn + 8 * j + g;
        split2<FP16>(Bs[cidx][ks + 2 * t], Bs[cidx][ks + 2 * t + 1], bh[j][0], bl[j][0]);
        split2<FP16>(Bs[cidx][ks + 2 * t + 8], Bs[cidx][ks + 2 * t + 9], bh[j][1], bl[j][1]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          mma16816<FP16>(acc[i][j], al[i], bh[j]);
          mma16816<FP16>(acc[i][j], ah[i], bl[j]);
          mma16816<FP16>(acc[i][j], ah[i], bh[j]);
        }
    }
    __syncthreads();
  }
  // epilogue: write the 64 x 64 tile
  const float out_scale = 1.0f / in_scale;  // exact: a power of two
  // rows -> x0, columns -> x1, inverse columns -> x1, inverse rows -> x0
  float* out = (MODE == 0 || MODE == 3) ? T.x0 + s * 2 * N * N : T.x1 + s * 2 * N * N;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gm = m0 + wm + 16 * i + g + 8 * h;
        const int gn = n0 + wn + 8 * j + 2 * t;
        float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
        if constexpr (MODE == 0) {  // out[c'][y][kx] from column (c', kx)
          v0 *= out_scale;
          v1 *= out_scale;
          const int c = gn / N, kx = gn % N;
          *reinterpret_cast<float2*>(out + (c * N + gm) * N + kx) = make_float2(v0, v1);
        } else if constexpr (MODE == 3) {  // real response s[y][x]
          *reinterpret_cast<float2*>(out + gm * N + gn) = make_float2(v0 * out_scale, v1 * out_scale);
        } else {  // out[(c', ky)][x]
          v0 *= out_scale;
          v1 *= out_scale;
          *reinterpret_cast<float2*>(out + static_cast<size_t>(gm) * N + gn) = make_float2(v0, v1);
        }
      }
}

// ---------------------------------------------------------------------------
// unpack M, R from Z = DFT(m' + i r'), C = M conj(R), whitening (planar, all bins)
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) tc_whiten_kernel(const MatchLaunch L, const TcLaunch T) {
  const long long s = blockIdx.x / (N * N / 256 / 4);
  const int blk = blockIdx.x % (N * N / 256 / 4);
  if (stat_status(T.stats[s]) != SWIFT_WIN_OK) return;
  const float* z = T.x1 + s * 2 * N * N;
  float* g = T.x0 + s * 2 * N * N;
  const float half_w = -0.5f * L.w;
  const float inv_n2 = 1.0f / (static_cast<float>(N) * static_cast<float>(N));
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int e = (blk * 4 + r) * 256 + threadIdx.x;
    const int ky = e / N, kx = e % N;
    const int nky = (N - ky) & (N - 1), nkx = (N - kx) & (N - 1);
    const float2 a = make_float2(z[ky * N + kx], z[N * N + ky * N + kx]);
    const float2 bb = make_float2(z[nky * N + nkx], z[N * N + nky * N + nkx]);
    const float2 c = make_float2(0.5f * fmaf(a.x, bb.y, a.y * bb.x),
                                 0.25f * ((a.x * a.x + a.y * a.y) - (bb.x * bb.x + bb.y * bb.y)));
    const float mag2 = fmaf(c.x, c.x, c.y * c.y);
    float sc = mag2 > 0.f ? exp2f(half_w * log2f(mag2)) * inv_n2 : 0.f;
    if (e == 0) sc = 0.f;  // G[0,0] = 0
    g[ky * N + kx] = c.x * sc;
    g[N * N + ky * N + kx] = c.y * sc;
  }
}

// ---------------------------------------------------------------------------
// argmax and FP64 sums of the response, in the block-partial layout of the
// streaming finalize kernel (first block slot holds the window's totals)
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) tc_reduce_kernel(const TcLaunch T, unsigned long long* part) {
  using G = StreamGeom<N>;
  const long long s = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ unsigned long long wk[8];
  __shared__ double ws[8][2];
  if (stat_status(T.stats[s]) != SWIFT_WIN_OK) return;
  const float* sv = T.x0 + s * 2 * N * N;
  unsigned long long best = 0ull;
  float s1 = 0.f, s2 = 0.f;
  for (int e = tid; e < N * N; e += 256) {
    const float v = sv[e];
    const unsigned long long k = argmax_key(v, static_cast<uint32_t>(e));
    best = k > best ? k : best;
    s1 += v;
    s2 = fmaf(v, v, s2);
  }
  best = warp_max_u64(best);
  const double d1 = warp_sum_f64(s1), d2 = warp_sum_f64(s2);
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
    unsigned long long* p = part + 3 * s * G::NB3;
    p[0] = k;
    p[1] = static_cast<unsigned long long>(__double_as_longlong(a));
    p[2] = static_cast<unsigned long long>(__double_as_longlong(c));
    for (int q = 1; q < G::NB3; ++q) {
      p[3 * q] = 0ull;
      p[3 * q + 1] = 0ull;
      p[3 * q + 2] = 0ull;
    }
  }
}

}  // namespace swift
