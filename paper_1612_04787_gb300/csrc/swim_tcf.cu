// Launchers and tables of the tensor-core precision variant.
#include <math.h>

#include <vector>

#include "swim_tcf.cuh"

namespace swift {

namespace {

// Per-lane constant fragments from FP32 cos/sin tables (FP64-computed on the
// host): the real 32 x 32 block form of the 16-point DFT as A fragments and
// the 16 x 16 block form of the 8-point DFT as B fragments, each split into
// hi = round16(v) and lo = round16(v - hi).
template <bool FP16>
__global__ void tcf_frag_kernel(const float2* cs16, const float2* cs8, uint32_t* out) {
  const int lane = threadIdx.x, g = lane >> 2, t = lane & 3;
  // F16big[r][c] = [[cos, sin], [-sin, cos]] blocks (rows re / im of k1, columns re / im of n1)
  auto f16 = [&](int r, int c) -> float {
    const float2 w = cs16[((r & 15) * (c & 15)) & 15];
    const bool rim = r >= 16, cim = c >= 16;
    if (rim == cim) return w.x;
    return cim ? w.y : -w.y;
  };
  // F8big[r][c] = [[cos, -sin], [sin, cos]] blocks (rows re / im of n2, columns re / im of k2)
  auto f8 = [&](int r, int c) -> float {
    const float2 w = cs8[((r & 7) * (c & 7)) & 7];
    const bool rim = r >= 8, cim = c >= 8;
    if (rim == cim) return w.x;
    return cim ? -w.y : w.y;
  };
  auto split = [&](float a, float b, uint32_t& hi, uint32_t& lo) {
    if constexpr (FP16) {
      const __half2 h = __floats2half2_rn(a, b);
      const float2 hf = __half22float2(h);
      const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
      hi = *reinterpret_cast<const uint32_t*>(&h);
      lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
      const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
      const float2 hf = __bfloat1622float2(h);
      const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
      hi = *reinterpret_cast<const uint32_t*>(&h);
      lo = *reinterpret_cast<const uint32_t*>(&l);
    }
  };
  uint32_t* o = out + lane * kTcfFragRegs;
  for (int mt = 0; mt < 2; ++mt)
    for (int ks = 0; ks < 2; ++ks) {
      const int f = 4 * (2 * mt + ks);
      const int r0 = 16 * mt + g, c0 = 16 * ks + 2 * t;
      split(f16(r0, c0), f16(r0, c0 + 1), o[f + 0], o[16 + f + 0]);
      split(f16(r0 + 8, c0), f16(r0 + 8, c0 + 1), o[f + 1], o[16 + f + 1]);
      split(f16(r0, c0 + 8), f16(r0, c0 + 9), o[f + 2], o[16 + f + 2]);
      split(f16(r0 + 8, c0 + 8), f16(r0 + 8, c0 + 9), o[f + 3], o[16 + f + 3]);
    }
  for (int nt = 0; nt < 2; ++nt) {
    const int col = 8 * nt + g;
    split(f8(2 * t, col), f8(2 * t + 1, col), o[32 + 2 * nt], o[36 + 2 * nt]);
    split(f8(2 * t + 8, col), f8(2 * t + 9, col), o[32 + 2 * nt + 1], o[36 + 2 * nt + 1]);
  }
}

template <int N, bool FP16, typename TIn>
cudaError_t tcf_n(const MatchLaunch& L, const StreamWork& W, const TcfLaunch& T, cudaStream_t st) {
  const unsigned S = static_cast<unsigned>(W.count);
  if (S == 0) return cudaSuccess;
  auto mark = [&](int k) {
    if (W.ev) cudaEventRecord(W.ev[k], st);
  };
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static unsigned m1 = 0;
  if ((e = smem_optin(tcf_rows_kernel<N, FP16, TIn>, tcf_rows_smem<N, TIn>(), m1, dev)) != cudaSuccess) return e;
  mark(0);
  stream_stats_kernel<N, TIn><<<S, 256, 0, st>>>(L, W);
  mark(1);
  tcf_rows_kernel<N, FP16, TIn><<<S * (N / kTcfRowsPerCta), 256, tcf_rows_smem<N, TIn>(), st>>>(L, W, T);
  mark(2);
  tcf_cols_kernel<N, FP16><<<S * (N / 16), 256, 0, st>>>(L, W, T);
  mark(3);
  tcf_irows_kernel<N, FP16><<<S * StreamGeom<N>::NB3, 256, 0, st>>>(L, W, T);
  mark(4);
  stream_final_kernel<N><<<S, 32, 0, st>>>(L, W);
  mark(5);
  return cudaGetLastError();
}

template <bool FP16>
cudaError_t tcf_dispatch(int n, swift_dtype dtype, const MatchLaunch& L, const StreamWork& W, const TcfLaunch& T,
                         cudaStream_t st) {
  const bool u8 = dtype == SWIFT_IN_U8;
  switch (n) {
    case 128:
      return u8 ? tcf_n<128, FP16, uint8_t>(L, W, T, st) : tcf_n<128, FP16, float>(L, W, T, st);
    case 256:
      return u8 ? tcf_n<256, FP16, uint8_t>(L, W, T, st) : tcf_n<256, FP16, float>(L, W, T, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t tcf_table_bytes(int n) { return sizeof(uint32_t) * 32 * kTcfFragRegs + sizeof(float2) * (n + 16 + 8); }

cudaError_t tcf_build_tables(int n, bool fp16, void* dst) {
  // host tables in FP64, stored as FP32: twiddles exp(-2 pi i m / n), cos/sin of 2 pi m / 16 and 2 pi m / 8
  std::vector<float2> h(n + 16 + 8);
  for (int m = 0; m < n; ++m) {
    const double a = 2.0 * M_PI * m / n;
    h[m] = make_float2(static_cast<float>(cos(a)), static_cast<float>(-sin(a)));
  }
  for (int m = 0; m < 16; ++m) {
    const double a = 2.0 * M_PI * m / 16;
    h[n + m] = make_float2(static_cast<float>(cos(a)), static_cast<float>(sin(a)));
  }
  for (int m = 0; m < 8; ++m) {
    const double a = 2.0 * M_PI * m / 8;
    h[n + 16 + m] = make_float2(static_cast<float>(cos(a)), static_cast<float>(sin(a)));
  }
  uint32_t* frag = static_cast<uint32_t*>(dst);
  float2* tabs = reinterpret_cast<float2*>(frag + 32 * kTcfFragRegs);
  cudaError_t e = cudaMemcpy(tabs, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  if (fp16)
    tcf_frag_kernel<true><<<1, 32>>>(tabs + n, tabs + n + 16, frag);
  else
    tcf_frag_kernel<false><<<1, 32>>>(tabs + n, tabs + n + 16, frag);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaDeviceSynchronize();
}

TcfLaunch tcf_tables(const void* dst) {
  TcfLaunch T;
  T.frag = static_cast<const uint32_t*>(dst);
  T.tw = reinterpret_cast<const float2*>(T.frag + 32 * kTcfFragRegs);
  return T;
}

cudaError_t launch_tcf(int n, swift_dtype dtype, bool fp16, const MatchLaunch& L, const StreamWork& W,
                       const TcfLaunch& T, cudaStream_t st) {
  return fp16 ? tcf_dispatch<true>(n, dtype, L, W, T, st) : tcf_dispatch<false>(n, dtype, L, W, T, st);
}

}  // namespace swift
