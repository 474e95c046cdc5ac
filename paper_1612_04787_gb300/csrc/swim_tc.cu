// Launchers of the tensor-core precision variant and its DFT block matrices.
#include <math.h>
#include <vector>

#include "swim_tc.cuh"

namespace swift {

namespace {

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

template <int N, bool FP16, typename TIn>
cudaError_t tc_n(const MatchLaunch& L, const StreamWork& W, const TcLaunch& T, cudaStream_t st) {
  const unsigned S = static_cast<unsigned>(W.count);
  if (S == 0) return cudaSuccess;
  constexpr int Q = N / 64;
  auto mark = [&](int k) {
    if (W.ev) cudaEventRecord(W.ev[k], st);
  };
  mark(0);
  stream_stats_kernel<N, TIn><<<S, 256, 0, st>>>(L, W);
  mark(1);
  tc_gemm_kernel<N, 0, FP16, TIn><<<S * Q * 2 * Q, 128, 0, st>>>(L, T);
  tc_gemm_kernel<N, 1, FP16, TIn><<<S * 2 * Q * Q, 128, 0, st>>>(L, T);
  mark(2);
  tc_whiten_kernel<N><<<S * (N * N / 1024), 256, 0, st>>>(L, T);
  mark(3);
  tc_gemm_kernel<N, 2, FP16, TIn><<<S * 2 * Q * Q, 128, 0, st>>>(L, T);
  tc_gemm_kernel<N, 3, FP16, TIn><<<S * Q * Q, 128, 0, st>>>(L, T);
  mark(4);
  tc_reduce_kernel<N><<<S, 256, 0, st>>>(T, W.part);
  stream_final_kernel<N><<<S, 32, 0, st>>>(L, W);
  mark(5);
  return cudaGetLastError();
}

template <bool FP16>
cudaError_t tc_dispatch(int n, swift_dtype dtype, const MatchLaunch& L, const StreamWork& W, const TcLaunch& T,
                        cudaStream_t st) {
  const bool u8 = dtype == SWIFT_IN_U8;
  switch (n) {
    case 128:
      return u8 ? tc_n<128, FP16, uint8_t>(L, W, T, st) : tc_n<128, FP16, float>(L, W, T, st);
    case 256:
      return u8 ? tc_n<256, FP16, uint8_t>(L, W, T, st) : tc_n<256, FP16, float>(L, W, T, st);
    default:
      return cudaErrorInvalidValue;
  }
}

int nb3(int n) { return n == 128 ? StreamGeom<128>::NB3 : StreamGeom<256>::NB3; }

}  // namespace

size_t tc_bytes_per_window(int n) {
  const size_t nn = static_cast<size_t>(n) * n;
  return 2 * 2 * sizeof(float) * nn + sizeof(float4) + 3 * sizeof(unsigned long long) * nb3(n);
}

size_t tc_matrix_floats(int n) { return 4 * static_cast<size_t>(2 * n) * (2 * n); }

// DFT block matrices in FP64, stored as FP32: [Wr | Wc | Wri | Wci], each (2n)^2
void tc_build_matrices(int n, float* m) {
  const size_t K = 2 * static_cast<size_t>(n);
  float* wr = m;
  float* wc = m + K * K;
  float* wri = m + 2 * K * K;
  float* wci = m + 3 * K * K;
  for (size_t i = 0; i < 4 * K * K; ++i) m[i] = 0.f;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      const double th = 2.0 * M_PI * static_cast<double>((static_cast<long long>(a) * b) % n) / n;
      const float c = static_cast<float>(cos(th)), s = static_cast<float>(sin(th));
      // rows: Wr[(c, x)][(c', kx)], x = a, kx = b; out_re = in_re cos + in_im sin, out_im = -in_re sin + in_im cos
      wr[(0 * n + a) * K + (0 * n + b)] = c;
      wr[(1 * n + a) * K + (0 * n + b)] = s;
      wr[(0 * n + a) * K + (1 * n + b)] = -s;
      wr[(1 * n + a) * K + (1 * n + b)] = c;
      // columns: Wc[(c', ky)][(c, y)], ky = a, y = b
      wc[(0 * n + a) * K + (0 * n + b)] = c;
      wc[(0 * n + a) * K + (1 * n + b)] = s;
      wc[(1 * n + a) * K + (0 * n + b)] = -s;
      wc[(1 * n + a) * K + (1 * n + b)] = c;
      // inverse columns: Wci[(c', y)][(c, ky)], y = a, ky = b; e^{+i th}
      wci[(0 * n + a) * K + (0 * n + b)] = c;
      wci[(0 * n + a) * K + (1 * n + b)] = -s;
      wci[(1 * n + a) * K + (0 * n + b)] = s;
      wci[(1 * n + a) * K + (1 * n + b)] = c;
      // inverse rows, real part: Wri[(c, kx)][x] (row stride n), kx = a, x = b
      wri[(0 * n + a) * n + b] = c;
      wri[(1 * n + a) * n + b] = -s;
    }
}

TcLaunch tc_carve(void* base, long long capacity, int n, const float* mats, long long b0, long long count,
                  StreamWork* W) {
  const size_t nn = static_cast<size_t>(n) * n;
  unsigned char* p = static_cast<unsigned char*>(base);
  TcLaunch T;
  T.mats = mats;
  T.x0 = reinterpret_cast<float*>(p);
  p += align256(2 * sizeof(float) * nn * capacity);
  T.x1 = reinterpret_cast<float*>(p);
  p += align256(2 * sizeof(float) * nn * capacity);
  T.stats = reinterpret_cast<float4*>(p);
  p += align256(sizeof(float4) * capacity);
  W->stats = T.stats;
  W->zr = reinterpret_cast<float2*>(T.x0);  // the response lives in x0, stride 2 n^2 floats
  W->h = nullptr;
  W->part = reinterpret_cast<unsigned long long*>(p);
  W->b0 = b0;
  W->count = count;
  W->ev = nullptr;
  T.b0 = b0;
  T.count = count;
  return T;
}

cudaError_t launch_tc(int n, swift_dtype dtype, bool fp16, const MatchLaunch& L, const StreamWork& W,
                      const TcLaunch& T, cudaStream_t st) {
  return fp16 ? tc_dispatch<true>(n, dtype, L, W, T, st) : tc_dispatch<false>(n, dtype, L, W, T, st);
}

}  // namespace swift
