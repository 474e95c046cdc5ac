// Register-resident small DFTs (radix 4, 8, 16) for the window transforms.
//
// DIR = -1 is the forward transform e^{-2 pi i k n / R}, DIR = +1 the inverse
// (unnormalised).  Inputs and outputs are in natural order.  The twiddle
// constants are cos/sin of multiples of pi/8, written out to float precision.
#pragma once
#include <cuda_runtime.h>

namespace swift {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// a * (DIR * i)
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// cos / sin of e * pi / 8, e = 0..15
__device__ constexpr float kC16[16] = {
    1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508978f,
    0.0f, -0.38268343236508978f, -0.70710678118654752f, -0.92387953251128674f,
    -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508978f,
    0.0f, 0.38268343236508978f, 0.70710678118654752f, 0.92387953251128674f};
__device__ constexpr float kS16[16] = {
    0.0f, 0.38268343236508978f, 0.70710678118654752f, 0.92387953251128674f,
    1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508978f,
    0.0f, -0.38268343236508978f, -0.70710678118654752f, -0.92387953251128674f,
    -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508978f};

// a * W16^(DIR * E), W16 = e^{2 pi i / 16}; E known at compile time
template <int DIR, int E>
__device__ __forceinline__ float2 tw16(float2 a) {
  constexpr int e = E & 15;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (e == 4) {
    return mul_i<DIR>(a);
  } else if constexpr (e == 8) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (e == 12) {
    return mul_i<-DIR>(a);
  } else if constexpr (e == 2 || e == 6 || e == 10 || e == 14) {
    // (c, DIR*s) with |c| == |s| == 1/sqrt(2)
    constexpr float c = kC16[e];
    constexpr float s = DIR * kS16[e];
    return make_float2(c * a.x - s * a.y, c * a.y + s * a.x);
  } else {
    constexpr float c = kC16[e];
    constexpr float s = DIR * kS16[e];
    return make_float2(fmaf(c, a.x, -s * a.y), fmaf(c, a.y, s * a.x));
  }
}

template <int DIR>
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
  float2 t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = mul_i<DIR>(csub(b, d));
  a = cadd(t0, t2);
  c = csub(t0, t2);
  b = cadd(t1, t3);
  d = csub(t1, t3);
}

// 8-point DFT: n = 2 n1 + n2, k = k1 + 4 k2
template <int DIR>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
  dft4<DIR>(v[0], v[2], v[4], v[6]);
  dft4<DIR>(v[1], v[3], v[5], v[7]);
  // v[n2 + 2 k1] = y[k1][n2]; twiddle W8^(n2 k1) = W16^(2 n2 k1)
  v[3] = tw16<DIR, 2>(v[3]);
  v[5] = tw16<DIR, 4>(v[5]);
  v[7] = tw16<DIR, 6>(v[7]);
  float2 o[8];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    o[k1] = cadd(v[2 * k1], v[2 * k1 + 1]);
    o[k1 + 4] = csub(v[2 * k1], v[2 * k1 + 1]);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = o[i];
}

// 16-point DFT: n = 4 n1 + n2, k = k1 + 4 k2
template <int DIR>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<DIR>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // v[n2 + 4 k1] = y[k1][n2]; twiddle W16^(n2 k1)
  v[5] = tw16<DIR, 1>(v[5]);
  v[6] = tw16<DIR, 2>(v[6]);
  v[7] = tw16<DIR, 3>(v[7]);
  v[9] = tw16<DIR, 2>(v[9]);
  v[10] = tw16<DIR, 4>(v[10]);
  v[11] = tw16<DIR, 6>(v[11]);
  v[13] = tw16<DIR, 3>(v[13]);
  v[14] = tw16<DIR, 6>(v[14]);
  v[15] = tw16<DIR, 9>(v[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<DIR>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // X[k1 + 4 k2] sits in v[4 k1 + k2]
  float2 o[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = o[i];
}

// cos / sin of e * pi / 16, e = 0..15 (the twiddles W32^e)
__device__ constexpr float kC32[16] = {
    1.0f, 0.98078528040323043f, 0.92387953251128674f, 0.83146961230254524f,
    0.70710678118654752f, 0.55557023301960218f, 0.38268343236508978f, 0.19509032201612826f,
    0.0f, -0.19509032201612826f, -0.38268343236508978f, -0.55557023301960218f,
    -0.70710678118654752f, -0.83146961230254524f, -0.92387953251128674f, -0.98078528040323043f};
__device__ constexpr float kS32[16] = {
    0.0f, 0.19509032201612826f, 0.38268343236508978f, 0.55557023301960218f,
    0.70710678118654752f, 0.83146961230254524f, 0.92387953251128674f, 0.98078528040323043f,
    1.0f, 0.98078528040323043f, 0.92387953251128674f, 0.83146961230254524f,
    0.70710678118654752f, 0.55557023301960218f, 0.38268343236508978f, 0.19509032201612826f};

// 32-point DFT: even / odd 16-point halves, then X[k] = E[k] + W^k O[k],
// X[k + 16] = E[k] - W^k O[k] with W = exp(DIR 2 pi i / 32)
template <int DIR>
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
  float2 e[16], o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft16<DIR>(e);
  dft16<DIR>(o);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float c = kC32[k], sn = DIR * kS32[k];
    const float2 t = k == 0 ? o[k] : make_float2(fmaf(c, o[k].x, -sn * o[k].y), fmaf(c, o[k].y, sn * o[k].x));
    v[k] = cadd(e[k], t);
    v[k + 16] = csub(e[k], t);
  }
}

template <int R, int DIR>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
  if constexpr (R == 32) dft32<DIR>(v);
  else if constexpr (R == 16) dft16<DIR>(v);
  else if constexpr (R == 8) dft8<DIR>(v);
  else static_assert(R == 8 || R == 16 || R == 32, "radix");
}

}  // namespace swift
