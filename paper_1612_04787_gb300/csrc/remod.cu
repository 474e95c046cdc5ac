// Pyramid and model steps around the match (Sec. III module list):
//   iscale  box-mean downsampling by an integer factor f (2, 3, 5, ...):
//           output (y, x) is the mean of the f x f block at (f y, f x),
//           partial edge blocks dropped.  uint8: exact integer sum, rounded
//           half to even; float32: float32 sum in row-major block order
//           divided by f^2 (one IEEE division).
//   remod   Z-averaged model of every section of a uint8 stack: the mean of
//           the valid sections within +-k of z, z itself excluded; with no
//           valid neighbour, the section itself.  float32 output
//           = float32(integer sum) / float32(count).
// Both are memory-bound streaming kernels.  The model kernel gives each
// thread one pixel column (four pixels with 4-byte loads when aligned) and
// walks z with running integer sums, so every section is read from memory a
// bounded number of times (entering the window, leaving it, as the centre).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/swift.h"

namespace swift {

namespace {

__device__ __forceinline__ uint32_t round_half_even_div(uint32_t s, uint32_t d) {
  uint32_t q = s / d;
  const uint32_t r = s - q * d;
  if (2 * r > d || (2 * r == d && (q & 1))) q += 1;
  return q;
}

// uint8, f = 2 or 4, four outputs per thread from 8- or 16-byte row loads
template <int F, int OUT>
__global__ void downsample_u8_vec_kernel(const uint8_t* src, long long pitch, long long stride, uint8_t* out,
                                         long long out_pitch, long long out_stride, int H, int W) {
  // OUT outputs per thread from F rows of F * OUT bytes (8 or 16-byte loads)
  static_assert((F == 2 && (OUT == 4 || OUT == 8)) || (F == 4 && OUT == 4), "vector shapes");
  const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * OUT;
  const int y = blockIdx.y;
  if (x0 >= W) return;
  const uint8_t* b = src + blockIdx.z * stride + static_cast<long long>(F) * y * pitch + static_cast<long long>(F) * x0;
  uint32_t sum[OUT];
#pragma unroll
  for (int o = 0; o < OUT; ++o) sum[o] = 0u;
#pragma unroll
  for (int i = 0; i < F; ++i) {
    if constexpr (F == 2 && OUT == 4) {
      const uint2 v = __ldg(reinterpret_cast<const uint2*>(b + i * pitch));
      const uint32_t w[2] = {v.x, v.y};
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const uint32_t word = w[o >> 1];
        const int sh = 16 * (o & 1);
        sum[o] += ((word >> sh) & 0xffu) + ((word >> (sh + 8)) & 0xffu);
      }
    } else if constexpr (F == 2) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(b + i * pitch));
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const uint32_t word = w[o >> 1];
        const int sh = 16 * (o & 1);
        sum[o] += ((word >> sh) & 0xffu) + ((word >> (sh + 8)) & 0xffu);
      }
    } else {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(b + i * pitch));
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int o = 0; o < 4; ++o)
        sum[o] += (w[o] & 0xffu) + ((w[o] >> 8) & 0xffu) + ((w[o] >> 16) & 0xffu) + (w[o] >> 24);
    }
  }
  uint32_t packed[OUT / 4];
#pragma unroll
  for (int o = 0; o < OUT; ++o) {
    const uint32_t r = round_half_even_div(sum[o], F * F) << (8 * (o & 3));
    packed[o >> 2] = (o & 3) ? (packed[o >> 2] | r) : r;
  }
  uint8_t* op = out + blockIdx.z * out_stride + static_cast<long long>(y) * out_pitch + x0;
  if constexpr (OUT == 8) {
    *reinterpret_cast<uint2*>(op) = make_uint2(packed[0], packed[1]);
  } else {
    *reinterpret_cast<uint32_t*>(op) = packed[0];
  }
}

template <typename T>
__global__ void downsample_kernel(const T* src, long long pitch, long long stride, T* out, long long out_pitch,
                                  long long out_stride, int H, int W, int f) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= W) return;
  src += blockIdx.z * stride;
  out += blockIdx.z * out_stride;
  const T* b = src + static_cast<long long>(f) * y * pitch + static_cast<long long>(f) * x;
  if constexpr (sizeof(T) == 1) {
    int s = 0;
    for (int i = 0; i < f; ++i)
      for (int j = 0; j < f; ++j) s += __ldg(b + i * pitch + j);
    const int d = f * f;
    out[static_cast<long long>(y) * out_pitch + x] =
        static_cast<T>(round_half_even_div(static_cast<uint32_t>(s), static_cast<uint32_t>(d)));
  } else {
    float s = 0.f;
    for (int i = 0; i < f; ++i)
      for (int j = 0; j < f; ++j) s = __fadd_rn(s, __ldg(b + i * pitch + j));
    out[static_cast<long long>(y) * out_pitch + x] = __fdiv_rn(s, static_cast<float>(f * f));
  }
}

// V pixels per thread (V = 4: 4-byte loads / 16-byte (float) or 4-byte
// (uint8) stores, rows aligned); TOut float: float32(sum) / float32(count),
// uint8: the exact mean rounded half to even
template <int V, typename TOut>
__global__ void zmodel_kernel(const uint8_t* stack, long long stride, int Z, int H, int W, long long pitch, int k,
                              const uint8_t* valid, TOut* out, long long out_stride, long long out_pitch) {
  const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  const int y = blockIdx.y;
  if (x0 >= W) return;
  const uint8_t* col = stack + static_cast<long long>(y) * pitch + x0;
  TOut* ocol = out + static_cast<long long>(y) * out_pitch + x0;
  auto ok = [&](int j) { return valid == nullptr || __ldg(valid + j) != 0; };
  auto load = [&](int j, int (&v)[V]) {
    const uint8_t* p = col + static_cast<long long>(j) * stride;
    if constexpr (V == 16) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
      const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = (w4[i >> 2] >> (8 * (i & 3))) & 0xff;
    } else if constexpr (V == 4) {
      const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(p));
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = (w >> (8 * i)) & 0xff;
    } else {
      v[0] = __ldg(p);
    }
  };
  int S[V], t[V];
#pragma unroll
  for (int i = 0; i < V; ++i) S[i] = 0;
  int C = 0;
  // window [0 - k, 0 + k] clipped: sections 0 .. k
  for (int j = 0; j <= k && j < Z; ++j) {
    if (!ok(j)) continue;
    load(j, t);
#pragma unroll
    for (int i = 0; i < V; ++i) S[i] += t[i];
    C += 1;
  }
  for (int z = 0; z < Z; ++z) {
    if (z > 0) {  // slide: z + k enters, z - k - 1 leaves
      const int jin = z + k, jout = z - k - 1;
      if (jin < Z && ok(jin)) {
        load(jin, t);
#pragma unroll
        for (int i = 0; i < V; ++i) S[i] += t[i];
        C += 1;
      }
      if (jout >= 0 && ok(jout)) {
        load(jout, t);
#pragma unroll
        for (int i = 0; i < V; ++i) S[i] -= t[i];
        C -= 1;
      }
    }
    int c[V];
    load(z, c);
    const bool vz = ok(z);
    const int n = C - (vz ? 1 : 0);
    TOut* op = ocol + static_cast<long long>(z) * out_stride;
    if constexpr (sizeof(TOut) == 4) {
      float o[V];
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const int s = S[i] - (vz ? c[i] : 0);
        o[i] = n > 0 ? __fdiv_rn(static_cast<float>(s), static_cast<float>(n)) : static_cast<float>(c[i]);
      }
      if constexpr (V >= 4) {
#pragma unroll
        for (int i = 0; i < V; i += 4)
          __stcs(reinterpret_cast<float4*>(op + i), make_float4(o[i], o[i + 1], o[i + 2], o[i + 3]));
      } else {
        __stcs(op, o[0]);
      }
    } else {
      uint32_t o[V];
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const int s = S[i] - (vz ? c[i] : 0);
        o[i] = n > 0 ? round_half_even_div(static_cast<uint32_t>(s), static_cast<uint32_t>(n))
                     : static_cast<uint32_t>(c[i]);
      }
      if constexpr (V == 16) {
        uint32_t w4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          w4[i] = o[4 * i] | (o[4 * i + 1] << 8) | (o[4 * i + 2] << 16) | (o[4 * i + 3] << 24);
        *reinterpret_cast<uint4*>(op) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
      } else if constexpr (V == 4) {
        *reinterpret_cast<uint32_t*>(op) = o[0] | (o[1] << 8) | (o[2] << 16) | (o[3] << 24);
      } else {
        *op = static_cast<uint8_t>(o[0]);
      }
    }
  }
}

}  // namespace

}  // namespace swift

extern "C" swift_status swift_downsample(const swift_image* src, swift_dtype dtype, int32_t factor, void* out,
                                         int64_t out_pitch, void* stream) {
  if (!src || !src->data || !out || factor < 1 || factor > 64) return SWIFT_ERR_INVALID_ARG;
  if (dtype != SWIFT_IN_U8 && dtype != SWIFT_IN_F32) return SWIFT_ERR_INVALID_ARG;
  if (src->height < 0 || src->width < 0 || src->pitch < src->width || src->count < 1) return SWIFT_ERR_INVALID_ARG;
  if (src->count > 1 && src->stride < src->pitch * src->height) return SWIFT_ERR_INVALID_ARG;
  const int H = src->height / factor, W = src->width / factor;
  if (out_pitch < W) return SWIFT_ERR_INVALID_ARG;
  if (H == 0 || W == 0) return SWIFT_OK;
  if (H > 65535 || src->count > 65535) return SWIFT_ERR_UNSUPPORTED;  // grid limits
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  const long long out_stride = out_pitch * H;  // output planes follow each other
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == SWIFT_IN_U8) {
    const uint8_t* s8 = static_cast<const uint8_t*>(src->data);
    uint8_t* o8 = static_cast<uint8_t*>(out);
    const int F = factor;
    const bool vec = (F == 2 || F == 4) && W % 4 == 0 && src->pitch % (4 * F) == 0 &&
                     (src->count == 1 || src->stride % (4 * F) == 0) &&
                     (reinterpret_cast<uintptr_t>(s8) % (4 * F)) == 0 && out_pitch % 4 == 0 &&
                     (reinterpret_cast<uintptr_t>(o8) % 4) == 0;
    // 2x: eight outputs per thread from 16-byte loads when the rows allow it
    const bool vec8 = vec && F == 2 && W % 8 == 0 && src->pitch % 16 == 0 &&
                      (src->count == 1 || src->stride % 16 == 0) && (reinterpret_cast<uintptr_t>(s8) % 16) == 0 &&
                      out_pitch % 8 == 0 && (reinterpret_cast<uintptr_t>(o8) % 8) == 0;
    if (vec8) {
      const dim3 grid((W / 8 + 127) / 128, H, src->count);
      swift::downsample_u8_vec_kernel<2, 8><<<grid, 128, 0, st>>>(s8, src->pitch, src->stride, o8, out_pitch,
                                                                  out_stride, H, W);
    } else if (vec) {
      const dim3 grid((W / 4 + 127) / 128, H, src->count);
      if (F == 2)
        swift::downsample_u8_vec_kernel<2, 4><<<grid, 128, 0, st>>>(s8, src->pitch, src->stride, o8, out_pitch,
                                                                    out_stride, H, W);
      else
        swift::downsample_u8_vec_kernel<4, 4><<<grid, 128, 0, st>>>(s8, src->pitch, src->stride, o8, out_pitch,
                                                                    out_stride, H, W);
    } else {
      const dim3 grid((W + 255) / 256, H, src->count);
      swift::downsample_kernel<uint8_t><<<grid, 256, 0, st>>>(s8, src->pitch, src->stride, o8, out_pitch,
                                                                out_stride, H, W, factor);
    }
  } else {
    const dim3 grid((W + 255) / 256, H, src->count);
    swift::downsample_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(src->data), src->pitch,
                                                            src->stride, static_cast<float*>(out), out_pitch,
                                                            out_stride, H, W, factor);
  }
  return cudaGetLastError() == cudaSuccess ? SWIFT_OK : SWIFT_ERR_CUDA;
}

extern "C" swift_status swift_zmodel(const uint8_t* stack, int64_t stride, int32_t n_sections, int32_t height,
                                     int32_t width, int64_t pitch, int32_t k, const uint8_t* valid, void* out,
                                     swift_dtype out_dtype, int64_t out_stride, int64_t out_pitch, void* stream) {
  if (!stack || !out || n_sections < 0 || height < 0 || width < 0 || k < 0 || pitch < width || out_pitch < width)
    return SWIFT_ERR_INVALID_ARG;
  if (out_dtype != SWIFT_IN_U8 && out_dtype != SWIFT_IN_F32) return SWIFT_ERR_INVALID_ARG;
  if (n_sections > 1 && (stride < pitch * height || out_stride < out_pitch * height)) return SWIFT_ERR_INVALID_ARG;
  if (n_sections == 0 || height == 0 || width == 0) return SWIFT_OK;
  if (height > 65535) return SWIFT_ERR_UNSUPPORTED;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool f32 = out_dtype == SWIFT_IN_F32;
  const int oalign = f32 ? 15 : 3;  // 16-byte float4 / 4-byte packed stores
  const bool vec = width % 4 == 0 && pitch % 4 == 0 && stride % 4 == 0 && out_pitch % 4 == 0 && out_stride % 4 == 0 &&
                   (reinterpret_cast<uintptr_t>(stack) & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & oalign) == 0;
  // 16 pixels per thread when every row and section start is 16-byte aligned (input and output)
  const bool vec16 = vec && width % 16 == 0 && pitch % 16 == 0 && stride % 16 == 0 && out_pitch % 16 == 0 &&
                     out_stride % 16 == 0 && (reinterpret_cast<uintptr_t>(stack) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  const dim3 grid_v((width / 4 + 127) / 128, height), grid_s((width + 127) / 128, height);
  const dim3 grid_16((width / 16 + 127) / 128, height);
  if (f32) {
    float* o = static_cast<float*>(out);
    if (vec16)
      swift::zmodel_kernel<16, float><<<grid_16, 128, 0, st>>>(stack, stride, n_sections, height, width, pitch, k,
                                                               valid, o, out_stride, out_pitch);
    else if (vec)
      swift::zmodel_kernel<4, float><<<grid_v, 128, 0, st>>>(stack, stride, n_sections, height, width, pitch, k,
                                                             valid, o, out_stride, out_pitch);
    else
      swift::zmodel_kernel<1, float><<<grid_s, 128, 0, st>>>(stack, stride, n_sections, height, width, pitch, k,
                                                             valid, o, out_stride, out_pitch);
  } else {
    uint8_t* o = static_cast<uint8_t*>(out);
    if (vec16)
      swift::zmodel_kernel<16, uint8_t><<<grid_16, 128, 0, st>>>(stack, stride, n_sections, height, width, pitch, k,
                                                                 valid, o, out_stride, out_pitch);
    else if (vec)
      swift::zmodel_kernel<4, uint8_t><<<grid_v, 128, 0, st>>>(stack, stride, n_sections, height, width, pitch, k,
                                                               valid, o, out_stride, out_pitch);
    else
      swift::zmodel_kernel<1, uint8_t><<<grid_s, 128, 0, st>>>(stack, stride, n_sections, height, width, pitch, k,
                                                               valid, o, out_stride, out_pitch);
  }
  return cudaGetLastError() == cudaSuccess ? SWIFT_OK : SWIFT_ERR_CUDA;
}
