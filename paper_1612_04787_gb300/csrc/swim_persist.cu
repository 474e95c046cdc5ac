// Launcher of the persistent forward schedule (swim_persist.cuh).
#include "swim_persist.cuh"

namespace swift {

namespace {

size_t round256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

template <typename TIn>
constexpr size_t smem_for() {
  size_t m = 0;
  const size_t v[] = {rows_smem<64, TIn>(),  rows_smem<128, TIn>(),  rows_smem<256, TIn>(), cpair_smem<64>(),
                      cpair_smem<128>(),     cpair_smem<256>(),      irows_smem<64>(),      irows_smem<128>(),
                      irows_smem<256>()};
  for (size_t x : v) m = x > m ? x : m;
  return m;
}

template <typename TIn>
cudaError_t grid_for(int dev, int* grid) {
  static int cached[64] = {};
  if (dev >= 0 && dev < 64 && cached[dev] > 0) {
    *grid = cached[dev];
    return cudaSuccess;
  }
  cudaError_t e = cudaFuncSetAttribute(swim_persistent_kernel<TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem_for<TIn>()));
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, swim_persistent_kernel<TIn>, 256,
                                                         smem_for<TIn>())) != cudaSuccess)
    return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  *grid = (per_sm > 0 ? per_sm : 1) * sms;
  if (dev >= 0 && dev < 64) cached[dev] = *grid;
  return cudaSuccess;
}

}  // namespace

// Workspace: control words and slot words (cleared before every launch), then
// per-window statistics and partials, per-level lists, and the two rings.
size_t persist_bytes(int n_levels, long long B, int nmax, int ring) {
  const size_t nn = static_cast<size_t>(nmax) * nmax;
  return round256(sizeof(unsigned int) * (4 + kPersistMaxLevels)) + round256(sizeof(unsigned long long) * ring) +
         round256(sizeof(float4) * B) + round256(sizeof(unsigned long long) * kPersistPartStride * B) +
         round256(sizeof(float) * kPersistRowBlocks * 8 * B) + round256(sizeof(int) * n_levels * B) + round256(sizeof(float2) * nn * ring) +
         round256(sizeof(float2) * nn / 2 * ring);
}

cudaError_t launch_persist(PersistLaunch P, void* work, swift_dtype dtype, cudaStream_t st) {
  if (P.B <= 0 || P.n_levels <= 0) return cudaSuccess;
  unsigned char* p = static_cast<unsigned char*>(work);
  unsigned int* ctrl = reinterpret_cast<unsigned int*>(p);
  P.queue = ctrl;
  P.comp_done = ctrl + 1;
  P.abort = ctrl + 2;
  P.lcount = ctrl + 4;
  p += round256(sizeof(unsigned int) * (4 + kPersistMaxLevels));
  P.slot = reinterpret_cast<unsigned long long*>(p);
  p += round256(sizeof(unsigned long long) * P.ring);
  const size_t cleared = static_cast<size_t>(p - static_cast<unsigned char*>(work));
  P.stats = reinterpret_cast<float4*>(p);
  p += round256(sizeof(float4) * P.B);
  P.part = reinterpret_cast<unsigned long long*>(p);
  p += round256(sizeof(unsigned long long) * kPersistPartStride * P.B);
  P.rstat = reinterpret_cast<float*>(p);
  p += round256(sizeof(float) * kPersistRowBlocks * 8 * P.B);
  P.lists = reinterpret_cast<int*>(p);
  p += round256(sizeof(int) * P.n_levels * P.B);
  const size_t nn = static_cast<size_t>(P.nmax) * P.nmax;
  P.zr = reinterpret_cast<float2*>(p);
  p += round256(sizeof(float2) * nn * P.ring);
  P.h = reinterpret_cast<float2*>(p);
  P.n_compact = P.level_idx != nullptr ? static_cast<int>((P.B + kCompactWindows - 1) / kCompactWindows) : 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(work, 0, cleared, st)) != cudaSuccess) return e;
  int grid = 0;
  if (dtype == SWIFT_IN_U8) {
    if ((e = grid_for<uint8_t>(dev, &grid)) != cudaSuccess) return e;
    swim_persistent_kernel<uint8_t><<<grid, 256, smem_for<uint8_t>(), st>>>(P);
  } else {
    if ((e = grid_for<float>(dev, &grid)) != cudaSuccess) return e;
    swim_persistent_kernel<float><<<grid, 256, smem_for<float>(), st>>>(P);
  }
  return cudaGetLastError();
}

}  // namespace swift
