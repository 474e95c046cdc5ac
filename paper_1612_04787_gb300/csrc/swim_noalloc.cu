// Allocation-free forward match: the streaming kernels with their scratch in a
// file-scope device array instead of a plan workspace.
//
// For callers that cannot allocate device memory: code that runs inside
// another allocator's callback, real-time loops whose memory must not change
// after start-up, or hosts where the memory pool is owned by a framework.
// Every call computes its small taper and twiddle tables on the device (one
// tiny kernel on the caller's stream, straight into the static array; no
// host buffer is involved), then runs the same streaming kernels as the plan
// path.
#include <cuda_runtime.h>
#include <initializer_list>
#include <math.h>
#include <mutex>
#include <stdint.h>

#include "../../include/swift.h"
#include "swift_internal.h"

namespace {

// Static scratch shared by every call on a device (held until the process exits).
constexpr size_t kNoAllocBytes = 24u << 20;  // 24 MiB
constexpr size_t kTableBytes = 8192;         // taper (n floats, at 0), twiddles (n complex, at 2048) and
                                             // the taper's transform (n floats, at 6144)
constexpr size_t kDoneBytes = 2048;          // per-window finalize counters (512), after the tables; they
                                             // start at zero (static storage) and every call leaves them zero
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array, looked up once per device with that device
// current (the host-side symbol is only a stand-in, not a device address).
void* g_scratch_ptr[64] = {};
std::mutex g_scratch_mutex;

cudaError_t scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

long long capacity_for(int n) {
  const size_t per = swift::stream_bytes_per_window(n);
  return static_cast<long long>((kNoAllocBytes - kTableBytes - kDoneBytes - 4 * 256) / per);
}

// taper (n floats), twiddle table (n complex, [m][j] with j < r1) and the
// taper's transform (n floats) of a level, from the same definitions the plan
// path evaluates (the transform with the same device function as its kernel)
__global__ void noalloc_tables_kernel(int n, int apod, float alpha, int r1, float* tap, float2* tw, float* ahat) {
  __shared__ float cos_tab[512];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    tap[k] = static_cast<float>(swift::taper_value(n, apod, static_cast<double>(alpha), k));
    tw[k] = swift::twiddle_entry(n, r1, k);
  }
  __syncthreads();
  swift::taper_spectrum(n, apod, alpha, tap, ahat, cos_tab, threadIdx.x, blockDim.x);
}

}  // namespace

extern "C" swift_status swift_match_batch_noalloc(const swift_level* level, swift_dtype in, const swift_batch* batch,
                                                  swift_result* out, void* stream) {
  if (!level || !batch) return SWIFT_ERR_INVALID_ARG;
  const swift_level lv = *level;
  if (lv.n != 64 && lv.n != 128 && lv.n != 256 && lv.n != 512) return SWIFT_ERR_UNSUPPORTED;
  if (in != SWIFT_IN_U8 && in != SWIFT_IN_F32) return SWIFT_ERR_INVALID_ARG;
  if (!(lv.whiten_exponent >= 0.f && lv.whiten_exponent <= 1.f)) return SWIFT_ERR_INVALID_ARG;
  if (lv.apod != SWIFT_APOD_NONE && lv.apod != SWIFT_APOD_HANN && lv.apod != SWIFT_APOD_TUKEY)
    return SWIFT_ERR_INVALID_ARG;
  if (lv.apod == SWIFT_APOD_TUKEY && !(lv.tukey_alpha > 0.f && lv.tukey_alpha <= 1.f)) return SWIFT_ERR_INVALID_ARG;
  if (!(lv.snr_exclusion_radius >= 0.f) || !(lv.snr_exclusion_radius < 0.25f * lv.n)) return SWIFT_ERR_INVALID_ARG;
  const long long B = batch->n_windows;
  if (B < 0) return SWIFT_ERR_INVALID_ARG;
  if (B > capacity_for(lv.n)) return SWIFT_ERR_CAPACITY;
  if (B == 0) return SWIFT_OK;
  if (!out || !batch->ref || !batch->mov || batch->level) return SWIFT_ERR_INVALID_ARG;
  const int pm = batch->patch_mode ? 1 : 0;
  if (!pm && (!batch->ref_origin || !batch->mov_origin)) return SWIFT_ERR_INVALID_ARG;
  const swift_image& ri = batch->ref[0];
  const swift_image& mi = batch->mov[0];
  for (const swift_image* im : {&ri, &mi}) {
    if (!im->data || im->count < 1) return SWIFT_ERR_INVALID_ARG;
    if (pm) {
      if (im->count != 1 || (B > 1 && im->stride < static_cast<int64_t>(lv.n) * lv.n)) return SWIFT_ERR_INVALID_ARG;
    } else if (im->height < 1 || im->width < 1 || im->pitch < im->width ||
               (im->count > 1 && im->stride < im->pitch * im->height)) {
      return SWIFT_ERR_INVALID_ARG;
    }
  }
  if (mi.count != 1) return SWIFT_ERR_INVALID_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SWIFT_ERR_CUDA;
  void* scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) return SWIFT_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // tables: taper at the start of the array, twiddles at byte 2048
  const int n = lv.n;
  int r1 = 0, r2 = 0;
  swift::stream_radices(n, &r1, &r2);
  double sum_a = 0.0;  // host copy of the taper's sum, for the mean's normalisation
  for (int k = 0; k < n; ++k) sum_a += swift::taper_value(n, lv.apod, lv.tukey_alpha, k);
  unsigned char* base = static_cast<unsigned char*>(scratch);
  noalloc_tables_kernel<<<1, 256, 0, st>>>(n, lv.apod, lv.tukey_alpha, r1, reinterpret_cast<float*>(base),
                                           reinterpret_cast<float2*>(base + 2048),
                                           reinterpret_cast<float*>(base + 6144));

  swift::MatchLaunch L;
  L.ref = ri.data;
  L.mov = mi.data;
  L.ref_pitch = pm ? n : ri.pitch;
  L.mov_pitch = pm ? n : mi.pitch;
  L.ref_stride = pm ? (ri.stride ? ri.stride : static_cast<long long>(n) * n) : ri.stride;
  L.mov_stride = pm ? (mi.stride ? mi.stride : static_cast<long long>(n) * n) : mi.stride;
  L.ref_h = ri.height;
  L.ref_w = ri.width;
  L.mov_h = mi.height;
  L.mov_w = mi.width;
  L.ref_count = ri.count;
  L.patch_mode = pm;
  L.ref_origin = batch->ref_origin;
  L.mov_origin = batch->mov_origin;
  L.level_idx = nullptr;
  L.level = 0;
  L.n_windows = B;
  L.w = lv.whiten_exponent;
  L.radius2 = static_cast<float>(floor(static_cast<double>(lv.snr_exclusion_radius) * lv.snr_exclusion_radius));
  L.inv_sum_a = 1.0 / (sum_a * sum_a);
  L.taper = reinterpret_cast<const float*>(base);
  L.twiddle = reinterpret_cast<const float2*>(base + 2048);
  L.ahat = reinterpret_cast<const float*>(base + 6144);
  L.out = out;
  swift::StreamWork W = swift::stream_carve(base + kTableBytes + kDoneBytes, capacity_for(n), n, 0, B);
  W.done = reinterpret_cast<unsigned int*>(base + kTableBytes);
  if (swift::launch_stream(n, in, L, W, st) != cudaSuccess) return SWIFT_ERR_CUDA;
  return SWIFT_OK;
}
