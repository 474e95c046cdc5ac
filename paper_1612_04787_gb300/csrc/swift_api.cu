// Host side of the C ABI: plans (taper and twiddle tables), argument checks,
// dispatch to the per-size kernels.  No exceptions cross this boundary.
#include <cuda_runtime.h>
#include <math.h>
#include <new>
#include <stdint.h>
#include <string.h>

#include "../../include/swift.h"
#include "swift_internal.h"

namespace {

constexpr int kMaxLevels = 16;
constexpr int kTimingSets = 1024;
constexpr int kNumSizes = 4;
constexpr int kSizes[kNumSizes] = {64, 128, 256, 512};

int size_slot(int n) {
  for (int i = 0; i < kNumSizes; ++i)
    if (kSizes[i] == n) return i;
  return -1;
}
// window sizes with a fused (cluster) kernel; 512 x 512 windows always stream
bool has_fused(int n) { return n <= 256; }

// 1D taper of a level in FP64 (swift::taper_value)
void taper_table(int n, int apod, double alpha, double* a) {
  for (int k = 0; k < n; ++k) a[k] = swift::taper_value(n, apod, alpha, k);
}

}  // namespace

struct swift_plan_s {
  int n_levels = 0;
  swift_level levels[kMaxLevels];
  swift_dtype dtype = SWIFT_IN_U8;
  swift_precision prec = SWIFT_PREC_FP32;
  int64_t max_windows = 0;
  int device = 0;
  float* taper[kMaxLevels] = {};
  float* ahat[kMaxLevels] = {};  // DFT of each level's 1D taper (swift::launch_taper_spectrum)
  double inv_sum_a[kMaxLevels] = {};
  float2* twiddle[kNumSizes] = {};
  // tensor-core precision variant: fragment and twiddle tables per window size
  void* tc_tab[kNumSizes] = {};
  // forward schedule of each level (SWIFT_SCHED_FUSED / _STREAM / _PERSISTENT)
  int sched[kMaxLevels] = {};
  // streaming forward path: its workspace
  void* work = nullptr;
  long long work_windows = 0;  // windows per slice with one lane (of the largest streamed size)
  size_t work_per = 0;         // workspace bytes per window at the largest streamed size
  long long lane_cap = 0;      // windows per streaming slice in each of two lanes (workspace part of each)
  unsigned int* done = nullptr;  // per-window block counters of the streaming finalize (kept zero)
  // lanes: the streams one forward call spreads its launch units over (the
  // call's stream and one auxiliary stream), each with its own part of the
  // workspace; fork / join events order the auxiliary lane with the call
  int lanes = 2;
  int row_tma = 1;  // swift_plan_set_row_tma
  cudaStream_t aux = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  // affine-warp forward and backward: allocated on first use
  void* bwork = nullptr;
  long long bwork_windows = 0;
  double* gw_acc = nullptr;  // [kMaxLevels] accumulated dL/dw
  // persistent schedule: workspace (grown to the largest batch seen), skew
  // and ring of its work order, the bound of its waits, and its test hook
  void* pwork = nullptr;
  size_t pwork_bytes = 0;
  int pskew = 16;
  long long pspin = 4000000000ll;  // clock cycles (about 2 s at 2 GHz)
  long long phold = -1;            // swift_plan_set_test_hold
  // per-kernel timing (swift_plan_set_timing / swift_plan_timings): a ring
  // of event sets, one set per streaming slice or fused launch
  bool test_stall = false;  // swift_plan_set_test_stall
  bool test_stale_ok = false;  // swift_plan_set_test_stale_status
  bool timing = false;
  cudaEvent_t* tev = nullptr;   // [kTimingSets][6]
  int* tkind = nullptr;         // [kTimingSets] 0 = streaming set (five kernels), 1 = fused launch,
                                // 2 = persistent launch, 8 | bits = FP32 streaming set (bit 1: no
                                // finalize kernel, bit 2: no statistics kernel)
  int tcount = 0;               // sets used since the last read
  // one captured forward call (swift_plan_capture / swift_plan_replay)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  // every call of the plan shares its workspace: an event recorded after each
  // call, which a call arriving on another stream waits for first
  cudaEvent_t order_ev = nullptr;
  cudaStream_t order_stream = nullptr;
  bool order_used = false;
};

namespace {
// windows per slice of the streaming path (bounds its workspace)
#ifndef SWIFT_STREAM_SLICE
#define SWIFT_STREAM_SLICE 2048
#endif
constexpr long long kStreamSlice = SWIFT_STREAM_SLICE;
// windows per slice of the affine / backward path
constexpr long long kBackSlice = 1024;
// default forward schedule: 128 x 128 and larger windows stream their
// intermediates through the workspace; 64 x 64 windows use the fused kernel
// (the persistent one-launch schedule measured slower on every workload)
int default_sched(int n) { return n >= 128 ? SWIFT_SCHED_STREAM : SWIFT_SCHED_FUSED; }
bool has_persistent(int n) { return n == 64 || n == 128 || n == 256; }
// ring slots of the persistent schedule for skew D (RING > 4 D); skews tried
// by the autotuner
int persist_ring(int skew) { return 5 * skew + 4; }
constexpr int kMaxSkew = 16;
constexpr int kSkews[] = {4, 8, 12, 16};
// lanes of a forward call: windows per streaming slice and the byte stride of
// the lanes' workspace parts (256-aligned: the carve aligns within a part)
constexpr int kMaxLanes = 2;
long long lane_capacity(long long work_windows, int lanes) { return (work_windows + lanes - 1) / lanes; }
// each lane's workspace part holds a full single-lane slice while that is at
// most this many bytes, else half of one
constexpr size_t kLaneBytes = size_t(2) << 30;
constexpr long long kMinLaneSlice = 256;
size_t lane_stride(size_t per, long long capacity) {
  return ((per * static_cast<size_t>(capacity) + 255) & ~static_cast<size_t>(255)) + 1024;
}
// the streams of one forward call: lane 0 is the call's stream; units (a
// fused launch, a streaming slice) go to the lane with the least work queued
struct Lanes {
  cudaStream_t s[kMaxLanes] = {};
  int n = 1;
  double load[kMaxLanes] = {};
};
int lane_pick(Lanes& ls, double cost) {
  int k = 0;
  for (int i = 1; i < ls.n; ++i)
    if (ls.load[i] < ls.load[k]) k = i;
  ls.load[k] += cost;
  return k;
}
}  // namespace

static swift_status release(swift_plan p) {
  if (!p) return SWIFT_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != p->device) cudaSetDevice(p->device);
  for (int l = 0; l < kMaxLevels; ++l) {
    if (p->taper[l]) cudaFree(p->taper[l]);
    if (p->ahat[l]) cudaFree(p->ahat[l]);
  }
  for (int i = 0; i < kNumSizes; ++i) {
    if (p->twiddle[i]) cudaFree(p->twiddle[i]);
    if (p->tc_tab[i]) cudaFree(p->tc_tab[i]);
  }
  if (p->work) cudaFree(p->work);
  if (p->done) cudaFree(p->done);
  if (p->bwork) cudaFree(p->bwork);
  if (p->pwork) cudaFree(p->pwork);
  if (p->tev) {
    for (int i = 0; i < 6 * kTimingSets; ++i) cudaEventDestroy(p->tev[i]);
    delete[] p->tev;
    delete[] p->tkind;
  }
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->gw_acc) cudaFree(p->gw_acc);
  if (p->order_ev) cudaEventDestroy(p->order_ev);
  if (p->fork_ev) cudaEventDestroy(p->fork_ev);
  if (p->join_ev) cudaEventDestroy(p->join_ev);
  if (p->aux) cudaStreamDestroy(p->aux);
  if (cur != p->device) cudaSetDevice(cur);
  delete p;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_create(const swift_level* levels, int32_t n_levels, swift_dtype in,
                                          swift_precision prec, int64_t max_windows, swift_plan* out) {
  if (out) *out = nullptr;
  if (!out || !levels || n_levels < 1 || n_levels > kMaxLevels || max_windows <= 0) return SWIFT_ERR_INVALID_ARG;
  if (in != SWIFT_IN_U8 && in != SWIFT_IN_F32) return SWIFT_ERR_INVALID_ARG;
  if (prec != SWIFT_PREC_FP32 && prec != SWIFT_PREC_BF16X2 && prec != SWIFT_PREC_FP16X2) return SWIFT_ERR_INVALID_ARG;
  for (int l = 0; l < n_levels; ++l) {
    const swift_level& lv = levels[l];
    // the tensor-core variant is built for 128 x 128 and 256 x 256 windows
    if (prec != SWIFT_PREC_FP32 && lv.n != 128 && lv.n != 256) return SWIFT_ERR_UNSUPPORTED;
    if (lv.n < 2 || (lv.n & (lv.n - 1)) != 0) return SWIFT_ERR_INVALID_ARG;
    if (!(lv.whiten_exponent >= 0.f && lv.whiten_exponent <= 1.f)) return SWIFT_ERR_INVALID_ARG;
    if (lv.apod != SWIFT_APOD_NONE && lv.apod != SWIFT_APOD_HANN && lv.apod != SWIFT_APOD_TUKEY)
      return SWIFT_ERR_INVALID_ARG;
    if (lv.apod == SWIFT_APOD_TUKEY && !(lv.tukey_alpha > 0.f && lv.tukey_alpha <= 1.f)) return SWIFT_ERR_INVALID_ARG;
    if (!(lv.snr_exclusion_radius >= 0.f) || !(lv.snr_exclusion_radius < 0.25f * lv.n)) return SWIFT_ERR_INVALID_ARG;
    if (size_slot(lv.n) < 0) return SWIFT_ERR_UNSUPPORTED;
  }
  swift_plan p = new (std::nothrow) swift_plan_s();
  if (!p) return SWIFT_ERR_OOM;
  p->n_levels = n_levels;
  memcpy(p->levels, levels, sizeof(swift_level) * n_levels);
  p->dtype = in;
  p->prec = prec;
  p->max_windows = max_windows;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return SWIFT_ERR_CUDA;
  }
  if (cudaEventCreateWithFlags(&p->order_ev, cudaEventDisableTiming) != cudaSuccess) {
    p->order_ev = nullptr;
    release(p);
    cudaGetLastError();
    return SWIFT_ERR_CUDA;
  }
  double a[512];
  float af[512];
  for (int l = 0; l < n_levels; ++l) {
    const int n = levels[l].n;
    taper_table(n, levels[l].apod, levels[l].tukey_alpha, a);
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
      s += a[k];
      af[k] = static_cast<float>(a[k]);
    }
    p->inv_sum_a[l] = 1.0 / (s * s);
    // the taper's transform, computed on the device from the FP32 taper (the
    // allocation-free path computes it with the same kernel)
    if (cudaMalloc(&p->taper[l], sizeof(float) * n) != cudaSuccess ||
        cudaMemcpy(p->taper[l], af, sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc(&p->ahat[l], sizeof(float) * n) != cudaSuccess ||
        swift::launch_taper_spectrum(n, levels[l].apod, levels[l].tukey_alpha, p->taper[l], p->ahat[l], nullptr) !=
            cudaSuccess ||
        cudaStreamSynchronize(nullptr) != cudaSuccess) {
      release(p);
      cudaGetLastError();
      return SWIFT_ERR_OOM;
    }
    // twiddle table W_n^{j m} = exp(-2 pi i j m / n), j < R1, m < R2, stored [m][j]
    const int slot = size_slot(n);
    if (!p->twiddle[slot]) {
      int r1 = 0, r2 = 0;
      swift::stream_radices(n, &r1, &r2);
      float2 tw[512];
      for (int i = 0; i < r1 * r2; ++i) tw[i] = swift::twiddle_entry(n, r1, i);
      if (cudaMalloc(&p->twiddle[slot], sizeof(float2) * n) != cudaSuccess ||
          cudaMemcpy(p->twiddle[slot], tw, sizeof(float2) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
        release(p);
        cudaGetLastError();
        return SWIFT_ERR_OOM;
      }
    }
    if (prec != SWIFT_PREC_FP32 && !p->tc_tab[slot]) {
      if (cudaMalloc(&p->tc_tab[slot], swift::tcf_table_bytes(n)) != cudaSuccess ||
          swift::tcf_build_tables(n, prec == SWIFT_PREC_FP16X2, p->tc_tab[slot]) != cudaSuccess) {
        release(p);
        cudaGetLastError();
        return SWIFT_ERR_OOM;
      }
    }
  }
  // workspace of the streaming forward path (also used by the tensor-core variant)
  // sized for the largest level, so any level can be switched to streaming
  size_t per = 0;
  for (int l = 0; l < n_levels; ++l) {
    p->sched[l] = default_sched(levels[l].n);
    const size_t b = swift::stream_bytes_per_window(levels[l].n);
    per = b > per ? b : per;
  }
  if (per > 0) {
    p->work_windows = max_windows < kStreamSlice ? max_windows : kStreamSlice;
    p->work_per = per;
    // room for kMaxLanes lanes of lane_cap windows each (together at least
    // the single-lane slice of work_windows)
    p->lane_cap = per * static_cast<size_t>(p->work_windows) <= kLaneBytes ? p->work_windows
                                                                         : lane_capacity(p->work_windows, kMaxLanes);
    const long long c = p->lane_cap;
    const size_t bytes = kMaxLanes * lane_stride(per, c) + 4096;
    if (cudaMalloc(&p->work, bytes) != cudaSuccess ||
        cudaMalloc(&p->done, sizeof(unsigned int) * kMaxLanes * c) != cudaSuccess ||
        cudaMemset(p->done, 0, sizeof(unsigned int) * kMaxLanes * c) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming) != cudaSuccess) {
      release(p);
      cudaGetLastError();
      return SWIFT_ERR_OOM;
    }
  }
  *out = p;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_destroy(swift_plan plan) { return release(plan); }

// levels a batch uses: all of the plan's when it carries a level array or
// level offsets, else level 0 only
static int batch_levels(swift_plan plan, const swift_batch* batch) {
  return (batch->level || batch->level_offsets) ? plan->n_levels : 1;
}

// window range [*b0, *b0 + *cnt) of level l: the whole batch, or the level's
// range of a batch sorted by level
static void level_range(const swift_batch* batch, int l, int64_t* b0, int64_t* cnt) {
  if (batch->level_offsets) {
    *b0 = batch->level_offsets[l];
    *cnt = batch->level_offsets[l + 1] - batch->level_offsets[l];
  } else {
    *b0 = 0;
    *cnt = batch->n_windows;
  }
}

static bool image_ok(const swift_image& im, int n, int patch_mode, int64_t B) {
  if (!im.data || im.count < 1) return false;
  if (patch_mode) {
    if (im.stride < static_cast<int64_t>(n) * n && B > 1) return false;
    return im.count == 1;
  }
  if (im.height < 1 || im.width < 1 || im.pitch < im.width) return false;
  if (im.count > 1 && im.stride < im.pitch * im.height) return false;
  return true;
}

// Launch description of level l of a forward batch (section or patch mode).
static swift::MatchLaunch level_launch_forward(swift_plan plan, const swift_batch* batch, int l, swift_result* out) {
  const int64_t B = batch->n_windows;
  const int pm = batch->patch_mode ? 1 : 0;
  const swift_level& lv = plan->levels[l];
  const swift_image& ri = batch->ref[l];
  const swift_image& mi = batch->mov[l];
  swift::MatchLaunch L;
  L.ref = ri.data;
  L.mov = mi.data;
  L.ref_pitch = pm ? lv.n : ri.pitch;
  L.mov_pitch = pm ? lv.n : mi.pitch;
  L.ref_stride = pm ? (ri.stride ? ri.stride : static_cast<long long>(lv.n) * lv.n) : ri.stride;
  L.mov_stride = pm ? (mi.stride ? mi.stride : static_cast<long long>(lv.n) * lv.n) : mi.stride;
  L.ref_h = ri.height;
  L.ref_w = ri.width;
  L.mov_h = mi.height;
  L.mov_w = mi.width;
  L.ref_count = ri.count;
  L.patch_mode = pm;
  L.ref_origin = batch->ref_origin;
  L.mov_origin = batch->mov_origin;
  L.level_idx = batch->level;
  L.level = l;
  L.n_windows = B;
  L.w = lv.whiten_exponent;
  const double r2 = static_cast<double>(lv.snr_exclusion_radius) * lv.snr_exclusion_radius;
  L.radius2 = static_cast<float>(floor(r2));
  L.inv_sum_a = plan->inv_sum_a[l];
  L.taper = plan->taper[l];
  L.ahat = plan->ahat[l];
  L.twiddle = plan->twiddle[size_slot(lv.n)];
  L.stall_tx = plan->test_stall ? 16u : 0u;
  L.stale_ok = plan->test_stale_ok ? 1 : 0;
  L.row_tma = plan->row_tma;
  L.out = out;
  if (batch->level_offsets) {
    // a batch sorted by level: this level's windows only, as a batch of their own
    int64_t b0 = 0, cnt = 0;
    level_range(batch, l, &b0, &cnt);
    const size_t es = plan->dtype == SWIFT_IN_U8 ? 1 : 4;
    if (pm) {
      L.ref = static_cast<const unsigned char*>(L.ref) + es * b0 * L.ref_stride;
      L.mov = static_cast<const unsigned char*>(L.mov) + es * b0 * L.mov_stride;
    } else {
      L.ref_origin += 2 * b0;
      L.mov_origin += 2 * b0;
    }
    L.out = out ? out + b0 : nullptr;
    L.level_idx = nullptr;
    L.n_windows = cnt;
  }
  return L;
}

// Slices of a level's B streaming windows over the call's lanes: one lane
// takes slices of the plan's full slice; two lanes split the level into
// about equal slices (at least kMinLaneSlice, at most lane_cap windows), lane
// k in its own part of the workspace and of the finalize counters.
struct LaneSlices {
  long long cap;       // windows per slice
  size_t stride;       // bytes between the lanes' workspace parts
  long long done_off;  // counters between the lanes' parts
};
static LaneSlices lane_slices(swift_plan plan, int lanes, long long B) {
  if (lanes <= 1) return {plan->work_windows, 0, 0};
  // a level is split only into slices of at least kMinLaneSlice windows (smaller
  // levels take one slice each and alternate between the lanes)
  long long cap = lane_capacity(B, lanes);
  if (cap < kMinLaneSlice) cap = kMinLaneSlice;
  if (cap > plan->lane_cap) cap = plan->lane_cap;
  if (cap < 1) cap = 1;
  return {cap, lane_stride(plan->work_per, plan->lane_cap), plan->lane_cap};
}

// Launch the windows of level l with the level's schedule (fused or
// streaming) over the call's lanes: each streaming slice (at most the lane
// capacity) and each fused launch goes to the least-loaded lane, a slice in
// that lane's part of the workspace.
static swift_status run_level(swift_plan plan, const swift_batch* batch, int l, swift_result* out, Lanes& ls) {
  const cudaStream_t st = ls.s[0];
  int64_t B0 = 0, B = 0;
  level_range(batch, l, &B0, &B);
  if (B == 0) return SWIFT_OK;
  const int pm = batch->patch_mode ? 1 : 0;
  const swift_level& lv = plan->levels[l];
  const swift_image& ri = batch->ref[l];
  const swift_image& mi = batch->mov[l];
  const swift::MatchLaunch L = level_launch_forward(plan, batch, l, out);
  if (plan->prec != SWIFT_PREC_FP32) {
    // the tensor-core schedule's slices spread over the lanes like the FP32 ones
    const bool fp16 = plan->prec == SWIFT_PREC_FP16X2;
    const LaneSlices sl = lane_slices(plan, ls.n, B);
    const long long cap = sl.cap;
    const size_t stride = sl.stride;
    for (long long b0 = 0; b0 < B; b0 += cap) {
      const long long cnt = (B - b0) < cap ? (B - b0) : cap;
      const int k = lane_pick(ls, static_cast<double>(cnt) * lv.n * lv.n);
      swift::StreamWork W = swift::stream_carve(static_cast<unsigned char*>(plan->work) + k * stride, cap, lv.n, b0, cnt);
      if (plan->timing) {
        const int set = plan->tcount++ % kTimingSets;
        plan->tkind[set] = 0;
        W.ev = plan->tev + 6 * set;
      }
      const swift::TcfLaunch T = swift::tcf_tables(plan->tc_tab[size_slot(lv.n)]);
      if (swift::launch_tcf(lv.n, plan->dtype, fp16, L, W, T, ls.s[k]) != cudaSuccess) return SWIFT_ERR_CUDA;
    }
    return SWIFT_OK;
  }
  if (plan->sched[l] != SWIFT_SCHED_FUSED) {
    const LaneSlices sl = lane_slices(plan, ls.n, B);
    const long long cap = sl.cap;
    const size_t stride = sl.stride;
    for (long long b0 = 0; b0 < B; b0 += cap) {
      const long long cnt = (B - b0) < cap ? (B - b0) : cap;
      const int k = lane_pick(ls, static_cast<double>(cnt) * lv.n * lv.n);
      swift::StreamWork W = swift::stream_carve(static_cast<unsigned char*>(plan->work) + k * stride, cap, lv.n, b0, cnt);
      W.done = plan->done + k * sl.done_off;
      if (plan->timing) {
        const int set = plan->tcount++ % kTimingSets;
        // the launcher folds the finalize into the inverse rows for n <= 256 and radii below 8 px
        // (kind bit 1), and the statistics into the rows for n <= 256 (kind bit 2)
        plan->tkind[set] = 8 | ((lv.n <= 256 && L.radius2 < 64.f) ? 1 : 0) |
                           (swift::stream_stats_folded(lv.n, L) ? 2 : 0);
        W.ev = plan->tev + 6 * set;
      }
      if (swift::launch_stream(lv.n, plan->dtype, L, W, ls.s[k]) != cudaSuccess) return SWIFT_ERR_CUDA;
    }
    return SWIFT_OK;
  }
  const bool bulk = plan->dtype == SWIFT_IN_U8 && !pm && ri.count == 1 &&
                    (reinterpret_cast<uintptr_t>(ri.data) % 16) == 0 &&
                    (reinterpret_cast<uintptr_t>(mi.data) % 16) == 0 && ri.pitch % 16 == 0 &&
                    mi.pitch % 16 == 0 && ri.width % 16 == 0 && mi.width % 16 == 0;
  const cudaStream_t fs = ls.s[lane_pick(ls, static_cast<double>(B) * lv.n * lv.n)];
  cudaEvent_t* ev = nullptr;
  if (plan->timing) {
    const int set = plan->tcount++ % kTimingSets;
    plan->tkind[set] = 1;
    ev = plan->tev + 6 * set;
    cudaEventRecord(ev[0], fs);
  }
  if (swift::launch_forward(lv.n, plan->dtype, bulk, L, fs) != cudaSuccess) return SWIFT_ERR_CUDA;
  if (ev) cudaEventRecord(ev[1], fs);
  return SWIFT_OK;
}

static swift_status check_warp_batch(swift_plan plan, const swift_batch* batch);
static swift_status warp_forward(swift_plan plan, const swift_batch* batch, swift_result* out, cudaStream_t st);

// Calls of one plan share its workspace.  A call that arrives on a stream
// other than the previous call's first makes its stream wait, on the device,
// for the previous call's work; every call then records the plan's event.
// Work being captured into a graph is left out (a capturing stream may not
// wait on an event recorded outside the capture); swift_plan_replay orders the
// graph's launches instead.
static swift_status order_begin(swift_plan p, cudaStream_t st, bool* captured) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return SWIFT_ERR_CUDA;
  }
  *captured = cs != cudaStreamCaptureStatusNone;
  if (*captured || !p->order_used || p->order_stream == st) return SWIFT_OK;
  if (cudaStreamWaitEvent(st, p->order_ev, 0) != cudaSuccess) {
    cudaGetLastError();
    return SWIFT_ERR_CUDA;
  }
  return SWIFT_OK;
}

static void order_end(swift_plan p, cudaStream_t st, bool captured) {
  if (captured) return;
  if (cudaEventRecord(p->order_ev, st) == cudaSuccess) {
    p->order_stream = st;
    p->order_used = true;
  }
}

// The levels of the batch with the persistent schedule, all in one launch.
static swift_status run_persistent(swift_plan plan, const swift_batch* batch, unsigned int mask, swift_result* out,
                                   cudaStream_t st) {
  const int64_t B = batch->n_windows;
  const int used_levels = batch_levels(plan, batch);
  swift::PersistLaunch P = {};
  P.n_levels = used_levels;
  P.level_mask = mask;
  P.B = B;
  P.level_idx = batch->level_offsets ? nullptr : batch->level;
  P.sorted = batch->level_offsets ? 1 : 0;
  for (int l = 0; l <= used_levels && batch->level_offsets; ++l) P.level_off[l] = batch->level_offsets[l];
  P.skew = plan->pskew;
  P.ring = persist_ring(plan->pskew);
  P.spin_limit = plan->phold >= 0 ? 20000000ll : plan->pspin;  // the test hook waits about 10 ms
  P.hold_s1 = plan->phold;
  P.nmax = 0;
  for (int l = 0; l < used_levels; ++l) {
    if (!((mask >> l) & 1u)) continue;
    swift_batch whole = *batch;
    whole.level_offsets = nullptr;  // the persistent kernel indexes the whole batch itself
    P.lv[l].L = level_launch_forward(plan, &whole, l, out);
    P.lv[l].n = plan->levels[l].n;
    P.nmax = plan->levels[l].n > P.nmax ? plan->levels[l].n : P.nmax;
  }
  for (int l = 0; l < used_levels; ++l)
    if (!((mask >> l) & 1u)) P.lv[l].n = P.nmax;  // not run: any built size
  // workspace, grown to the largest batch and ring seen (before any capture:
  // swift_plan_capture makes an uncaptured call first)
  const size_t need = swift::persist_bytes(used_levels, B, 256, persist_ring(kMaxSkew));
  if (need > plan->pwork_bytes) {
    bool captured = false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess) captured = cs != cudaStreamCaptureStatusNone;
    if (captured) return SWIFT_ERR_INVALID_ARG;  // a capture needs the same batch size as the call before it
    if (plan->pwork) {
      cudaStreamSynchronize(st);
      cudaFree(plan->pwork);
      plan->pwork = nullptr;
      plan->pwork_bytes = 0;
    }
    if (cudaMalloc(&plan->pwork, need) != cudaSuccess) {
      plan->pwork = nullptr;
      cudaGetLastError();
      return SWIFT_ERR_OOM;
    }
    plan->pwork_bytes = need;
  }
  cudaEvent_t* ev = nullptr;
  if (plan->timing) {
    const int set = plan->tcount++ % kTimingSets;
    plan->tkind[set] = 2;
    ev = plan->tev + 6 * set;
    cudaEventRecord(ev[0], st);
  }
  if (swift::launch_persist(P, plan->pwork, plan->dtype, st) != cudaSuccess) return SWIFT_ERR_CUDA;
  if (ev) cudaEventRecord(ev[1], st);
  return SWIFT_OK;
}

// the launches of one validated forward call
static swift_status match_launches(swift_plan plan, const swift_batch* batch, swift_result* out, cudaStream_t st) {
  if (batch->affine) return warp_forward(plan, batch, out, st);
  const int used_levels = batch_levels(plan, batch);
  Lanes ls;
  ls.s[0] = st;
  ls.s[1] = plan->aux;
  // forward calls spread over the lanes; the auxiliary lane first waits
  // for what the call's stream has queued (the fork) and the call's stream
  // finally waits for the auxiliary lane (the join), so the call stays one
  // ordered unit of its stream (and of a captured graph)
  ls.n = (plan->lanes > 1 && plan->aux) ? plan->lanes : 1;
  if (ls.n > 1 && (cudaEventRecord(plan->fork_ev, st) != cudaSuccess ||
                   cudaStreamWaitEvent(plan->aux, plan->fork_ev, 0) != cudaSuccess)) {
    cudaGetLastError();
    return SWIFT_ERR_CUDA;
  }
  unsigned int mask = 0;
  swift_status e = SWIFT_OK;
  for (int l = 0; l < used_levels && e == SWIFT_OK; ++l) {
    if (plan->prec == SWIFT_PREC_FP32 && plan->sched[l] == SWIFT_SCHED_PERSISTENT && has_persistent(plan->levels[l].n) &&
        batch->n_windows < (1ll << 24)) {
      mask |= 1u << l;
      continue;
    }
    e = run_level(plan, batch, l, out, ls);
  }
  if (e == SWIFT_OK && mask) e = run_persistent(plan, batch, mask, out, st);
  if (ls.n > 1 && (cudaEventRecord(plan->join_ev, plan->aux) != cudaSuccess ||
                   cudaStreamWaitEvent(st, plan->join_ev, 0) != cudaSuccess) && e == SWIFT_OK) {
    e = SWIFT_ERR_CUDA;
  }
  if (e != SWIFT_OK) return e;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  return SWIFT_OK;
}

extern "C" swift_status swift_match_batch(swift_plan plan, const swift_batch* batch, swift_result* out,
                                          void* stream) {
  if (!plan || !batch) return SWIFT_ERR_INVALID_ARG;
  const int64_t B = batch->n_windows;
  if (B < 0 || B > plan->max_windows) return SWIFT_ERR_INVALID_ARG;
  if (B == 0) return SWIFT_OK;
  if (!out || !batch->ref || !batch->mov) return SWIFT_ERR_INVALID_ARG;
  if (B * 4 > static_cast<int64_t>(0x7fffffff)) return SWIFT_ERR_INVALID_ARG;  // grid limit
  const int pm = batch->patch_mode ? 1 : 0;
  if (!pm && (!batch->ref_origin || !batch->mov_origin)) return SWIFT_ERR_INVALID_ARG;
  const int used_levels = batch_levels(plan, batch);
  for (int l = 0; l < used_levels; ++l) {
    const int n = plan->levels[l].n;
    if (!image_ok(batch->ref[l], n, pm, B) || !image_ok(batch->mov[l], n, pm, B)) return SWIFT_ERR_INVALID_ARG;
    if (batch->mov[l].count != 1) return SWIFT_ERR_INVALID_ARG;
  }
  if (batch->level_offsets) {
    const int64_t* o = batch->level_offsets;
    if (o[0] != 0 || o[plan->n_levels] != B) return SWIFT_ERR_INVALID_ARG;
    for (int l = 0; l < plan->n_levels; ++l)
      if (o[l + 1] < o[l]) return SWIFT_ERR_INVALID_ARG;
  }
  // report (and clear) an asynchronous failure left by earlier work
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  if (batch->affine) {
    const swift_status e = check_warp_batch(plan, batch);
    if (e != SWIFT_OK) return e;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool captured = false;
  const swift_status oe = order_begin(plan, st, &captured);
  if (oe != SWIFT_OK) return oe;
  const swift_status e = match_launches(plan, batch, out, st);
  order_end(plan, st, captured);
  return e;
}

// Launch description of level l (shared by the warp and backward paths).
static swift::MatchLaunch level_launch(swift_plan plan, const swift_batch* batch, int l, swift_result* out) {
  const swift_level& lv = plan->levels[l];
  const swift_image& ri = batch->ref[l];
  const swift_image& mi = batch->mov[l];
  swift::MatchLaunch L;
  L.ref = ri.data;
  L.mov = mi.data;
  L.ref_pitch = ri.pitch;
  L.mov_pitch = mi.pitch;
  L.ref_stride = ri.stride;
  L.mov_stride = mi.stride;
  L.ref_h = ri.height;
  L.ref_w = ri.width;
  L.mov_h = mi.height;
  L.mov_w = mi.width;
  L.ref_count = ri.count;
  L.patch_mode = 0;
  L.ref_origin = batch->ref_origin;
  L.mov_origin = batch->mov_origin;
  L.level_idx = batch->level;
  L.level = l;
  L.n_windows = batch->n_windows;
  L.w = lv.whiten_exponent;
  L.radius2 = static_cast<float>(floor(static_cast<double>(lv.snr_exclusion_radius) * lv.snr_exclusion_radius));
  L.inv_sum_a = plan->inv_sum_a[l];
  L.taper = plan->taper[l];
  L.twiddle = plan->twiddle[size_slot(lv.n)];
  L.stall_tx = plan->test_stall ? 16u : 0u;
  L.stale_ok = plan->test_stale_ok ? 1 : 0;
  L.out = out;
  L.pre_status = nullptr;
  return L;
}

// extra workspace of the warp / backward path, allocated on first use
static swift_status ensure_bwork(swift_plan plan) {
  if (plan->bwork) return SWIFT_OK;
  size_t per = 0;
  for (int l = 0; l < plan->n_levels; ++l) {
    const size_t b = swift::back_bytes_per_window(plan->levels[l].n);
    per = b > per ? b : per;
  }
  const long long cap = plan->max_windows < kBackSlice ? plan->max_windows : kBackSlice;
  if (cudaMalloc(&plan->bwork, per * cap + 16 * 4096) != cudaSuccess) {
    plan->bwork = nullptr;
    cudaGetLastError();
    return SWIFT_ERR_OOM;
  }
  if (cudaMalloc(&plan->gw_acc, sizeof(double) * kMaxLevels) != cudaSuccess) {
    cudaFree(plan->bwork);
    plan->bwork = nullptr;
    plan->gw_acc = nullptr;
    cudaGetLastError();
    return SWIFT_ERR_OOM;
  }
  plan->bwork_windows = cap;
  return SWIFT_OK;
}

// validation shared by the warp forward and the backward (section mode)
static swift_status check_warp_batch(swift_plan plan, const swift_batch* batch) {
  if (!plan || !batch) return SWIFT_ERR_INVALID_ARG;
  if (plan->prec != SWIFT_PREC_FP32) return SWIFT_ERR_UNSUPPORTED;  // warp / backward are FP32 only
  for (int l = 0; l < plan->n_levels; ++l)
    if (plan->levels[l].n > 256) return SWIFT_ERR_UNSUPPORTED;  // warp / backward are built up to 256 x 256
  const int64_t B = batch->n_windows;
  if (B < 0 || B > plan->max_windows) return SWIFT_ERR_INVALID_ARG;
  if (B == 0) return SWIFT_OK;
  if (batch->patch_mode || !batch->ref || !batch->mov || !batch->ref_origin || !batch->mov_origin)
    return SWIFT_ERR_INVALID_ARG;
  if (batch->level_offsets && !batch->level) return SWIFT_ERR_UNSUPPORTED;  // warped windows need the level array
  const int used = batch->level ? plan->n_levels : 1;
  for (int l = 0; l < used; ++l) {
    if (!image_ok(batch->ref[l], plan->levels[l].n, 0, B) || !image_ok(batch->mov[l], plan->levels[l].n, 0, B))
      return SWIFT_ERR_INVALID_ARG;
    if (batch->mov[l].count != 1 || batch->mov[l].height < 2 || batch->mov[l].width < 2) return SWIFT_ERR_INVALID_ARG;
  }
  return SWIFT_OK;
}

static swift_status warp_forward(swift_plan plan, const swift_batch* batch, swift_result* out, cudaStream_t st) {
  swift_status e = ensure_bwork(plan);
  if (e != SWIFT_OK) return e;
  const int used = batch->level ? plan->n_levels : 1;
  const long long B = batch->n_windows;
  for (int l = 0; l < used; ++l) {
    const swift::MatchLaunch L = level_launch(plan, batch, l, out);
    swift::BackLaunch K = {batch->affine, nullptr, nullptr, nullptr, nullptr};
    for (long long b0 = 0; b0 < B; b0 += plan->bwork_windows) {
      const long long cnt = (B - b0) < plan->bwork_windows ? (B - b0) : plan->bwork_windows;
      const swift::BackWork BW = swift::back_carve(plan->bwork, plan->bwork_windows, plan->levels[l].n, cnt);
      if (swift::launch_prepare(plan->levels[l].n, plan->dtype, L, K, BW, b0, st) != cudaSuccess ||
          swift::launch_prepared_forward(plan->levels[l].n, L, BW, b0, st) != cudaSuccess)
        return SWIFT_ERR_CUDA;
    }
  }
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  return SWIFT_OK;
}

static swift_status backward_launches(swift_plan plan, const swift_batch* batch, const float* grad_peak,
                                      const float* grad_snr, float* grad_affine, float* grad_w, cudaStream_t st);

extern "C" swift_status swift_match_backward(swift_plan plan, const swift_batch* batch, const float* grad_peak,
                                             const float* grad_snr, float* grad_affine, float* grad_w,
                                             void* stream) {
  swift_status e = check_warp_batch(plan, batch);
  if (e != SWIFT_OK) return e;
  const long long B = batch->n_windows;
  if (!grad_w) return SWIFT_ERR_INVALID_ARG;
  if (B > 0 && (!grad_peak || !grad_snr || !grad_affine)) return SWIFT_ERR_INVALID_ARG;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  if ((e = ensure_bwork(plan)) != SWIFT_OK) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool captured = false;
  if ((e = order_begin(plan, st, &captured)) != SWIFT_OK) return e;
  e = backward_launches(plan, batch, grad_peak, grad_snr, grad_affine, grad_w, st);
  order_end(plan, st, captured);
  return e;
}

// the launches of one validated backward call
static swift_status backward_launches(swift_plan plan, const swift_batch* batch, const float* grad_peak,
                                      const float* grad_snr, float* grad_affine, float* grad_w, cudaStream_t st) {
  const long long B = batch->n_windows;
  if (cudaMemsetAsync(plan->gw_acc, 0, sizeof(double) * kMaxLevels, st) != cudaSuccess) return SWIFT_ERR_CUDA;
  const int used = batch->level ? plan->n_levels : 1;
  for (int l = 0; l < used && B > 0; ++l) {
    const swift::MatchLaunch L = level_launch(plan, batch, l, nullptr);
    const swift::BackLaunch K = {batch->affine, grad_peak, grad_snr, grad_affine, plan->gw_acc + l};
    for (long long b0 = 0; b0 < B; b0 += plan->bwork_windows) {
      const long long cnt = (B - b0) < plan->bwork_windows ? (B - b0) : plan->bwork_windows;
      const swift::BackWork BW = swift::back_carve(plan->bwork, plan->bwork_windows, plan->levels[l].n, cnt);
      if (swift::launch_prepare(plan->levels[l].n, plan->dtype, L, K, BW, b0, st) != cudaSuccess ||
          swift::launch_backward(plan->levels[l].n, plan->dtype, L, K, BW, b0, st) != cudaSuccess)
        return SWIFT_ERR_CUDA;
    }
  }
  if (swift::launch_wout(plan->gw_acc, grad_w, plan->n_levels, st) != cudaSuccess) return SWIFT_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return SWIFT_ERR_CUDA;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_set_schedule(swift_plan plan, int32_t level, int32_t schedule) {
  if (!plan || level < 0 || level >= plan->n_levels) return SWIFT_ERR_INVALID_ARG;
  const int n = plan->levels[level].n;
  if (schedule == SWIFT_SCHED_DEFAULT) {
    plan->sched[level] = default_sched(n);
  } else if (schedule == SWIFT_SCHED_FUSED || schedule == SWIFT_SCHED_STREAM || schedule == SWIFT_SCHED_PERSISTENT) {
    if (schedule == SWIFT_SCHED_FUSED && !has_fused(n)) return SWIFT_ERR_UNSUPPORTED;
    if (schedule == SWIFT_SCHED_PERSISTENT && !has_persistent(n)) return SWIFT_ERR_UNSUPPORTED;
    plan->sched[level] = schedule;
  } else {
    return SWIFT_ERR_INVALID_ARG;
  }
  return SWIFT_OK;
}

// time `reps` forward calls of the batch on `st` (after one warm-up call)
static swift_status time_calls(swift_plan plan, const swift_batch* batch, swift_result* out, cudaStream_t st,
                               cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  swift_status e = match_launches(plan, batch, out, st);  // warm-up
  if (e != SWIFT_OK) return e;
  cudaEventRecord(e0, st);
  for (int rep = 0; rep < 3 && e == SWIFT_OK; ++rep) e = match_launches(plan, batch, out, st);
  cudaEventRecord(e1, st);
  if (e != SWIFT_OK) return e;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) return SWIFT_ERR_CUDA;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_autotune(swift_plan plan, const swift_batch* batch, swift_result* out,
                                            void* stream, int32_t* chosen) {
  if (!plan || !batch) return SWIFT_ERR_INVALID_ARG;
  if (batch->affine) return SWIFT_ERR_INVALID_ARG;
  // run once with the current schedules: validates the batch and does the set-up
  swift_status e = swift_match_batch(plan, batch, out, stream);
  if (e != SWIFT_OK) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return SWIFT_ERR_CUDA;
  }
  const int used = batch_levels(plan, batch);
  // (a) per level: the faster of the fused and streaming schedules, each
  // level timed alone
  int per_level[kMaxLevels];
  for (int l = 0; l < used && e == SWIFT_OK; ++l) {
    float best = 3.4e38f;
    per_level[l] = SWIFT_SCHED_STREAM;
    for (int s : {SWIFT_SCHED_FUSED, SWIFT_SCHED_STREAM}) {
      if (s == SWIFT_SCHED_FUSED && !has_fused(plan->levels[l].n)) continue;
      plan->sched[l] = s;
      Lanes one;
      one.s[0] = st;
      if ((e = run_level(plan, batch, l, out, one)) != SWIFT_OK) break;  // warm-up
      cudaEventRecord(e0, st);
      for (int rep = 0; rep < 3 && e == SWIFT_OK; ++rep) e = run_level(plan, batch, l, out, one);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (e != SWIFT_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        e = SWIFT_ERR_CUDA;
        break;
      }
      if (ms < best) {
        best = ms;
        per_level[l] = s;
      }
    }
  }
  float best_ms = 3.4e38f;
  int best_skew = plan->pskew;
  bool best_persist = false;
  if (e == SWIFT_OK) {
    for (int l = 0; l < used; ++l) plan->sched[l] = per_level[l];
    e = time_calls(plan, batch, out, st, e0, e1, &best_ms);
  }
  // (b) every level that has it in one persistent launch, for each skew of
  // its work order (ring and L2 working set grow with the skew)
  bool any = false;
  for (int l = 0; l < used; ++l) any = any || (plan->prec == SWIFT_PREC_FP32 && has_persistent(plan->levels[l].n));
  for (int k = 0; any && e == SWIFT_OK && k < static_cast<int>(sizeof(kSkews) / sizeof(kSkews[0])); ++k) {
    for (int l = 0; l < used; ++l) plan->sched[l] = has_persistent(plan->levels[l].n) ? SWIFT_SCHED_PERSISTENT : per_level[l];
    plan->pskew = kSkews[k];
    float ms = 0.f;
    if ((e = time_calls(plan, batch, out, st, e0, e1, &ms)) != SWIFT_OK) break;
    if (ms < best_ms) {
      best_ms = ms;
      best_skew = kSkews[k];
      best_persist = true;
    }
  }
  for (int l = 0; l < used; ++l)
    plan->sched[l] = best_persist && has_persistent(plan->levels[l].n) ? SWIFT_SCHED_PERSISTENT : per_level[l];
  plan->pskew = best_skew;
  // (c) one lane or two for the chosen schedules
  if (e == SWIFT_OK && plan->aux) {
    float lane_ms[kMaxLanes + 1] = {};
    int best_lanes = plan->lanes;
    for (int k = 1; k <= kMaxLanes && e == SWIFT_OK; ++k) {
      plan->lanes = k;
      e = time_calls(plan, batch, out, st, e0, e1, &lane_ms[k]);
      if (e == SWIFT_OK && (k == 1 || lane_ms[k] < lane_ms[best_lanes])) best_lanes = k;
    }
    plan->lanes = best_lanes;
  }
  if (chosen)
    for (int l = 0; l < used; ++l) chosen[l] = plan->sched[l];
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != SWIFT_OK) return e;
  // leave `out` holding the results of the chosen schedules
  return swift_match_batch(plan, batch, out, stream);
}

extern "C" swift_status swift_plan_capture(swift_plan plan, const swift_batch* batch, swift_result* out,
                                           void* stream) {
  if (!plan || !batch || !stream) return SWIFT_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // an uncaptured call first: checks the batch and does every one-time set-up
  swift_status e = swift_match_batch(plan, batch, out, stream);
  if (e != SWIFT_OK) return e;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SWIFT_ERR_CUDA;
  if (plan->graph_exec) cudaGraphExecDestroy(plan->graph_exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  plan->graph_exec = nullptr;
  plan->graph = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SWIFT_ERR_CUDA;
  e = swift_match_batch(plan, batch, out, stream);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(st, &g);
  if (e != SWIFT_OK || ce != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return e != SWIFT_OK ? e : SWIFT_ERR_CUDA;
  }
  cudaGraphExec_t x = nullptr;
  if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return SWIFT_ERR_CUDA;
  }
  plan->graph = g;
  plan->graph_exec = x;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_replay(swift_plan plan, void* stream) {
  if (!plan || !plan->graph_exec) return SWIFT_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool captured = false;
  const swift_status oe = order_begin(plan, st, &captured);
  if (oe != SWIFT_OK) return oe;
  const cudaError_t ge = cudaGraphLaunch(plan->graph_exec, st);
  order_end(plan, st, captured);
  if (ge != cudaSuccess) {
    cudaGetLastError();
    return SWIFT_ERR_CUDA;
  }
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_set_test_stall(swift_plan plan, int32_t enable) {
  if (!plan) return SWIFT_ERR_INVALID_ARG;
  plan->test_stall = enable != 0;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_set_skew(swift_plan plan, int32_t skew) {
  if (!plan || skew < 1 || skew > kMaxSkew) return SWIFT_ERR_INVALID_ARG;
  plan->pskew = skew;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_set_lanes(swift_plan plan, int32_t lanes) {
  if (!plan || lanes < 1 || lanes > kMaxLanes) return SWIFT_ERR_INVALID_ARG;
  if (lanes > 1 && !plan->aux) return SWIFT_ERR_INVALID_ARG;  // no streaming workspace: nothing to spread
  plan->lanes = lanes;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_get_lanes(swift_plan plan, int32_t* lanes) {
  if (!plan || !lanes) return SWIFT_ERR_INVALID_ARG;
  *lanes = plan->aux ? plan->lanes : 1;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_set_row_tma(swift_plan plan, int32_t mode) {
  if (!plan || mode < 0 || mode > 2) return SWIFT_ERR_INVALID_ARG;
  plan->row_tma = mode;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_get_row_tma(swift_plan plan, int32_t* mode) {
  if (!plan || !mode) return SWIFT_ERR_INVALID_ARG;
  *mode = plan->row_tma;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_set_test_hold(swift_plan plan, int64_t window) {
  if (!plan || window < -1) return SWIFT_ERR_INVALID_ARG;
  plan->phold = window;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_set_test_stale_status(swift_plan plan, int32_t enable) {
  if (!plan) return SWIFT_ERR_INVALID_ARG;
  plan->test_stale_ok = enable != 0;
  return SWIFT_OK;
}

extern "C" int32_t swift_window_check(int32_t n, int32_t level, int32_t want_level, const int32_t* ref_origin,
                                      const int32_t* mov_origin, int32_t ref_h, int32_t ref_w, int32_t mov_h,
                                      int32_t mov_w) {
  if (!ref_origin || !mov_origin || n < 1) return SWIFT_WIN_OUT_OF_BOUNDS;
  return swift::window_check(n, level, want_level, ref_origin[0], ref_origin[1], mov_origin[0], mov_origin[1], ref_h,
                             ref_w, mov_h, mov_w);
}

extern "C" swift_status swift_plan_set_timing(swift_plan plan, int32_t enable) {
  if (!plan) return SWIFT_ERR_INVALID_ARG;
  if (enable && !plan->tev) {
    plan->tev = new (std::nothrow) cudaEvent_t[6 * kTimingSets];
    plan->tkind = new (std::nothrow) int[kTimingSets];
    if (!plan->tev || !plan->tkind) {
      delete[] plan->tev;
      delete[] plan->tkind;
      plan->tev = nullptr;
      plan->tkind = nullptr;
      return SWIFT_ERR_OOM;
    }
    for (int i = 0; i < 6 * kTimingSets; ++i) {
      if (cudaEventCreate(&plan->tev[i]) != cudaSuccess) {
        for (int k = 0; k < i; ++k) cudaEventDestroy(plan->tev[k]);
        delete[] plan->tev;
        delete[] plan->tkind;
        plan->tev = nullptr;
        plan->tkind = nullptr;
        cudaGetLastError();
        return SWIFT_ERR_CUDA;
      }
    }
  }
  plan->timing = enable != 0;
  plan->tcount = 0;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_timings(swift_plan plan, float* kernel_ms, int32_t* launches) {
  if (!plan || !kernel_ms || !launches) return SWIFT_ERR_INVALID_ARG;
  for (int k = 0; k < 8; ++k) {
    kernel_ms[k] = 0.f;
    launches[k] = 0;
  }
  if (!plan->tev) return SWIFT_OK;
  const int used = plan->tcount < kTimingSets ? plan->tcount : kTimingSets;
  for (int set = 0; set < used; ++set) {
    cudaEvent_t* ev = plan->tev + 6 * set;
    const int kind = plan->tkind[set];
    const bool streaming = kind == 0 || (kind & 8);
    const int nk = streaming ? 5 : 1;  // 1: fused launch, 2: persistent launch
    if (cudaEventSynchronize(ev[nk]) != cudaSuccess) return SWIFT_ERR_CUDA;
    for (int k = 0; k < nk; ++k) {
      // no finalize / statistics kernel ran between these events
      if (((kind & 8) && (kind & 1) && k == 4) || ((kind & 8) && (kind & 2) && k == 0)) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) != cudaSuccess) return SWIFT_ERR_CUDA;
      const int slot = streaming ? k : (kind == 1 ? 5 : 6);
      kernel_ms[slot] += ms;
      launches[slot] += 1;
    }
  }
  plan->tcount = 0;
  return SWIFT_OK;
}

extern "C" swift_status swift_plan_set_whitening(swift_plan plan, int32_t level, float w) {
  if (!plan || level < 0 || level >= plan->n_levels || !(w >= 0.f && w <= 1.f)) return SWIFT_ERR_INVALID_ARG;
  plan->levels[level].whiten_exponent = w;
  return SWIFT_OK;
}

extern "C" const char* swift_status_string(swift_status s) {
  switch (s) {
    case SWIFT_OK:
      return "SWIFT_OK";
    case SWIFT_ERR_INVALID_ARG:
      return "SWIFT_ERR_INVALID_ARG";
    case SWIFT_ERR_UNSUPPORTED:
      return "SWIFT_ERR_UNSUPPORTED";
    case SWIFT_ERR_CUDA:
      return "SWIFT_ERR_CUDA";
    case SWIFT_ERR_OOM:
      return "SWIFT_ERR_OOM";
    case SWIFT_ERR_TIMEOUT:
      return "SWIFT_ERR_TIMEOUT";
    case SWIFT_ERR_CAPACITY:
      return "SWIFT_ERR_CAPACITY";
  }
  return "SWIFT_ERR_UNKNOWN";
}

extern "C" const char* swift_version(void) { return "swift-gb300 0.1 sm_103a"; }
