// Internal launch descriptors shared by the host API and the kernels.
#pragma once
#include <cuda.h>  // CUtensorMap (the structure; the encoder is fetched at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/swift.h"

namespace swift {

// ---------------------------------------------------------------------------
// Window guard.  Window b of a launch may be read only when it belongs to the
// launch's level and, in section mode, both n x n windows lie inside their
// images.  Every kernel that turns an origin into an address evaluates this
// itself from the level and origin arrays (a few integer compares per CTA), so
// no status word in a shared workspace ever decides whether a read is made.
// ---------------------------------------------------------------------------
constexpr int kWindowOtherLevel = -1;  // window of another level: skipped, no result written

__host__ __device__ inline bool window_inside(int n, int y, int x, int h, int w) {
  return y >= 0 && x >= 0 && y <= h - n && x <= w - n;
}

// SWIFT_WIN_OK, SWIFT_WIN_OUT_OF_BOUNDS or kWindowOtherLevel
__host__ __device__ inline int window_check(int n, int level, int want_level, int ry, int rx, int my, int mx,
                                            int ref_h, int ref_w, int mov_h, int mov_w) {
  if (level != want_level) return kWindowOtherLevel;
  return window_inside(n, ry, rx, ref_h, ref_w) && window_inside(n, my, mx, mov_h, mov_w) ? SWIFT_WIN_OK
                                                                                          : SWIFT_WIN_OUT_OF_BOUNDS;
}

// ---------------------------------------------------------------------------
// Per-level tables, shared by the plan (built on the host) and the
// allocation-free entry point (built on the device).
// ---------------------------------------------------------------------------
// 1D taper in FP64 (Sec. III: cosine taper).  Periodic convention: Hann is
// a[k] = (1 - cos(2 pi k / n)) / 2; Tukey(alpha) has raised-cosine ramps of
// alpha*n/2 samples at each edge and is 1 in between; NONE is 1.
__host__ __device__ inline double taper_value(int n, int apod, double alpha, int k) {
  if (apod == SWIFT_APOD_NONE) return 1.0;
  if (apod == SWIFT_APOD_HANN) alpha = 1.0;
  const double ramp = alpha * n / 2.0;
  const double pi = 3.14159265358979323846;
  if (k < ramp) return 0.5 * (1.0 - cos(pi * k / ramp));
  if (k > n - ramp) return 0.5 * (1.0 - cos(pi * (n - k) / ramp));
  return 1.0;
}

// Entry i of the streaming kernels' twiddle table, stored [m][j] (j < r1):
// W_n^(j m) = exp(-2 pi i (j m mod n) / n), rounded to FP32.
__host__ __device__ inline float2 twiddle_entry(int n, int r1, int i) {
  const int j = i % r1, m = i / r1;
  const double ang = -2.0 * 3.14159265358979323846 * ((j * m) % n) / n;
  return make_float2(static_cast<float>(cos(ang)), static_cast<float>(sin(ang)));
}

// Everything one forward launch needs, passed by value as the kernel argument.
struct MatchLaunch {
  const void* ref;  // reference image (or first of ref_count sections)
  const void* mov;  // moving image
  long long ref_pitch, mov_pitch;    // elements between rows
  long long ref_stride, mov_stride;  // elements between stacked sections / patches
  int ref_h, ref_w, mov_h, mov_w;    // image sizes (section mode)
  int ref_count;                     // sections averaged into the reference (>= 1)
  int patch_mode;                    // 1: window b is the patch at data + b * stride
  const int* ref_origin;             // [B][2] (y, x), section mode
  const int* mov_origin;
  const int* level_idx;              // [B] or null
  int level;                         // windows of this level only (when level_idx != null)
  long long n_windows;
  float w;                           // whitening exponent
  float radius2;                     // floor(r^2): background iff dy^2 + dx^2 > radius2
  double inv_sum_a;                  // 1 / sum over the window of the 2D taper
  const float* taper;                // [n] 1D taper
  const float2* twiddle;             // [R2][R1] forward W_n^{j m}
  const float* ahat = nullptr;       // [n] DFT of the 1D taper (real: the taper is symmetric), or null
  swift_result* out;                 // [B]
  const int* pre_status = nullptr;   // [slice] status decided before the statistics (or null)
  unsigned int stall_tx = 0;         // test hook: bytes the row staging copies wait for that never arrive
  int row_tma = 1;                   // uint8 section rows through tensor maps: 0 never, 1 windows whose
                                     // rows start off a 16-byte boundary, 2 every window (RowMaps)
  int stale_ok = 0;                  // test hook: statistics report OK for windows of other levels
};

// Tensor maps of the row kernel's uint8 window tiles, one per section image:
// the image seen as [height][width / 16][16] bytes (row stride the pitch),
// box [RB][n / 16 + 1][16], i.e. the RB rows of a row block from the 16-byte
// chunk that holds the window's first column through the chunk after its
// last, into shared memory rows of n + 16 bytes.  The copy's innermost
// coordinate is always 0 (16-byte aligned whatever the origin); the kernel
// reads the window from byte x mod 16 of each row.  Needs 16-byte aligned
// data, pitch and width (else `on` stays 0 and the rows load without them).
struct RowMaps {
  CUtensorMap mov, ref;
  int on;   // 1: both maps hold
  int all;  // 1: every window loads through the maps; 0: only windows whose rows start off a 16-byte boundary
};

// Workspace of the streaming forward path for one slice of windows.
struct StreamWork {
  float4* stats;             // [S] (mu_m, mu_r, status bits, unused)
  float2* zr;                // [S][n][n] row spectra; reused for the match response (float [n][n])
  float2* h;                 // [S][n][n/2] inverse-column output
  unsigned long long* part;  // [S][blocks][3] block argmax key, FP64 sum of s, FP64 sum of s^2
  long long b0;              // first window of the slice
  long long count;           // windows in the slice
  cudaEvent_t* ev = nullptr; // host: 6 events recorded around the five kernels (timing), or null
  unsigned int* done = nullptr;  // [S] finished inverse-row blocks per window (zero between calls), or
                                 // null: the finalize then runs as a kernel of its own
  float* rstat = nullptr;        // [S][n / RB][8] row-block statistics records (stream_carve)
};

// Whether a plain FP32 forward slice of n x n windows runs without the
// statistics kernel: the row kernel records each block's sums and flatness,
// and the column-pair kernel removes the means in the spectrum (needs the
// taper's transform, MatchLaunch::ahat).
inline bool stream_stats_folded(int n, const MatchLaunch& L) {
  return n <= 256 && L.ahat != nullptr && L.pre_status == nullptr;
}

// The DFT of a level's 1D taper, Ahat[k] = sum_j a[j] cos(2 pi j k / n) (the
// sine part vanishes: the periodic taper is symmetric), for k < n, into a
// device array: closed forms for no taper (n at k = 0) and the Hann taper
// (n / 2 at 0, -n / 4 at +-1, 0 elsewhere), else the FP32 sum over j in order
// with cos from cospif.  One kernel on `stream`; the plan path and the
// allocation-free path both call it, so their tables are equal.
cudaError_t launch_taper_spectrum(int n, int apod, float alpha, const float* taper, float* out, cudaStream_t stream);
// the same in one CTA (threads tid of nth); cos_tab: n floats of shared
// memory; the taper must be visible to the whole CTA
__device__ __forceinline__ void taper_spectrum(int n, int apod, float alpha, const float* taper, float* out,
                                               float* cos_tab, int tid, int nth) {
  const bool hann = apod == SWIFT_APOD_HANN || (apod == SWIFT_APOD_TUKEY && alpha >= 1.f);
  if (apod == SWIFT_APOD_NONE || hann) {
    for (int k = tid; k < n; k += nth) {
      float v = 0.f;
      if (apod == SWIFT_APOD_NONE) {
        v = k == 0 ? static_cast<float>(n) : 0.f;
      } else if (k == 0) {
        v = 0.5f * static_cast<float>(n);
      } else if (k == 1 || k == n - 1) {
        v = -0.25f * static_cast<float>(n);
      }
      out[k] = v;
    }
    return;
  }
  for (int m = tid; m < n; m += nth) cos_tab[m] = cospif(2.f * static_cast<float>(m) / static_cast<float>(n));
  __syncthreads();
  for (int k = tid; k < n; k += nth) {
    float acc = 0.f;
    for (int j = 0; j < n; ++j) acc = fmaf(taper[j], cos_tab[(j * k) & (n - 1)], acc);
    out[k] = acc;
  }
}

// streaming forward path (swim_stream.cu): bytes of workspace per window, launch of one slice
size_t stream_bytes_per_window(int n);
StreamWork stream_carve(void* base, long long capacity, int n, long long b0, long long count);
cudaError_t launch_stream(int n, swift_dtype dtype, const MatchLaunch& L, const StreamWork& W, cudaStream_t stream);

// Extra workspace of the affine-warp forward and the backward pass (one slice).
// The backward reuses the forward's H for the inverse-column output of dL/dM
// and Zr (as float [n][n]) for dL/dm'.
struct BackWork {
  StreamWork fw;   // forward workspace
  float* mp;       // [S][n][n] prepared moving windows (affine-resampled)
  float* rp;       // [S][n][n] prepared reference windows (gathered / projected)
  int* pre_status; // [S] bounds / level decided by the preparation kernel
  float2* cr;      // [S][2][n][n/2+1] C = M conj(R) and R, kx in [0, n/2]
  double* bst;     // [S][8] mu_bg, sigma_bg, snr, peak, py, px, status, n_bg
  float2* gr;      // [S][n][n/2+1] row spectra of dL/ds
  double* gwp;     // [S][blocks] partial dL/dw
  double* gsum;    // [S][blocks] partial sum of A dL/dm'
  double* gwin;    // [S] dL/dw of each window
};

struct BackLaunch {
  const float* affine;     // [B][6] (a_yy, a_yx, t_y, a_xy, a_xx, t_x) or null (identity)
  const float* grad_peak;  // [B]
  const float* grad_snr;   // [B]
  float* grad_affine;      // [B][6]
  double* gw_acc;          // accumulated dL/dw of this level (device, one double)
};

// affine-warp forward and backward (swim_backward.cu)
size_t back_bytes_per_window(int n);
BackWork back_carve(void* base, long long capacity, int n, long long count);
// prepare windows (resample / gather) for a slice [b0, b0 + count) of the batch
cudaError_t launch_prepare(int n, swift_dtype dtype, const MatchLaunch& L, const BackLaunch& K, const BackWork& BW,
                           long long b0, cudaStream_t stream);
// forward on the prepared windows (results to L.out)
cudaError_t launch_prepared_forward(int n, const MatchLaunch& L, const BackWork& BW, long long b0,
                                    cudaStream_t stream);
// backward on the prepared windows (accumulates into K.gw_acc, writes K.grad_affine)
cudaError_t launch_backward(int n, swift_dtype dtype, const MatchLaunch& L, const BackLaunch& K, const BackWork& BW,
                            long long b0, cudaStream_t stream);

// tensor-core precision variant (swim_tcf.cu): tables per window size, and
// the five-kernel schedule on the streaming workspace
struct TcfLaunch {
  const uint32_t* frag;  // [32][40] per-lane constant DFT fragments (hi / lo)
  const float2* tw;      // [n] W_n^m = exp(-2 pi i m / n)
};
size_t tcf_table_bytes(int n);
cudaError_t tcf_build_tables(int n, bool fp16, void* dst);
TcfLaunch tcf_tables(const void* dst);
cudaError_t launch_tcf(int n, swift_dtype dtype, bool fp16, const MatchLaunch& L, const StreamWork& W,
                       const TcfLaunch& T, cudaStream_t stream);

// persistent forward schedule (swim_persist.cu): every window of the levels
// in one launch; bytes of its workspace, and the launch (the launch
// description's workspace pointers are filled in from `work`)
constexpr int kPersistMaxLevels = 16;
constexpr int kPersistStages = 5;
constexpr int kPersistPartStride = 24;  // u64 partials per window (NB3 <= 8, three each)
constexpr int kPersistRowBlocks = 16;   // row blocks per window (n / RB <= 16 up to 256 x 256)
constexpr int kCompactWindows = 2048;   // windows per compaction item
struct PersistLevel {
  MatchLaunch L;  // the level's launch (tables, images, origins, results)
  int n;          // window side (64, 128, 256)
};

struct PersistLaunch {
  PersistLevel lv[kPersistMaxLevels];
  int n_levels;
  int ring, skew;                // RING slots (shared by the levels), skew D (RING > 4 D)
  long long B;                   // windows in the batch
  const int* level_idx;          // [B] or null (every window is level 0)
  unsigned int level_mask;       // levels run by this launch (bit l)
  int sorted;                    // windows sorted by level: level l is [level_off[l], level_off[l + 1])
  long long level_off[kPersistMaxLevels + 1];
  int* lists;                    // [n_levels][B] window indices per level
  unsigned int* lcount;          // [kPersistMaxLevels] windows per level
  float4* stats;                 // [B]
  unsigned long long* part;      // [B][kPersistPartStride]
  float* rstat;                  // [B][kPersistRowBlocks][8] row-block statistics records
  float2* zr;                    // ring [RING][nmax][nmax] row spectra
  float2* h;                     // ring [RING][nmax][nmax/2] inverse-column output
  int nmax;                      // largest window side of the launch
  unsigned long long* slot;      // [RING] tag (bits 40-63: window + 1) and per-stage counts (8 bits each)
  unsigned int* queue;           // next item
  unsigned int* comp_done;       // compaction items done
  unsigned int* abort;           // nonzero once a wait ran out
  int n_compact;                 // compaction items (0 without a level array)
  long long spin_limit;          // clock cycles a wait may take
  long long hold_s1;             // test hook: window (sequence position) whose S1 items never signal, or -1
};

size_t persist_bytes(int n_levels, long long B, int nmax, int ring);
cudaError_t launch_persist(PersistLaunch P, void* work, swift_dtype dtype, cudaStream_t stream);

// float32 copy of the accumulated dL/dw of n levels
cudaError_t launch_wout(const double* acc, float* out, int n, cudaStream_t stream);

// forward launchers (one per window size), defined in swim_forward.cu
// bulk: stage uint8 section rows with cp.async.bulk (needs 16-byte aligned
// base pointers, pitches and widths, and a single reference section)
cudaError_t launch_forward(int n, swift_dtype dtype, bool bulk, const MatchLaunch& L, cudaStream_t stream);
// radix split (R1, R2) used by the kernel for window size n; false if n is not built
// radices (R1, R2) of the streaming kernels' 1D transforms, n = R1 R2
bool stream_radices(int n, int* r1, int* r2);
bool forward_radices(int n, int* r1, int* r2);

}  // namespace swift
