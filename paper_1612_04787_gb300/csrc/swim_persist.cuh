// Persistent forward schedule: every window of every level of a batch in one
// launch.
//
// The five steps of the streaming schedule (statistics S0, rows S1, column
// pairs S2, inverse rows S3, finalize S4) become work items of one kernel.
// CTAs claim items in a fixed global order from an atomic counter and run
// the same stage functions as the five-kernel schedule, so every window's
// results equal that schedule's bit for bit.  An item waits for the items it
// depends on through per-slot completion counters:
//
//   S0(j)  after S4 of the window that last used j's ring slot
//   S1(j)  after S0(j)              S2(j)  after all S1(j)
//   S3(j)  after all S2(j)          S4(j)  after all S3(j)
//
// The levels' windows form one sequence (level 0's list, then level 1's, ...);
// window g of it uses ring slot g mod RING for its row spectra Zr and
// inverse-column output H (sized for the largest window).  Each slot has one
// 64-bit word: the tag g + 1 of its current window and that window's count
// of finished items per stage.  Within a level the order is skewed: stage k
// of the level's j-th window sits at time j + k D, items sorted by time (later
// stages first within a time), and the levels follow one another.  Every item
// therefore depends only on items earlier in the order (RING > 4 D), and since
// a CTA only claims an item while it runs, the earliest unfinished item always
// has its inputs: the schedule cannot deadlock, whether or not all CTAs are
// resident.  With D of a dozen steps the items in flight span a few dozen
// windows, so a window's Zr and H (768 KB at 256 x 256) are written and read
// back within L2.
//
// Windows with a level array are first gathered into per-level lists by the
// leading "compaction" items (atomics on per-level counts); every pipeline
// item waits until they are done.  Every wait is bounded (spin_limit clock
// cycles): a wait that runs out raises the launch's abort flag, after which
// every later wait returns at once, stages do no work, and each finalize item
// writes SWIFT_WIN_TIMEOUT for its window.  Nothing waits without a bound.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "swim_stream.cuh"

namespace swift {


// items per window and stage at window size N
template <int N>
struct PersistItems {
  static constexpr int n1 = N / StreamGeom<N>::RB;
  static constexpr int n2 = PairGeom<N>::NB;
  static constexpr int n3 = StreamGeom<N>::NB3;
};

__host__ __device__ inline void persist_stage_items(int n, int (&nk)[kPersistStages]) {
  // matches PersistItems<N> for the built sizes
  nk[0] = 1;
  nk[4] = 1;
  if (n == 256) {
    nk[1] = 16, nk[2] = 8, nk[3] = 8;
  } else if (n == 128) {
    nk[1] = 4, nk[2] = 2, nk[3] = 2;
  } else {
    nk[1] = 2, nk[2] = 1, nk[3] = 1;
  }
}

// items of a level with C windows whose time (j + k D) is below tau
__host__ __device__ inline long long persist_items_before(long long tau, long long C, int D,
                                                          const int (&nk)[kPersistStages]) {
  long long f = 0;
  for (int k = 0; k < kPersistStages; ++k) {
    long long c = tau - static_cast<long long>(k) * D;
    c = c < 0 ? 0 : (c > C ? C : c);
    f += nk[k] * c;
  }
  return f;
}

// item i (0 <= i < C * sum(nk)) of a level -> stage k, sub-block, window j.
// Between the fill and the drain (4 D <= time <= C) every time holds S =
// sum(nk) items, so there the time is one division; the binary search covers
// the fill and the drain.
__host__ __device__ inline void persist_decode(long long i, long long C, int D, const int (&nk)[kPersistStages],
                                               int* stage, int* sub, long long* j) {
  const long long S = nk[0] + nk[1] + nk[2] + nk[3] + nk[4];
  const long long K1 = nk[1] + 2 * nk[2] + 3 * nk[3] + 4 * nk[4];  // sum of k nk[k]
  const long long fill = static_cast<long long>(kPersistStages - 1) * D;
  long long lo;
  if (C > fill && i >= S * fill - D * K1 && i < S * C - D * K1) {
    lo = (i + D * K1) / S;  // F(t) = S t - D K1 there
  } else {
    lo = 0;
    long long hi = C + fill;  // time in [lo, hi)
    while (hi - lo > 1) {
      const long long mid = (lo + hi) / 2;
      if (persist_items_before(mid, C, D, nk) <= i) lo = mid;
      else hi = mid;
    }
  }
  long long r = i - persist_items_before(lo, C, D, nk);
  for (int k = kPersistStages - 1; k >= 0; --k) {
    const long long w = lo - static_cast<long long>(k) * D;
    if (w < 0 || w >= C) continue;
    if (r < nk[k]) {
      *stage = k;
      *sub = static_cast<int>(r);
      *j = w;
      return;
    }
    r -= nk[k];
  }
  *stage = -1;  // not reached for i in range
  *sub = 0;
  *j = 0;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// a slot word holds window tag t (window + 1) and stage k's count c
__device__ __forceinline__ bool slot_ready(unsigned long long w, unsigned long long tag, int k, unsigned int c) {
  return (w >> 40) == tag && static_cast<unsigned int>((w >> (8 * k)) & 0xffu) >= c;
}

// thread 0: wait until the launch's ready(), or false if the launch aborted
// or the wait ran out (which aborts the launch).  The abort flag is read
// after ready(): an item skipped because of an abort still reports
// completion, and a consumer that sees that report then also sees the abort,
// so no item ever runs on a skipped item's output.
template <typename Ready>
__device__ __forceinline__ bool persist_wait(unsigned int* abort, long long spin_limit, Ready ready) {
  const long long t0 = clock64();
  while (true) {
    const bool r = ready();
    if (ld_acquire_u32(abort) != 0u) return false;
    if (r) return true;
    if (clock64() - t0 > spin_limit) {
      atomicExch(abort, 1u);
      return false;
    }
    __nanosleep(128);
  }
}

// all threads: this item's global writes are done; thread 0 publishes them
// with a release reduction (the barrier orders the other threads' writes
// before it)
__device__ __forceinline__ void persist_signal(unsigned int* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
}

// one thread, after a barrier that follows the item's writes: stage k of
// window g is one item further (release: the barrier orders the other
// threads' writes before it); S0 also tags the slot
constexpr int kSignalThread = 224;  // lane 0 of the last warp
__device__ __forceinline__ void persist_slot_signal(unsigned long long* w, long long g, int k) {
  if (k == 0) {
    const unsigned long long v = (static_cast<unsigned long long>(g + 1) << 40) | 1ull;
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(w), "l"(v) : "memory");
  } else {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(w), "l"(1ull << (8 * k)) : "memory");
  }
}

// The stage bodies are called, not inlined: each gets its own register
// allocation (within the kernel's bound) instead of one allocation for the
// union of all fifteen, which spilled heavily.
// As in the streaming schedule (n <= 256, plain forward) the rows record each
// block's statistics and the column pairs remove the means in the spectrum,
// so the statistics item has no work of its own: it stays in the order as the
// point where a window takes over its ring slot.
template <int N, typename TIn>
__device__ __noinline__ void persist_s0(const MatchLaunch*, WinRef) {}
template <int N, typename TIn>
__device__ __noinline__ void persist_s1(const MatchLaunch* L, WinRef R, int sub) {
  rows_stage<N, TIn, true>(*L, R, sub);
}
template <int N>
__device__ __noinline__ void persist_s2(const MatchLaunch* L, WinRef R, int sub) {
  cpair_stage<N, true>(*L, R, sub);
}
template <int N>
__device__ __noinline__ void persist_s3(const MatchLaunch* L, WinRef R, int sub) {
  irows_stage<N, false>(*L, R, sub);
}
template <int N>
__device__ __noinline__ void persist_s4(const MatchLaunch* L, WinRef R) {
  // the same finalize as the streaming schedule's (folded into its last
  // inverse-row block below an 8 px radius, a kernel of its own above)
  if (L->radius2 < 64.f) {
    const int st = stat_status(load_stats(R));
    if (st == SWIFT_WIN_OK) {
      disc_stage<N>(*L, R);
    } else if (st != kStatusSkip && threadIdx.x == 0) {
      swift_result r = {0, 0, 0.f, 0.f, 0.f, 0.f, st, 0};
      L->out[R.b] = r;
    }
  } else {
    peak_stage<N, 256>(*L, R);
  }
}

template <int N, typename TIn>
__device__ __forceinline__ void persist_stage(const PersistLaunch& P, const MatchLaunch* L, int l, int stage, int sub,
                                              long long j, long long g, long long loff, bool live) {
  const long long slot = static_cast<int>(g) % P.ring;
  WinRef R;
  if (P.sorted) R.b = loff + j;
  else if (P.level_idx != nullptr) R.b = static_cast<long long>(__ldcg(P.lists + static_cast<long long>(l) * P.B + j));
  else R.b = j;
  R.stats = P.stats + R.b;
  R.zr = P.zr + slot * P.nmax * P.nmax;
  R.h = P.h + slot * P.nmax * (P.nmax / 2);
  R.part = P.part + kPersistPartStride * R.b;
  R.pre = nullptr;
  R.done = nullptr;  // the finalize is an item of its own
  R.rstat = P.rstat + static_cast<long long>(kPersistRowBlocks) * 8 * R.b;
  if (!live) {
    // the launch aborted: no work; a finalize item reports the window
    if (stage == 4 && threadIdx.x == 0) {
      swift_result r = {0, 0, 0.f, 0.f, 0.f, 0.f, SWIFT_WIN_TIMEOUT, 0};
      L->out[R.b] = r;
    }
    return;
  }
  switch (stage) {
    case 0:
      persist_s0<N, TIn>(L, R);
      break;
    case 1:
      persist_s1<N, TIn>(L, R, sub);
      break;
    case 2:
      persist_s2<N>(L, R, sub);
      break;
    case 3:
      persist_s3<N>(L, R, sub);
      break;
    default:
      persist_s4<N>(L, R);
      break;
  }
}

template <typename TIn>
__global__ void __launch_bounds__(256, 2) swim_persistent_kernel(const PersistLaunch P) {
  __shared__ long long s_off[kPersistMaxLevels + 1];   // first item of each level
  __shared__ long long s_base[kPersistMaxLevels + 1];  // first sequence position of each level
  __shared__ int s_info[4];                            // level, stage, sub, live
  __shared__ long long s_j, s_g;
  __shared__ unsigned int s_item, s_next;
  __shared__ int s_ready;
  __shared__ MatchLaunch s_L;  // the current item's level launch (copied from the parameters)
  __shared__ int s_n[kPersistMaxLevels];  // window side of each level
  __shared__ int s_nlev;                  // window side of the current item's level
  __shared__ long long s_loff[kPersistMaxLevels + 1];  // level offsets of a sorted batch
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_item = atomicAdd(P.queue, 1u);
    s_ready = 0;
  }
#pragma unroll
  for (int k = 0; k < kPersistMaxLevels; ++k)
    if (tid == k) s_n[k] = P.lv[k].n;
#pragma unroll
  for (int k = 0; k <= kPersistMaxLevels; ++k)
    if (tid == 32 + k) s_loff[k] = P.level_off[k];
  __syncthreads();
  while (true) {
    const unsigned int item = s_item;
    if (static_cast<int>(item) < P.n_compact) {
      // gather windows into per-level lists
      const long long b0 = static_cast<long long>(item) * kCompactWindows;
      for (long long b = b0 + tid; b < b0 + kCompactWindows && b < P.B; b += blockDim.x) {
        const int l = __ldg(P.level_idx + b);
        if (l >= 0 && l < P.n_levels && ((P.level_mask >> l) & 1u)) {
          const unsigned int pos = atomicAdd(P.lcount + l, 1u);
          P.lists[static_cast<long long>(l) * P.B + pos] = static_cast<int>(b);
        }
      }
      persist_signal(P.comp_done);
    } else {
      if (tid == 0) {
        if (!s_ready) {
          // level sizes: the batch itself, or the lists once every compaction item is done
          bool ok = true;
          if (P.n_compact > 0)
            ok = persist_wait(P.abort, P.spin_limit, [comp = P.comp_done, nc = static_cast<unsigned int>(P.n_compact)] {
              return ld_acquire_u32(comp) >= nc;
            });
          long long off = P.n_compact, base = 0;
          for (int l = 0; l < P.n_levels; ++l) {
            s_off[l] = off;
            s_base[l] = base;
            long long C;
            if (P.sorted) C = ((P.level_mask >> l) & 1u) ? s_loff[l + 1] - s_loff[l] : 0;
            else if (P.level_idx != nullptr) C = ok ? static_cast<long long>(ld_acquire_u32(P.lcount + l)) : 0;
            else C = l == 0 ? P.B : 0;
            int nk[kPersistStages];
            persist_stage_items(s_n[l], nk);
            off += C * (nk[0] + nk[1] + nk[2] + nk[3] + nk[4]);
            base += C;
          }
          s_off[P.n_levels] = off;
          s_base[P.n_levels] = base;
          s_ready = 1;
        }
        int l = -1;
        for (int k = 0; k < P.n_levels; ++k)
          if (static_cast<long long>(item) >= s_off[k] && static_cast<long long>(item) < s_off[k + 1]) l = k;
        s_info[0] = l;
        if (l >= 0) {
          int nk[kPersistStages];
          persist_stage_items(s_n[l], nk);
          s_nlev = s_n[l];
          const long long C = s_base[l + 1] - s_base[l];
          int stage, sub;
          long long j;
          persist_decode(static_cast<long long>(item) - s_off[l], C, P.skew, nk, &stage, &sub, &j);
          const long long g = s_base[l] + j;  // position in the sequence of all levels' windows
          const unsigned long long* w = P.slot + static_cast<int>(g) % P.ring;
          bool live;
          if (stage == 0) {
            // the slot's previous window (g - RING) has finished every stage
            const unsigned long long prev = static_cast<unsigned long long>(g - P.ring + 1);
            live = g < P.ring || persist_wait(P.abort, P.spin_limit, [w, prev] { return slot_ready(ld_acquire_u64(w), prev, 4, 1u); });
          } else {
            const unsigned long long tag = static_cast<unsigned long long>(g + 1);
            const int k = stage - 1;
            const unsigned int need = static_cast<unsigned int>(nk[k]);
            live = persist_wait(P.abort, P.spin_limit, [w, tag, k, need] { return slot_ready(ld_acquire_u64(w), tag, k, need); });
          }
          s_info[1] = stage;
          s_info[2] = sub;
          s_info[3] = live ? 1 : 0;
          s_j = j;
          s_g = g;
          // constant indices into the parameter block (a runtime index would
          // make the compiler copy the whole block to local memory)
          switch (l) {
            case 0:
              s_L = P.lv[0].L;
              break;
            case 1:
              s_L = P.lv[1].L;
              break;
            case 2:
              s_L = P.lv[2].L;
              break;
            case 3:
              s_L = P.lv[3].L;
              break;
            case 4:
              s_L = P.lv[4].L;
              break;
            case 5:
              s_L = P.lv[5].L;
              break;
            case 6:
              s_L = P.lv[6].L;
              break;
            case 7:
              s_L = P.lv[7].L;
              break;
            case 8:
              s_L = P.lv[8].L;
              break;
            case 9:
              s_L = P.lv[9].L;
              break;
            case 10:
              s_L = P.lv[10].L;
              break;
            case 11:
              s_L = P.lv[11].L;
              break;
            case 12:
              s_L = P.lv[12].L;
              break;
            case 13:
              s_L = P.lv[13].L;
              break;
            case 14:
              s_L = P.lv[14].L;
              break;
            case 15:
              s_L = P.lv[15].L;
              break;
          }
        }
      }
      __syncthreads();
      const int l = s_info[0];
      if (l < 0) break;  // every item is claimed
      const int stage = s_info[1], sub = s_info[2];
      const bool live = s_info[3] != 0;
      const long long j = s_j, g = s_g;
      switch (s_info[0] >= 0 ? s_nlev : 0) {
        case 64:
          persist_stage<64, TIn>(P, &s_L, l, stage, sub, j, g, s_loff[l], live);
          break;
        case 128:
          persist_stage<128, TIn>(P, &s_L, l, stage, sub, j, g, s_loff[l], live);
          break;
        default:
          persist_stage<256, TIn>(P, &s_L, l, stage, sub, j, g, s_loff[l], live);
          break;
      }
      // the item's writes are done: one thread of the last warp publishes them
      // while thread 0 claims the next item
      __syncthreads();
      if (tid == kSignalThread && !(stage == 1 && g == P.hold_s1))  // test hook: never signals
        persist_slot_signal(P.slot + static_cast<int>(g) % P.ring, g, stage);
    }
    if (tid == 0) s_next = atomicAdd(P.queue, 1u);
    __syncthreads();
    if (tid == 0) s_item = s_next;
    __syncthreads();
  }
}

}  // namespace swift
