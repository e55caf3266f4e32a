// Persistent batched sweep: cooperative launches that each advance every
// replica of every lattice (uneven L included) through one part of a sweep
// -- its Metropolis passes, or its over-relaxation passes with, on measured
// or exchanging sweeps, the fused measurement in the last white half-sweep
// and the on-device exchange of Sec. II, Eq. (3) -- so that each part's
// kernel keeps its own register budget (one kernel holding every variant
// needed 246 registers a thread for the direct tile, two warps per
// scheduler).  Each half-sweep is one list of tile work items (lattice,
// slot, tile), sorted by the host by decreasing cost; the blocks take items
// from the list in that order through one atomic counter, so the longest
// items start first and a block that finishes early takes the next one
// (longest-processing-time-first, balanced by the actual run times); a
// bounded grid barrier separates the half-sweeps inside a launch, and the
// launch boundary separates the parts.
//
// The barrier is two levels of monotonically increasing arrival counters:
// block b arrives on group counter b mod kBarGroups (each on its own 128-byte
// line, so arrivals are spread over L2 slices instead of serialising on one
// address); the block that completes its group's count for this barrier
// instance adds one to the top counter, which every block polls with
// acquire loads.  Barrier instance k completes when the top counter reaches
// (k + 1) * (number of non-empty groups); instances are numbered across the
// launches of one xy_sweep call (the host passes each launch the number
// completed before it), and the counters are cleared once per call.  Every
// wait is bounded by a %globaltimer budget; when it runs out the block sets
// the status word to XY_ERR_TIMEOUT and every block leaves at its next
// barrier (and later launches return at once), so a missing block ends the
// call with an error, never a hang.  Co-residency of all blocks is
// guaranteed by the cooperative launch.
#pragma once
#include <cstdint>

#include "kernels.cuh"
#include "sweep.cuh"

namespace xy {

constexpr int kBarGroups = 16;
constexpr int kBarStride = 16;  // 64-bit words between counters (128 bytes)
// The work counter sits after the barrier's group and top counters.
constexpr int kBarWords = (kBarGroups + 2) * kBarStride;

// The update passes one persistent launch runs.  The launch that ends a
// measured or exchanging sweep (FIN) runs that sweep's last half-sweep (the
// last pass's white sites) with the fused measurement, then the slots'
// sums, records and exchange; the launch before it stops one half-sweep
// short.
enum PersistentPart : int { kPartMetropolis = 0, kPartOverrelax = 1 };

struct PersistentArgs {
  PassParams pp;            // mpass_off and measure are set per pass
  FinishParams fp;          // offsets, record and swap set by the host per sweep (FIN)
  const Lattice* lats;
  const int4* items;        // (lattice, local slot, tile, unused), by decreasing cost
  int n_items;              // items of one half-sweep
  int n_lat;
  int n_half;               // half-sweeps of this launch (black, white, black, ...; FIN: 1, white)
  uint64_t mpass_off;       // kPartMetropolis: pass counter offset of its first half-sweep's pass
  unsigned long long bar0;  // barrier instances completed before this launch
  unsigned long long work0; // work-counter value at this launch's first half-sweep
  unsigned long long* bar;  // kBarGroups group counters, the top counter, then
                            // the work counter, kBarStride words apart, zero at
                            // the call's start
  int* status;              // 0, or XY_ERR_TIMEOUT
  long long budget_ns;      // bound of one barrier wait
  int poison;               // test hook: the first barrier expects one block too many
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long atom_acq_rel_add(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

// Barrier instance `k` (0-based).  Returns false if the launch has failed
// (this or another block timed out).
__device__ __forceinline__ bool grid_barrier(const PersistentArgs& a, unsigned long long k) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const unsigned G = gridDim.x;
    const unsigned g = blockIdx.x % kBarGroups;
    const unsigned n_groups = G < kBarGroups ? G : kBarGroups;
    const unsigned long long n_in_group = G / kBarGroups + (g < G % kBarGroups ? 1u : 0u);
    unsigned long long* top = a.bar + kBarGroups * kBarStride;
    __threadfence();
    const unsigned long long old = atom_acq_rel_add(a.bar + g * kBarStride, 1ull);
    if (old + 1 == (k + 1) * n_in_group) red_release_add(top, 1ull);
    const unsigned long long target = (k + 1) * n_groups + (a.poison ? 1ull : 0ull);
    const long long t0 = global_ns();
    int good = 1;
    while (ld_acquire(top) < target) {
      if (*reinterpret_cast<volatile int*>(a.status) != 0) {
        good = 0;
        break;
      }
      if (global_ns() - t0 > a.budget_ns) {
        atomicCAS(a.status, 0, XY_ERR_TIMEOUT);
        good = 0;
        break;
      }
      __nanosleep(32);
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// Barrier instances one launch runs: one between consecutive half-sweeps,
// and when finishing a sweep one before the slots' sums and one before the
// exchange.
__host__ __device__ inline unsigned long long persistent_barriers(int n_half, bool fin, bool swap) {
  return static_cast<unsigned long long>(n_half) - 1ull + (fin ? (swap ? 2ull : 1ull) : 0ull);
}

// Every lattice of a persistent launch uses tile kind KIND, with blocks of
// at most 256 threads, and each part's kernel is compiled for the blocks per
// SM its kind keeps: the block kind three (at most 80 registers), the march,
// the direct and the angle kinds two (at most 128).  FIN: the launch ends a
// measured or exchanging sweep.  The direct kind's other-colour
// loads go through L1: a half-sweep starts after the launch boundary or a
// grid barrier whose acquire (by one thread, then the block barrier) orders
// the block's later loads after every block's writes of the previous
// half-sweep, as the launch boundary does for the per-launch kernels.
constexpr int kPersistentBlockThreads = 256;

template <int KIND, int PART, bool FIN>
__global__ void __launch_bounds__(kPersistentBlockThreads, KIND == kTileBlock ? 3 : 2)
    k_persistent(PersistentArgs a) {
  extern __shared__ __align__(16) float sm[];
  unsigned long long nbar = a.bar0;
  if (a.poison) {  // test hook: the first barrier waits for one arrival too many
    grid_barrier(a, 0);
    return;
  }
  if (*reinterpret_cast<volatile int*>(a.status) != 0) return;  // an earlier launch failed
  const int tid = threadIdx.x, B = blockDim.x;
  unsigned long long* const work = a.bar + (kBarGroups + 1) * kBarStride;
  // Every block makes one failing grab per half-sweep, so each half-sweep
  // advances the counter by exactly n_items + gridDim.x.
  unsigned long long base = a.work0;
  __shared__ int s_item;
  // One half-sweep of colour `colour` over the tile items the block takes.
  // The measuring variant (the last white half-sweep of a finishing launch)
  // is the per-launch path's fused pass, so the records are identical.
  auto tile_items = [&](auto mode, auto meas, int colour, const PassParams& pp) {
    constexpr int MODE = decltype(mode)::value;
    constexpr bool MEAS = decltype(meas)::value != 0;
    for (;;) {
      if (tid == 0) {
        const unsigned long long t = atomicAdd(work, 1ull) - base;
        s_item = t < static_cast<unsigned long long>(a.n_items) ? static_cast<int>(t) : -1;
      }
      __syncthreads();
      const int it = s_item;
      __syncthreads();  // every thread has read s_item before it is written again
      if (it < 0) break;
      const int4 w = a.items[it];
      const Lattice lat = a.lats[w.x];
      const int TX = lat.L >> 3;
      const int tx = tid % TX, rest = tid / TX;
      const int yt = w.z % lat.nyt, zt = w.z / lat.nyt;
      float acc[kNumSums];
#pragma unroll
      for (int j = 0; j < kNumSums; ++j) acc[j] = 0.f;
      uint32_t n_acc = 0u;
      if (KIND == kTileBlock) {
        const int ty = rest % lat.ty, tz = rest / lat.ty;
        tile_block<MODE, MEAS>(lat, w.y, yt, zt, colour, tx, ty, tz, tz < lat.tz, pp, sm, acc, n_acc);
      } else if (KIND == kTileDirect) {
        // threads beyond the tile's rows return at once
        tile_direct<MODE, MEAS>(lat, w.y, yt, zt, colour, tx, rest, pp, acc, n_acc);
      } else if (KIND == kTileAngle) {
        tile_angle<MODE, MEAS>(lat, w.y, yt, zt, colour, tx, rest, pp, acc, n_acc);
      } else {
        tile_pass<MODE, MEAS>(lat, w.y, yt, zt, colour, tx, rest, rest < lat.ty, pp, sm, acc, n_acc);
      }
      if (MODE == kMetropolis) block_count_to(pp.acc_met + lat.slot0 + w.y, n_acc, tid, B);
      if (MEAS) {
        double* red = reinterpret_cast<double*>(sm + tile_floats(lat.kind, lat.L, lat.ty, lat.tz));
        const long long part = lat.part0 + static_cast<long long>(w.y) * lat.nyt * lat.nzt + w.z;
        block_sums_to(pp.partials + part * kNumSums, acc, tid, B, red);
      }
    }
    base += static_cast<unsigned long long>(a.n_items) + gridDim.x;
  };
  constexpr int MODE = PART == kPartMetropolis ? kMetropolis : kOverrelax;
  if (!FIN) {
    for (int h = 0; h < a.n_half; ++h) {
      if (h > 0)
        if (!grid_barrier(a, nbar++)) return;
      PassParams pp = a.pp;
      pp.mpass_off = PART == kPartMetropolis ? a.mpass_off + static_cast<uint64_t>(h >> 1) : 0ull;
      pp.measure = 0;
      tile_items(IC<MODE>{}, IC<0>{}, h & 1, pp);
    }
  } else {
    PassParams pp = a.pp;
    pp.mpass_off = PART == kPartMetropolis ? a.mpass_off : 0ull;
    pp.measure = 1;
    tile_items(IC<MODE>{}, IC<1>{}, 1, pp);
    if (!grid_barrier(a, nbar++)) return;
    // every slot's sums and record on its own warp, spread over the grid,
    // then (after a barrier) each ladder's exchange on one block
    const FinishParams& fp = a.fp;
    const int lane = tid & 31, nwb = B >> 5;
    for (int g = blockIdx.x * nwb + (tid >> 5); g < fp.n_slots; g += gridDim.x * nwb) {
      int lo = 0, hi = a.n_lat - 1;  // the lattice of slot g
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.lats[mid].slot0 <= g) lo = mid;
        else hi = mid - 1;
      }
      finish_slot(a.lats[lo], g - a.lats[lo].slot0, fp, lane);
    }
    if (fp.swap) {
      if (!grid_barrier(a, nbar++)) return;
      for (int l = blockIdx.x; l < a.n_lat; l += gridDim.x) exchange_ladder(a.lats[l], l, fp, tid, B);
    }
  }
}

}  // namespace xy
