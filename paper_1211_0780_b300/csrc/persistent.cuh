// Persistent batched sweep: one cooperative launch advances every replica of
// every lattice (uneven L included) through n_sweeps sweeps, with the fused
// measurement and the on-device exchange of Sec. II, Eq. (3).  Each
// half-sweep is a list of tile work items (lattice, slot, tile) that the host
// scheduler spreads over the blocks by longest-processing-time-first; a
// bounded grid barrier separates half-sweeps.
//
// The barrier is two levels of monotonically increasing arrival counters:
// block b arrives on group counter b mod kBarGroups (each on its own 128-byte
// line, so arrivals are spread over L2 slices instead of serialising on one
// address); the block that completes its group's count for this barrier
// instance adds one to the top counter, which every block polls with
// acquire loads.  Barrier instance k completes when the top counter reaches
// (k + 1) * (number of non-empty groups).  Every wait is bounded by a
// %globaltimer budget; when it runs out the block sets the status word to
// XY_ERR_TIMEOUT and every block leaves at its next barrier, so a missing
// block ends the launch with an error, never a hang.  Co-residency of all
// blocks is guaranteed by the cooperative launch.
#pragma once
#include <cstdint>

#include "kernels.cuh"
#include "sweep.cuh"

namespace xy {

constexpr int kBarGroups = 16;
constexpr int kBarStride = 16;  // 64-bit words between counters (128 bytes)

struct PersistentArgs {
  PassParams pp;            // mpass_off and measure are set per pass
  FinishParams fp;          // offsets, record and swap are set per sweep
  const Lattice* lats;
  const int4* items;        // (lattice, local slot, tile, unused)
  const int* offs;          // items of block b: offs[b] .. offs[b+1]-1
  int n_lat;
  int nM, nOR, n_sweeps, me, se;
  unsigned long long* bar;  // kBarGroups group counters then the top counter,
                            // kBarStride words apart, zero at launch
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

__device__ __forceinline__ bool due_dev(uint64_t s, int every) {
  return every > 0 && (s + 1) % static_cast<uint64_t>(every) == 0;
}

// Every lattice of a persistent launch uses tile kind KIND, with blocks of
// at most 256 threads: the block kind with at least three blocks resident
// per SM (80 registers); the march kind with two (128 registers; it spills
// 272 bytes there, and ran 19% faster on a 64^3 x 32 ladder than with its
// 217 registers unbounded); the direct kind with its registers unbounded
// (246; at 128 it spilled 1.2 KB and ran 10% slower).  The direct kind's other-colour
// loads go through L1: every half-sweep starts after a grid barrier whose
// acquire (by one thread, then the block barrier) orders the block's later
// loads after every block's writes of the previous half-sweep, as the
// launch boundary does for the per-launch kernels.
constexpr int kPersistentBlockThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kPersistentBlockThreads, KIND == kTileBlock ? 3 : (KIND == kTileMarch ? 2 : 1))
    k_persistent(PersistentArgs a) {
  extern __shared__ __align__(16) float sm[];
  unsigned long long nbar = 0;
  if (a.poison) {  // test hook: the first barrier waits for one arrival too many
    grid_barrier(a, 0);
    return;
  }
  const int tid = threadIdx.x, B = blockDim.x;
  const uint64_t s_base = a.pp.ctr[kCtrSweep];
  const int n_pass = a.nM + a.nOR;
  const int i0 = a.offs[blockIdx.x], i1 = a.offs[blockIdx.x + 1];
  uint64_t n_rec = 0, n_swp = 0;
  // One pass of colour `colour` over this block's tile items.  The update
  // passes never measure: the lattice sums of a measured sweep come from a
  // measure-only pass after its last half-sweep, which forms the same
  // per-thread sums in the same order as the per-launch path's fused pass
  // (the white sites' stored spins are the updated ones), so the records
  // are identical; keeping the measuring update variants out of this kernel
  // lets the march kind keep two blocks per SM.
  auto tile_items = [&](auto mode, int colour, const PassParams& pp) {
    constexpr int MODE = decltype(mode)::value;
    constexpr bool MEAS = MODE == kMeasureOnly;
    for (int it = i0; it < i1; ++it) {
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
  };
  for (int s = 0; s < a.n_sweeps; ++s) {
    const uint64_t sw = s_base + s;
    const bool meas = due_dev(sw, a.me), swp = due_dev(sw, a.se);
    for (int p = 0; p < n_pass; ++p) {
      const bool is_met = p < a.nM;
      for (int colour = 0; colour < 2; ++colour) {
        PassParams pp = a.pp;
        pp.mpass_off = is_met ? static_cast<uint64_t>(s) * a.nM + p : 0ull;
        pp.measure = 0;
        if (is_met)
          tile_items(IC<kMetropolis>{}, colour, pp);
        else
          tile_items(IC<kOverrelax>{}, colour, pp);
        if (!grid_barrier(a, nbar++)) return;
      }
    }
    if (meas || swp) {
      PassParams pp = a.pp;
      pp.measure = 1;
      tile_items(IC<kMeasureOnly>{}, 1, pp);
      if (!grid_barrier(a, nbar++)) return;
    }
    if (meas || swp) {
      FinishParams fp = a.fp;
      fp.sweep_off = s;
      fp.series_off = n_rec;
      fp.swap_off = n_swp;
      fp.record = meas ? 1 : 0;
      fp.swap = swp ? 1 : 0;
      // every slot's sums and record on its own warp, spread over the grid,
      // then (after a barrier) each ladder's exchange on one block
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
      if (swp) {
        if (!grid_barrier(a, nbar++)) return;
        for (int l = blockIdx.x; l < a.n_lat; l += gridDim.x) exchange_ladder(a.lats[l], l, fp, tid, B);
      }
      n_rec += meas ? 1 : 0;
      n_swp += swp ? 1 : 0;
      if (!grid_barrier(a, nbar++)) return;
    }
  }
}

}  // namespace xy
