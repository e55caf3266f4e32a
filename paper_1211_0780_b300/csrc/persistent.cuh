// Persistent batched sweep: launches that each advance every replica of
// every lattice (uneven L included) through one part of a sweep -- its
// Metropolis passes, or its over-relaxation passes with, on measured or
// exchanging sweeps, the fused measurement in the last white half-sweep and
// the on-device exchange of Sec. II, Eq. (3) -- so that each part's kernel
// keeps its own register budget (one kernel holding the Metropolis and the
// over-relaxation update spills more than a kilobyte a thread for the
// direct tile and runs at half the speed).
//
// A launch is one list of work items: the tile items (lattice, slot, tile)
// of its first half-sweep, sorted by the host by decreasing cost, then the
// same list for each later half-sweep, then (finishing launch) the slots'
// finishing items, one slot per warp.  Blocks take items in that order
// through one atomic counter, so the longest items start first and a block
// that finishes early takes the next one.  There is no grid-wide barrier:
// the half-sweeps of one slot depend only on that slot's previous
// half-sweep (the checkerboard of Sec. II reads the other colour's
// neighbours, which the previous half-sweep wrote, and overwrites the
// colour the previous half-sweep read) and, after an exchange, on its
// ladder's exchange (which changes the slot's beta).  So each slot counts
// what it has finished in the xy_sweep call -- one per tile item, and one
// per finishing step (its own sums, or its ladder's exchange) -- and a
// block starts an item once the item's slot has counted everything before
// it.  Slots of a replica ladder or of other lattices keep running
// meanwhile, so a half-sweep's last tiles overlap the next half-sweep's
// first ones.  The launches of one call are chained by programmatic
// dependent launch without griddepcontrol.wait: a launch's blocks start as
// the previous launch's blocks leave, and the counts alone order the work.
//
// Waiting never deadlocks.  Within a launch a block waits only for items
// placed before its own in the list, which running blocks took earlier (a
// block holds one item at a time), so the earliest unfinished item always
// has its inputs and runs.  Across launches, a launch's blocks are started
// only once every block of the previous launch has taken its last item
// (each block signals griddepcontrol.launch_dependents after the grab that
// finds the list empty), so every item of the previous launch is held by a
// running block that waits for nothing of the later launch.  The counts
// are released (a release add) by the block's first thread after a block
// barrier, or by a warp's lanes after a warp barrier, and acquired by the
// waiting block's first thread before a block barrier; the acquire also
// orders the direct tile's L1 loads after the counted writes.  Every wait
// is bounded by a %globaltimer budget: when it runs out the block sets the
// status word to XY_ERR_TIMEOUT, and every block leaves at its next wait,
// so a missing item ends the call with an error, never a hang.  The
// counters are cleared at the call's start.
#pragma once
#include <cstdint>

#include "kernels.cuh"
#include "sweep.cuh"

namespace xy {

// The synchronisation area: two item counters (launches of even and odd
// position in the call take turns: a launch starts only after every block
// of the one before has made its last grab, so the launch two back has
// finished grabbing), then from word kSyncSlot0 on one completion count
// per slot; all zero at an xy_sweep call's start.  Each counter has a
// 128-byte line of its own.
constexpr int kSyncWork1 = 16;
constexpr int kSyncSlot0 = 32;

// The update passes one persistent launch runs.  The launch that ends a
// measured or exchanging sweep (FIN) runs that sweep's last half-sweep (the
// last pass's white sites) with the fused measurement, then the slots'
// sums, records and exchange; the launch before it stops one half-sweep
// short.
enum PersistentPart : int { kPartMetropolis = 0, kPartOverrelax = 1 };

struct PersistentArgs {
  PassParams pp;                 // mpass_off: the pass counter offset of a Metropolis launch's first pass
  FinishParams fp;               // offsets, record and swap set by the host per sweep (FIN)
  const Lattice* lats;
  const int4* items;             // (lattice, local slot, tile, unused), by decreasing cost
  int n_items;                   // tile items of one half-sweep
  int n_lat;
  int n_half;                    // half-sweeps of this launch (black, white, black, ...; FIN: 1, white)
  unsigned long long hs0;        // half-sweeps every slot finished before this launch in the call
  unsigned long long fin0;       // finishing steps every slot finished before this launch in the call
  unsigned long long work0;      // this launch's item counter's value at its start
  unsigned long long* work;      // this launch's item counter
  unsigned long long* cnt;       // the slot counts
  int* status;                   // 0, or XY_ERR_TIMEOUT
  long long budget_ns;           // bound of one wait
  int poison;                    // test hook: every block waits for a count nothing reaches
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// By the block's first thread: waits until *p >= target (bounded), polling
// with relaxed loads and acquiring once the count is there (polling with
// acquire loads measured slower: an acquire makes the SM drop cached lines
// the other blocks on it are using).  Returns false if the launch has
// failed (this or another block timed out).
__device__ __forceinline__ bool wait_count(const PersistentArgs& a, const unsigned long long* p,
                                           unsigned long long target) {
  if (ld_acquire(p) >= target) return true;
  const long long t0 = global_ns();
  while (ld_relaxed(p) < target) {
    if (*reinterpret_cast<volatile int*>(a.status) != 0) return false;
    if (global_ns() - t0 > a.budget_ns) {
      atomicCAS(a.status, 0, XY_ERR_TIMEOUT);
      return false;
    }
    __nanosleep(64);
  }
  return ld_acquire(p) >= target;  // the count only grows
}

__device__ __forceinline__ int lattice_of_slot(const Lattice* lats, int n_lat, int g) {
  int lo = 0, hi = n_lat - 1;  // the last lattice with slot0 <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (lats[mid].slot0 <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Work items of one launch: its tile items, then (FIN) its finishing items
// of one slot per warp.
__host__ __device__ inline long long persistent_items(int n_half, int n_items, bool fin, int n_slots,
                                                      int block_threads) {
  const int nwb = block_threads / 32;
  return static_cast<long long>(n_half) * n_items + (fin ? (n_slots + nwb - 1) / nwb : 0);
}

// Finishing step of slot g, by one warp: the slot's sums and record (the
// per-launch path's k_finish), then its count; on an exchanging sweep the
// warp that finishes a ladder's last slot runs the ladder's exchange and
// counts it for every slot of the ladder.
__device__ __noinline__ void finish_counted(const PersistentArgs& a, int g, int lane) {
  const int l = lattice_of_slot(a.lats, a.n_lat, g);
  const Lattice& lat = a.lats[l];
  const FinishParams& fp = a.fp;
  finish_slot(lat, g - lat.slot0, fp, lane);
  if (!fp.swap) {
    if (lane == 0) red_release_add(a.cnt + g, 1ull);  // lane 0 wrote the slot's results
    return;
  }
  __threadfence();
  int last = 0;
  if (lane == 0) last = (atomicAdd(fp.done + l, 1) == lat.R - 1) ? 1 : 0;
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  exchange_ladder(lat, l, fp, lane, 32);
  if (lane == 0) fp.done[l] = 0;
  __syncwarp();  // every lane's exchange writes precede every lane's release
  for (int r = lane; r < lat.R; r += 32) red_release_add(a.cnt + lat.slot0 + r, 1ull);
}

// The finishing items of a FIN launch, from item `it` (the first the block
// took past the tile items) on.  Kept out of line so that the tile loop
// keeps its registers.
__device__ __noinline__ void finish_items(const PersistentArgs& a, long long it, long long n_tile, long long n_all,
                                          long long* s_item, int* s_ok) {
  const int tid = threadIdx.x, nwb = blockDim.x >> 5;
  for (;;) {
    // every warp's slot has its measured half-sweep finished
    if (tid == 0) {
      int ok = 1;
      const int g0 = static_cast<int>(it - n_tile) * nwb;
      for (int g = g0; g < min(g0 + nwb, a.fp.n_slots) && ok; ++g) {
        const Lattice& lat = a.lats[lattice_of_slot(a.lats, a.n_lat, g)];
        const unsigned long long T = static_cast<unsigned long long>(lat.nyt) * lat.nzt;
        ok = wait_count(a, a.cnt + g, (a.hs0 + 1ull) * T + a.fin0);
      }
      *s_ok = ok;
    }
    __syncthreads();
    if (!*s_ok) return;
    const int g = static_cast<int>(it - n_tile) * nwb + (tid >> 5);
    if (g < a.fp.n_slots) finish_counted(a, g, tid & 31);
    if (tid == 0) {
      const unsigned long long t = atomicAdd(a.work, 1ull) - a.work0;
      *s_item = t < static_cast<unsigned long long>(n_all) ? static_cast<long long>(t) : -1ll;
    }
    __syncthreads();
    it = *s_item;
    if (it < 0) {
      launch_dependents();  // every item of this launch is taken
      return;
    }
    __syncthreads();  // every thread has read s_item before it is written again
  }
}

// Every lattice of a persistent launch uses tile kind KIND, with blocks of
// at most 256 threads, and each part's kernel is compiled for the blocks per
// SM its kind keeps: the block kind three (at most 80 registers), the march,
// the direct and the angle kinds two (at most 128).  FIN: the launch ends a
// measured or exchanging sweep; EO (FIN): the sweep only exchanges, and the
// direct and angle kinds' half-sweep sums the energy alone (the other kinds
// read that from pp.measure).
constexpr int kPersistentBlockThreads = 256;

template <int KIND, int PART, bool FIN, bool EO = false>
__global__ void __launch_bounds__(kPersistentBlockThreads, KIND == kTileBlock ? 3 : 2)
    k_persistent(PersistentArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x, B = blockDim.x;
  __shared__ long long s_item;  // the item taken, or -1
  __shared__ int s_ok;          // its inputs are ready (0: the launch has failed)
  __shared__ int s_h, s_i;      // its half-sweep and its place in the half-sweep's list
  if (a.poison) {  // test hook: slot 0's count never reaches the target
    if (tid == 0) wait_count(a, a.cnt, 1ull);
    return;
  }
  if (*reinterpret_cast<volatile int*>(a.status) != 0) return;  // an earlier launch failed
  constexpr int MODE = PART == kPartMetropolis ? kMetropolis : kOverrelax;
  for (;;) {
    // the first thread takes the next item and waits for everything the
    // item's slot had to finish before it
    if (tid == 0) {
      const long long n_tile = static_cast<long long>(a.n_half) * a.n_items;
      const long long n_all = persistent_items(a.n_half, a.n_items, FIN, a.fp.n_slots, B);
      const unsigned long long t = atomicAdd(a.work, 1ull) - a.work0;
      const long long it = t < static_cast<unsigned long long>(n_all) ? static_cast<long long>(t) : -1ll;
      int ok = 1;
      if (it >= 0 && it < n_tile) {
        const long long h = it / a.n_items;
        s_h = static_cast<int>(h);
        s_i = static_cast<int>(it - h * a.n_items);
        const int4 w = a.items[s_i];
        const Lattice& lat = a.lats[w.x];
        const unsigned long long T = static_cast<unsigned long long>(lat.nyt) * lat.nzt;
        ok = wait_count(a, a.cnt + lat.slot0 + w.y, (a.hs0 + static_cast<unsigned long long>(h)) * T + a.fin0);
      }
      s_item = it;
      s_ok = ok;
    }
    __syncthreads();
    const long long it = s_item;
    if (it < 0) launch_dependents();  // every item of this launch is taken
    if (it < 0 || !s_ok) return;
    if (FIN && it >= static_cast<long long>(a.n_half) * a.n_items) {
      __syncthreads();  // every thread has read s_item before it is written again
      finish_items(a, it, static_cast<long long>(a.n_half) * a.n_items,
                   persistent_items(a.n_half, a.n_items, FIN, a.fp.n_slots, B), &s_item, &s_ok);
      return;
    }
    const int h = FIN ? 0 : s_h;  // FIN: one half-sweep
    const int4 w = a.items[s_i];
    const Lattice lat = a.lats[w.x];
    const int TX = lat.L >> 3;
    const int tx = tid % TX, rest = tid / TX;
    const int yt = w.z % lat.nyt, zt = w.z / lat.nyt;
    // FIN: one half-sweep, the last pass's white sites, measured (the
    // per-launch path's fused pass, so the records are identical)
    const int colour = FIN ? 1 : (h & 1);
    const PassParams& pp = a.pp;
    const uint32_t pass_add = PART == kPartMetropolis ? static_cast<uint32_t>(h >> 1) : 0u;
    float acc[kNumSums];
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) acc[j] = 0.f;
    uint32_t n_acc = 0u;
    if (KIND == kTileBlock) {
      const int ty = rest % lat.ty, tz = rest / lat.ty;
      tile_block<MODE, FIN>(lat, w.y, yt, zt, colour, tx, ty, tz, tz < lat.tz, pp, sm, acc, n_acc, pass_add);
    } else if (KIND == kTileDirect) {
      // threads beyond the tile's rows return at once
      tile_direct<MODE, FIN, 0, false, EO ? 1 : 0>(lat, w.y, yt, zt, colour, tx, rest, pp, acc, n_acc, pass_add);
    } else if (KIND == kTileAngle) {
      tile_angle<MODE, FIN, EO ? 1 : 0>(lat, w.y, yt, zt, colour, tx, rest, rest < lat.ty, pp, sm, acc, n_acc,
                                        pass_add);
    } else {
      tile_pass<MODE, FIN>(lat, w.y, yt, zt, colour, tx, rest, rest < lat.ty, pp, sm, acc, n_acc, pass_add);
    }
    if (MODE == kMetropolis) block_count_to(pp.acc_met + lat.slot0 + w.y, n_acc, tid, B);
    if (FIN) {
      double* red = reinterpret_cast<double*>(sm + tile_floats(lat.kind, lat.L, lat.ty, lat.tz));
      const long long part = lat.part0 + static_cast<long long>(w.y) * lat.nyt * lat.nzt + w.z;
      block_sums_to(pp.partials + part * kNumSums, acc, tid, B, red);
    }
    // every thread's writes of the tile precede the count: the block
    // barrier orders them before the first thread's release, whose
    // cumulativity makes them visible to whoever acquires the count
    __syncthreads();
    if (tid == 0) red_release_add(a.cnt + lat.slot0 + w.y, 1ull);
  }
}

}  // namespace xy
