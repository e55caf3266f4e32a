// Kernels of the sweep path: initial state, one half-sweep per launch,
// the deterministic FP64 finishing reduction with the record append and the
// on-device replica exchange (Sec. II, Eq. 3), the counter advance and the
// Philox draw dump used by the parity tests.
#pragma once
#include <cstdint>

#include "../../include/xy.h"
#include "philox.cuh"
#include "sweep.cuh"

namespace xy {

static_assert(sizeof(xy_record) == 96, "xy_record layout");

// theta = 2 pi u from the initial-state stream, stored as (cos, sin) with
// the accurate sincosf (once per run); one Philox call per packed pair
// (2q, 2q+1) of one colour of one slot.
__global__ void k_init(Lattice lat, uint64_t seed) {
  const long long N = static_cast<long long>(lat.L) * lat.L * lat.L;
  const long long Q = N >> 2;  // pairs per colour
  const long long total = static_cast<long long>(lat.R) * 2 * Q;
  const PhiloxKey key = philox_key(seed);
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i / (2 * Q));
    const int c = static_cast<int>((i / Q) & 1);
    const uint32_t q = static_cast<uint32_t>(i % Q);
    const uint32_t tagw = (static_cast<uint32_t>(lat.slot0 + r) << 4) |
                          (static_cast<uint32_t>(c) << 3) | kTagInit;
    const uint4 w = philox4x32_10(make_uint4(q, 0u, 0u, tagw), key);
    float* a = lat.spins + 2 * r * N + c * N + 2 * static_cast<long long>(q);
    float c0, s0, c1, s1;
    sincosf(u24(w.x) * kTwoPi, &s0, &c0);
    sincosf(u24(w.z) * kTwoPi, &s1, &c1);
    *reinterpret_cast<float2*>(a) = make_float2(c0, c1);
    *reinterpret_cast<float2*>(a + (N >> 1)) = make_float2(s0, s1);
  }
}

// An angle taken into [0, 2 pi) (a value that rounds to 2 pi is 0).
__device__ __forceinline__ float mod_two_pi(float t) {
  t = fmodf(t, kTwoPi);
  t = t < 0.f ? t + kTwoPi : t;
  return t >= kTwoPi ? 0.f : t;
}

// Angles of one slot in the packed order (colour 0 then colour 1, N/2 each):
// theta = atan2(sin, cos) taken into [0, 2 pi), or the stored angle itself
// (angle storage, kTileAngle).
__global__ void k_to_angles(const float* __restrict__ spins, long long N, float* __restrict__ out, int angles) {
  const long long half = N >> 1;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long c = i / half, p = i - c * half;
    const float* base = spins + c * N;
    out[i] = angles ? base[p] : wrap_angle(atan2f(base[p + half], base[p]));
  }
}

// The inverse: packed angles of one slot to stored (cos, sin) with sincosf,
// or (angle storage) to the stored angle taken into [0, 2 pi).
__global__ void k_from_angles(const float* __restrict__ in, long long N, float* __restrict__ spins, int angles) {
  const long long half = N >> 1;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long c = i / half, p = i - c * half;
    if (angles) {
      spins[c * N + p] = mod_two_pi(in[i]);
      continue;
    }
    float sn, cs;
    sincosf(in[i], &sn, &cs);
    spins[c * N + p] = cs;
    spins[c * N + half + p] = sn;
  }
}

// In place, for n_slots slots of 2N floats: every stored vector (cos, sin)
// becomes its angle atan2(sin, cos) in [0, 2 pi), written where the cosine
// was (the change to angle storage, kTileAngle).
__global__ void k_vectors_to_angles(float* __restrict__ spins, long long N, int n_slots) {
  const long long half = N >> 1;
  const long long total = static_cast<long long>(n_slots) * N;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = i / N, q = i - r * N, c = q / half, p = q - c * half;
    float* base = spins + 2 * r * N + c * N;
    base[p] = wrap_angle(atan2f(base[half + p], base[p]));
  }
}

// In place: the angle stored in each cos slot of n_slots slots (each 2N
// floats: colour 0's N/2 cosines, its N/2 sines, colour 1's ...) becomes
// the (cos, sin) pair, with sincosf as k_from_angles uses it; or, for a
// lattice kept as angles (angles != 0), is taken into [0, 2 pi) and stays.
__global__ void k_angles_in_place(float* __restrict__ spins, long long N, int n_slots, int angles) {
  const long long half = N >> 1;
  const long long total = static_cast<long long>(n_slots) * N;  // angles
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = i / N, q = i - r * N, c = q / half, p = q - c * half;
    float* base = spins + 2 * r * N + c * N;
    if (angles) {
      base[p] = mod_two_pi(base[p]);
      continue;
    }
    float sn, cs;
    sincosf(base[p], &sn, &cs);
    base[p] = cs;
    base[half + p] = sn;
  }
}

// One half-sweep of one lattice: grid (tiles per slot, R); block (L/8, ty) for
// the march kind, (L/8, ty, tz) for the block kind, 32 (ceil(L ty / 256) + 1)
// threads in x for the stream kind.  MEAS: the variant that
// fuses the lattice sums (white passes of measured sweeps and the
// measurement-only pass).
template <int MODE, bool MEAS, int KIND>
__global__ void __launch_bounds__(512) k_half(Lattice lat, int colour, PassParams pp) {
  extern __shared__ __align__(16) float sm[];
  chain_wait_and_release();
  const int r = blockIdx.y;
  const int t = blockIdx.x;
  const int yt = t % lat.nyt, zt = t / lat.nyt;
  float acc[kNumSums];
#pragma unroll
  for (int j = 0; j < kNumSums; ++j) acc[j] = 0.f;
  uint32_t n_acc = 0u;
  if (KIND == kTileBlock)
    tile_block<MODE, MEAS>(lat, r, yt, zt, colour, threadIdx.x, threadIdx.y, threadIdx.z, true, pp, sm, acc, n_acc);
  else if (KIND == kTileStream)
    tile_stream<MODE, MEAS>(lat, r, yt, zt, colour, threadIdx.x, pp, sm, acc, n_acc);
  else
    tile_pass<MODE, MEAS>(lat, r, yt, zt, colour, threadIdx.x, threadIdx.y, true, pp, sm, acc, n_acc);
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nth = blockDim.x * blockDim.y * blockDim.z;
  if (MODE == kMetropolis) block_count_to(pp.acc_met + lat.slot0 + r, n_acc, tid, nth);
  if (MEAS) {
    double* red = reinterpret_cast<double*>(sm + tile_floats(KIND, lat.L, lat.ty, lat.tz));
    const long long part = lat.part0 + static_cast<long long>(r) * lat.nyt * lat.nzt + t;
    block_sums_to(pp.partials + part * kNumSums, acc, tid, nth, red);
  }
}

// Draws the calls [pp.gen_begin, pp.gen_end) of the Metropolis words of
// lattice lat for the pass with counter ctr[kCtrMpass] + pp.gen_mpass, one
// call per thread of the grid at a time: call i is call q = i mod N/4 of
// colour c of local slot r, (2 r + c) = i / (N/4), with the counter
// (q, pass, 0, tag) that the Metropolis update would use.
__device__ __forceinline__ void draw_words(const Lattice& lat, const PassParams& pp) {
  const uint32_t quarter = static_cast<uint32_t>(lat.L) * static_cast<uint32_t>(lat.L) * static_cast<uint32_t>(lat.L) / 4u;
  const uint64_t mp = pp.ctr[kCtrMpass] + pp.gen_mpass;
  const uint32_t mlo = static_cast<uint32_t>(mp), mhi = static_cast<uint32_t>(mp >> 32);
  const uint32_t nth = gridDim.x * gridDim.y * blockDim.x * blockDim.y;
  const uint32_t t0 = ((blockIdx.y * gridDim.x + blockIdx.x) * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  for (uint32_t i = pp.gen_begin + t0; i < pp.gen_end; i += nth) {
    const uint32_t sc = i / quarter;
    const uint32_t q = i - sc * quarter;
    const uint32_t tagw = ((static_cast<uint32_t>(lat.slot0) + (sc >> 1)) << 4) | ((sc & 1u) << 3) | kTagMet;
    __stcg(pp.words + i, philox4x32_10(make_uint4(q, mlo, mhi, tagw), pp.rk));
  }
}

// One half-sweep of one lattice with the kTileDirect tile: grid (tiles per
// slot, R), block (L/8, ty); shared memory only for the reduction of the
// measuring variant.  LC: the lattice size fixed at compile time, or 0.
// WG: 1, a Metropolis half-sweep that reads its pass's words (pp.words)
// instead of drawing them; 2, an over-relaxation half-sweep that also draws
// calls of the next Metropolis pass's words (before griddepcontrol.wait in
// library-chained launches: no launch in flight reads them).  EO: the
// measuring variant sums the energy alone (an exchange that records
// nothing), at the plain over-relaxation kernel's register limit.
template <int MODE, bool MEAS, int LC, int WG = 0, bool EO = false>
__global__ void __maxnreg__(MODE == kOverrelax && (!MEAS || EO) ? kDirectMaxRegsOR : kDirectMaxRegs) k_half_direct(Lattice lat, int colour, PassParams pp) {
  extern __shared__ __align__(16) float sm[];
  if (!pp.own_ready) chain_wait_and_release();  // else tile_direct waits after its own-colour loads
  if (WG == 2) draw_words(lat, pp);
  const int r = blockIdx.y;
  const int t = blockIdx.x;
  const int yt = t % lat.nyt, zt = t / lat.nyt;
  float acc[kNumSums];
#pragma unroll
  for (int j = 0; j < kNumSums; ++j) acc[j] = 0.f;
  uint32_t n_acc = 0u;
  tile_direct<MODE, MEAS, LC, WG == 1, EO ? 1 : 0>(lat, r, yt, zt, colour, threadIdx.x, threadIdx.y, pp, acc, n_acc);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nth = blockDim.x * blockDim.y;
  if (MODE == kMetropolis) block_count_to(pp.acc_met + lat.slot0 + r, n_acc, tid, nth);
  if (MEAS) {
    const long long part = lat.part0 + static_cast<long long>(r) * lat.nyt * lat.nzt + t;
    block_sums_to(pp.partials + part * kNumSums, acc, tid, nth, reinterpret_cast<double*>(sm));
  }
}

// One half-sweep of one lattice with the kTileAngle tile (angle storage):
// grid (tiles per slot, R), block (L/8, ty); shared memory: the tile's
// plane buffers, then the reduction area of the measuring variant.  EO:
// the measuring variant sums the energy alone (an exchange that records
// nothing); with that sum the over-relaxation kernel keeps the plain one's
// register limit.
template <int MODE, bool MEAS, bool EO = false>
__global__ void __maxnreg__(MODE == kOverrelax && (!MEAS || EO) ? kAngleMaxRegsOR : kDirectMaxRegs) k_half_angle(Lattice lat, int colour, PassParams pp) {
  extern __shared__ __align__(16) float sm[];
  if (!pp.own_ready) chain_wait_and_release();  // else tile_angle waits after its own-colour loads
  const int r = blockIdx.y;
  const int t = blockIdx.x;
  const int yt = t % lat.nyt, zt = t / lat.nyt;
  float acc[kNumSums];
#pragma unroll
  for (int j = 0; j < kNumSums; ++j) acc[j] = 0.f;
  uint32_t n_acc = 0u;
  tile_angle<MODE, MEAS, EO ? 1 : 0>(lat, r, yt, zt, colour, threadIdx.x, threadIdx.y, true, pp, sm, acc, n_acc);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nth = blockDim.x * blockDim.y;
  if (MODE == kMetropolis) block_count_to(pp.acc_met + lat.slot0 + r, n_acc, tid, nth);
  if (MEAS) {
    double* red = reinterpret_cast<double*>(sm + tile_floats(kTileAngle, lat.L, lat.ty, lat.tz));
    const long long part = lat.part0 + static_cast<long long>(r) * lat.nyt * lat.nzt + t;
    block_sums_to(pp.partials + part * kNumSums, acc, tid, nth, red);
  }
}

struct FinishParams {
  const double* partials;
  double* sums_slot;            // [slots][kNumSums]
  double* E_slot;               // [slots]
  const uint64_t* ctr;
  uint64_t sweep_off;           // record sweep index = ctr[kCtrSweep] + sweep_off
  uint64_t series_off;          // record event = ctr[kCtrSeries] + series_off
  uint64_t swap_off;            // exchange event = ctr[kCtrSwap] + swap_off
  xy_record* series;
  int n_slots;
  int record;
  int swap;
  int parity;                   // < 0: the event counter's parity
  int* perm;                    // [slots]: ladder l's entries at slot0(l) + k
  const double* ladder_beta;    // [slots]: ascending betas of each ladder
  float* beta_slot;             // [slots]
  double* beta_slot64;          // [slots]
  int* bidx_slot;               // [slots]
  unsigned long long* acc_swap; // [slots]
  uint64_t seed;
  int* n_swapped;               // nullable
  int* done;                    // [lattices]: slots of the current event finished
                                // (k_finish), back to 0 after the exchange
};

// Sums of slot r of lattice lat, by one warp: fixed-order FP64 sum of the
// slot's tile partials (lane-strided sequential sums, then a fixed shuffle
// tree); lane 0 writes the slot's sums, its energy and, when recording, its
// record.  Partials are read through L2 because the persistent kernel's
// other blocks wrote them in the same launch.
__device__ void finish_slot(const Lattice& lat, int r, const FinishParams& fp, int lane) {
  const int ntile = lat.nyt * lat.nzt;
  const double* P = fp.partials + (static_cast<long long>(lat.part0) + static_cast<long long>(r) * ntile) * kNumSums;
  double v[kNumSums];
#pragma unroll
  for (int j = 0; j < kNumSums; ++j) v[j] = 0.0;
  for (int t = lane; t < ntile; t += 32) {
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) v[j] += __ldcg(P + t * kNumSums + j);
  }
#pragma unroll
  for (int j = 0; j < kNumSums; ++j) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], off);
  }
  if (lane == 0) {
    const int g = lat.slot0 + r;
    for (int j = 0; j < kNumSums; ++j) fp.sums_slot[g * kNumSums + j] = v[j];
    const double E = -(v[2] + v[3] + v[4]);
    fp.E_slot[g] = E;
    if (fp.record) {
      const uint64_t ev = fp.ctr[kCtrSeries] + fp.series_off;
      xy_record rec;
      rec.E = E;
      rec.Mx = v[0];
      rec.My = v[1];
      for (int mu = 0; mu < 3; ++mu) {
        rec.C[mu] = v[2 + mu];
        rec.S[mu] = v[5 + mu];
      }
      rec.beta = fp.beta_slot64[g];
      rec.slot = g;
      rec.beta_index = fp.bidx_slot[g];
      rec.sweep = fp.ctr[kCtrSweep] + fp.sweep_off;
      fp.series[ev * fp.n_slots + g] = rec;
    }
  }
}

// The exchange of Eq. (3) on ladder l.  The pairs (k, k+1) with k of the
// event's parity are disjoint, so thread t of nt decides the pairs
// k = par + 2t, par + 2(t + nt), ...; the outcome does not depend on nt.
// Energies are read through L2 (other warps wrote them).
__device__ void exchange_ladder(const Lattice& lat, int l, const FinishParams& fp, int t, int nt) {
  const uint64_t n = fp.ctr[kCtrSwap] + fp.swap_off;
  const int par = fp.parity < 0 ? static_cast<int>(n & 1ull) : (fp.parity & 1);
  const PhiloxKey key = philox_key(fp.seed);
  const uint32_t tagw = (static_cast<uint32_t>(l) << 4) | kTagPt;
  const int s0 = lat.slot0;
  int count = 0;
  for (int k = par + 2 * t; k + 1 < lat.R; k += 2 * nt) {
    const int a = fp.perm[s0 + k], b = fp.perm[s0 + k + 1];
    const double bk = fp.ladder_beta[s0 + k], bk1 = fp.ladder_beta[s0 + k + 1];
    const double expo = (bk - bk1) * (__ldcg(fp.E_slot + s0 + a) - __ldcg(fp.E_slot + s0 + b));
    const uint4 w = philox4x32_10(
        make_uint4(static_cast<uint32_t>(k), static_cast<uint32_t>(n), static_cast<uint32_t>(n >> 32), tagw), key);
    const double thr = expo >= 0.0 ? 1.0 : exp(expo);
    if (u24d(w.x) < thr) {
      fp.perm[s0 + k] = b;
      fp.perm[s0 + k + 1] = a;
      fp.beta_slot[s0 + b] = static_cast<float>(bk);
      fp.beta_slot64[s0 + b] = bk;
      fp.bidx_slot[s0 + b] = k;
      fp.beta_slot[s0 + a] = static_cast<float>(bk1);
      fp.beta_slot64[s0 + a] = bk1;
      fp.bidx_slot[s0 + a] = k + 1;
      fp.acc_swap[s0 + k] += 1ull;
      ++count;
    }
  }
  if (fp.n_swapped && count) atomicAdd(fp.n_swapped, count);
}

// Finishing step of slot g, by one warp: its sums and record; on an
// exchanging sweep a lattice's slots are counted on fp.done[l] as they
// finish (after a fence), and the warp that finishes the last one runs the
// lattice's exchange and resets the count.  No warp waits for another.
__device__ __forceinline__ void finish_slot_and_exchange(const Lattice* lats, int n_lat, const FinishParams& fp,
                                                         int g, int lane) {
  int lo = 0, hi = n_lat - 1;  // the lattice of slot g: the last with slot0 <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (lats[mid].slot0 <= g) lo = mid;
    else hi = mid - 1;
  }
  const Lattice lat = lats[lo];
  finish_slot(lat, g - lat.slot0, fp, lane);
  if (!fp.swap) return;
  __threadfence();
  int last = 0;
  if (lane == 0) last = (atomicAdd(fp.done + lo, 1) == lat.R - 1) ? 1 : 0;
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  exchange_ladder(lat, lo, fp, lane, 32);
  if (lane == 0) fp.done[lo] = 0;
}

// Per-launch finishing step: one warp (block of 32 threads) per slot, for
// the slots g0, g0 + 1, ... (all of them, or one lattice's), so the FP64 sums
// of the slots run on as many SMs.
__global__ void k_finish(const Lattice* lats, int n_lat, FinishParams fp, int g0) {
  chain_wait_and_release();
  finish_slot_and_exchange(lats, n_lat, fp, g0 + static_cast<int>(blockIdx.x), threadIdx.x & 31);
}

__global__ void k_advance(uint64_t* ctr, uint64_t d_mpass, uint64_t d_sweep, uint64_t d_swap,
                          uint64_t d_records, uint64_t d_series) {
  chain_wait_and_release();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctr[kCtrMpass] += d_mpass;
    ctr[kCtrSweep] += d_sweep;
    ctr[kCtrSwap] += d_swap;
    ctr[kCtrRecords] += d_records;
    ctr[kCtrSeries] += d_series;
  }
}

// The fast-math expressions of the Metropolis update, evaluated one by one
// for accuracy checks with the same device functions the sweep kernels
// call.  kind 0: in = proposal words; out[2i], out[2i+1] = the proposal
// vector (cos, sin) of proposal_angle(w).  kind 1: in = exponents x (FP32);
// out[i] = accept_threshold(x).
__global__ void k_fast_math(int kind, long long n, const void* __restrict__ in, float* __restrict__ out) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    if (kind == 0) {
      float c, s;
      spin(proposal_angle(static_cast<const uint32_t*>(in)[i]), c, s);
      out[2 * i] = c;
      out[2 * i + 1] = s;
    } else if (kind == 1) {
      out[i] = accept_threshold(static_cast<const float*>(in)[i]);
    } else {
      // lane 0 of the paired atan2 the tile uses (both lanes take the pair)
      const float* xy2 = static_cast<const float*>(in);
      const float x = xy2[2 * i], y = xy2[2 * i + 1];
      out[i] = atan2_poly2(make_float2(y, y), make_float2(x, x)).x;
    }
  }
}

// Raw words of every site of one colour of local slot r, natural order of
// those sites (x fastest), two per site.
__global__ void k_draws(Lattice lat, int r, int colour, uint32_t tag, uint64_t count,
                        uint64_t seed, uint32_t* out) {
  const int L = lat.L, H = L >> 1;
  const long long half = static_cast<long long>(L) * L * L / 2;
  const PhiloxKey key = philox_key(seed);
  const uint32_t tagw = (static_cast<uint32_t>(lat.slot0 + r) << 4) |
                        (static_cast<uint32_t>(colour) << 3) | (tag & 7u);
  for (long long n = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; n < half;
       n += static_cast<long long>(gridDim.x) * blockDim.x) {
    // n-th site of this colour in natural order: row (y, z) = n / H, k = n % H.
    const long long row = n / H;
    const int k = static_cast<int>(n % H);
    const long long p = row * H + k;  // packed index equals the order index
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(p >> 1), static_cast<uint32_t>(count),
                                             static_cast<uint32_t>(count >> 32), tagw), key);
    out[2 * n] = (p & 1) ? w.z : w.x;
    out[2 * n + 1] = (p & 1) ? w.w : w.y;
  }
}

}  // namespace xy
