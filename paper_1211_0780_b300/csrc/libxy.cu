// libxy: the C-ABI of the XY sweep path (declared in include/xy.h).
//
// Host-side responsibilities: validate arguments, carve the caller's device
// workspace, issue the half-sweep kernels in the sweep schedule (plain
// launches, a captured CUDA graph, or persistent launches, one per part of
// a sweep),
// keep host mirrors of the device counters, and marshal state between the
// natural host layout and the packed device layout.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/xy.h"
#include "kernels.cuh"
#include "persistent.cuh"

using namespace xy;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
int conv_blocks(long long n) { return static_cast<int>(std::min<long long>((n + 255) / 256, 4096)); }

struct LatHost {
  int L, R, slot0;
  int kind;  // kTileMarch, kTileBlock, kTileStream or kTileDirect
  int ty, tz;
  size_t spin_off;  // floats from the spin base (2N per slot)
  long long words_off;  // uint4s from the words base (R N/2), or -1: no words region
  int part0;         // first partial slot
  int part_cap;      // partial slots reserved per slot
  long long N() const { return static_cast<long long>(L) * L * L; }
  int nyt() const { return (L + ty - 1) / ty; }
  int nzt() const { return (L + tz - 1) / tz; }
  int threads() const { return tile_threads(kind, L, ty, tz); }
  int smem() const { return tile_bytes(kind, L, ty, tz); }
};

// Partial capacity per slot: tiles of at least 4 sites x rows x planes.
int part_cap_for(int L) { return std::max(1, (L * L) / 4); }

struct Layout {
  size_t spins, ladder_beta, perm, beta_slot, beta_slot64, bidx_slot, E_slot, sums_slot, partials,
      acc_met, acc_swap, ctr, status, sync, nswapped, fin_done, words, words_bytes, lats, staging, plan_items, series, total;
};

constexpr int kMaxPlanBlocks = 8192;
// The persistent launches' item counter and per-slot completion counts.
size_t sync_bytes(long long slots) { return static_cast<size_t>(kSyncSlot0 + slots) * 8; }

bool valid_lattices(int n, const int* L, const int* R) {
  if (n <= 0 || n > 4096 || !L || !R) return false;
  for (int i = 0; i < n; ++i) {
    if (L[i] < 8 || L[i] > 1024 || L[i] % 8 != 0) return false;
    if (R[i] <= 0 || R[i] > (1 << 20)) return false;
  }
  return true;
}

// Whether a context keeps a words region: its (cos, sin) state, 8 bytes per
// site, at most 40 MB, so that state and words (another 8 bytes per site)
// fit in L2 together.
constexpr long long kWordsMaxStateBytes = 40ll << 20;
bool words_region(long long spin_floats) { return spin_floats * 4 <= kWordsMaxStateBytes; }

Layout layout_for(int n, const int* L, const int* R, int64_t series_cap) {
  Layout o{};
  size_t off = 0;
  long long spin_floats = 0, slots = 0, parts = 0, maxN = 0;
  for (int i = 0; i < n; ++i) {
    const long long N = static_cast<long long>(L[i]) * L[i] * L[i];
    spin_floats += 2 * N * R[i];  // (cos, sin) per site
    slots += R[i];
    parts += static_cast<long long>(part_cap_for(L[i])) * R[i];
    maxN = std::max(maxN, N);
  }
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  o.spins = take(static_cast<size_t>(spin_floats) * 4);
  o.ladder_beta = take(slots * 8);
  o.perm = take(slots * 4);
  o.beta_slot = take(slots * 4);
  o.beta_slot64 = take(slots * 8);
  o.bidx_slot = take(slots * 4);
  o.E_slot = take(slots * 8);
  o.sums_slot = take(slots * kNumSums * 8);
  o.partials = take(static_cast<size_t>(parts) * kNumSums * 8);
  o.acc_met = take(slots * 8);
  o.acc_swap = take(slots * 8);
  o.ctr = take(kNumCounters * 8);
  o.status = take(64);
  o.sync = take(sync_bytes(slots));
  o.nswapped = take(64);
  o.fin_done = take(static_cast<size_t>(n) * 4);
  // Metropolis words drawn ahead: one pass of every slot (16 B per two
  // sites), only for a vector state small enough that state and words stay
  // in L2 together
  o.words_bytes = words_region(spin_floats) ? static_cast<size_t>(spin_floats) * 4 : 0;
  o.words = take(o.words_bytes);
  o.lats = take(static_cast<size_t>(n) * sizeof(Lattice));
  o.staging = take(static_cast<size_t>(maxN) * 4);
  o.plan_items = take(static_cast<size_t>(parts) * sizeof(int4));
  o.series = take(static_cast<size_t>(std::max<int64_t>(series_cap, 0)) * slots * sizeof(xy_record));
  o.total = off;
  return o;
}

int lcm_int(int a, int b) { return a / std::gcd(a, b) * b; }

// The period after which the pattern of measured and exchanging sweeps
// repeats: lcm(me, se) of the periods that are set (1 if neither is).
uint64_t sweep_period(int me, int se) {
  const uint64_t a = me > 0 ? static_cast<uint64_t>(me) : 1u, b = se > 0 ? static_cast<uint64_t>(se) : 1u;
  return a / std::gcd(a, b) * b;
}

}  // namespace

struct xy_ctx {
  int n_lat = 0;
  int n_slots = 0;
  std::vector<LatHost> lat;
  std::vector<double> betas;  // ladder betas, slot-indexed per lattice
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  // One stream per lattice: the lattices' half-sweep chains run as
  // concurrent branches between the points where they must meet.
  std::vector<cudaStream_t> lat_streams;
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
  int device = 0;
  int num_sms = 0;
  int max_block = 1024;  // threads per block the half-sweep kernels can launch with
  Layout lay{};
  char* ws = nullptr;
  int64_t series_cap = 0;
  uint64_t h_ctr[kNumCounters] = {0};
  int exec = XY_EXEC_PLAIN;
  int sticky = XY_OK;
  std::map<std::tuple<int, int, int, int, int, long long, int>, cudaGraphExec_t> graphs;
  struct Plan {
    int G = 0, B = 0, smem = 0, kind = 0, n_items = 0;
    bool graph_ok = true;
  } plan;
  bool plan_valid = false;

  template <typename T>
  T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
  float* spins() const { return at<float>(lay.spins); }
  uint64_t* ctr() const { return at<uint64_t>(lay.ctr); }
  Lattice dev_lat(int i) const {
    const LatHost& h = lat[i];
    Lattice d;
    d.spins = spins() + h.spin_off;
    d.L = h.L;
    d.R = h.R;
    d.slot0 = h.slot0;
    d.ty = h.ty;
    d.tz = h.tz;
    d.nyt = h.nyt();
    d.nzt = h.nzt();
    d.kind = h.kind;
    d.part0 = h.part0;
    return d;
  }
  PassParams pass_params(bool use_ctr, uint64_t mpass_off, int measure) const {
    PassParams p{};
    p.rk = philox_round_keys(seed);
    p.ctr = use_ctr ? ctr() : nullptr;
    p.mpass_off = mpass_off;
    p.beta_slot = at<float>(lay.beta_slot);
    p.partials = at<double>(lay.partials);
    p.acc_met = at<unsigned long long>(lay.acc_met);
    p.measure = measure;
    p.poison = 0;
    p.own_ready = 0;
    p.status = at<int>(lay.status);
    p.wait_ns = 1000000000ll;  // a copied plane lands in microseconds
    return p;
  }
};

namespace {

thread_local char g_last_cuda_error[256] = {0};

// Threads a tile of this kind may have: the kTileDirect kernels are compiled
// for smaller blocks than the others.
int kind_max_threads(const xy_ctx* c, int kind) {
  return (kind == kTileDirect || kind == kTileAngle) ? std::min(c->max_block, kDirectMaxThreads) : c->max_block;
}

int fail_cuda(xy_ctx* c, cudaError_t e, const char* what) {
  std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s: %s", what, cudaGetErrorString(e));
  if (c) c->sticky = XY_ERR_CUDA;
  return XY_ERR_CUDA;
}

#define XY_TRY(c, call)                                      \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return fail_cuda((c), e_, #call); \
  } while (0)

#define XY_CHECK_LAUNCH(c) XY_TRY(c, cudaGetLastError())

// An NVTX range over one C-ABI call (host-side timeline markers for
// profilers; header-only, a no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

#define XY_ENTER(c)                                          \
  do {                                                       \
    if (!(c)) return XY_ERR_ARG;                             \
    if ((c)->sticky != XY_OK) return XY_ERR_STATE;           \
    XY_TRY((c), cudaSetDevice((c)->device));                 \
  } while (0)

// Synchronises the context's stream and reads the device status word: a
// bounded wait that ran out inside a kernel (a stream tile waiting for a
// copied plane, a persistent launch's wait for a slot's tiles) fails the context with
// XY_ERR_TIMEOUT.
int sync_checked(xy_ctx* c) {
  int st = 0;
  XY_TRY(c, cudaMemcpyAsync(&st, c->ws + c->lay.status, 4, cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  if (st != 0) {
    c->sticky = st == XY_ERR_BOUNDS ? XY_ERR_BOUNDS : XY_ERR_TIMEOUT;
    return c->sticky;
  }
  return XY_OK;
}

// Default tile: the block kind with up to 8 x 8 rows and at most 256 threads.
void default_tile(LatHost& h) {
  h.kind = kTileBlock;
  h.ty = std::min(h.L, 8);
  h.tz = std::min(h.L, 8);
  while (h.threads() > 256 && (h.ty > 1 || h.tz > 1)) {
    if (h.tz >= h.ty) h.tz = std::max(1, h.tz / 2);
    else h.ty = std::max(1, h.ty / 2);
  }
}

// Converts lattice i's stored state in place between vectors and angles
// when a change of tile kind changes its storage (kTileAngle keeps angles,
// every other kind vectors).  Ordered on the context's stream.
int convert_storage(xy_ctx* c, int i, bool to_angles) {
  const LatHost& h = c->lat[i];
  const long long N = h.N(), n = N * h.R;
  float* dst = c->spins() + h.spin_off;
  const int blocks = static_cast<int>(std::min<long long>((n + 255) / 256, 4096));
  if (to_angles)
    k_vectors_to_angles<<<blocks, 256, 0, c->stream>>>(dst, N, h.R);
  else
    k_angles_in_place<<<blocks, 256, 0, c->stream>>>(dst, N, h.R, 0);
  XY_CHECK_LAUNCH(c);
  return XY_OK;
}

int sync_lats(xy_ctx* c) {
  std::vector<Lattice> d(c->n_lat);
  for (int i = 0; i < c->n_lat; ++i) d[i] = c->dev_lat(i);
  XY_TRY(c, cudaMemcpyAsync(c->at<Lattice>(c->lay.lats), d.data(), sizeof(Lattice) * c->n_lat,
                            cudaMemcpyHostToDevice, c->stream));
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  return XY_OK;
}

void drop_graphs(xy_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  c->plan_valid = false;
}

// Launches a kernel of the half-sweep chain with programmatic stream
// serialization, so it is launched while its predecessor still runs and
// starts its work (after griddepcontrol.wait) as soon as that one is done.
template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                           Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// kTileDirect half-sweep, the kernel compiled for lattice size LC (0: any).
template <int MODE, int LC>
cudaError_t launch_direct(dim3 grid, dim3 block, int smem, cudaStream_t st, const Lattice& d, int colour,
                          const PassParams& pp) {
  static_assert(sizeof(kDirectSizes) / sizeof(kDirectSizes[0]) == 5, "one case per fixed size");
  constexpr int M = MODE == kMeasureOnly ? kOverrelax : MODE;
  if (MODE == kMeasureOnly) return launch_chained(k_half_direct<kMeasureOnly, true, LC>, grid, block, smem, st, d, colour, pp);
  if (pp.measure == 2 && colour == 1)
    return launch_chained(k_half_direct<M, true, LC, 0, true>, grid, block, smem, st, d, colour, pp);
  if (pp.measure && colour == 1) return launch_chained(k_half_direct<M, true, LC>, grid, block, smem, st, d, colour, pp);
  if (MODE == kMetropolis && pp.words && pp.words_read)
    return launch_chained(k_half_direct<M, false, LC, 1>, grid, block, smem, st, d, colour, pp);
  if (MODE == kOverrelax && pp.words && pp.gen_end > pp.gen_begin)
    return launch_chained(k_half_direct<M, false, LC, 2>, grid, block, smem, st, d, colour, pp);
  return launch_chained(k_half_direct<M, false, LC>, grid, block, smem, st, d, colour, pp);
}

// kTileAngle half-sweep (angle storage; L read at run time).
template <int MODE>
cudaError_t launch_angle(dim3 grid, dim3 block, int smem, cudaStream_t st, const Lattice& d, int colour,
                         const PassParams& pp) {
  constexpr int M = MODE == kMeasureOnly ? kOverrelax : MODE;
  if (MODE == kMeasureOnly) return launch_chained(k_half_angle<kMeasureOnly, true>, grid, block, smem, st, d, colour, pp);
  if (pp.measure == 2 && colour == 1)
    return launch_chained(k_half_angle<M, true, true>, grid, block, smem, st, d, colour, pp);
  if (pp.measure && colour == 1) return launch_chained(k_half_angle<M, true>, grid, block, smem, st, d, colour, pp);
  return launch_chained(k_half_angle<M, false>, grid, block, smem, st, d, colour, pp);
}

template <int MODE, int KIND>
cudaError_t launch_half_kind(const LatHost& h, const Lattice& d, cudaStream_t st, int colour,
                             const PassParams& pp) {
  const dim3 grid(h.nyt() * h.nzt(), h.R);
  const dim3 block = KIND == kTileBlock    ? dim3(h.L / 8, h.ty, h.tz)
                     : KIND == kTileStream ? dim3(tile_threads(KIND, h.L, h.ty, h.tz))
                                           : dim3(h.L / 8, h.ty);
  const int smem = h.smem();
  constexpr int M = MODE == kMeasureOnly ? kOverrelax : MODE;
  if constexpr (KIND == kTileDirect) {
    switch (h.L) {
      case kDirectSizes[0]: return launch_direct<MODE, kDirectSizes[0]>(grid, block, smem, st, d, colour, pp);
      case kDirectSizes[1]: return launch_direct<MODE, kDirectSizes[1]>(grid, block, smem, st, d, colour, pp);
      case kDirectSizes[2]: return launch_direct<MODE, kDirectSizes[2]>(grid, block, smem, st, d, colour, pp);
      case kDirectSizes[3]: return launch_direct<MODE, kDirectSizes[3]>(grid, block, smem, st, d, colour, pp);
      case kDirectSizes[4]: return launch_direct<MODE, kDirectSizes[4]>(grid, block, smem, st, d, colour, pp);
      default: return launch_direct<MODE, 0>(grid, block, smem, st, d, colour, pp);
    }
  } else if constexpr (KIND == kTileAngle) {
    return launch_angle<MODE>(grid, block, smem, st, d, colour, pp);
  } else {
    if (MODE == kMeasureOnly) return launch_chained(k_half<kMeasureOnly, true, KIND>, grid, block, smem, st, d, colour, pp);
    if (pp.measure && colour == 1) return launch_chained(k_half<M, true, KIND>, grid, block, smem, st, d, colour, pp);
    return launch_chained(k_half<M, false, KIND>, grid, block, smem, st, d, colour, pp);
  }
}

// The Metropolis words drawn ahead, for one half-sweep of issue_sweeps: a
// Metropolis half-sweep of a sweep's first pass reads the words the previous
// sweep's over-relaxation half-sweeps drew (read); over-relaxation
// half-sweep `part` of `parts` draws that share of the next sweep's words,
// for the pass counter offset `mpass`.  Only lattices on the direct tile in
// a context with a words region take part.
struct WordPlan {
  int read = 0;
  int part = 0, parts = 0;
  uint64_t mpass = 0;
};

template <int MODE>
int launch_half(xy_ctx* c, cudaStream_t st, int i, int colour, const PassParams& pp, const WordPlan& wp = WordPlan()) {
  const LatHost& h = c->lat[i];
  const Lattice d = c->dev_lat(i);
  PassParams q = pp;
  q.words = nullptr;
  q.words_read = 0;
  q.gen_begin = q.gen_end = 0;
  if (h.kind == kTileDirect && h.words_off >= 0 && (wp.read || wp.parts > 0)) {
    q.words = c->at<uint4>(c->lay.words) + h.words_off;
    q.words_read = wp.read;
    if (wp.parts > 0) {
      const uint64_t calls = static_cast<uint64_t>(h.R) * static_cast<uint64_t>(h.N() / 2);
      q.gen_begin = static_cast<uint32_t>(calls * wp.part / wp.parts);
      q.gen_end = static_cast<uint32_t>(calls * (wp.part + 1) / wp.parts);
      q.gen_mpass = wp.mpass;
    }
  }
  const cudaError_t e = h.kind == kTileBlock    ? launch_half_kind<MODE, kTileBlock>(h, d, st, colour, q)
                       : h.kind == kTileStream ? launch_half_kind<MODE, kTileStream>(h, d, st, colour, q)
                       : h.kind == kTileDirect ? launch_half_kind<MODE, kTileDirect>(h, d, st, colour, q)
                       : h.kind == kTileAngle  ? launch_half_kind<MODE, kTileAngle>(h, d, st, colour, q)
                                               : launch_half_kind<MODE, kTileMarch>(h, d, st, colour, q);
  XY_TRY(c, e);
  return XY_OK;
}

template <int MODE>
int launch_half_all(xy_ctx* c, cudaStream_t st, int colour, const PassParams& pp, const WordPlan& wp = WordPlan()) {
  for (int i = 0; i < c->n_lat; ++i) {
    const int rc = launch_half<MODE>(c, st, i, colour, pp, wp);
    if (rc != XY_OK) return rc;
  }
  return XY_OK;
}

FinishParams finish_params(xy_ctx* c) {
  FinishParams f{};
  f.partials = c->at<double>(c->lay.partials);
  f.sums_slot = c->at<double>(c->lay.sums_slot);
  f.E_slot = c->at<double>(c->lay.E_slot);
  f.ctr = c->ctr();
  f.series = c->at<xy_record>(c->lay.series);
  f.n_slots = c->n_slots;
  f.parity = -1;
  f.perm = c->at<int>(c->lay.perm);
  f.ladder_beta = c->at<double>(c->lay.ladder_beta);
  f.beta_slot = c->at<float>(c->lay.beta_slot);
  f.beta_slot64 = c->at<double>(c->lay.beta_slot64);
  f.bidx_slot = c->at<int>(c->lay.bidx_slot);
  f.acc_swap = c->at<unsigned long long>(c->lay.acc_swap);
  f.seed = c->seed;
  f.n_swapped = nullptr;
  f.done = c->at<int>(c->lay.fin_done);
  return f;
}

// The finishing step of slots [g0, g0 + n) (every slot: 0, n_slots).
int launch_finish(xy_ctx* c, cudaStream_t st, const FinishParams& f, int g0, int n) {
  XY_TRY(c, launch_chained(k_finish, dim3(n), dim3(32), 0, st,
                           static_cast<const Lattice*>(c->at<Lattice>(c->lay.lats)), c->n_lat, f, g0));
  return XY_OK;
}

bool due(uint64_t s, int every) { return every > 0 && (s + 1) % static_cast<uint64_t>(every) == 0; }

struct BlockCounts {
  uint64_t mpass = 0, sweeps = 0, swaps = 0, records = 0;
};

// Issues `ns` sweeps starting at host sweep index s0, relative to the device
// counters, followed by the counter advance.  No synchronisation.
// Lattices share nothing within a call (each has its own ladder, partial
// sums, records and words), so with several lattices each runs all of its
// sweeps, finishing steps and exchanges included, on its own stream: one
// fork and one join per call, and no lattice waits for another's sweep.
int issue_sweeps(xy_ctx* c, cudaStream_t st, int nM, int nOR, int ns, int me, int se, uint64_t s0,
                 BlockCounts* out) {
  // the call's counter offsets at the start of each sweep (at[ns]: the total)
  std::vector<BlockCounts> at(static_cast<size_t>(ns) + 1);
  for (int j = 0; j < ns; ++j) {
    const uint64_t s = s0 + j;
    at[j + 1] = at[j];
    at[j + 1].mpass += nM;
    at[j + 1].sweeps += 1;
    at[j + 1].records += due(s, me) ? 1 : 0;
    at[j + 1].swaps += due(s, se) ? 1 : 0;
  }
  const int n_pass = nM + nOR;
  const bool branches = c->n_lat > 1;
  if (branches) {
    XY_TRY(c, cudaEventRecord(c->fork_ev, st));
    for (int i = 0; i < c->n_lat; ++i) XY_TRY(c, cudaStreamWaitEvent(c->lat_streams[i], c->fork_ev, 0));
  }
  for (int i = 0; i < (branches ? c->n_lat : 1); ++i) {
    cudaStream_t ls = branches ? c->lat_streams[i] : st;
    for (int j = 0; j < ns; ++j) {
      const uint64_t s = s0 + j;
      const bool meas = due(s, me), swp = due(s, se);
      const bool needE = meas || swp;
      uint64_t mp = at[j].mpass;
      for (int p = 0; p < n_pass; ++p) {
        const bool last = (p == n_pass - 1);
        for (int colour = 0; colour < 2; ++colour) {
          // the sweep's last half-sweep measures: every sum when it records,
          // the energy alone when it only exchanges
          const int measure = (needE && last && colour == 1) ? (meas ? 1 : 2) : 0;
          PassParams pp = c->pass_params(true, p < nM ? mp : 0, measure);
          // Every half-sweep of a sweep but the first is chained behind the
          // other colour's half-sweep on the same stream (see tile_direct).
          pp.own_ready = (p > 0 || colour > 0) ? 1 : 0;
          // Metropolis words drawn ahead: the over-relaxation half-sweeps
          // after the sweep's first and before its last draw the next
          // sweep's first-pass words (no launch in flight reads them then:
          // the Metropolis half-sweeps that read the current ones completed
          // before the first of those launches passed its wait, and the next
          // sweep's first Metropolis half-sweep starts after the last one's),
          // which that pass reads instead of drawing.
          WordPlan wp;
          const int k = 2 * (p - nM) + colour;  // over-relaxation half-sweep of the sweep
          if (p == 0 && nM > 0 && nOR >= 2 && j > 0) wp.read = 1;
          if (p >= nM && nM > 0 && j + 1 < ns && k >= 1 && k <= 2 * nOR - 2 && !measure) {
            wp.part = k - 1;
            wp.parts = 2 * nOR - 2;
            wp.mpass = at[j].mpass + nM;
          }
          int rc;
          if (branches)
            rc = p < nM ? launch_half<kMetropolis>(c, ls, i, colour, pp, wp)
                        : launch_half<kOverrelax>(c, ls, i, colour, pp, wp);
          else
            rc = p < nM ? launch_half_all<kMetropolis>(c, ls, colour, pp, wp)
                        : launch_half_all<kOverrelax>(c, ls, colour, pp, wp);
          if (rc != XY_OK) return rc;
        }
        if (p < nM) mp += 1;
      }
      if (needE) {
        FinishParams f = finish_params(c);
        f.sweep_off = at[j].sweeps;
        f.series_off = at[j].records;
        f.swap_off = at[j].swaps;
        f.record = meas ? 1 : 0;
        f.swap = swp ? 1 : 0;
        const int rc = branches ? launch_finish(c, ls, f, c->lat[i].slot0, c->lat[i].R)
                                : launch_finish(c, ls, f, 0, c->n_slots);
        if (rc != XY_OK) return rc;
      }
    }
  }
  if (branches) {
    for (int i = 0; i < c->n_lat; ++i) {
      XY_TRY(c, cudaEventRecord(c->join_ev[i], c->lat_streams[i]));
      XY_TRY(c, cudaStreamWaitEvent(st, c->join_ev[i], 0));
    }
  }
  const BlockCounts& bc = at[ns];
  XY_TRY(c, launch_chained(k_advance, dim3(1), dim3(1), 0, st, c->ctr(), bc.mpass, bc.sweeps, bc.swaps,
                           bc.records, bc.records));
  if (out) *out = bc;
  return XY_OK;
}

void mirror_advance(xy_ctx* c, const BlockCounts& bc) {
  c->h_ctr[kCtrMpass] += bc.mpass;
  c->h_ctr[kCtrSweep] += bc.sweeps;
  c->h_ctr[kCtrSwap] += bc.swaps;
  c->h_ctr[kCtrRecords] += bc.records;
  c->h_ctr[kCtrSeries] += bc.records;
}

uint64_t count_due(uint64_t s0, uint64_t n, int every) {
  if (every <= 0) return 0;
  const uint64_t e = static_cast<uint64_t>(every);
  return (s0 + n) / e - s0 / e;
}

int run_graph_block(xy_ctx* c, int nM, int nOR, int me, int se, int P, uint64_t s0) {
  const auto key = std::make_tuple(nM, nOR, me, se, P, static_cast<long long>(s0 % P), 0);
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    XY_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    BlockCounts bc;
    const int rc = issue_sweeps(c, c->cap_stream, nM, nOR, P, me, se, s0, &bc);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (rc != XY_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail_cuda(c, e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e2 = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return fail_cuda(c, e2, "cudaGraphInstantiate");
    it = c->graphs.emplace(key, ex).first;
  }
  XY_TRY(c, cudaGraphLaunch(it->second, c->stream));
  return XY_OK;
}

int persistent_sweeps(xy_ctx* c, int nM, int nOR, int ns, int me, int se);

}  // namespace

// ------------------------------------------------------------------ C-ABI

extern "C" {

const char* xy_strerror(int status) {
  switch (status) {
    case XY_OK: return "ok";
    case XY_ERR_ARG: return "invalid argument";
    case XY_ERR_CUDA: return g_last_cuda_error[0] ? g_last_cuda_error : "CUDA error";
    case XY_ERR_TIMEOUT: return "device-side wait timed out";
    case XY_ERR_STATE: return "context is in an error state";
    case XY_ERR_NOMEM: return "buffer too small";
    case XY_ERR_BOUNDS: return "out-of-bounds access skipped (bounds-checked build)";
    default: return "unknown status";
  }
}

size_t xy_workspace_bytes(int n_lattices, const int* L, const int* n_replicas, int64_t series_capacity) {
  if (!valid_lattices(n_lattices, L, n_replicas) || series_capacity < 0) return 0;
  return layout_for(n_lattices, L, n_replicas, series_capacity).total;
}

int xy_init(xy_ctx** out, int n_lattices, const int* L, const int* n_replicas, const double* betas,
            uint64_t seed, void* d_workspace, size_t ws_bytes, int64_t series_capacity, void* stream) {
  if (!out) return XY_ERR_ARG;
  *out = nullptr;
  if (!valid_lattices(n_lattices, L, n_replicas) || !betas || !d_workspace || series_capacity < 0)
    return XY_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_workspace) % kAlign != 0) return XY_ERR_ARG;
  int off = 0;
  for (int i = 0; i < n_lattices; ++i) {
    for (int k = 0; k < n_replicas[i]; ++k) {
      const double b = betas[off + k];
      if (!std::isfinite(b) || b < 0.0) return XY_ERR_ARG;
      if (k > 0 && !(b > betas[off + k - 1])) return XY_ERR_ARG;
    }
    off += n_replicas[i];
  }
  const Layout lay = layout_for(n_lattices, L, n_replicas, series_capacity);
  if (ws_bytes < lay.total) return XY_ERR_NOMEM;

  xy_ctx* c = new xy_ctx();
  c->n_lat = n_lattices;
  c->seed = seed;
  c->stream = static_cast<cudaStream_t>(stream);
  c->lay = lay;
  c->ws = static_cast<char*>(d_workspace);
  c->series_cap = series_capacity;
  size_t aoff = 0;
  int slot = 0, part = 0;
  for (int i = 0; i < n_lattices; ++i) {
    LatHost h;
    h.L = L[i];
    h.R = n_replicas[i];
    h.slot0 = slot;
    default_tile(h);
    h.spin_off = aoff;
    // the words region mirrors the spin region: R N/2 uint4s per lattice
    h.words_off = lay.words_bytes ? static_cast<long long>(aoff / 4) : -1;
    h.part_cap = part_cap_for(h.L);
    h.part0 = part;
    aoff += 2 * static_cast<size_t>(h.N()) * h.R;  // (cos, sin) per site
    slot += h.R;
    part += h.part_cap * h.R;
    c->lat.push_back(h);
  }
  c->n_slots = slot;
  c->betas.assign(betas, betas + slot);

  auto bail = [&](int rc) {
    xy_destroy(c);
    return rc;
  };
  // The workspace's device is the context's device.
  cudaPointerAttributes pa{};
  cudaError_t e = cudaPointerGetAttributes(&pa, d_workspace);
  if (e != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    xy_destroy(c);
    return XY_ERR_ARG;
  }
  c->device = pa.device;
  e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return bail(fail_cuda(nullptr, e, "cudaSetDevice"));
  e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) return bail(fail_cuda(nullptr, e, "cudaDeviceGetAttribute"));
  e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(fail_cuda(nullptr, e, "cudaStreamCreateWithFlags"));
  if (n_lattices > 1) {
    e = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(fail_cuda(nullptr, e, "cudaEventCreateWithFlags"));
    c->lat_streams.assign(n_lattices, nullptr);
    c->join_ev.assign(n_lattices, nullptr);
    for (int i = 0; i < n_lattices; ++i) {
      e = cudaStreamCreateWithFlags(&c->lat_streams[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join_ev[i], cudaEventDisableTiming);
      if (e != cudaSuccess) return bail(fail_cuda(nullptr, e, "lattice streams"));
    }
  }
  const void* half_kernels[15] = {
      reinterpret_cast<const void*>(k_half<kMetropolis, false, kTileMarch>),
      reinterpret_cast<const void*>(k_half<kMetropolis, true, kTileMarch>),
      reinterpret_cast<const void*>(k_half<kOverrelax, false, kTileMarch>),
      reinterpret_cast<const void*>(k_half<kOverrelax, true, kTileMarch>),
      reinterpret_cast<const void*>(k_half<kMeasureOnly, true, kTileMarch>),
      reinterpret_cast<const void*>(k_half<kMetropolis, false, kTileBlock>),
      reinterpret_cast<const void*>(k_half<kMetropolis, true, kTileBlock>),
      reinterpret_cast<const void*>(k_half<kOverrelax, false, kTileBlock>),
      reinterpret_cast<const void*>(k_half<kOverrelax, true, kTileBlock>),
      reinterpret_cast<const void*>(k_half<kMeasureOnly, true, kTileBlock>),
      reinterpret_cast<const void*>(k_half<kMetropolis, false, kTileStream>),
      reinterpret_cast<const void*>(k_half<kMetropolis, true, kTileStream>),
      reinterpret_cast<const void*>(k_half<kOverrelax, false, kTileStream>),
      reinterpret_cast<const void*>(k_half<kOverrelax, true, kTileStream>),
      reinterpret_cast<const void*>(k_half<kMeasureOnly, true, kTileStream>)};
  for (const void* fn : half_kernels) {
    // Tiles need up to ~64 KB of shared memory on the largest lattices.
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return bail(fail_cuda(nullptr, e, "cudaFuncSetAttribute"));
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return bail(fail_cuda(nullptr, e, "cudaFuncGetAttributes"));
    c->max_block = std::min(c->max_block, fa.maxThreadsPerBlock);
  }
  // The kTileDirect and kTileAngle kernels: their own block limit
  // (kDirectMaxThreads); the angle tile keeps its plane buffers in shared
  // memory (up to ~50 KB at L = 1024).
  const void* direct_kernels[14] = {
      reinterpret_cast<const void*>(k_half_direct<kMetropolis, false, 0>),
      reinterpret_cast<const void*>(k_half_direct<kMetropolis, true, 0>),
      reinterpret_cast<const void*>(k_half_direct<kOverrelax, false, 0>),
      reinterpret_cast<const void*>(k_half_direct<kOverrelax, true, 0>),
      reinterpret_cast<const void*>(k_half_direct<kMetropolis, true, 0, 0, true>),
      reinterpret_cast<const void*>(k_half_direct<kOverrelax, true, 0, 0, true>),
      reinterpret_cast<const void*>(k_half_direct<kMeasureOnly, true, 0>),
      reinterpret_cast<const void*>(k_half_angle<kMetropolis, false>),
      reinterpret_cast<const void*>(k_half_angle<kMetropolis, true>),
      reinterpret_cast<const void*>(k_half_angle<kOverrelax, false>),
      reinterpret_cast<const void*>(k_half_angle<kOverrelax, true>),
      reinterpret_cast<const void*>(k_half_angle<kMetropolis, true, true>),
      reinterpret_cast<const void*>(k_half_angle<kOverrelax, true, true>),
      reinterpret_cast<const void*>(k_half_angle<kMeasureOnly, true>)};
  for (const void* fn : direct_kernels) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return bail(fail_cuda(nullptr, e, "cudaFuncSetAttribute"));
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return bail(fail_cuda(nullptr, e, "cudaFuncGetAttributes"));
    if (fa.maxThreadsPerBlock < kDirectMaxThreads) return bail(XY_ERR_CUDA);
  }
  for (LatHost& h : c->lat)
    while (h.threads() > c->max_block && (h.ty > 1 || h.tz > 1)) {
      if (h.tz >= h.ty) h.tz = std::max(1, h.tz / 2);
      else h.ty = std::max(1, h.ty / 2);
    }

  // Ladder tables: identity permutation, each slot at its own beta.
  std::vector<int> perm(slot), bidx(slot);
  std::vector<float> bs(slot);
  for (const LatHost& h : c->lat)
    for (int k = 0; k < h.R; ++k) {
      perm[h.slot0 + k] = k;
      bidx[h.slot0 + k] = k;
      bs[h.slot0 + k] = static_cast<float>(betas[h.slot0 + k]);
    }
  cudaStream_t st = c->stream;
  auto cp = [&](size_t off, const void* src, size_t n) {
    return cudaMemcpyAsync(c->ws + off, src, n, cudaMemcpyHostToDevice, st);
  };
  if ((e = cp(lay.ladder_beta, betas, slot * 8)) != cudaSuccess ||
      (e = cp(lay.perm, perm.data(), slot * 4)) != cudaSuccess ||
      (e = cp(lay.beta_slot, bs.data(), slot * 4)) != cudaSuccess ||
      (e = cp(lay.beta_slot64, betas, slot * 8)) != cudaSuccess ||
      (e = cp(lay.bidx_slot, bidx.data(), slot * 4)) != cudaSuccess)
    return bail(fail_cuda(nullptr, e, "cudaMemcpyAsync"));
  if ((e = cudaMemsetAsync(c->ws + lay.acc_met, 0, slot * 8, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->ws + lay.acc_swap, 0, slot * 8, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->ws + lay.ctr, 0, kNumCounters * 8, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->ws + lay.status, 0, 64, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->ws + lay.fin_done, 0, static_cast<size_t>(n_lattices) * 4, st)) != cudaSuccess)
    return bail(fail_cuda(nullptr, e, "cudaMemsetAsync"));
  int rc = sync_lats(c);
  if (rc != XY_OK) return bail(rc);
  for (int i = 0; i < n_lattices; ++i) {
    const long long pairs = c->lat[i].N() / 2 * c->lat[i].R;
    const int blocks = static_cast<int>(std::min<long long>((pairs + 255) / 256, 65535));
    k_init<<<blocks, 256, 0, st>>>(c->dev_lat(i), seed);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bail(fail_cuda(nullptr, e, "k_init"));
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bail(fail_cuda(nullptr, e, "cudaStreamSynchronize"));
  *out = c;
  return XY_OK;
}

int xy_destroy(xy_ctx* c) {
  if (!c) return XY_OK;
  // let the context's work finish before its graphs, streams and events go
  // (and before the caller frees the workspace); a failed context's error
  // is not reported again here
  cudaStreamSynchronize(c->stream);
  if (c->cap_stream) cudaStreamSynchronize(c->cap_stream);
  drop_graphs(c);
  for (cudaStream_t s : c->lat_streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t ev : c->join_ev)
    if (ev) cudaEventDestroy(ev);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return XY_OK;
}

int xy_set_exec(xy_ctx* c, int mode) {
  XY_ENTER(c);
  if (mode != XY_EXEC_PLAIN && mode != XY_EXEC_GRAPH && mode != XY_EXEC_PERSISTENT) return XY_ERR_ARG;
  c->exec = mode;
  return XY_OK;
}

int xy_sweep(xy_ctx* c, int nM, int nOR, int n_sweeps, int me, int se) {
  const NvtxRange nvtx_range("xy_sweep");
  XY_ENTER(c);
  if (nM < 0 || nOR < 0 || n_sweeps < 0 || me < 0 || se < 0) return XY_ERR_ARG;
  if (n_sweeps == 0) return XY_OK;
  if (nM + nOR == 0) return XY_ERR_ARG;
  const uint64_t s0 = c->h_ctr[kCtrSweep];
  const uint64_t n_meas = count_due(s0, n_sweeps, me);
  if (c->h_ctr[kCtrSeries] + n_meas > static_cast<uint64_t>(c->series_cap)) return XY_ERR_NOMEM;

  if (c->exec == XY_EXEC_PERSISTENT) return persistent_sweeps(c, nM, nOR, n_sweeps, me, se);

  if (c->exec == XY_EXEC_GRAPH) {
    const int P0 = lcm_int(me > 0 ? me : 1, se > 0 ? se : 1);
    if (P0 <= 64 && n_sweeps >= P0) {
      // a graph holds P sweeps: whole periods, up to ~16 sweeps
      const int P = P0 * std::max(1, std::min(16 / P0, n_sweeps / P0));
      int done = 0;
      while (n_sweeps - done >= P) {
        const uint64_t s = c->h_ctr[kCtrSweep];
        const int rc = run_graph_block(c, nM, nOR, me, se, P, s);
        if (rc != XY_OK) return rc;
        BlockCounts bc;
        bc.mpass = static_cast<uint64_t>(nM) * P;
        bc.sweeps = P;
        bc.swaps = count_due(s, P, se);
        bc.records = count_due(s, P, me);
        mirror_advance(c, bc);
        done += P;
      }
      if (done < n_sweeps) {
        BlockCounts bc;
        const int rc = issue_sweeps(c, c->stream, nM, nOR, n_sweeps - done, me, se, c->h_ctr[kCtrSweep], &bc);
        if (rc != XY_OK) return rc;
        mirror_advance(c, bc);
      }
      return XY_OK;
    }
  }
  BlockCounts bc;
  const int rc = issue_sweeps(c, c->stream, nM, nOR, n_sweeps, me, se, s0, &bc);
  if (rc != XY_OK) return rc;
  mirror_advance(c, bc);
  return XY_OK;
}

int xy_metropolis_half(xy_ctx* c, int colour, uint64_t mpass) {
  XY_ENTER(c);
  if (colour != 0 && colour != 1) return XY_ERR_ARG;
  return launch_half_all<kMetropolis>(c, c->stream, colour, c->pass_params(false, mpass, 0));
}

int xy_overrelax_half(xy_ctx* c, int colour) {
  XY_ENTER(c);
  if (colour != 0 && colour != 1) return XY_ERR_ARG;
  return launch_half_all<kOverrelax>(c, c->stream, colour, c->pass_params(false, 0, 0));
}

static int measure_now(xy_ctx* c, int swap, int parity) {
  int rc = launch_half_all<kMeasureOnly>(c, c->stream, 1, c->pass_params(false, 0, 1));
  if (rc != XY_OK) return rc;
  FinishParams f = finish_params(c);
  f.record = 0;
  f.swap = swap;
  f.parity = parity;
  f.n_swapped = swap ? c->at<int>(c->lay.nswapped) : nullptr;
  return launch_finish(c, c->stream, f, 0, c->n_slots);
}

int xy_measure(xy_ctx* c, xy_record* out) {
  const NvtxRange nvtx_range("xy_measure");
  XY_ENTER(c);
  if (!out) return XY_ERR_ARG;
  int rc = measure_now(c, 0, 0);
  if (rc != XY_OK) return rc;
  const int S = c->n_slots;
  std::vector<double> sums(static_cast<size_t>(S) * kNumSums), E(S), b64(S);
  std::vector<int> bidx(S);
  XY_TRY(c, cudaMemcpyAsync(sums.data(), c->ws + c->lay.sums_slot, sums.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaMemcpyAsync(E.data(), c->ws + c->lay.E_slot, S * 8, cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaMemcpyAsync(b64.data(), c->ws + c->lay.beta_slot64, S * 8, cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaMemcpyAsync(bidx.data(), c->ws + c->lay.bidx_slot, S * 4, cudaMemcpyDeviceToHost, c->stream));
  if ((rc = sync_checked(c)) != XY_OK) return rc;
  for (int g = 0; g < S; ++g) {
    xy_record& r = out[g];
    const double* v = &sums[static_cast<size_t>(g) * kNumSums];
    r.E = E[g];
    r.Mx = v[0];
    r.My = v[1];
    for (int mu = 0; mu < 3; ++mu) {
      r.C[mu] = v[2 + mu];
      r.S[mu] = v[5 + mu];
    }
    r.beta = b64[g];
    r.slot = g;
    r.beta_index = bidx[g];
    r.sweep = c->h_ctr[kCtrSweep];
  }
  return XY_OK;
}

int xy_pt_swap(xy_ctx* c, int parity, int* n_accepted_out) {
  const NvtxRange nvtx_range("xy_pt_swap");
  XY_ENTER(c);
  if (parity != 0 && parity != 1) return XY_ERR_ARG;
  XY_TRY(c, cudaMemsetAsync(c->ws + c->lay.nswapped, 0, 4, c->stream));
  int rc = measure_now(c, 1, parity);
  if (rc != XY_OK) return rc;
  k_advance<<<1, 1, 0, c->stream>>>(c->ctr(), 0, 0, 1, 0, 0);
  XY_CHECK_LAUNCH(c);
  c->h_ctr[kCtrSwap] += 1;
  int n = 0;
  XY_TRY(c, cudaMemcpyAsync(&n, c->ws + c->lay.nswapped, 4, cudaMemcpyDeviceToHost, c->stream));
  if ((rc = sync_checked(c)) != XY_OK) return rc;
  if (n_accepted_out) *n_accepted_out = n;
  return XY_OK;
}

int xy_series_count(xy_ctx* c, int64_t* n_out) {
  XY_ENTER(c);
  if (!n_out) return XY_ERR_ARG;
  *n_out = static_cast<int64_t>(c->h_ctr[kCtrSeries]) * c->n_slots;
  return XY_OK;
}

int xy_read_series(xy_ctx* c, xy_record* buf, int64_t cap, int64_t* n_out) {
  XY_ENTER(c);
  if (!n_out || (cap > 0 && !buf) || cap < 0) return XY_ERR_ARG;
  const int64_t n = static_cast<int64_t>(c->h_ctr[kCtrSeries]) * c->n_slots;
  *n_out = 0;
  if (n > cap) return XY_ERR_NOMEM;
  if (n > 0) {
    XY_TRY(c, cudaMemcpyAsync(buf, c->ws + c->lay.series, n * sizeof(xy_record), cudaMemcpyDeviceToHost, c->stream));
  }
  XY_TRY(c, cudaMemsetAsync(c->ws + c->lay.ctr + kCtrSeries * 8, 0, 8, c->stream));
  const int rc = sync_checked(c);
  if (rc != XY_OK) return rc;
  c->h_ctr[kCtrSeries] = 0;
  *n_out = n;
  return XY_OK;
}

int xy_get_state(xy_ctx* c, float* host_angles, int32_t* perm, uint64_t* counters) {
  XY_ENTER(c);
  if (host_angles) {
    size_t at = 0;
    for (const LatHost& h : c->lat) {
      const long long N = h.N();
      const int Hh = h.L / 2;
      std::vector<float> packed(static_cast<size_t>(N));
      for (int r = 0; r < h.R; ++r) {
        float* stage = c->at<float>(c->lay.staging);
        k_to_angles<<<conv_blocks(N), 256, 0, c->stream>>>(c->spins() + h.spin_off + 2 * r * N, N, stage,
                                                           angle_storage(h.kind) ? 1 : 0);
        XY_CHECK_LAUNCH(c);
        XY_TRY(c, cudaMemcpyAsync(packed.data(), stage, N * 4, cudaMemcpyDeviceToHost, c->stream));
        XY_TRY(c, cudaStreamSynchronize(c->stream));
        float* dst = host_angles + at;
        for (int z = 0; z < h.L; ++z)
          for (int y = 0; y < h.L; ++y)
            for (int x = 0; x < h.L; ++x) {
              const int col = (x + y + z) & 1;
              const long long p = (x >> 1) + static_cast<long long>(Hh) * (y + static_cast<long long>(h.L) * z);
              dst[x + static_cast<long long>(h.L) * (y + static_cast<long long>(h.L) * z)] = packed[col * (N / 2) + p];
            }
        at += static_cast<size_t>(N);
      }
    }
  }
  if (perm) XY_TRY(c, cudaMemcpyAsync(perm, c->ws + c->lay.perm, c->n_slots * 4, cudaMemcpyDeviceToHost, c->stream));
  if (counters) XY_TRY(c, cudaMemcpyAsync(counters, c->ctr(), 4 * 8, cudaMemcpyDeviceToHost, c->stream));
  return sync_checked(c);
}

int xy_set_state(xy_ctx* c, const float* host_angles, const int32_t* perm, const uint64_t* counters) {
  XY_ENTER(c);
  if (perm) {
    for (const LatHost& h : c->lat) {
      std::vector<int> seen(h.R, 0);
      for (int k = 0; k < h.R; ++k) {
        const int v = perm[h.slot0 + k];
        if (v < 0 || v >= h.R || seen[v]) return XY_ERR_ARG;
        seen[v] = 1;
      }
    }
  }
  if (host_angles) {
    size_t at = 0;
    for (const LatHost& h : c->lat) {
      const long long N = h.N();
      const int Hh = h.L / 2;
      std::vector<float> packed(static_cast<size_t>(N));
      for (int r = 0; r < h.R; ++r) {
        const float* src = host_angles + at;
        for (int z = 0; z < h.L; ++z)
          for (int y = 0; y < h.L; ++y)
            for (int x = 0; x < h.L; ++x) {
              const int col = (x + y + z) & 1;
              const long long p = (x >> 1) + static_cast<long long>(Hh) * (y + static_cast<long long>(h.L) * z);
              float v = src[x + static_cast<long long>(h.L) * (y + static_cast<long long>(h.L) * z)];
              if (!std::isfinite(v)) return XY_ERR_ARG;
              packed[col * (N / 2) + p] = v;
            }
        float* stage = c->at<float>(c->lay.staging);
        XY_TRY(c, cudaMemcpyAsync(stage, packed.data(), N * 4, cudaMemcpyHostToDevice, c->stream));
        k_from_angles<<<conv_blocks(N), 256, 0, c->stream>>>(stage, N, c->spins() + h.spin_off + 2 * r * N,
                                                             angle_storage(h.kind) ? 1 : 0);
        XY_CHECK_LAUNCH(c);
        XY_TRY(c, cudaStreamSynchronize(c->stream));
        at += static_cast<size_t>(N);
      }
    }
  }
  if (perm) {
    const int S = c->n_slots;
    std::vector<int> pv(perm, perm + S), bidx(S);
    std::vector<float> bs(S);
    std::vector<double> b64(S);
    for (const LatHost& h : c->lat)
      for (int k = 0; k < h.R; ++k) {
        const int g = h.slot0 + pv[h.slot0 + k];
        bidx[g] = k;
        b64[g] = c->betas[h.slot0 + k];
        bs[g] = static_cast<float>(b64[g]);
      }
    XY_TRY(c, cudaMemcpyAsync(c->ws + c->lay.perm, pv.data(), S * 4, cudaMemcpyHostToDevice, c->stream));
    XY_TRY(c, cudaMemcpyAsync(c->ws + c->lay.bidx_slot, bidx.data(), S * 4, cudaMemcpyHostToDevice, c->stream));
    XY_TRY(c, cudaMemcpyAsync(c->ws + c->lay.beta_slot, bs.data(), S * 4, cudaMemcpyHostToDevice, c->stream));
    XY_TRY(c, cudaMemcpyAsync(c->ws + c->lay.beta_slot64, b64.data(), S * 8, cudaMemcpyHostToDevice, c->stream));
  }
  if (counters) {
    uint64_t v[kNumCounters] = {0};
    for (int i = 0; i < 4; ++i) v[i] = counters[i];
    v[kCtrSeries] = c->h_ctr[kCtrSeries];
    XY_TRY(c, cudaMemcpyAsync(c->ctr(), v, 4 * 8, cudaMemcpyHostToDevice, c->stream));
    for (int i = 0; i < 4; ++i) c->h_ctr[i] = counters[i];
  }
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  return XY_OK;
}

int xy_set_betas(xy_ctx* c, int lattice, const double* betas) {
  XY_ENTER(c);
  if (lattice < 0 || lattice >= c->n_lat || !betas) return XY_ERR_ARG;
  const LatHost& h = c->lat[lattice];
  for (int k = 0; k < h.R; ++k) {
    if (!std::isfinite(betas[k])) return XY_ERR_ARG;
    if (k > 0 && !(betas[k] > betas[k - 1])) return XY_ERR_ARG;
  }
  // The permutation (beta index -> slot) stays; every slot takes the new
  // beta of its index.
  std::vector<int> perm(h.R);
  XY_TRY(c, cudaMemcpyAsync(perm.data(), c->ws + c->lay.perm + 4 * static_cast<size_t>(h.slot0), 4 * h.R,
                            cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  std::vector<double> b64(h.R);
  std::vector<float> bs(h.R);
  for (int k = 0; k < h.R; ++k) {
    c->betas[h.slot0 + k] = betas[k];
    b64[perm[k]] = betas[k];
    bs[perm[k]] = static_cast<float>(betas[k]);
  }
  const size_t o8 = 8 * static_cast<size_t>(h.slot0), o4 = 4 * static_cast<size_t>(h.slot0);
  XY_TRY(c, cudaMemcpyAsync(c->ws + c->lay.ladder_beta + o8, betas, 8 * h.R, cudaMemcpyHostToDevice, c->stream));
  XY_TRY(c, cudaMemcpyAsync(c->ws + c->lay.beta_slot64 + o8, b64.data(), 8 * h.R, cudaMemcpyHostToDevice, c->stream));
  XY_TRY(c, cudaMemcpyAsync(c->ws + c->lay.beta_slot + o4, bs.data(), 4 * h.R, cudaMemcpyHostToDevice, c->stream));
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  return XY_OK;
}

int xy_get_packed(xy_ctx* c, float* host_packed) {
  XY_ENTER(c);
  if (!host_packed) return XY_ERR_ARG;
  size_t n = 0;
  for (const LatHost& h : c->lat) n += 2 * static_cast<size_t>(h.N()) * h.R;
  XY_TRY(c, cudaMemcpyAsync(host_packed, c->spins(), n * 4, cudaMemcpyDeviceToHost, c->stream));
  return sync_checked(c);
}

int xy_set_packed(xy_ctx* c, const float* host_packed) {
  XY_ENTER(c);
  if (!host_packed) return XY_ERR_ARG;
  size_t n = 0;
  for (const LatHost& h : c->lat) n += 2 * static_cast<size_t>(h.N()) * h.R;
  XY_TRY(c, cudaMemcpyAsync(c->spins(), host_packed, n * 4, cudaMemcpyHostToDevice, c->stream));
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  return XY_OK;
}

int xy_set_packed_angles(xy_ctx* c, const float* host_angles) {
  XY_ENTER(c);
  if (!host_angles) return XY_ERR_ARG;
  size_t at = 0;
  for (const LatHost& h : c->lat) {
    const long long N = h.N();
    float* dst = c->spins() + h.spin_off;
    // each slot's colour 0 and colour 1 angles (N/2 each) into the two
    // colours' cos arrays (N floats apart), then converted in place
    XY_TRY(c, cudaMemcpy2DAsync(dst, static_cast<size_t>(N) * 4, host_angles + at, static_cast<size_t>(N / 2) * 4,
                                static_cast<size_t>(N / 2) * 4, static_cast<size_t>(2 * h.R), cudaMemcpyHostToDevice,
                                c->stream));
    const long long n = N * h.R;
    k_angles_in_place<<<static_cast<int>(std::min<long long>((n + 255) / 256, 4096)), 256, 0, c->stream>>>(
        dst, N, h.R, angle_storage(h.kind) ? 1 : 0);
    XY_CHECK_LAUNCH(c);
    at += static_cast<size_t>(n);
  }
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  return XY_OK;
}

int xy_host_alloc(size_t bytes, void** out) {
  if (!out || bytes == 0) return XY_ERR_ARG;
  *out = nullptr;
  void* p = nullptr;
  if (cudaHostAlloc(&p, bytes, cudaHostAllocPortable) != cudaSuccess) {
    cudaGetLastError();  // not sticky: nothing else depends on this call
    return XY_ERR_CUDA;
  }
  *out = p;
  return XY_OK;
}

int xy_host_free(void* p) {
  if (!p) return XY_OK;
  if (cudaFreeHost(p) != cudaSuccess) {
    cudaGetLastError();
    return XY_ERR_CUDA;
  }
  return XY_OK;
}

int xy_get_packed_angles(xy_ctx* c, float* host_angles) {
  XY_ENTER(c);
  if (!host_angles) return XY_ERR_ARG;
  size_t at = 0;
  float* stage = c->at<float>(c->lay.staging);
  for (const LatHost& h : c->lat) {
    const long long N = h.N();
    for (int r = 0; r < h.R; ++r) {
      k_to_angles<<<conv_blocks(N), 256, 0, c->stream>>>(c->spins() + h.spin_off + 2 * r * N, N, stage,
                                                         angle_storage(h.kind) ? 1 : 0);
      XY_CHECK_LAUNCH(c);
      XY_TRY(c, cudaMemcpyAsync(host_angles + at, stage, static_cast<size_t>(N) * 4, cudaMemcpyDeviceToHost,
                                c->stream));
      XY_TRY(c, cudaStreamSynchronize(c->stream));
      at += static_cast<size_t>(N);
    }
  }
  return sync_checked(c);
}

int xy_get_accepts(xy_ctx* c, uint64_t* met, uint64_t* swap) {
  XY_ENTER(c);
  if (met) XY_TRY(c, cudaMemcpyAsync(met, c->ws + c->lay.acc_met, c->n_slots * 8, cudaMemcpyDeviceToHost, c->stream));
  if (swap) XY_TRY(c, cudaMemcpyAsync(swap, c->ws + c->lay.acc_swap, c->n_slots * 8, cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  return XY_OK;
}

int xy_debug_draws(xy_ctx* c, int slot, int colour, int tag, uint64_t count, uint32_t* host_words) {
  XY_ENTER(c);
  if (!host_words || slot < 0 || slot >= c->n_slots || (colour != 0 && colour != 1) || tag < 0 || tag > 7)
    return XY_ERR_ARG;
  int i = 0;
  while (!(slot >= c->lat[i].slot0 && slot < c->lat[i].slot0 + c->lat[i].R)) ++i;
  const LatHost& h = c->lat[i];
  const long long half = h.N() / 2;
  uint32_t* dev = c->at<uint32_t>(c->lay.staging);  // room for N words = 2 * half
  const int blocks = static_cast<int>(std::min<long long>((half + 255) / 256, 65535));
  k_draws<<<blocks, 256, 0, c->stream>>>(c->dev_lat(i), slot - h.slot0, colour, static_cast<uint32_t>(tag), count, c->seed, dev);
  XY_CHECK_LAUNCH(c);
  XY_TRY(c, cudaMemcpyAsync(host_words, dev, 2 * half * 4, cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  return XY_OK;
}

int xy_debug_fast_math(int kind, int64_t n, const void* d_in, float* d_out, void* stream) {
  if (kind < 0 || kind > 2 || n < 0 || (n > 0 && (!d_in || !d_out))) return XY_ERR_ARG;
  if (n == 0) return XY_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, 16384));
  k_fast_math<<<blocks, 256, 0, st>>>(kind, static_cast<long long>(n), d_in, d_out);
  XY_TRY(nullptr, cudaGetLastError());
  XY_TRY(nullptr, cudaStreamSynchronize(st));
  return XY_OK;
}

int xy_set_tile(xy_ctx* c, int lattice, int kind, int ty, int tz) {
  XY_ENTER(c);
  if (lattice < 0 || lattice >= c->n_lat) return XY_ERR_ARG;
  if (kind != kTileMarch && kind != kTileBlock && kind != kTileStream && kind != kTileDirect && kind != kTileAngle)
    return XY_ERR_ARG;
  LatHost h = c->lat[lattice];
  h.kind = kind;
  h.ty = ty;
  h.tz = tz;
  if (ty < 1 || tz < 1 || ty > h.L || tz > h.L || h.threads() > kind_max_threads(c, kind)) return XY_ERR_ARG;
  if (kind == kTileBlock && tz > 64) return XY_ERR_ARG;  // block z extent
  if (h.nyt() * h.nzt() > h.part_cap) return XY_ERR_ARG;
  if (h.smem() > 200 * 1024) return XY_ERR_ARG;
  if (angle_storage(h.kind) != angle_storage(c->lat[lattice].kind)) {
    const int rc = convert_storage(c, lattice, angle_storage(h.kind));
    if (rc != XY_OK) return rc;
  }
  c->lat[lattice] = h;
  drop_graphs(c);
  return sync_lats(c);
}

int xy_get_tile(xy_ctx* c, int lattice, int* kind, int* ty, int* tz) {
  XY_ENTER(c);
  if (lattice < 0 || lattice >= c->n_lat || !kind || !ty || !tz) return XY_ERR_ARG;
  *kind = c->lat[lattice].kind;
  *ty = c->lat[lattice].ty;
  *tz = c->lat[lattice].tz;
  return XY_OK;
}

int xy_device_status(xy_ctx* c, int* status_out) {
  XY_ENTER(c);
  if (!status_out) return XY_ERR_ARG;
  XY_TRY(c, cudaMemcpyAsync(status_out, c->ws + c->lay.status, 4, cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  return XY_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ persistent path

namespace {

// The persistent kernel of one tile kind, sweep part and finishing flag.
// eo (fin): the finishing launch of a sweep that only exchanges.
const void* persistent_kernel(int kind, int part, bool fin, bool eo) {
#define XY_PK(K)                                                                                              \
  (part == kPartMetropolis                                                                                    \
       ? (fin ? (eo ? reinterpret_cast<const void*>(k_persistent<K, kPartMetropolis, true, true>)             \
                    : reinterpret_cast<const void*>(k_persistent<K, kPartMetropolis, true>))                  \
              : reinterpret_cast<const void*>(k_persistent<K, kPartMetropolis, false>))                       \
   : fin ? (eo ? reinterpret_cast<const void*>(k_persistent<K, kPartOverrelax, true, true>)                   \
               : reinterpret_cast<const void*>(k_persistent<K, kPartOverrelax, true>))                        \
         : reinterpret_cast<const void*>(k_persistent<K, kPartOverrelax, false>))
  return kind == kTileBlock    ? XY_PK(kTileBlock)
         : kind == kTileDirect ? XY_PK(kTileDirect)
         : kind == kTileAngle  ? XY_PK(kTileAngle)
                               : XY_PK(kTileMarch);
#undef XY_PK
}

// The tile work items of one half-sweep in decreasing order of cost (the
// blocks take them in this order: longest-processing-time-first) and the
// grid of the persistent launches.  Cost of a tile ~ (rows + 2)(planes + 2)
// x row length: the update work including the halos.
int build_plan(xy_ctx* c) {
  if (c->plan_valid) return XY_OK;
  int B = 64, smem = 0;
  const int kind = c->lat[0].kind;
  for (const LatHost& h : c->lat) {
    if (h.kind != kind) return XY_ERR_ARG;  // one tile kind per persistent launch
    // stream tiles copy planes with TMA, which does not see what other blocks
    // of the same launch wrote
    if (h.kind == kTileStream) return XY_ERR_ARG;
    B = std::max(B, h.threads());
    smem = std::max(smem, h.smem());
  }
  B = (B + 31) / 32 * 32;
  // Every part's kernel runs on the same grid and item plan: the grid is
  // sized by the part that keeps the fewest blocks per SM.
  int nb = 1 << 30;
  for (int v = 0; v < 6; ++v) {  // (part, fin) = (v >> 1, v & 1); v = 4, 5: the energy-only finishing parts
    const void* fn = v < 4 ? persistent_kernel(kind, v >> 1, (v & 1) != 0, false)
                           : persistent_kernel(kind, v - 4, true, true);
    cudaFuncAttributes fa{};
    XY_TRY(c, cudaFuncGetAttributes(&fa, fn));
    if (B > fa.maxThreadsPerBlock) return XY_ERR_ARG;  // a tile wider than one persistent block
    XY_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    int n = 0;
    XY_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, B, smem));
    nb = std::min(nb, n);
  }
  if (nb <= 0) return XY_ERR_ARG;
  struct Item {
    int4 w;
    double cost;
  };
  std::vector<Item> items;
  for (int i = 0; i < c->n_lat; ++i) {
    const LatHost& h = c->lat[i];
    for (int r = 0; r < h.R; ++r)
      for (int t = 0; t < h.nyt() * h.nzt(); ++t) {
        const int yt = t % h.nyt(), zt = t / h.nyt();
        const int tya = std::min(h.ty, h.L - yt * h.ty), tza = std::min(h.tz, h.L - zt * h.tz);
        items.push_back({make_int4(i, r, t, 0), double(tya + 2) * double(tza + 2) * (h.L / 8)});
      }
  }
  const int G = static_cast<int>(std::min<long long>(
      std::min<long long>(static_cast<long long>(nb) * c->num_sms, kMaxPlanBlocks), std::max<size_t>(items.size(), 1)));
  std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.cost > b.cost; });
  std::vector<int4> flat(items.size());
  for (size_t i = 0; i < items.size(); ++i) flat[i] = items[i].w;
  XY_TRY(c, cudaMemcpyAsync(c->ws + c->lay.plan_items, flat.data(), flat.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream));
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  c->plan.G = G;
  c->plan.n_items = static_cast<int>(items.size());
  c->plan.B = B;
  c->plan.smem = smem;
  c->plan.kind = kind;
  c->plan_valid = true;
  return XY_OK;
}

PersistentArgs persistent_args(xy_ctx* c) {
  PersistentArgs a{};
  a.pp = c->pass_params(true, 0, 0);
  a.fp = finish_params(c);
  a.lats = c->at<Lattice>(c->lay.lats);
  a.items = c->at<int4>(c->lay.plan_items);
  a.n_items = c->plan.n_items;
  a.n_lat = c->n_lat;
  unsigned long long* sync = c->at<unsigned long long>(c->lay.sync);
  a.work = sync;
  a.cnt = sync + kSyncSlot0;
  a.status = c->at<int>(c->lay.status);
  a.budget_ns = 2000000000ll;
  a.poison = 0;
  return a;
}

// One persistent launch; `chained`: programmatic dependent launch after the
// previous persistent launch of the same call (its blocks start as the
// previous launch's blocks leave; the slot counts order the work).
cudaError_t launch_persistent(xy_ctx* c, cudaStream_t st, const PersistentArgs& a, int part, bool fin,
                              bool chained) {
  const bool eo = fin && a.pp.measure == 2;  // a finishing launch that sums the energy alone
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(c->plan.G);
  cfg.blockDim = dim3(c->plan.B);
  cfg.dynamicSmemBytes = c->plan.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  void* args[] = {const_cast<PersistentArgs*>(&a)};
  return cudaLaunchKernelExC(&cfg, persistent_kernel(c->plan.kind, part, fin, eo), args);
}

// Issues the persistent launches of `ns` sweeps starting at host sweep
// index s0 on `st` -- the counters' reset, then per sweep the Metropolis
// part and the over-relaxation part, the last of them finishing measured or
// exchanging sweeps -- followed by the counter advance.  No
// synchronisation.
cudaError_t issue_persistent(xy_ctx* c, cudaStream_t st, int nM, int nOR, int ns, int me, int se, uint64_t s0,
                             const BlockCounts& bc) {
  PersistentArgs a = persistent_args(c);
  unsigned long long* const work[2] = {a.work, a.work + kSyncWork1};
  unsigned long long work_base[2] = {0ull, 0ull};
  cudaError_t e = cudaMemsetAsync(a.work, 0, sync_bytes(c->n_slots), st);
  uint64_t n_rec = 0, n_swp = 0;
  int n_launch = 0;
  a.hs0 = 0;
  a.fin0 = 0;
  for (int s = 0; s < ns && e == cudaSuccess; ++s) {
    const bool meas = due(s0 + s, me), swp = due(s0 + s, se);
    for (int part = kPartMetropolis; part <= kPartOverrelax && e == cudaSuccess; ++part) {
      const int n_pass = part == kPartMetropolis ? nM : nOR;
      if (n_pass == 0) continue;
      // the sweep's last part leaves its last half-sweep to the finishing launch
      const bool finishes = (meas || swp) && (part == kPartOverrelax || nOR == 0);
      a.fp.sweep_off = s;
      a.fp.series_off = n_rec;
      a.fp.swap_off = n_swp;
      a.fp.record = meas ? 1 : 0;
      a.fp.swap = swp ? 1 : 0;
      for (int fin = 0; fin < (finishes ? 2 : 1) && e == cudaSuccess; ++fin) {
        a.n_half = fin ? 1 : 2 * n_pass - (finishes ? 1 : 0);
        if (a.n_half == 0) continue;
        // the pass counter offset of the launch's first pass (the kernel
        // adds the later passes' index)
        a.pp.mpass_off = part == kPartMetropolis ? static_cast<uint64_t>(s) * nM + (fin ? n_pass - 1 : 0) : 0ull;
        // the finishing launch's half-sweep measures every sum when the
        // sweep records, the energy alone when it only exchanges
        a.pp.measure = fin ? (meas ? 1 : 2) : 0;
        const int q = n_launch & 1;
        a.work = work[q];
        a.work0 = work_base[q];
        e = launch_persistent(c, st, a, part, fin != 0, n_launch > 0);
        // every block makes one grab that finds the list empty
        work_base[q] += static_cast<unsigned long long>(
                            persistent_items(a.n_half, c->plan.n_items, fin != 0, c->n_slots, c->plan.B)) +
                        static_cast<unsigned long long>(c->plan.G);
        a.hs0 += static_cast<unsigned long long>(a.n_half);
        if (fin) a.fin0 += 1ull;
        ++n_launch;
      }
    }
    n_rec += meas ? 1 : 0;
    n_swp += swp ? 1 : 0;
  }
  if (e == cudaSuccess) {
    k_advance<<<1, 1, 0, st>>>(c->ctr(), bc.mpass, bc.sweeps, bc.swaps, bc.records, bc.records);
    e = cudaGetLastError();
  }
  return e;
}

int persistent_sweeps(xy_ctx* c, int nM, int nOR, int ns, int me, int se) {
  int rc = build_plan(c);
  if (rc != XY_OK) return rc;
  const uint64_t s0 = c->h_ctr[kCtrSweep];
  BlockCounts bc;
  bc.mpass = static_cast<uint64_t>(nM) * ns;
  bc.sweeps = ns;
  bc.swaps = count_due(s0, ns, se);
  bc.records = count_due(s0, ns, me);
  bool launched = false;
  if (c->plan.graph_ok) {
    // The kernels read the device counters; which sweeps measure or
    // exchange, and the counter advance, depend on the phase of s0 against
    // the two periods.
    const auto key = std::make_tuple(nM, nOR, ns, me, se, static_cast<long long>(s0 % sweep_period(me, se)), 1);
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return fail_cuda(c, e, "cudaStreamBeginCapture");
      const cudaError_t e2 = issue_persistent(c, c->cap_stream, nM, nOR, ns, me, se, s0, bc);
      e = cudaStreamEndCapture(c->cap_stream, &g);
      if (e2 == cudaSuccess && e == cudaSuccess) {
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail_cuda(c, e, "cudaGraphInstantiate");
        it = c->graphs.emplace(key, ex).first;
      } else {
        // The launches could not be captured: launch directly.
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        c->plan.graph_ok = false;
      }
    }
    if (c->plan.graph_ok) {
      XY_TRY(c, cudaGraphLaunch(it->second, c->stream));
      launched = true;
    }
  }
  if (!launched) XY_TRY(c, issue_persistent(c, c->stream, nM, nOR, ns, me, se, s0, bc));
  mirror_advance(c, bc);
  return sync_checked(c);
}

}  // namespace

extern "C" {

int xy_debug_barrier_timeout(xy_ctx* c, int budget_us, int* status_out) {
  XY_ENTER(c);
  if (budget_us <= 0 || budget_us > 2000000) return XY_ERR_ARG;
  int rc = build_plan(c);
  if (rc != XY_OK) return rc;
  PersistentArgs a = persistent_args(c);
  a.poison = 1;
  a.budget_ns = static_cast<long long>(budget_us) * 1000;
  XY_TRY(c, cudaMemsetAsync(a.work, 0, sync_bytes(c->n_slots), c->stream));
  XY_TRY(c, cudaMemsetAsync(a.status, 0, 4, c->stream));
  a.n_half = 1;
  XY_TRY(c, launch_persistent(c, c->stream, a, kPartOverrelax, false, false));
  int st = 0;
  XY_TRY(c, cudaMemcpyAsync(&st, a.status, 4, cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaMemsetAsync(a.status, 0, 4, c->stream));
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  if (status_out) *status_out = st;
  return st == 0 ? XY_OK : XY_ERR_TIMEOUT;
}

int xy_debug_stream_timeout(xy_ctx* c, int budget_us, int* status_out) {
  XY_ENTER(c);
  if (budget_us <= 0 || budget_us > 2000000) return XY_ERR_ARG;
  if (c->lat[0].kind != kTileStream) return XY_ERR_ARG;
  PassParams pp = c->pass_params(false, 0, 0);
  pp.poison = 1;
  pp.wait_ns = static_cast<long long>(budget_us) * 1000;
  XY_TRY(c, cudaMemsetAsync(pp.status, 0, 4, c->stream));
  const int rc = launch_half<kOverrelax>(c, c->stream, 0, 0, pp);
  if (rc != XY_OK) return rc;
  int st = 0;
  XY_TRY(c, cudaMemcpyAsync(&st, pp.status, 4, cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaMemsetAsync(pp.status, 0, 4, c->stream));
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  if (status_out) *status_out = st;
  return st == 0 ? XY_OK : XY_ERR_TIMEOUT;
}

int xy_autotune(xy_ctx* c, int nM, int nOR) {
  const NvtxRange nvtx_range("xy_autotune");
  XY_ENTER(c);
  if (nM < 0 || nOR < 0 || nM + nOR == 0) return XY_ERR_ARG;
  // Save what trial sweeps change: spins, counters, Metropolis accepts, and
  // (persistent trials exchange on ladders of two or more replicas) the
  // ladders' permutations, couplings and exchange counts.
  const size_t spin_bytes = c->lay.ladder_beta - c->lay.spins;
  const size_t S = static_cast<size_t>(c->n_slots);
  std::vector<char> saved(spin_bytes);
  std::vector<char> ctr(kNumCounters * 8), acc(S * 8);
  const std::pair<size_t, size_t> ladder_parts[] = {{c->lay.perm, S * 4},        {c->lay.beta_slot, S * 4},
                                                    {c->lay.beta_slot64, S * 8}, {c->lay.bidx_slot, S * 4},
                                                    {c->lay.acc_swap, S * 8}};
  std::vector<std::vector<char>> ladder(5);
  XY_TRY(c, cudaMemcpyAsync(saved.data(), c->ws + c->lay.spins, spin_bytes, cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaMemcpyAsync(ctr.data(), c->ws + c->lay.ctr, ctr.size(), cudaMemcpyDeviceToHost, c->stream));
  XY_TRY(c, cudaMemcpyAsync(acc.data(), c->ws + c->lay.acc_met, acc.size(), cudaMemcpyDeviceToHost, c->stream));
  for (int k = 0; k < 5; ++k) {
    ladder[k].resize(ladder_parts[k].second);
    XY_TRY(c, cudaMemcpyAsync(ladder[k].data(), c->ws + ladder_parts[k].first, ladder_parts[k].second,
                              cudaMemcpyDeviceToHost, c->stream));
  }
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  uint64_t h_ctr[kNumCounters];
  std::memcpy(h_ctr, c->h_ctr, sizeof h_ctr);
  const int exec = c->exec;
  c->exec = XY_EXEC_PLAIN;
  cudaEvent_t e0, e1;
  XY_TRY(c, cudaEventCreate(&e0));
  XY_TRY(c, cudaEventCreate(&e1));
  int rc = XY_OK;
  const bool persistent = exec == XY_EXEC_PERSISTENT;
  // Angle storage (kTileAngle) is a candidate only when the context's
  // vector state does not fit in L2: there the half-sweeps are bound by HBM
  // bytes, which it halves; an L2-resident state keeps its vectors.
  int l2 = 0;
  XY_TRY(c, cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device));
  const bool allow_angle = spin_bytes > static_cast<size_t>(l2);
  const int kind_end = allow_angle ? kTileAngle + 1 : kTileAngle;
  // The storage each lattice's state is in now (trial sweeps of a kind run
  // on its storage; the saved state is in the storage of the starting kind).
  std::vector<char> stored_ang(c->n_lat), start_ang(c->n_lat);
  for (int i = 0; i < c->n_lat; ++i) stored_ang[i] = start_ang[i] = angle_storage(c->lat[i].kind) ? 1 : 0;
  auto ensure_storage = [&](int i, int kind) {
    const char want = angle_storage(kind) ? 1 : 0;
    if (rc == XY_OK && stored_ang[i] != want) {
      rc = convert_storage(c, i, want != 0);
      stored_ang[i] = want;
    }
  };
  // Fastest tile of lattice i among kinds [k0, k1) and blocks of at most
  // max_threads threads, timed on half-sweep launches.
  auto search = [&](int i, int k0, int k1, int max_threads) {
    LatHost& h = c->lat[i];
    const LatHost start = h;
    float best = 1e30f;
    LatHost best_h = h;
    const int zs[] = {1, 2, 4, 8, 16, 32};
    for (int kind = k0; kind < k1 && rc == XY_OK; ++kind) {
      for (int ty = 1; ty <= h.L && rc == XY_OK; ++ty) {
        if (h.L % ty != 0) continue;
        for (int tz : zs) {
          if (tz > h.L || h.L % tz != 0) continue;
          LatHost cand = start;
          cand.kind = kind;
          cand.ty = ty;
          cand.tz = tz;
          if (kind != kTileBlock && tz < 2) continue;  // a march covers two planes or more
          if (cand.threads() > std::min(max_threads, kind_max_threads(c, kind)) || cand.threads() < 32) continue;
          if (cand.nyt() * cand.nzt() > h.part_cap || cand.smem() > 200 * 1024) continue;
          ensure_storage(i, kind);
          if (rc != XY_OK) break;
          h = cand;
          if ((rc = sync_lats(c)) != XY_OK) break;
          auto run = [&](int reps) {
            int r2 = XY_OK;
            for (int rep = 0; rep < reps && r2 == XY_OK; ++rep)
              for (int p = 0; p < nM + nOR && r2 == XY_OK; ++p)
                for (int col = 0; col < 2 && r2 == XY_OK; ++col)
                  r2 = p < nM ? launch_half<kMetropolis>(c, c->stream, i, col, c->pass_params(false, 0, 0))
                              : launch_half<kOverrelax>(c, c->stream, i, col, c->pass_params(false, 0, 0));
            return r2;
          };
          if ((rc = run(1)) != XY_OK) break;
          // the faster of two timed trials (close candidates are otherwise
          // ordered by timing noise)
          float ms = 1e30f;
          for (int trial = 0; trial < 2 && rc == XY_OK; ++trial) {
            if (cudaEventRecord(e0, c->stream) != cudaSuccess) { rc = fail_cuda(c, cudaGetLastError(), "autotune"); break; }
            if ((rc = run(3)) != XY_OK) break;
            float t = 0.f;
            if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
              rc = fail_cuda(c, cudaGetLastError(), "autotune");
              break;
            }
            ms = std::min(ms, t);
          }
          if (rc != XY_OK) break;
          if (ms < best) {
            best = ms;
            best_h = h;
          }
        }
      }
    }
    h = best_h;
  };
  // Whole sweeps are timed on sweeps that end with an exchange when a ladder
  // has two or more replicas (parallel tempering; the finishing step's cost
  // differs between kinds and shapes), else on plain sweeps, in the
  // context's execution mode.
  int swap_every = 0;
  for (const LatHost& h : c->lat) swap_every = h.R > 1 ? 1 : swap_every;
  // four sweeps: long enough that timing noise orders close sets rarely
  constexpr int kTrialSweeps = 4;
  auto trial_sweeps = [&]() -> int {
    if (persistent) return persistent_sweeps(c, nM, nOR, kTrialSweeps, 0, swap_every);
    if (exec == XY_EXEC_GRAPH) {
      c->exec = XY_EXEC_GRAPH;
      const int r = xy_sweep(c, nM, nOR, kTrialSweeps, 0, swap_every);
      c->exec = XY_EXEC_PLAIN;
      return r;
    }
    return issue_sweeps(c, c->stream, nM, nOR, kTrialSweeps, 0, swap_every, c->h_ctr[kCtrSweep], nullptr);
  };
  // Time of a few sweeps with a set of tiles: an untimed call first (it
  // builds the call's graph: capture and instantiation are host work that
  // would otherwise fall inside the timed region), then the fastest of three
  // timed calls; 1e30 for a set the execution mode cannot run.
  auto time_set = [&](const std::vector<LatHost>& set) -> float {
    c->lat = set;
    for (int i = 0; i < c->n_lat; ++i) ensure_storage(i, c->lat[i].kind);
    if (rc != XY_OK) return 1e30f;
    drop_graphs(c);
    if ((rc = sync_lats(c)) != XY_OK) return 1e30f;
    if (trial_sweeps() != XY_OK) {
      rc = c->sticky;
      return 1e30f;
    }
    float ms = 1e30f;
    for (int trial = 0; trial < 3 && rc == XY_OK; ++trial) {
      if (cudaEventRecord(e0, c->stream) != cudaSuccess) { rc = fail_cuda(c, cudaGetLastError(), "autotune"); break; }
      if ((rc = trial_sweeps()) != XY_OK) break;
      float t = 0.f;
      if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
        rc = fail_cuda(c, cudaGetLastError(), "autotune");
        break;
      }
      ms = std::min(ms, t);
    }
    return ms;
  };
  // The shapes come from per-launch timings of one lattice at a time:
  // refine a set on whole sweeps of every lattice together, one lattice at
  // a time (largest first), by doubling or halving its tile's rows or
  // planes within the blocks of at most max_threads threads, keeping a
  // change that is at least 1% faster.
  auto refine = [&](std::vector<LatHost> cur, float best, int max_threads) {
    std::vector<int> order(c->n_lat);
    for (int i = 0; i < c->n_lat; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return cur[a].N() * cur[a].R > cur[b].N() * cur[b].R; });
    for (int i : order) {
      if (rc != XY_OK || best >= 1e29f) break;
      const LatHost h0 = cur[i];
      const int cand_ty[4] = {h0.ty * 2, h0.ty / 2, h0.ty, h0.ty};
      const int cand_tz[4] = {h0.tz, h0.tz, h0.tz * 2, h0.tz / 2};
      for (int k = 0; k < 4 && rc == XY_OK; ++k) {
        LatHost h = h0;
        h.ty = cand_ty[k];
        h.tz = cand_tz[k];
        if (h.ty < 1 || h.tz < 1 || h.ty > h.L || h.tz > h.L || h.L % h.ty != 0 || h.L % h.tz != 0) continue;
        if (h.kind != kTileBlock && h.tz < 2) continue;
        if (h.tz > 32) continue;  // the range the per-launch search covers
        if (h.threads() > std::min(max_threads, kind_max_threads(c, h.kind)) || h.threads() < 32) continue;
        if (h.nyt() * h.nzt() > h.part_cap || h.smem() > 200 * 1024) continue;
        std::vector<LatHost> cand = cur;
        cand[i] = h;
        const float ms = time_set(cand);
        if (rc == XY_OK && ms < 0.99f * best) {
          best = ms;
          cur = cand;
        }
      }
    }
    return cur;
  };
  if (!persistent) {
    for (int i = 0; i < c->n_lat && rc == XY_OK; ++i) search(i, 0, kind_end, c->max_block);
    if (rc == XY_OK) {
      const std::vector<LatHost> found = c->lat;
      const std::vector<LatHost> cur = refine(found, time_set(found), c->max_block);
      if (rc == XY_OK) c->lat = cur;
    }
  } else {
    // One tile kind and one block size serve every lattice of a persistent
    // launch (the block is as wide as the widest tile): for each kind (not
    // the stream kind) and each cap on the tile's threads (64, 128, 256),
    // take each lattice's best tile under the cap, then time the persistent
    // launch itself with each set, keep the fastest and refine it.
    const int kinds[4] = {kTileMarch, kTileBlock, kTileDirect, kTileAngle};
    const int n_sets = 3 * (allow_angle ? 4 : 3);
    std::vector<std::vector<LatHost>> sets(n_sets);
    const std::vector<LatHost> start = c->lat;
    for (int q = 0; q < n_sets && rc == XY_OK; ++q) {
      const int kind = kinds[q / 3], cap = 64 << (q % 3);
      c->lat = start;
      for (int i = 0; i < c->n_lat && rc == XY_OK; ++i) search(i, kind, kind + 1, cap);
      sets[q] = c->lat;
    }
    float best = 1e30f;
    int best_q = n_sets - 1;
    for (int q = 0; q < n_sets && rc == XY_OK; ++q) {
      const float ms = time_set(sets[q]);
      if (rc == XY_OK && ms < best) {
        best = ms;
        best_q = q;
      }
    }
    const std::vector<LatHost> cur = refine(sets[best_q], best, kPersistentBlockThreads);
    if (rc == XY_OK) c->lat = cur;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->exec = exec;
  if (rc != XY_OK) return rc;
  rc = sync_lats(c);
  if (rc != XY_OK) return rc;
  XY_TRY(c, cudaMemcpyAsync(c->ws + c->lay.spins, saved.data(), spin_bytes, cudaMemcpyHostToDevice, c->stream));
  XY_TRY(c, cudaMemcpyAsync(c->ws + c->lay.ctr, ctr.data(), ctr.size(), cudaMemcpyHostToDevice, c->stream));
  XY_TRY(c, cudaMemcpyAsync(c->ws + c->lay.acc_met, acc.data(), acc.size(), cudaMemcpyHostToDevice, c->stream));
  for (int k = 0; k < 5; ++k)
    XY_TRY(c, cudaMemcpyAsync(c->ws + ladder_parts[k].first, ladder[k].data(), ladder_parts[k].second,
                              cudaMemcpyHostToDevice, c->stream));
  // the restored state is in each lattice's starting storage
  for (int i = 0; i < c->n_lat; ++i)
    if ((angle_storage(c->lat[i].kind) ? 1 : 0) != start_ang[i]) {
      rc = convert_storage(c, i, start_ang[i] == 0);
      if (rc != XY_OK) return rc;
    }
  XY_TRY(c, cudaStreamSynchronize(c->stream));
  std::memcpy(c->h_ctr, h_ctr, sizeof h_ctr);
  drop_graphs(c);
  return XY_OK;
}

}  // extern "C"
