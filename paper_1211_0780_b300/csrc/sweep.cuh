// Checkerboard half-sweep of the 3D XY model on sm_103a: Metropolis
// (Sec. II, Fig. 2), over-relaxation (Sec. II, Eq. 2) and the lattice sums of
// Eqs. (4)-(6), fused into one tile pass.
//
// State.  A spin is stored as its unit vector S = (cos theta, sin theta) in
// FP32, not as its angle: the reflection of Eq. (2) is then plain vector
// arithmetic, S' = 2 (S.h / h.h) h - S, and neither the neighbour cos/sin nor
// an arctangent is evaluated on the hot path.  Metropolis proposals
// theta' = 2 pi u are turned into vectors once, when drawn.  Angles are
// computed only when the state is read out.
//
// Layout.  Each slot (replica) of an L^3 lattice holds colour 0 then colour
// 1; each colour is a packed cos array then a packed sin array of N/2 floats;
// site (x, y, z) of colour c = (x+y+z) & 1 sits at p = (x >> 1) + (L/2)(y + L z)
// of both arrays of colour c.  A row (y, z) of one colour is L/2 contiguous
// floats per component, so a thread owns one float4 per component = 4
// same-colour sites of a row (x = 2k + s, k = 4 tx .. 4 tx + 3, with
// s = (y + z + c) & 1).  Its six neighbours are all of the other colour:
//   x-1, x+1 -> same row, packed k-1+s and k+s (one element comes from the
//               neighbouring float4, with periodic wrap along the row);
//   y+-1, z+-1 -> the other colour's rows (y+-1, z), (y, z+-1) at the same k.
//
// Tile (the march, kTileMarch).  A thread block covers full rows in x, `ty`
// rows in y and marches over `tz` planes in z.  A thread loads its own row
// of the other colour's plane z+1 and keeps planes z-1, z, z+1 of its own
// column in registers; planes are shared through three shared-memory
// buffers (one barrier per plane) for the y neighbours and the x halo
// element.  The thread rows at the tile's y edges also load the halo rows
// y0-1 and y0+ty.  The plane loop is unrolled three times so the register
// planes and the buffer indices rotate without copies.  The other tile kinds
// (block, stream, direct; see TileKind) keep this thread layout or this
// update and change how neighbour rows reach the thread.
//
// Accuracy.  The reflection renormalises its result with one Newton step
// towards |S| = 1, so stored vectors stay within a few ulp of the unit
// circle however many reflections a spin goes through; the direction (the
// angle) is not changed by that step.  Proposal vectors use the fast sincos,
// evaluated at theta - pi inside [-pi, pi) (absolute error ~2^-21.4).
#pragma once
#include <cstdint>

#include "../../include/xy.h"
#include "atan_poly.cuh"
#include "philox.cuh"

namespace xy {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kTwoPiOver2p24 = 6.28318530717958647692f / 16777216.0f;  // exact scaling
constexpr uint32_t kTagInit = 1u, kTagMet = 2u, kTagPt = 3u;
constexpr int kNumSums = 8;                       // Mx, My, Cx, Cy, Cz, Sx, Sy, Sz
constexpr int kReduceBytes = kNumSums * 32 * 8;   // per-warp FP64 partials

enum Mode : int { kMetropolis = 0, kOverrelax = 1, kMeasureOnly = 2 };

// Tile kinds.  kTileMarch: a block of (L/8) x ty threads marches over tz
// planes (each other-colour site loaded ~once, but the planes are processed
// in sequence).  kTileBlock: a block of (L/8) x ty x tz threads updates its
// whole tile at once after one cooperative staging of the tile's
// other-colour rows and face halos (more loads, no sequence).
// kTileStream: the march of kTileMarch, but every plane the tile needs
// (the other colour's rows with their y halo, the own colour's rows) is
// brought into a ring of shared-memory stages by bulk asynchronous copies
// (TMA) that run ahead of the computation; threads only read shared memory
// and store their results.
// kTileDirect: the march of kTileMarch without shared memory and without a
// block barrier: each thread loads its y-neighbour rows and its x-halo
// element itself, through the L1 cache (the rows it reads are the rows its
// neighbouring threads load for their own columns), one plane ahead, so
// every warp marches on its own.  In the persistent kernel the grid
// barrier between half-sweeps (an acquire, then the block barrier) orders
// these loads after the previous half-sweep's writes.
// kTileAngle: the direct tile on a lattice stored as FP32 angles instead of
// vectors (4 instead of 8 bytes per spin, for lattices that do not fit in
// L2, where the half-sweep is bound by HBM bytes): every angle read is
// turned into its vector with the fast sincos, and the update stores the
// new angle (the proposal's, or atan2 of the reflected vector).
enum TileKind : int { kTileMarch = 0, kTileBlock = 1, kTileStream = 2, kTileDirect = 3, kTileAngle = 4 };

// Whether a tile kind keeps the lattice as angles (else as vectors).
__host__ __device__ inline bool angle_storage(int kind) { return kind == kTileAngle; }

// Threads of a kTileDirect block at most, and the registers a thread of its
// kernel may use.  Each of an SM's four schedulers holds 16K registers, so
// at 128 registers a thread it keeps four warps and three blocks of 160
// threads (a 160^3 tile of 8 rows) stay resident per SM; at 129-136 only
// three warps per scheduler and two blocks fit.  (The measuring variants
// spill some words at this limit; measured on B300 that is faster than two
// blocks per SM.)
// The plain over-relaxation variant runs 1% faster at 120 (measured at
// 160^3; Metropolis runs 4% slower there).
constexpr int kDirectMaxThreads = 240;
constexpr int kDirectMaxRegs = 128;
constexpr int kDirectMaxRegsOR = 120;
// The angle tile's plain over-relaxation variant at most 96 registers
// (81 used, no spills): five to six blocks of 128 threads per SM instead of
// four, which the plane barrier and the load latency of the 128^3 x 16
// half-sweep need (277 -> 329 updates/ns on the 8 x 16 tile; Metropolis
// keeps kDirectMaxRegs, where a cap cost it 10%).
constexpr int kAngleMaxRegsOR = 96;
// Lattice sizes for which the kTileDirect kernels are also compiled with L
// fixed: those of the paper's runs (Sec. III: L = 64, 80, 96, 128, 160);
// other sizes use the kernels that read L at run time.  (At 160^3 the fixed
// size makes both half-sweeps about 3% faster.)
constexpr int kDirectSizes[] = {64, 80, 96, 128, 160};

// Stages of the kTileStream ring: planes z-1, z, z+1 in use, the rest in
// flight.
constexpr int kStreamStages = 5;

// Device-resident counters (graph replays read them instead of baking
// values into kernel arguments).
enum Counter : int {
  kCtrMpass = 0,    // Metropolis passes done
  kCtrSweep = 1,    // sweeps done
  kCtrSwap = 2,     // exchange events done
  kCtrRecords = 3,  // measurement events done over the context's life
  kCtrSeries = 4,   // measurement events waiting in the series buffer
  kNumCounters = 8
};

// One lattice (= one exchange ladder) as the kernels see it.
struct Lattice {
  float* spins;   // slot r, colour c: cos at spins + 2rN + cN, sin N/2 further
  int L;
  int R;
  int slot0;      // global index of local slot 0
  int ty, tz;     // tile: ty rows x tz planes, full rows in x
  int nyt, nzt;   // tiles per slot along y and z
  int kind;       // kTileMarch or kTileBlock
  int part0;      // first tile partial of this lattice; slot r tile t at
                  // part0 + r*nyt*nzt + t, t = yt + nyt*zt
};

struct PassParams {
  PhiloxRoundKeys rk;           // round keys of the seed
  const uint64_t* ctr;          // device counters (may be null: mpass_off absolute)
  uint64_t mpass_off;           // pass counter = ctr[kCtrMpass] + mpass_off
  const float* beta_slot;       // FP32 beta of every global slot
  double* partials;             // [tiles][kNumSums], written when measuring
  unsigned long long* acc_met;  // accepted proposals per global slot
  int measure;                  // fuse the lattice sums (white passes only):
                                // 1 all of them, 2 the energy alone (an
                                // exchange that records nothing)
  int poison;                   // test hook (kTileStream): plane 2 is never copied
  int own_ready;                // kTileDirect launches chained by the library: the
                                // own colour and the pass counter are final before
                                // griddepcontrol.wait (see tile_direct)
  int* status;                  // set to XY_ERR_TIMEOUT when a bounded wait runs out
  long long wait_ns;            // bound of one wait for a copied plane
  // Metropolis words drawn ahead (kTileDirect, per-launch path): the words
  // of one Metropolis pass of the launch's lattice, one Philox4x32-10 output
  // per call, at (slot * 2 + colour) * N/4 + call; null: none.
  uint4* words;
  int words_read;               // Metropolis: read the pass's words instead of drawing them
  uint32_t gen_begin, gen_end;  // over-relaxation: draw the calls [begin, end) of the words
  uint64_t gen_mpass;           // the pass counter of the words drawn = ctr[kCtrMpass] + gen_mpass
};

// Shared-memory bytes of one tile pass: three plane buffers of ty+2 rows of
// L/2 (cos, sin) pairs, then the reduction area.
__host__ __device__ inline int tile_plane_floats(int L, int ty) { return 3 * (ty + 2) * L; }
__host__ __device__ inline int tile_smem_bytes(int L, int ty) {
  return tile_plane_floats(L, ty) * 4 + kReduceBytes;
}
// kTileBlock: (ty+2) x (tz+2) rows of L/2 (cos, sin) pairs.
__host__ __device__ inline int block_tile_floats(int L, int ty, int tz) { return (ty + 2) * (tz + 2) * L; }
// kTileStream: per stage, the cosines of the other colour's ty+2 rows, their
// sines, then the cosines and the sines of the own colour's ty rows (L/2
// floats per row); after the stages, a "full" and an "empty" 8-byte
// mbarrier per stage.
__host__ __device__ inline int stream_stage_floats(int L, int ty) { return (2 * ty + 2) * L; }
__host__ __device__ inline int stream_tile_floats(int L, int ty) {
  return kStreamStages * stream_stage_floats(L, ty) + 4 * kStreamStages;  // + full and empty mbarriers
}
// kTileStream: compute warps covering (L/8) x ty threads, then one producer warp.
__host__ __device__ inline int stream_compute_warps(int L, int ty) { return ((L / 8) * ty + 31) / 32; }
__host__ __device__ inline int tile_threads(int kind, int L, int ty, int tz) {
  return kind == kTileBlock    ? (L / 8) * ty * tz
         : kind == kTileStream ? 32 * (stream_compute_warps(L, ty) + 1)
                               : (L / 8) * ty;
}
// kTileDirect and kTileAngle keep no tile in shared memory (only the
// reduction area).
__host__ __device__ inline int tile_floats(int kind, int L, int ty, int tz) {
  return kind == kTileBlock                            ? block_tile_floats(L, ty, tz)
         : kind == kTileStream                         ? stream_tile_floats(L, ty)
         : kind == kTileDirect                         ? 0
                                                       : tile_plane_floats(L, ty);
}
__host__ __device__ inline int tile_bytes(int kind, int L, int ty, int tz) {
  return tile_floats(kind, L, ty, tz) * 4 + kReduceBytes;
}

// Programmatic dependent launch: a kernel of the half-sweep chain waits for
// its predecessor's results (griddepcontrol.wait returns once the previous
// grid has completed and its memory is visible; it is a no-op for launches
// without the attribute), then lets its own successor be launched early.
__device__ __forceinline__ void chain_wait_and_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void spin(float th, float& c, float& s) {
  float sn, cs;
  __sincosf(th - kPi, &sn, &cs);
  c = -cs;
  s = -sn;
}

// The Metropolis proposal angle theta' = 2 pi u0 of a proposal word: the
// 24-bit integer (w >> 8) times 2 pi / 2^24 in FP32.
__device__ __forceinline__ float proposal_angle(uint32_t w) {
  return static_cast<float>(w >> 8) * kTwoPiOver2p24;
}

// The acceptance threshold of u1 < exp(x) in units of the accept word:
// u1 < exp(x)  <=>  (w >> 8) < exp(x) 2^24 (the scaling by 2^24 is exact),
// with the fast exponential.
__device__ __forceinline__ float accept_threshold(float x) { return __expf(x) * 16777216.0f; }

struct Spins4 {
  float4 c, s;
};

// An angle in [0, 2 pi) from atan2's (-pi, pi]; a value that rounds to 2 pi
// is 0.
__device__ __forceinline__ float wrap_angle(float t) {
  t = t < 0.f ? t + kTwoPi : t;
  return t >= kTwoPi ? 0.f : t;
}

// atan2(y, x) in [-pi, pi] of two pairs (x, y) != (0, 0) at once, without
// a division: the octant reduction r = min(|x|, |y|) / max(|x|, |y|) in
// [0, 1] (the approximate reciprocal and one Newton correction of the
// quotient), the minimax polynomial atan(r) ~ r P(r^2) of atan_poly.cuh,
// then pi/2 - a where |y| > |x|, pi - a where x < 0 (each constant as a
// rounded value plus its FP32 remainder), and the sign of y.  The quotient
// and the polynomial run in the paired FP32 instructions (each lane rounds
// as the scalar ones).  Measured against FP64 atan2: at most 3.0e-7 rad
// (tests/test_gpu_accuracy.py).
__device__ __forceinline__ float2 atan2_poly2(float2 y, float2 x) {
  constexpr float kPio2Hi = 1.57079637e+00f, kPio2Lo = -4.37113883e-08f;
  constexpr float kPiHi = 3.14159274e+00f, kPiLo = -8.74227766e-08f;
  const float2 ax = make_float2(fabsf(x.x), fabsf(x.y)), ay = make_float2(fabsf(y.x), fabsf(y.y));
  const float2 mx = make_float2(fmaxf(ax.x, ay.x), fmaxf(ax.y, ay.y));
  const float2 mn = make_float2(fminf(ax.x, ay.x), fminf(ax.y, ay.y));
  float2 inv;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv.x) : "f"(mx.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv.y) : "f"(mx.y));
  const float2 q = __fmul2_rn(mn, inv);
  const float2 r = __ffma2_rn(__ffma2_rn(make_float2(-q.x, -q.y), mx, mn), inv, q);
  float2 a = __fmul2_rn(r, atan_poly2(__fmul2_rn(r, r)));
  a.x = ay.x > ax.x ? (kPio2Hi - a.x) + kPio2Lo : a.x;
  a.y = ay.y > ax.y ? (kPio2Hi - a.y) + kPio2Lo : a.y;
  a.x = x.x < 0.f ? (kPiHi - a.x) + kPiLo : a.x;
  a.y = x.y < 0.f ? (kPiHi - a.y) + kPiLo : a.y;
  return make_float2(copysignf(a.x, y.x), copysignf(a.y, y.y));
}

// The reflection of Eq. (2) of an angle t in [0, 2 pi) about the field
// (hx, hy) != 0: 2 phi - t with phi = atan2(hy, hx) in [-pi, pi], taken into
// [0, 2 pi) (2 phi - t lies in (-4 pi, 2 pi]; 2 phi is exact, so the fused
// multiply-add rounds once).  Two sites at once.
__device__ __forceinline__ float wrap_two_periods(float u) {
  u = u < 0.f ? u + kTwoPi : u;
  u = u < 0.f ? u + kTwoPi : u;
  return u >= kTwoPi ? 0.f : u;
}
__device__ __forceinline__ float2 reflect_angle2(float2 hx, float2 hy, float2 t) {
  const float2 u = __ffma2_rn(make_float2(2.f, 2.f), atan2_poly2(hy, hx), make_float2(-t.x, -t.y));
  return make_float2(wrap_two_periods(u.x), wrap_two_periods(u.y));
}

// The vectors of four stored angles (kTileAngle), with the fast sincos of
// spin() (the stored angles lie in [0, 2 pi)).
__device__ __forceinline__ Spins4 spins_of_angles(const float4& a) {
  Spins4 v;
  spin(a.x, v.c.x, v.s.x);
  spin(a.y, v.c.y, v.s.y);
  spin(a.z, v.c.z, v.s.z);
  spin(a.w, v.c.w, v.s.w);
  return v;
}

// Bounds of the spin accesses of one tile pass: the slot's 2N floats.  In a
// build with XY_BOUNDS_CHECK defined (the debug library, in place of
// compute-sanitizer) every global spin access is checked against them; one
// outside is skipped (loads read zeros) and the status word is set to
// XY_ERR_BOUNDS, so the host reports it and nothing faults.  Otherwise the
// guard is empty and the checks compile away.
struct SpinGuard {
#ifdef XY_BOUNDS_CHECK
  const float* lo;
  const float* hi;
  int* status;
  __device__ __forceinline__ bool ok(const float* p, int n) const {
    if (p >= lo && p + n <= hi) return true;
    atomicCAS(status, 0, XY_ERR_BOUNDS);
    return false;
  }
#else
  __device__ __forceinline__ bool ok(const float*, int) const { return true; }
#endif
};
__device__ __forceinline__ SpinGuard spin_guard(const float* slot, size_t n_floats, int* status) {
#ifdef XY_BOUNDS_CHECK
  return SpinGuard{slot, slot + n_floats, status};
#else
  (void)slot;
  (void)n_floats;
  (void)status;
  return SpinGuard{};
#endif
}

// Spin loads and stores go through L2 (.cg): the persistent kernel reads
// values other blocks wrote earlier in the same launch.
__device__ __forceinline__ float4 ld4(const float* p) {
  return __ldcg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ void st4(float* p, float4 v) {
  __stcg(reinterpret_cast<float4*>(p), v);
}

// The 4 spins of one thread's row segment: cos at p, sin at p + half.
__device__ __forceinline__ Spins4 ld_spins(const SpinGuard& g, const float* p, uint32_t half) {
  Spins4 v{};
  if (g.ok(p, 4) && g.ok(p + half, 4)) {
    v.c = ld4(p);
    v.s = ld4(p + half);
  }
  return v;
}
__device__ __forceinline__ void st_spins(const SpinGuard& g, float* p, uint32_t half, const float4& c,
                                         const float4& s) {
  if (g.ok(p, 4) && g.ok(p + half, 4)) {
    st4(p, c);
    st4(p + half, s);
  }
}

__device__ __forceinline__ void put_row(float* row, int H, int tx, const Spins4& v) {
  reinterpret_cast<float4*>(row)[tx] = v.c;
  reinterpret_cast<float4*>(row + H)[tx] = v.s;
}

__device__ __forceinline__ float comp(const float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

template <int N>
struct IC {
  static constexpr int value = N;
};

// Per-thread accumulators of the fused lattice sums (present only in the
// measuring variants).
template <bool MEAS>
struct SumAcc {
  __device__ __forceinline__ void add_plane(const float*) {}
  __device__ __forceinline__ void export_to(float*) const {}
};
template <>
struct SumAcc<true> {
  float2 acc[kNumSums / 2];
  float2 err[kNumSums / 2];
  __device__ __forceinline__ SumAcc() {
#pragma unroll
    for (int j = 0; j < kNumSums / 2; ++j) acc[j] = err[j] = make_float2(0.f, 0.f);
  }
  // Compensated (Kahan) accumulation of one plane's terms, so the per-thread
  // FP32 sums stay within a few roundings of the terms whatever the depth;
  // two sums at a time in the paired FP32 instructions (each lane rounds as
  // the scalar instruction would).
  __device__ __forceinline__ void add_plane(const float* step) {
#pragma unroll
    for (int j = 0; j < kNumSums / 2; ++j) {
      const float2 yv = __fadd2_rn(make_float2(step[2 * j], step[2 * j + 1]),
                                   make_float2(-err[j].x, -err[j].y));
      const float2 t = __fadd2_rn(acc[j], yv);
      err[j] = __fadd2_rn(__fadd2_rn(t, make_float2(-acc[j].x, -acc[j].y)), make_float2(-yv.x, -yv.y));
      acc[j] = t;
    }
  }
  __device__ __forceinline__ void export_to(float* out) const {
#pragma unroll
    for (int j = 0; j < kNumSums / 2; ++j) {
      out[2 * j] = acc[j].x;
      out[2 * j + 1] = acc[j].y;
    }
  }
};

__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The reflection of Eq. (2) for two sites at once, in the paired FP32
// instructions of sm_100 and later (each lane rounds exactly as the scalar
// instruction would): S' = 2 (S.h / h.h) h - S, then one Newton step of the
// norm, S' *= 3/2 - |S'|^2 / 2.  h = 0 leaves S (Sec. II reading: no field,
// no reflection); so does a field whose squared length underflows.
__device__ __forceinline__ void reflect2(float2 hx, float2 hy, float2 c, float2 s, float2& c1, float2& s1) {
  const float2 n2 = __ffma2_rn(hy, hy, __fmul2_rn(hx, hx));
  const float2 rn = make_float2(rcp_approx(n2.x), rcp_approx(n2.y));
  const float2 d = __ffma2_rn(s, hy, __fmul2_rn(c, hx));
  const float2 k = __fmul2_rn(__fadd2_rn(d, d), rn);
  const float2 a = __ffma2_rn(k, hx, neg2(c)), b = __ffma2_rn(k, hy, neg2(s));
  const float2 f = __ffma2_rn(make_float2(-0.5f, -0.5f), __ffma2_rn(b, b, __fmul2_rn(a, a)), make_float2(1.5f, 1.5f));
  const float2 ca = __fmul2_rn(a, f), sb = __fmul2_rn(b, f);
  c1 = make_float2(n2.x > 0.f ? ca.x : c.x, n2.y > 0.f ? ca.y : c.y);
  s1 = make_float2(n2.x > 0.f ? sb.x : s.x, n2.y > 0.f ? sb.y : s.y);
}

// The update of one thread's 4 same-colour sites (one float4 per component
// of a row, packed k = 4t .. 4t+3), shared by every tile kind so that all of
// them produce bit-identical spins.  z: the other colour's float4 of the same
// row (cos, sin), h: its x-halo element, s: the row's parity (x = 2k + s), so
// the -x and +x neighbours of site e are X[e] and X[e+1] with X = (z0, z1,
// z2, z3, h) if s = 1 and (h, z0, z1, z2, z3) if s = 0; ym, yp, zm, zp: the
// other colour's float4s of rows y-1, y+1 and planes z-1, z+1 at the same k;
// o: the own spins.  w0, w1: the Philox words of sites (0, 1) and (2, 3)
// (Metropolis).  Returns the new spins; accumulates the accepted proposals
// and, when measuring, this plane's lattice-sum terms (stepv).  ANG (angle
// storage): *oa holds the own angles, and *na receives the new angles: the
// proposal's where accepted, 2 phi - theta (reflect_angle2) where reflected,
// the old angle elsewhere (also where the field is zero); the new spins n
// are then the vectors of those angles when measuring (o is not read by
// the over-relaxation update).  e_only (measuring): the energy's term alone.
template <int MODE, bool MEAS, bool ANG = false>
__device__ __forceinline__ void update4(const Spins4& z, float hc, float hs, int s, const Spins4& ym,
                                        const Spins4& yp, const Spins4& zm, const Spins4& zp, const Spins4& o,
                                        const uint4& w0, const uint4& w1, float beta, Spins4& n, uint32_t& n_acc,
                                        float* stepv, const float4* oa = nullptr, float4* na = nullptr,
                                        bool e_only = false) {
  float2 nang[2];
  float Xc[5], Xs[5];
#pragma unroll
  for (int e = 0; e < 5; ++e) {
    const float a_c = (e < 4) ? comp(z.c, e < 4 ? e : 0) : hc, a_s = (e < 4) ? comp(z.s, e < 4 ? e : 0) : hs;
    const float b_c = (e == 0) ? hc : comp(z.c, e == 0 ? 0 : e - 1);
    const float b_s = (e == 0) ? hs : comp(z.s, e == 0 ? 0 : e - 1);
    Xc[e] = s ? a_c : b_c;
    Xs[e] = s ? a_s : b_s;
  }
  // field h = (x- + x+) + (y- + y+) + (z- + z+), sites in pairs
  float2 hx[2], hy[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float2 xx = make_float2(Xc[2 * q] + Xc[2 * q + 1], Xc[2 * q + 1] + Xc[2 * q + 2]);
    const float2 xy = make_float2(Xs[2 * q] + Xs[2 * q + 1], Xs[2 * q + 1] + Xs[2 * q + 2]);
    const float2 yyc = q ? __fadd2_rn(hi2(ym.c), hi2(yp.c)) : __fadd2_rn(lo2(ym.c), lo2(yp.c));
    const float2 yys = q ? __fadd2_rn(hi2(ym.s), hi2(yp.s)) : __fadd2_rn(lo2(ym.s), lo2(yp.s));
    const float2 zzc = q ? __fadd2_rn(hi2(zm.c), hi2(zp.c)) : __fadd2_rn(lo2(zm.c), lo2(zp.c));
    const float2 zzs = q ? __fadd2_rn(hi2(zm.s), hi2(zp.s)) : __fadd2_rn(lo2(zm.s), lo2(zp.s));
    hx[q] = __fadd2_rn(__fadd2_rn(xx, yyc), zzc);
    hy[q] = __fadd2_rn(__fadd2_rn(xy, yys), zzs);
  }
  float2 nc[2], ns[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float2 co = q ? hi2(o.c) : lo2(o.c), so = q ? hi2(o.s) : lo2(o.s);
    if (MODE == kMetropolis) {
      const uint4& w = q ? w1 : w0;
      // proposal theta' = 2 pi u0 (words 0 and 2), acceptance u1 (words 1 and 3)
      const float2 tp = make_float2(proposal_angle(w.x), proposal_angle(w.z));
      float2 cp, sp;
      spin(tp.x, cp.x, sp.x);
      spin(tp.y, cp.y, sp.y);
      // -beta dE with dE = -[h_x (cos t' - cos t) + h_y (sin t' - sin t)]
      const float2 x = __fmul2_rn(make_float2(beta, beta),
                                  __ffma2_rn(hx[q], __fadd2_rn(cp, neg2(co)), __fmul2_rn(hy[q], __fadd2_rn(sp, neg2(so)))));
      const bool a0 = static_cast<float>(w.y >> 8) < accept_threshold(x.x);
      const bool a1 = static_cast<float>(w.w >> 8) < accept_threshold(x.y);
      n_acc += (a0 ? 1u : 0u) + (a1 ? 1u : 0u);
      nc[q] = make_float2(a0 ? cp.x : co.x, a1 ? cp.y : co.y);
      ns[q] = make_float2(a0 ? sp.x : so.x, a1 ? sp.y : so.y);
      if (ANG) {
        const float2 ta = q ? make_float2(oa->z, oa->w) : make_float2(oa->x, oa->y);
        nang[q] = make_float2(a0 ? tp.x : ta.x, a1 ? tp.y : ta.y);
      }
    } else if (MODE == kOverrelax) {
      if (ANG) {
        // Eq. (2) on the stored angle itself: theta' = 2 phi - theta with
        // phi the field's angle (no vector of the own site is needed)
        const float2 ta = q ? make_float2(oa->z, oa->w) : make_float2(oa->x, oa->y);
        const float2 n2 = __ffma2_rn(hy[q], hy[q], __fmul2_rn(hx[q], hx[q]));
        const float2 rf = reflect_angle2(hx[q], hy[q], ta);
        nang[q] = make_float2(n2.x > 0.f ? rf.x : ta.x, n2.y > 0.f ? rf.y : ta.y);
        nc[q] = co;  // unused: the measuring variant forms the vectors of the new angles
        ns[q] = so;
      } else {
        reflect2(hx[q], hy[q], co, so, nc[q], ns[q]);
      }
    } else {
      nc[q] = co;
      ns[q] = so;
      if (ANG) nang[q] = q ? make_float2(oa->z, oa->w) : make_float2(oa->x, oa->y);
    }
  }
  n.c = make_float4(nc[0].x, nc[0].y, nc[1].x, nc[1].y);
  n.s = make_float4(ns[0].x, ns[0].y, ns[1].x, ns[1].y);
  if (ANG) {
    *na = make_float4(nang[0].x, nang[0].y, nang[1].x, nang[1].y);
    // the sums measure the stored state: the vectors of the stored angles,
    // as a later measure-only pass forms them
    if (MEAS) n = spins_of_angles(*na);
  }
  if (MEAS && e_only) {
    // The energy alone (Eq. 1; an exchange that records nothing): the same
    // bonds as C_x + C_y + C_z below, grouped by white site, w . h with h the
    // sum of its six neighbours (the field of the update), in slot 2 (the
    // other slots stay 0; the finishing step takes E = -(slots 2 + 3 + 4)).
    const float2 t = __ffma2_rn(hi2(n.c), hx[1], __ffma2_rn(hi2(n.s), hy[1], __ffma2_rn(lo2(n.c), hx[0],
                                __fmul2_rn(lo2(n.s), hy[0]))));
    stepv[2] += t.x + t.y;
  } else if (MEAS) {
    // Bonds (w, w+mu) and (w-mu, w) of the white site w: every bond has
    // exactly one white end, so each is counted once.  C_mu: cos of the
    // bond's angle difference, w . (w+mu + w-mu); S_mu: sin,
    // w x (w+mu - w-mu); M: the white site and the black site of this
    // column.  Sites in pairs, the two pairs added lane-wise, then the
    // lanes.
    float2 t[kNumSums];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float2 c2 = q ? hi2(n.c) : lo2(n.c), s2 = q ? hi2(n.s) : lo2(n.s);
      float2 v[kNumSums];
      v[0] = __fadd2_rn(c2, q ? hi2(z.c) : lo2(z.c));
      v[1] = __fadd2_rn(s2, q ? hi2(z.s) : lo2(z.s));
      // +mu and -mu neighbours of the pair's two sites along x, y, z
      const float2 pc[3] = {make_float2(Xc[2 * q + 1], Xc[2 * q + 2]), q ? hi2(yp.c) : lo2(yp.c),
                            q ? hi2(zp.c) : lo2(zp.c)};
      const float2 mc[3] = {make_float2(Xc[2 * q], Xc[2 * q + 1]), q ? hi2(ym.c) : lo2(ym.c),
                            q ? hi2(zm.c) : lo2(zm.c)};
      const float2 ps[3] = {make_float2(Xs[2 * q + 1], Xs[2 * q + 2]), q ? hi2(yp.s) : lo2(yp.s),
                            q ? hi2(zp.s) : lo2(zp.s)};
      const float2 ms[3] = {make_float2(Xs[2 * q], Xs[2 * q + 1]), q ? hi2(ym.s) : lo2(ym.s),
                            q ? hi2(zm.s) : lo2(zm.s)};
#pragma unroll
      for (int mu = 0; mu < 3; ++mu) {
        v[2 + mu] = __ffma2_rn(c2, __fadd2_rn(pc[mu], mc[mu]), __fmul2_rn(s2, __fadd2_rn(ps[mu], ms[mu])));
        v[5 + mu] = __ffma2_rn(s2, __fadd2_rn(pc[mu], neg2(mc[mu])),
                               __fmul2_rn(neg2(c2), __fadd2_rn(ps[mu], neg2(ms[mu]))));
      }
#pragma unroll
      for (int j = 0; j < kNumSums; ++j) t[j] = q ? __fadd2_rn(t[j], v[j]) : v[j];
    }
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) stepv[j] += t[j].x + t[j].y;
  }
}

// One tile of one half-sweep of colour `colour` on local slot r.
// (tx, ty): thread coordinates, tx in [0, L/8); in_block = the thread maps
// onto the tile at all (the persistent kernel's flat blocks have spares).
// Every thread of the block must call this (it contains barriers).
// acc_out[] receives this thread's FP32 lattice-sum partials (MEAS);
// n_acc its accepted Metropolis proposals; pass_add is added to the
// Metropolis pass counter (a persistent launch's later passes).
template <int MODE, bool MEAS>
__device__ __forceinline__ void tile_pass(const Lattice& lat, int r, int yt, int zt, int colour,
                                          int tx, int ty, bool in_block, const PassParams& pp,
                                          float* sm, float* acc_out, uint32_t& n_acc, uint32_t pass_add = 0) {
  static_assert(MODE != kMeasureOnly || MEAS, "measure-only pass measures");
  const int L = lat.L;
  const int H = L >> 1;
  const uint32_t PS = static_cast<uint32_t>(H) * static_cast<uint32_t>(L);  // plane stride
  const uint32_t half = PS * static_cast<uint32_t>(L);                       // N / 2
  const int y0 = yt * lat.ty, z0 = zt * lat.tz;
  const int TYa = min(lat.ty, L - y0), TZa = min(lat.tz, L - z0);
  const bool act = in_block && ty < TYa;
  const int y = y0 + ty;
  float* const slot = lat.spins + static_cast<size_t>(r) * (4 * static_cast<size_t>(half));
  const SpinGuard sg = spin_guard(slot, 4 * static_cast<size_t>(half), pp.status);
  float* const own = slot + colour * (2 * half);            // cos; sin at + half
  const float* const oth = slot + (colour ^ 1) * (2 * half);
  const int rows = lat.ty + 2;
  const int ym = (y0 == 0 ? L : y0) - 1;          // halo row y0 - 1 (periodic)
  const int yp = (y0 + TYa == L) ? 0 : y0 + TYa;  // halo row y0 + TYa
  const bool top = act && ty == 0;
  const bool bot = act && ty == TYa - 1;
  const uint32_t offy = static_cast<uint32_t>(H * y + 4 * tx);
  const uint32_t offym = static_cast<uint32_t>(H * ym + 4 * tx);
  const uint32_t offyp = static_cast<uint32_t>(H * yp + 4 * tx);
  auto row_ptr = [&](int b, int rr) -> float* { return sm + (b * rows + rr) * 2 * H; };
  // x-halo element of this thread's row: k = 4 tx - 1 (s = 0) or 4 tx + 4 (s = 1)
  const int kh0 = (tx == 0) ? H - 1 : 4 * tx - 1;
  const int kh1 = (4 * tx + 4 == H) ? 0 : 4 * tx + 4;

  float beta = 0.f;
  uint32_t tagw = 0u, mlo = 0u, mhi = 0u;
  if (MODE == kMetropolis) {
    beta = __ldcg(pp.beta_slot + lat.slot0 + r);
    tagw = (static_cast<uint32_t>(lat.slot0 + r) << 4) | (static_cast<uint32_t>(colour) << 3) |
           kTagMet;
    const uint64_t mp = (pp.ctr ? pp.ctr[kCtrMpass] : 0ull) + pp.mpass_off + pass_add;
    mlo = static_cast<uint32_t>(mp);
    mhi = static_cast<uint32_t>(mp >> 32);
  }
  SumAcc<MEAS> sums;

  Spins4 pa{}, pb{}, pc{};  // rotating register planes (other colour, own column)
  Spins4 nx_oth{}, nx_own{}, nx_h0{}, nx_h1{};
  if (act) {
    const uint32_t zb = static_cast<uint32_t>((z0 == 0 ? L : z0) - 1) * PS;
    const uint32_t zz = static_cast<uint32_t>(z0) * PS;
    const uint32_t z1 = static_cast<uint32_t>((z0 + 1 == L) ? 0 : z0 + 1) * PS;
    pa = ld_spins(sg, oth + offy + zb, half);
    pb = ld_spins(sg, oth + offy + zz, half);
    put_row(row_ptr(0, ty + 1), H, tx, pb);
    if (top) put_row(row_ptr(0, 0), H, tx, ld_spins(sg, oth + offym + zz, half));
    if (bot) put_row(row_ptr(0, TYa + 1), H, tx, ld_spins(sg, oth + offyp + zz, half));
    nx_oth = ld_spins(sg, oth + offy + z1, half);
    nx_own = ld_spins(sg, own + offy + zz, half);
    if (TZa > 1) {
      if (top) nx_h0 = ld_spins(sg, oth + offym + z1, half);
      if (bot) nx_h1 = ld_spins(sg, oth + offyp + z1, half);
    }
  }
  __syncthreads();

  // One plane: zm, zc = planes z-1, z (registers); zn receives plane z+1.
  auto step = [&](auto bc, Spins4& zm, Spins4& zc, Spins4& zn, int i) {
    constexpr int b0 = decltype(bc)::value;
    constexpr int b1 = b0 == 2 ? 0 : b0 + 1;
    const int z = z0 + i;
    if (act) {
      const Spins4 t_own = nx_own;
      zn = nx_oth;
      if (i + 1 < TZa) {
        put_row(row_ptr(b1, ty + 1), H, tx, zn);
        if (top) put_row(row_ptr(b1, 0), H, tx, nx_h0);
        if (bot) put_row(row_ptr(b1, TYa + 1), H, tx, nx_h1);
        // prefetch the next plane's operands
        const uint32_t pz1 = static_cast<uint32_t>(z + 1) * PS;
        const uint32_t pz2 = static_cast<uint32_t>(z + 2 >= L ? z + 2 - L : z + 2) * PS;
        nx_oth = ld_spins(sg, oth + offy + pz2, half);
        nx_own = ld_spins(sg, own + offy + pz1, half);
        if (i + 2 < TZa) {
          if (top) nx_h0 = ld_spins(sg, oth + offym + pz2, half);
          if (bot) nx_h1 = ld_spins(sg, oth + offyp + pz2, half);
        }
      }
      const float* rm = row_ptr(b0, ty);
      const float* rp = row_ptr(b0, ty + 2);
      const float* r0 = row_ptr(b0, ty + 1);
      Spins4 ysm, ysp;
      ysm.c = reinterpret_cast<const float4*>(rm)[tx];
      ysm.s = reinterpret_cast<const float4*>(rm + H)[tx];
      ysp.c = reinterpret_cast<const float4*>(rp)[tx];
      ysp.s = reinterpret_cast<const float4*>(rp + H)[tx];
      const int s = (y + z + colour) & 1;
      const int kh = s ? kh1 : kh0;
      const float hc = r0[kh], hs = r0[H + kh];
      const uint32_t offz = offy + static_cast<uint32_t>(z) * PS;
      uint4 w0 = make_uint4(0u, 0u, 0u, 0u), w1 = w0;
      if (MODE == kMetropolis) {
        const uint32_t q0 = offz >> 1;
        w0 = philox4x32_10(make_uint4(q0, mlo, mhi, tagw), pp.rk);
        w1 = philox4x32_10(make_uint4(q0 + 1u, mlo, mhi, tagw), pp.rk);
      }
      float stepv[kNumSums];
#pragma unroll
      for (int j = 0; j < kNumSums; ++j) stepv[j] = 0.f;
      Spins4 nw;
      update4<MODE, MEAS>(zc, hc, hs, s, ysm, ysp, zm, zn, t_own, w0, w1, beta, nw, n_acc, stepv, nullptr, nullptr,
                          pp.measure == 2);
      if (MEAS) sums.add_plane(stepv);
      if (MODE != kMeasureOnly) st_spins(sg, own + offz, half, nw.c, nw.s);
    }
    __syncthreads();
  };

  for (int i = 0; i < TZa; i += 3) {
    step(IC<0>{}, pa, pb, pc, i);
    if (i + 1 >= TZa) break;
    step(IC<1>{}, pb, pc, pa, i + 1);
    if (i + 2 >= TZa) break;
    step(IC<2>{}, pc, pa, pb, i + 2);
  }
  if (MEAS) sums.export_to(acc_out);
}

// The 4 spins of one thread's row segment through L1 (other-colour reads of
// kTileDirect).  The other colour is not written during a half-sweep
// launch, and a launch starts reading only after its predecessor has
// completed and its writes are visible (griddepcontrol.wait), so no cached
// line is stale.
__device__ __forceinline__ Spins4 ld_spins_l1(const SpinGuard& g, const float* p, uint32_t half) {
  Spins4 v{};
  if (g.ok(p, 4) && g.ok(p + half, 4)) {
    v.c = __ldca(reinterpret_cast<const float4*>(p));
    v.s = __ldca(reinterpret_cast<const float4*>(p + half));
  }
  return v;
}
__device__ __forceinline__ float ld1_l1(const SpinGuard& g, const float* p) {
  return g.ok(p, 1) ? __ldca(p) : 0.f;
}

// One tile of one half-sweep, kTileDirect: the thread layout and the plane
// march of tile_pass (planes of the thread's column rotate through
// registers), but the y-neighbour rows (y-1, y+1) and the x-halo element of
// plane z are loaded by the thread itself, through L1, while it updates
// plane z-1, and nothing is shared through shared memory: no block barrier,
// every warp marches at its own pace.  Threads with ty >= the tile's rows
// return at once.  acc_out / n_acc as tile_pass.  LC > 0: the lattice size
// fixed at compile time (it must equal lat.L), so that plane strides and the
// cos-to-sin offset are constants folded into the addressing.
// EO (measuring): 1 the energy alone, 0 every sum, -1 as pp.measure says.
template <int MODE, bool MEAS, int LC = 0, bool WORDS = false, int EO = -1>
__device__ __forceinline__ void tile_direct(const Lattice& lat, int r, int yt, int zt, int colour, int tx,
                                            int ty, const PassParams& pp, float* acc_out, uint32_t& n_acc, uint32_t pass_add = 0) {
  static_assert(MODE != kMeasureOnly || MEAS, "measure-only pass measures");
  static_assert(LC % 8 == 0, "L % 8 == 0");
  const int L = LC ? LC : lat.L;
  const int H = L >> 1;
  const uint32_t PS = static_cast<uint32_t>(H) * static_cast<uint32_t>(L);  // plane stride
  const uint32_t half = PS * static_cast<uint32_t>(L);                       // N / 2
  const int y0 = yt * lat.ty, z0 = zt * lat.tz;
  const int TYa = min(lat.ty, L - y0), TZa = min(lat.tz, L - z0);
  if (ty >= TYa) return;
  const int y = y0 + ty;
  float* const slot = lat.spins + static_cast<size_t>(r) * (4 * static_cast<size_t>(half));
  const SpinGuard sg = spin_guard(slot, 4 * static_cast<size_t>(half), pp.status);
  float* const own = slot + colour * (2 * half);  // cos; sin at + half
  const float* const oth = slot + (colour ^ 1) * (2 * half);
  const int ym = (y == 0 ? L : y) - 1;  // periodic y neighbours of this row
  const int yp = (y + 1 == L) ? 0 : y + 1;
  const uint32_t offy = static_cast<uint32_t>(H * y + 4 * tx);
  const uint32_t offym = static_cast<uint32_t>(H * ym + 4 * tx);
  const uint32_t offyp = static_cast<uint32_t>(H * yp + 4 * tx);
  // x-halo element of this thread's row: k = 4 tx - 1 (s = 0) or 4 tx + 4 (s = 1)
  const uint32_t offh0 = static_cast<uint32_t>(H * y + ((tx == 0) ? H - 1 : 4 * tx - 1));
  const uint32_t offh1 = static_cast<uint32_t>(H * y + ((4 * tx + 4 == H) ? 0 : 4 * tx + 4));

  uint32_t tagw = 0u, mlo = 0u, mhi = 0u;
  if (MODE == kMetropolis) {
    tagw = (static_cast<uint32_t>(lat.slot0 + r) << 4) | (static_cast<uint32_t>(colour) << 3) |
           kTagMet;
    const uint64_t mp = (pp.ctr ? pp.ctr[kCtrMpass] : 0ull) + pp.mpass_off + pass_add;
    mlo = static_cast<uint32_t>(mp);
    mhi = static_cast<uint32_t>(mp >> 32);
  }
  SumAcc<MEAS> sums;

  // Registers: four other-colour planes of the column rotate (z-1, z, z+1 in
  // use, z+2 being loaded), and two sets of the other operands alternate
  // (this plane's, the next plane's, loaded one plane ahead); the plane loop
  // is unrolled four times so that every load lands in a free register and
  // nothing is copied.  The Metropolis words of a plane are drawn with its
  // operands, one plane ahead, so that the Philox integer work of the next
  // plane overlaps this plane's update (8.7 instead of 9.1 us at 160^3).
  struct Operands {
    Spins4 own, ym, yp;  // own spins; other colour's rows y-1, y+1
    float hc, hs;        // x-halo element
    uint4 w0, w1;        // Metropolis words of sites (0, 1) and (2, 3)
  };
  Spins4 P0, P1, P2, P3{};
  Operands A, B;
  // The own colour's spins and the Metropolis words of one plane.
  const uint4* const wrow =
      WORDS ? pp.words + static_cast<size_t>(2 * r + colour) * static_cast<size_t>(half >> 1) : nullptr;
  auto load_own = [&](Operands& o, uint32_t pz) {
    o.own = ld_spins(sg, own + offy + pz, half);
    if (MODE == kMetropolis && WORDS) {
      // the pass's words, drawn ahead by the preceding over-relaxation
      // launches (the same Philox outputs)
      const uint32_t q0 = (offy + pz) >> 1;
      o.w0 = __ldcg(wrow + q0);
      o.w1 = __ldcg(wrow + q0 + 1u);
    } else if (MODE == kMetropolis) {
      const uint32_t q0 = (offy + pz) >> 1;
      o.w0 = philox4x32_10(make_uint4(q0, mlo, mhi, tagw), pp.rk);
      o.w1 = philox4x32_10(make_uint4(q0 + 1u, mlo, mhi, tagw), pp.rk);
    } else {
      o.w0 = o.w1 = make_uint4(0u, 0u, 0u, 0u);
    }
  };
  // The other colour's operands of one plane (rows y -+ 1, x halo).
  auto load_other = [&](Operands& o, int z, uint32_t pz) {
    o.ym = ld_spins_l1(sg, oth + offym + pz, half);
    o.yp = ld_spins_l1(sg, oth + offyp + pz, half);
    const uint32_t oh = (((y + z + colour) & 1) ? offh1 : offh0) + pz;
    o.hc = ld1_l1(sg, oth + oh);
    o.hs = ld1_l1(sg, oth + oh + half);
  };
  auto load_operands = [&](Operands& o, int z, uint32_t pz) {
    load_own(o, pz);
    load_other(o, z, pz);
  };
  float beta = 0.f;
  {
    const uint32_t zz = static_cast<uint32_t>(z0) * PS;
    // A launch chained by the library behind the other colour's half-sweep
    // (pp.own_ready) reads its own colour and draws its first plane's words
    // before griddepcontrol.wait: its predecessor writes only the other
    // colour, and the own colour's last writer, the launch before that, has
    // completed once the predecessor passed its own wait, which it did
    // before releasing this launch (so have the launches that drew words
    // read here: never the predecessor).  Everything the predecessor may
    // write (the other colour, the coupling after an exchange) is read
    // after it.
    if (pp.own_ready) {
      load_own(A, zz);
      chain_wait_and_release();
    }
    if (MODE == kMetropolis) beta = __ldcg(pp.beta_slot + lat.slot0 + r);
    P3 = ld_spins_l1(sg, oth + offy + static_cast<uint32_t>((z0 == 0 ? L : z0) - 1) * PS, half);
    P0 = ld_spins_l1(sg, oth + offy + zz, half);
    P1 = ld_spins_l1(sg, oth + offy + static_cast<uint32_t>((z0 + 1 == L) ? 0 : z0 + 1) * PS, half);
    if (pp.own_ready)
      load_other(A, z0, zz);
    else
      load_operands(A, z0, zz);
  }

  // One plane: zm, zc, zn = planes z-1, z, z+1; zf receives plane z+2; cur
  // holds this plane's operands, nxt receives the next plane's.
  auto step = [&](Spins4& zm, Spins4& zc, Spins4& zn, Spins4& zf, Operands& cur, Operands& nxt, int i) {
    const int z = z0 + i;
    if (i + 1 < TZa) {
      zf = ld_spins_l1(sg, oth + offy + static_cast<uint32_t>(z + 2 >= L ? z + 2 - L : z + 2) * PS, half);
      load_operands(nxt, z + 1, static_cast<uint32_t>(z + 1) * PS);
    }
    const int s = (y + z + colour) & 1;
    const uint32_t offz = offy + static_cast<uint32_t>(z) * PS;
    float stepv[kNumSums];
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) stepv[j] = 0.f;
    Spins4 nw;
    update4<MODE, MEAS>(zc, cur.hc, cur.hs, s, cur.ym, cur.yp, zm, zn, cur.own, cur.w0, cur.w1, beta, nw, n_acc,
                        stepv, nullptr, nullptr, EO > 0 || (EO < 0 && pp.measure == 2));
    if (MEAS) sums.add_plane(stepv);
    if (MODE != kMeasureOnly) st_spins(sg, own + offz, half, nw.c, nw.s);
  };

  for (int i = 0; i < TZa; i += 4) {
    step(P3, P0, P1, P2, A, B, i);
    if (i + 1 >= TZa) break;
    step(P0, P1, P2, P3, B, A, i + 1);
    if (i + 2 >= TZa) break;
    step(P1, P2, P3, P0, A, B, i + 2);
    if (i + 3 >= TZa) break;
    step(P2, P3, P0, P1, B, A, i + 3);
  }
  if (MEAS) sums.export_to(acc_out);
}

// Four stored angles (kTileAngle): through L2 (own colour) or L1 (other
// colour, as the direct tile's vectors).
__device__ __forceinline__ float4 ld_ang(const SpinGuard& g, const float* p) {
  return g.ok(p, 4) ? ld4(p) : make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ float4 ld_ang_l1(const SpinGuard& g, const float* p) {
  return g.ok(p, 4) ? __ldca(reinterpret_cast<const float4*>(p)) : make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void st_ang(const SpinGuard& g, float* p, const float4& v) {
  if (g.ok(p, 4)) st4(p, v);
}

// One tile of one half-sweep, kTileAngle: a lattice stored as angles, each
// colour's N/2 FP32 angles at the places of its cosines (the sine places are
// unused), so a half-sweep moves 12 bytes per update instead of 24.  The
// march's thread layout and plane march (tile_pass): every thread loads its
// row of the other colour's next plane as angles and turns them into
// vectors (the fast sincos) once; the row goes to a shared-memory plane
// buffer, where the threads of rows y-1 and y+1 read it, and stays in the
// thread's registers for its three uses as planes z+1, z and z-1 (the
// tile's edge rows and planes are turned by the threads next to them).  So
// each other-colour angle of the tile becomes a vector once, not once per
// reader.  The update (update4: the field and the Metropolis test are the
// same arithmetic as every tile kind's on those vectors) stores the new
// angle: the proposal's where a Metropolis move is accepted, the reflection
// of Eq. (2) taken on the angle itself (2 phi - theta, phi the field's angle
// by atan2) where the field is non-zero, the old angle otherwise.  The spins
// therefore differ from the vector kinds' by the fast sincos of the
// neighbours (a few 1e-7 per vector) and by the reflection's arithmetic, and
// do not depend on the tile.
// Arguments as tile_pass; every thread of the block must call it (it
// contains barriers).  Library-chained launches (pp.own_ready) load the own
// colour's first plane before griddepcontrol.wait, as tile_direct does.
// EO (measuring): 1 the energy alone, 0 every sum, -1 as pp.measure says.
template <int MODE, bool MEAS, int EO = -1>
__device__ __forceinline__ void tile_angle(const Lattice& lat, int r, int yt, int zt, int colour, int tx, int ty,
                                           bool in_block, const PassParams& pp, float* sm, float* acc_out,
                                           uint32_t& n_acc, uint32_t pass_add = 0) {
  static_assert(MODE != kMeasureOnly || MEAS, "measure-only pass measures");
  const int L = lat.L;
  const int H = L >> 1;
  const uint32_t PS = static_cast<uint32_t>(H) * static_cast<uint32_t>(L);  // plane stride
  const uint32_t half = PS * static_cast<uint32_t>(L);                       // N / 2
  const int y0 = yt * lat.ty, z0 = zt * lat.tz;
  const int TYa = min(lat.ty, L - y0), TZa = min(lat.tz, L - z0);
  const bool act = in_block && ty < TYa;
  const int y = y0 + ty;
  float* const slot = lat.spins + static_cast<size_t>(r) * (4 * static_cast<size_t>(half));
  const SpinGuard sg = spin_guard(slot, 4 * static_cast<size_t>(half), pp.status);
  float* const own = slot + colour * (2 * half);  // angles where the cosines of the vector layout are
  const float* const oth = slot + (colour ^ 1) * (2 * half);
  const int rows = lat.ty + 2;
  const int ym = (y0 == 0 ? L : y0) - 1;          // halo row y0 - 1 (periodic)
  const int yp = (y0 + TYa == L) ? 0 : y0 + TYa;  // halo row y0 + TYa
  const bool top = act && ty == 0;
  const bool bot = act && ty == TYa - 1;
  const uint32_t offy = static_cast<uint32_t>(H * y + 4 * tx);
  const uint32_t offym = static_cast<uint32_t>(H * ym + 4 * tx);
  const uint32_t offyp = static_cast<uint32_t>(H * yp + 4 * tx);
  auto row_ptr = [&](int b, int rr) -> float* { return sm + (b * rows + rr) * 2 * H; };
  const int kh0 = (tx == 0) ? H - 1 : 4 * tx - 1;
  const int kh1 = (4 * tx + 4 == H) ? 0 : 4 * tx + 4;

  float beta = 0.f;
  uint32_t tagw = 0u, mlo = 0u, mhi = 0u;
  if (MODE == kMetropolis) {
    tagw = (static_cast<uint32_t>(lat.slot0 + r) << 4) | (static_cast<uint32_t>(colour) << 3) | kTagMet;
  }
  SumAcc<MEAS> sums;

  Spins4 pa{}, pb{}, pc{};  // rotating register planes: vectors of the other colour's column rows
  float4 nx_oth{}, nx_own{}, nx_h0{}, nx_h1{};  // the next plane's angles
  const uint32_t zz = static_cast<uint32_t>(z0) * PS;
  if (act) nx_own = ld_ang(sg, own + offy + zz);
  if (pp.own_ready) chain_wait_and_release();
  if (MODE == kMetropolis) {
    beta = __ldcg(pp.beta_slot + lat.slot0 + r);
    const uint64_t mp = (pp.ctr ? pp.ctr[kCtrMpass] : 0ull) + pp.mpass_off + pass_add;
    mlo = static_cast<uint32_t>(mp);
    mhi = static_cast<uint32_t>(mp >> 32);
  }
  if (act) {
    const uint32_t zb = static_cast<uint32_t>((z0 == 0 ? L : z0) - 1) * PS;
    const uint32_t z1 = static_cast<uint32_t>((z0 + 1 == L) ? 0 : z0 + 1) * PS;
    pa = spins_of_angles(ld_ang_l1(sg, oth + offy + zb));
    pb = spins_of_angles(ld_ang_l1(sg, oth + offy + zz));
    put_row(row_ptr(0, ty + 1), H, tx, pb);
    if (top) put_row(row_ptr(0, 0), H, tx, spins_of_angles(ld_ang_l1(sg, oth + offym + zz)));
    if (bot) put_row(row_ptr(0, TYa + 1), H, tx, spins_of_angles(ld_ang_l1(sg, oth + offyp + zz)));
    nx_oth = ld_ang_l1(sg, oth + offy + z1);
    if (TZa > 1) {
      if (top) nx_h0 = ld_ang_l1(sg, oth + offym + z1);
      if (bot) nx_h1 = ld_ang_l1(sg, oth + offyp + z1);
    }
  }
  __syncthreads();

  // One plane: zm, zc = the vectors of planes z-1, z (registers); zn
  // receives plane z+1's.
  auto step = [&](auto bc, Spins4& zm, Spins4& zc, Spins4& zn, int i) {
    constexpr int b0 = decltype(bc)::value;
    constexpr int b1 = b0 == 2 ? 0 : b0 + 1;
    const int z = z0 + i;
    if (act) {
      const float4 t_own = nx_own;
      zn = spins_of_angles(nx_oth);
      if (i + 1 < TZa) {
        put_row(row_ptr(b1, ty + 1), H, tx, zn);
        if (top) put_row(row_ptr(b1, 0), H, tx, spins_of_angles(nx_h0));
        if (bot) put_row(row_ptr(b1, TYa + 1), H, tx, spins_of_angles(nx_h1));
        // prefetch the next plane's operands
        const uint32_t pz1 = static_cast<uint32_t>(z + 1) * PS;
        const uint32_t pz2 = static_cast<uint32_t>(z + 2 >= L ? z + 2 - L : z + 2) * PS;
        nx_oth = ld_ang_l1(sg, oth + offy + pz2);
        nx_own = ld_ang(sg, own + offy + pz1);
        if (i + 2 < TZa) {
          if (top) nx_h0 = ld_ang_l1(sg, oth + offym + pz2);
          if (bot) nx_h1 = ld_ang_l1(sg, oth + offyp + pz2);
        }
      }
      const float* rm = row_ptr(b0, ty);
      const float* rp = row_ptr(b0, ty + 2);
      const float* r0 = row_ptr(b0, ty + 1);
      Spins4 ysm, ysp;
      ysm.c = reinterpret_cast<const float4*>(rm)[tx];
      ysm.s = reinterpret_cast<const float4*>(rm + H)[tx];
      ysp.c = reinterpret_cast<const float4*>(rp)[tx];
      ysp.s = reinterpret_cast<const float4*>(rp + H)[tx];
      const int s = (y + z + colour) & 1;
      const int kh = s ? kh1 : kh0;
      const float hc = r0[kh], hs = r0[H + kh];
      const uint32_t offz = offy + static_cast<uint32_t>(z) * PS;
      uint4 w0 = make_uint4(0u, 0u, 0u, 0u), w1 = w0;
      if (MODE == kMetropolis) {
        const uint32_t q0 = offz >> 1;
        w0 = philox4x32_10(make_uint4(q0, mlo, mhi, tagw), pp.rk);
        w1 = philox4x32_10(make_uint4(q0 + 1u, mlo, mhi, tagw), pp.rk);
      }
      float stepv[kNumSums];
#pragma unroll
      for (int j = 0; j < kNumSums; ++j) stepv[j] = 0.f;
      Spins4 nw;
      float4 na;
      update4<MODE, MEAS, true>(zc, hc, hs, s, ysm, ysp, zm, zn, spins_of_angles(t_own), w0, w1, beta, nw, n_acc,
                                stepv, &t_own, &na, EO > 0 || (EO < 0 && pp.measure == 2));
      if (MEAS) sums.add_plane(stepv);
      if (MODE != kMeasureOnly) st_ang(sg, own + offz, na);
    }
    __syncthreads();
  };

  for (int i = 0; i < TZa; i += 3) {
    step(IC<0>{}, pa, pb, pc, i);
    if (i + 1 >= TZa) break;
    step(IC<1>{}, pb, pc, pa, i + 1);
    if (i + 2 >= TZa) break;
    step(IC<2>{}, pc, pa, pb, i + 2);
  }
  if (MEAS) sums.export_to(acc_out);
}

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Arrives once on the barrier and adds `bytes` to the transfer count its
// current phase waits for.
__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for the phase with the given parity to complete, at most `budget_ns`
// of %globaltimer time; false if the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget_ns) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = global_ns();
  while (!mbar_test(bar, parity))
    if (global_ns() - t0 > budget_ns) return false;
  return true;
}

// Bulk asynchronous copy (TMA) of `bytes` (a multiple of 16; both addresses
// 16-byte aligned) from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const float* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// One tile of one half-sweep, kTileStream, warp-specialised: a producer warp
// streams every plane the tile reads into a ring of kStreamStages
// shared-memory stages with bulk asynchronous copies (TMA), and the compute
// warps update the sites with no block-wide barrier.  Stage j mod
// kStreamStages holds plane z0-1+j: the other colour's rows y0-1 .. y0+TYa
// and, for the planes the tile updates, the own colour's rows y0 .. y0+TYa-1
// (cosines of all rows, then sines).  Each stage has a "full" mbarrier (the
// producer arms it with the plane's byte count; the copies complete it) and
// an "empty" one (every compute warp arrives once it no longer reads the
// plane).  Compute thread t < (L/8) ty is (tx, ty) = (t mod L/8, t div
// L/8) of the march; it keeps planes z-1 and z of its column in registers
// and reads plane z+1's row, the y neighbours, its own spins and the x halo
// from the ring.  Plane p is read by the updates of planes p-1 (as z+1) and
// p (current), so it is released after the update of plane p; the producer
// refills its stage with plane p + kStreamStages, which the compute warps
// need kStreamStages - 1 updates later.  Every wait is bounded by
// pp.wait_ns of %globaltimer: when one runs out the block sets *pp.status
// to XY_ERR_TIMEOUT, every warp leaves its loop (their waits are bounded
// too), the producer lets the copies it issued land (bounded again) and
// the tile returns with nothing more written.  Not for the persistent
// kernel, whose other blocks write the planes within one launch.
template <int MODE, bool MEAS>
__device__ __forceinline__ void tile_stream(const Lattice& lat, int r, int yt, int zt, int colour, int tid,
                                            const PassParams& pp, float* sm, float* acc_out, uint32_t& n_acc, uint32_t pass_add = 0) {
  static_assert(MODE != kMeasureOnly || MEAS, "measure-only pass measures");
  constexpr int D = kStreamStages;
  const int L = lat.L;
  const int H = L >> 1, TX = L >> 3;
  const uint32_t PS = static_cast<uint32_t>(H) * static_cast<uint32_t>(L);
  const uint32_t half = PS * static_cast<uint32_t>(L);
  const int y0 = yt * lat.ty, z0 = zt * lat.tz;
  const int TYa = min(lat.ty, L - y0), TZa = min(lat.tz, L - z0);
  const int NC = TX * lat.ty;
  const int nwc = (NC + 31) >> 5;
  const int warp = tid >> 5, lane = tid & 31;
  const int tx = tid % TX, ty = tid / TX;
  const bool act = tid < NC && ty < TYa;
  const int y = y0 + ty;
  float* const slot = lat.spins + static_cast<size_t>(r) * (4 * static_cast<size_t>(half));
  const SpinGuard sg = spin_guard(slot, 4 * static_cast<size_t>(half), pp.status);
  float* const own = slot + colour * (2 * half);
  const float* const oth = slot + (colour ^ 1) * (2 * half);
  const int SF = stream_stage_floats(L, lat.ty);
  const int OS = (lat.ty + 2) * H;           // other sin rows
  const int WC = 2 * (lat.ty + 2) * H;       // own cos rows
  const int WS = WC + lat.ty * H;            // own sin rows
  const uint32_t full0 = smem_addr(sm + D * SF), empty0 = full0 + 8u * D;
  const int n_planes = TZa + 2;              // planes z0-1 .. z0+TZa
  __shared__ int s_abort;

  if (tid == 0) {
    for (int st = 0; st < D; ++st) {
      mbar_init(full0 + 8u * st, 1u);
      mbar_init(empty0 + 8u * st, static_cast<uint32_t>(nwc));
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  if (warp == nwc) {
    // ---------------------------------------------------------- producer
    const int ym = (y0 == 0 ? L : y0) - 1;
    const int yp = (y0 + TYa == L) ? 0 : y0 + TYa;
    const uint32_t row = static_cast<uint32_t>(H) * 4u;
    int n_issued = 0;
    bool ok = true;
    for (int j = 0; j < n_planes && ok; ++j) {
      const int st = j % D;
      if (j >= D) {
        // every compute warp has released plane j - D
        bool got = true;
        if (lane == 0) got = mbar_wait(empty0 + 8u * st, static_cast<uint32_t>((j / D - 1) & 1), pp.wait_ns);
        ok = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
        if (!ok || *reinterpret_cast<volatile int*>(&s_abort)) {
          ok = false;
          break;
        }
      }
      if (!(pp.poison && j == 2)) {
        int zz = z0 - 1 + j;
        zz += zz < 0 ? L : 0;
        zz -= zz >= L ? L : 0;
        const bool has_own = j >= 1 && j <= TZa;
        const uint32_t bar = full0 + 8u * st;
        if (lane == 0) mbar_arrive_expect(bar, 2u * row * static_cast<uint32_t>(TYa + 2 + (has_own ? TYa : 0)));
        __syncwarp();
        if (lane < 8) {
          const uint32_t zoff = static_cast<uint32_t>(zz) * PS;
          const uint32_t dst0 = smem_addr(sm + st * SF);
          // Rows y0-1 .. y0+TYa of one component are contiguous unless the
          // tile touches y = 0 or y = L-1: then one copy per component
          // (lanes 0, 3), else three (top halo row, body rows, bottom halo
          // row: lanes 0-2 cos, 3-5 sin).  Lanes 6 and 7: own cos and sin.
          const bool merged = ym + 1 == y0 && yp == y0 + TYa;
          if (lane < 6) {
            const int cs = lane / 3, part = lane % 3;
            if (!merged || part == 0) {
              const int yrow = part == 0 ? ym : (part == 1 ? y0 : yp);
              const int srow = part == 0 ? 0 : (part == 1 ? 1 : TYa + 1);
              const int nrow = merged ? TYa + 2 : (part == 1 ? TYa : 1);
              const float* src = oth + cs * half + zoff + static_cast<uint32_t>(H) * static_cast<uint32_t>(yrow);
              if (sg.ok(src, H * nrow))
                bulk_copy_g2s(dst0 + 4u * static_cast<uint32_t>(cs * OS + srow * H), src, row * nrow, bar);
            }
          } else if (has_own) {
            const int cs = lane - 6;
            const float* src = own + cs * half + zoff + static_cast<uint32_t>(H) * static_cast<uint32_t>(y0);
            if (sg.ok(src, H * TYa)) bulk_copy_g2s(dst0 + 4u * static_cast<uint32_t>(cs ? WS : WC), src, row * TYa, bar);
          }
        }
      }
      n_issued = j + 1;
    }
    if (!ok) {
      if (lane == 0) {
        atomicCAS(pp.status, 0, XY_ERR_TIMEOUT);
        s_abort = 1;
        // the copies of the last D issued planes may still be landing
        for (int j = max(0, n_issued - D); j < n_issued; ++j)
          if (!(pp.poison && j == 2)) mbar_wait(full0 + 8u * (j % D), static_cast<uint32_t>((j / D) & 1), pp.wait_ns);
      }
      __syncwarp();
    }
  } else {
    // ---------------------------------------------------------- compute
    float beta = 0.f;
    uint32_t tagw = 0u, mlo = 0u, mhi = 0u;
    if (MODE == kMetropolis) {
      beta = __ldcg(pp.beta_slot + lat.slot0 + r);
      tagw = (static_cast<uint32_t>(lat.slot0 + r) << 4) | (static_cast<uint32_t>(colour) << 3) | kTagMet;
      const uint64_t mp = (pp.ctr ? pp.ctr[kCtrMpass] : 0ull) + pp.mpass_off + pass_add;
      mlo = static_cast<uint32_t>(mp);
      mhi = static_cast<uint32_t>(mp >> 32);
    }
    SumAcc<MEAS> sums;
    const uint32_t offy = static_cast<uint32_t>(H * y + 4 * tx);
    const int kh0 = (tx == 0) ? H - 1 : 4 * tx - 1;
    const int kh1 = (4 * tx + 4 == H) ? 0 : 4 * tx + 4;
    // per-thread float offsets inside a stage
    const int o_row = (ty + 1) * H + 4 * tx, o_ym = ty * H + 4 * tx, o_yp = (ty + 2) * H + 4 * tx;
    const int o_own = WC + ty * H + 4 * tx;
    auto ld2 = [&](const float* st, int oc, int os) {
      Spins4 v;
      v.c = *reinterpret_cast<const float4*>(st + oc);
      v.s = *reinterpret_cast<const float4*>(st + os);
      return v;
    };
    // warp-uniform outcome (a lane whose wait ran out takes the warp with it)
    auto wait_plane = [&](int j) -> bool {
      const bool got = mbar_wait(full0 + 8u * (j % D), static_cast<uint32_t>((j / D) & 1), pp.wait_ns);
      return __all_sync(0xffffffffu, got);
    };
    auto release = [&](int j) {
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8u * (j % D));
    };
    bool ok = wait_plane(0) && wait_plane(1);
    Spins4 pa{}, pb{}, pc{};
    if (ok && act) {
      pa = ld2(sm, o_row, OS + o_row);
      pb = ld2(sm + SF, o_row, OS + o_row);
    }
    if (ok) release(0);
    int s1 = 1;  // stage of plane i+1 (the current plane of update i)
    auto step = [&](Spins4& zm, Spins4& zc, Spins4& zn, int i) {
      const int s2 = s1 + 1 == D ? 0 : s1 + 1;
      ok = ok && wait_plane(i + 2);
      if (!ok) return;
      if (act) {
        const int z = z0 + i;
        const float* cur = sm + s1 * SF;
        zn = ld2(sm + s2 * SF, o_row, OS + o_row);
        const Spins4 ysm = ld2(cur, o_ym, OS + o_ym), ysp = ld2(cur, o_yp, OS + o_yp);
        const Spins4 t_own = ld2(cur, o_own, o_own + lat.ty * H);
        const int s = (y + z + colour) & 1;
        const int kh = (ty + 1) * H + (s ? kh1 : kh0);
        const float hc = cur[kh], hs = cur[OS + kh];
        const uint32_t offz = offy + static_cast<uint32_t>(z) * PS;
        uint4 w0 = make_uint4(0u, 0u, 0u, 0u), w1 = w0;
        if (MODE == kMetropolis) {
          const uint32_t q0 = offz >> 1;
          w0 = philox4x32_10(make_uint4(q0, mlo, mhi, tagw), pp.rk);
          w1 = philox4x32_10(make_uint4(q0 + 1u, mlo, mhi, tagw), pp.rk);
        }
        float stepv[kNumSums];
#pragma unroll
        for (int q = 0; q < kNumSums; ++q) stepv[q] = 0.f;
        Spins4 nw;
        update4<MODE, MEAS>(zc, hc, hs, s, ysm, ysp, zm, zn, t_own, w0, w1, beta, nw, n_acc, stepv, nullptr,
                            nullptr, pp.measure == 2);
        if (MEAS) sums.add_plane(stepv);
        if (MODE != kMeasureOnly) st_spins(sg, own + offz, half, nw.c, nw.s);
      }
      release(i + 1);
      s1 = s2;
    };
    for (int i = 0; i < TZa && ok; i += 3) {
      step(pa, pb, pc, i);
      if (i + 1 >= TZa || !ok) break;
      step(pb, pc, pa, i + 1);
      if (i + 2 >= TZa || !ok) break;
      step(pc, pa, pb, i + 2);
    }
    if (!ok) {
      if (lane == 0) atomicCAS(pp.status, 0, XY_ERR_TIMEOUT);
      s_abort = 1;
    }
    if (MEAS) sums.export_to(acc_out);
  }
}

// One tile of one half-sweep, kTileBlock: thread (tx, ty, tz) owns the 4
// sites at row y0+ty of plane z0+tz.  Prologue: every thread stages the
// other-colour spins of its own row in shared memory; threads on the tile's
// faces also stage the face-halo rows (y0-1, y0+TYa at each plane; z0-1,
// z0+TZa at each row).  One barrier, then each thread reads its six
// neighbours from shared memory.  The per-site arithmetic (field in the same
// association order, Metropolis, reflection, lattice sums) is the march
// kind's, so both kinds give bit-identical spins.
template <int MODE, bool MEAS>
__device__ __forceinline__ void tile_block(const Lattice& lat, int r, int yt, int zt, int colour,
                                           int tx, int ty, int tz, bool in_block, const PassParams& pp,
                                           float* sm, float* acc_out, uint32_t& n_acc, uint32_t pass_add = 0) {
  static_assert(MODE != kMeasureOnly || MEAS, "measure-only pass measures");
  const int L = lat.L;
  const int H = L >> 1;
  const uint32_t PS = static_cast<uint32_t>(H) * static_cast<uint32_t>(L);
  const uint32_t half = PS * static_cast<uint32_t>(L);
  const int y0 = yt * lat.ty, z0 = zt * lat.tz;
  const int TYa = min(lat.ty, L - y0), TZa = min(lat.tz, L - z0);
  const bool act = in_block && ty < TYa && tz < TZa;
  const int y = y0 + ty, z = z0 + tz;
  float* const slot = lat.spins + static_cast<size_t>(r) * (4 * static_cast<size_t>(half));
  const SpinGuard sg = spin_guard(slot, 4 * static_cast<size_t>(half), pp.status);
  float* const own = slot + colour * (2 * half);            // cos; sin at + half
  const float* const oth = slot + (colour ^ 1) * (2 * half);
  const int stride_z = lat.ty + 2;  // rows per plane in shared memory
  auto row_ptr = [&](int dy, int dz) -> float* { return sm + (dz * stride_z + dy) * 2 * H; };
  const uint32_t offy = static_cast<uint32_t>(H * y + 4 * tx);
  const uint32_t offz = offy + static_cast<uint32_t>(z) * PS;
  const int kh0 = (tx == 0) ? H - 1 : 4 * tx - 1;
  const int kh1 = (4 * tx + 4 == H) ? 0 : 4 * tx + 4;

  float beta = 0.f;
  uint32_t tagw = 0u, mlo = 0u, mhi = 0u;
  if (MODE == kMetropolis) {
    beta = __ldcg(pp.beta_slot + lat.slot0 + r);
    tagw = (static_cast<uint32_t>(lat.slot0 + r) << 4) | (static_cast<uint32_t>(colour) << 3) |
           kTagMet;
    const uint64_t mp = (pp.ctr ? pp.ctr[kCtrMpass] : 0ull) + pp.mpass_off + pass_add;
    mlo = static_cast<uint32_t>(mp);
    mhi = static_cast<uint32_t>(mp >> 32);
  }

  Spins4 t_own{};
  if (act) {
    t_own = ld_spins(sg, own + offz, half);
    const bool zlo = tz == 0, zhi = tz == TZa - 1, ylo = ty == 0, yhi = ty == TYa - 1;
    const uint32_t pzm = static_cast<uint32_t>(z == 0 ? L - 1 : z - 1) * PS;
    const uint32_t pzp = static_cast<uint32_t>(z + 1 == L ? 0 : z + 1) * PS;
    const uint32_t oym = static_cast<uint32_t>(H * (y == 0 ? L - 1 : y - 1) + 4 * tx);
    const uint32_t oyp = static_cast<uint32_t>(H * (y + 1 == L ? 0 : y + 1) + 4 * tx);
    const Spins4 a0 = ld_spins(sg, oth + offz, half);
    Spins4 a1 = a0, a2 = a0, a3 = a0, a4 = a0;
    if (zlo) a1 = ld_spins(sg, oth + offy + pzm, half);
    if (zhi) a2 = ld_spins(sg, oth + offy + pzp, half);
    if (ylo) a3 = ld_spins(sg, oth + oym + static_cast<uint32_t>(z) * PS, half);
    if (yhi) a4 = ld_spins(sg, oth + oyp + static_cast<uint32_t>(z) * PS, half);
    put_row(row_ptr(ty + 1, tz + 1), H, tx, a0);
    if (zlo) put_row(row_ptr(ty + 1, 0), H, tx, a1);
    if (zhi) put_row(row_ptr(ty + 1, TZa + 1), H, tx, a2);
    if (ylo) put_row(row_ptr(0, tz + 1), H, tx, a3);
    if (yhi) put_row(row_ptr(TYa + 1, tz + 1), H, tx, a4);
  }
  __syncthreads();
  if (act) {
    const float* r0 = row_ptr(ty + 1, tz + 1);
    const float* rm = row_ptr(ty, tz + 1);
    const float* rp = row_ptr(ty + 2, tz + 1);
    const float* rzm = row_ptr(ty + 1, tz);
    const float* rzp = row_ptr(ty + 1, tz + 2);
    auto row = [&](const float* r) {
      Spins4 v;
      v.c = reinterpret_cast<const float4*>(r)[tx];
      v.s = reinterpret_cast<const float4*>(r + H)[tx];
      return v;
    };
    const Spins4 zc = row(r0), ysm = row(rm), ysp = row(rp), zsm = row(rzm), zsp = row(rzp);
    const int s = (y + z + colour) & 1;
    const int kh = s ? kh1 : kh0;
    const float hc = r0[kh], hs = r0[H + kh];
    uint4 w0 = make_uint4(0u, 0u, 0u, 0u), w1 = w0;
    if (MODE == kMetropolis) {
      const uint32_t q0 = offz >> 1;
      w0 = philox4x32_10(make_uint4(q0, mlo, mhi, tagw), pp.rk);
      w1 = philox4x32_10(make_uint4(q0 + 1u, mlo, mhi, tagw), pp.rk);
    }
    float stepv[kNumSums];
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) stepv[j] = 0.f;
    Spins4 nw;
    update4<MODE, MEAS>(zc, hc, hs, s, ysm, ysp, zsm, zsp, t_own, w0, w1, beta, nw, n_acc, stepv, nullptr, nullptr,
                        pp.measure == 2);
    if (MEAS) {
#pragma unroll
      for (int j = 0; j < kNumSums; ++j) acc_out[j] = stepv[j];
    }
    if (MODE != kMeasureOnly) st_spins(sg, own + offz, half, nw.c, nw.s);
  }
  // The shared rows may be overwritten by the caller's next tile.
  __syncthreads();
}

// Error-free sum of two floats (Knuth's TwoSum): s + e equals a + b
// exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Fixed-order block reduction of the FP32 partials into FP64 (a deterministic
// tree: warp shuffles, then warp totals in order).  Within a warp the tree
// carries each value as an unevaluated FP32 sum s + c, every addition split
// exactly by TwoSum (FP64 arithmetic is a small fraction of the FP32 rate on
// sm_103a, and eight five-level FP64 trees per warp cost as much as the
// half-sweep's update work); lane 0 adds s and c in FP64 and the warp totals
// are summed in FP64.  Thread 0..kNumSums-1 write out[j].  `red` must hold
// kReduceBytes.  Every thread of the block calls it.
__device__ __forceinline__ void block_sums_to(double* out, const float acc[kNumSums], int tid,
                                              int nthreads, double* red) {
  const int lane = tid & 31, warp = tid >> 5;
  const int nw = (nthreads + 31) >> 5;
  const int wn = min(32, nthreads - warp * 32);
  const unsigned mask = wn == 32 ? 0xffffffffu : ((1u << wn) - 1u);
#pragma unroll
  for (int j = 0; j < kNumSums; ++j) {
    float v = acc[j], c = 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ov = __shfl_down_sync(mask, v, off), oc = __shfl_down_sync(mask, c, off);
      if (lane + off < wn) {
        float e;
        two_sum(v, ov, v, e);
        c += oc + e;
      }
    }
    if (lane == 0) red[j * 32 + warp] = static_cast<double>(v) + static_cast<double>(c);
  }
  __syncthreads();
  if (tid < kNumSums) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[tid * 32 + w];
    out[tid] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ void block_count_to(unsigned long long* dst, uint32_t n, int tid,
                                               int nthreads) {
  const int lane = tid & 31, warp = tid >> 5;
  const int wn = min(32, nthreads - warp * 32);
  const unsigned mask = wn == 32 ? 0xffffffffu : ((1u << wn) - 1u);
  const unsigned t = __reduce_add_sync(mask, n);
  if (lane == 0 && t) atomicAdd(dst, static_cast<unsigned long long>(t));
}

}  // namespace xy
