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
// Tile.  A thread block covers full rows in x, `ty` rows in y and marches
// over `tz` planes in z.  A thread loads its own row of the other colour's
// plane z+1 and keeps planes z-1, z, z+1 of its own column in registers;
// planes are shared through three shared-memory buffers (one barrier per
// plane) for the y neighbours and the x halo element.  The thread rows at the
// tile's y edges also load the halo rows y0-1 and y0+ty.  The plane loop is
// unrolled three times so the register planes and the buffer indices rotate
// without copies.
//
// Accuracy.  The reflection renormalises its result with one Newton step
// towards |S| = 1, so stored vectors stay within a few ulp of the unit
// circle however many reflections a spin goes through; the direction (the
// angle) is not changed by that step.  Proposal vectors use the fast sincos,
// evaluated at theta - pi inside [-pi, pi) (absolute error ~2^-21.4).
#pragma once
#include <cstdint>

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
enum TileKind : int { kTileMarch = 0, kTileBlock = 1 };

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
  int measure;                  // fuse the lattice sums (white passes only)
};

// Shared-memory bytes of one tile pass: three plane buffers of ty+2 rows of
// L/2 (cos, sin) pairs, then the reduction area.
__host__ __device__ inline int tile_plane_floats(int L, int ty) { return 3 * (ty + 2) * L; }
__host__ __device__ inline int tile_smem_bytes(int L, int ty) {
  return tile_plane_floats(L, ty) * 4 + kReduceBytes;
}
// kTileBlock: (ty+2) x (tz+2) rows of L/2 (cos, sin) pairs.
__host__ __device__ inline int block_tile_floats(int L, int ty, int tz) { return (ty + 2) * (tz + 2) * L; }
__host__ __device__ inline int tile_floats(int kind, int L, int ty, int tz) {
  return kind == kTileBlock ? block_tile_floats(L, ty, tz) : tile_plane_floats(L, ty);
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

// The reflection of Eq. (2) at the field h = sum of the six neighbour
// vectors: S' = 2 (S.h / h.h) h - S, followed by one Newton step of the norm
// (S' *= 3/2 - |S'|^2 / 2).  h = 0 leaves S (Sec. II reading: no field, no
// reflection); so does a field whose squared length underflows.
__device__ __forceinline__ void reflect(float hx, float hy, float c, float s, float& c1, float& s1) {
  const float n2 = fmaf(hy, hy, hx * hx);
  float rn;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rn) : "f"(n2));
  const float k = 2.f * fmaf(s, hy, c * hx) * rn;
  const float a = fmaf(k, hx, -c), b = fmaf(k, hy, -s);
  const float f = fmaf(-0.5f, fmaf(b, b, a * a), 1.5f);
  const bool keep = !(n2 > 0.f);
  c1 = keep ? c : a * f;
  s1 = keep ? s : b * f;
}

struct Spins4 {
  float c[4];
  float s[4];
};

// Spin loads and stores go through L2 (.cg): the persistent kernel reads
// values other blocks wrote earlier in the same launch.
__device__ __forceinline__ float4 ld4(const float* p) {
  return __ldcg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ void st4(float* p, float4 v) {
  __stcg(reinterpret_cast<float4*>(p), v);
}

// The 4 spins of one thread's row segment: cos at p, sin at p + half.
__device__ __forceinline__ Spins4 ld_spins(const float* p, uint32_t half) {
  const float4 c = ld4(p), s = ld4(p + half);
  Spins4 v;
  v.c[0] = c.x; v.c[1] = c.y; v.c[2] = c.z; v.c[3] = c.w;
  v.s[0] = s.x; v.s[1] = s.y; v.s[2] = s.z; v.s[3] = s.w;
  return v;
}
__device__ __forceinline__ void st_spins(float* p, uint32_t half, const float c[4], const float s[4]) {
  st4(p, make_float4(c[0], c[1], c[2], c[3]));
  st4(p + half, make_float4(s[0], s[1], s[2], s[3]));
}

__device__ __forceinline__ void put_row(float* row, int H, int tx, const Spins4& v) {
  reinterpret_cast<float4*>(row)[tx] = make_float4(v.c[0], v.c[1], v.c[2], v.c[3]);
  reinterpret_cast<float4*>(row + H)[tx] = make_float4(v.s[0], v.s[1], v.s[2], v.s[3]);
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
  float acc[kNumSums];
  float err[kNumSums];
  __device__ __forceinline__ SumAcc() {
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) acc[j] = err[j] = 0.f;
  }
  // Compensated (Kahan) accumulation of one plane's terms, so the per-thread
  // FP32 sums stay within a few roundings of the terms whatever the depth.
  __device__ __forceinline__ void add_plane(const float* step) {
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) {
      const float yv = step[j] - err[j];
      const float t = acc[j] + yv;
      err[j] = (t - acc[j]) - yv;
      acc[j] = t;
    }
  }
  __device__ __forceinline__ void export_to(float* out) const {
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) out[j] = acc[j];
  }
};

// One tile of one half-sweep of colour `colour` on local slot r.
// (tx, ty): thread coordinates, tx in [0, L/8); in_block = the thread maps
// onto the tile at all (the persistent kernel's flat blocks have spares).
// Every thread of the block must call this (it contains barriers).
// acc_out[] receives this thread's FP32 lattice-sum partials (MEAS);
// n_acc its accepted Metropolis proposals.
template <int MODE, bool MEAS>
__device__ __forceinline__ void tile_pass(const Lattice& lat, int r, int yt, int zt, int colour,
                                          int tx, int ty, bool in_block, const PassParams& pp,
                                          float* sm, float* acc_out, uint32_t& n_acc) {
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
    const uint64_t mp = (pp.ctr ? pp.ctr[kCtrMpass] : 0ull) + pp.mpass_off;
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
    pa = ld_spins(oth + offy + zb, half);
    pb = ld_spins(oth + offy + zz, half);
    put_row(row_ptr(0, ty + 1), H, tx, pb);
    if (top) put_row(row_ptr(0, 0), H, tx, ld_spins(oth + offym + zz, half));
    if (bot) put_row(row_ptr(0, TYa + 1), H, tx, ld_spins(oth + offyp + zz, half));
    nx_oth = ld_spins(oth + offy + z1, half);
    nx_own = ld_spins(own + offy + zz, half);
    if (TZa > 1) {
      if (top) nx_h0 = ld_spins(oth + offym + z1, half);
      if (bot) nx_h1 = ld_spins(oth + offyp + z1, half);
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
        nx_oth = ld_spins(oth + offy + pz2, half);
        nx_own = ld_spins(own + offy + pz1, half);
        if (i + 2 < TZa) {
          if (top) nx_h0 = ld_spins(oth + offym + pz2, half);
          if (bot) nx_h1 = ld_spins(oth + offyp + pz2, half);
        }
      }
      const float* rm = row_ptr(b0, ty);
      const float* rp = row_ptr(b0, ty + 2);
      const float* r0 = row_ptr(b0, ty + 1);
      const float4 ymc = reinterpret_cast<const float4*>(rm)[tx];
      const float4 yms = reinterpret_cast<const float4*>(rm + H)[tx];
      const float4 ypc = reinterpret_cast<const float4*>(rp)[tx];
      const float4 yps = reinterpret_cast<const float4*>(rp + H)[tx];
      const int s = (y + z + colour) & 1;
      const int kh = s ? kh1 : kh0;
      const float hc = r0[kh], hs = r0[H + kh];
      // X[e] = the -x neighbour of site e, X[e+1] its +x neighbour.
      float Xc[5], Xs[5];
#pragma unroll
      for (int e = 0; e < 5; ++e) {
        const float a_c = (e < 4) ? zc.c[e] : hc, a_s = (e < 4) ? zc.s[e] : hs;
        const float b_c = (e == 0) ? hc : zc.c[e - 1 < 0 ? 0 : e - 1];
        const float b_s = (e == 0) ? hs : zc.s[e - 1 < 0 ? 0 : e - 1];
        Xc[e] = s ? a_c : b_c;
        Xs[e] = s ? a_s : b_s;
      }
      const uint32_t offz = offy + static_cast<uint32_t>(z) * PS;
      float nc[4], ns[4];
      uint4 w0 = make_uint4(0u, 0u, 0u, 0u), w1 = w0;
      if (MODE == kMetropolis) {
        const uint32_t q0 = offz >> 1;
        w0 = philox4x32_10(make_uint4(q0, mlo, mhi, tagw), pp.rk);
        w1 = philox4x32_10(make_uint4(q0 + 1u, mlo, mhi, tagw), pp.rk);
      }
      float stepv[kNumSums];
#pragma unroll
      for (int j = 0; j < kNumSums; ++j) stepv[j] = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float hx = (Xc[e] + Xc[e + 1]) + (comp(ymc, e) + comp(ypc, e)) + (zm.c[e] + zn.c[e]);
        const float hy = (Xs[e] + Xs[e + 1]) + (comp(yms, e) + comp(yps, e)) + (zm.s[e] + zn.s[e]);
        const float co = t_own.c[e], so = t_own.s[e];
        if (MODE == kMetropolis) {
          const uint4& w = (e < 2) ? w0 : w1;
          const uint32_t wprop = (e & 1) ? w.z : w.x;
          const uint32_t wacc = (e & 1) ? w.w : w.y;
          const float tp = static_cast<float>(wprop >> 8) * kTwoPiOver2p24;  // = u0 * 2 pi
          float cp, sp;
          spin(tp, cp, sp);
          // -beta dE with dE = -[h_x (cos t' - cos t) + h_y (sin t' - sin t)]
          const float x = beta * (hx * (cp - co) + hy * (sp - so));
          // u1 < exp(x)  <=>  (w >> 8) < exp(x) 2^24 (exact scaling)
          const bool accept = static_cast<float>(wacc >> 8) < __expf(x) * 16777216.0f;
          n_acc += accept ? 1u : 0u;
          nc[e] = accept ? cp : co;
          ns[e] = accept ? sp : so;
        } else if (MODE == kOverrelax) {
          reflect(hx, hy, co, so, nc[e], ns[e]);  // reflection about the field
        } else {
          nc[e] = co;
          ns[e] = so;
        }
        if (MEAS) {
          // Bonds (w, w+mu) and (w-mu, w) of the white site w: every bond has
          // exactly one white end, so each is counted once.
          const float c = nc[e], sn = ns[e];
          const float pxc = Xc[e + 1], qxc = Xc[e], pxs = Xs[e + 1], qxs = Xs[e];
          const float pyc = comp(ypc, e), qyc = comp(ymc, e), pys = comp(yps, e), qys = comp(yms, e);
          const float pzc = zn.c[e], qzc = zm.c[e], pzs = zn.s[e], qzs = zm.s[e];
          stepv[0] += c + zc.c[e];  // white site + the black site of this column
          stepv[1] += sn + zc.s[e];
          stepv[2] += c * (pxc + qxc) + sn * (pxs + qxs);
          stepv[3] += c * (pyc + qyc) + sn * (pys + qys);
          stepv[4] += c * (pzc + qzc) + sn * (pzs + qzs);
          stepv[5] += sn * (pxc - qxc) - c * (pxs - qxs);
          stepv[6] += sn * (pyc - qyc) - c * (pys - qys);
          stepv[7] += sn * (pzc - qzc) - c * (pzs - qzs);
        }
      }
      if (MEAS) sums.add_plane(stepv);
      if (MODE != kMeasureOnly) st_spins(own + offz, half, nc, ns);
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
                                           float* sm, float* acc_out, uint32_t& n_acc) {
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
    const uint64_t mp = (pp.ctr ? pp.ctr[kCtrMpass] : 0ull) + pp.mpass_off;
    mlo = static_cast<uint32_t>(mp);
    mhi = static_cast<uint32_t>(mp >> 32);
  }

  Spins4 t_own{};
  if (act) {
    t_own = ld_spins(own + offz, half);
    const bool zlo = tz == 0, zhi = tz == TZa - 1, ylo = ty == 0, yhi = ty == TYa - 1;
    const uint32_t pzm = static_cast<uint32_t>(z == 0 ? L - 1 : z - 1) * PS;
    const uint32_t pzp = static_cast<uint32_t>(z + 1 == L ? 0 : z + 1) * PS;
    const uint32_t oym = static_cast<uint32_t>(H * (y == 0 ? L - 1 : y - 1) + 4 * tx);
    const uint32_t oyp = static_cast<uint32_t>(H * (y + 1 == L ? 0 : y + 1) + 4 * tx);
    const Spins4 a0 = ld_spins(oth + offz, half);
    Spins4 a1 = a0, a2 = a0, a3 = a0, a4 = a0;
    if (zlo) a1 = ld_spins(oth + offy + pzm, half);
    if (zhi) a2 = ld_spins(oth + offy + pzp, half);
    if (ylo) a3 = ld_spins(oth + oym + static_cast<uint32_t>(z) * PS, half);
    if (yhi) a4 = ld_spins(oth + oyp + static_cast<uint32_t>(z) * PS, half);
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
    const float4 zcc = reinterpret_cast<const float4*>(r0)[tx];
    const float4 zcs = reinterpret_cast<const float4*>(r0 + H)[tx];
    const float4 ymc = reinterpret_cast<const float4*>(rm)[tx];
    const float4 yms = reinterpret_cast<const float4*>(rm + H)[tx];
    const float4 ypc = reinterpret_cast<const float4*>(rp)[tx];
    const float4 yps = reinterpret_cast<const float4*>(rp + H)[tx];
    const float4 zmc = reinterpret_cast<const float4*>(rzm)[tx];
    const float4 zms = reinterpret_cast<const float4*>(rzm + H)[tx];
    const float4 zpc = reinterpret_cast<const float4*>(rzp)[tx];
    const float4 zps = reinterpret_cast<const float4*>(rzp + H)[tx];
    const int s = (y + z + colour) & 1;
    const int kh = s ? kh1 : kh0;
    const float hc = r0[kh], hs = r0[H + kh];
    float Xc[5], Xs[5];
#pragma unroll
    for (int e = 0; e < 5; ++e) {
      const float a_c = (e < 4) ? comp(zcc, e < 4 ? e : 0) : hc;
      const float a_s = (e < 4) ? comp(zcs, e < 4 ? e : 0) : hs;
      const float b_c = (e == 0) ? hc : comp(zcc, e == 0 ? 0 : e - 1);
      const float b_s = (e == 0) ? hs : comp(zcs, e == 0 ? 0 : e - 1);
      Xc[e] = s ? a_c : b_c;
      Xs[e] = s ? a_s : b_s;
    }
    float nc[4], ns[4];
    uint4 w0 = make_uint4(0u, 0u, 0u, 0u), w1 = w0;
    if (MODE == kMetropolis) {
      const uint32_t q0 = offz >> 1;
      w0 = philox4x32_10(make_uint4(q0, mlo, mhi, tagw), pp.rk);
      w1 = philox4x32_10(make_uint4(q0 + 1u, mlo, mhi, tagw), pp.rk);
    }
    float stepv[kNumSums];
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) stepv[j] = 0.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float hx = (Xc[e] + Xc[e + 1]) + (comp(ymc, e) + comp(ypc, e)) + (comp(zmc, e) + comp(zpc, e));
      const float hy = (Xs[e] + Xs[e + 1]) + (comp(yms, e) + comp(yps, e)) + (comp(zms, e) + comp(zps, e));
      const float co = t_own.c[e], so = t_own.s[e];
      if (MODE == kMetropolis) {
        const uint4& w = (e < 2) ? w0 : w1;
        const uint32_t wprop = (e & 1) ? w.z : w.x;
        const uint32_t wacc = (e & 1) ? w.w : w.y;
        const float tp = static_cast<float>(wprop >> 8) * kTwoPiOver2p24;
        float cp, sp;
        spin(tp, cp, sp);
        const float x = beta * (hx * (cp - co) + hy * (sp - so));
        const bool accept = static_cast<float>(wacc >> 8) < __expf(x) * 16777216.0f;
        n_acc += accept ? 1u : 0u;
        nc[e] = accept ? cp : co;
        ns[e] = accept ? sp : so;
      } else if (MODE == kOverrelax) {
        reflect(hx, hy, co, so, nc[e], ns[e]);
      } else {
        nc[e] = co;
        ns[e] = so;
      }
      if (MEAS) {
        const float c = nc[e], sn = ns[e];
        const float pxc = Xc[e + 1], qxc = Xc[e], pxs = Xs[e + 1], qxs = Xs[e];
        const float pyc = comp(ypc, e), qyc = comp(ymc, e), pys = comp(yps, e), qys = comp(yms, e);
        const float pzc = comp(zpc, e), qzc = comp(zmc, e), pzs = comp(zps, e), qzs = comp(zms, e);
        stepv[0] += c + comp(zcc, e);
        stepv[1] += sn + comp(zcs, e);
        stepv[2] += c * (pxc + qxc) + sn * (pxs + qxs);
        stepv[3] += c * (pyc + qyc) + sn * (pys + qys);
        stepv[4] += c * (pzc + qzc) + sn * (pzs + qzs);
        stepv[5] += sn * (pxc - qxc) - c * (pxs - qxs);
        stepv[6] += sn * (pyc - qyc) - c * (pys - qys);
        stepv[7] += sn * (pzc - qzc) - c * (pzs - qzs);
      }
    }
    if (MEAS) {
#pragma unroll
      for (int j = 0; j < kNumSums; ++j) acc_out[j] = stepv[j];
    }
    if (MODE != kMeasureOnly) st_spins(own + offz, half, nc, ns);
  }
  // The shared rows may be overwritten by the caller's next tile.
  __syncthreads();
}

// Fixed-order block reduction of the FP32 partials into FP64 (a deterministic
// tree: warp shuffles, then warp totals in order).  Thread 0..kNumSums-1 write
// out[j].  `red` must hold kReduceBytes.  Every thread of the block calls it.
__device__ __forceinline__ void block_sums_to(double* out, const float acc[kNumSums], int tid,
                                              int nthreads, double* red) {
  const int lane = tid & 31, warp = tid >> 5;
  const int nw = (nthreads + 31) >> 5;
  const int wn = min(32, nthreads - warp * 32);
  const unsigned mask = wn == 32 ? 0xffffffffu : ((1u << wn) - 1u);
#pragma unroll
  for (int j = 0; j < kNumSums; ++j) {
    double v = static_cast<double>(acc[j]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_down_sync(mask, v, off);
      if (lane + off < wn) v += o;
    }
    if (lane == 0) red[j * 32 + warp] = v;
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
