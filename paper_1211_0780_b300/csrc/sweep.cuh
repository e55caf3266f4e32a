// Checkerboard half-sweep of the 3D XY model on sm_103a: Metropolis
// (Sec. II, Fig. 2), over-relaxation (Sec. II, Eq. 2) and the lattice sums of
// Eqs. (4)-(6), fused into one tile pass.
//
// Layout.  Each slot (replica) of an L^3 lattice holds two packed FP32 angle
// arrays, colour 0 then colour 1, of N/2 floats each; site (x, y, z) of colour
// c = (x+y+z) & 1 sits at p = (x >> 1) + (L/2)(y + L z) of array c.  A row
// (y, z) of one colour is L/2 contiguous floats, so a thread owns one float4
// = 4 same-colour sites of a row (x = 2k + s, k = 4 tx .. 4 tx + 3, with
// s = (y + z + c) & 1).  Its six neighbours are all of the other colour:
//   x-1, x+1 -> same row, packed k-1+s and k+s (one element comes from the
//               neighbouring float4, with periodic wrap along the row);
//   y+-1, z+-1 -> the other colour's rows (y+-1, z), (y, z+-1) at the same k.
//
// Tile.  A thread block covers full rows in x, `ty` rows in y and marches
// over `tz` planes in z.  The cos/sin of every other-colour site it needs is
// evaluated once per block: a thread evaluates its own row of plane z+1 and
// keeps planes z-1, z, z+1 of its own column in registers; planes are shared
// through three shared-memory buffers (one barrier per plane) for the y
// neighbours and the x halo element.  The thread rows at the tile's y edges
// also evaluate the halo rows y0-1 and y0+ty.  Cost per update:
// (ty+2)(tz+2)/(ty tz) sincos evaluations instead of six.
//
// Accuracy.  Angles live in [0, 2 pi); the fast sincos is evaluated at
// theta - pi, inside [-pi, pi) where its absolute error is ~2^-21.4, and
// negated.
#pragma once
#include <cstdint>

#include "philox.cuh"

namespace xy {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr uint32_t kTagInit = 1u, kTagMet = 2u, kTagPt = 3u;
constexpr int kNumSums = 8;                       // Mx, My, Cx, Cy, Cz, Sx, Sy, Sz
constexpr int kReduceBytes = kNumSums * 32 * 8;   // per-warp FP64 partials

enum Mode : int { kMetropolis = 0, kOverrelax = 1, kMeasureOnly = 2 };

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
  float* angles;  // slot r, colour c at angles + r*N + c*(N/2)
  int L;
  int R;
  int slot0;      // global index of local slot 0
  int ty, tz;     // tile: ty rows x tz planes, full rows in x
  int nyt, nzt;   // tiles per slot along y and z
  int part0;      // first tile partial of this lattice; slot r tile t at
                  // part0 + r*nyt*nzt + t, t = yt + nyt*zt
};

struct PassParams {
  uint64_t seed;
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

__device__ __forceinline__ void spin(float th, float& c, float& s) {
  float sn, cs;
  __sincosf(th - kPi, &sn, &cs);
  c = -cs;
  s = -sn;
}

struct Spins4 {
  float c[4];
  float s[4];
};

__device__ __forceinline__ Spins4 spins4(float4 t) {
  Spins4 v;
  spin(t.x, v.c[0], v.s[0]);
  spin(t.y, v.c[1], v.s[1]);
  spin(t.z, v.c[2], v.s[2]);
  spin(t.w, v.c[3], v.s[3]);
  return v;
}

// Angle loads and stores go through L2 (.cg): the persistent kernel reads
// values other blocks wrote earlier in the same launch.
__device__ __forceinline__ float4 ld4(const float* p) {
  return __ldcg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ void st4(float* p, float4 v) {
  __stcg(reinterpret_cast<float4*>(p), v);
}

__device__ __forceinline__ void put_row(float* row, int H, int tx, const Spins4& v) {
  reinterpret_cast<float4*>(row)[tx] = make_float4(v.c[0], v.c[1], v.c[2], v.c[3]);
  reinterpret_cast<float4*>(row + H)[tx] = make_float4(v.s[0], v.s[1], v.s[2], v.s[3]);
}

__device__ __forceinline__ float comp(const float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// One tile of one half-sweep of colour `colour` on local slot r.
// (tx, ty): thread coordinates, tx in [0, L/8); in_block = the thread maps
// onto the tile at all (the persistent kernel's flat blocks have spares).
// Every thread of the block must call this (it contains barriers).
// acc[] receives this thread's FP32 lattice-sum partials when measuring;
// n_acc its accepted Metropolis proposals.
template <int MODE>
__device__ __forceinline__ void tile_pass(const Lattice& lat, int r, int yt, int zt, int colour,
                                          int tx, int ty, bool in_block, const PassParams& pp,
                                          float* sm, float acc[kNumSums], uint32_t& n_acc) {
  const int L = lat.L;
  const int H = L >> 1;
  const long long N = static_cast<long long>(L) * L * L;
  const int y0 = yt * lat.ty, z0 = zt * lat.tz;
  const int TYa = min(lat.ty, L - y0), TZa = min(lat.tz, L - z0);
  const bool act = in_block && ty < TYa;
  const int y = y0 + ty;
  float* own = lat.angles + r * N + colour * (N >> 1);
  const float* oth = lat.angles + r * N + (colour ^ 1) * (N >> 1);
  const int rows = lat.ty + 2;
  const int ym = (y0 == 0 ? L : y0) - 1;          // halo row y0 - 1 (periodic)
  const int yp = (y0 + TYa == L) ? 0 : y0 + TYa;  // halo row y0 + TYa
  const bool top = act && ty == 0;
  const bool bot = act && ty == TYa - 1;
  const bool meas = (MODE == kMeasureOnly) || (pp.measure && colour == 1);
  auto idx = [&](int yy, int zz) -> long long {
    return static_cast<long long>(H) * (yy + static_cast<long long>(L) * zz) + 4 * tx;
  };
  auto row_ptr = [&](int b, int rr) -> float* { return sm + (b * rows + rr) * 2 * H; };

  float beta = 0.f;
  PhiloxKey key{0u, 0u};
  uint32_t tagw = 0u;
  uint64_t mp = 0ull;
  if (MODE == kMetropolis) {
    beta = __ldcg(pp.beta_slot + lat.slot0 + r);
    key = philox_key(pp.seed);
    tagw = (static_cast<uint32_t>(lat.slot0 + r) << 4) | (static_cast<uint32_t>(colour) << 3) |
           kTagMet;
    mp = (pp.ctr ? pp.ctr[kCtrMpass] : 0ull) + pp.mpass_off;
  }

  Spins4 zm{}, zc{}, zn{};  // other colour, own column: planes z-1, z, z+1
  float4 nx_oth = make_float4(0.f, 0.f, 0.f, 0.f), nx_own = nx_oth, nx_h0 = nx_oth, nx_h1 = nx_oth;
  if (act) {
    const int zb = (z0 == 0 ? L : z0) - 1;
    const int z1 = (z0 + 1 == L) ? 0 : z0 + 1;
    zm = spins4(ld4(oth + idx(y, zb)));
    zc = spins4(ld4(oth + idx(y, z0)));
    put_row(row_ptr(0, ty + 1), H, tx, zc);
    if (top) put_row(row_ptr(0, 0), H, tx, spins4(ld4(oth + idx(ym, z0))));
    if (bot) put_row(row_ptr(0, TYa + 1), H, tx, spins4(ld4(oth + idx(yp, z0))));
    nx_oth = ld4(oth + idx(y, z1));
    nx_own = ld4(own + idx(y, z0));
    if (TZa > 1) {
      if (top) nx_h0 = ld4(oth + idx(ym, z1));
      if (bot) nx_h1 = ld4(oth + idx(yp, z1));
    }
  }
  __syncthreads();

  int b0 = 0, b1 = 1;
  for (int i = 0; i < TZa; ++i) {
    const int z = z0 + i;
    if (act) {
      const float4 t_oth = nx_oth, t_own = nx_own, t_h0 = nx_h0, t_h1 = nx_h1;
      if (i + 1 < TZa) {  // prefetch the next plane's operands
        const int z1 = z + 1;
        const int z2 = (z1 + 1 == L) ? 0 : z1 + 1;
        nx_oth = ld4(oth + idx(y, z2));
        nx_own = ld4(own + idx(y, z1));
        if (i + 2 < TZa) {
          if (top) nx_h0 = ld4(oth + idx(ym, z2));
          if (bot) nx_h1 = ld4(oth + idx(yp, z2));
        }
      }
      zn = spins4(t_oth);
      if (i + 1 < TZa) {
        put_row(row_ptr(b1, ty + 1), H, tx, zn);
        if (top) put_row(row_ptr(b1, 0), H, tx, spins4(t_h0));
        if (bot) put_row(row_ptr(b1, TYa + 1), H, tx, spins4(t_h1));
      }
      const float* rm = row_ptr(b0, ty);
      const float* rp = row_ptr(b0, ty + 2);
      const float* r0 = row_ptr(b0, ty + 1);
      const float4 ymc = reinterpret_cast<const float4*>(rm)[tx];
      const float4 yms = reinterpret_cast<const float4*>(rm + H)[tx];
      const float4 ypc = reinterpret_cast<const float4*>(rp)[tx];
      const float4 yps = reinterpret_cast<const float4*>(rp + H)[tx];
      const int s = (y + z + colour) & 1;
      const int kh = s ? ((4 * tx + 4 == H) ? 0 : 4 * tx + 4) : (tx == 0 ? H - 1 : 4 * tx - 1);
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
      const float th[4] = {t_own.x, t_own.y, t_own.z, t_own.w};
      float tn[4], nc[4], ns[4];
      uint4 w0 = make_uint4(0u, 0u, 0u, 0u), w1 = w0;
      if (MODE == kMetropolis) {
        const uint32_t q0 = static_cast<uint32_t>(idx(y, z) >> 1);
        const uint32_t mlo = static_cast<uint32_t>(mp), mhi = static_cast<uint32_t>(mp >> 32);
        w0 = philox4x32_10(make_uint4(q0, mlo, mhi, tagw), key);
        w1 = philox4x32_10(make_uint4(q0 + 1u, mlo, mhi, tagw), key);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float hx = (Xc[e] + Xc[e + 1]) + (comp(ymc, e) + comp(ypc, e)) + (zm.c[e] + zn.c[e]);
        const float hy = (Xs[e] + Xs[e + 1]) + (comp(yms, e) + comp(yps, e)) + (zm.s[e] + zn.s[e]);
        if (MODE == kMetropolis) {
          const uint4& w = (e < 2) ? w0 : w1;
          const uint32_t wprop = (e & 1) ? w.z : w.x;
          const uint32_t wacc = (e & 1) ? w.w : w.y;
          const float tp = u24(wprop) * kTwoPi;
          float cp, sp, co, so;
          spin(tp, cp, sp);
          spin(th[e], co, so);
          // -beta dE with dE = -[h_x (cos t' - cos t) + h_y (sin t' - sin t)]
          const float x = beta * (hx * (cp - co) + hy * (sp - so));
          const bool accept = u24(wacc) < __expf(x);
          n_acc += accept ? 1u : 0u;
          tn[e] = accept ? tp : th[e];
          nc[e] = accept ? cp : co;
          ns[e] = accept ? sp : so;
        } else if (MODE == kOverrelax) {
          float t = th[e];
          if (hx != 0.f || hy != 0.f) {
            t = fmaf(2.f, atan2f(hy, hx), -th[e]);  // reflection about the field
            if (t < 0.f) t += kTwoPi;
            if (t < 0.f) t += kTwoPi;
            if (t >= kTwoPi) t -= kTwoPi;
          }
          tn[e] = t;
          if (meas) spin(t, nc[e], ns[e]);
        } else {
          tn[e] = th[e];
          spin(th[e], nc[e], ns[e]);
        }
        if (meas) {
          // Bonds (w, w+mu) and (w-mu, w) of the white site w: every bond has
          // exactly one white end, so each is counted once.
          const float c = nc[e], sn = ns[e];
          const float pxc = Xc[e + 1], qxc = Xc[e], pxs = Xs[e + 1], qxs = Xs[e];
          const float pyc = comp(ypc, e), qyc = comp(ymc, e), pys = comp(yps, e), qys = comp(yms, e);
          const float pzc = zn.c[e], qzc = zm.c[e], pzs = zn.s[e], qzs = zm.s[e];
          acc[0] += c + zc.c[e];  // white site + the black site of this column
          acc[1] += sn + zc.s[e];
          acc[2] += c * (pxc + qxc) + sn * (pxs + qxs);
          acc[3] += c * (pyc + qyc) + sn * (pys + qys);
          acc[4] += c * (pzc + qzc) + sn * (pzs + qzs);
          acc[5] += sn * (pxc - qxc) - c * (pxs - qxs);
          acc[6] += sn * (pyc - qyc) - c * (pys - qys);
          acc[7] += sn * (pzc - qzc) - c * (pzs - qzs);
        }
      }
      if (MODE != kMeasureOnly) st4(own + idx(y, z), make_float4(tn[0], tn[1], tn[2], tn[3]));
    }
    zm = zc;
    zc = zn;
    b0 = b0 == 2 ? 0 : b0 + 1;
    b1 = b1 == 2 ? 0 : b1 + 1;
    __syncthreads();
  }
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
