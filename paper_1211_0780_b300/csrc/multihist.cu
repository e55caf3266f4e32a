// Multi-histogram reweighting (Ferrenberg and Swendsen, 1989) of the series
// of all temperatures of a parallel-tempering ladder (the paper reweights
// nothing: it bins its series on the host, Sec. II; this combines every
// replica's data into one estimate at any beta').
//
// Records t = 1..T, pooled over the R couplings beta_m, N_m of them sampled
// at beta_m.  With free energies f_m (f_0 = 0),
//   log D_t = log sum_m N_m exp(f_m - beta_m E_t),
//   f_k     = -log sum_t exp(-beta_k E_t - log D_t)          (*)
// and at any beta'
//   <O>_beta' = sum_t O_t exp(-beta' E_t - log D_t) / sum_t exp(...).
// (*) are the stationarity conditions of the convex function
//   F(f) = sum_t log D_t(f) - sum_m N_m f_m,
//   dF/df_k = sum_t p_kt - N_k,  p_kt = N_k exp(f_k - beta_k E_t) / D_t,
//   d2F/df_k df_l = sum_t (delta_kl p_kt - p_kt p_lt),
// so they are solved by Newton's method on F (f_0 held at 0, a backtracking
// line search on F), which takes a handful of steps where the textbook
// fixed-point iteration of (*) takes hundreds.  Everything in FP64 with
// log-sum-exp shifts: per record for log D (the largest of its R terms),
// per coupling for the sums over records (a separate max pass).
// Reductions are fixed-order (deterministic).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/xy.h"

namespace {

constexpr int kMaxR = 64;        // couplings of one ladder (Newton: R(R+1)/2 Hessian terms)
constexpr int kBlock = 256;
constexpr int kNSum = 11;        // as the single-histogram sums
constexpr int kKT = 4;           // target couplings per thread
constexpr int kChunk = 256;

// Newton sums: R gradient terms, R(R+1)/2 Hessian terms (upper triangle),
// then sum_t log D_t.
__host__ __device__ inline int newton_items(int R) { return R + R * (R + 1) / 2 + 1; }

struct Plan {
  int n_tblocks;                 // blocks over records (f iteration, max pass)
  int n_kblocks, n_tchunks;      // sums pass
  int64_t t_per_chunk;
  size_t off_logD, off_coef, off_part, off_tot, off_group, off_max, off_kmax, off_stats, off_sums, total;
};

Plan plan_for(int64_t T, int R, int K) {
  Plan p{};
  p.n_tblocks = static_cast<int>(std::min<int64_t>(512, (T + kBlock - 1) / kBlock));
  p.n_kblocks = std::max(1, (K + kKT * kBlock - 1) / (kKT * kBlock));  // K = 0: solving only
  const int64_t want = std::max<int64_t>(1, 4 * 148 / p.n_kblocks);  // four full waves on 148 SMs
  p.n_tchunks = static_cast<int>(std::min<int64_t>(want, (T + kChunk - 1) / kChunk));
  p.t_per_chunk = (T + p.n_tchunks - 1) / p.n_tchunks;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t at = off;
    off = (off + b + 255) / 256 * 256;
    return at;
  };
  p.off_logD = take(static_cast<size_t>(T) * 8);
  p.off_coef = take(static_cast<size_t>(3 * kMaxR) * 8);  // log N + f, betas, log N
  p.off_part = take(static_cast<size_t>(p.n_tblocks) * newton_items(R) * 8);
  p.off_tot = take(static_cast<size_t>(newton_items(R)) * 8);
  p.off_group = take(static_cast<size_t>(2 * R + 1) * 8);  // group offsets, then group mean energies
  p.off_max = take(static_cast<size_t>(p.n_tblocks) * std::max(K, 1) * 8);
  p.off_kmax = take(static_cast<size_t>(std::max(K, 1)) * 8);
  p.off_stats = take(4 * 8);
  p.off_sums = take(static_cast<size_t>(p.n_tchunks) * std::max(K, 1) * kNSum * 8);
  p.total = off;
  return p;
}

// coef[m] = log N_m + f_m, coef[R + m] = beta_m, coef[2R + m] = log N_m.
// log D_t = log sum_m exp(coef[m] - beta_m E_t), shifted by the largest term.
__global__ void k_mh_logD(int64_t T, const double* __restrict__ E, int R, const double* __restrict__ coef,
                          double* __restrict__ logD) {
  __shared__ double s_a[kMaxR], s_b[kMaxR];
  for (int m = threadIdx.x; m < R; m += blockDim.x) {
    s_a[m] = coef[m];
    s_b[m] = coef[R + m];
  }
  __syncthreads();
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < T;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double e = E[t];
    double mx = -INFINITY;
    for (int m = 0; m < R; ++m) mx = fmax(mx, fma(-s_b[m], e, s_a[m]));
    double s = 0.0;
    for (int m = 0; m < R; ++m) s += exp(fma(-s_b[m], e, s_a[m]) - mx);
    logD[t] = mx + log(s);
  }
}

constexpr int kNewtonRecords = 32;   // records staged per step in shared memory
constexpr int kMaxItemsPerThread = (kMaxR + kMaxR * (kMaxR + 1) / 2 + 1 + kBlock - 1) / kBlock;

// Per block: the Newton sums over its records, item q of newton_items(R):
// q < R: sum_t p_qt; then the upper triangle (k <= l) of sum_t p_kt p_lt in
// row order; last: sum_t log D_t.  p_kt = exp(coef[k] - beta_k E_t - log D_t)
// (coef[k] = log N_k + f_k), staged kNewtonRecords records at a time.
__global__ void __launch_bounds__(kBlock) k_mh_newton(int64_t T, const double* __restrict__ E,
                                                      const double* __restrict__ logD, int R,
                                                      const double* __restrict__ coef, double* __restrict__ part) {
  __shared__ double s_p[kNewtonRecords][kMaxR];
  __shared__ double s_l[kNewtonRecords];
  __shared__ unsigned char s_k[kMaxR * (kMaxR + 1) / 2], s_kl[kMaxR * (kMaxR + 1) / 2];
  const int Q = newton_items(R), P = R * (R + 1) / 2;
  for (int k = threadIdx.x; k < R; k += blockDim.x) {
    const int off = k * R - k * (k - 1) / 2;
    for (int l = k; l < R; ++l) {
      s_k[off + l - k] = static_cast<unsigned char>(k);
      s_kl[off + l - k] = static_cast<unsigned char>(l);
    }
  }
  double acc[kMaxItemsPerThread];
#pragma unroll
  for (int i = 0; i < kMaxItemsPerThread; ++i) acc[i] = 0.0;
  const int64_t per = (T + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = blockIdx.x * per, t1 = (t0 + per < T) ? t0 + per : T;
  for (int64_t tb = t0; tb < t1; tb += kNewtonRecords) {
    const int n = static_cast<int>((t1 - tb) < kNewtonRecords ? (t1 - tb) : kNewtonRecords);
    __syncthreads();
    for (int q = threadIdx.x; q < n * R; q += blockDim.x) {
      const int j = q / R, k = q - j * R;
      const double e = E[tb + j], lD = logD[tb + j];
      s_p[j][k] = exp(fma(-coef[R + k], e, coef[k]) - lD);
      if (k == 0) s_l[j] = lD;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kMaxItemsPerThread; ++i) {
      const int q = threadIdx.x + i * blockDim.x;
      if (q >= Q) break;
      double v = acc[i];
      if (q < R) {
        for (int j = 0; j < n; ++j) v += s_p[j][q];
      } else if (q < R + P) {
        const int k = s_k[q - R], l = s_kl[q - R];
        for (int j = 0; j < n; ++j) v = fma(s_p[j][k], s_p[j][l], v);
      } else {
        for (int j = 0; j < n; ++j) v += s_l[j];
      }
      acc[i] = v;
    }
  }
#pragma unroll
  for (int i = 0; i < kMaxItemsPerThread; ++i) {
    const int q = threadIdx.x + i * blockDim.x;
    if (q < Q) part[static_cast<int64_t>(blockIdx.x) * Q + q] = acc[i];
  }
}

// Block partials of each item added in block order.
__global__ void k_mh_total(int nblk, int Q, const double* __restrict__ part, double* __restrict__ tot) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  double v = 0.0;
  for (int b = 0; b < nblk; ++b) v += part[static_cast<int64_t>(b) * Q + q];
  tot[q] = v;
}

// Per block: sum of log D_t over the block's records (for F alone).
__global__ void k_mh_logD_sum(int64_t T, const double* __restrict__ logD, double* __restrict__ part) {
  __shared__ double s[kBlock];
  const int64_t per = (T + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = blockIdx.x * per, t1 = (t0 + per < T) ? t0 + per : T;
  double v = 0.0;
  for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) v += logD[t];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// Mean energy of each coupling's records (records grouped by coupling, group
// m = [off[m], off[m+1])), one block per group, fixed-order tree.
__global__ void k_mh_group_mean(const double* __restrict__ E, const int64_t* __restrict__ off,
                                double* __restrict__ mean) {
  __shared__ double s[kBlock];
  const int m = blockIdx.x;
  const int64_t a = off[m], b = off[m + 1];
  double v = 0.0;
  for (int64_t t = a + threadIdx.x; t < b; t += blockDim.x) v += E[t];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) mean[m] = s[0] / static_cast<double>(b - a);
}

// Solves the symmetric positive definite system A x = b (n x n, row-major,
// overwritten) by Cholesky factorisation; false if A is not positive
// definite to working precision.
bool cholesky_solve(std::vector<double>& A, std::vector<double>& b, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = A[i * n + j];
      for (int k = 0; k < j; ++k) v -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = v / d;
    }
  }
  for (int i = 0; i < n; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= A[i * n + k] * b[k];
    b[i] = v / A[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = b[i];
    for (int k = i + 1; k < n; ++k) v -= A[k * n + i] * b[k];
    b[i] = v / A[i * n + i];
  }
  return true;
}

// Evaluation.  Max pass: per block, max over its records of
// x_kt = -beta'_k E_t - log D_t for every k.
__global__ void k_mh_max(int64_t T, const double* __restrict__ E, const double* __restrict__ logD, int K,
                         const double* __restrict__ betap, double* __restrict__ part) {
  __shared__ double s_e[kChunk], s_l[kChunk];
  const int64_t per = (T + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = blockIdx.x * per, t1 = (t0 + per < T) ? t0 + per : T;
  for (int k = threadIdx.x; k < K; k += blockDim.x) part[static_cast<int64_t>(blockIdx.x) * K + k] = -INFINITY;
  for (int64_t tb = t0; tb < t1; tb += kChunk) {
    const int n = static_cast<int>((t1 - tb) < kChunk ? (t1 - tb) : kChunk);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      s_e[j] = E[tb + j];
      s_l[j] = logD[tb + j];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      const double b = betap[k];
      double mx = part[static_cast<int64_t>(blockIdx.x) * K + k];
      for (int j = 0; j < n; ++j) mx = fmax(mx, fma(-b, s_e[j], -s_l[j]));
      part[static_cast<int64_t>(blockIdx.x) * K + k] = mx;
    }
  }
}

__global__ void k_mh_max_finish(int K, int nblk, const double* __restrict__ part, double* __restrict__ kmax) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double mx = -INFINITY;
  for (int b = 0; b < nblk; ++b) mx = fmax(mx, part[static_cast<int64_t>(b) * K + k]);
  kmax[k] = mx;
}

// Grid step (beta'_K-1 - beta'_0) / (K - 1), and whether the couplings of the
// thread group starting at k0 sit on it to a few ulps (then the group steps
// its weights by a per-sample factor instead of one exp per pair).
__device__ __forceinline__ double grid_step(int K, const double* betap) {
  return K > 1 ? (betap[K - 1] - betap[0]) / (K - 1) : 0.0;
}
__device__ __forceinline__ bool group_on_grid(int k0, int K, const double* betap, double step) {
  if (step == 0.0 || k0 + 1 >= K) return false;
  bool even = true;
  for (int i = 1; i < kKT && k0 + i < K; ++i)
    even = even && fabs(betap[k0 + i] - (betap[k0] + i * step)) <= 8.0 * 2.220446049250313e-16 * fabs(betap[k0 + i]);
  return even;
}

// Sums pass: chunk partial sums of w x_j, w = exp(x_kt - max_k), x_j in
// {1, e, e^2, m2, m2 e, m4, m4 e, c, c e, s2, s2 e}, e = E - Ebar (Ebar =
// stats[0], the record mean); each thread owns kKT consecutive k.
__global__ void __launch_bounds__(kBlock) k_mh_sums(int64_t T, int64_t t_per_chunk, const double* __restrict__ E,
                                                    const double* __restrict__ logD, const float* __restrict__ m2,
                                                    const float* __restrict__ m4, const float* __restrict__ c,
                                                    const float* __restrict__ s2, int K,
                                                    const double* __restrict__ betap, const double* __restrict__ kmax,
                                                    const double* __restrict__ stats, double* __restrict__ sums) {
  __shared__ double s_E[kChunk], s_l[kChunk], s_m2[kChunk], s_m4[kChunk], s_c[kChunk], s_s2[kChunk], s_rho[kChunk];
  // e = E - Ebar and its products with the observables, staged once per
  // block so that every accumulation below is one fused multiply-add by w
  __shared__ double s_e[kChunk], s_ee[kChunk], s_em2[kChunk], s_em4[kChunk], s_ec[kChunk], s_es2[kChunk];
  const int chunk = blockIdx.y;
  const int64_t t0 = chunk * t_per_chunk, t1 = (t0 + t_per_chunk < T) ? t0 + t_per_chunk : T;
  const int k0 = (blockIdx.x * blockDim.x + threadIdx.x) * kKT;
  const double Ebar = stats[0];
  // On the grid, coupling k0+i uses the shift max_k0 - i step Ebar, so that
  // its weight is the first one times rho_t^i, rho_t = exp(-step (E_t -
  // Ebar)) (evaluated once per sample by the block); the exponent stays
  // below kKT |step| max |E - Ebar|.
  const double step = grid_step(K, betap);
  const bool even = k0 < K && group_on_grid(k0, K, betap, step);
  double b[kKT], mx[kKT];
  int nk = 0;
#pragma unroll
  for (int i = 0; i < kKT; ++i) {
    const int k = k0 + i;
    b[i] = k < K ? betap[k] : 0.0;
    mx[i] = k < K ? kmax[k] : 0.0;
    nk += k < K ? 1 : 0;
  }
  double S[kKT][kNSum];
#pragma unroll
  for (int i = 0; i < kKT; ++i)
#pragma unroll
    for (int j = 0; j < kNSum; ++j) S[i][j] = 0.0;
  for (int64_t tb = t0; tb < t1; tb += kChunk) {
    const int n = static_cast<int>((t1 - tb) < kChunk ? (t1 - tb) : kChunk);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int64_t t = tb + j;
      s_E[j] = E[t];
      s_l[j] = logD[t];
      s_m2[j] = static_cast<double>(m2[t]);
      s_m4[j] = static_cast<double>(m4[t]);
      s_c[j] = static_cast<double>(c[t]) + static_cast<double>(c[T + t]) + static_cast<double>(c[2 * T + t]);
      s_s2[j] = static_cast<double>(s2[t]) + static_cast<double>(s2[T + t]) + static_cast<double>(s2[2 * T + t]);
      s_rho[j] = exp(-step * (s_E[j] - Ebar));
      const double e = s_E[j] - Ebar;
      s_e[j] = e;
      s_ee[j] = e * e;
      s_em2[j] = e * s_m2[j];
      s_em4[j] = e * s_m4[j];
      s_ec[j] = e * s_c[j];
      s_es2[j] = e * s_s2[j];
    }
    __syncthreads();
    if (nk > 0) {
      for (int j = 0; j < n; ++j) {
        const double Et = s_E[j], e = s_e[j], lD = s_l[j];
        const double x2 = s_m2[j], x4 = s_m4[j], xc = s_c[j], xs = s_s2[j];
        const double ee = s_ee[j], ex2 = s_em2[j], ex4 = s_em4[j], exc = s_ec[j], exs = s_es2[j];
        double w = exp(fma(-b[0], Et, -lD) - mx[0]);
        const double rho = s_rho[j];
#pragma unroll
        for (int i = 0; i < kKT; ++i) {
          if (i > 0) w = even ? w * rho : exp(fma(-b[i], Et, -lD) - mx[i]);
          S[i][0] += w;
          S[i][1] = fma(w, e, S[i][1]);
          S[i][2] = fma(w, ee, S[i][2]);
          S[i][3] = fma(w, x2, S[i][3]);
          S[i][4] = fma(w, ex2, S[i][4]);
          S[i][5] = fma(w, x4, S[i][5]);
          S[i][6] = fma(w, ex4, S[i][6]);
          S[i][7] = fma(w, xc, S[i][7]);
          S[i][8] = fma(w, exc, S[i][8]);
          S[i][9] = fma(w, xs, S[i][9]);
          S[i][10] = fma(w, exs, S[i][10]);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kKT; ++i)
    if (i < nk) {
      double* dst = sums + (static_cast<int64_t>(chunk) * K + k0 + i) * kNSum;
#pragma unroll
      for (int j = 0; j < kNSum; ++j) dst[j] = S[i][j];
    }
}

// Record mean of E in a fixed order (one block).
__global__ void k_mh_mean(int64_t T, const double* __restrict__ E, double* stats) {
  __shared__ double s[kBlock];
  double v = 0.0;
  for (int64_t t = threadIdx.x; t < T; t += blockDim.x) v += E[t];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) stats[0] = s[0] / static_cast<double>(T);
}

// Outputs in the layout of xy_reweight_forward: out[6][K] = {log Z (up to a
// constant common to all k: log sum_t exp(-beta' E_t - log D_t)), <E>,
// <m2>, <m4>, <c>, <s2>}, obs[3][K] = {U_L, rho_s L, q2}, cov[5][K] = cov with E
// of {E, m2, m4, c, s2}.
__global__ void k_mh_finish(int K, int n_tchunks, const double* __restrict__ betap, int L,
                            const double* __restrict__ kmax, const double* __restrict__ stats,
                            const double* __restrict__ sums, double* out, double* obs, double* cov) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double S[kNSum];
#pragma unroll
  for (int j = 0; j < kNSum; ++j) S[j] = 0.0;
  for (int ch = 0; ch < n_tchunks; ++ch) {
    const double* src = sums + (static_cast<int64_t>(ch) * K + k) * kNSum;
#pragma unroll
    for (int j = 0; j < kNSum; ++j) S[j] += src[j];
  }
  const double inv = 1.0 / S[0];
  const double me = S[1] * inv, mm2 = S[3] * inv, mm4 = S[5] * inv, mc = S[7] * inv, ms2 = S[9] * inv;
  const double bp = betap[k];
  // the shift the sums pass used for k (see k_mh_sums)
  const int g0 = (k / kKT) * kKT;
  const double step = grid_step(K, betap);
  const double shift = group_on_grid(g0, K, betap, step) ? kmax[g0] - (k - g0) * step * stats[0] : kmax[k];
  out[0 * K + k] = log(S[0]) + shift;
  out[1 * K + k] = stats[0] + me;
  out[2 * K + k] = mm2;
  out[3 * K + k] = mm4;
  out[4 * K + k] = mc;
  out[5 * K + k] = ms2;
  cov[0 * K + k] = S[2] * inv - me * me;
  cov[1 * K + k] = S[4] * inv - mm2 * me;
  cov[2 * K + k] = S[6] * inv - mm4 * me;
  cov[3 * K + k] = S[8] * inv - mc * me;
  cov[4 * K + k] = S[10] * inv - ms2 * me;
  obs[0 * K + k] = 1.0 - mm4 / (3.0 * mm2 * mm2);
  obs[1 * K + k] = L / 3.0 * (mc - bp * ms2);
  obs[2 * K + k] = mm4 / (mm2 * mm2);  // q2 of Eq. (11)
}

bool valid_ladder(int R, const double* betas, const int64_t* counts, int64_t T) {
  if (R < 1 || R > kMaxR || !betas || !counts) return false;
  int64_t total = 0;
  for (int m = 0; m < R; ++m) {
    if (!std::isfinite(betas[m]) || counts[m] < 1) return false;
    if (m > 0 && !(betas[m] > betas[m - 1])) return false;
    total += counts[m];
  }
  return total == T;
}

}  // namespace

extern "C" {

size_t xy_multihist_scratch_bytes(int64_t T, int R, int K) {
  if (T < 1 || R < 1 || R > kMaxR || K < 0) return 0;
  return plan_for(T, R, K).total;
}

int xy_multihist_solve(int64_t T, const double* d_E, int R, const double* betas, const int64_t* counts, double tol,
                       int max_iter, double* f, int* iters_out, void* d_scratch, size_t scratch_bytes,
                       void* stream) {
  if (T < 1 || !d_E || !f || !d_scratch || !(tol > 0.0) || max_iter < 1) return XY_ERR_ARG;
  if (!valid_ladder(R, betas, counts, T)) return XY_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_scratch) % 256 != 0) return XY_ERR_ARG;
  const Plan p = plan_for(T, R, 0);
  if (scratch_bytes < p.total) return XY_ERR_NOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_scratch);
  double* logD = reinterpret_cast<double*>(ws + p.off_logD);
  double* coef = reinterpret_cast<double*>(ws + p.off_coef);
  double* part = reinterpret_cast<double*>(ws + p.off_part);
  double* tot = reinterpret_cast<double*>(ws + p.off_tot);
  const int Q = newton_items(R), n = R - 1;
  std::vector<double> logN(R), x(R), h_coef(2 * R), h_tot(Q);
  bool guess = true;  // a caller's non-zero finite f is a starting point
  for (int m = 0; m < R; ++m) {
    logN[m] = std::log(static_cast<double>(counts[m]));
    h_coef[R + m] = betas[m];
    guess = guess && std::isfinite(f[m]);
  }
  bool all_zero = true;
  for (int m = 0; m < R; ++m) all_zero = all_zero && f[m] == 0.0;
  if (guess && !all_zero) {
    for (int m = 0; m < R; ++m) x[m] = f[m] - f[0];
  } else {
    // Thermodynamic integration between neighbouring couplings: df/dbeta =
    // <E>, trapezoid rule on the group means (records are grouped by
    // coupling in the order of betas), exact to O(dbeta^3) per step.
    std::vector<int64_t> off(R + 1, 0);
    for (int m = 0; m < R; ++m) off[m + 1] = off[m] + counts[m];
    int64_t* d_off = reinterpret_cast<int64_t*>(ws + p.off_group);
    double* d_mean = reinterpret_cast<double*>(ws + p.off_group) + (R + 1);
    std::vector<double> mean(R);
    if (cudaMemcpyAsync(d_off, off.data(), (R + 1) * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) return XY_ERR_CUDA;
    k_mh_group_mean<<<R, kBlock, 0, st>>>(d_E, d_off, d_mean);
    if (cudaMemcpyAsync(mean.data(), d_mean, R * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return XY_ERR_CUDA;
    x[0] = 0.0;
    for (int m = 1; m < R; ++m) x[m] = x[m - 1] + (betas[m] - betas[m - 1]) * 0.5 * (mean[m] + mean[m - 1]);
  }
  x[0] = 0.0;
  // F(x) and, with `newton`, its gradient and Hessian sums (into h_tot).
  auto evaluate = [&](const std::vector<double>& xv, bool newton, double& F) -> int {
    for (int m = 0; m < R; ++m) h_coef[m] = logN[m] + xv[m];
    if (cudaMemcpyAsync(coef, h_coef.data(), 2 * R * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) return XY_ERR_CUDA;
    k_mh_logD<<<p.n_tblocks, kBlock, 0, st>>>(T, d_E, R, coef, logD);
    double sum_logD = 0.0;
    if (newton) {
      k_mh_newton<<<p.n_tblocks, kBlock, 0, st>>>(T, d_E, logD, R, coef, part);
      k_mh_total<<<(Q + 127) / 128, 128, 0, st>>>(p.n_tblocks, Q, part, tot);
      if (cudaMemcpyAsync(h_tot.data(), tot, Q * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return XY_ERR_CUDA;
      sum_logD = h_tot[Q - 1];
    } else {
      k_mh_logD_sum<<<p.n_tblocks, kBlock, 0, st>>>(T, logD, part);
      k_mh_total<<<1, 32, 0, st>>>(p.n_tblocks, 1, part, tot);
      if (cudaMemcpyAsync(&sum_logD, tot, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return XY_ERR_CUDA;
    }
    F = sum_logD;
    for (int m = 0; m < R; ++m) F -= static_cast<double>(counts[m]) * xv[m];
    return cudaGetLastError() == cudaSuccess ? XY_OK : XY_ERR_CUDA;
  };
  int it = 0;
  bool converged = (R == 1);
  for (; it < max_iter && !converged; ++it) {
    double F = 0.0;
    int rc = evaluate(x, true, F);
    if (rc != XY_OK) return rc;
    // reduced system over k, l >= 1 (f_0 = 0 fixes the common shift)
    std::vector<double> H(static_cast<size_t>(n) * n), g(n);
    for (int k = 1; k < R; ++k) {
      g[k - 1] = h_tot[k] - static_cast<double>(counts[k]);
      for (int l = k; l < R; ++l) {
        const double pkl = h_tot[R + k * R - k * (k - 1) / 2 + (l - k)];
        const double v = (k == l ? h_tot[k] : 0.0) - pkl;
        H[(k - 1) * n + (l - 1)] = v;
        H[(l - 1) * n + (k - 1)] = v;
      }
    }
    std::vector<double> dx(n);
    for (int i = 0; i < n; ++i) dx[i] = -g[i];
    std::vector<double> Hc(H);
    bool ok = cholesky_solve(Hc, dx, n);
    for (int i = 0; i < n && ok; ++i) ok = std::isfinite(dx[i]);
    if (!ok) {
      // Hessian not positive definite to working precision (far from the
      // solution, or couplings without overlap): the fixed-point step of (*),
      // f_k -> f_k - log(sum_t p_kt / N_k), renormalised to f_0 = 0.
      const double r0 = std::log(h_tot[0] / static_cast<double>(counts[0]));
      for (int k = 1; k < R; ++k) dx[k - 1] = -(std::log(h_tot[k] / static_cast<double>(counts[k])) - r0);
    }
    double big = 0.0;
    for (int i = 0; i < n; ++i) big = std::fmax(big, std::fabs(dx[i]));
    if (big > 20.0)  // trust region: at most e^20 in any weight per step
      for (int i = 0; i < n; ++i) dx[i] *= 20.0 / big;
    double step = 0.0, slope = 0.0;
    for (int i = 0; i < n; ++i) {
      step = std::fmax(step, std::fabs(dx[i]));
      slope += g[i] * dx[i];
    }
    // backtracking (Armijo) line search on F
    double alpha = 1.0;
    std::vector<double> xt(x);
    bool moved = false;
    for (int ls = 0; ls < 40; ++ls) {
      for (int i = 0; i < n; ++i) xt[i + 1] = x[i + 1] + alpha * dx[i];
      double Ft = 0.0;
      if ((rc = evaluate(xt, false, Ft)) != XY_OK) return rc;
      if (Ft <= F + 1e-4 * alpha * slope || step * alpha <= tol) {
        moved = true;
        break;
      }
      alpha *= 0.5;
    }
    if (!moved) break;
    x = xt;
    converged = step * alpha <= tol;
  }
  for (int m = 0; m < R; ++m) f[m] = x[m];
  if (iters_out) *iters_out = it;
  return converged ? XY_OK : XY_ERR_TIMEOUT;
}

int xy_multihist_forward(int64_t T, const double* d_E, const float* d_m2, const float* d_m4, const float* d_c,
                         const float* d_s2, int R, const double* betas, const int64_t* counts, const double* f,
                         int K, const double* d_betap, int L, double* d_out, double* d_obs, double* d_cov,
                         void* d_scratch, size_t scratch_bytes, void* stream) {
  if (T < 1 || K < 1 || L < 1 || !d_E || !d_m2 || !d_m4 || !d_c || !d_s2 || !f || !d_betap || !d_out || !d_obs ||
      !d_cov || !d_scratch)
    return XY_ERR_ARG;
  if (!valid_ladder(R, betas, counts, T)) return XY_ERR_ARG;
  for (int m = 0; m < R; ++m)
    if (!std::isfinite(f[m])) return XY_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_scratch) % 256 != 0) return XY_ERR_ARG;
  const Plan p = plan_for(T, R, K);
  if (scratch_bytes < p.total) return XY_ERR_NOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_scratch);
  double* logD = reinterpret_cast<double*>(ws + p.off_logD);
  double* coef = reinterpret_cast<double*>(ws + p.off_coef);
  double* mpart = reinterpret_cast<double*>(ws + p.off_max);
  double* kmax = reinterpret_cast<double*>(ws + p.off_kmax);
  double* stats = reinterpret_cast<double*>(ws + p.off_stats);
  double* sums = reinterpret_cast<double*>(ws + p.off_sums);
  std::vector<double> h_coef(2 * R);
  for (int m = 0; m < R; ++m) {
    h_coef[m] = std::log(static_cast<double>(counts[m])) + (f[m] - f[0]);
    h_coef[R + m] = betas[m];
  }
  if (cudaMemcpyAsync(coef, h_coef.data(), 2 * R * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) return XY_ERR_CUDA;
  k_mh_logD<<<p.n_tblocks, kBlock, 0, st>>>(T, d_E, R, coef, logD);
  k_mh_mean<<<1, kBlock, 0, st>>>(T, d_E, stats);
  k_mh_max<<<p.n_tblocks, kBlock, 0, st>>>(T, d_E, logD, K, d_betap, mpart);
  k_mh_max_finish<<<(K + 127) / 128, 128, 0, st>>>(K, p.n_tblocks, mpart, kmax);
  k_mh_sums<<<dim3(p.n_kblocks, p.n_tchunks), kBlock, 0, st>>>(T, p.t_per_chunk, d_E, logD, d_m2, d_m4, d_c, d_s2, K,
                                                                  d_betap, kmax, stats, sums);
  k_mh_finish<<<(K + 127) / 128, 128, 0, st>>>(K, p.n_tchunks, d_betap, L, kmax, stats, sums, d_out, d_obs, d_cov);
  return cudaGetLastError() == cudaSuccess ? XY_OK : XY_ERR_CUDA;
}

}  // extern "C"
