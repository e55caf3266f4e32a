// Single-histogram reweighting of a measured series to K target couplings,
// forward and backward, all FP64 (the method is Ferrenberg-Swendsen's; the
// paper bins its series on the host instead, Sec. II).
//
// For samples t with energy E_t and observables O_t measured at beta0, and
// Delta_k = beta'_k - beta0:
//   w_kt = exp(-Delta_k (e_t - e_ref)),   e_t = E_t - Ebar (centred),
//   S_k[O] = sum_t w_kt O_t,   <O>_k = S_k[O] / S_k[1],
//   log Z_k = log S_k[1] - Delta_k (e_ref + Ebar),
//   cov_k(O, E) = S_k[O e] / S_k[1] - <O>_k <e>_k.
// e_ref = min_t e_t for Delta >= 0 and max_t e_t otherwise, so every
// exponent is <= 0 (the log-sum-exp shift, known in closed form from the
// extremes of the series).
//
// Work split.  Pass 1 reduces (sum E, min E, max E) in a fixed order and
// takes the grid step (beta'_K-1 - beta'_0) / (K - 1).  Pass 2: a block owns
// 4 * blockDim.x consecutive k and one chunk of t; each thread owns 4
// consecutive k.  It evaluates the weight of its first k exactly and, when
// its four couplings sit on the grid step (the usual linspace grid), steps
// to the next ones by multiplying with rho_t = exp(-step (e_t - e_ref)),
// whose sample-dependent factor exp(-step (e_t - e_mid)) the block
// evaluates once per staged sample in shared memory (one FP64 exp per four
// (k, t) pairs; relative error of the stepped weights <= 5 roundings).  The
// per-chunk partial sums go to scratch; pass 3 adds the chunks in chunk
// order (deterministic) and forms the outputs.  The FP64 pipe bounds pass 2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/xy.h"

namespace {

constexpr int kKT = 4;          // couplings per thread
constexpr int kBlock = 256;     // threads per block in pass 2
constexpr int kChunk = 256;     // samples staged in shared memory at a time
constexpr int kNSum = 11;       // 1, e, e^2, m2, m2 e, m4, m4 e, c, c e, s2, s2 e
constexpr int kStatBlocks = 256;
// Pass-2 grids are sized in whole waves of B300's 148 SMs: one 256-thread
// block of the sums kernel fits per SM (178 registers a thread), so a grid
// of 4 x 148 blocks runs as four full waves with no partial last wave.
constexpr int kWaveBlocks = 4 * 148;

// Chunks per bin (1..8) whose grid n_kblocks * n_bins * c fills its last
// wave of 148 blocks best (the smallest on ties).
int chunks_for_waves(int64_t n_kblocks, int64_t n_bins, int64_t max_c) {
  int best = 1;
  double best_eff = 0.0;
  for (int c = 1; c <= 8 && c <= max_c; ++c) {
    const double waves = static_cast<double>(n_kblocks * n_bins * c) / 148.0;
    const double eff = waves / std::ceil(waves);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = c;
    }
  }
  return best;
}

struct Plan {
  int n_kblocks, n_tchunks;
  int64_t t_per_chunk;
  size_t off_stat_part, off_stats, off_sums, total;
};

Plan plan_for(int64_t T, int K) {
  Plan p{};
  p.n_kblocks = (K + kKT * kBlock - 1) / (kKT * kBlock);
  const int64_t want = std::max<int64_t>(1, kWaveBlocks / p.n_kblocks);
  p.n_tchunks = static_cast<int>(std::min<int64_t>(want, (T + kChunk - 1) / kChunk));
  p.t_per_chunk = (T + p.n_tchunks - 1) / p.n_tchunks;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t at = off;
    off = (off + b + 255) / 256 * 256;
    return at;
  };
  p.off_stat_part = take(static_cast<size_t>(kStatBlocks) * 3 * 8);
  p.off_stats = take(4 * 8);
  p.off_sums = take(static_cast<size_t>(p.n_tchunks) * K * kNSum * 8);
  p.total = off;
  return p;
}

__device__ __forceinline__ double dmin(double a, double b) { return a < b ? a : b; }
__device__ __forceinline__ double dmax(double a, double b) { return a > b ? a : b; }

// Pass 1a: per-block (sum, min, max) of E in a fixed order.
__global__ void k_rw_stats(int64_t T, const double* __restrict__ E, double* part) {
  __shared__ double s_sum[kBlock], s_min[kBlock], s_max[kBlock];
  double sum = 0.0, mn = INFINITY, mx = -INFINITY;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < T;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double e = E[t];
    sum += e;
    mn = dmin(mn, e);
    mx = dmax(mx, e);
  }
  s_sum[threadIdx.x] = sum;
  s_min[threadIdx.x] = mn;
  s_max[threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_sum[threadIdx.x] += s_sum[threadIdx.x + w];
      s_min[threadIdx.x] = dmin(s_min[threadIdx.x], s_min[threadIdx.x + w]);
      s_max[threadIdx.x] = dmax(s_max[threadIdx.x], s_max[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = s_sum[0];
    part[3 * blockIdx.x + 1] = s_min[0];
    part[3 * blockIdx.x + 2] = s_max[0];
  }
}

// Pass 1b: stats = {Ebar, e_min, e_max, grid step} with e = E - Ebar and
// grid step = (beta'_K-1 - beta'_0) / (K - 1) (0 for K = 1).
__global__ void k_rw_stats_finish(int64_t T, int nblk, const double* part, int K, const double* betap,
                                  double* stats) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double sum = 0.0, mn = INFINITY, mx = -INFINITY;
  for (int b = 0; b < nblk; ++b) {
    sum += part[3 * b];
    mn = dmin(mn, part[3 * b + 1]);
    mx = dmax(mx, part[3 * b + 2]);
  }
  const double mean = sum / static_cast<double>(T);
  stats[0] = mean;
  stats[1] = mn - mean;
  stats[2] = mx - mean;
  stats[3] = K > 1 ? (betap[K - 1] - betap[0]) / (K - 1) : 0.0;
}

// Sample range of chunk `chunk`: uniform chunks of t_per_chunk samples, or,
// with n_bins > 0, chunks_per_bin chunks inside each of n_bins equal bins
// (bin b = samples [b T / n_bins, (b + 1) T / n_bins)), so that no chunk
// straddles two bins.
__device__ __forceinline__ void chunk_range(int chunk, int64_t T, int64_t t_per_chunk, int n_bins,
                                            int chunks_per_bin, int64_t& t0, int64_t& t1) {
  if (n_bins <= 0) {
    t0 = chunk * t_per_chunk;
    t1 = (t0 + t_per_chunk < T) ? t0 + t_per_chunk : T;
    return;
  }
  const int b = chunk / chunks_per_bin, j = chunk - b * chunks_per_bin;
  const int64_t b0 = T * b / n_bins, b1 = T * (b + 1) / n_bins;
  const int64_t per = (b1 - b0 + chunks_per_bin - 1) / chunks_per_bin;
  t0 = b0 + j * per;
  t0 = t0 < b1 ? t0 : b1;
  t1 = (t0 + per < b1) ? t0 + per : b1;
}

// Pass 2: chunk partial sums S[chunk][k][kNSum].
__global__ void __launch_bounds__(kBlock) k_rw_sums(int64_t T, int64_t t_per_chunk, int n_bins, int chunks_per_bin,
                                                    const double* __restrict__ E, const float* __restrict__ m2,
                                                    const float* __restrict__ m4, const float* __restrict__ c,
                                                    const float* __restrict__ s2, double beta0, int K,
                                                    const double* __restrict__ betap, const double* __restrict__ stats,
                                                    double* __restrict__ sums) {
  // the sample's observables and their products with e, staged once per
  // block so that every accumulation below is one fused multiply-add by w
  __shared__ double s_e[kChunk], s_m2[kChunk], s_m4[kChunk], s_c[kChunk], s_s2[kChunk], s_rho[kChunk];
  __shared__ double s_ee[kChunk], s_em2[kChunk], s_em4[kChunk], s_ec[kChunk], s_es2[kChunk];
  const int chunk = blockIdx.y;
  int64_t t0, t1;
  chunk_range(chunk, T, t_per_chunk, n_bins, chunks_per_bin, t0, t1);
  const int k0 = (blockIdx.x * blockDim.x + threadIdx.x) * kKT;
  const double Ebar = stats[0], emin = stats[1], emax = stats[2], gstep = stats[3];
  const double emid = 0.5 * (emin + emax);

  double d[kKT];
  int nk = 0;
#pragma unroll
  for (int i = 0; i < kKT; ++i) {
    const int k = k0 + i;
    d[i] = (k < K) ? betap[k] - beta0 : 0.0;
    nk += (k < K) ? 1 : 0;
  }
  const double eref = d[0] >= 0.0 ? emin : emax;
  // Even spacing of this thread's couplings (to rounding) at the grid's
  // step allows stepping: w_{i+1} = w_i rho_t with rho_t = exp(-step (e_t -
  // eref)) = exp(-step (e_t - emid)) exp(-step (emid - eref)); the first
  // factor is the same for every thread, so the block evaluates it once per
  // sample into shared memory, and each thread multiplies by its constant.
  const double step = gstep;
  bool even = nk > 1 && step != 0.0;
#pragma unroll
  for (int i = 1; i < kKT; ++i)
    if (i < nk)  // a few ulps of the couplings themselves (grids from linspace round to them)
      even = even && fabs(d[i] - (d[0] + i * step)) <= 8.0 * 2.220446049250313e-16 * (fabs(beta0) + fabs(d[i]));
  const double rho_c = even ? exp(-step * (emid - eref)) : 0.0;
  // Stepping from a coupling whose shift differs in sign is also fine: the
  // exponent stays bounded by |step| * kKT * (emax - emin).

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
      s_e[j] = E[t] - Ebar;
      s_m2[j] = static_cast<double>(m2[t]);
      s_m4[j] = static_cast<double>(m4[t]);
      s_c[j] = static_cast<double>(c[t]) + static_cast<double>(c[T + t]) + static_cast<double>(c[2 * T + t]);
      s_s2[j] = static_cast<double>(s2[t]) + static_cast<double>(s2[T + t]) + static_cast<double>(s2[2 * T + t]);
      s_rho[j] = exp(-step * (s_e[j] - emid));
      s_ee[j] = s_e[j] * s_e[j];
      s_em2[j] = s_e[j] * s_m2[j];
      s_em4[j] = s_e[j] * s_m4[j];
      s_ec[j] = s_e[j] * s_c[j];
      s_es2[j] = s_e[j] * s_s2[j];
    }
    __syncthreads();
    if (nk > 0) {
      for (int j = 0; j < n; ++j) {
        const double e = s_e[j], x2 = s_m2[j], x4 = s_m4[j], xc = s_c[j], xs = s_s2[j];
        const double ee = s_ee[j], ex2 = s_em2[j], ex4 = s_em4[j], exc = s_ec[j], exs = s_es2[j];
        const double de = e - eref;
        double w = exp(-d[0] * de);
        const double rho = even ? s_rho[j] * rho_c : 0.0;
#pragma unroll
        for (int i = 0; i < kKT; ++i) {
          if (i > 0) w = even ? w * rho : exp(-d[i] * de);
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
  for (int i = 0; i < kKT; ++i) {
    if (i < nk) {
      double* dst = sums + (static_cast<int64_t>(chunk) * K + k0 + i) * kNSum;
#pragma unroll
      for (int j = 0; j < kNSum; ++j) dst[j] = S[i][j];
    }
  }
}

// Pass 3: chunk sums in chunk order, then the outputs of each k.
__global__ void k_rw_finish(int K, int n_tchunks, double beta0, const double* __restrict__ betap, int L,
                            const double* __restrict__ stats, const double* __restrict__ sums, double* out,
                            double* obs, double* cov) {
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
  const double Ebar = stats[0];
  const double bp = betap[k];
  const double dk = bp - beta0;
  // The shift reference of pass 2 is that of the thread group's first k.
  const double d0 = betap[(k / kKT) * kKT] - beta0;
  const double eref = d0 >= 0.0 ? stats[1] : stats[2];
  const double inv = 1.0 / S[0];
  const double me = S[1] * inv;
  const double mm2 = S[3] * inv, mm4 = S[5] * inv, mc = S[7] * inv, ms2 = S[9] * inv;
  out[0 * K + k] = log(S[0]) - dk * (eref + Ebar);
  out[1 * K + k] = Ebar + me;
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
  obs[2 * K + k] = mm4 / (mm2 * mm2);  // q2 of Eq. (11) = 3 (1 - U_L)
}

// Backward: d<O>/dbeta' = -cov(O, E), chain rule to U_L and rho_s L.
__global__ void k_rw_backward(int K, const double* __restrict__ betap, int L, const double* __restrict__ out,
                              const double* __restrict__ cov, const double* __restrict__ gU,
                              const double* __restrict__ gR, double* grad, double* dobs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double mm2 = out[2 * K + k], mm4 = out[3 * K + k], ms2 = out[5 * K + k];
  const double d2 = -cov[1 * K + k], d4 = -cov[2 * K + k], dc = -cov[3 * K + k], ds2 = -cov[4 * K + k];
  const double bp = betap[k];
  const double dU = -(d4 / (3.0 * mm2 * mm2) - 2.0 * mm4 * d2 / (3.0 * mm2 * mm2 * mm2));
  const double dR = L / 3.0 * (dc - ms2 - bp * ds2);
  if (dobs) {
    dobs[k] = dU;
    dobs[K + k] = dR;
    dobs[2 * K + k] = -3.0 * dU;  // d q2 / d beta', q2 = 3 (1 - U_L)
  }
  if (grad) grad[k] = (gU ? gU[k] * dU : 0.0) + (gR ? gR[k] * dR : 0.0);
}

thread_local char g_rw_err[160];

}  // namespace

extern "C" {

size_t xy_reweight_scratch_bytes(int64_t T, int K) {
  if (T < 2 || K < 1) return 0;
  return plan_for(T, K).total;
}

int xy_reweight_forward(int64_t T, const double* d_E, const float* d_m2, const float* d_m4, const float* d_c,
                        const float* d_s2, double beta0, int K, const double* d_betap, int L, double* d_out,
                        double* d_obs, double* d_cov, void* d_scratch, size_t scratch_bytes, void* stream) {
  if (T < 2 || K < 1 || L < 1 || !std::isfinite(beta0)) return XY_ERR_ARG;
  if (!d_E || !d_m2 || !d_m4 || !d_c || !d_s2 || !d_betap || !d_out || !d_obs || !d_cov || !d_scratch)
    return XY_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_scratch) % 256 != 0) return XY_ERR_ARG;
  const Plan p = plan_for(T, K);
  if (scratch_bytes < p.total) return XY_ERR_NOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_scratch);
  double* part = reinterpret_cast<double*>(ws + p.off_stat_part);
  double* stats = reinterpret_cast<double*>(ws + p.off_stats);
  double* sums = reinterpret_cast<double*>(ws + p.off_sums);
  k_rw_stats<<<kStatBlocks, kBlock, 0, st>>>(T, d_E, part);
  k_rw_stats_finish<<<1, 32, 0, st>>>(T, kStatBlocks, part, K, d_betap, stats);
  k_rw_sums<<<dim3(p.n_kblocks, p.n_tchunks), kBlock, 0, st>>>(T, p.t_per_chunk, 0, 1, d_E, d_m2, d_m4, d_c, d_s2,
                                                                  beta0, K, d_betap, stats, sums);
  k_rw_finish<<<(K + 127) / 128, 128, 0, st>>>(K, p.n_tchunks, beta0, d_betap, L, stats, sums, d_out, d_obs, d_cov);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_rw_err, sizeof g_rw_err, "%s", cudaGetErrorString(e));
    return XY_ERR_CUDA;
  }
  return XY_OK;
}

int xy_reweight_backward(int K, const double* d_betap, int L, const double* d_out, const double* d_cov,
                         const double* d_gU, const double* d_grhoL, double* d_grad_betap, double* d_dobs,
                         void* stream) {
  if (K < 1 || L < 1 || !d_betap || !d_out || !d_cov || (!d_grad_betap && !d_dobs)) return XY_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_rw_backward<<<(K + 127) / 128, 128, 0, st>>>(K, d_betap, L, d_out, d_cov, d_gU, d_grhoL, d_grad_betap, d_dobs);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? XY_OK : XY_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of the reweighting forward pass.
//
// Some callers cannot hand the library a scratch buffer: code that runs with a
// fixed device-memory budget decided up front, code that must not call the
// CUDA allocator (or a framework's caching allocator) between set-up and
// shutdown, and plugins hosted by a framework that owns all device
// allocations.  For them the forward pass can run out of one file-scope
// device array of a fixed size that every GPU loading this library holds
// until the process exits.
//
// The kernels are the same as xy_reweight_forward's; only the number of
// sample chunks is capped so that the per-chunk partial sums fit the array.
// Every scratch word the kernels read is written earlier in the same call,
// so nothing needs clearing between calls.  All calls share the one array:
// calls that overlap on the GPU (other streams, other host threads) race.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB per device
static __device__ __align__(256) unsigned char g_rw_static_scratch[kStaticScratchBytes];

// Device address of g_rw_static_scratch per device, looked up once with that
// device current (in host code the array's name is only a host-side handle).
std::mutex g_static_mu;
void* g_static_addr[64] = {nullptr};

int static_scratch_address(int device, void** out) {
  if (device < 0 || device >= 64) return XY_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_rw_static_scratch);
    if (e != cudaSuccess || !p) {
      snprintf(g_rw_err, sizeof g_rw_err, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return XY_ERR_CUDA;
    }
    g_static_addr[device] = p;
  }
  *out = g_static_addr[device];
  return XY_OK;
}

// Layout inside the array: stat partials, stats, then n_tchunks x K x kNSum
// chunk sums.
constexpr size_t kStaticOffStats = (static_cast<size_t>(kStatBlocks) * 3 * 8 + 255) / 256 * 256;
constexpr size_t kStaticOffSums = kStaticOffStats + 256;

// The forward pass on `device` (current) out of the static array.
int forward_on_static_scratch(int64_t T, const double* d_E, const float* d_m2, const float* d_m4, const float* d_c,
                              const float* d_s2, double beta0, int K, const double* d_betap, int L, double* d_out,
                              double* d_obs, double* d_cov, const Plan& p, int device, cudaStream_t st) {
  void* base = nullptr;
  const int rc = static_scratch_address(device, &base);
  if (rc != XY_OK) return rc;
  char* ws = static_cast<char*>(base);
  double* part = reinterpret_cast<double*>(ws);
  double* stats = reinterpret_cast<double*>(ws + kStaticOffStats);
  double* sums = reinterpret_cast<double*>(ws + kStaticOffSums);
  k_rw_stats<<<kStatBlocks, kBlock, 0, st>>>(T, d_E, part);
  k_rw_stats_finish<<<1, 32, 0, st>>>(T, kStatBlocks, part, K, d_betap, stats);
  k_rw_sums<<<dim3(p.n_kblocks, p.n_tchunks), kBlock, 0, st>>>(T, p.t_per_chunk, 0, 1, d_E, d_m2, d_m4, d_c, d_s2,
                                                                  beta0, K, d_betap, stats, sums);
  k_rw_finish<<<(K + 127) / 128, 128, 0, st>>>(K, p.n_tchunks, beta0, d_betap, L, stats, sums, d_out, d_obs, d_cov);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_rw_err, sizeof g_rw_err, "%s", cudaGetErrorString(e));
    return XY_ERR_CUDA;
  }
  return XY_OK;
}

}  // namespace

extern "C" {

size_t xy_reweight_noalloc_capacity_bytes(void) { return kStaticScratchBytes; }

int xy_reweight_forward_noalloc(int64_t T, const double* d_E, const float* d_m2, const float* d_m4,
                                const float* d_c, const float* d_s2, double beta0, int K,
                                const double* d_betap, int L, double* d_out, double* d_obs, double* d_cov,
                                void* stream) {
  if (T < 2 || K < 1 || L < 1 || !std::isfinite(beta0)) return XY_ERR_ARG;
  if (!d_E || !d_m2 || !d_m4 || !d_c || !d_s2 || !d_betap || !d_out || !d_obs || !d_cov) return XY_ERR_ARG;
  const size_t per_chunk = static_cast<size_t>(K) * kNSum * 8;
  if (kStaticOffSums + per_chunk > kStaticScratchBytes) return XY_ERR_NOMEM;  // K too large
  Plan p = plan_for(T, K);
  const int cap = static_cast<int>((kStaticScratchBytes - kStaticOffSums) / per_chunk);
  if (p.n_tchunks > cap) {
    p.n_tchunks = cap;
    p.t_per_chunk = (T + cap - 1) / cap;
  }
  // The device of the outputs (device or managed memory) is the device to
  // run on; the first call on a device looks the array's address up (do it
  // before any stream capture).  The caller's current device is restored
  // before returning.
  cudaPointerAttributes pa{};
  const cudaError_t e = cudaPointerGetAttributes(&pa, d_out);
  if (e != cudaSuccess || (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device < 0) {
    cudaGetLastError();
    return XY_ERR_ARG;
  }
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || (prev != pa.device && cudaSetDevice(pa.device) != cudaSuccess)) {
    snprintf(g_rw_err, sizeof g_rw_err, "%s", cudaGetErrorString(cudaGetLastError()));
    return XY_ERR_CUDA;
  }
  const int rc = forward_on_static_scratch(T, d_E, d_m2, d_m4, d_c, d_s2, beta0, K, d_betap, L, d_out, d_obs, d_cov,
                                           p, pa.device, static_cast<cudaStream_t>(stream));
  if (prev != pa.device) cudaSetDevice(prev);
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Per-bin reweighting sums, for error analysis by resampling whole bins.
//
// The series is cut into n_bins equal contiguous bins (the paper bins its
// measurements before any analysis, Sec. II).  The pass-2 chunks are laid
// out inside the bins, and pass 3 adds each bin's chunks in order, giving
// S[b][k][j] for every bin b with the same shift per k for all bins: bin
// sums add, so the sums of any multiset of bins (a bootstrap or jackknife
// resample) are a weighted sum of these, and any ratio of them is a
// reweighted average of that resample.
// ---------------------------------------------------------------------------

namespace {

struct BinPlan {
  int n_kblocks, chunks_per_bin, n_tchunks;
  size_t off_stat_part, off_stats, off_sums, total;
};

BinPlan bin_plan_for(int64_t T, int K, int n_bins) {
  BinPlan p{};
  p.n_kblocks = (K + kKT * kBlock - 1) / (kKT * kBlock);
  const int64_t per_bin = T / n_bins + 1;
  p.chunks_per_bin = chunks_for_waves(p.n_kblocks, n_bins, (per_bin + kChunk - 1) / kChunk);
  p.n_tchunks = p.chunks_per_bin * n_bins;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t at = off;
    off = (off + b + 255) / 256 * 256;
    return at;
  };
  p.off_stat_part = take(static_cast<size_t>(kStatBlocks) * 3 * 8);
  p.off_stats = take(4 * 8);
  p.off_sums = take(static_cast<size_t>(p.n_tchunks) * K * kNSum * 8);
  p.total = off;
  return p;
}

// S[b][k][j] = sum of the chunk partials of bin b in chunk order.
__global__ void k_rw_bin_sums(int n_bins, int chunks_per_bin, int K, const double* __restrict__ sums,
                              double* __restrict__ bins) {
  const int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;  // (k, j)
  const int b = blockIdx.y;
  if (q >= static_cast<int64_t>(K) * kNSum) return;
  double v = 0.0;
  for (int ch = 0; ch < chunks_per_bin; ++ch)
    v += sums[(static_cast<int64_t>(b) * chunks_per_bin + ch) * K * kNSum + q];
  bins[static_cast<int64_t>(b) * K * kNSum + q] = v;
}

}  // namespace

extern "C" {

size_t xy_reweight_bins_scratch_bytes(int64_t T, int K, int n_bins) {
  if (T < 2 || K < 1 || n_bins < 1 || n_bins > T || n_bins > 65535) return 0;
  return bin_plan_for(T, K, n_bins).total;
}

int xy_reweight_bins(int64_t T, const double* d_E, const float* d_m2, const float* d_m4, const float* d_c,
                     const float* d_s2, double beta0, int K, const double* d_betap, int n_bins, double* d_binsums,
                     double* d_stats, void* d_scratch, size_t scratch_bytes, void* stream) {
  if (T < 2 || K < 1 || n_bins < 1 || n_bins > T || n_bins > 65535 || !std::isfinite(beta0)) return XY_ERR_ARG;
  if (!d_E || !d_m2 || !d_m4 || !d_c || !d_s2 || !d_betap || !d_binsums || !d_scratch) return XY_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_scratch) % 256 != 0) return XY_ERR_ARG;
  const BinPlan p = bin_plan_for(T, K, n_bins);
  if (scratch_bytes < p.total) return XY_ERR_NOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_scratch);
  double* part = reinterpret_cast<double*>(ws + p.off_stat_part);
  double* stats = reinterpret_cast<double*>(ws + p.off_stats);
  double* sums = reinterpret_cast<double*>(ws + p.off_sums);
  k_rw_stats<<<kStatBlocks, kBlock, 0, st>>>(T, d_E, part);
  k_rw_stats_finish<<<1, 32, 0, st>>>(T, kStatBlocks, part, K, d_betap, stats);
  k_rw_sums<<<dim3(p.n_kblocks, p.n_tchunks), kBlock, 0, st>>>(T, 0, n_bins, p.chunks_per_bin, d_E, d_m2, d_m4, d_c,
                                                                  d_s2, beta0, K, d_betap, stats, sums);
  const int64_t nq = static_cast<int64_t>(K) * kNSum;
  k_rw_bin_sums<<<dim3(static_cast<unsigned>((nq + 255) / 256), n_bins), 256, 0, st>>>(n_bins, p.chunks_per_bin, K,
                                                                                        sums, d_binsums);
  if (d_stats) {
    const cudaError_t ce = cudaMemcpyAsync(d_stats, stats, 3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (ce != cudaSuccess) return XY_ERR_CUDA;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_rw_err, sizeof g_rw_err, "%s", cudaGetErrorString(e));
    return XY_ERR_CUDA;
  }
  return XY_OK;
}

}  // extern "C"
