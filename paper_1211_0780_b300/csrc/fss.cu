// Finite-size-scaling analysis on the device (Sec. III): resampled
// reweighted curves of the Binder cumulant U_L (Eq. 5) and of rho_s L
// (Eq. 6, scaled by L), their beta' derivatives, and the crossings of two
// sizes' curves with the slopes there, from which 1/nu follows.
//
// Inputs are the per-bin reweighting sums of xy_reweight_bins: for each bin
// b, target coupling k and j in {1, e, e^2, m2, m2 e, m4, m4 e, c, c e, s2,
// s2 e}, S[b][k][j] = sum over the bin's samples of w_kt x_j with a weight
// shift common to all bins.  A resample (bootstrap: bins drawn with
// replacement, Sec. III; jackknife: all bins but one) is a vector of bin
// multiplicities; its sums are the multiplicity-weighted sums of the bins'.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/xy.h"

namespace {

constexpr int kNSum = 11;

// out[r][q] = sum_b counts[r][b] S[b][q], q = (k, j), bins in order.
__global__ void k_fss_resample(int n_bins, int64_t nq, const double* __restrict__ bins,
                               const int32_t* __restrict__ counts, double* __restrict__ out) {
  extern __shared__ double s_cnt[];
  const int r = blockIdx.y;
  for (int b = threadIdx.x; b < n_bins; b += blockDim.x)
    s_cnt[b] = static_cast<double>(counts[static_cast<int64_t>(r) * n_bins + b]);
  __syncthreads();
  const int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (q >= nq) return;
  double v = 0.0;
  for (int b = 0; b < n_bins; ++b) v = fma(s_cnt[b], bins[static_cast<int64_t>(b) * nq + q], v);
  out[static_cast<int64_t>(r) * nq + q] = v;
}

// U_L = 1 - <m4> / (3 <m2>^2) (Eq. 5) and rho_s L = (L/3)(<c> - beta' <s2>)
// (Eq. 6 with c, s2 the bond sums per site), and their beta' derivatives
// from d<O>/dbeta' = -(<O e> - <O><e>), for every (resample, k).
__global__ void k_fss_curves(int B, int K, const double* __restrict__ betap, double L,
                             const double* __restrict__ sums, double* __restrict__ curves) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<int64_t>(B) * K) return;
  const int r = static_cast<int>(i / K), k = static_cast<int>(i - static_cast<int64_t>(r) * K);
  const double* S = sums + i * kNSum;
  const double inv = 1.0 / S[0];
  const double me = S[1] * inv, mm2 = S[3] * inv, mm4 = S[5] * inv, mc = S[7] * inv, ms2 = S[9] * inv;
  const double d2 = -(S[4] * inv - mm2 * me), d4 = -(S[6] * inv - mm4 * me);
  const double dc = -(S[8] * inv - mc * me), ds2 = -(S[10] * inv - ms2 * me);
  const double bp = betap[k];
  double* out = curves + static_cast<int64_t>(r) * 4 * K;
  out[k] = 1.0 - mm4 / (3.0 * mm2 * mm2);
  out[K + k] = L / 3.0 * (mc - bp * ms2);
  out[2 * K + k] = -(d4 / (3.0 * mm2 * mm2) - 2.0 * mm4 * d2 / (3.0 * mm2 * mm2 * mm2));
  out[3 * K + k] = L / 3.0 * (dc - ms2 - bp * ds2);
}

// Cubic Hermite basis on [0, 1] and its derivative.
__device__ __forceinline__ double hermite(double t, double f0, double d0, double f1, double d1, double h) {
  const double t2 = t * t, t3 = t2 * t;
  return (2 * t3 - 3 * t2 + 1) * f0 + (t3 - 2 * t2 + t) * h * d0 + (-2 * t3 + 3 * t2) * f1 + (t3 - t2) * h * d1;
}
__device__ __forceinline__ double hermite_d(double t, double f0, double d0, double f1, double d1, double h) {
  const double t2 = t * t;
  return ((6 * t2 - 6 * t) * f0 + (3 * t2 - 4 * t + 1) * h * d0 + (-6 * t2 + 6 * t) * f1 + (3 * t2 - 2 * t) * h * d1) / h;
}

// Crossing of two sizes' curves (row `which` of each: 0 = U_L, 1 = rho_s L)
// for every resample, one warp per resample: the first k (ascending beta')
// where the difference g = A - B changes sign (lanes test 32 consecutive
// intervals at a time; a ballot picks the lowest), refined on the cubic
// Hermite interpolant of g (values and derivatives at both grid points) by
// bisection; the slopes of A and B there come from their own Hermite
// interpolants.  Since a dimensionless ratio Q scales as Q(t L^{1/nu}),
// dQ/dbeta at the crossing grows as L^{1/nu}: 1/nu = ln(|dB| / |dA|) /
// ln(L_B / L_A).  out[r] = {beta*, dA, dB, 1/nu, nu}; NaN when the curves
// do not cross.
__global__ void k_fss_crossings(int B, int K, const double* __restrict__ betap, double LA,
                                const double* __restrict__ curvesA, double LB, const double* __restrict__ curvesB,
                                int which, double* __restrict__ out) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= B) return;  // whole warps leave together
  const double* A = curvesA + static_cast<int64_t>(r) * 4 * K + which * K;
  const double* dA = curvesA + static_cast<int64_t>(r) * 4 * K + (2 + which) * K;
  const double* Bv = curvesB + static_cast<int64_t>(r) * 4 * K + which * K;
  const double* dB = curvesB + static_cast<int64_t>(r) * 4 * K + (2 + which) * K;
  double* o = out + static_cast<int64_t>(r) * 5;
  int found = -1;
  for (int k0 = 0; k0 + 1 < K && found < 0; k0 += 32) {
    const int k = k0 + lane;
    bool hit = false;
    if (k + 1 < K) {
      const double g0 = A[k] - Bv[k], g1 = A[k + 1] - Bv[k + 1];
      // NaN (an empty resample) never brackets; g1 == 0 is the next interval's
      hit = g0 == g0 && g1 == g1 && g1 != 0.0 && (g0 == 0.0 || (g0 < 0.0) != (g1 < 0.0));
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (m) found = k0 + __ffs(m) - 1;
  }
  if (lane != 0) return;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  if (found < 0) {
    o[0] = o[1] = o[2] = o[3] = o[4] = nan;
    return;
  }
  const int k = found;
  const double g0 = A[k] - Bv[k], g1 = A[k + 1] - Bv[k + 1];
  const double h = betap[k + 1] - betap[k];
  const double dg0 = dA[k] - dB[k], dg1 = dA[k + 1] - dB[k + 1];
  double lo = 0.0, hi = 1.0;
  if (g0 != 0.0) {
    const bool neg0 = g0 < 0.0;
    for (int it = 0; it < 64; ++it) {
      const double mid = 0.5 * (lo + hi);
      const double gm = hermite(mid, g0, dg0, g1, dg1, h);
      if ((gm < 0.0) == neg0) lo = mid;
      else hi = mid;
    }
  } else {
    hi = 0.0;
  }
  const double t = 0.5 * (lo + hi);
  const double sA = hermite_d(t, A[k], dA[k], A[k + 1], dA[k + 1], h);
  const double sB = hermite_d(t, Bv[k], dB[k], Bv[k + 1], dB[k + 1], h);
  const double inv_nu = log(fabs(sB) / fabs(sA)) / log(LB / LA);
  o[0] = betap[k] + t * h;
  o[1] = sA;
  o[2] = sB;
  o[3] = inv_nu;
  o[4] = 1.0 / inv_nu;
}

int launch_status() { return cudaGetLastError() == cudaSuccess ? XY_OK : XY_ERR_CUDA; }

}  // namespace

extern "C" {

int xy_fss_resample(int n_bins, int K, const double* d_binsums, int B, const int32_t* d_counts, double* d_sums,
                    void* stream) {
  if (n_bins < 1 || K < 1 || B < 1 || B > 65535 || !d_binsums || !d_counts || !d_sums) return XY_ERR_ARG;
  if (n_bins > 6144) return XY_ERR_ARG;  // multiplicities staged in 48 KB of shared memory
  const int64_t nq = static_cast<int64_t>(K) * kNSum;
  k_fss_resample<<<dim3(static_cast<unsigned>((nq + 255) / 256), B), 256, n_bins * sizeof(double),
                   static_cast<cudaStream_t>(stream)>>>(n_bins, nq, d_binsums, d_counts, d_sums);
  return launch_status();
}

int xy_fss_curves(int B, int K, const double* d_betap, int L, const double* d_sums, double* d_curves, void* stream) {
  if (B < 1 || K < 1 || L < 1 || !d_betap || !d_sums || !d_curves) return XY_ERR_ARG;
  const int64_t n = static_cast<int64_t>(B) * K;
  k_fss_curves<<<static_cast<unsigned>((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      B, K, d_betap, static_cast<double>(L), d_sums, d_curves);
  return launch_status();
}

int xy_fss_crossings(int B, int K, const double* d_betap, int LA, const double* d_curvesA, int LB,
                     const double* d_curvesB, int which, double* d_out, void* stream) {
  if (B < 1 || K < 2 || LA < 1 || LB < 1 || LA == LB || (which != 0 && which != 1)) return XY_ERR_ARG;
  if (!d_betap || !d_curvesA || !d_curvesB || !d_out) return XY_ERR_ARG;
  k_fss_crossings<<<(B + 3) / 4, 128, 0, static_cast<cudaStream_t>(stream)>>>(
      B, K, d_betap, static_cast<double>(LA), d_curvesA, static_cast<double>(LB), d_curvesB, which, d_out);
  return launch_status();
}

}  // extern "C"
