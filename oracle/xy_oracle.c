/*
 * Oracle for the 3D XY Monte Carlo hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU implementation of what the method computes, written
 * step by step from Lan, Hsieh & Kao, "High-precision Monte Carlo study of
 * the three-dimensional XY model on GPU" (arXiv:1211.0780):
 *   - the Hamiltonian H = -J sum_<ij> cos(theta_i - theta_j), J = 1,
 *     periodic boundaries (Sec. II, Eq. 1);
 *   - checkerboard Metropolis single-spin flips, all black sites then all
 *     white sites (Sec. II, Fig. 2);
 *   - microcanonical over-relaxation, S' = -S + 2 (S.H)/H^2 H with the local
 *     molecular field H = -sum_j S_j (Sec. II, Eq. 2);
 *   - the parallel-tempering swap W = min[1, exp((1/T_m - 1/T_n)(E_m - E_n))]
 *     (Sec. II, Eq. 3);
 *   - the lattice sums behind the estimators of m, U_L and rho_s
 *     (Sec. II, Eqs. 4-6);
 *   - single-histogram reweighting of a measured series to beta' (not in
 *     the paper: the standard Ferrenberg-Swendsen method).
 * Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11), implemented here
 * from that paper's definition.  The counter layout is the one fixed in the
 * library's header; this file shares no code with the CUDA library.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this code.  The product path never calls it.
 *
 * Lattice storage here is the natural one: theta[x + Lx*(y + Ly*z)].  An
 * extent of 1 along an axis means "no bonds along that axis" (used for the
 * Lx x 1 x 1 ring checks); other extents must be even so the two-colour
 * checkerboard is consistent under the periodic wrap.
 *
 * Readings of the paper where it is silent (fixed in writing before code):
 *   - proposal: theta' uniform in [0, 2pi), independent of theta;
 *   - accept iff u < exp(-beta dE) (strict); dE <= 0 therefore always
 *     accepts because u < 1;
 *   - sweep order: colour 0 ("black", (x+y+z) even) then colour 1;
 *   - over-relaxation is also a checkerboard pass; H = 0 leaves the spin;
 *   - angles are wrapped into [0, 2pi); a value that rounds to 2pi is 0;
 *   - swaps alternate even/odd pairs of the beta-sorted ladder and exchange
 *     the beta labels (a permutation), not the configurations.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define XO_TAG_INIT 1u
#define XO_TAG_MET 2u
#define XO_TAG_PT 3u

static const double XO_TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 3.3).                          */
/* One round maps (c0,c1,c2,c3) with key (k0,k1) to                          */
/*   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),       */
/* and the key advances by the Weyl constants between rounds.               */
/* ------------------------------------------------------------------------ */
void xo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                      uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* 24-bit uniform in [0, 1): (w >> 8) * 2^-24, exact in FP64. */
double xo_u01(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* The two words a site draws.  Packed index p = (x >> 1) + (Lx/2)(y + Ly z)
 * numbers the sites of one colour; one Philox call serves the packed pair
 * (2q, 2q+1): the even site takes words 0 and 1, the odd site 2 and 3. */
static void site_words(uint64_t seed, uint32_t slot, uint32_t colour,
                       uint32_t tag, uint64_t count, uint32_t p, uint32_t *wa,
                       uint32_t *wb) {
  uint32_t ctr[4], key[2], w[4];
  ctr[0] = p >> 1;
  ctr[1] = (uint32_t)count;
  ctr[2] = (uint32_t)(count >> 32);
  ctr[3] = (slot << 4) | (colour << 3) | tag;
  key[0] = (uint32_t)seed;
  key[1] = (uint32_t)(seed >> 32);
  xo_philox4x32_10(ctr, key, w);
  if (p & 1u) {
    *wa = w[2];
    *wb = w[3];
  } else {
    *wa = w[0];
    *wb = w[1];
  }
}

/* Raw words for every site of one colour, natural-layout order of those
 * sites (x fastest); two words per site. */
void xo_draw_words(int Lx, int Ly, int Lz, uint64_t seed, uint32_t slot,
                   int colour, int tag, uint64_t count, uint32_t *out) {
  long n = 0;
  for (int z = 0; z < Lz; ++z)
    for (int y = 0; y < Ly; ++y)
      for (int x = 0; x < Lx; ++x) {
        if (((x + y + z) & 1) != colour) continue;
        uint32_t p = (uint32_t)((x >> 1) + (Lx / 2) * (y + Ly * z));
        site_words(seed, slot, (uint32_t)colour, (uint32_t)tag, count, p,
                   &out[2 * n], &out[2 * n + 1]);
        ++n;
      }
}

static inline long site(int Lx, int Ly, int x, int y, int z) {
  return (long)x + (long)Lx * ((long)y + (long)Ly * (long)z);
}

static inline int wrap(int a, int L) { return a < 0 ? a + L : (a >= L ? a - L : a); }

/* Sum of the neighbour spin vectors, sum_j (cos theta_j, sin theta_j), over
 * the up-to-6 nearest neighbours (axes of extent 1 carry no bonds). */
static void neighbour_sum(int Lx, int Ly, int Lz, const double *th, int x,
                          int y, int z, double *sx, double *sy) {
  double ax = 0.0, ay = 0.0;
  const int L[3] = {Lx, Ly, Lz};
  for (int mu = 0; mu < 3; ++mu) {
    if (L[mu] == 1) continue;
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      int c[3] = {x, y, z};
      c[mu] = wrap(c[mu] + sgn, L[mu]);
      double t = th[site(Lx, Ly, c[0], c[1], c[2])];
      ax += cos(t);
      ay += sin(t);
    }
  }
  *sx = ax;
  *sy = ay;
}

/* Initial state: theta = 2 pi u, u from the INIT stream (count 0). */
void xo_init_uniform(int Lx, int Ly, int Lz, uint64_t seed, uint32_t slot,
                     double *th) {
  for (int z = 0; z < Lz; ++z)
    for (int y = 0; y < Ly; ++y)
      for (int x = 0; x < Lx; ++x) {
        int colour = (x + y + z) & 1;
        uint32_t p = (uint32_t)((x >> 1) + (Lx / 2) * (y + Ly * z));
        uint32_t wa, wb;
        site_words(seed, slot, (uint32_t)colour, XO_TAG_INIT, 0, p, &wa, &wb);
        th[site(Lx, Ly, x, y, z)] = XO_TWO_PI * xo_u01(wa);
      }
}

/* One Metropolis half-sweep over the sites of `colour` (Sec. II, Fig. 2).
 * For each site: field h = sum_j S_j; proposal theta' = 2 pi u0;
 * dE = E' - E = -[h_x (cos theta' - cos theta) + h_y (sin theta' - sin theta)];
 * accept iff u1 < exp(-beta dE).  Same-colour sites share no bond, so the
 * in-place update is order independent.  `mpass` is the Metropolis-pass
 * counter placed in the Philox counter.  If `margin` is not NULL, the
 * accept margin |u1 - exp(-beta dE)| of every updated site is written at
 * its natural index.  Returns the number of accepted proposals. */
long xo_metropolis_half(int Lx, int Ly, int Lz, double *th, double beta,
                        uint64_t seed, uint32_t slot, uint64_t mpass,
                        int colour, double *margin) {
  long accepted = 0;
#pragma omp parallel for collapse(2) reduction(+ : accepted) schedule(static) \
    if ((long)Lx * Ly * Lz >= 32768)
  for (int z = 0; z < Lz; ++z)
    for (int y = 0; y < Ly; ++y)
      for (int x = 0; x < Lx; ++x) {
        if (((x + y + z) & 1) != colour) continue;
        long i = site(Lx, Ly, x, y, z);
        double hx, hy;
        neighbour_sum(Lx, Ly, Lz, th, x, y, z, &hx, &hy);
        uint32_t p = (uint32_t)((x >> 1) + (Lx / 2) * (y + Ly * z));
        uint32_t wprop, wacc;
        site_words(seed, slot, (uint32_t)colour, XO_TAG_MET, mpass, p, &wprop,
                   &wacc);
        double t_old = th[i];
        double t_new = XO_TWO_PI * xo_u01(wprop);
        double dE = -(hx * (cos(t_new) - cos(t_old)) +
                      hy * (sin(t_new) - sin(t_old)));
        double a = exp(-beta * dE);
        double u = xo_u01(wacc);
        if (margin) margin[i] = fabs(u - a);
        if (u < a) {
          th[i] = t_new;
          accepted += 1;
        }
      }
  return accepted;
}

/* One over-relaxation half-sweep over the sites of `colour`, Eq. (2) in its
 * vector form: H = -sum_j S_j, S' = -S + 2 (S.H)/H^2 H, then theta' =
 * atan2(S'_y, S'_x) wrapped into [0, 2pi).  H = 0 leaves the spin alone. */
void xo_overrelax_half(int Lx, int Ly, int Lz, double *th, int colour) {
#pragma omp parallel for collapse(2) schedule(static) \
    if ((long)Lx * Ly * Lz >= 32768)
  for (int z = 0; z < Lz; ++z)
    for (int y = 0; y < Ly; ++y)
      for (int x = 0; x < Lx; ++x) {
        if (((x + y + z) & 1) != colour) continue;
        long i = site(Lx, Ly, x, y, z);
        double sx, sy;
        neighbour_sum(Lx, Ly, Lz, th, x, y, z, &sx, &sy);
        double Hx = -sx, Hy = -sy;
        double H2 = Hx * Hx + Hy * Hy;
        if (H2 == 0.0) continue;
        double Sx = cos(th[i]), Sy = sin(th[i]);
        double d = Sx * Hx + Sy * Hy;
        double Spx = -Sx + 2.0 * d / H2 * Hx;
        double Spy = -Sy + 2.0 * d / H2 * Hy;
        double t = atan2(Spy, Spx);
        if (t < 0.0) t += XO_TWO_PI;
        if (t >= XO_TWO_PI) t = 0.0;
        th[i] = t;
      }
}

/* Lattice sums behind Eqs. (4)-(6).  out[0] = E = -sum_<ij> cos(theta_i -
 * theta_j); out[1..2] = (M_x, M_y) = sum_i (cos theta_i, sin theta_i);
 * out[3+mu] = C_mu = sum over bonds (i, i+mu) of cos(theta_i - theta_{i+mu});
 * out[6+mu] = S_mu = the same sum of sin(theta_i - theta_{i+mu}).  Each bond
 * is visited once, from its lower end i, with the orientation i -> i+mu. */
void xo_measure(int Lx, int Ly, int Lz, const double *th, double out[9]) {
  double Mx = 0.0, My = 0.0, C[3] = {0, 0, 0}, S[3] = {0, 0, 0};
  const int L[3] = {Lx, Ly, Lz};
  for (int z = 0; z < Lz; ++z)
    for (int y = 0; y < Ly; ++y)
      for (int x = 0; x < Lx; ++x) {
        double ti = th[site(Lx, Ly, x, y, z)];
        Mx += cos(ti);
        My += sin(ti);
        for (int mu = 0; mu < 3; ++mu) {
          if (L[mu] == 1) continue;
          int c[3] = {x, y, z};
          c[mu] = wrap(c[mu] + 1, L[mu]);
          double tj = th[site(Lx, Ly, c[0], c[1], c[2])];
          C[mu] += cos(ti - tj);
          S[mu] += sin(ti - tj);
        }
      }
  out[0] = -(C[0] + C[1] + C[2]);
  out[1] = Mx;
  out[2] = My;
  for (int mu = 0; mu < 3; ++mu) {
    out[3 + mu] = C[mu];
    out[6 + mu] = S[mu];
  }
}

/* A single-slot chain under the sweep schedule: per sweep, nM Metropolis
 * passes (black then white; the pass counter starts at mpass0 and advances
 * by one per pass), then nOR over-relaxation passes (black then white).
 * After every measure_every-th sweep the nine lattice sums of xo_measure
 * are appended to `series` (row-major [n_meas][9]).  Returns the number of
 * accepted Metropolis proposals. */
long xo_run_chain(int Lx, int Ly, int Lz, double *th, double beta,
                  uint64_t seed, uint32_t slot, uint64_t mpass0, int nM,
                  int nOR, int n_sweeps, int measure_every, double *series) {
  long accepted = 0;
  uint64_t mpass = mpass0;
  long m = 0;
  for (int s = 0; s < n_sweeps; ++s) {
    for (int i = 0; i < nM; ++i) {
      accepted += xo_metropolis_half(Lx, Ly, Lz, th, beta, seed, slot, mpass, 0, NULL);
      accepted += xo_metropolis_half(Lx, Ly, Lz, th, beta, seed, slot, mpass, 1, NULL);
      ++mpass;
    }
    for (int i = 0; i < nOR; ++i) {
      xo_overrelax_half(Lx, Ly, Lz, th, 0);
      xo_overrelax_half(Lx, Ly, Lz, th, 1);
    }
    if (measure_every > 0 && (s + 1) % measure_every == 0 && series) {
      xo_measure(Lx, Ly, Lz, th, &series[9 * m]);
      ++m;
    }
  }
  return accepted;
}

/* The Philox draw of one ladder pair: counter (k, sweep_lo, sweep_hi,
 * ladder << 4 | TAG_PT), word 0. */
double xo_pt_uniform(uint64_t seed, uint32_t ladder, uint64_t sweep, int k) {
  uint32_t ctr[4], key[2], w[4];
  ctr[0] = (uint32_t)k;
  ctr[1] = (uint32_t)sweep;
  ctr[2] = (uint32_t)(sweep >> 32);
  ctr[3] = (ladder << 4) | XO_TAG_PT;
  key[0] = (uint32_t)seed;
  key[1] = (uint32_t)(seed >> 32);
  xo_philox4x32_10(ctr, key, w);
  return xo_u01(w[0]);
}

/* Parallel-tempering exchange on one ladder, Eq. (3).  betas[k] ascending;
 * perm[k] = the replica slot (0..R-1 within the ladder) currently at
 * betas[k]; E[r] = total energy of slot r.  Pairs (k, k+1) with k of the
 * given parity are tried; the pair swaps its beta labels with probability
 * min[1, exp((beta_k - beta_{k+1}) (E_perm[k] - E_perm[k+1]))].  accepted[k]
 * (nullable) is set to 1 for each accepted pair, else 0.  Returns the
 * number of accepted swaps. */
int xo_pt_swap(int R, const double *betas, const double *E, int *perm,
               uint64_t seed, uint32_t ladder, uint64_t sweep, int parity,
               int *accepted) {
  int n = 0;
  if (accepted)
    for (int k = 0; k < R; ++k) accepted[k] = 0;
  for (int k = parity & 1; k + 1 < R; k += 2) {
    int rm = perm[k], rn = perm[k + 1];
    double expo = (betas[k] - betas[k + 1]) * (E[rm] - E[rn]);
    double u = xo_pt_uniform(seed, ladder, sweep, k);
    double w = expo >= 0.0 ? 1.0 : exp(expo);
    if (u < w) {
      perm[k] = rn;
      perm[k + 1] = rm;
      if (accepted) accepted[k] = 1;
      ++n;
    }
  }
  return n;
}

/* Single-histogram reweighting of a series (E_t, O_t) measured at beta0 to
 * each target beta'_k: l_kt = -(beta'_k - beta0) E_t; log Z_k = log sum_t
 * exp(l_kt) (max-shifted); <O>_k = sum_t exp(l_kt - log Z_k) O_t.  O is
 * row-major [T][n_obs].  Outputs (row-major over k): logZ[K],
 * meanE[K], mean[K][n_obs], cov[K][n_obs] = <O E>_k - <O>_k <E>_k, the
 * fluctuation formula whose negative is d<O>/dbeta'. */
void xo_reweight(long T, const double *E, int n_obs, const double *O,
                 double beta0, int K, const double *betap, double *logZ,
                 double *meanE, double *mean, double *cov) {
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < K; ++k) {
    double db = betap[k] - beta0;
    double lmax = -INFINITY;
    for (long t = 0; t < T; ++t) {
      double l = -db * E[t];
      if (l > lmax) lmax = l;
    }
    double s = 0.0;
    for (long t = 0; t < T; ++t) s += exp(-db * E[t] - lmax);
    double lz = lmax + log(s);
    double sE = 0.0;
    double *sO = (double *)calloc((size_t)n_obs, sizeof(double));
    double *sOE = (double *)calloc((size_t)n_obs, sizeof(double));
    for (long t = 0; t < T; ++t) {
      double w = exp(-db * E[t] - lz);
      sE += w * E[t];
      for (int j = 0; j < n_obs; ++j) {
        sO[j] += w * O[t * n_obs + j];
        sOE[j] += w * O[t * n_obs + j] * E[t];
      }
    }
    logZ[k] = lz;
    meanE[k] = sE;
    for (int j = 0; j < n_obs; ++j) {
      mean[(long)k * n_obs + j] = sO[j];
      cov[(long)k * n_obs + j] = sOE[j] - sO[j] * sE;
    }
    free(sO);
    free(sOE);
  }
}
