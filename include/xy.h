/*
 * libxy -- B300-native (sm_103a) hot path of the 3D XY Monte Carlo method of
 * Lan, Hsieh & Kao, "High-precision Monte Carlo study of the
 * three-dimensional XY model on GPU" (arXiv:1211.0780): checkerboard
 * Metropolis and over-relaxation sweeps of classical O(2) spins on periodic
 * L x L x L cubic lattices, run across parallel-tempering replicas, with the
 * energy, magnetisation and helicity sums fused into the sweep, plus FP64
 * single-histogram reweighting of the measured series.
 *
 * Conventions (every entry point):
 *   - Returns an int status (XY_OK or a negative XY_ERR_*); never throws.
 *   - Host pointers are plain host memory owned by the caller and are only
 *     read or written during the call.  Device pointers (d_*) are owned by
 *     the caller and must stay valid for as long as the library uses them.
 *   - The library allocates no device memory: all device state lives in the
 *     caller's workspace (xy_workspace_bytes) handed to xy_init.
 *   - Work is ordered on the stream given to xy_init (a cudaStream_t passed
 *     as void*; NULL = the legacy default stream).  Calls that return host
 *     data synchronise that stream.
 *   - Errors are sticky per context: after XY_ERR_CUDA, XY_ERR_TIMEOUT or
 *     XY_ERR_BOUNDS every call on the context returns XY_ERR_STATE until
 *     xy_destroy.
 *   - A spin is stored on the device as its unit vector (cos theta,
 *     sin theta) in FP32 (as its FP32 angle on tile kind 4, see
 *     xy_set_tile).  Angles exchanged with the host (xy_get_state /
 *     xy_set_state) are FP32 radians in [0, 2 pi).
 *
 * Lattice, colours and layout.  Site (x, y, z), 0 <= x, y, z < L, has colour
 * c = (x + y + z) mod 2 (0 = "black", 1 = "white"; Sec. II, Fig. 2).  L must
 * be a multiple of 8 (8 <= L <= 1024).  Host-side angle arrays use the
 * natural layout theta[x + L (y + L z)]; on the device each colour is a
 * packed cos array and a packed sin array, both indexed
 * p = (x >> 1) + (L/2)(y + L z).
 *
 * Random numbers.  Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) with
 * key = (seed & 0xffffffff, seed >> 32).  The site with packed index p and
 * colour c of global slot g draws from the call with counter
 *   (p >> 1, count & 0xffffffff, count >> 32, g << 4 | c << 3 | tag),
 * taking words 0 and 1 if p is even, 2 and 3 if p is odd; a word w maps to
 * u = (w >> 8) 2^-24 in [0, 1).  tag 1 = initial state (count 0, theta =
 * 2 pi u of the first word), tag 2 = Metropolis (count = the Metropolis-pass
 * counter; first word -> proposal, second -> acceptance).  Exchange draws
 * use counter (k, n & 0xffffffff, n >> 32, ladder << 4 | 3), word 0, for
 * pair k of exchange event n.
 *
 * Slots and ladders.  xy_init takes n_lattices lattices; lattice l has edge
 * L[l] and n_replicas[l] replicas ("slots"), numbered globally (lattice 0's
 * first).  Each lattice is one parallel-tempering ladder whose betas are
 * given in ascending order; initially the k-th replica sits at the k-th
 * beta.  An exchange swaps beta labels (a permutation), not configurations.
 */
#ifndef XY_H
#define XY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  XY_OK = 0,
  XY_ERR_ARG = -1,     /* invalid argument; nothing was done             */
  XY_ERR_CUDA = -2,    /* a CUDA call failed; the context is now unusable */
  XY_ERR_TIMEOUT = -3, /* a bounded device-side wait ran out               */
  XY_ERR_STATE = -4,   /* the context is in a sticky error state          */
  XY_ERR_NOMEM = -5,   /* workspace or series buffer too small            */
  XY_ERR_BOUNDS = -6   /* bounds-checked build (XY_BOUNDS_CHECK, libxy_check)
                          only: a kernel skipped an access outside its buffer */
};

/* Execution modes of xy_sweep. */
enum {
  XY_EXEC_PLAIN = 0,      /* one kernel launch per half-sweep per lattice          */
  XY_EXEC_GRAPH = 1,      /* the same launches captured once into a CUDA graph     */
  XY_EXEC_PERSISTENT = 2  /* persistent launches, each running one part of a
                             sweep (its Metropolis passes, its over-relaxation
                             passes, the last half-sweep with the measurement and
                             the exchange) for every lattice and replica as one
                             list of tile items; no grid barrier: an item waits
                             (bounded) only for its own slot's previous work,
                             counted per slot; the launches are chained by
                             programmatic dependent launch; one CUDA graph per
                             xy_sweep call                                          */
};

typedef struct xy_ctx xy_ctx; /* opaque; owned by the library */

/* One measurement of one slot: the lattice sums behind the estimators of
 * Sec. II, Eqs. (4)-(6).  E = -sum_<ij> cos(theta_i - theta_j) (Eq. 1);
 * (Mx, My) = sum_i (cos theta_i, sin theta_i); C[mu] and S[mu] = the sums
 * over bonds (i, i + mu) of cos and sin of (theta_i - theta_{i+mu}).  Then
 * m = sqrt(Mx^2 + My^2) / N (Eq. 4) and rho_s = (1/3N) sum_mu (C[mu] -
 * beta S[mu]^2) (Eq. 6). */
typedef struct xy_record {
  double E;
  double Mx, My;
  double C[3];
  double S[3];
  double beta;        /* the beta of the slot when measured            */
  int32_t slot;       /* global slot                                    */
  int32_t beta_index; /* position of that beta in its ladder           */
  uint64_t sweep;     /* 0-based index of the sweep just completed      */
} xy_record;          /* 96 bytes                                       */

/* Bytes of device workspace xy_init needs for these lattices and a series
 * buffer of `series_capacity` measurement events (each event holds one
 * record per slot).  When the lattices' vector state (8 bytes per site) is
 * at most 40 MB the workspace also holds one Metropolis pass's Philox words
 * (another 8 bytes per site), which the over-relaxation half-sweeps of
 * XY_EXEC_PLAIN and XY_EXEC_GRAPH draw ahead for the direct tile (kind 3).
 * Returns 0 for invalid arguments. */
size_t xy_workspace_bytes(int n_lattices, const int *L, const int *n_replicas,
                          int64_t series_capacity);

/* Creates a context over caller-owned device memory `d_workspace` (at least
 * xy_workspace_bytes, 256-byte aligned; it must outlive the context) and
 * writes the initial state: theta = 2 pi u from the initial-state stream,
 * uniform in [0, 2 pi) as in the hot start of the benchmark configurations.
 * `betas` holds sum(n_replicas) inverse temperatures, lattice by lattice,
 * each lattice's ascending.  The paper's single-lattice call
 * xy_init(L, betas, seed) is n_lattices = 1.  `stream` is a cudaStream_t or
 * NULL.  Errors: XY_ERR_ARG (L not a multiple of 8 or out of range, a
 * non-positive replica count, betas not finite or not ascending, NULL
 * pointers), XY_ERR_NOMEM (ws_bytes too small), XY_ERR_CUDA. */
int xy_init(xy_ctx **out, int n_lattices, const int *L, const int *n_replicas,
            const double *betas, uint64_t seed, void *d_workspace,
            size_t ws_bytes, int64_t series_capacity, void *stream);

/* Releases the context (not the workspace) after synchronising its stream,
 * so the caller may free the workspace once it returns.  Safe on NULL;
 * always returns XY_OK (a failed context's error is not reported again). */
int xy_destroy(xy_ctx *ctx);

/* Selects how xy_sweep issues its work (XY_EXEC_*).  All modes give
 * bit-identical states and records. */
int xy_set_exec(xy_ctx *ctx, int mode);

/* Runs n_sweeps sweeps on every slot (Sec. II: "one Monte Carlo step").
 * One sweep = n_metropolis Metropolis passes then n_overrelax
 * over-relaxation passes; a pass is a black half-sweep then a white one.
 * After sweep s (0-based, counted over the context's life):
 *   - if measure_every > 0 and (s + 1) % measure_every == 0, one record per
 *     slot is appended to the series buffer (fused into the last white
 *     half-sweep);
 *   - if pt_swap_every > 0 and (s + 1) % pt_swap_every == 0, one exchange
 *     event runs on every ladder with the energies of the final state
 *     (Sec. II, Eq. 3), alternating even and odd pairs between events; a
 *     sweep that exchanges without recording sums the energy alone, as
 *     -E = sum over white sites of w . h (h the six neighbours' sum: the
 *     same bonds as the record's C_x + C_y + C_z, in another order).
 * Metropolis half-sweep (Sec. II): each site of the colour proposes
 * theta' = 2 pi u0 and accepts iff u1 < exp(-beta dE), with dE = -[h_x
 * (cos theta' - cos theta) + h_y (sin theta' - sin theta)] and h the sum of
 * the six neighbour spin vectors.  Over-relaxation half-sweep (Eq. 2): the
 * spin is reflected about its local field, S' = 2 (S.h / h.h) h - S (as an
 * angle theta' = 2 atan2(h_y, h_x) - theta mod 2 pi); h = 0 leaves it.  The
 * Philox words of a Metropolis pass depend only on the seed, the pass
 * counter, the slot, the colour and the site, so with a words region (see
 * xy_workspace_bytes) the over-relaxation half-sweeps between a sweep's
 * first and last draw the next sweep's first-pass words and that pass reads
 * them: the same words, the same spins.  Errors: XY_ERR_ARG (negative counts,
 * n_metropolis + n_overrelax == 0 with n_sweeps > 0), XY_ERR_NOMEM (the
 * series buffer would overflow: read it first), XY_ERR_TIMEOUT, XY_ERR_CUDA. */
int xy_sweep(xy_ctx *ctx, int n_metropolis, int n_overrelax, int n_sweeps,
             int measure_every, int pt_swap_every);

/* One Metropolis half-sweep of `colour` on every slot (Sec. II, the
 * checkerboard update of Fig. 2) with Metropolis-pass counter `mpass` (the
 * counters of the context are not advanced). */
int xy_metropolis_half(xy_ctx *ctx, int colour, uint64_t mpass);

/* One over-relaxation half-sweep of `colour` on every slot (Eq. 2). */
int xy_overrelax_half(xy_ctx *ctx, int colour);

/* Measures the current state of every slot (Eqs. 4-6 sums) into
 * host_out[total slots]; synchronises the stream. */
int xy_measure(xy_ctx *ctx, xy_record *host_out);

/* One exchange event on every ladder (Eq. 3) with freshly measured
 * energies: pairs (k, k+1), k = parity, parity + 2, ...; accept with
 * min[1, exp((beta_k - beta_{k+1})(E_k - E_{k+1}))] where E_k is the energy
 * of the slot at beta_k.  Uses and advances the exchange-event counter.
 * *n_accepted_out (nullable) receives the number of accepted swaps over all
 * ladders; synchronises the stream. */
int xy_pt_swap(xy_ctx *ctx, int parity, int *n_accepted_out);

/* The measurement series (Sec. II: the per-sweep values that are binned).
 * Copies the records appended since the last read (oldest first) into
 * host_buf (room for `cap` records) and empties the buffer.  *n_out = the
 * number copied.  XY_ERR_NOMEM if cap is too small (nothing is copied). */
int xy_read_series(xy_ctx *ctx, xy_record *host_buf, int64_t cap,
                   int64_t *n_out);

/* Number of records waiting in the series buffer. */
int xy_series_count(xy_ctx *ctx, int64_t *n_out);

/* The spin configuration theta_i of H = -J sum cos(theta_i - theta_j)
 * (Sec. II), for parity checks and checkpoints.  host_angles: all slots
 * concatenated, natural layout, sum over slots of L^3 floats; get_state
 * returns atan2(sin, cos) of the stored vectors taken into [0, 2 pi),
 * set_state stores (cos, sin) of the given angles (sincosf; every angle
 * must be finite); on tile kind 4 (angle storage) the stored angles are
 * returned as they are and the given ones stored taken into [0, 2 pi).  perm: for each ladder in order, n_replicas entries
 * (beta index -> local slot).  counters[4] = {Metropolis passes, sweeps,
 * exchange events, records}.  Any pointer may be NULL to skip that part.
 * Every draw is a pure function of (seed, counters, slot, site), so
 * restoring the counters and the packed state (xy_set_packed) resumes a run
 * bit-exactly; restoring angles resumes it up to the FP32 rounding of the
 * angle <-> vector conversion. */
int xy_get_state(xy_ctx *ctx, float *host_angles, int32_t *perm,
                 uint64_t *counters);
int xy_set_state(xy_ctx *ctx, const float *host_angles, const int32_t *perm,
                 const uint64_t *counters);

/* The spins of every slot in the device's packed layout (for each slot:
 * colour 0's N/2 cosines, its N/2 sines, then colour 1's, indexed
 * p = (x >> 1) + (L/2)(y + L z)), copied stream-ordered between the
 * workspace and a host buffer of sum over slots of 2 L^3 floats (pinned
 * memory makes the copy asynchronous; the call returns after it completes).
 * Bit-exact checkpoints and host round trips without the conversion of
 * xy_get_state / xy_set_state; set_packed takes the vectors as given.  A
 * lattice on tile kind 4 (angle storage) holds its angles where the
 * cosines are (the sine places are unused); a packed state is restored on a
 * lattice of the same storage. */
int xy_get_packed(xy_ctx *ctx, float *host_packed);
int xy_set_packed(xy_ctx *ctx, const float *host_packed);

/* The spins as FP32 angles in the packed order (for each slot: colour 0's
 * N/2 angles, then colour 1's, at p = (x >> 1) + (L/2)(y + L z)); a host
 * buffer of sum over slots of L^3 floats, half the bytes of the packed
 * vectors.  set: stream-ordered copy into the workspace and conversion on
 * the device with sincosf (the values must be finite; they are not
 * inspected; on tile kind 4 the angles are taken into [0, 2 pi) and kept);
 * get: atan2 on the device, wrapped into [0, 2 pi) as xy_get_state (on
 * tile kind 4 the stored angles themselves).  Both return after the copy completes (pinned memory makes
 * it asynchronous to the host until then). */
int xy_set_packed_angles(xy_ctx *ctx, const float *host_angles);
int xy_get_packed_angles(xy_ctx *ctx, float *host_angles);

/* Page-locked host memory for the host buffers of the calls above
 * (cudaHostAlloc, portable to every device), so that their copies run at
 * the full host-to-device rate: on some hosts memory pinned by other means
 * (page by page) moved at a quarter of it.  The one allocation call of the
 * library, on the host only; the caller frees the block with xy_host_free
 * (NULL is a no-op).  Errors: XY_ERR_ARG (NULL out, zero bytes),
 * XY_ERR_CUDA (the allocation failed; *out = NULL, no context is affected). */
int xy_host_alloc(size_t bytes, void **out);
int xy_host_free(void *p);

/* The parallel-tempering temperature set (Sec. II, Eq. 3).
 * Replaces the betas of ladder `lattice` (n_replicas ascending finite
 * values) in a running context: every slot takes the new beta of its beta
 * index (the exchange permutation is kept).  Used by an adaptive ladder
 * (xy_ladder_update); counters, states and records are untouched. */
int xy_set_betas(xy_ctx *ctx, int lattice, const double *betas);

/* Equal-acceptance ladder update (host only; Sec. II: the temperature set
 * is chosen so that the exchange acceptance rate does not depend on the
 * temperature).  betas[R] ascending; acceptance[R-1] = the measured
 * exchange acceptance of pair (k, k+1).  Model: Gaussian energy
 * distributions of a common width sigma_k near each pair, for which
 * A_k = erfc(Delta_k sigma_k / 2); the target widths are Delta*_k =
 * W (Delta_k / x_k) / sum_j (Delta_j / x_j) with x_k = erfcinv(A_k) (rates
 * clamped to [1e-6, 1 - 1e-9]) and W = beta_R-1 - beta_0, which equalises
 * the modelled acceptances.  new_betas[R] keeps both ends and moves each
 * width the fraction `damping` in [0, 1] of the way to its target.
 * Errors: XY_ERR_ARG (R < 2, a non-ascending ladder, a rate outside
 * [0, 1], damping outside [0, 1], NULL). */
int xy_ladder_update(int R, const double *betas, const double *acceptance,
                     double damping, double *new_betas);

/* Accepted-move counters of the Metropolis test (Sec. II) and of the
 * exchanges (Eq. 3): met[total slots] = accepted Metropolis proposals
 * per slot; swap[total slots] = accepted exchanges per ladder pair (entry
 * slot0(l) + k for pair (k, k+1) of ladder l).  Either may be NULL. */
int xy_get_accepts(xy_ctx *ctx, uint64_t *met, uint64_t *swap);

/* Philox4x32-10 (Salmon et al., SC'11; it replaces the Warp Generator of
 * Sec. II).  Raw words of every site of one colour of slot `slot` for stream
 * `tag` and counter `count`, natural order of those sites (x fastest), two
 * words per site, drawn on the device by the same code the sweeps use. */
int xy_debug_draws(xy_ctx *ctx, int slot, int colour, int tag, uint64_t count,
                   uint32_t *host_words);

/* The fast-math expressions of the Metropolis update (Sec. II: proposal
 * theta' uniform in [0, 2 pi), acceptance u < exp(-beta dE)), evaluated
 * element by element on the device by the same device functions the sweep
 * kernels inline, for accuracy checks against FP64.  kind 0: d_in holds n
 * uint32 proposal words w; d_out[2i], d_out[2i+1] receive the proposal
 * vector (cos theta', sin theta') of theta' = (w >> 8) 2 pi / 2^24 (FP32
 * product) as the update forms it with the fast sincos.  kind 1: d_in holds
 * n FP32 exponents x = -beta dE; d_out[i] receives the threshold exp(x) 2^24
 * (fast exponential) that the update compares the acceptance word's
 * (w >> 8) with.  kind 2: d_in holds n FP32 pairs (x, y), not both zero;
 * d_out[i] receives the angle-storage tile's atan2(y, x) (the field's
 * angle of the over-relaxation of Eq. 2 on stored angles).  Device pointers
 * owned by the caller, on the current device; ordered on `stream`, which
 * the call synchronises.  XY_ERR_ARG for another kind, n < 0 or a null
 * pointer with n > 0. */
int xy_debug_fast_math(int kind, int64_t n, const void *d_in, float *d_out,
                       void *stream);

/* Tile of lattice `lattice`.  kind 0 (march): a thread block of (L/8) x ty
 * threads covers full rows in x and ty rows in y and marches over tz planes
 * in z, loading each other-colour spin about once.  kind 1 (block): a
 * thread block of (L/8) x ty x tz threads covers ty rows x tz planes at
 * once after one cooperative staging of the tile's other-colour rows and
 * face halos.  kind 2 (stream): the march's thread layout, with every plane
 * the tile reads (the other colour's rows with their y halo, the own
 * colour's rows) copied ahead into a ring of shared-memory stages by bulk
 * asynchronous copies (TMA); not run by XY_EXEC_PERSISTENT, whose blocks
 * write planes other blocks read within one launch.  kind 3 (direct): the
 * march's thread layout and plane march without shared memory or block
 * barriers: each thread loads its y-neighbour rows and x-halo element
 * itself through the L1 cache, one plane ahead (in XY_EXEC_PERSISTENT the
 * acquire of the slot's count before each tile orders those loads after
 * the previous half-sweep's writes).  kind 4 (angle): the march's thread
 * layout on a lattice kept as FP32 angles in [0, 2 pi) instead of vectors
 * (4 instead of 8 bytes per spin; each colour's angles sit where its
 * cosines are in the vector layout): every other-colour angle of the tile
 * is turned into its vector once by the fast sincos and shared through the
 * shared-memory plane buffers, and the update stores the new angle (the
 * proposal's, or 2 phi - theta with phi the field's angle, Eq. 2).
 * Changing a lattice between kind 4 and another kind converts its state in
 * place (atan2f / sincosf, within 1e-6 rad).
 * xy_set_tile checks 1 <= ty, tz <= L, the block size against
 * the kernels' limit (512 threads at their register use on sm_103a; 240
 * for kinds 3 and 4), tz <= 64 for kind 1, and that the tile count fits the
 * partial-sum area (ceil(L/ty) ceil(L/tz) <= L^2/4).  Spins do not depend
 * on the tile among kinds 0-3 (the lattice sums only through FP64 summation
 * order), nor on the shape within kind 4; kind 4 differs from the others by
 * the fast sincos of the neighbours (a few 1e-7 per vector). */
int xy_set_tile(xy_ctx *ctx, int lattice, int kind, int ty, int tz);
int xy_get_tile(xy_ctx *ctx, int lattice, int *kind, int *ty, int *tz);

/* Picks each lattice's tile (kind and shape) by timing the candidates on
 * the device for sweeps of `n_metropolis` + `n_overrelax` passes (the spins,
 * counters, accept counts and the ladders' permutations, couplings and
 * exchange counts are saved and restored); the choice stays in the
 * context.  Outside XY_EXEC_PERSISTENT every kind (0-3) is a candidate,
 * and kind 4 too when the context's vector state is larger than the
 * device's L2 cache (there a half-sweep is bound by HBM bytes, which angle
 * storage halves); each lattice's best tile is found on its own half-sweep
 * launches.  In XY_EXEC_PERSISTENT mode one tile kind serves every lattice
 * (xy_sweep returns XY_ERR_ARG otherwise) and the block is as wide as the
 * widest tile: for the march, the block, the direct (and, as above, the
 * angle) kind and for tiles of at most 64, 128 and 256 threads, each
 * lattice's best tile is found as above, the sets are timed in the
 * persistent launch itself, and the fastest is kept.  In every mode the
 * kept set is then refined on whole sweeps of all lattices together, in
 * the context's execution mode (ending with an exchange when a ladder has
 * two or more replicas): lattice by lattice, largest first, a tile's rows
 * or planes doubled or halved, a change kept when it is at least 1%
 * faster. */
int xy_autotune(xy_ctx *ctx, int n_metropolis, int n_overrelax);

/* Device-side status word of the last persistent launch (0 = fine). */
int xy_device_status(xy_ctx *ctx, int *status_out);

/* Test hook for the bounded waits of XY_EXEC_PERSISTENT: runs one
 * persistent launch whose blocks each wait for a slot count that nothing
 * raises, so every wait runs out after `budget_us` microseconds and the
 * kernel returns XY_ERR_TIMEOUT through the status word without hanging.
 * The context stays usable (the timeout is reported, not made sticky).  No
 * GPU fault is involved. */
int xy_debug_barrier_timeout(xy_ctx *ctx, int budget_us, int *status_out);

/* Test hook for the bounded plane waits of stream tiles (kind 2): lattice 0
 * must use a stream tile.  Runs one over-relaxation half-sweep of colour 0
 * of lattice 0 in which no block copies its third plane, so every block's
 * wait for it runs out after `budget_us` microseconds; the blocks set the
 * status word to XY_ERR_TIMEOUT, update nothing, let their other copies
 * land and return.  The state is unchanged and the context stays usable
 * (the timeout is reported, not made sticky).  No GPU fault is involved. */
int xy_debug_stream_timeout(xy_ctx *ctx, int budget_us, int *status_out);

/* Throughput probe of one hardware unit, for roofline denominators:
 * kind 0 = special-function unit sin+cos (2 ops per pair), 1 = ex2,
 * 2 = FP32 FMA, 3 = FP64 FMA, 4 = 32x32->64 integer multiply (the Philox
 * round's operation), 5 = L2 read bytes (a 32 MiB L2-resident buffer).
 * Writes operations (or bytes) per second to *ops_per_s.  d_scratch: device
 * memory owned by the caller, >= 64 MiB for kind 5 and >= 4 bytes
 * otherwise.  Runs on the current device and `stream`; synchronises it. */
int xy_peak_probe(int kind, void *d_scratch, size_t scratch_bytes,
                  double *ops_per_s, void *stream);

/* Human-readable text of a status code. */
const char *xy_strerror(int status);

/* ------------------------------------------------------------------------
 * Single-histogram reweighting (Ferrenberg-Swendsen; not in the paper,
 * which bins the series on the host, Sec. II).  For a series of T samples
 * measured at beta0 and targets beta'_k (k < K):
 *   l_kt = -(beta'_k - beta0) E_t,   log Z_k = log sum_t exp(l_kt),
 *   <O>_k = sum_t exp(l_kt - log Z_k) O_t,
 * for O in {E, m2, m4, csum = sum_mu c_mu, s2sum = sum_mu s2_mu}, where
 * m2 = (|M|/N)^2, m4 = m2^2, c_mu = C_mu / N, s2_mu = S_mu^2 / N.  Derived:
 *   U_L(beta')   = 1 - <m4> / (3 <m2>^2)               (Eq. 5)
 *   rho_s L      = L/3 (<csum> - beta' <s2sum>)         (Eq. 6 scaled by L
 *                                                        as in Eq. 8)
 * and their d/dbeta' from d<O>/dbeta' = -(<O E> - <O><E>).
 * All arithmetic is FP64.  Device pointers; layout:
 *   d_E[T] f64, d_m2[T] f32, d_m4[T] f32, d_c[3][T] f32, d_s2[3][T] f32,
 *   d_betap[K] f64.
 * Outputs (device, f64):
 *   d_out[6][K]  = rows {logZ, <E>, <m2>, <m4>, <csum>, <s2sum>};
 *   d_obs[3][K]  = {U_L, rho_s L, q2 = <m4>/<m2>^2 (Eq. 11) = 3 (1 - U_L)};
 *   d_cov[5][K]  = {var E, cov(m2,E), cov(m4,E), cov(csum,E), cov(s2sum,E)}.
 * d_scratch: xy_reweight_scratch_bytes(T, K) bytes of caller-owned device
 * memory.  Errors: XY_ERR_ARG (T < 2, K < 1, L < 1, NULL pointers,
 * non-finite beta0), XY_ERR_NOMEM (scratch too small), XY_ERR_CUDA. */
size_t xy_reweight_scratch_bytes(int64_t T, int K);

int xy_reweight_forward(int64_t T, const double *d_E, const float *d_m2,
                        const float *d_m4, const float *d_c, const float *d_s2,
                        double beta0, int K, const double *d_betap, int L,
                        double *d_out, double *d_obs, double *d_cov,
                        void *d_scratch, size_t scratch_bytes, void *stream);

/* Allocation-free forward pass.  The paper has no counterpart: this entry
 * point exists for callers that cannot give the library scratch memory --
 * code working inside a device-memory budget fixed at start-up, code that
 * must not call the CUDA allocator (or a framework's caching allocator)
 * once running, and plugins whose host framework owns every device
 * allocation.  It computes exactly what xy_reweight_forward computes (same
 * kernels, outputs equal to FP64 rounding) but takes its scratch from one
 * library-owned device array of xy_reweight_noalloc_capacity_bytes() bytes
 * (8 MiB), which every GPU that loads the library holds until the process
 * exits.  The number of sample chunks is capped so their partial sums fit:
 * K may be at most about 95,000 target couplings; larger K returns
 * XY_ERR_NOMEM (T is unrestricted).  The call allocates nothing.  It runs on
 * the device that owns d_out (device or managed memory; made current for the
 * call, and the caller's current device restored before it returns) and, on
 * its first call on a device, looks up the array's device address and keeps
 * it for the life of the process -- make that first call before any stream
 * capture, and do not call this entry point on a device after a
 * cudaDeviceReset of it (the kept address then belongs to the torn-down
 * context).  Every call shares the array and leaves its contents behind;
 * nothing needs clearing because each call writes every word it later
 * reads, but calls that overlap on the GPU race.  Errors as for
 * xy_reweight_forward. */
size_t xy_reweight_noalloc_capacity_bytes(void);

int xy_reweight_forward_noalloc(int64_t T, const double *d_E, const float *d_m2,
                                const float *d_m4, const float *d_c,
                                const float *d_s2, double beta0, int K,
                                const double *d_betap, int L, double *d_out,
                                double *d_obs, double *d_cov, void *stream);

/* Multi-histogram reweighting (Ferrenberg and Swendsen, 1989) of the
 * pooled series of a whole ladder (not in the paper, which bins each
 * temperature's series separately, Sec. II).  T records pooled over R <= 64
 * couplings betas[m] (host, ascending), counts[m] >= 1 of them measured at
 * betas[m] (host, sum = T), grouped by coupling in that order.  Free
 * energies: log D_t = log sum_m counts[m] exp(f_m - betas[m] E_t) and
 * f_k = -log sum_t exp(-betas[k] E_t - log D_t), solved as the minimum of
 * the convex F(f) = sum_t log D_t - sum_m counts[m] f_m by Newton's method
 * (f_0 = 0, backtracking line search, steps capped at 20 in any f_k; the
 * fixed-point step of the equations where the Hessian is not positive
 * definite) until the step is at most tol.  Start: the caller's f if it is
 * finite and not all zero, else thermodynamic integration of the group
 * mean energies.  All FP64 with log-sum-exp shifts; deterministic.
 * Returns XY_OK, or XY_ERR_TIMEOUT if max_iter steps did not converge (f
 * holds the last iterate); *iters_out (nullable) gets the number of Newton
 * steps.  Scratch: xy_multihist_scratch_bytes(T, R, K) bytes (K = 0 for
 * solving only).  Synchronises `stream` a few times per step. */
size_t xy_multihist_scratch_bytes(int64_t T, int R, int K);
int xy_multihist_solve(int64_t T, const double *d_E, int R,
                       const double *betas, const int64_t *counts, double tol,
                       int max_iter, double *f, int *iters_out,
                       void *d_scratch, size_t scratch_bytes, void *stream);

/* Averages at K target couplings from the pooled series and solved f:
 * <O>_beta' = sum_t O_t exp(-beta' E_t - log D_t) / sum_t exp(...), with the
 * columns and outputs of xy_reweight_forward (d_out[6][K]: log of the
 * denominator sum, <E>, <m2>, <m4>, <c>, <s2>; d_obs[3][K]: U_L, rho_s L, q2;
 * d_cov[5][K]: covariances with E, so xy_reweight_backward gives the
 * beta' derivatives). */
int xy_multihist_forward(int64_t T, const double *d_E, const float *d_m2,
                         const float *d_m4, const float *d_c, const float *d_s2,
                         int R, const double *betas, const int64_t *counts,
                         const double *f, int K, const double *d_betap, int L,
                         double *d_out, double *d_obs, double *d_cov,
                         void *d_scratch, size_t scratch_bytes, void *stream);

/* Per-bin reweighting sums for error analysis by resampling (the paper
 * blocks its measurements into bins and resamples them, Sec. II-III).  The
 * series (as for xy_reweight_forward) is cut into n_bins equal contiguous
 * bins, bin b = samples [b T / n_bins, (b+1) T / n_bins).  d_binsums
 * [n_bins][K][11] (device f64, caller-owned) receives, for each bin and
 * target coupling k, the sums over the bin of w_kt x_j for x_j in {1, e,
 * e^2, m2, m2 e, m4, m4 e, c, c e, s2, s2 e} with e = E - Ebar, c and s2 the
 * three-direction sums, and w_kt = exp(-(beta'_k - beta0)(e - e_ref)) with a
 * shift e_ref per k common to all bins: bin sums add, and ratios of
 * (resampled) sums are reweighted averages.  d_stats[3] (nullable) receives
 * {Ebar, min e, max e}.  d_scratch: xy_reweight_bins_scratch_bytes(T, K,
 * n_bins) bytes.  Errors: XY_ERR_ARG (T < 2, K < 1, n_bins outside
 * [1, min(T, 65535)], NULL pointers), XY_ERR_NOMEM, XY_ERR_CUDA. */
size_t xy_reweight_bins_scratch_bytes(int64_t T, int K, int n_bins);
int xy_reweight_bins(int64_t T, const double *d_E, const float *d_m2,
                     const float *d_m4, const float *d_c, const float *d_s2,
                     double beta0, int K, const double *d_betap, int n_bins,
                     double *d_binsums, double *d_stats, void *d_scratch,
                     size_t scratch_bytes, void *stream);

/* Resampled sums: d_sums[r][K][11] = sum_b d_counts[r][b] d_binsums[b][K][11]
 * for B resamples given as bin multiplicities (int32 [B][n_bins], device;
 * bootstrap: drawn with replacement; jackknife: all ones but one zero).
 * Bins are added in order (deterministic).  n_bins <= 6144, B <= 65535. */
int xy_fss_resample(int n_bins, int K, const double *d_binsums, int B,
                    const int32_t *d_counts, double *d_sums, void *stream);

/* Curves of each resample: d_curves[r][4][K] = {U_L (Eq. 5, 1 - <m4> /
 * (3 <m2>^2)), rho_s L (Eq. 6, (L/3)(<c> - beta' <s2>)), dU_L/dbeta',
 * d(rho_s L)/dbeta'} from resampled sums, the derivatives by
 * d<O>/dbeta' = -(<O e> - <O><e>). */
int xy_fss_curves(int B, int K, const double *d_betap, int L,
                  const double *d_sums, double *d_curves, void *stream);

/* Crossing of two sizes' curves, row `which` (0 = U_L, 1 = rho_s L), for
 * each resample (Sec. III: the curves of different L intersect at T_c): the
 * first grid interval (ascending beta') where A - B changes sign, refined on
 * the cubic Hermite interpolant of A - B (values and derivatives at the two
 * grid points) by bisection; slopes of A and B at the crossing from their
 * Hermite interpolants; 1/nu = ln(|slope B| / |slope A|) / ln(LB / LA),
 * since a dimensionless ratio scales as Q(t L^{1/nu}).  d_out[B][5] =
 * {beta*, slope A, slope B, 1/nu, nu}, NaN where the curves do not cross. */
int xy_fss_crossings(int B, int K, const double *d_betap, int LA,
                     const double *d_curvesA, int LB, const double *d_curvesB,
                     int which, double *d_out, void *stream);

/* Backward: given upstream gradients g_U[K] and g_rhoL[K] (device f64) and
 * the forward's d_out, d_cov, returns grad_betap[K] = g_U dU/dbeta' +
 * g_rhoL d(rho_s L)/dbeta' (each output depends only on its own beta'_k).
 * d_dobs[3][K] (nullable) receives {dU/dbeta', d(rho_s L)/dbeta',
 * dq2/dbeta' = -3 dU/dbeta'}. */
int xy_reweight_backward(int K, const double *d_betap, int L,
                         const double *d_out, const double *d_cov,
                         const double *d_gU, const double *d_grhoL,
                         double *d_grad_betap, double *d_dobs, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* XY_H */
