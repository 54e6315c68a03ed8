/*
 * tnlbm.h - C ABI of the GB300 MPS lattice Boltzmann library (libtnlbm.so).
 *
 * The method (Gross et al., "Tensor Network Lattice Boltzmann Method for
 * Data-Compressed Fluid Simulations"): every particle distribution function
 * f_i of a D3Q19 / D3Q15 BGK lattice Boltzmann model is stored as a matrix
 * product state (MPS, Eq. MPS) over the scale-ordered binary digits of the
 * cell coordinates (Sec. 2.4, Eq. scale_ordering); one time step (Sec. 3.2)
 * is carried out entirely on those encodings with no dense grid:
 *   collision from moments, a Taylor-expanded 1/rho and compressed products
 *   (Sec. 2.3, Sec. 3.2, App. A), streaming as shift-MPO x MPS (Sec. 2.5),
 *   bounce-back walls and objects through mask MPS (Eqs. boundaries2, objects),
 *   and TT-rounding of every sum (Eq. svd-move).
 *
 * Conventions (all entry points)
 *   - Return 0 on success, a negative TNLBM_E_* code on failure; no exception
 *     crosses the ABI.  tnlbm_last_error() returns a thread-local message.
 *   - Binary sites: an N^3 lattice with N = 2^n has L = 3n sites; site k holds
 *     bit (n-1 - k/3) of axis k%3 (axis 0 = x), most significant bits first.
 *   - Dense fields are [x][y][z] row-major (z fastest).
 *   - "Flat MPS layout" (host or device): for L sites and capacity cap, bond k
 *     has capacity cap_k = cap for 0 < k < L and cap_0 = cap_L = 1; core k
 *     occupies a slot of cap_k * 2 * cap_(k+1) elements starting at
 *     tnlbm_mps_offset(L, cap, k); inside the slot the core is packed
 *     [r_k][2][r_(k+1)] row-major with its realised bonds r.  Realised bonds
 *     are an int32 array r[0..L] with r[0] = r[L] = 1.
 *   - precision: TNLBM_FP64 buffers hold double, TNLBM_FP32, TNLBM_TF32,
 *     TNLBM_MIXED and TNLBM_BF16 buffers float.
 *   - stream arguments are cudaStream_t values passed as void* (NULL = legacy
 *     default stream).  Primitive calls are asynchronous on that stream unless
 *     stated; they allocate their own scratch with cudaMalloc and free it
 *     after synchronising the stream.
 */
#ifndef TNLBM_H
#define TNLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TNLBM_OK = 0,
  TNLBM_E_ARG = -1,      /* invalid argument or configuration            */
  TNLBM_E_OOM = -2,      /* device or host allocation failed             */
  TNLBM_E_CUDA = -3,     /* a CUDA runtime call failed                   */
  TNLBM_E_TIMEOUT = -4,  /* a bounded device-side wait ran out           */
  TNLBM_E_NOCONV = -5,   /* a Jacobi SVD hit its sweep limit             */
  TNLBM_E_NAN = -6,      /* non-finite values detected                   */
  TNLBM_E_CAPACITY = -7  /* a realised bond exceeded a buffer capacity   */
};

/* Precision of a simulation or primitive call:
 *   TNLBM_FP64   cores, contractions, QR and SVD in FP64
 *   TNLBM_FP32   FP32 cores, contractions, QR and one-sided Jacobi SVD; the
 *                singular-value tails and the rank rule in FP64
 *   TNLBM_TF32   as TNLBM_FP32, with the fit's core contractions on the tensor
 *                cores (TF32 operands, FP32 sums)
 *   TNLBM_MIXED  FP32 cores, contractions and QR sweeps; the centre SVD of every
 *                rounding step (Eq. svd-move: the singular values whose tail is
 *                the discarded weight, and the kept singular vectors) by an
 *                FP64 one-sided Jacobi on the FP32 centre matrix X, run to the
 *                FP64 stopping rule, with the inner products, norms and tails
 *                in FP64.  It starts from the V of FP32 sweeps on X, made
 *                orthogonal in FP64 by one Newton-Schulz step (W = X V formed
 *                in FP64).  On one GPU the FP64 part of a rounding is shared by
 *                a thread-block cluster of up to 16 CTAs
 *                (tnlbm_config.max_cluster); with one CTA per job the FP64
 *                Jacobi runs from V = I.
 *   TNLBM_BF16   as TNLBM_MIXED, with the fit's core contractions on the tensor
 *                cores as BF16 x BF16 products summed in FP32 (tcgen05.mma
 *                kind::f16); cores and every other contraction stay FP32. */
enum { TNLBM_FP64 = 0, TNLBM_FP32 = 1, TNLBM_TF32 = 2, TNLBM_MIXED = 3, TNLBM_BF16 = 4 };
enum { TNLBM_D3Q19 = 19, TNLBM_D3Q15 = 15 };
enum { TNLBM_HADAMARD_FIT = 0, TNLBM_HADAMARD_EXACT = 1, TNLBM_HADAMARD_ZIPUP = 2 };

/* ------------------------------------------------------------ simulation */

typedef struct tnlbm_sim tnlbm_sim; /* opaque; owns all its device memory */

typedef struct {
  int n_per_axis;          /* bits per axis n, N = 2^n, 2 <= n <= 10           */
  int lattice;             /* TNLBM_D3Q19 or TNLBM_D3Q15 (Sec. 3.1)            */
  double tau;              /* BGK relaxation time (Eq. collision), > 0.5       */
  int periodic[3];         /* per axis: 1 = cyclic shift S, 0 = wall: non-cyclic
                              shift plus halfway bounce-back (Eq. boundaries2)   */
  const uint8_t *solid;    /* host N^3 voxels [x][y][z], 1 = solid, or NULL;
                              copied during create; compressed on the GPU by
                              TT-SVD (Eq. svd-comp) to chi_mask / eps_mask      */
  int chi_mask;            /* bond cap of the object mask MPS                  */
  double eps_mask;         /* relative tolerance of the mask TT-SVD            */
  const double *mask_cores;/* alternative to solid: host mask MPS m_O in flat
                              layout (FP64, capacity mask_cap), or NULL         */
  const int *mask_ranks;   /* its realised bonds r[0..L]                       */
  int mask_cap;
  double force[3];         /* body force density F (App. A), lattice units     */
  int chi_max;             /* bond cap chi of every rounding (Sec. 2.1)        */
  double eps;              /* relative rounding tolerance: keep the smallest
                              rank whose discarded tail is <= eps*||T||/sqrt(L-1) */
  int precision;           /* TNLBM_FP64, TNLBM_FP32, TNLBM_TF32, TNLBM_MIXED or
                              TNLBM_BF16 (see the enum above).  Near tau = 1/2 (weakly
                              damped flows) the FP32 one-sided Jacobi of
                              TNLBM_FP32 / TNLBM_TF32 leaves errors the
                              collision does not damp: use TNLBM_MIXED,
                              TNLBM_BF16 or TNLBM_FP64                          */
  int hadamard;            /* TNLBM_HADAMARD_FIT (Sec. 2.3, default), _EXACT
                              (Eq. mul followed by a rounding) or _ZIPUP (the
                              zip-up pass, then a rounding; chi_max <= 512)     */
  int sweeps;              /* round trips of the product fit (Sec. 2.3: 2)     */
  int n_modes;             /* 0: start at rest, f_i = w_i (1 - m_O);  > 0:
                              f_i = w_i (1 + sum_m (a_rho + 3 c_i.a_u) cos(2 pi
                              k.x/N + phase)), rounded once                     */
  const double *modes;     /* host [n_modes][8]: kx ky kz phase a_rho a_ux a_uy a_uz */
  int max_jobs_in_flight;  /* 0 = default; caps rounding CTAs per launch        */
  int conserve_mass;       /* 1: after every step, rescale all populations by
                              M0 / M (M = sum_i <f_i, 1> in FP64, M0 its value
                              at the start): removes the ~1e-6-per-step mass
                              drift of FP32 core storage.  Not part of the
                              paper's method; default 0                         */
  /* Boundary function of each face on the non-periodic axes (Eq. boundaries2),
   * faces ordered x-, x+, y-, y+, z-, z+ (x- = the plane x = 0):
   *   TNLBM_FACE_WALL      halfway bounce-back (Eq. no_slip), the default
   *   TNLBM_FACE_VELOCITY  inlet at velocity face_u: f_i = f*_opp(i) +
   *                        2 w_i rho_0 (c_i . u_b) / c_s^2, c_i pointing into
   *                        the domain (moving-wall bounce-back, rho_b = rho_0);
   *                        tnlbm_set_face_velocity changes u_b between steps
   *   TNLBM_FACE_PRESSURE  outlet at density face_rho: f_i = -f*_opp(i) +
   *                        2 w_i rho_b (1 + (c_i.u)^2 / (2 c_s^4) - u.u / (2 c_s^2))
   *                        with the local velocity, u_d u_e = P_de / rho_0
   * A cell entered through several wall faces takes the face of lowest axis.
   * All faces TNLBM_FACE_WALL reproduces the plain bounce-back step.  Faces on
   * periodic axes must stay TNLBM_FACE_WALL (they are not used). */
  int face_kind[6];
  double face_u[6][3];
  double face_rho[6];
  int block_sums;          /* 1: the moments as one rounding of the block sum of
                              all Q populations (Eq. add over all terms) instead
                              of the pairwise tree; needs Q chi_max <= 1024     */
  int learned_rank;        /* learned rounding from the start (not in the paper):
                              0 off; 1 log spectra and training rows (as
                              tnlbm_learn_configure mode 1); 3 randomized
                              truncation at the previous step's rank (mode 3).
                              Mode 2 (the rank model) needs a trained model:
                              tnlbm_learn_set_mlp, then tnlbm_learn_configure.
                              The Gaussian test matrix is drawn from `seed`;
                              oversampling 8, one power step, eta 0.2           */
  uint64_t seed;           /* seed of that test matrix (SplitMix64 stream,
                              Box-Muller normals)                               */
  int jacobi_max_sweeps;   /* sweep limit of every one-sided Jacobi SVD (0 = 60);
                              a rounding that reaches it makes tnlbm_step return
                              TNLBM_E_NOCONV                                   */
  long long wait_limit_ns; /* limit of every wait between the CTAs of a cluster
                              (0 = 5 s); running out makes tnlbm_step return
                              TNLBM_E_TIMEOUT (the simulation can be destroyed) */
  int max_cluster;         /* CTAs per rounding job for the FP64 centre SVDs
                              (TNLBM_FP64, TNLBM_MIXED, TNLBM_BF16): 0 =
                              automatic (the largest size <= 16 at which every
                              job of a dependency level is resident at once;
                              tnlbm_tune_clusters measures it instead), 1 = one
                              CTA per job, else a cap (<= 16)                   */
} tnlbm_config;

enum { TNLBM_FACE_WALL = 0, TNLBM_FACE_VELOCITY = 1, TNLBM_FACE_PRESSURE = 2 };

typedef struct {
  int64_t steps;             /* steps taken so far                               */
  int max_bond;              /* largest realised bond over all populations       */
  double mean_bond;          /* mean realised bond over all bonds/populations    */
  double nvps;               /* sum over populations of sum_k r_k*2*r_(k+1)      */
  double compression_ratio;  /* Q*N^3 / nvps                                     */
  double rho0;               /* last mean density rho_0 (Sec. 3.2)               */
  int status;                /* device status word (0 = fine)                    */
  int gpu_launches_per_step; /* kernels launched by one tnlbm_step(1)            */
  int round_jobs_per_step;   /* rounding jobs in one step                       */
  int product_jobs_per_step; /* fit or zip-up product jobs in one step           */
  double mass;               /* sum of rho over all cells at the last rho_0 node
                                (rho_0 * N_fluid)                                */
  double discarded2;         /* sum over every rounding since creation of the
                                squared norm discarded at each truncation
                                (Eq. svd-move tails); difference two calls for
                                a step's share                                  */
  int round_ctas_per_step;   /* CTAs of all rounding launches of one step (a job
                                runs on a cluster of CTAs when its centre SVDs
                                are FP64)                                       */
  int max_cluster;           /* largest cluster of a rounding launch            */
} tnlbm_stats;

/* Build a simulation: shift MPOs, mask MPS, initial populations, and a CUDA
 * graph of one time step.  Uses the current CUDA device.  On failure *out is
 * NULL and everything allocated is released. */
int tnlbm_create(const tnlbm_config *cfg, tnlbm_sim **out);

/* Advance k >= 0 time steps (Sec. 3.2, Eq. evolution); synchronous. */
int tnlbm_step(tnlbm_sim *s, int k);

/* Contract the populations to dense fields (host, caller-owned, FP64):
 * rho[N^3] = sum_i f_i and u[3][N^3] = (sum_i c_i f_i + F (1 - m_O)/2) / rho
 * where rho > 0.5, else 0.  Either pointer may be NULL.  Synchronous. */
int tnlbm_macroscopic(tnlbm_sim *s, double *rho, double *u);

/* The plane coordinate[axis] = index (axis 0..2 = x, y, z) of the same
 * fields, contracted from the MPS with that axis's sites fixed (no N^3 field
 * is formed; for large N where rho and u do not fit host memory):
 * rho[N^2], u[3][N^2], indexed [a][b] with a, b the two other coordinates in
 * increasing axis order.  Host buffers, caller-owned; NULL skips a field.
 * Synchronous. */
int tnlbm_macroscopic_slice(tnlbm_sim *s, int axis, int index, double *rho, double *u);

/* Populations as MPS: host buffers of Q * tnlbm_mps_size(L, chi_max) doubles
 * (flat layout, capacity chi_max, population-major) and Q*(L+1) ints.
 * get = checkpoint, set = resume / custom initial state. Synchronous. */
int tnlbm_get_populations(tnlbm_sim *s, double *cores, int *ranks);
int tnlbm_set_populations(tnlbm_sim *s, const double *cores, const int *ranks);

int tnlbm_stats_get(tnlbm_sim *s, tnlbm_stats *out);

/* Inlet velocity u_b of a TNLBM_FACE_VELOCITY face (0..5) from the next step
 * on (a time-dependent inflow sets it before every step); synchronous. */
int tnlbm_set_face_velocity(tnlbm_sim *s, int face, const double *u);

/* Change the Jacobi sweep limit and the cross-CTA wait limit of every rounding
 * of the simulation's step from the next step on (meaning and defaults as the
 * tnlbm_config members jacobi_max_sweeps and wait_limit_ns; >= 0).  A step
 * whose Jacobi reaches the limit returns TNLBM_E_NOCONV, one whose wait runs
 * out TNLBM_E_TIMEOUT; either way the simulation stays valid for
 * tnlbm_destroy (its populations are then unreliable).  Synchronous. */
int tnlbm_set_limits(tnlbm_sim *s, int jacobi_max_sweeps, long long wait_limit_ns);

/* Advance k steps through the captured graph and return the device time of
 * the k launches in *ms (CUDA events on the simulation's stream). */
int tnlbm_step_timed(tnlbm_sim *s, int k, double *ms);

/* ------------------------------------------------------------------ cluster sizes
 * Each dependency level of a step is one rounding launch.  In TNLBM_FP64,
 * TNLBM_MIXED and TNLBM_BF16 a job of that launch runs on a thread-block
 * cluster of P CTAs (1 <= P <= TNLBM_CLUSTER_MAX) that share its FP64 centre
 * SVDs.  tnlbm_create picks P per level from occupancy (the largest size at
 * which every job of the level is resident at once, capped by
 * tnlbm_config.max_cluster); these calls read, set or measure it. */
enum { TNLBM_CLUSTER_MAX = 16 };

/* Per-level cluster sizes: clusters[l] (0 for a level without roundings) and
 * jobs[l] (the rounding jobs of level l) for l < min(cap, levels); either
 * array may be NULL; *nlevels (may be NULL) = the number of levels.  Host
 * only. */
int tnlbm_clusters(tnlbm_sim *s, int *clusters, int *jobs, int cap, int *nlevels);

/* Sets the cluster size of every level with roundings from
 * clusters[0..nlevels) (nlevels must equal the level count; entries of levels
 * without roundings are ignored) and re-captures the step's graph.  Each size
 * is 1..16 and fits on the device; FP32 and TF32 simulations take 1 only.
 * Otherwise TNLBM_E_ARG with nothing changed.  Synchronous. */
int tnlbm_set_clusters(tnlbm_sim *s, const int *clusters, int nlevels);

/* Measures the cluster size of every level.  Runs one step eagerly, level by
 * level, and times each rounding launch (CUDA events; the minimum of reps >= 1
 * launches) at the level's current size, at P = 16, 8, 4, 2, 1 (going down
 * until a size is 1.5x slower than the best so far), then at 3/4 and 3/2 of
 * the fastest, among the sizes <= tnlbm_config.max_cluster that fit on the
 * device.  Each level keeps its fastest
 * size (the current one unless another is 2 % faster); the graph is then
 * re-captured.  The step's copy into the populations (and the mass correction
 * before it) is left out: the populations, the step count and the total
 * discarded weight are unchanged.  ms (may be NULL; ms_cap doubles):
 * ms[l * (TNLBM_CLUSTER_MAX + 1) + P] = level l's launch time at P CTAs per
 * job in ms, -1 where not timed.  FP32 / TF32 simulations time nothing.  Not
 * allowed once the learned rounding is configured (TNLBM_E_ARG); a failing
 * rounding returns its code and keeps the old sizes.  Synchronous. */
int tnlbm_tune_clusters(tnlbm_sim *s, int reps, double *ms, int ms_cap);

/* Kernel classes reported by tnlbm_profile_step (array index). */
enum { TNLBM_K_ROUND = 0, TNLBM_K_FIT_GEMM = 1, TNLBM_K_FIT_QR = 2, TNLBM_K_FIT_MISC = 3,
       TNLBM_K_RHO0 = 4, TNLBM_K_COPY = 5, TNLBM_K_ZIPUP = 6, TNLBM_K_COUNT = 7 };

/* Advance one step with eager (non-graph), serialised launches and report per
 * kernel class: device milliseconds ms[TNLBM_K_COUNT] (CUDA events after every
 * launch), algorithmic FLOPs flops[] (counted on the device from the realised
 * bonds: 2MNK per GEMM, LAPACK-style counts for QR and SVD), and launches[].
 * phases (nullable, 22 doubles): SM cycles of the rounding kernel's phases
 * summed over its jobs: term formation, R*W product, QR, Jacobi, SVD outputs,
 * Q*US product (indices 0..5); Jacobi sweeps and SVD count (6, 7); Jacobi
 * cycles and count of the SVDs whose matrices did not fit in shared memory
 * (8, 9); FLOPs of the FP64 centre SVDs of TNLBM_MIXED / cluster runs: the
 * algorithmic (Golub-Kahan) count 4 M N^2 + 8 N^3 (10) and the FP64 FLOPs
 * the cluster Jacobi executed (11); cycles of the cluster Jacobi's FP64
 * sweeps (leader CTA) in the column norms, forming and sending the pair inner
 * products, waiting for the other CTAs' parts, the rotation angles and the
 * rotations (12..16); for TNLBM_MIXED the cycles of the leader's FP32 sweeps,
 * of the Newton-Schulz step and of the product X V that start the FP64
 * sweeps, and the FP32 sweeps (17..20); rounds of the FP64 cluster sweeps
 * (21). */
int tnlbm_profile_step(tnlbm_sim *s, double *ms, double *flops, int *launches, double *phases);
int tnlbm_destroy(tnlbm_sim *s); /* NULL-safe */
const char *tnlbm_last_error(void);

/* ------------------------------------------------------------ layout helpers */

size_t tnlbm_mps_size(int L, int cap);      /* elements of one flat MPS  */
size_t tnlbm_mps_offset(int L, int cap, int k); /* element offset of core k */

/* ------------------------------------------------------------ primitives
 * Batched operations on caller-owned DEVICE buffers in the flat layout.
 * Pointer arrays ("const void *const *src" etc.) are HOST arrays of length
 * `batch` holding device pointers.  All MPS of one call have L = 3*n_bits. */

enum {
  TNLBM_TERM_PLAIN = 0, /* coef * X                                           */
  TNLBM_TERM_SHIFT = 1, /* coef * S X: 1-D shift MPO along `axis` (Sec. 2.5),
                           (S X)(x) = X(x + offset e_axis), offset = +1 / -1,
                           cyclic (S) or non-cyclic (S^, zero where x+offset
                           leaves the domain)                                 */
  TNLBM_TERM_MASK1 = 2, /* coef * (m . X), m a rank-1 MPS given by per-site
                           2-vectors mask[k][2] (exact product, Eq. mul)      */
  TNLBM_TERM_KRON = 3,  /* coef * (X . Y) exact product by Eq. (mul)          */
  TNLBM_TERM_ONES = 4   /* coef * 1, the rank-1 all-ones MPS                  */
};

typedef struct {
  int kind;
  double coef;
  const void *x; const int *x_ranks; int x_cap; /* device MPS (not for ONES) */
  const void *y; const int *y_ranks; int y_cap; /* KRON second factor        */
  int axis, offset, cyclic;                     /* SHIFT                     */
  const double *mask;                           /* MASK1: host [L][2]        */
} tnlbm_term;

/* dst[b] = round(sum_t terms[b*nterms + t]) : block-diagonal sum (Eq. add) of
 * the (exactly formed) terms, then a left-orthogonalising QR sweep and a
 * right-to-left truncated SVD sweep (Eq. svd-move) with bond cap chi_max and
 * relative tolerance eps.  dst capacity must be >= chi_max.  TNLBM_BF16 rounds
 * as TNLBM_MIXED (a rounding has no contraction that BF16 would take). */
int tnlbm_lincomb_round(int precision, int n_bits, int batch, int nterms,
                        const tnlbm_term *terms, void *const *dst,
                        int *const *dst_ranks, int dst_cap, int chi_max,
                        double eps, void *stream);

/* Same result as tnlbm_lincomb_round, for callers that cannot allocate device
 * memory at the point of the call: code whose device memory is entirely held
 * by a pool allocator, and code that must not stall the device (cudaFree
 * synchronises it).  The paper has no counterpart to this entry point.
 * It calls no cudaMalloc / cudaFree: its workspace is a fixed 16 MiB array, a
 * table of 64 jobs and 64 rank-1 masks in the library's static device memory,
 * held by every GPU that loads the library until the process exits.  Requests
 * that need more return TNLBM_E_ARG with a message.  All calls share these
 * arrays (and fixed host staging tables): calls whose work overlaps on the GPU,
 * or that come from several host threads at once, race.  The status word is
 * cleared at the start of each call.  The first call on a device looks up the
 * arrays' device addresses (cudaGetSymbolAddress) and should come before any
 * stream capture that includes this call.  Synchronous on `stream`. */
int tnlbm_lincomb_round_noalloc(int precision, int n_bits, int batch, int nterms,
                                const tnlbm_term *terms, void *const *dst,
                                int *const *dst_ranks, int dst_cap, int chi_max,
                                double eps, void *stream);

/* dst[b] = the single term, formed exactly without rounding (bond grows:
 * SHIFT doubles it inside the axis span, KRON multiplies bonds). */
int tnlbm_materialize(int precision, int n_bits, int batch,
                      const tnlbm_term *terms, void *const *dst,
                      int *const *dst_ranks, int dst_cap, void *stream);

/* A[b] ~ B[b] . C[b] by the zip-up pass, the alternative to the fit that
 * Sec. 2.3 names: copies of B and C are brought to right-canonical form, one
 * left-to-right pass contracts each site's product core into the carried
 * matrix and truncates it (QR of the unfolding, Jacobi SVD of R, chi_max and
 * the tail rule with delta = eps ||T_0|| / sqrt(L-1), T_0 the first site's
 * unfolding), and the result is rounded (chi_max, eps) into A.  Caps of B and
 * C <= 512, chi_max <= 512, capA >= chi_max; B and C are not modified.
 * Allocates its scratch (cudaMalloc) and synchronises `stream`.
 * Not in the paper's own runs (it uses the fit). */
int tnlbm_hadamard_zipup(int precision, int n_bits, int batch,
                         const void *const *B, const int *const *rB, int capB,
                         const void *const *C, const int *const *rC, int capC,
                         void *const *A, int *const *rA, int capA, int chi_max,
                         double eps, void *stream);

/* A[b] ~ B[b] . C[b] by the single-site variational fit of Sec. 2.3: candidate
 * A = B (bonds unchanged), `sweeps` round trips of local updates and QR/LQ
 * centre shifts.  A must have capacity >= B's.  precision TNLBM_TF32 /
 * TNLBM_BF16: float buffers, the contractions on the tensor cores (TF32 or
 * BF16 operands, FP32 sums); TNLBM_MIXED: float buffers, FP32 contractions. */
int tnlbm_hadamard_fit(int precision, int n_bits, int batch,
                       const void *const *B, const int *const *rB, int capB,
                       const void *const *C, const int *const *rC, int capC,
                       void *const *A, int *const *rA, int capA, int sweeps,
                       void *stream);

/* out[b] (device doubles) = <X[b], 1>, the sum of all entries (Sec. 3.2). */
int tnlbm_inner_ones(int precision, int n_bits, int batch,
                     const void *const *X, const int *const *rX, int capX,
                     double *out, void *stream);

/* dense[x][y][z] (device, N^3 elements of the precision's type) = contraction
 * of the MPS (Eq. MPS). */
int tnlbm_to_dense(int precision, int n_bits, const void *X, const int *rX,
                   int capX, void *dense, void *stream);

/* TT-SVD of a dense device field [x][y][z] into an MPS (Eq. svd-comp, the mask
 * builder), truncating each bond to chi_max / eps.  The singular values come
 * from FP64 Gram matrices, so tails below ~1e-8 of the norm are not resolved. */
int tnlbm_from_dense(int precision, int n_bits, const void *dense, void *dst,
                     int *dst_ranks, int dst_cap, int chi_max, double eps,
                     void *stream);

/* Mask combined on separate length scales (App. D): an inner geometry on a
 * (2^n_inner)^3 grid repeated where an outer mask on a (2^n_outer)^3 grid is
 * one, i.e. m(x) = m_outer(x >> n_inner) m_inner(x mod 2^n_inner) per axis, on
 * (2^(n_outer + n_inner))^3 cells.  Each part is compressed on its own grid
 * (TT-SVD as tnlbm_from_dense, chi_max / eps relative to its own norm) and the
 * outer cores are followed by the inner ones: the largest bond is the larger
 * of the two, with bond 1 at the junction, and no dense field of the combined
 * size is formed.  outer_dense / inner_dense: DEVICE [x][y][z] arrays of the
 * precision's type; dst: DEVICE MPS of L = 3 (n_outer + n_inner) sites and
 * capacity dst_cap >= chi_max.  Allocates temporaries; synchronous. */
int tnlbm_mask_product(int precision, int n_outer, const void *outer_dense,
                       int n_inner, const void *inner_dense, void *dst,
                       int *dst_ranks, int dst_cap, int chi_max, double eps,
                       void *stream);

/* ------------------------------------------------------------------ batched simulations
 * Several independent simulations (same precision and fit sweeps; lattice
 * size, velocity set, geometry, walls, tau, force, chi, eps and start may
 * differ) stepped together: each dependency level of the step (Sec. 3.2)
 * launches the roundings and fits of that level of every simulation at once,
 * and one CUDA graph holds the whole batched step.  The paper runs one simulation at a
 * time; results are bitwise those of the simulations stepped alone when the
 * rounding launches use the same cluster sizes (always in TNLBM_FP32 and
 * TNLBM_TF32, where every job runs on one CTA). */
typedef struct tnlbm_batch tnlbm_batch; /* opaque; owns its simulations */

/* Creates cfgs[0..nsim) (1 <= nsim <= 64) as for tnlbm_create.  Batched steps
 * round with the full truncated SVD: every learned_rank must be 0
 * (TNLBM_E_ARG otherwise).  On error no simulation is left allocated. */
int tnlbm_batch_create(const tnlbm_config *cfgs, int nsim, tnlbm_batch **out);
/* k batched steps; synchronous; device status checked after the last. */
int tnlbm_batch_step(tnlbm_batch *b, int k);
/* k batched steps timed with CUDA events on the batch's stream (ms). */
int tnlbm_batch_step_timed(tnlbm_batch *b, int k, double *ms);
/* Borrowed handle of simulation i (owned by the batch: never destroy it).
 * tnlbm_macroscopic / get / set populations / stats work on it between
 * batched steps; stepping it alone is allowed too.  NULL on bad arguments. */
tnlbm_sim *tnlbm_batch_sim(tnlbm_batch *b, int i);
/* Simulations, kernel launches per batched step, jobs (roundings + fits) per
 * batched step; any pointer may be NULL. */
int tnlbm_batch_info(tnlbm_batch *b, int *nsim, int *launches_per_step,
                     int *jobs_per_step);
/* tnlbm_clusters / tnlbm_set_clusters / tnlbm_tune_clusters for the batched
 * step, whose rounding launch of a level holds the jobs of every simulation;
 * the cap is the smallest max_cluster of the simulations.  Tuning leaves every
 * simulation's populations, step count and discarded weight unchanged. */
int tnlbm_batch_clusters(tnlbm_batch *b, int *clusters, int *jobs, int cap, int *nlevels);
int tnlbm_batch_set_clusters(tnlbm_batch *b, const int *clusters, int nlevels);
int tnlbm_batch_tune_clusters(tnlbm_batch *b, int reps, double *ms, int ms_cap);
int tnlbm_batch_destroy(tnlbm_batch *b);

/* ------------------------------------------------------------------ learned rounding
 * Not part of the paper: the full SVD of each right-to-left step of the
 * rounding (Eq. svd-move) may be replaced by a randomized truncation at a
 * target rank k, which is accepted only when its error is certified.
 *   l = min(max(k + oversample, 16), m, n) samples;  Y = C Omega[:n, :l];
 *   `power` times: Y = C orth(C^T orth(Y))  (orth = Householder Q factor);
 *   Q = orth(Y);  B = Q^T C;  B = U S V^T (one-sided Jacobi);
 *   err(r)^2 = ||C - Q B||_F^2 + sum_{j>=r} s_j^2  (exact, measured);
 *   r = smallest rank <= chi_max with err(r) <= delta (delta as in the full
 *   rounding), accepted iff that rule is met inside the sample (or r reaches
 *   chi_max) and either err(r) <= delta or ||C - Q B||^2 <= max(eta err(r)^2,
 *   (floor_rel ||C||_F)^2) -- the latter proves err(r)^2 <= opt(r)^2/(1-eta)
 *   (Ky Fan on C^T C = B^T B + E^T E); otherwise the full SVD runs on C.
 * C is the m x n centre matrix of the step.  Omega is a fixed Gaussian matrix
 * supplied by the caller (row-major, omega_rows x omega_ld); the randomized
 * path is skipped where n > omega_rows or l > omega_ld. */

/* tnlbm_lincomb_round with the randomized truncation at given target ranks.
 * targets: host, batch x (3 n_bits + 1) ints, entry k = target at bond k
 * (0 = full SVD there; entries 0 and L are ignored).  omega: DEVICE array of
 * the precision's type.  counters (host int[3], may be NULL) receives
 * accepted / fell back / full-SVD step counts.  0 < eta < 1, floor_rel >= 0,
 * 0 <= power <= 4.
 * Synchronous on `stream`. */
int tnlbm_lincomb_round_rsvd(int precision, int n_bits, int batch, int nterms,
                             const tnlbm_term *terms, void *const *dst,
                             int *const *dst_ranks, int dst_cap, int chi_max,
                             double eps, const int *targets, const void *omega,
                             int omega_rows, int omega_ld, int oversample,
                             int power, double eta, double floor_rel,
                             int *counters, void *stream);

/* Rank model: 18 -> 64 -> 64 -> 1 ReLU network mapping a bond's features
 * (top-16 log10 singular values of the previous step relative to the largest,
 * padded with -20; bond / L; min(step / 1000, 1)) to retained rank / chi_max.
 * Parameters: one flat array of tnlbm_mlp_param_count() values, W1[64][18],
 * b1[64], W2[64][64], b2[64], W3[64], b3.  Forward and backward passes use the
 * parameters rounded to FP16, with FP32 arithmetic.  All pointers are DEVICE
 * pointers; X is M x 18 row-major FP32, y and out are M FP32 values.
 * Asynchronous on `stream`. */
int tnlbm_mlp_param_count(void);
int tnlbm_mlp_forward(const float *params, int M, const float *X, float *out,
                      void *stream);
/* loss = mean (out - y)^2 (device float), grad = d loss / d params (device). */
int tnlbm_mlp_loss_grad(const float *params, int M, const float *X,
                        const float *y, float *loss, float *grad, void *stream);
/* `iters` Adam steps (beta 0.9 / 0.999, eps 1e-8, rate lr) on minibatches of
 * `batch` consecutive samples (cyclic over the M samples; shuffle beforehand),
 * starting at Adam step step0 (0 for a fresh start).  master (FP32), adam_m and
 * adam_v (zero for a fresh start) are updated in place; half_out (device
 * __half[param_count], may be NULL) receives the FP16 copy after every step;
 * loss_hist (device float[iters], may be NULL) the minibatch losses. */
int tnlbm_mlp_train(float *master, float *adam_m, float *adam_v, void *half_out,
                    int M, const float *X, const float *y, int iters, int batch,
                    int step0, float lr, float *loss_hist, void *stream);

/* Learned rounding inside a simulation.  mode 0: off (the default; the step is
 * unchanged).  mode 1: every rounding step logs its spectrum; from the second
 * step on, each step also appends one training row per bond (the 18 features
 * of the previous step's spectrum at that bond, then the rank kept now /
 * chi_max) to a device log of dataset_cap rows.  mode 2: as mode 1, and the
 * rank model (tnlbm_learn_set_mlp, required first) predicts each bond's target
 * rank from the previous step's spectrum for the randomized truncation above.
 * mode 3: as mode 2 with the previous step's kept rank as the target (the
 * baseline the rank model is measured against).
 * omega: HOST doubles, omega_rows >= 2 chi_max.  Re-captures the step graph;
 * clears the logs and counters. */
int tnlbm_learn_configure(tnlbm_sim *s, int mode, const double *omega,
                          int omega_rows, int omega_ld, int oversample,
                          int power, double eta, double floor_rel,
                          int dataset_cap);
/* Copies the FP16 rank model (host or device pointer, param_count values). */
int tnlbm_learn_set_mlp(tnlbm_sim *s, const void *params_f16);
/* Copies up to cap logged rows (19 floats each) to out (host or device);
 * *count = rows logged so far (may exceed the log's capacity). */
int tnlbm_learn_dataset(tnlbm_sim *s, float *out, int cap, int *count,
                        int reset);
/* out[0..2]: randomized truncations accepted, fallen back, full SVDs. */
int tnlbm_learn_counters(tnlbm_sim *s, long long *out, int reset);

#ifdef __cplusplus
}
#endif
#endif /* TNLBM_H */
