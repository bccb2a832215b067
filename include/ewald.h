/*
 * ewald.h - C ABI of the GB300 Ewald summation library (libewald.so).
 *
 * The library evaluates the classical Ewald sum of the paper "Long range forces in a
 * performance portable Molecular Dynamics framework" (arXiv 1708.01135): Coulomb energy and
 * forces of N point charges in a periodic cubic box of side L (Section 3.1, Eq. 2), split
 * into
 *   - a real-space pair sum of erfc-screened charges inside a cutoff r_c
 *     (Section 3.1.1; Eq. 4; Listing 1),
 *   - a reciprocal-space sum over the wave vectors k = 2 pi m / L, m in Z^3, m != 0,
 *     |m|^2 <= k_max^2 (Section 3.1.2; the two matrix-vector products of Eq. 3, built as
 *     structure factors S(k) = sum_j q_j exp(i k.r_j) (Algorithm 1) and scattered back to
 *     every particle as forces and potentials (Algorithm 2)),
 *   - the self-energy term (Section 3.2.2).
 * Units are Gaussian with the Coulomb constant 1.  The k = 0 term is dropped (neutral
 * systems only, footnote of Section 3.1.2): the conducting ("tin-foil") boundary condition.
 *
 * Splitting parameter: every call takes beta (1/length), the coefficient inside erfc.  The
 * paper writes the Gaussian exponent alpha = beta^2 (erfc(sqrt(alpha) r)).
 *
 * Conventions for every function:
 *   - Positions are float64, array-of-structs [n][3] (x, y, z); charges float64 [n];
 *     forces float64 [n][3] in the caller's particle order.  Positions may lie outside
 *     [0, L): they are wrapped (x - L floor(x / L)).
 *   - "dev" pointers are CUDA device pointers on the current device; "host" pointers are
 *     host memory (pinned or pageable).  The caller owns every buffer it passes; the library
 *     owns the plan and server objects and their device workspaces.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - No exception or longjmp crosses this ABI; every fallible call returns an
 *     ewald_status code, and ewald_strerror() names it.
 *   - A plan is not thread-safe: one plan, one stream at a time.  Distinct plans are
 *     independent.
 */
#ifndef EWALD_H
#define EWALD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ewald_plan *ewald_plan_t;     /* opaque, library-owned */
typedef struct ewald_server *ewald_server_t; /* opaque, library-owned */

typedef enum ewald_status {
    EWALD_OK = 0,
    EWALD_PENDING = 1,          /* ewald_poll: the request has not finished yet            */
    EWALD_E_INVAL = -1,         /* bad argument (NULL pointer, L <= 0, k_max < 1, ...)     */
    EWALD_E_NONNEUTRAL = -2,    /* |sum q| > 1e-10 sum |q|: the paper treats neutral only  */
    EWALD_E_CUTOFF = -3,        /* r_c > L/2 (minimum image) or r_c <= 0                   */
    EWALD_E_NOMEM = -4,         /* device or host allocation failed / over the HBM budget  */
    EWALD_E_CUDA = -5,          /* a CUDA runtime call failed                              */
    EWALD_E_TIMEOUT = -6,       /* a bounded wait gave up (device pipeline or server)      */
    EWALD_E_BUSY = -7,          /* server: no free slot / queue full                       */
    EWALD_E_NOTFOUND = -8,      /* server: unknown or already collected ticket             */
    EWALD_E_NONFINITE = -9,     /* a position or charge is NaN or infinite                 */
    EWALD_E_UNSUPPORTED = -10   /* parameters outside what this build implements           */
} ewald_status;

/* Most particle types of the Lennard-Jones pair table (ewald_set_lj). */
#define EWALD_LJ_MAX_TYPES 8

typedef enum ewald_precision {
    /* FP64 everywhere on CUDA cores: real-space pairs, per-axis phase recurrences,
     * structure factors and back-scatter as FP64 products.  The plain FP64 GPU Ewald. */
    EWALD_FP64 = 0,
    /* Real-space pairs in FP32 on cell-local coordinates; S(k) and the force back-scatter
     * as complex matrix products on the tcgen05 tensor cores with every operand split into
     * two FP16 terms (hi + lo, three products per term pair) and FP32 accumulation; FP64
     * base phases, per-k energy and all global reductions. */
    EWALD_MIXED = 1,
    /* As EWALD_MIXED with BF16 instead of FP16 operand terms (wider range, 8 fewer
     * mantissa bits per term). */
    EWALD_MIXED_BF16 = 2,
    /* FP32 on CUDA cores for pairs and for the matrix products (no tensor cores). */
    EWALD_FP32 = 3
} ewald_precision;

/* Bit mask selecting the parts of the sum that ewald_compute_async evaluates. */
enum {
    EWALD_PART_REAL = 1,   /* real-space pairs                                   */
    EWALD_PART_RECIP = 2,  /* reciprocal space (S(k), energy, back-scatter)      */
    EWALD_PART_SELF = 4,   /* self-energy                                        */
    EWALD_PART_ALL = 7
};

/* Index of every entry of an energy[4] array. */
enum { EWALD_E_REAL = 0, EWALD_E_RECIP = 1, EWALD_E_SELF = 2, EWALD_E_TOTAL = 3 };

/*
 * ewald_create - make a plan for a box and a set of Ewald parameters.
 *   L          box side (> 0)
 *   beta       splitting parameter (> 0, 1/length); the paper's alpha is beta^2
 *   r_c        real-space cutoff, 0 < r_c <= L/2 (pairs with distance < r_c are summed,
 *              strict inequality as in Listing 1)
 *   k_max      integer reciprocal cutoff: m != 0 with |m|^2 <= k_max^2 (1 <= k_max <= 127)
 *   precision  one of ewald_precision
 *   out        receives the plan
 * The plan holds the cell grid (cell side >= r_c / 2 where the box allows), the half-space
 * k set and its row tables, and device workspaces that grow on the first compute with a
 * larger n.  Uses the device current at creation; every later call must run with that
 * device current.  Returns EWALD_OK, EWALD_E_INVAL, EWALD_E_CUTOFF, EWALD_E_UNSUPPORTED,
 * EWALD_E_NOMEM or EWALD_E_CUDA.
 */
int ewald_create(double L, double beta, double r_c, int k_max, int precision, ewald_plan_t *out);

/* ewald_destroy - free a plan and its device memory (synchronises its last stream).
 * NULL is ignored. */
void ewald_destroy(ewald_plan_t plan);

/*
 * ewald_compute - one energy + force evaluation, device buffers, synchronous energies.
 *   pos     dev float64 [n][3]
 *   q       dev float64 [n]
 *   forces  dev float64 [n][3], overwritten with F_i = -dU/dr_i (all three parts)
 *   energy  host float64 [4]: real, reciprocal, self, total (EWALD_E_* indices)
 *   stream  cudaStream_t (void*)
 * Launches the whole pipeline on `stream`, then synchronises that stream to return the
 * energies and the validation status.  n == 0 gives zero energies.  Errors:
 * EWALD_E_INVAL, EWALD_E_NONNEUTRAL, EWALD_E_NONFINITE (checked on the device, reported
 * here), EWALD_E_NOMEM (workspace growth), EWALD_E_TIMEOUT (a bounded device wait gave
 * up), EWALD_E_CUDA.  On a validation error forces and energies are unspecified.
 */
int ewald_compute(ewald_plan_t plan, int64_t n, const double *pos, const double *q,
                  double *forces, double energy[4], void *stream);

/*
 * ewald_compute_async - as ewald_compute, but fully asynchronous on `stream`.
 *   energy_dev  dev float64 [4] (real, reciprocal, self, total), written on the stream
 *   parts       EWALD_PART_* mask; forces and energies contain only the selected parts
 *               (unselected energy entries are 0)
 * Host-side argument errors are returned immediately.  Device-side validation (neutrality,
 * finiteness) and bounded-wait timeouts are recorded in the plan and returned by the next
 * ewald_status_sync() call.  Workspace growth (the first call with a larger n) allocates
 * device memory and is therefore not capturable in a CUDA graph; later calls with n no
 * larger than before allocate nothing.
 */
int ewald_compute_async(ewald_plan_t plan, int64_t n, const double *pos, const double *q,
                        double *forces, double *energy_dev, int parts, void *stream);

/*
 * ewald_compute_phi_async - as ewald_compute_async, and also the electrostatic potential at
 * every particle (the per-particle u of Algorithm 2 for the reciprocal part, phi of Eq. 4 for
 * the real-space part):
 *   phi_dev  dev float64 [n], caller order: phi_i = phi_i^real + phi_i^recip - 2 beta q_i /
 *            sqrt(pi) over the selected parts, the potential at r_i of all other charges and of
 *            all periodic images, so that the total energy is 1/2 sum_i q_i phi_i (the last
 *            term is each particle's share of the self energy).
 * Errors as ewald_compute_async; phi_dev may not be NULL when n > 0.
 */
int ewald_compute_phi_async(ewald_plan_t plan, int64_t n, const double *pos, const double *q,
                            double *forces, double *phi_dev, double *energy_dev, int parts,
                            void *stream);

/*
 * ewald_compute_virial_async - as ewald_compute_async, and also the virial tensor of every
 * part: W_ab = -dE/d(eps_ab), the derivative of the energy when the box and all positions
 * are strained by (1 + eps) at fixed beta.  The configurational pressure tensor is W / V
 * (V = L^3); the paper states the energies and forces (Section 3.1, Eqs. 2-4) and this is
 * their strain derivative:
 *   real:  W_ab = 1/2 sum_i sum_{j,n} q_i q_j psi(d) d_a d_b / d over the pairs of Eq. 4,
 *          psi(d) = erfc(beta d)/d^2 + 2 beta/sqrt(pi) exp(-beta^2 d^2)/d, d_vec = r_i-r_j-nL;
 *   recip: W_ab = sum_{k in K_half} g(k) |S(k)|^2 [delta_ab - 2 k_a k_b (1/k^2 + 1/(4 beta^2))]
 *          (Eq. 3: V grows by tr eps, k shrinks by eps k, S(k) is unchanged);
 *   self:  zero (the self energy does not change under the strain at fixed beta).
 *   virial_dev  dev float64 [4][3][3]: the real, reciprocal and self tensors and their sum
 *               (selected parts only; unselected parts are zero), row-major and symmetric.
 *               For converged cutoffs tr W = E_total (the Coulomb energy is homogeneous of
 *               degree -1 in the coordinates).
 * The real-space kernel accumulates the six tensor entries next to the force in FP32 (mixed
 * precisions) or FP64; the reciprocal tensor is an FP64 sum over the modes of S(k).  Sums are
 * in a fixed order, so repeated calls give identical bits.
 * Errors as ewald_compute_async; virial_dev may not be NULL.
 */
int ewald_compute_virial_async(ewald_plan_t plan, int64_t n, const double *pos,
                               const double *q, double *forces, double *virial_dev,
                               double *energy_dev, int parts, void *stream);

/*
 * ewald_set_near_pairs - arithmetic of the near real-space Coulomb pairs of every later
 * evaluation of this plan (EWALD_MIXED, EWALD_MIXED_BF16 and EWALD_FP32 plans; FP64 plans
 * accept the call and are unchanged).  Near pairs are those with 0 < d < r_near,
 * r_near = min(2.5 (L^3 / n)^(1/3), r_c): the pairs that carry most of the force on a
 * particle (the real-space sum of Eq. 4, Section 2).
 *   double_float  0 (the default): FP32 with the exact r^2 (a first-order correction of the
 *                 pair terms for the rounding of r^2), about 1e-7 of every pair term;
 *                 1: double-float arithmetic (pairs of FP32 numbers), about 1e-8.
 * Where the net force on a particle is a small sum of large pair forces (ionic crystals)
 * the FP32 rounding of the near pairs is amplified: on a rock-salt crystal it gives about
 * 1e-6 of the RMS force with 0 and 2e-7 with 1; on disordered systems both are below
 * 2e-7.  Mode 1 costs a second scan of the staged candidates within r_near (measured on
 * GB300, real-space kernel alone: +15 % at 2,097,152 ions, r_c = 10.7; +30 % at 262,144,
 * r_c = 7.6; +80 % at 32,768, r_c = 4).  Returns EWALD_OK or EWALD_E_INVAL (NULL plan, a
 * mode other than 0 or 1).  Synchronises the plan's streams; not thread-safe against a
 * running evaluation of the same plan.
 */
int ewald_set_near_pairs(ewald_plan_t plan, int double_float);

/*
 * ewald_set_lj - fuse short-range Lennard-Jones pairs into the real-space kernel of every
 * later evaluation of this plan (the paper's NaCl benchmark adds such a repulsion to the
 * Coulomb sum, Section 4; its parameters are not printed, so they are the caller's).
 *   ntypes    0 (switch the pairs off; the other arguments are ignored) or
 *             1..EWALD_LJ_MAX_TYPES
 *   epsilon   host float64 [ntypes][ntypes], symmetric, >= 0 and finite (copied)
 *   sigma     host float64 [ntypes][ntypes], symmetric, > 0 and finite (copied)
 *   type_dev  dev int32 [n], the type of every particle in caller order, for the n of each
 *             later call.  NOT copied: the caller keeps it alive and unchanged while the plan
 *             evaluates with it (a type outside [0, ntypes) makes that evaluation report
 *             EWALD_E_INVAL through its device status, with the type taken as 0).
 * Every pair with 0 < d < r_c (the real-space cutoff, minimum image) adds the truncated and
 * shifted potential u(d) = 4 eps [(sigma/d)^12 - (sigma/d)^6] - u_0 with u_0 its value at r_c,
 * evaluated in the arithmetic of the real-space pairs (FP32 on the mixed and FP32 paths).
 * The Lennard-Jones force is part of the returned forces, its energy part of energy[3] (the
 * total potential energy) but not of energy[0..2], so E_LJ = energy[3] - energy[0] -
 * energy[1] - energy[2]; likewise its virial is part of the sum tensor of
 * ewald_compute_virial_async only.  The pairs are evaluated whenever EWALD_PART_REAL is
 * selected, and ewald_md integrates with them.
 * Synchronises the plan's streams.  Returns EWALD_E_INVAL for bad arguments.
 */
int ewald_set_lj(ewald_plan_t plan, int ntypes, const double *epsilon, const double *sigma,
                 const int32_t *type_dev);

/*
 * ewald_set_spme - compute the reciprocal part of every later evaluation of this plan by
 * smooth particle-mesh Ewald (Essmann et al., J. Chem. Phys. 103, 8577 (1995)), the
 * successor that the paper names for large N (Sections 1 and 5), instead of the classical
 * sum over the k set of Eq. 3.  The real-space and self parts, the energies layout, the
 * forces, potentials, virial, Lennard-Jones pairs and ewald_md are unchanged; k_max is not
 * used while SPME is on, and ewald_structure_factor returns EWALD_E_UNSUPPORTED.
 *   K      mesh points per side (even order <= K <= 1024), or 0 to return to the classical sum
 *   order  B-spline order p: 4, 6, 8, 10 or 12
 * Charges are spread with p^3 weights per particle, brick by brick of the cell grid in shared
 * memory, and the brick sums are added to a fixed-point mesh (64-bit integer atomics, 2^-36
 * resolution), so results repeat bit for bit; an evaluation with sum |q| >= 2^26 reports
 * EWALD_E_UNSUPPORTED (the mesh could overflow).  The mesh, its
 * transforms (cuFFT) and the particle-side splines are FP32 on the mixed and FP32 plans,
 * FP64 on the FP64 plan.  The error of the mesh approximation falls with K and p (about
 * (beta L / (pi K))^p); it adds to the real-space and k-space truncation errors.
 * Synchronises the plan's streams; allocates the mesh (about 8 + 4 (or 8) x 2 bytes per
 * mesh point) and two cuFFT plans.  The first evaluation after a change of the particle
 * count or cell grid also sets the brick sizes of the spreading (host work only).  Returns EWALD_E_INVAL, EWALD_E_NOMEM,
 * EWALD_E_UNSUPPORTED (cuFFT plan failure) or EWALD_E_CUDA.
 */
int ewald_set_spme(ewald_plan_t plan, int K, int order);

/*
 * ewald_probe_timeout - diagnostic of the failure path of the device-side waits (not part of
 * the paper's method).  Every wait of the library's kernels on an asynchronous copy gives up
 * after about one second and records EWALD_E_TIMEOUT in the plan's status instead of hanging
 * the GPU.  This call launches, on `stream`, one warp that waits in the same way on a
 * barrier that nothing completes, so the next ewald_status_sync of the plan returns
 * EWALD_E_TIMEOUT (about one second later) and the device stays usable.  Returns
 * EWALD_E_INVAL for a null plan, EWALD_E_CUDA if the launch fails.
 */
int ewald_probe_timeout(ewald_plan_t plan, void *stream);

/*
 * ewald_fma_peak - measured fused multiply-add rate of the CUDA cores of the current device
 * (a diagnostic with no counterpart in the paper: the denominator of the roofline of the
 * arithmetic-bound pair kernels and of the CUDA-core reciprocal products).
 *   precision  EWALD_FP32 or EWALD_FP64 (anything else: EWALD_E_INVAL)
 *   tflops     host out: TFLOP/s (two flops per FMA) of a bounded FMA loop on every SM,
 *              timed with CUDA events (synchronous; a few tenths of a second)
 */
int ewald_fma_peak(int precision, double *tflops);

/* ewald_status_sync - synchronise the plan's last stream and return (and clear) the
 * device-side status of the last evaluation: EWALD_OK, EWALD_E_NONNEUTRAL,
 * EWALD_E_NONFINITE, EWALD_E_TIMEOUT or EWALD_E_CUDA. */
int ewald_status_sync(ewald_plan_t plan);

/*
 * ewald_compute_host - end-to-end evaluation from host buffers: copies pos and q to the
 * device (plan-owned staging buffers), runs the pipeline, copies forces and the four
 * energies back, and synchronises.  pos, q, forces, energy are HOST pointers with the
 * same layouts as ewald_compute.  Pinned host memory gives asynchronous copies.
 */
int ewald_compute_host(ewald_plan_t plan, int64_t n, const double *pos_host,
                       const double *q_host, double *forces_host, double energy_host[4],
                       void *stream);

/*
 * ewald_profile - per-stage timing of later evaluations with CUDA events recorded on the
 * stream each stage runs on (off by default; recording adds a few event records per call).
 *   enable    1 to record from the next evaluation on, 0 to stop, -1 to leave unchanged
 *   times_ms  host float64 [EWALD_PROFILE_TIMES] or NULL: synchronises and returns the
 *             durations of the last recorded evaluation.  Spans between stage boundaries
 *             of one stream (they include waits for the other stream):
 *             [0] binning and packing (a1-a3), [1] from the end of binning to the end of
 *             the real-space pairs (the forward operands and the pair kernel, a4),
 *             [2] phases and structure-factor product (a5-a6), [3] S(k) reduction, energy
 *             and coefficients (a6-a7), [4] back-scatter product and its reduction (a8),
 *             [5] from the end of the real-space pairs to the end of the evaluation (the
 *             wait for the reciprocal branch, then a9), [6] whole evaluation,
 *             [7] reciprocal branch (stages 2-4 on their stream).
 *             Single kernels (bracketed by their own events): [8] the real-space pair
 *             kernel, [9] the back-scatter product kernel, [10] the self term, totals and
 *             unsort (a9) after the join.  -1 where a span was not recorded: [2]-[4], [7]
 *             and [9] when the evaluation had no reciprocal part, [9] for the mesh
 *             reciprocal part.
 *   launches  host int or NULL: kernels launched by the last evaluation
 */
#define EWALD_PROFILE_TIMES 11
int ewald_profile(ewald_plan_t plan, int enable, double times_ms[EWALD_PROFILE_TIMES],
                  int *launches);

/* ewald_plan_info - read plan parameters chosen at creation.
 *   info[0] = number of cells per side, info[1] = stencil half-width in cells
 *   (0 = all pairs with the minimum image), info[2] = |K_half|, info[3] = number of
 *   (m_y, m_z) rows, info[4] = k_max, info[5] = precision.  Any pointer may be NULL. */
int ewald_plan_info(ewald_plan_t plan, int64_t info[6]);

/*
 * ewald_kset - the plan's half-space k set K_half, in the order used by
 * ewald_structure_factor: m_z ascending, then m_y ascending, then m_x ascending; m != 0,
 * |m|^2 <= k_max^2, and (m_z > 0) or (m_z = 0, m_y > 0) or (m_z = m_y = 0, m_x > 0).
 *   m_host  host int32 [cap][3] or NULL;  *count receives |K_half|.
 * Writes min(cap, |K_half|) triples.
 */
int ewald_kset(ewald_plan_t plan, int32_t *m_host, int64_t cap, int64_t *count);

/* ewald_structure_factor - copy S(k) = sum_j q_j exp(i k.r_j) of the last evaluation
 * that included EWALD_PART_RECIP, as float64 (re, im) pairs [|K_half|][2] in ewald_kset
 * order, into the device buffer S_dev, on `stream`. */
int ewald_structure_factor(ewald_plan_t plan, double *S_dev, void *stream);

/* ewald_cell_sort - debug view of the integer binning of the last evaluation: copies, on
 * `stream`, the cell index of every particle in caller order (int32 [n], key =
 * (c_z n_c + c_y) n_c + c_x) and the sorted order (int32 [n]: slot s holds particle
 * perm[s]) into device buffers.  Either pointer may be NULL.  The order is stable by key;
 * where the FP32 real-space kernel cuts its ranges to x windows (stencil half-width >= 5,
 * r_c plus one cell side below L/2), every cell of at most 256 particles is then ordered
 * by round(x 2^32 / L) mod 2^32 relative to its centre's fraction, ties in key order. */
int ewald_cell_sort(ewald_plan_t plan, int32_t *key_dev, int32_t *perm_dev, void *stream);

/* Index of every entry of one ewald_md energy record (EWALD_MD_RECORD doubles). */
enum { EWALD_MD_REAL = 0, EWALD_MD_RECIP = 1, EWALD_MD_SELF = 2, EWALD_MD_POT = 3,
       EWALD_MD_KIN = 4, EWALD_MD_TOTAL = 5, EWALD_MD_RECORD = 6 };

/*
 * ewald_md - molecular dynamics with the Ewald forces: `steps` velocity-Verlet time steps
 * of N charges in the plan's periodic box, every step ending with a full evaluation (the
 * per-timestep force computation of Section 2.1; the paper benchmarks such time steps of
 * an NaCl system in Section 4).  Per step, with a = F / m:
 *     v <- v + (dt/2) a(x);   x <- x + dt v;   F <- forces at x (ewald_compute_async);
 *     v <- v + (dt/2) a(x)
 * The forces at the initial positions are evaluated first, so a call costs steps + 1
 * evaluations.
 *   pos         dev float64 [n][3], advanced in place (not wrapped: trajectories stay
 *               continuous; every evaluation wraps internally)
 *   vel         dev float64 [n][3], advanced in place
 *   q           dev float64 [n]
 *   mass        dev float64 [n] (every entry > 0), or NULL for unit masses
 *   dt          time step (> 0, finite); steps >= 0
 *   forces      dev float64 [n][3]: on return the forces at the final positions
 *   energy_log  dev float64 [steps + 1][EWALD_MD_RECORD] or NULL: record s holds, after s
 *               steps, E_real, E_recip, E_self, E_pot = their sum, the kinetic energy
 *               1/2 sum m v^2 and E_pot + E_kin (record 0: the initial state)
 *   stream      cudaStream_t; the call is asynchronous on it (it never synchronises except
 *               for the first call with a larger n, which grows the plan's workspaces)
 * Host-side argument errors are returned immediately (EWALD_E_INVAL).  Device-side
 * validation of every evaluation of the run (neutrality, finiteness, bounded waits) is
 * accumulated and returned by the next ewald_status_sync().  Every reduction has a fixed
 * order: repeated runs from the same state give bit-identical trajectories.
 */
int ewald_md(ewald_plan_t plan, int64_t n, double *pos, double *vel, const double *q,
             const double *mass, double dt, int steps, double *forces, double *energy_log,
             void *stream);

/*
 * ewald_tune - choose (beta, r_c, k_max) for a target relative RMS force error.
 *   n, L      particle count and box side
 *   tol       target relative RMS force error (e.g. 1e-6), 1e-15 < tol < 1e-1
 *   r_c       in: a fixed cutoff (> 0), or <= 0 to let the tuner choose; out: the cutoff
 *   beta, k_max  out
 * Both truncation errors decay as exp(-p^2) with p = beta r_c = pi k_max / (beta L)
 * (Section 3.1.3: r_c ~ alpha^-1/2, k_c ~ alpha^1/2); p is set from tol.  With r_c free,
 * the tuner picks r_c <= L/2 minimising a cost model of pair candidates plus k modes.
 * The tolerance is relative to the RMS force, and both the truncation errors and the RMS
 * force scale with the charges squared, so no sum of q^2 enters (the absolute-error forms
 * of the estimates that Section 3.1.3 points to carry one; for a relative target it
 * cancels).  r_c is an in/out argument so that a caller can fix the cutoff (a cell grid, a
 * Lennard-Jones range) and have beta and k_max follow.
 */
int ewald_tune(int64_t n, double L, double tol, double *r_c, double *beta, int *k_max);

/*
 * ewald_real_noalloc - the real-space part alone, without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers of this library that
 * cannot allocate device memory -- code running while a stream is being captured into a
 * CUDA graph (allocation is not allowed there), programs whose device memory is owned by
 * another allocator or capped by a quota, and latency-critical loops that must never enter
 * the allocator.  The plan-based calls above allocate workspaces on first use; this one
 * does not call cudaMalloc, cudaFree or any routine that allocates.
 *
 *   L, beta, r_c   as in ewald_create (0 < r_c <= L/2)
 *   n              0 <= n <= EWALD_NOALLOC_MAX_N particles; larger n returns
 *                  EWALD_E_UNSUPPORTED without doing anything
 *   pos, q         dev float64 [n][3], [n]
 *   forces         dev float64 [n][3], overwritten with the real-space forces (caller order)
 *   energy_dev     dev float64 [4]: E_real, 0, 0, E_real (the reciprocal and self parts are
 *                  not evaluated)
 *   stream         cudaStream_t; the call is asynchronous on it
 * Results equal ewald_compute_async(..., EWALD_PART_REAL) of an EWALD_FP64 plan up to
 * floating-point summation order (every pair is visited with the minimum image).  There is
 * no device-side validation: non-neutral input is not reported and non-finite input gives
 * non-finite output.
 *
 * Scratch: a fixed device array inside the library (packed particles and per-tile energy
 * partials for EWALD_NOALLOC_MAX_N particles, about 516 KB), present on every GPU that loads
 * the library until the process exits.  Every call shares it: calls whose GPU work overlaps
 * (different streams, or unordered calls from several host threads) race and give undefined
 * results.  Every call looks up the array's device address in the current context (a host
 * lookup that allocates nothing) and asks for its kernels' attributes, which loads them into
 * the context if they are not loaded yet; the first call on a device, with any n (n = 0
 * included), may therefore load the library's device code, so make it before any stream
 * capture.  A launch failure of this call returns EWALD_E_CUDA; errors left pending by other
 * work are not reported or cleared.
 */
#define EWALD_NOALLOC_MAX_N 16384
int ewald_real_noalloc(double L, double beta, double r_c, int64_t n, const double *pos,
                       const double *q, double *forces, double *energy_dev, void *stream);

/* ewald_strerror - static, NUL-terminated name of a status code. */
const char *ewald_strerror(int status);

/* ------------------------------------------------------------------------------------
 * Serving: continuous batching of independent Ewald evaluations.
 *
 * A server owns a scheduler thread, a pool of CUDA streams and a pool of reusable plans
 * ("slots").  ewald_submit() queues a request; the scheduler admits queued requests in
 * arrival order whenever a slot is free and the request's device footprint fits in the
 * remaining HBM budget, and launches its whole pipeline on the slot's stream, so that
 * requests admitted while others run overlap on the device.  ewald_poll() returns the
 * result once the request's stream has finished.
 * ---------------------------------------------------------------------------------- */

typedef struct ewald_request {
    double L, beta, r_c;
    int k_max;
    int precision;       /* ewald_precision */
    int64_t n;
    const double *pos;   /* dev [n][3]; must stay valid until ewald_poll returns final */
    const double *q;     /* dev [n] */
    double *forces;      /* dev [n][3], written by the server */
    void *stream;        /* cudaStream_t on which pos and q were produced (NULL: legacy
                            default stream); the request starts after the work queued on
                            it before ewald_submit */
} ewald_request;

typedef struct ewald_result {
    int status;          /* EWALD_OK or an error code of the evaluation */
    double energy[4];    /* real, reciprocal, self, total */
    double t_submit;     /* seconds on the server's monotonic clock */
    double t_admit;      /* when the scheduler launched the request */
    double t_done;       /* when the scheduler saw the request's stream finish */
    int64_t footprint_bytes; /* device memory charged against the budget */
} ewald_result;

/*
 * ewald_server_create - start a server on the current device.
 *   max_slots         concurrent requests on the device (1..64)
 *   hbm_budget_bytes  device memory the server may hold for request workspaces
 *                     (0 = 80 % of the free memory at creation)
 *   out               receives the server
 */
int ewald_server_create(int max_slots, size_t hbm_budget_bytes, ewald_server_t *out);

/* ewald_submit - queue a request (copied; the buffers it points to are not).  Returns
 * EWALD_OK and a ticket, EWALD_E_INVAL for a request that can never run (bad
 * parameters, footprint above the whole budget), or EWALD_E_BUSY when the queue is full. */
int ewald_submit(ewald_server_t srv, const ewald_request *req, uint64_t *ticket);

/* ewald_poll - non-blocking: EWALD_PENDING while queued or running; otherwise fills
 * *out, forgets the ticket and returns EWALD_OK (the request's own status is in
 * out->status).  EWALD_E_NOTFOUND for an unknown ticket. */
int ewald_poll(ewald_server_t srv, uint64_t ticket, ewald_result *out);

/* ewald_wait - blocking poll with a time limit in seconds; EWALD_E_TIMEOUT when it runs
 * out (the request stays queued or running and can be polled again). */
int ewald_wait(ewald_server_t srv, uint64_t ticket, double timeout_s, ewald_result *out);

/* ewald_server_stats - counters since creation: stats[0] submitted, [1] completed,
 * [2] admitted bytes now, [3] peak admitted bytes, [4] peak concurrent requests. */
int ewald_server_stats(ewald_server_t srv, int64_t stats[5]);

/* ewald_server_destroy - drain: wait for running requests, cancel queued ones (their
 * poll results are dropped), stop the scheduler and free everything. */
int ewald_server_destroy(ewald_server_t srv);

/*
 * ewald_server_simulate - replay the server's admission policy on the host with a simulated
 * executor (no device work; the policy function is the one the scheduler thread runs).
 * Request i (0 <= i < n, arrivals in non-decreasing t_arrive, index order at equal times)
 * holds footprint[i] bytes (<= budget) and runs for duration[i] seconds once admitted; a
 * finished slot keeps its memory until the policy reclaims it.  After every arrival or
 * completion the admission pass runs: first fit in arrival order on the idle slot holding the
 * most memory, idle slots' memory reclaimed while a request does not fit, and at most 64
 * admissions past a waiting head of the queue.  Writes order[k] = the k-th admitted request,
 * t_admit[i] = its admission time and *peak_held = the largest total held.  Returns
 * EWALD_E_INVAL for bad arguments.
 */
int ewald_server_simulate(int max_slots, int64_t budget, int n, const int64_t *footprint,
                          const double *t_arrive, const double *duration, int64_t *order,
                          double *t_admit, int64_t *peak_held);

#ifdef __cplusplus
}
#endif

#endif /* EWALD_H */
