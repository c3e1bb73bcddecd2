/*
 * susp.h -- C ABI of the GB300 library that advances the minimal
 * dense-suspension model of Li, Royer & Ness (arXiv 2307.13802):
 * spheres under contact forces with Coulomb-capped tangential history
 * (Sec. II.A, Eqs. 3-4), one-body Stokes drag (Sec. II.B, Eqs. 5-6),
 * regularised pairwise lubrication (Sec. II.B, Eqs. 8-18), one-body and
 * pairwise Brownian forces tied to those resistances (Sec. II.C,
 * Eqs. 19-24), integrated by Velocity-Verlet (Sec. II, Eqs. 1-2) in a
 * tilted periodic box sheared at a fixed rate with the strain flip of
 * Sec. II.E, and reporting the pair-virial stress (Sec. II.A, II.B, II.D).
 * Optional: the short-range repulsion of Sec. IV.E (Eq. 34) and the
 * structural Brownian stress of Sec. II.D (Eqs. 25-26) with its Green-Kubo
 * viscosity (Sec. III.D, Eq. 33).
 *
 * Conventions used by every call:
 *   - Particles are identified by their tag = index in the caller's arrays.
 *     For a batch of R replicas the tags of replica r are offset_r + local
 *     index, offset_r = sum of the sizes of the replicas before r.
 *   - Vectors are passed as row-major arrays of shape [count][3] (x, y, z).
 *     Host pointers are read or written in tag order whatever order the
 *     library keeps internally.
 *   - Flow x, gradient y, vorticity z; the imposed flow is
 *     U_inf = rate (y - Ly/2) x, Omega_inf = -(rate/2) z.  The box is
 *     [0,Lx) x [0,Ly) x [0,Lz) in the sliding-brick form of the tilted box:
 *     the image above in y is shifted by tilt = strain * Ly in x.
 *   - The force on sphere i from sphere j (i the lower tag, n the unit vector
 *     from i to j) is applied to i and its negative to j; the stress is
 *     sigma = (1/V) sum_pairs F_{i<-j} (x) r_ij (tension positive).
 *   - All calls are synchronous with respect to the host unless stated.
 *     One handle must not be used by two host threads at once.
 *   - Every call returns SUSP_OK or an error code; after an error the handle
 *     stays valid and susp_last_error() gives a message.  No call throws.
 *
 * Ownership: input arrays are copied before the call returns; the library
 * owns its device memory (allocated through the hook of
 * susp_set_allocator() if one is set, else cudaMalloc) and frees it in
 * susp_destroy().  Output arrays are caller-owned and must hold the stated
 * number of elements.
 */
#ifndef SUSP_H
#define SUSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SUSP_OK 0
#define SUSP_EINVAL 1    /* invalid argument (NULL, N <= 0, radius <= 0,    */
                         /* box < 3 list cutoffs, dt <= 0, kT < 0, mu < 0)  */
#define SUSP_ENOMEM 2    /* device or host allocation failed                */
#define SUSP_ECUDA 3     /* a CUDA runtime call failed                      */
#define SUSP_ESTATE 4    /* call order (e.g. step before set_state)         */
#define SUSP_ENEIGH 5    /* neighbour row exceeded its capacity (at 64, or  */
                         /* inside a call's steps before it could grow)     */
#define SUSP_EUNSTABLE 6 /* non-finite position/velocity or runaway overlap */
                         /* 7 is not used: no call waits on the device      */
                         /* with a time limit                               */
#define SUSP_ENODEV 8    /* no CUDA device is visible                       */

/* ---- parameters --------------------------------------------------------- */
#define SUSP_FP64 0  /* every step in double precision                      */
#define SUSP_MIXED 1 /* pair arithmetic in single precision on gaps formed  */
                     /* from double-float positions (pairs of floats, a    */
                     /* 48-bit significand); positions, velocities and the */
                     /* tangential history kept and integrated in          */
                     /* double-float; per-warp virial sums in single       */
                     /* precision, folded per block and summed over blocks */
                     /* and time in double                                 */

typedef struct susp_params {
  double eta;         /* liquid viscosity                                   */
  double rho;         /* particle density; m = 4/3 pi rho a^3, I = 2/5 m a^2 */
  double kn;          /* normal contact stiffness (Eq. 3)                   */
  double kt;          /* tangential stiffness (Eq. 3); used when mu > 0      */
  double mu;          /* static friction coefficient, 0 = frictionless       */
  double xi_min;      /* regularised gap xi_eff (paper: 1e-3)               */
  double xi_max;      /* lubrication cutoff on xi (paper: 0.05)             */
  double skin;        /* neighbour-list skin, length units                  */
  double shear_rate;  /* batch handles: this replica's shear rate           */
  double kT;          /* batch handles: this replica's thermal energy       */
  double torque_sign; /* sign of the chi term of T_ji in Eq. 24; -1 makes    */
                      /* the pair noise covariance (2kT/dt) R exactly        */
  double dt;          /* timestep used by susp_evaluate() before any step;  */
                      /* each susp_step*() call replaces it with its own dt */
  uint64_t seed;      /* batch handles: this replica's Philox key           */
  int32_t precision;  /* SUSP_FP64 or SUSP_MIXED                            */
  int32_t noise;      /* 1: Brownian terms on                               */
  int32_t lubrication;/* 1: lubrication and pair noise on                   */
  int32_t onebody;    /* 1: one-body drag and noise on                      */
  int32_t contact;    /* 1: contact forces on                               */
  int32_t sample_every;/* accumulate the stress every this many steps (>=1) */
  int32_t kmax;       /* initial neighbour row capacity (0: default 48);    */
                      /* it grows, up to 64, before a call whose rebuilds  */
                      /* could fill it: when a rebuild asked for by the    */
                      /* host (new state, skin or clock) overflows, and    */
                      /* when the last build's longest row came within a   */
                      /* quarter of it                                      */
  int32_t threads_per_particle; /* 0 = autotune, else 1, 2, 4 or 8          */
  int32_t use_graphs; /* 1: replay steps as CUDA graphs (default)           */
  int32_t structural; /* 1: sample the structural Brownian stress (Eq. 26)  */
  int32_t series_cap; /* per replica, samples of Sigma^B_xy kept for        */
                      /* Green-Kubo (0: none); needs structural = 1         */
  int32_t rebuild_every; /* n > 0: rebuild the neighbour list at least every */
                      /* n steps (the displacement bound of the skin may    */
                      /* rebuild sooner); 0: only when that bound requires  */
  double rep_A;       /* repulsion force scale A of Eq. 34 (0: off);        */
                      /* batch handles: this replica's A                    */
  double rep_cut;     /* repulsion acts for h <= rep_cut kappa,             */
                      /* kappa = 0.01 (a_i + a_j) (default 10)              */
  double shell;       /* structural shell Delta / a_i (paper: 0.05)         */
  int32_t deterministic; /* 0: force sums use atomics, so their order (and */
                      /* the last bits) may change from run to run; 1      */
                      /* (SUSP_FP64 only, kmax * N < 2^31): each pair's     */
                      /* shares go to its own slot and every sphere sums    */
                      /* them in a fixed order, so repeated runs are        */
                      /* bitwise equal (a step costs about 4% more at 1M    */
                      /* spheres; the reverse list takes 4 B per slot and  */
                      /* the shares 72 B per slot).                         */
                      /* The stress reductions are always in a fixed order  */
  int32_t autotune;   /* 1: the first step call of the handle runs          */
                      /* susp_autotune() over the skins 0.2, 0.3, 0.45,    */
                      /* 0.6 and 0.8 (100 trial steps each) and keeps the  */
                      /* fastest                                            */
} susp_params;

/* Fills *p with the defaults: eta = rho = 1, kn = 1e4, kt = 0, mu = 0,
 * xi_min = 1e-3, xi_max = 0.05, skin = 0.3, shear_rate = 1, kT = 0,
 * torque_sign = -1, dt = 1e-4, seed = 0, FP64, all terms on, sample_every = 1,
 * kmax = 48, autotuned threads per particle, graphs on, no repulsion
 * (rep_A = 0, rep_cut = 10), no structural stress (shell = 0.05), no series,
 * rebuild_every = 0, deterministic = 0, autotune = 0. */
void susp_default_params(susp_params* p);

typedef struct susp_s susp_t;

/* ---- lifetime ----------------------------------------------------------- */
/* One system of N spheres with the given radii (N doubles, all > 0; on the
 * mixed path at most 2^27 - 1 spheres in all, the capacity of a neighbour
 * entry's index field) in the
 * box [0,box[0]) x [0,box[1]) x [0,box[2]) with tilt 0.  Each box edge must
 * be at least three neighbour-list cutoffs, 3 * (2 a_max (1 + xi_max/2) +
 * skin).  Selects device 0 (or the current device).  Nothing is allocated on
 * the device until susp_set_state(). */
int susp_create(susp_t** out, int64_t N, const double* radii,
                const double box[3], const susp_params* p);

/* R independent replicas stepped together (Sec. II.E: ensembles of 10-800
 * realisations).  N_r[R] sizes, radii[sum N_r], boxes[R][3], p_r[R]
 * parameters (eta, rho, kn, kt, mu, shear_rate, kT, seed, rep_A may differ
 * per replica; xi_min, xi_max, skin, rep_cut, shell, series_cap, precision
 * and the switches are taken from p_r[0]). */
int susp_create_batch(susp_t** out, int32_t R, const int64_t* N_r,
                      const double* radii, const double* boxes,
                      const susp_params* p_r);

/* Frees all device and host memory of the handle.  NULL is a no-op. */
void susp_destroy(susp_t* h);

/* Message of the last failing call on this handle ("" if none).  The string
 * is owned by the handle and valid until its next call. */
const char* susp_last_error(const susp_t* h);

/* Message of the last susp_create*() or susp_pair_stress_noalloc() failure in
 * this thread. */
const char* susp_create_error(void);

/* ---- plumbing ----------------------------------------------------------- */
/* Work is issued on this cudaStream_t; NULL selects the handle's own
 * non-blocking stream (the default).  The legacy default stream cannot be
 * captured into graphs, so pass a created stream.  Takes effect for later
 * calls; captured graphs are rebuilt. */
int susp_set_stream(susp_t* h, void* cuda_stream);

/* Device memory comes from alloc(bytes, ctx) and is returned with
 * free(ptr, ctx).  Must be called before the first susp_set_state(). */
int susp_set_allocator(susp_t* h, void* (*alloc)(size_t, void*),
                       void (*release)(void*, void*), void* ctx);

/* ---- state -------------------------------------------------------------- */
/* Positions x[N][3] (wrapped into the box), velocities U[N][3] and angular
 * velocities Omega[N][3] from HOST memory; U or Omega NULL means zero.
 * Forces are re-evaluated (without advancing time) before the next step. */
int susp_set_state(susp_t* h, const double* x, const double* U,
                   const double* Omega);

/* Same, from DEVICE memory of the handle's device (e.g. tensors). */
int susp_set_state_device(susp_t* h, const double* x, const double* U,
                          const double* Omega);

/* Sets the evaluation counter k used as the noise counter (the forces held
 * after a step of index n have k = n + 1; setup forces have the k in
 * effect) and the strain of replica `replica` (-1: all), within
 * (-Lx/(2Ly), Lx/(2Ly)].  Forces are re-evaluated before the next step. */
int susp_set_clock(susp_t* h, int64_t k, int32_t replica, double strain);

/* Copies positions, velocities and angular velocities to HOST arrays
 * [N][3] in tag order; any pointer may be NULL. */
int susp_get_state(susp_t* h, double* x, double* U, double* Omega);

/* Forces F[N][3] and torques T[N][3] of the last evaluation, tag order. */
int susp_get_forces(susp_t* h, double* F, double* T);

/* ---- the method ----------------------------------------------------------- */
/* Cell binning by a counting sort on the cell key, then the skin-padded
 * half neighbour list: every unordered pair with |r|^2 < (r_int + skin)^2,
 * stored once, where r_int is the widest interaction range in use:
 * (a_i + a_j)(1 + xi_max/2) (lubrication cutoff xi <= xi_max, Sec. II.B),
 * with repulsion also (a_i + a_j)(1 + 0.01 rep_cut), with the structural
 * stress also a_i + a_j + shell max(a_i, a_j); the skin is that of Sec. II.
 * The tangential history of touching pairs is carried over.  Done
 * automatically by the step when the displacement bound exceeds the skin. */
int susp_build_neighbors(susp_t* h);

/* Sets the neighbour-list skin (length units, >= 0): the cell grid is laid
 * out again for the new list cutoff and the list is rebuilt before the next
 * evaluation.  SUSP_EINVAL if a box then holds fewer than 3 cells along an
 * axis.  Batch handles: one skin for all replicas. */
int susp_set_skin(susp_t* h, double skin);

/* Autotuner: for each candidate skin[c] (c < n) advances trial_steps steps
 * of size dt from the current state (after an untimed pass of up to 64
 * steps that captures the graphs), times them with CUDA events on the
 * handle's stream and writes the device milliseconds per step to
 * ms_per_step[c] (NaN where the skin is not possible; the array may be
 * NULL).  The fastest skin is kept and written to *chosen, and the state,
 * forces, tangential history, clock and stress sums are put back as they
 * were, so tuning leaves the run unchanged.  The cell size follows from the
 * skin (cells are one list cutoff thick); the pair kernels map one list
 * item per lane whatever the row lengths, so there is no threads-per-
 * particle choice to make. */
int susp_autotune(susp_t* h, int64_t trial_steps, double dt, const double* skins,
                  int32_t n, double* ms_per_step, double* chosen);

/* Evaluates forces, torques and pair stresses at the current state without
 * advancing time (tangential history is not incremented). */
int susp_evaluate(susp_t* h);

/* Advances n_steps Velocity-Verlet steps of a single-replica handle with the
 * given shear rate, thermal energy, timestep and Philox seed (Sec. II,
 * Eqs. 1-24, Sec. II.E).  Returns SUSP_EUNSTABLE on non-finite state and
 * SUSP_ENEIGH if a neighbour row overflowed. */
int susp_step(susp_t* h, int64_t n_steps, double shear_rate, double kT,
              double dt, uint64_t seed);

/* Advances every replica of a batch handle n_steps steps of size dt with the
 * per-replica rate, kT and seed given at creation. */
int susp_step_batch(susp_t* h, int64_t n_steps, double dt);

/* Measures where the time goes: advances n_steps exactly as
 * susp_step()/susp_step_batch() would (same physics, the parameters of the
 * last step call), but launches every kernel eagerly between two CUDA events
 * recorded on the handle's stream, and a neighbour rebuild only when it is
 * due.  out[SUSP_PROFILE_LEN] holds, for each kernel family f -- 0 integrator
 * (kick, drift, wrap), 1 neighbour rebuild (binning, sort, list, history),
 * 2 pair forces, 3 stress reduction, 4 closing half kick --
 * out[3f] the total device milliseconds, out[3f+1] the number of launches and
 * out[3f+2] the mean milliseconds per launch. */
#define SUSP_PROFILE_LEN 15
int susp_profile(susp_t* h, int64_t n_steps, double dt, double* out);

/* Stress of replica `replica` averaged over the sampled evaluations since
 * the previous call (which it resets).  out[SUSP_STRESS_LEN]:
 *   [ 0.. 8] contact        sigma^C  (row-major 3x3, Sec. II.A)
 *   [ 9..17] lubrication    sigma^HL (Sec. II.B)
 *   [18..26] pair Brownian  sigma^BL (Sec. II.D, averages to zero)
 *   [27..35] drag stresslet (20/3) pi eta sum a^3 E / V (Sec. II.B)
 *   [36..44] kinetic        sum m (U - U_inf)(U - U_inf) / V (full steps)
 *   [45..53] rotational kinetic sum I (W - W_inf)(W - W_inf) / V
 *   [54] eta_r = (sigma^C + sigma^HL + drag + sigma^R)_xy / (eta rate)
 *   [55] N1 = sigma_xx - sigma_yy, [56] N2 = sigma_yy - sigma_zz of that sum
 *   [57] number of sampled evaluations
 *   [58..66] repulsion      sigma^R (Eq. 34; zero when rep_A = 0)
 *   [67..75] structural Brownian Sigma^B, Eq. 26: -kT/V sum_i (a_i/Delta)
 *            sum_{j: h_ij <= Delta} n_ij n_ij with Delta = shell a_i, overlaps
 *            included (zero unless structural = 1; not added to eta_r) */
#define SUSP_STRESS_LEN 76
int susp_stress(susp_t* h, double* out, int32_t replica);

/* The current half neighbour list as tag pairs ij[count][2] with i < j in
 * lexicographic order; *count receives the number of pairs, at most cap are
 * written (cap = 0 only counts). */
int susp_get_pairs(susp_t* h, int32_t* ij, int64_t cap, int64_t* count);

/* Touching pairs carrying tangential history: ij[count][2] (i < j, sorted)
 * and xi_t[count][3]; as susp_get_pairs for cap and count. */
int susp_get_history(susp_t* h, int32_t* ij, double* xi_t, int64_t cap,
                     int64_t* count);

/* Diagnostics, info[SUSP_INFO_LEN]: [0] k, [1] neighbour builds so far,
 * [2] longest row at the last build, [3] row capacity, [4] pairs in the
 * list, [5] strain of replica 0, [6] tilt of replica 0, [7] threads per
 * particle in use, [8] precision, [9] replicas, [10] total spheres,
 * [11] steps replayed through graphs, [12] device bytes held, [13] kernels
 * launched so far (eager launches, graph kernel nodes per replay, and the
 * kernels of each rebuild taken inside a replay). */
#define SUSP_INFO_LEN 14
int susp_get_info(susp_t* h, double* info);

/* ---- Green-Kubo (Sec. III.D) -------------------------------------------------- */
/* The Sigma^B_xy of each sampled evaluation of replica `replica` since the
 * record was last reset, oldest first: *count receives the number recorded
 * and *dropped (may be NULL) the number dropped because series_cap samples
 * were already held.  With out NULL or cap 0 only the counts are returned;
 * otherwise min(count, cap) samples are copied to out and the record is
 * reset. */
int susp_get_series(susp_t* h, int32_t replica, double* out, int64_t cap,
                    int64_t* count, int64_t* dropped);

/* Green-Kubo viscosity of a stress series x[n] sampled every dt (Eq. 33):
 * C[m] = sum_{t < n-m} x[t+m] x[t] / (n - m) for m < max_lag (computed on the
 * current device), eta[m] = V/kT dt sum of the trapezoids of C up to m
 * (eta[0] = 0), and fit[2] = (eta_phi, tau_phi) of the least-squares fit
 * eta ~ eta_phi (1 - exp(-t/tau_phi)) over tau_g = dt (10 max_lag)^(g/(G-1)),
 * g < G = 400.  x is a HOST array; C, eta (max_lag each) and fit are host
 * outputs (C may be NULL).  Errors: SUSP_EINVAL (NULL, n < 2, max_lag < 2 or
 * > n, dt, V or kT <= 0), SUSP_ENODEV, SUSP_ENOMEM, SUSP_ECUDA; message in
 * susp_create_error(). */
int susp_green_kubo(const double* x, int64_t n, int64_t max_lag, double dt,
                    double V, double kT, double* C, double* eta, double* fit);

/* ---- diagnostics ------------------------------------------------------------- */
/* Measured peak multiply-add rates of the current device, the denominators
 * of the arithmetic rooflines: out[0] FP64 and out[1] FP32 GFLOP/s (two
 * operations per fused multiply-add), from a kernel of eight independent
 * multiply-add chains per thread on 8 blocks of 256 threads per SM, the best
 * of three launches timed with CUDA events on the legacy default stream.
 * Errors: SUSP_EINVAL (NULL), SUSP_ENODEV, SUSP_ENOMEM, SUSP_ECUDA; message
 * in susp_create_error(). */
int susp_measure_peaks(double* out);

/* ---- without allocation ------------------------------------------------------ */
/* The paper has no counterpart to this call; it is a service for callers
 * that cannot allocate device memory where they need the answer (code
 * running inside another framework's memory arena, threads that must not
 * touch the allocator, tools that only borrow buffers they do not own).
 *
 * Pair stresses of one evaluation, (1/V) sum over the listed pairs of
 * F_{i<-j} (x) r_ij for the contact (normal part), lubrication and pair
 * Brownian terms, computed as the double-precision evaluation of a handle
 * does but with the tangential history taken as zero, and written to
 * stress_out[27] (row-major 3x3 blocks in the order contact, lubrication,
 * Brownian, like out[0..26] of susp_stress() after one sampled
 * evaluation).  Every pointer except box and p is a DEVICE pointer of the
 * current device and stays owned by the caller: x, U, Omega [N][3]
 * (positions wrapped into the box), radii [N], ij [npairs][2] (pairs by
 * index, either order; pairs beyond the lubrication cutoff add nothing),
 * stress_out [27].  p supplies eta, kn, xi_min, xi_max, shear_rate, kT,
 * torque_sign, seed and the noise/lubrication/contact switches; strain is
 * the box strain, dt the timestep and k the noise counter.  Work is
 * enqueued on `stream` (a cudaStream_t, NULL = the legacy default stream)
 * and the call returns without waiting for it.
 *
 * The call allocates nothing: its scratch is a fixed array in device memory
 * that every GPU which loads the library holds until the process exits.
 * npairs above SUSP_NOALLOC_MAX_PAIRS is rejected with SUSP_EINVAL.  The
 * first call in each CUDA context (the device's primary context unless the
 * caller made another one current) looks up that array's device address in
 * that context, so make the first call before any stream capture; a device
 * reset or another context gets a fresh look-up.  All
 * calls share the array: calls whose work overlaps on the GPU (several
 * streams, or several host threads) race and give wrong results; calls on
 * one stream are ordered and safe.  Errors: SUSP_EINVAL (NULL pointer,
 * N <= 0, npairs out of range, dt <= 0, kT < 0, box <= 0), SUSP_ENODEV,
 * SUSP_ECUDA; the message is read with susp_create_error(). */
#define SUSP_NOALLOC_MAX_PAIRS (1 << 21)
int susp_pair_stress_noalloc(int64_t N, const double* x, const double* U,
                             const double* Omega, const double* radii,
                             int64_t npairs, const int32_t* ij,
                             const double box[3], double strain,
                             const susp_params* p, double dt, int64_t k,
                             double* stress_out, void* stream);

/* ---- checkpoint ------------------------------------------------------------- */
/* Writes / reads positions, velocities, forces, tangential history, k,
 * strains and the step counters; resuming reproduces the run it was taken
 * from (counter-based noise carries no generator state). */
int susp_save(susp_t* h, const char* path);
int susp_load(susp_t* h, const char* path);

#ifdef __cplusplus
}
#endif
#endif /* SUSP_H */
