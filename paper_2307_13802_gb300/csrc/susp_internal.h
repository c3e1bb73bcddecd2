// susp_internal.h -- device-side data layout shared by the library's CUDA
// translation units (not part of the public ABI).
//
// Layout in HBM.  Particles live in "sorted" order p: grouped by replica,
// then by cell key (counting sort on the cell of the tilted grid), then by
// tag.  Every per-particle array that is permuted at a rebuild exists twice
// (index [0]/[1]); Ctl::cur names the live copy, so a neighbour rebuild
// inside a captured CUDA graph permutes into the other copy and flips `cur`
// without any pointer change in the graph.
//   pos  double4_32a (x, y, z, a)            lab frame, wrapped into the box
//   vel  double4_32a (Ux, Uy, Uz, m)          lab-frame velocity, mass
//   omg  double4_32a (Wx, Wy, Wz, I)          angular velocity, moment of inertia
//   frc  double [3][Npad]                 force (SoA; accumulated by atomics)
//   trq  double [3][Npad]                 torque
//   tag  int32                            global tag (caller index)
//   rep  int32                            replica of the particle
//   nbr  int32  [kmax][Npad]              half list, slot-major (coalesced)
//   nnb  int32  [Npad]                    row lengths
//   hist double [3][kmax][Npad]           tangential history per slot (mu>0);
//                                         mixed: [kmax][Npad] 32-byte records
//                                         (x, y, z as hi/lo float pairs)
//   cmsk uint64 [Npad]                    slot s in contact at last evaluation
//   mirror (mixed precision)  posm: two float4 (hi, lo) of (dx, dy, dz, a),
//                               the offset from the home-cell origin;
//                               float4 velm (u - U_inf, tag); the spins
//                               are read from the high halves of omg;
//                               int32 cell (packed home cell coordinates)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace susp {

constexpr int kBlock = 256;          // threads per block of particle kernels
constexpr int kStressComp = 3;       // contact, lubrication, pair Brownian
constexpr int kVirLen = 27;          // their virials: 3 components x 9 entries
constexpr int kRepOff = 27;          // repulsion virial (9) in a block partial
constexpr int kStrOff = 36;          // structural sums sum w n n (9), Eq. 26
constexpr int kPartialLen = 45;      // pair entries of a block partial
// A neighbour-list entry holds the partner's sorted index in its low 27 bits;
// on the mixed path the top 5 bits hold the partner's home cell relative to
// the owner's, (dcx + 1) 3 + (dcy + 1) + 9 (dcz + 1) with dc in {-1, 0, 1}^3
// (the stencil offset the list build found it at), so the pair kernel needs
// neither home cell.
constexpr int kNbrIndexBits = 27;
constexpr int kNbrIndexMask = (1 << kNbrIndexBits) - 1;
constexpr int kKinLen = 18;          // translational + rotational kinetic
// per-replica stress accumulator: [0, 45) pair, [45, 63) kinetic, sample counts
constexpr int kAccStride = 72;
constexpr int kAccNp = 63;           // pair samples
constexpr int kAccNk = 64;           // kinetic samples
constexpr int kChunk = 64;           // blocks per chunk of the stress reduction

// error bits of Ctl::err
constexpr int kErrNonFinite = 1;
constexpr int kErrOverflow = 2;
constexpr int kErrOverlap = 4;
constexpr int kErrWrap = 8;

struct Replica {
  double L[3];
  double iL[3];      // 1 / L
  double rate;       // shear rate
  double rate_dt;    // rate * dt (set per step call)
  double kT;
  double noise_c;    // sqrt(2 kT / dt)
  double eta, kn, kt, mu;
  double rep_A;      // repulsion scale of Eq. 34 (0: off)
  double V;
  double flip_at;    // 0.5 Lx / Ly
  double flip_by;    // Lx / Ly
  double strain;     // current strain (advanced on the device)
  double tilt;       // strain * Ly
  double hcell[3];   // cell extents in fractional units (1/nc)
  uint32_t key0, key1;   // Philox key (seed)
  int32_t nc[3];     // cell grid
  int32_t pad0;
  int64_t cell_base; // first cell key of this replica
  int64_t p0, n;     // particle range (tags and sorted order)
  // single-precision and double-float copies for the mixed path; the
  // strain-dependent ones are refreshed by refresh_strain_fields()
  float rate_f, noise_cf, eta_f, kn_f, kt_f, mu_f;
  float cwf[3];                 // cell widths L / nc
  float ctilt_f;                // current tilt / ncy
  float L_hi[3], L_lo[3];       // box edges
  float yc_hi, yc_lo;           // Ly / 2
  float dux_hi, dux_lo;         // rate * Ly: velocity jump across y
  float rate_hi, rate_lo;
  float cw_hi[3], cw_lo[3];     // cell widths
  float ct_hi, ct_lo;           // current tilt / ncy
  float nt_hi, nt_lo;           // tilt after the next strain advance
  float nct_hi, nct_lo;         // that tilt / ncy
  float rep_A_f;
  float pad1;
};

// Next strain of the box with the flip of Sec. II.E.
__host__ __device__ __forceinline__ double advance_strain(double st, double rate_dt,
                                                          double flip_at, double flip_by) {
  st = st + rate_dt;
  if (st > flip_at) st = st - flip_by;
  return st;
}

__host__ __device__ __forceinline__ void split_df(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// Strain-dependent single/double-float fields of the mixed path.
__host__ __device__ inline void refresh_strain_fields(Replica& R) {
  R.ctilt_f = (float)(R.tilt * R.hcell[1]);
  split_df(R.tilt * R.hcell[1], R.ct_hi, R.ct_lo);
  const double nst = advance_strain(R.strain, R.rate_dt, R.flip_at, R.flip_by);
  const double ntilt = nst * R.L[1];
  split_df(ntilt, R.nt_hi, R.nt_lo);
  split_df(ntilt * R.hcell[1], R.nct_hi, R.nct_lo);
}

// Constant single/double-float fields of the mixed path.
inline void refresh_constant_fields(Replica& R) {
  R.rate_f = (float)R.rate;
  R.noise_cf = (float)R.noise_c;
  R.eta_f = (float)R.eta;
  R.kn_f = (float)R.kn;
  R.kt_f = (float)R.kt;
  R.mu_f = (float)R.mu;
  R.rep_A_f = (float)R.rep_A;
  for (int d = 0; d < 3; ++d) {
    R.cwf[d] = (float)(R.L[d] * R.hcell[d]);
    split_df(R.L[d], R.L_hi[d], R.L_lo[d]);
    split_df(R.L[d] * R.hcell[d], R.cw_hi[d], R.cw_lo[d]);
  }
  split_df(0.5 * R.L[1], R.yc_hi, R.yc_lo);
  split_df(R.rate * R.L[1], R.dux_hi, R.dux_lo);
  split_df(R.rate, R.rate_hi, R.rate_lo);
  refresh_strain_fields(R);
}

struct Ctl {
  long long k;                  // evaluation index of the forces held
  unsigned long long vmax_bits; // max peculiar speed of this step (double bits)
  unsigned int vmax_fbits;      // same, single precision bits (mixed path)
  double disp_bound;            // accumulated displacement bound D
  double t_since_build;
  long long steps_since_build;
  int need_rebuild;
  int err;
  int cur;                      // live copy of the double-buffered arrays
  int nbuilds;
  int max_row;                  // longest neighbour row at the last build
  unsigned int ticket;          // last-block detection in the integrator
  long long npairs;             // pairs in the list
  long long graph_steps;
};

// Per-block work map: block b handles sorted particles [start, end) of one
// replica, so block reductions are per replica and deterministic.
struct BlockMap {
  const int* rep;
  const int* start;
  const int* end;
  int nblocks;
};

template <typename T>
struct Pair2 {
  T* a[2];
  __host__ __device__ T* operator[](int i) const { return a[i]; }
};

// Mixed-precision layout (Arrays::mixed = 1): the 32-byte records of
// pos/vel/omg hold two float4 halves (hi, lo) of a double-float value:
//   pos = {x_hi, y_hi, z_hi, a}{x_lo, y_lo, z_lo, 0}
//   vel = {U_hi.., 1/m}{U_lo.., 0}      omg = {W_hi.., 1/I}{W_lo.., 0}
// frc/trq hold float4 accumulators (F, 0) / (T, 0); hist holds float2
// (hi, lo) per component at the double index of the FP64 layout.
struct Arrays {
  int64_t N;        // total particles
  int64_t Npad;     // padded stride of SoA arrays
  int kmax;
  int R;
  int mixed;        // 1: mixed-precision layout
  Pair2<double4_32a> pos, vel, omg;
  Pair2<double> frc, trq;
  Pair2<int> tag, rep;
  Pair2<int> nbr, nnb;
  Pair2<double> hist;
  Pair2<unsigned long long> cmsk;
  int* slot_of_tag;     // tag -> sorted index (live copy)
  // deterministic force sums (FP64 path, deterministic = 1)
  int det;              // 1: pair shares go to per-slot records
  double* det_slot;     // [9][kmax * Npad]: force and torque on the row's
                        // sphere, torque on the partner
  double* det_own;      // [6][Npad]: one-body force and torque
  int* rev_cnt;         // [N + 1] times each sphere is a partner
  int* rev_fill;        // [N + 1] fill counters
  int* rev_off;         // [N + 1] offsets into rev_ent
  int* rev_ent;         // [kmax * Npad] slots (sl * Npad + p) of each partner
  int* rev_part;        // scan block totals
  int* cell;            // home cell of sorted particle (new order after build),
                        // coordinates packed cx | cy << 10 | cz << 20
  float4* posm;         // mixed-precision mirrors: cell-relative position
  float4* velm;         // and velocity relative to the imposed flow
  // neighbour-build scratch
  int* key;             // cell key per particle (old order)
  int* perm;            // new sorted index -> old sorted index
  int* cell_count;      // [ncell_total + 1]
  int* cell_start;      // [ncell_total + 1]
  int* cell_fill;       // [ncell_total]
  int* scan_part;       // block sums of the scan
  int64_t ncell;
  // reductions
  double* pair_partial; // [nblocks][27]
  double* pair_partial_w; // [2][nblocks][45] block partials of the mixed path
                          // (single-precision warp sums folded in double): two
                          // buffers, so that a pair launch can reduce the
                          // previous launch's partials while writing its own
  double* kin_partial;  // [nblocks][18]
  double* stress_acc;   // [R][kAccStride]: 45 pair, 18 kinetic, pair / kinetic counts
  double* series;       // [R][series_cap] Sigma^B_xy per sampled evaluation
  long long* series_n;  // [2R]: samples recorded, samples dropped
  int series_cap;
  double shell;         // structural shell Delta / a_i
  int* rep_bstart;      // [R + 1] first block of each replica
  // two-level stress reduction: chunks of up to kChunk consecutive blocks of
  // one replica; chunk c covers blocks [chunk_b[c], chunk_b[c + 1]) -- the
  // array holds nchunk + 1 entries and chunk ends coincide with replica
  // ends -- and replica r owns chunks [rep_cstart[r], rep_cstart[r + 1])
  int* chunk_b;
  int* rep_cstart;
  int nchunk;
  double* chunk_partial; // [nchunk][kPartialLen + kKinLen]
  int* chunk_rep;         // [nchunk] replica of each chunk
  // per-replica arrival counters of the reduction fused into the mixed pair
  // kernel; zero between launches (the last arrival resets its counter)
  unsigned int* rep_tk;   // [R]
  Replica* repl;        // [R]
  Ctl* ctl;
};

struct StepArgs {
  double dt;
  double hdt;        // dt / 2
  double xi_min, xi_max, skin;
  double rcmax;      // largest interaction range (list cutoff without skin)
  double rate_max;   // largest |rate| over replicas
  double torque_sign;
  int noise, lubrication, onebody, contact, friction;
  int rep_on;        // some replica has repulsion (Eq. 34)
  int structural;    // structural Brownian sums (Eq. 26) on sampled steps
  int rebuild_every; // > 0: rebuild at least every this many steps
  double rep_fac;    // 1 + 0.01 rep_cut: repulsion range over a_i + a_j
  double rep_cut;    // repulsion for h <= rep_cut kappa, kappa = 0.01 (a_i + a_j)
  double rep_hc;     // 0.01 rep_cut: repulsion gap cutoff over a_i + a_j
  double shell;      // structural shell Delta / a_i
  int advance;       // 1: time advanced since the previous evaluation
  int sample;        // 1: accumulate stresses at this evaluation
  int ppar;          // mixed path: pair_partial_w buffer this evaluation writes
  int fuse_red;      // mixed path: the pair kernel first reduces the previous
                     // sampled step (buffer ppar ^ 1 and the kinetic partials
                     // of the integrator launch before it)
  // single-precision copies for the mixed path (set on the host)
  float dt_f, hdt_f, xi_min_f, xi_max_f, tsign_f;
  float rep_fac_f, rep_hc_f, shell_f;
};

// ---- host-side launchers (defined in the .cu files) ----------------------
void launch_integrate_fp64(const Arrays& A, const BlockMap& bm,
                           const StepArgs& s, int close, int sample_kin,
                           cudaStream_t st, unsigned long long cond_handle,
                           int use_cond);
void launch_finalize_fp64(const Arrays& A, const BlockMap& bm,
                          const StepArgs& s, int sample_kin, cudaStream_t st);
void launch_pair_fp64(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                      int tpp, cudaStream_t st);
// raises the FP64 pair kernels' dynamic shared-memory limit on the current
// device; 0 or the CUDA error code
int prepare_pair_fp64();
// deterministic sums (k_det.cu): the reverse list (gated, in the rebuild)
// and the per-sphere gather after the pair kernel
void launch_rev_build(const Arrays& A, cudaStream_t st);
void launch_det_gather(const Arrays& A, cudaStream_t st);
void launch_integrate_mixed(const Arrays& A, const BlockMap& bm,
                            const StepArgs& s, int close, int sample_kin,
                            cudaStream_t st, unsigned long long cond_handle,
                            int use_cond);
void launch_finalize_mixed(const Arrays& A, const BlockMap& bm,
                           const StepArgs& s, int sample_kin, cudaStream_t st);
void launch_mirror(const Arrays& A, const BlockMap& bm, cudaStream_t st);
void launch_pair_mixed(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                       int tpp, cudaStream_t st);
void launch_autocorr(const double* x, int64_t n, int64_t max_lag, double* C,
                     cudaStream_t st);
void launch_fma_peak(int fp64, void* sink, int blocks, int iters, cudaStream_t st);
// ppar: the pair_partial_w buffer to read (mixed path)
void launch_reduce_stress(const Arrays& A, const BlockMap& bm, int sample_pair,
                          int sample_kin, int ppar, cudaStream_t st);
// neighbour rebuild: `gated` kernels return at once unless ctl->need_rebuild
void launch_rebuild(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                    cudaStream_t st, int mixed);
void launch_mirror_gated_next(const Arrays& A, cudaStream_t st);
void launch_request_rebuild(const Arrays& A, cudaStream_t st);
void launch_load_state(const Arrays& A, const double* x, const double* U,
                       const double* W, const double* radius,
                       const double* mass, const double* inertia,
                       const int* rep_of, cudaStream_t st);
void launch_load_state_mixed(const Arrays& A, const double* x, const double* U,
                             const double* W, const double* radius,
                             const double* mass, const double* inertia,
                             const int* rep_of, cudaStream_t st);
void launch_zero_forces(const Arrays& A, cudaStream_t st);
void launch_gather(const Arrays& A, int what, double* out, cudaStream_t st);
void launch_row_counts(const Arrays& A, int with_history, long long* cnt,
                       cudaStream_t st);
void launch_list_pairs(const Arrays& A, const long long* off, int* ij,
                       int with_history, double* xi_t, cudaStream_t st);

}  // namespace susp
