// k_mixed.cu -- time update and state handling of the mixed-precision path.
//
// The state (positions, velocities, spins) is held in double-float form
// (dfloat.cuh) and advanced with FP32 instructions only: the same fused
// Velocity-Verlet step as the FP64 path (close the previous step with
// dt/2 F/m, open the next, drift, advance the strain with the flip of
// Sec. II.E, wrap with the Lees-Edwards shift), with forces read from the
// float4 accumulators the pair kernel fills.  Each step also writes the
// single-precision mirrors the pair kernel reads:
//   posm = (x - O_home, a) as a 32-byte double-float record (hi half, lo
//          half): offset from the lab position of the sphere's home cell
//          origin O_home = H(t) s_cell (H the tilted box matrix) at the
//          nearest periodic image.  Offsets are a few cell widths at most, so
//          the pair kernel rebuilds separations and the gap
//          h = (d^2 - S^2)/(d + S) to ~1e-12 for any box size;
//   velm = (U - U_inf(y), tag): velocity relative to the imposed flow.
// The pair kernel reads the spins from the high halves of the double-float
// records themselves (a normalised double-float's high word is its value in
// single precision), so they need no mirror.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "dfloat.cuh"
#include "susp_internal.h"

namespace susp {

struct DF3 {
  df x, y, z;
};

// One 32-byte record = two float4 halves (hi, lo); w / wl are the 4th words.
__device__ __forceinline__ void load_df3(const double4_32a* base, int64_t p, DF3& v,
                                         float& w, float* wl = nullptr) {
  const float4* r = reinterpret_cast<const float4*>(base + p);
  const float4 h = r[0], l = r[1];
  v.x = df{h.x, l.x};
  v.y = df{h.y, l.y};
  v.z = df{h.z, l.z};
  w = h.w;
  if (wl) *wl = l.w;
}

__device__ __forceinline__ void store_df3(double4_32a* base, int64_t p, const DF3& v,
                                          float w, float wl = 0.0f) {
  float4* r = reinterpret_cast<float4*>(base + p);
  r[0] = make_float4(v.x.hi, v.y.hi, v.z.hi, w);
  r[1] = make_float4(v.x.lo, v.y.lo, v.z.lo, wl);
}

// Mirrors of one sphere (see the file comment): pm[0]/pm[1] are the hi/lo
// halves of (offset, radius).  `ct` is tilt/ncy and `tilt` the tilt, both
// double-float, of the box the positions are wrapped in.
__device__ __forceinline__ void make_mirrors(const Replica& R, df tilt, df ct, int pack,
                                             const DF3& x, df a, const DF3& U, int tag,
                                             float4* pm, float4& vm) {
  // home cell coordinates, packed 10 bits per axis by the rebuild
  const int cx = pack & 1023, cy = (pack >> 10) & 1023, cz = pack >> 20;
  // home-cell origin in the lab frame
  const df ox = df_add(df_mul_f(df{R.cw_hi[0], R.cw_lo[0]}, (float)cx), df_mul_f(ct, (float)cy));
  const df oy = df_mul_f(df{R.cw_hi[1], R.cw_lo[1]}, (float)cy);
  const df oz = df_mul_f(df{R.cw_hi[2], R.cw_lo[2]}, (float)cz);
  df dx = df_sub(x.x, ox), dy = df_sub(x.y, oy), dz = df_sub(x.z, oz);
  // nearest image of the offset (a sphere wrapped across a face)
  const df Lx{R.L_hi[0], R.L_lo[0]}, Ly{R.L_hi[1], R.L_lo[1]}, Lz{R.L_hi[2], R.L_lo[2]};
  const float my = rintf(df_to_f(dy) / R.L_hi[1]);
  if (my != 0.0f) {
    dy = df_sub(dy, df_mul_f(Ly, my));
    dx = df_sub(dx, df_mul_f(tilt, my));
  }
  const float mx = rintf(df_to_f(dx) / R.L_hi[0]);
  if (mx != 0.0f) dx = df_sub(dx, df_mul_f(Lx, mx));
  const float mz = rintf(df_to_f(dz) / R.L_hi[2]);
  if (mz != 0.0f) dz = df_sub(dz, df_mul_f(Lz, mz));
  pm[0] = make_float4(dx.hi, dy.hi, dz.hi, a.hi);
  pm[1] = make_float4(dx.lo, dy.lo, dz.lo, a.lo);
  // U - rate (y - Ly/2)
  const df yrel = df_sub(x.y, df{R.yc_hi, R.yc_lo});
  const df ux = df_sub(U.x, df_mul(yrel, df{R.rate_hi, R.rate_lo}));
  vm = make_float4(df_to_f(ux), df_to_f(U.y), df_to_f(U.z), __int_as_float(tag));
}

__device__ __forceinline__ bool wrap_df(DF3& x, df& ux, const Replica& R, df tilt) {
  const df Lx{R.L_hi[0], R.L_lo[0]}, Ly{R.L_hi[1], R.L_lo[1]}, Lz{R.L_hi[2], R.L_lo[2]};
  const df du{R.dux_hi, R.dux_lo};
  if (!isfinite(x.x.hi + x.y.hi + x.z.hi)) return false;
  int guard = 0;
  while (df_ge(x.y, Ly) && guard < 64) { x.y = df_sub(x.y, Ly); x.x = df_sub(x.x, tilt); ux = df_sub(ux, du); ++guard; }
  while (df_lt0(x.y) && guard < 64) { x.y = df_add(x.y, Ly); x.x = df_add(x.x, tilt); ux = df_add(ux, du); ++guard; }
  while (df_ge(x.x, Lx) && guard < 64) { x.x = df_sub(x.x, Lx); ++guard; }
  while (df_lt0(x.x) && guard < 64) { x.x = df_add(x.x, Lx); ++guard; }
  while (df_ge(x.z, Lz) && guard < 64) { x.z = df_sub(x.z, Lz); ++guard; }
  while (df_lt0(x.z) && guard < 64) { x.z = df_add(x.z, Lz); ++guard; }
  return guard < 64;
}

__device__ __forceinline__ void kick(DF3& v, float4 f, float c) {
  v.x = df_add_f(v.x, c * f.x);
  v.y = df_add_f(v.y, c * f.y);
  v.z = df_add_f(v.z, c * f.z);
}

// Last-block bookkeeping (strain, k, rebuild decision) as in the FP64 path,
// plus the double-float fields the next step reads.  Every thread of the
// block that finishes last runs it: the replicas are advanced in parallel
// (thread t takes replicas t, t + blockDim, ...), then thread 0 does the
// global part.
__device__ void epilogue_mixed(const Arrays& A, const StepArgs& s,
                               unsigned long long cond_handle, int use_cond) {
  Ctl* ctl = A.ctl;
  for (int r = threadIdx.x; r < A.R; r += blockDim.x) {
    Replica& R = A.repl[r];
    const double st = advance_strain(R.strain, R.rate_dt, R.flip_at, R.flip_by);
    // a flip moves every home-cell origin by a fraction of Lx: the
    // cell-relative mirrors need fresh home cells (every thread that sees
    // one writes the same 1)
    if (st < R.strain && R.rate_dt > 0.0) ctl->need_rebuild = 1;
    R.strain = st;
    R.tilt = R.strain * R.L[1];
    refresh_strain_fields(R);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  ctl->k = ctl->k + 1;
  const double vmax = (double)__uint_as_float(ctl->vmax_fbits);
  ctl->vmax_fbits = 0u;
  ctl->disp_bound = ctl->disp_bound + s.dt * vmax;
  ctl->t_since_build = ctl->t_since_build + s.dt;
  const double D = ctl->disp_bound;
  const double drift = 2.0 * D + s.rate_max * ctl->t_since_build * (s.rcmax + 2.0 * D);
  if (drift >= s.skin) ctl->need_rebuild = 1;
  ctl->steps_since_build = ctl->steps_since_build + 1;
  if (s.rebuild_every > 0 && ctl->steps_since_build >= s.rebuild_every) ctl->need_rebuild = 1;
  if (use_cond)
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle,
                            ctl->need_rebuild ? 1u : 0u);
  ctl->ticket = 0u;
}

// resident blocks per SM the register allocation targets
#ifndef SUSP_INTEG_MINBLOCKS
#define SUSP_INTEG_MINBLOCKS 4
#endif

__global__ void __launch_bounds__(kBlock, SUSP_INTEG_MINBLOCKS)
k_integrate_mixed(Arrays A, BlockMap bm, StepArgs s, int close, int sample_kin,
                  unsigned long long cond_handle, int use_cond, float dt_hi, float dt_lo,
                  float hdt) {
  __shared__ double smem[(kBlock / 32) * kKinLen];
  const int b = blockIdx.x;
  const int r = bm.rep[b];
  const int p = bm.start[b] + threadIdx.x;
  const bool active = p < bm.end[b];
  Ctl* ctl = A.ctl;
  const int cur = ctl->cur;
  const Replica& RP = A.repl[r];
  const df tilt{RP.nt_hi, RP.nt_lo};   // tilt after this step's strain advance
  const df ct{RP.nct_hi, RP.nct_lo};
  const df dt{dt_hi, dt_lo};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* sk = reinterpret_cast<float*>(smem);
  float vpec = 0.0f;
  DF3 x{}, U{}, W{};
  float a = 0.0f, alo = 0.0f, im = 0.0f, iI = 0.0f;
  float4 f = make_float4(0.f, 0.f, 0.f, 0.f), t = f;
  int cellpk = 0, tagp = 0;
  float4* F4 = reinterpret_cast<float4*>(A.frc[cur]);
  float4* T4 = reinterpret_cast<float4*>(A.trq[cur]);
  if (active) {
    load_df3(A.pos[cur], p, x, a, &alo);
    load_df3(A.vel[cur], p, U, im);
    load_df3(A.omg[cur], p, W, iI);
    cellpk = A.cell[p];
    tagp = A.tag[cur][p];
  }
  // the state above is not written by the pair kernel; the forces are, and
  // the mirrors written below are read by it: wait for that grid here
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (active) {
    f = F4[p];
    t = T4[p];
  }
  const float cm = hdt * im, cI = hdt * iI;
  if (close) {
    kick(U, f, cm);
    kick(W, t, cI);
    if (sample_kin) {
      // kinetic tensors of the closed step, summed over the warp one entry
      // at a time into shared memory (all lanes take part; idle lanes add 0)
      float u[3] = {0.f, 0.f, 0.f}, w[3] = {0.f, 0.f, 0.f}, m = 0.f, I = 0.f;
      if (active) {
        const df yrel = df_sub(x.y, df{RP.yc_hi, RP.yc_lo});
        u[0] = df_to_f(df_sub(U.x, df_mul(yrel, df{RP.rate_hi, RP.rate_lo})));
        u[1] = df_to_f(U.y);
        u[2] = df_to_f(U.z);
        w[0] = df_to_f(W.x);
        w[1] = df_to_f(W.y);
        w[2] = df_to_f(W.z) + 0.5f * RP.rate_f;
        m = 1.0f / im;
        I = 1.0f / iI;
      }
#pragma unroll
      for (int q = 0; q < kKinLen; ++q) {
        const int al = (q % 9) / 3, be = q % 3;
        float v = q < 9 ? m * u[al] * u[be] : I * w[al] * w[be];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sk[warp * kKinLen + q] = v;
      }
    }
  }
  if (active) {
    kick(U, f, cm);
    kick(W, t, cI);
    x.x = df_add(x.x, df_mul(U.x, dt));
    x.y = df_add(x.y, df_mul(U.y, dt));
    x.z = df_add(x.z, df_mul(U.z, dt));
    if (!wrap_df(x, U.x, RP, tilt)) atomicOr(&ctl->err, kErrNonFinite);
    if (!isfinite(U.x.hi + U.y.hi + U.z.hi + W.x.hi + W.y.hi + W.z.hi))
      atomicOr(&ctl->err, kErrNonFinite);
    store_df3(A.pos[cur], p, x, a, alo);
    store_df3(A.vel[cur], p, U, im);
    store_df3(A.omg[cur], p, W, iI);
    F4[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    T4[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 pm[2], vm;
    make_mirrors(RP, tilt, ct, cellpk, x, df{a, alo}, U, tagp, pm, vm);
    A.posm[2 * p] = pm[0];
    A.posm[2 * p + 1] = pm[1];
    A.velm[p] = vm;
    vpec = sqrtf(vm.x * vm.x + vm.y * vm.y + vm.z * vm.z);
    if (!(vpec == vpec)) vpec = 0.0f;
  }
  // Block sums of the kinetic tensors (sampled steps; the warp sums are in
  // shared memory already) and the block max of the peculiar speed in single
  // precision, one barrier for both; thread 0 then publishes the max
  // (non-negative floats order like their bit patterns, so an integer
  // atomicMax is a float max), fences and takes the ticket, and the last
  // block runs the step's epilogue.
  __shared__ float svmax[kBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vpec = fmaxf(vpec, __shfl_down_sync(0xffffffffu, vpec, o));
  if (lane == 0) svmax[warp] = vpec;
  __syncthreads();
  if (close && sample_kin && threadIdx.x < kKinLen) {
    float sum = 0.0f;
    for (int w2 = 0; w2 < kBlock / 32; ++w2) sum += sk[w2 * kKinLen + threadIdx.x];
    A.kin_partial[(int64_t)b * kKinLen + threadIdx.x] = (double)sum;
  }
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    float bmax = 0.0f;
    for (int w2 = 0; w2 < kBlock / 32; ++w2) bmax = fmaxf(bmax, svmax[w2]);
    atomicMax(&ctl->vmax_fbits, __float_as_uint(bmax));
    __threadfence();
    const unsigned int tk = atomicAdd(&ctl->ticket, 1u);
    s_last = tk == (unsigned int)gridDim.x - 1u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    epilogue_mixed(A, s, cond_handle, use_cond);
  }
}

// Closing half kick at the end of a call (double-float).
__global__ void __launch_bounds__(kBlock)
k_finalize_mixed(Arrays A, BlockMap bm, StepArgs s, int sample_kin, float hdt) {
  __shared__ double smem[(kBlock / 32) * kKinLen];
  const int b = blockIdx.x;
  const int r = bm.rep[b];
  const int p = bm.start[b] + threadIdx.x;
  const bool active = p < bm.end[b];
  const int cur = A.ctl->cur;
  const Replica& RP = A.repl[r];
  float kin[kKinLen];
#pragma unroll
  for (int q = 0; q < kKinLen; ++q) kin[q] = 0.0f;
  if (active) {
    DF3 x, U, W;
    float a, im, iI;
    load_df3(A.pos[cur], p, x, a);
    load_df3(A.vel[cur], p, U, im);
    load_df3(A.omg[cur], p, W, iI);
    const float4 f = reinterpret_cast<const float4*>(A.frc[cur])[p];
    const float4 t = reinterpret_cast<const float4*>(A.trq[cur])[p];
    kick(U, f, hdt * im);
    kick(W, t, hdt * iI);
    store_df3(A.vel[cur], p, U, im);
    store_df3(A.omg[cur], p, W, iI);
    if (sample_kin) {
      const df yrel = df_sub(x.y, df{RP.yc_hi, RP.yc_lo});
      const float u[3] = {df_to_f(df_sub(U.x, df_mul(yrel, df{RP.rate_hi, RP.rate_lo}))),
                          df_to_f(U.y), df_to_f(U.z)};
      const float w[3] = {df_to_f(W.x), df_to_f(W.y), df_to_f(W.z) + 0.5f * RP.rate_f};
      const float m = 1.0f / im, I = 1.0f / iI;
#pragma unroll
      for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) {
          kin[3 * al + be] = m * u[al] * u[be];
          kin[9 + 3 * al + be] = I * w[al] * w[be];
        }
    }
  }
  if (sample_kin) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* sk = reinterpret_cast<float*>(smem);
#pragma unroll
    for (int q = 0; q < kKinLen; ++q) {
      float v = kin[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sk[warp * kKinLen + q] = v;
    }
    __syncthreads();
    if (threadIdx.x < kKinLen) {
      float sum = 0.0f;
      for (int w2 = 0; w2 < kBlock / 32; ++w2) sum += sk[w2 * kKinLen + threadIdx.x];
      A.kin_partial[(int64_t)b * kKinLen + threadIdx.x] = (double)sum;
    }
  }
  (void)s;
}

// Mirrors from the state: after a rebuild (gated, new order) or a state change.
__global__ void k_mirror_mixed(Arrays A, int gated, int use_next) {
  if (gated && *(volatile const int*)&A.ctl->need_rebuild == 0) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int c = use_next ? (A.ctl->cur ^ 1) : A.ctl->cur;
  const int r = A.rep[c][p];
  const Replica& R = A.repl[r];
  DF3 x, U, W;
  float a, alo, im, iI;
  load_df3(A.pos[c], p, x, a, &alo);
  load_df3(A.vel[c], p, U, im);
  load_df3(A.omg[c], p, W, iI);
  const df tilt = df_from_d(R.tilt);  // off the per-step path
  float4 pm[2], vm;
  make_mirrors(R, tilt, df{R.ct_hi, R.ct_lo}, A.cell[p], x, df{a, alo}, U, A.tag[c][p], pm,
               vm);
  A.posm[2 * p] = pm[0];
  A.posm[2 * p + 1] = pm[1];
  A.velm[p] = vm;
}

// Host state (tag order, doubles) into the live copy in double-float form.
__global__ void k_load_state_mixed(Arrays A, const double* __restrict__ x,
                                   const double* __restrict__ U,
                                   const double* __restrict__ W,
                                   const double* __restrict__ radius,
                                   const double* __restrict__ mass,
                                   const double* __restrict__ inertia,
                                   const int* __restrict__ rep_of) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int cur = A.ctl->cur;
  const int r = rep_of[p];
  const Replica& R = A.repl[r];
  double px = x[3 * p], py = x[3 * p + 1], pz = x[3 * p + 2];
  double ux = U ? U[3 * p] : 0.0, uy = U ? U[3 * p + 1] : 0.0, uz = U ? U[3 * p + 2] : 0.0;
  const double wx = W ? W[3 * p] : 0.0, wy = W ? W[3 * p + 1] : 0.0, wz = W ? W[3 * p + 2] : 0.0;
  const double dUx = R.rate * R.L[1];
  if (isfinite(px + py + pz)) {
    int guard = 0;
    while (py >= R.L[1] && guard < 1024) { py -= R.L[1]; px -= R.tilt; ux -= dUx; ++guard; }
    while (py < 0.0 && guard < 1024) { py += R.L[1]; px += R.tilt; ux += dUx; ++guard; }
    while (px >= R.L[0] && guard < 1024) { px -= R.L[0]; ++guard; }
    while (px < 0.0 && guard < 1024) { px += R.L[0]; ++guard; }
    while (pz >= R.L[2] && guard < 1024) { pz -= R.L[2]; ++guard; }
    while (pz < 0.0 && guard < 1024) { pz += R.L[2]; ++guard; }
    if (guard >= 1024) atomicOr(&A.ctl->err, kErrWrap);
  } else {
    atomicOr(&A.ctl->err, kErrNonFinite);
  }
  DF3 X{df_from_d(px), df_from_d(py), df_from_d(pz)};
  DF3 V{df_from_d(ux), df_from_d(uy), df_from_d(uz)};
  DF3 Om{df_from_d(wx), df_from_d(wy), df_from_d(wz)};
  const df arad = df_from_d(radius[p]);
  store_df3(A.pos[cur], p, X, arad.hi, arad.lo);
  store_df3(A.vel[cur], p, V, (float)(1.0 / mass[p]));
  store_df3(A.omg[cur], p, Om, (float)(1.0 / inertia[p]));
  reinterpret_cast<float4*>(A.frc[cur])[p] = make_float4(0.f, 0.f, 0.f, 0.f);
  reinterpret_cast<float4*>(A.trq[cur])[p] = make_float4(0.f, 0.f, 0.f, 0.f);
  A.tag[cur][p] = (int)p;
  A.rep[cur][p] = r;
  A.slot_of_tag[p] = (int)p;
  A.nnb[cur][p] = 0;
  A.cmsk[cur][p] = 0ull;
}

__global__ void k_zero_forces_mixed(Arrays A) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int cur = A.ctl->cur;
  reinterpret_cast<float4*>(A.frc[cur])[p] = make_float4(0.f, 0.f, 0.f, 0.f);
  reinterpret_cast<float4*>(A.trq[cur])[p] = make_float4(0.f, 0.f, 0.f, 0.f);
}

static inline unsigned grid_of(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

void launch_integrate_mixed(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                            int close, int sample_kin, cudaStream_t st,
                            unsigned long long cond_handle, int use_cond) {
  float dth, dtl;
  split_df(s.dt, dth, dtl);
  // programmatic dependent launch: the blocks may become resident during the
  // pair kernel's last wave and load their state before it ends
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)bm.nblocks);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_integrate_mixed, A, bm, s, close, sample_kin, cond_handle, use_cond,
                     dth, dtl, (float)s.hdt);
}

void launch_finalize_mixed(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                           int sample_kin, cudaStream_t st) {
  k_finalize_mixed<<<bm.nblocks, kBlock, 0, st>>>(A, bm, s, sample_kin, (float)s.hdt);
}

void launch_mirror(const Arrays& A, const BlockMap& bm, cudaStream_t st) {
  (void)bm;
  k_mirror_mixed<<<grid_of(A.N), kBlock, 0, st>>>(A, 0, 0);
}

void launch_mirror_gated_next(const Arrays& A, cudaStream_t st) {
  k_mirror_mixed<<<grid_of(A.N), kBlock, 0, st>>>(A, 1, 1);
}

void launch_load_state_mixed(const Arrays& A, const double* x, const double* U,
                             const double* W, const double* radius, const double* mass,
                             const double* inertia, const int* rep_of, cudaStream_t st) {
  k_load_state_mixed<<<grid_of(A.N), kBlock, 0, st>>>(A, x, U, W, radius, mass, inertia,
                                                      rep_of);
}

void launch_zero_forces_mixed(const Arrays& A, cudaStream_t st) {
  k_zero_forces_mixed<<<grid_of(A.N), kBlock, 0, st>>>(A);
}

}  // namespace susp
