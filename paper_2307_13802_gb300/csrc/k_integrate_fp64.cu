// k_integrate_fp64.cu -- Velocity-Verlet update (Sec. II) with the tilted,
// flipping periodic box (Sec. II.E), double precision, no multiply-add
// contraction.
//
// The two half kicks that surround a force evaluation are fused: the kernel
// that starts step n first closes step n-1 (U += dt/2 F/m with the forces of
// the last evaluation; skipped on the first step of a call, whose state is a
// full step), then opens step n (U += dt/2 F/m), drifts (x += dt U), advances
// the strain (flip 0.5 -> -0.5 in units of Lx/Ly), wraps the sphere into the
// box (a y crossing shifts x by the tilt and U_x by rate * Ly) and clears the
// force accumulators for the next evaluation.  The last block to finish
// advances the strain of every replica and the evaluation index k, and
// decides whether the neighbour list must be rebuilt: with D the accumulated
// bound on the displacement relative to the imposed flow, a rebuild is due
// once 2 D + rate t (r_c + 2 D) >= skin.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "susp_internal.h"

namespace susp {

// Advance strain by rate*dt with the flip of Sec. II.E.
__device__ __forceinline__ double next_strain(const Replica& R) {
  double st = R.strain + R.rate_dt;
  if (st > R.flip_at) st = st - R.flip_by;
  return st;
}

// Wrap into [0, L) (bounded loop: returns false if it cannot).
__device__ __forceinline__ bool wrap_le(double& x, double& y, double& z,
                                        double& ux, const double* L,
                                        double tilt, double dUx) {
  if (!isfinite(x + y + z)) return false;
  int guard = 0;
  while (y >= L[1] && guard < 64) { y = y - L[1]; x = x - tilt; ux = ux - dUx; ++guard; }
  while (y < 0.0 && guard < 64) { y = y + L[1]; x = x + tilt; ux = ux + dUx; ++guard; }
  while (x >= L[0] && guard < 64) { x = x - L[0]; ++guard; }
  while (x < 0.0 && guard < 64) { x = x + L[0]; ++guard; }
  while (z >= L[2] && guard < 64) { z = z - L[2]; ++guard; }
  while (z < 0.0 && guard < 64) { z = z + L[2]; ++guard; }
  return guard < 64;
}

// Last-block bookkeeping, run by every thread of the block that finishes
// last: the threads advance the replicas' strains in parallel (thread t takes
// replicas t, t + blockDim, ...), then thread 0 does the global part.
__device__ void integrator_epilogue(const Arrays& A, const StepArgs& s,
                                    unsigned long long cond_handle,
                                    int use_cond) {
  Ctl* ctl = A.ctl;
  for (int r = threadIdx.x; r < A.R; r += blockDim.x) {
    Replica& R = A.repl[r];
    const double st = next_strain(R);
    R.strain = st;
    R.tilt = st * R.L[1];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  ctl->k = ctl->k + 1;
  const double vmax = __longlong_as_double((long long)ctl->vmax_bits);
  ctl->vmax_bits = 0ull;
  ctl->disp_bound = ctl->disp_bound + s.dt * vmax;
  ctl->t_since_build = ctl->t_since_build + s.dt;
  const double D = ctl->disp_bound;
  const double drift = 2.0 * D + s.rate_max * ctl->t_since_build * (s.rcmax + 2.0 * D);
  if (drift >= s.skin) ctl->need_rebuild = 1;
  ctl->steps_since_build = ctl->steps_since_build + 1;
  if (s.rebuild_every > 0 && ctl->steps_since_build >= s.rebuild_every) ctl->need_rebuild = 1;
  if (use_cond) {
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle,
                            ctl->need_rebuild ? 1u : 0u);
  }
  ctl->ticket = 0u;
}

__global__ void __launch_bounds__(kBlock)
k_integrate_fp64(Arrays A, BlockMap bm, StepArgs s, int close, int sample_kin,
                 unsigned long long cond_handle, int use_cond) {
  __shared__ double smem[(kBlock / 32) * kKinLen];
  __shared__ bool last;
  const int b = blockIdx.x;
  const int r = bm.rep[b];
  const int p = bm.start[b] + threadIdx.x;
  const bool active = p < bm.end[b];
  Ctl* ctl = A.ctl;
  const int cur = ctl->cur;
  const Replica& RP = A.repl[r];
  const double L[3] = {RP.L[0], RP.L[1], RP.L[2]};
  const double rate = RP.rate;
  const double tilt = next_strain(RP) * L[1];
  const double hdt = s.hdt, dt = s.dt;
  const int64_t Np = A.Npad;

  double kin[kKinLen];
#pragma unroll
  for (int q = 0; q < kKinLen; ++q) kin[q] = 0.0;
  double vpec = 0.0;
  if (active) {
    double4_32a P = A.pos[cur][p];
    double4_32a V = A.vel[cur][p];
    double4_32a W = A.omg[cur][p];
    double* F = A.frc[cur];
    double* T = A.trq[cur];
    const double f0 = F[p], f1 = F[Np + p], f2 = F[2 * Np + p];
    const double t0 = T[p], t1 = T[Np + p], t2 = T[2 * Np + p];
    const double m = V.w, I = W.w;
    if (close) {
      V.x = V.x + hdt * f0 / m; V.y = V.y + hdt * f1 / m; V.z = V.z + hdt * f2 / m;
      W.x = W.x + hdt * t0 / I; W.y = W.y + hdt * t1 / I; W.z = W.z + hdt * t2 / I;
      if (sample_kin) {
        const double u[3] = {V.x - rate * (P.y - 0.5 * L[1]), V.y, V.z};
        const double w[3] = {W.x, W.y, W.z + 0.5 * rate};
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
          for (int be = 0; be < 3; ++be) {
            kin[3 * al + be] = m * u[al] * u[be];
            kin[9 + 3 * al + be] = I * w[al] * w[be];
          }
      }
    }
    V.x = V.x + hdt * f0 / m; V.y = V.y + hdt * f1 / m; V.z = V.z + hdt * f2 / m;
    W.x = W.x + hdt * t0 / I; W.y = W.y + hdt * t1 / I; W.z = W.z + hdt * t2 / I;
    P.x = P.x + dt * V.x; P.y = P.y + dt * V.y; P.z = P.z + dt * V.z;
    if (!wrap_le(P.x, P.y, P.z, V.x, L, tilt, rate * L[1]))
      atomicOr(&ctl->err, kErrNonFinite);
    if (!isfinite(V.x + V.y + V.z + W.x + W.y + W.z)) atomicOr(&ctl->err, kErrNonFinite);
    A.pos[cur][p] = P;
    A.vel[cur][p] = V;
    A.omg[cur][p] = W;
    F[p] = 0.0; F[Np + p] = 0.0; F[2 * Np + p] = 0.0;
    T[p] = 0.0; T[Np + p] = 0.0; T[2 * Np + p] = 0.0;
    const double ux = V.x - rate * (P.y - 0.5 * L[1]);
    vpec = sqrt(ux * ux + V.y * V.y + V.z * V.z);
    if (!(vpec == vpec)) vpec = 0.0;
  }
  const double bmax = block_max(vpec, smem);
  if (threadIdx.x == 0) atomicMax(&ctl->vmax_bits, (unsigned long long)__double_as_longlong(bmax));
  if (close && sample_kin)
    block_sum_write<kKinLen>(kin, smem, A.kin_partial + (int64_t)b * kKinLen);
  __threadfence();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(&ctl->ticket, 1u);
    last = (t == (unsigned int)gridDim.x - 1u);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    integrator_epilogue(A, s, cond_handle, use_cond);
  }
}

// Closing half kick at the end of a call: U += dt/2 F/m, W += dt/2 T/I.
__global__ void __launch_bounds__(kBlock)
k_finalize_fp64(Arrays A, BlockMap bm, StepArgs s, int sample_kin) {
  __shared__ double smem[(kBlock / 32) * kKinLen];
  const int b = blockIdx.x;
  const int r = bm.rep[b];
  const int p = bm.start[b] + threadIdx.x;
  const bool active = p < bm.end[b];
  const int cur = A.ctl->cur;
  const Replica& RP = A.repl[r];
  const double rate = RP.rate, Ly = RP.L[1];
  const double hdt = s.hdt;
  const int64_t Np = A.Npad;
  double kin[kKinLen];
#pragma unroll
  for (int q = 0; q < kKinLen; ++q) kin[q] = 0.0;
  if (active) {
    const double4_32a P = A.pos[cur][p];
    double4_32a V = A.vel[cur][p];
    double4_32a W = A.omg[cur][p];
    const double* F = A.frc[cur];
    const double* T = A.trq[cur];
    const double m = V.w, I = W.w;
    V.x = V.x + hdt * F[p] / m; V.y = V.y + hdt * F[Np + p] / m; V.z = V.z + hdt * F[2 * Np + p] / m;
    W.x = W.x + hdt * T[p] / I; W.y = W.y + hdt * T[Np + p] / I; W.z = W.z + hdt * T[2 * Np + p] / I;
    A.vel[cur][p] = V;
    A.omg[cur][p] = W;
    if (sample_kin) {
      const double u[3] = {V.x - rate * (P.y - 0.5 * Ly), V.y, V.z};
      const double w[3] = {W.x, W.y, W.z + 0.5 * rate};
#pragma unroll
      for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) {
          kin[3 * al + be] = m * u[al] * u[be];
          kin[9 + 3 * al + be] = I * w[al] * w[be];
        }
    }
  }
  if (sample_kin) block_sum_write<kKinLen>(kin, smem, A.kin_partial + (int64_t)b * kKinLen);
}

void launch_integrate_fp64(const Arrays& A, const BlockMap& bm,
                           const StepArgs& s, int close, int sample_kin,
                           cudaStream_t st, unsigned long long cond_handle,
                           int use_cond) {
  k_integrate_fp64<<<bm.nblocks, kBlock, 0, st>>>(A, bm, s, close, sample_kin,
                                                  cond_handle, use_cond);
}

void launch_finalize_fp64(const Arrays& A, const BlockMap& bm,
                          const StepArgs& s, int sample_kin, cudaStream_t st) {
  k_finalize_fp64<<<bm.nblocks, kBlock, 0, st>>>(A, bm, s, sample_kin);
}

}  // namespace susp
