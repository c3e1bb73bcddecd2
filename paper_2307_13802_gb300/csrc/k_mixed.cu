// k_mixed.cu -- mixed-precision form of the time update and of the pair
// force evaluation.
//
// Positions, velocities, spins, the tangential history and all stress and
// force accumulators stay in double precision.  The pair arithmetic of
// Sec. II.A-II.C (gap, resistances, lubrication, pair noise, contact) runs in
// single precision on mirrors the integrator writes each step:
//   posm = (x - O_home, a): offset of the sphere from the lab position of its
//          home cell's origin O_home = H(t) s_cell (H the tilted box matrix),
//          taken at the nearest periodic image, so |offset| stays below a
//          few cell widths and its single-precision rounding is ~1e-7 of a
//          radius;
//   velm = U - U_inf(y): velocity relative to the imposed flow;
//   omgm = Omega.
// The separation of a listed pair is rebuilt as
//   r = (posm_q - posm_p) + H(t) (c_q - c_p) / nc
// with the cell difference wrapped to {-1, 0, 1}: both terms are of order
// one cell, so the gap h = |r| - (a_i + a_j) keeps ~1e-7 absolute accuracy
// however large the box.  The relative velocity of the image of j is
// u_j - u_i + rate r_y x (the imposed flow difference across r), which
// includes the Lees-Edwards image velocity without a separate shift.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "philox.cuh"
#include "susp_internal.h"

namespace susp {

__device__ __forceinline__ double next_strain_m(const Replica& R) {
  double st = R.strain + R.rate_dt;
  if (st > R.flip_at) st = st - R.flip_by;
  return st;
}

// Offset of a sphere from its home-cell origin at the nearest image, in the
// box of tilt `tilt`; `cellkey` is the global cell key.
__device__ __forceinline__ float4 make_posm(const Replica& R, double tilt,
                                            int cellkey, double x, double y,
                                            double z, double a) {
  const int local = (int)(cellkey - R.cell_base);
  const int cx = local % R.nc[0], cy = (local / R.nc[0]) % R.nc[1],
            cz = local / (R.nc[0] * R.nc[1]);
  const double sx = cx * R.hcell[0], sy = cy * R.hcell[1], sz = cz * R.hcell[2];
  double dx = x - (R.L[0] * sx + tilt * sy);
  double dy = y - R.L[1] * sy;
  double dz = z - R.L[2] * sz;
  const double my = rint(dy / R.L[1]);
  dy -= my * R.L[1];
  dx -= my * tilt;
  dx -= rint(dx / R.L[0]) * R.L[0];
  dz -= rint(dz / R.L[2]) * R.L[2];
  return make_float4((float)dx, (float)dy, (float)dz, (float)a);
}

__device__ __forceinline__ bool wrap_le_m(double& x, double& y, double& z,
                                          double& ux, const double* L,
                                          double tilt, double dUx) {
  if (!isfinite(x + y + z)) return false;
  int guard = 0;
  while (y >= L[1] && guard < 64) { y -= L[1]; x -= tilt; ux -= dUx; ++guard; }
  while (y < 0.0 && guard < 64) { y += L[1]; x += tilt; ux += dUx; ++guard; }
  while (x >= L[0] && guard < 64) { x -= L[0]; ++guard; }
  while (x < 0.0 && guard < 64) { x += L[0]; ++guard; }
  while (z >= L[2] && guard < 64) { z -= L[2]; ++guard; }
  while (z < 0.0 && guard < 64) { z += L[2]; ++guard; }
  return guard < 64;
}

__device__ void integrator_epilogue_m(const Arrays& A, const StepArgs& s,
                                      unsigned long long cond_handle,
                                      int use_cond) {
  Ctl* ctl = A.ctl;
  for (int r = 0; r < A.R; ++r) {
    Replica& R = A.repl[r];
    const double st = next_strain_m(R);
    R.strain = st;
    R.tilt = st * R.L[1];
  }
  ctl->k = ctl->k + 1;
  const double vmax = __longlong_as_double((long long)ctl->vmax_bits);
  ctl->vmax_bits = 0ull;
  ctl->disp_bound = ctl->disp_bound + s.dt * vmax;
  ctl->t_since_build = ctl->t_since_build + s.dt;
  const double D = ctl->disp_bound;
  const double drift = 2.0 * D + s.rate_max * ctl->t_since_build * (s.rcmax + 2.0 * D);
  if (drift >= s.skin) ctl->need_rebuild = 1;
  if (use_cond)
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle,
                            ctl->need_rebuild ? 1u : 0u);
  ctl->ticket = 0u;
}

// Fused close/open half kicks, drift, strain advance, wrap, mirrors (see the
// FP64 integrator for the step structure).
__global__ void __launch_bounds__(kBlock)
k_integrate_mixed(Arrays A, BlockMap bm, StepArgs s, int close, int sample_kin,
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
  const double tilt = next_strain_m(RP) * L[1];
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
    const double im = 1.0 / V.w, iI = 1.0 / W.w;
    const double a0 = hdt * F[p] * im, a1 = hdt * F[Np + p] * im, a2 = hdt * F[2 * Np + p] * im;
    const double b0 = hdt * T[p] * iI, b1 = hdt * T[Np + p] * iI, b2 = hdt * T[2 * Np + p] * iI;
    if (close) {
      V.x += a0; V.y += a1; V.z += a2;
      W.x += b0; W.y += b1; W.z += b2;
      if (sample_kin) {
        const double u[3] = {V.x - rate * (P.y - 0.5 * L[1]), V.y, V.z};
        const double w[3] = {W.x, W.y, W.z + 0.5 * rate};
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
          for (int be = 0; be < 3; ++be) {
            kin[3 * al + be] = V.w * u[al] * u[be];
            kin[9 + 3 * al + be] = W.w * w[al] * w[be];
          }
      }
    }
    V.x += a0; V.y += a1; V.z += a2;
    W.x += b0; W.y += b1; W.z += b2;
    P.x += dt * V.x; P.y += dt * V.y; P.z += dt * V.z;
    if (!wrap_le_m(P.x, P.y, P.z, V.x, L, tilt, rate * L[1]))
      atomicOr(&ctl->err, kErrNonFinite);
    if (!isfinite(V.x + V.y + V.z + W.x + W.y + W.z)) atomicOr(&ctl->err, kErrNonFinite);
    A.pos[cur][p] = P;
    A.vel[cur][p] = V;
    A.omg[cur][p] = W;
    F[p] = 0.0; F[Np + p] = 0.0; F[2 * Np + p] = 0.0;
    T[p] = 0.0; T[Np + p] = 0.0; T[2 * Np + p] = 0.0;
    const double ux = V.x - rate * (P.y - 0.5 * L[1]);
    A.posm[p] = make_posm(RP, tilt, A.cell[p], P.x, P.y, P.z, P.w);
    A.velm[p] = make_float4((float)ux, (float)V.y, (float)V.z, 0.0f);
    A.omgm[p] = make_float4((float)W.x, (float)W.y, (float)W.z, 0.0f);
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
  if (last && threadIdx.x == 0) {
    __threadfence();
    integrator_epilogue_m(A, s, cond_handle, use_cond);
  }
}

__global__ void __launch_bounds__(kBlock)
k_finalize_mixed(Arrays A, BlockMap bm, StepArgs s, int sample_kin) {
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
    const double im = 1.0 / V.w, iI = 1.0 / W.w;
    V.x += hdt * F[p] * im; V.y += hdt * F[Np + p] * im; V.z += hdt * F[2 * Np + p] * im;
    W.x += hdt * T[p] * iI; W.y += hdt * T[Np + p] * iI; W.z += hdt * T[2 * Np + p] * iI;
    A.vel[cur][p] = V;
    A.omg[cur][p] = W;
    if (sample_kin) {
      const double u[3] = {V.x - rate * (P.y - 0.5 * Ly), V.y, V.z};
      const double w[3] = {W.x, W.y, W.z + 0.5 * rate};
#pragma unroll
      for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) {
          kin[3 * al + be] = V.w * u[al] * u[be];
          kin[9 + 3 * al + be] = W.w * w[al] * w[be];
        }
    }
  }
  if (sample_kin) block_sum_write<kKinLen>(kin, smem, A.kin_partial + (int64_t)b * kKinLen);
}

// Mirrors of the live copy from scratch (after a rebuild or a state change).
__global__ void k_mirror(Arrays A, int gated, int use_next) {
  if (gated && *(volatile const int*)&A.ctl->need_rebuild == 0) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int c = use_next ? (A.ctl->cur ^ 1) : A.ctl->cur;
  const int r = A.rep[c][p];
  const Replica& R = A.repl[r];
  const double4_32a P = A.pos[c][p];
  const double4_32a V = A.vel[c][p];
  const double4_32a W = A.omg[c][p];
  A.posm[p] = make_posm(R, R.tilt, A.cell[p], P.x, P.y, P.z, P.w);
  const double ux = V.x - R.rate * (P.y - 0.5 * R.L[1]);
  A.velm[p] = make_float4((float)ux, (float)V.y, (float)V.z, 0.0f);
  A.omgm[p] = make_float4((float)W.x, (float)W.y, (float)W.z, 0.0f);
}

// ---------------------------------------------------------------------------
// pair kernel, single-precision arithmetic
// ---------------------------------------------------------------------------
template <bool NOISE, bool FRIC, bool SAMPLE>
__global__ void __launch_bounds__(kBlock)
k_pair_mixed(Arrays A, BlockMap bm, StepArgs s) {
  __shared__ double smem[(kBlock / 32) * kPartialLen];
  const int b = blockIdx.x;
  const int r = bm.rep[b];
  const int p = bm.start[b] + threadIdx.x;
  const bool active = p < bm.end[b];
  const Ctl* ctl = A.ctl;
  const int cur = ctl->cur;
  const long long k = ctl->k;
  const Replica& RP = A.repl[r];
  const float rate = (float)RP.rate;
  const float eta = (float)RP.eta, kn = (float)RP.kn, kt = (float)RP.kt;
  const double mu = RP.mu, kt_d = RP.kt, kn_d = RP.kn;
  const float c = (float)RP.noise_c;
  const float cwx = (float)(RP.L[0] * RP.hcell[0]);
  const float cwy = (float)(RP.L[1] * RP.hcell[1]);
  const float cwz = (float)(RP.L[2] * RP.hcell[2]);
  const float ctilt = (float)(RP.tilt * RP.hcell[1]);
  const int ncx = RP.nc[0], ncy = RP.nc[1], ncz = RP.nc[2];
  const int64_t cbase = RP.cell_base;
  const uint32_t key0 = RP.key0, key1 = RP.key1;
  const int64_t t0 = RP.p0;
  const int64_t Np = A.Npad;
  const float xi_min = (float)s.xi_min, xi_max = (float)s.xi_max;
  const float tsign = (float)s.torque_sign;

  float vir[kPartialLen];
#pragma unroll
  for (int q = 0; q < kPartialLen; ++q) vir[q] = 0.0f;

  if (active) {
    const float4 P = A.posm[p];
    const float4 VP = A.velm[p];
    const float4 WP = A.omgm[p];
    const int tp = A.tag[cur][p];
    const int lp = A.cell[p] - (int)cbase;
    const int pcx = lp % ncx, pcy = (lp / ncx) % ncy, pcz = lp / (ncx * ncy);
    const float ap = P.w;
    float F[3] = {0.f, 0.f, 0.f}, T[3] = {0.f, 0.f, 0.f};
    if (s.onebody) {
      const float pi = 3.14159265358979f;
      const float gt = 6.0f * pi * eta * ap;
      const float gr = 8.0f * pi * eta * ap * ap * ap;
      float g[6] = {0, 0, 0, 0, 0, 0};
      if (NOISE) gauss6_f32(key0, key1, k, (uint32_t)(tp - t0), (uint32_t)(tp - t0), g);
      const float ct = c * sqrtf(gt), cr = c * sqrtf(gr);
      // U_inf - U = -u (peculiar velocity); Omega_inf - Omega
      F[0] = -gt * VP.x + (NOISE ? ct * g[0] : 0.f);
      F[1] = -gt * VP.y + (NOISE ? ct * g[1] : 0.f);
      F[2] = -gt * VP.z + (NOISE ? ct * g[2] : 0.f);
      T[0] = -gr * WP.x + (NOISE ? cr * g[3] : 0.f);
      T[1] = -gr * WP.y + (NOISE ? cr * g[4] : 0.f);
      T[2] = gr * (-0.5f * rate - WP.z) + (NOISE ? cr * g[5] : 0.f);
    }
    const int nn = A.nnb[cur][p];
    const int* __restrict__ row = A.nbr[cur] + p;
    unsigned long long cm_old = 0ull, cm_new = 0ull;
    if (FRIC) cm_old = A.cmsk[cur][p];
    double* __restrict__ hist = FRIC ? A.hist[cur] : nullptr;
    const int64_t hstride = (int64_t)A.kmax * Np;

    for (int sl = 0; sl < nn; ++sl) {
      const int q = __ldg(row + (int64_t)sl * Np);
      const float4 Q = __ldg(A.posm + q);
      const int lq = __ldg(A.cell + q) - (int)cbase;
      int dcx = lq % ncx - pcx, dcy = (lq / ncx) % ncy - pcy, dcz = lq / (ncx * ncy) - pcz;
      dcx = dcx > 1 ? dcx - ncx : (dcx < -1 ? dcx + ncx : dcx);
      dcy = dcy > 1 ? dcy - ncy : (dcy < -1 ? dcy + ncy : dcy);
      dcz = dcz > 1 ? dcz - ncz : (dcz < -1 ? dcz + ncz : dcz);
      float rpq[3];
      rpq[0] = (Q.x - P.x) + (cwx * (float)dcx + ctilt * (float)dcy);
      rpq[1] = (Q.y - P.y) + cwy * (float)dcy;
      rpq[2] = (Q.z - P.z) + cwz * (float)dcz;
      const float d2 = rpq[0] * rpq[0] + rpq[1] * rpq[1] + rpq[2] * rpq[2];
      const float S = ap + Q.w;
      const float d = sqrtf(d2);
      const float h = d - S;
      const float xi = 2.0f * h / S;
      if (xi > xi_max) continue;
      const float4 VQ = __ldg(A.velm + q);
      const float4 WQ = __ldg(A.omgm + q);
      const int tq = __ldg(A.tag[cur] + q);
      const bool p_is_i = tp < tq;
      const float sg = p_is_i ? 1.0f : -1.0f;
      const float rr[3] = {sg * rpq[0], sg * rpq[1], sg * rpq[2]};
      const float ai = p_is_i ? ap : Q.w, aj = p_is_i ? Q.w : ap;
      const float Ui[3] = {p_is_i ? VP.x : VQ.x, p_is_i ? VP.y : VQ.y, p_is_i ? VP.z : VQ.z};
      const float Uj[3] = {p_is_i ? VQ.x : VP.x, p_is_i ? VQ.y : VP.y, p_is_i ? VQ.z : VP.z};
      const float Wi[3] = {p_is_i ? WP.x : WQ.x, p_is_i ? WP.y : WQ.y, p_is_i ? WP.z : WQ.z};
      const float Wj[3] = {p_is_i ? WQ.x : WP.x, p_is_i ? WQ.y : WP.y, p_is_i ? WQ.z : WP.z};
      const float id = 1.0f / d;
      const float n[3] = {rr[0] * id, rr[1] * id, rr[2] * id};
      const float dU[3] = {Uj[0] - Ui[0] + rate * rr[1], Uj[1] - Ui[1], Uj[2] - Ui[2]};
      PairOut<float> o;
      if (s.lubrication) {
        const float xi_e = xi < xi_min ? xi_min : xi;
        const float lg = -__logf(xi_e);
        const Res8<float> R = resistances<float>(eta, ai, aj, xi_e, lg);
        float g[6] = {0, 0, 0, 0, 0, 0};
        const int li = (int)((p_is_i ? tp : tq) - t0);
        const int lj = (int)((p_is_i ? tq : tp) - t0);
        if (NOISE) gauss6_f32(key0, key1, k, (uint32_t)li, (uint32_t)lj, g);
        lub_brownian<float, NOISE>(R, n, dU, Wi, Wj, g, g + 3, c, tsign, o);
      } else {
#pragma unroll
        for (int q3 = 0; q3 < 3; ++q3) o.FL[q3] = o.FB[q3] = o.Ti[q3] = o.Tj[q3] = 0.f;
      }
      float FC[3] = {0.f, 0.f, 0.f}, TCi[3] = {0.f, 0.f, 0.f}, TCj[3] = {0.f, 0.f, 0.f};
      if (h < 0.0f && s.contact) {
        const float delta = -h;
        float Ft[3] = {0.f, 0.f, 0.f};
        if (FRIC && mu > 0.0) {
          double xt[3] = {0.0, 0.0, 0.0};
          const int64_t hi = (int64_t)sl * Np + p;
          if ((cm_old >> sl) & 1ull) {
            xt[0] = hist[hi]; xt[1] = hist[hi + hstride]; xt[2] = hist[hi + 2 * hstride];
          }
          if (s.advance) {
            const float ww[3] = {ai * Wi[0] + aj * Wj[0], ai * Wi[1] + aj * Wj[1],
                                 ai * Wi[2] + aj * Wj[2]};
            float wxn[3];
            cross3(ww, n, wxn);
            const double v[3] = {(double)(dU[0] - wxn[0]), (double)(dU[1] - wxn[1]),
                                 (double)(dU[2] - wxn[2])};
            const double nd[3] = {(double)n[0], (double)n[1], (double)n[2]};
            history_update(xt, nd, v, s.dt, kt_d, mu * kn_d * (double)delta);
          }
          hist[hi] = xt[0]; hist[hi + hstride] = xt[1]; hist[hi + 2 * hstride] = xt[2];
          cm_new |= 1ull << sl;
          Ft[0] = kt * (float)xt[0]; Ft[1] = kt * (float)xt[1]; Ft[2] = kt * (float)xt[2];
        }
#pragma unroll
        for (int q3 = 0; q3 < 3; ++q3) FC[q3] = -kn * delta * n[q3] + Ft[q3];
        float nxF[3];
        cross3(n, Ft, nxF);
#pragma unroll
        for (int q3 = 0; q3 < 3; ++q3) {
          TCi[q3] = ai * nxF[q3];
          TCj[q3] = aj * nxF[q3];
        }
      }
      float Fi[3], Ti_[3], Tj_[3];
#pragma unroll
      for (int q3 = 0; q3 < 3; ++q3) {
        Fi[q3] = FC[q3] + o.FL[q3] + o.FB[q3];
        Ti_[q3] = TCi[q3] + o.Ti[q3];
        Tj_[q3] = TCj[q3] + o.Tj[q3];
      }
      const int64_t qo = q;
#pragma unroll
      for (int q3 = 0; q3 < 3; ++q3) {
        F[q3] += sg * Fi[q3];
        T[q3] += p_is_i ? Ti_[q3] : Tj_[q3];
        atomicAdd(A.frc[cur] + q3 * Np + qo, (double)(-sg * Fi[q3]));
        atomicAdd(A.trq[cur] + q3 * Np + qo, (double)(p_is_i ? Tj_[q3] : Ti_[q3]));
      }
      if (SAMPLE) {
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
          for (int be = 0; be < 3; ++be) {
            vir[3 * al + be] += FC[al] * rr[be];
            vir[9 + 3 * al + be] += o.FL[al] * rr[be];
            vir[18 + 3 * al + be] += o.FB[al] * rr[be];
          }
      }
    }
    if (FRIC) A.cmsk[cur][p] = cm_new;
#pragma unroll
    for (int q3 = 0; q3 < 3; ++q3) {
      atomicAdd(A.frc[cur] + q3 * Np + p, (double)F[q3]);
      atomicAdd(A.trq[cur] + q3 * Np + p, (double)T[q3]);
    }
  }
  if (SAMPLE) {
    // per-thread single-precision partials, warp sums in single precision,
    // block and global accumulation in double
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int cc = 0; cc < kPartialLen; ++cc) {
      float x = vir[cc];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) smem[warp * kPartialLen + cc] = (double)x;
    }
    __syncthreads();
    if (threadIdx.x < kPartialLen) {
      double sum = 0.0;
      for (int w = 0; w < kBlock / 32; ++w) sum += smem[w * kPartialLen + threadIdx.x];
      A.pair_partial[(int64_t)b * kPartialLen + threadIdx.x] = sum;
    }
  }
}

template <bool NOISE, bool FRIC>
static void launch_pm(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                      cudaStream_t st) {
  if (s.sample)
    k_pair_mixed<NOISE, FRIC, true><<<bm.nblocks, kBlock, 0, st>>>(A, bm, s);
  else
    k_pair_mixed<NOISE, FRIC, false><<<bm.nblocks, kBlock, 0, st>>>(A, bm, s);
}

void launch_pair_mixed(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                       int tpp, cudaStream_t st) {
  (void)tpp;
  const bool noise = s.noise != 0, fric = s.friction != 0;
  if (noise && fric) launch_pm<true, true>(A, bm, s, st);
  else if (noise) launch_pm<true, false>(A, bm, s, st);
  else if (fric) launch_pm<false, true>(A, bm, s, st);
  else launch_pm<false, false>(A, bm, s, st);
}

void launch_integrate_mixed(const Arrays& A, const BlockMap& bm,
                            const StepArgs& s, int close, int sample_kin,
                            cudaStream_t st, unsigned long long cond_handle,
                            int use_cond) {
  k_integrate_mixed<<<bm.nblocks, kBlock, 0, st>>>(A, bm, s, close, sample_kin,
                                                   cond_handle, use_cond);
}

void launch_finalize_mixed(const Arrays& A, const BlockMap& bm,
                           const StepArgs& s, int sample_kin, cudaStream_t st) {
  k_finalize_mixed<<<bm.nblocks, kBlock, 0, st>>>(A, bm, s, sample_kin);
}

void launch_mirror(const Arrays& A, const BlockMap& bm, cudaStream_t st) {
  (void)bm;
  k_mirror<<<(unsigned)((A.N + kBlock - 1) / kBlock), kBlock, 0, st>>>(A, 0, 0);
}

void launch_mirror_gated_next(const Arrays& A, cudaStream_t st) {
  k_mirror<<<(unsigned)((A.N + kBlock - 1) / kBlock), kBlock, 0, st>>>(A, 1, 1);
}

}  // namespace susp
