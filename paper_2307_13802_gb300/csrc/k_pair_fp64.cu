// k_pair_fp64.cu -- per-timestep pair force evaluation in double precision
// (the plain FP64 path).  Compiled with multiply-add contraction (a product
// and a sum rounded once; about a sixth fewer FP64 instructions than the
// written order), and the resistances and the unit vector use reciprocal
// products in place of the printed quotients (a few ulps from the printed
// forms), which takes the FP64 divisions, each a long sequence on the FP64
// pipe, from 21 to 10 per lubricated pair.
//
// Each warp owns 32 spheres of the sorted order and flattens their half-list
// rows into one list of items.  A pass tests 32 items against the widest
// interaction range and queues those within it in shared memory, touching
// pairs apart from the others; the pair arithmetic then runs on full
// batches of 32 queued pairs, so rows of uneven length, pairs beyond the
// cutoff and the contact branch leave no lanes idle through the FP64
// arithmetic.  For each pair it forms the minimum-image gap
// h = |r| - (a_i + a_j) and xi = 2h/(a_i + a_j) (Sec. II.B); pairs with
// xi > xi_max are skipped.  Each remaining pair is oriented by tag
// (i = lower tag, n from i to j) and gets
//   - lubrication, Eqs. 8, 13, 14, with resistances Eqs. 9-12, 15-18 at
//     xi_eff = max(xi, xi_min);
//   - pair Brownian force and torques, Eqs. 22-24, Philox counter
//     (k, tag_i, tag_j);
//   - for h < 0 the contact force and torques, Eqs. 3-4, with tangential
//     history (double, per list slot) and the Coulomb cap.
// Both spheres' shares, and each sphere's one-body drag (Eqs. 5-6) and
// noise (Eqs. 20-21), are added with double atomics; the new contact bits of
// a warp's spheres are gathered in shared memory.  On sampled evaluations the pair virials F (x) r of the
// three components are reduced per block (Sec. II.A, II.B, II.D).
// Optional terms: the short-range repulsion of Eq. 34 (read as the force on
// j, so -(A/kappa) exp(-h/kappa) n on i) for h <= rep_cut kappa, with its
// own virial; and on sampled evaluations the structural Brownian sums of
// Eq. 26, sum over pairs of w n n with w the number of the two spheres whose
// shell h <= shell a holds the pair (scaled by -kT / (shell V) on the host).
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "philox.cuh"
#include "susp_internal.h"

namespace susp {

// DET: the shares go to per-slot and per-sphere records that k_det_gather
// sums in a fixed order, instead of double atomics
template <bool NOISE, bool FRIC, bool SAMPLE, bool DET>
__global__ void __launch_bounds__(kBlock, 2)
k_pair_fp64(Arrays A, BlockMap bm, StepArgs s) {
  __shared__ double smem[(kBlock / 32) * kPartialLen];
  const int b = blockIdx.x;
  const int r = bm.rep[b];
  const int p = bm.start[b] + threadIdx.x;
  const bool active = p < bm.end[b];
  const Ctl* ctl = A.ctl;
  const int cur = ctl->cur;
  const long long k = ctl->k;
  const Replica& RP = A.repl[r];
  const double L[3] = {RP.L[0], RP.L[1], RP.L[2]};
  const double iL[3] = {RP.iL[0], RP.iL[1], RP.iL[2]};
  const double tilt = RP.tilt;
  const double rate = RP.rate;
  const double eta = RP.eta, kn = RP.kn, kt = RP.kt, mu = RP.mu;
  const double c = RP.noise_c;
  const uint32_t key0 = RP.key0, key1 = RP.key1;
  const int64_t t0 = RP.p0;
  const int64_t Np = A.Npad;

  // pair virials of a sampled evaluation: each thread's own running sums in
  // shared memory (entry e of thread t at sVir[e * kBlock + t]), which keeps
  // them out of registers so that two blocks fit on an SM
  extern __shared__ double sVir[];
  if (SAMPLE) {
#pragma unroll
    for (int q = 0; q < kPartialLen; ++q) sVir[q * kBlock + threadIdx.x] = 0.0;
  }

  const int tid = threadIdx.x, lane = tid & 31;
  __shared__ unsigned long long sM[kBlock];  // new contact bits of the block's spheres
  sM[tid] = 0ull;
  int nn = 0;
  if (active) {
    nn = A.nnb[cur][p];
    if (s.onebody) {
      // Eqs. 5-6 and 20-21
      const double4_32a P = A.pos[cur][p];
      const double4_32a VP = A.vel[cur][p];
      const double4_32a WP = A.omg[cur][p];
      const int tp = A.tag[cur][p];
      const double ap = P.w;
      const double pi = 3.14159265358979323846;
      const double gt = 6.0 * pi * eta * ap;
      const double gr = 8.0 * pi * eta * ap * ap * ap;
      const double Uinf0 = rate * (P.y - 0.5 * L[1]);
      const double Winf2 = -0.5 * rate;
      double g[6] = {0, 0, 0, 0, 0, 0};
      if (NOISE) gauss6_f64(key0, key1, k, (uint32_t)(tp - t0), (uint32_t)(tp - t0), g);
      const double ct = c * sqrt(gt), cr = c * sqrt(gr);
      const double F[3] = {gt * (Uinf0 - VP.x) + (NOISE ? ct * g[0] : 0.0),
                           gt * (0.0 - VP.y) + (NOISE ? ct * g[1] : 0.0),
                           gt * (0.0 - VP.z) + (NOISE ? ct * g[2] : 0.0)};
      const double T[3] = {gr * (0.0 - WP.x) + (NOISE ? cr * g[3] : 0.0),
                           gr * (0.0 - WP.y) + (NOISE ? cr * g[4] : 0.0),
                           gr * (Winf2 - WP.z) + (NOISE ? cr * g[5] : 0.0)};
#pragma unroll
      for (int q3 = 0; q3 < 3; ++q3) {
        if (DET) {
          A.det_own[q3 * Np + p] = F[q3];
          A.det_own[(3 + q3) * Np + p] = T[q3];
        } else {
          atomicAdd(A.frc[cur] + q3 * Np + p, F[q3]);
          atomicAdd(A.trq[cur] + q3 * Np + p, T[q3]);
        }
      }
    } else if (DET) {
#pragma unroll
      for (int c6 = 0; c6 < 6; ++c6) A.det_own[c6 * Np + p] = 0.0;
    }
  }
  // the warp's 32 rows flattened into one list of items: lane l takes items
  // l, l + 32, ... whatever the rows' lengths
  int incl = nn;
#pragma unroll
  for (int o2 = 1; o2 < 32; o2 <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o2);
    if (lane >= o2) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  const int excl = incl - nn;
  double* __restrict__ hist = FRIC ? A.hist[cur] : nullptr;
  const int64_t hstride = (int64_t)A.kmax * Np;
  const int pw = bm.start[b] + (tid - lane);   // first sphere of the warp
  __syncwarp();
  // One listed pair (owner row ow of the warp, slot sl): the exact range
  // tests, then the pair's physics.  It has a single call site, in the
  // batch step of the work loop below.
  auto item = [&](int ow, int sl) {
    const int po = pw + ow;
    const int q = A.nbr[cur][(int64_t)sl * Np + po] & kNbrIndexMask;
    const double4_32a P = A.pos[cur][po];
    const double4_32a VP = A.vel[cur][po];
    const double4_32a WP = A.omg[cur][po];
    const int tp = A.tag[cur][po];
    const double ap = P.w;
    const double4_32a Q = A.pos[cur][q];
    double rpq[3], sy;
    min_image_f64(Q.x - P.x, Q.y - P.y, Q.z - P.z, L, iL, tilt, rpq, &sy);
    const double d2 = rpq[0] * rpq[0] + rpq[1] * rpq[1] + rpq[2] * rpq[2];
    const double d = sqrt(d2);
    const double S = ap + Q.w;
    const double h = d - S;
    const double xi = 2.0 * h / S;
    const double kappa = 0.01 * S;
    const bool lub = xi <= s.xi_max;
    const bool rep = s.rep_on && RP.rep_A > 0.0 && h <= s.rep_cut * kappa;
    const bool shp = SAMPLE && s.structural && h <= s.shell * ap;
    const bool shq = SAMPLE && s.structural && h <= s.shell * Q.w;
    if (lub || rep || shp || shq) {

    const double4_32a VQ = A.vel[cur][q];
    const double4_32a WQ = A.omg[cur][q];
    const int tq = A.tag[cur][q];
    const bool p_is_i = tp < tq;
    // orient: i = lower tag, n and r from i to j
    double rr[3], syij, ai, aj;
    double Ui[3], Uj[3], Wi[3], Wj[3];
    if (p_is_i) {
      rr[0] = rpq[0]; rr[1] = rpq[1]; rr[2] = rpq[2]; syij = sy;
      ai = ap; aj = Q.w;
      Ui[0] = VP.x; Ui[1] = VP.y; Ui[2] = VP.z; Uj[0] = VQ.x; Uj[1] = VQ.y; Uj[2] = VQ.z;
      Wi[0] = WP.x; Wi[1] = WP.y; Wi[2] = WP.z; Wj[0] = WQ.x; Wj[1] = WQ.y; Wj[2] = WQ.z;
    } else {
      rr[0] = -rpq[0]; rr[1] = -rpq[1]; rr[2] = -rpq[2]; syij = -sy;
      ai = Q.w; aj = ap;
      Ui[0] = VQ.x; Ui[1] = VQ.y; Ui[2] = VQ.z; Uj[0] = VP.x; Uj[1] = VP.y; Uj[2] = VP.z;
      Wi[0] = WQ.x; Wi[1] = WQ.y; Wi[2] = WQ.z; Wj[0] = WP.x; Wj[1] = WP.y; Wj[2] = WP.z;
    }
    const double id = 1.0 / d;
    const double n[3] = {rr[0] * id, rr[1] * id, rr[2] * id};
    const double dU[3] = {Uj[0] - syij * rate * L[1] - Ui[0], Uj[1] - Ui[1],
                          Uj[2] - Ui[2]};

    if (SAMPLE && (shp || shq)) {
      const double w = (shp ? 1.0 : 0.0) + (shq ? 1.0 : 0.0);
#pragma unroll
      for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) sVir[(kStrOff + 3 * al + be) * kBlock + tid] += w * n[al] * n[be];
    }
    double FR[3] = {0.0, 0.0, 0.0};
    if (rep) {
      const double f = RP.rep_A / kappa * exp(-h / kappa);
#pragma unroll
      for (int q3 = 0; q3 < 3; ++q3) FR[q3] = -f * n[q3];
    }

    PairOut<double> o;
    if (lub && s.lubrication) {
      const double xi_e = xi < s.xi_min ? s.xi_min : xi;
      const double ixi = 1.0 / xi_e;
      const double lg = log(ixi);
      const Res8<double> R = resistances_rcp(eta, ai, aj, ixi, lg);
      double g[6] = {0, 0, 0, 0, 0, 0};
      const int li = (int)((p_is_i ? tp : tq) - t0);
      const int lj = (int)((p_is_i ? tq : tp) - t0);
      if (NOISE) gauss6_f64(key0, key1, k, (uint32_t)li, (uint32_t)lj, g);
      lub_brownian<double, NOISE>(R, n, dU, Wi, Wj, g, g + 3, c, s.torque_sign, o);
    } else {
#pragma unroll
      for (int q3 = 0; q3 < 3; ++q3) o.FL[q3] = o.FB[q3] = o.Ti[q3] = o.Tj[q3] = 0.0;
    }

    double FC[3] = {0.0, 0.0, 0.0}, TCi[3] = {0.0, 0.0, 0.0}, TCj[3] = {0.0, 0.0, 0.0};
    if (h < 0.0 && s.contact) {
      const double delta = -h;
      double Ft[3] = {0.0, 0.0, 0.0};
      if (FRIC && mu > 0.0) {
        double xt[3] = {0.0, 0.0, 0.0};
        const int64_t hi = (int64_t)sl * Np + po;
        if ((A.cmsk[cur][po] >> sl) & 1ull) {
          xt[0] = hist[hi]; xt[1] = hist[hi + hstride]; xt[2] = hist[hi + 2 * hstride];
        }
        if (s.advance) {
          const double ww[3] = {ai * Wi[0] + aj * Wj[0], ai * Wi[1] + aj * Wj[1],
                                ai * Wi[2] + aj * Wj[2]};
          double wxn[3];
          cross3(ww, n, wxn);
          const double v[3] = {dU[0] - wxn[0], dU[1] - wxn[1], dU[2] - wxn[2]};
          history_update(xt, n, v, s.dt, kt, mu * kn * delta);
        }
        hist[hi] = xt[0]; hist[hi + hstride] = xt[1]; hist[hi + 2 * hstride] = xt[2];
        atomicOr(&sM[tid - lane + ow], 1ull << sl);
        Ft[0] = kt * xt[0]; Ft[1] = kt * xt[1]; Ft[2] = kt * xt[2];
      }
#pragma unroll
      for (int q3 = 0; q3 < 3; ++q3) FC[q3] = -kn * delta * n[q3] + Ft[q3];
      double nxF[3];
      cross3(n, Ft, nxF);
#pragma unroll
      for (int q3 = 0; q3 < 3; ++q3) {
        TCi[q3] = ai * nxF[q3];
        TCj[q3] = aj * nxF[q3];
      }
    }

    double Fi[3], Ti_[3], Tj_[3];
#pragma unroll
    for (int q3 = 0; q3 < 3; ++q3) {
      Fi[q3] = FC[q3] + o.FL[q3] + o.FB[q3] + FR[q3];
      Ti_[q3] = TCi[q3] + o.Ti[q3];
      Tj_[q3] = TCj[q3] + o.Tj[q3];
    }
    const int64_t qo = q;
    const double sgn = p_is_i ? 1.0 : -1.0;
    const double* To = p_is_i ? Ti_ : Tj_;
    const double* Tq = p_is_i ? Tj_ : Ti_;
    if (DET) {
      const int64_t e = (int64_t)sl * Np + po, KN = (int64_t)A.kmax * Np;
#pragma unroll
      for (int q3 = 0; q3 < 3; ++q3) {
        A.det_slot[q3 * KN + e] = sgn * Fi[q3];
        A.det_slot[(3 + q3) * KN + e] = To[q3];
        A.det_slot[(6 + q3) * KN + e] = Tq[q3];
      }
    } else {
#pragma unroll
      for (int q3 = 0; q3 < 3; ++q3) {
        atomicAdd(A.frc[cur] + q3 * Np + po, sgn * Fi[q3]);
        atomicAdd(A.trq[cur] + q3 * Np + po, To[q3]);
        atomicAdd(A.frc[cur] + q3 * Np + qo, -sgn * Fi[q3]);
        atomicAdd(A.trq[cur] + q3 * Np + qo, Tq[q3]);
      }
    }
    if (SAMPLE) {
#pragma unroll
      for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) {
          sVir[(3 * al + be) * kBlock + tid] += FC[al] * rr[be];
          sVir[(9 + 3 * al + be) * kBlock + tid] += o.FL[al] * rr[be];
          sVir[(18 + 3 * al + be) * kBlock + tid] += o.FB[al] * rr[be];
          sVir[(kRepOff + 3 * al + be) * kBlock + tid] += FR[al] * rr[be];
        }
    }
    } else if (DET) {
      // a listed pair that does not interact: its slot holds zeros
      const int64_t e = (int64_t)sl * Np + po, KN = (int64_t)A.kmax * Np;
#pragma unroll
      for (int c9 = 0; c9 < 9; ++c9) A.det_slot[c9 * KN + e] = 0.0;
    }
  };

  // Work loop of the warp, all decisions warp-uniform.  A pass reads the next
  // 32 list items and queues those within the widest interaction range
  // (touching pairs apart from the others) in two 64-entry rings in shared
  // memory; a batch runs 32 queued pairs of one ring, one per lane, so pairs
  // beyond the range and the contact branch leave no lanes idle through the
  // FP64 arithmetic.  What is left at the end runs as one or two batches.
  constexpr int kQ = 64;
  __shared__ int qE[2][kBlock / 32][kQ];   // ow | sl << 5
  const int warp = tid >> 5;
  // the range test widened by a relative 1e-9 above the rounding of the
  // exact tests, which decide in item()
  const double rcf = 1.0 + 0.5 * s.xi_max;
  const bool rep_any = s.rep_on && RP.rep_A > 0.0;
  const double repf = 1.0 + 0.01 * s.rep_cut;
  const bool strc = SAMPLE && s.structural;
  int h0 = 0, n0 = 0, h1 = 0, n1 = 0, base = 0;
  while (true) {
    int c0 = 0, c1 = 0;
    if (n0 >= 32) {
      c0 = 32;
    } else if (n1 >= 32) {
      c1 = 32;
    } else if (base < total) {
      const int t = base + lane;
      // owner row o of item t: the number of rows ending at or before t
      int ow = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, ow + step - 1);
        if (v <= t) ow += step;
      }
      const int sl = t - __shfl_sync(0xffffffffu, excl, ow);
      bool keep = false, touch = false;
      if (t < total) {
        const int po = pw + ow;
        const int q = A.nbr[cur][(int64_t)sl * Np + po] & kNbrIndexMask;
        const double4_32a P = A.pos[cur][po];
        const double4_32a Q = A.pos[cur][q];
        double rpq[3], sy;
        min_image_f64(Q.x - P.x, Q.y - P.y, Q.z - P.z, L, iL, tilt, rpq, &sy);
        const double d2 = rpq[0] * rpq[0] + rpq[1] * rpq[1] + rpq[2] * rpq[2];
        const double S = P.w + Q.w;
        double rc = S * rcf;
        if (rep_any) rc = fmax(rc, S * repf);
        if (strc) rc = fmax(rc, S + s.shell * fmax(P.w, Q.w));
        keep = d2 <= rc * rc * (1.0 + 1e-9);
        touch = keep && d2 <= S * S * (1.0 + 1e-9);
        if (DET && !keep) {
          // a listed pair beyond every range: its slot holds zeros
          const int64_t e = (int64_t)sl * Np + po, KN = (int64_t)A.kmax * Np;
#pragma unroll
          for (int c9 = 0; c9 < 9; ++c9) A.det_slot[c9 * KN + e] = 0.0;
        }
      }
      const unsigned m0 = __ballot_sync(0xffffffffu, keep && !touch);
      const unsigned m1 = __ballot_sync(0xffffffffu, touch);
      if (keep) {
        const unsigned below = (1u << lane) - 1u;
        const int e = touch ? (h1 + n1 + __popc(m1 & below)) & (kQ - 1)
                            : (h0 + n0 + __popc(m0 & below)) & (kQ - 1);
        qE[touch ? 1 : 0][warp][e] = ow | (sl << 5);
      }
      n0 += __popc(m0);
      n1 += __popc(m1);
      __syncwarp();
      base += 32;
      continue;
    } else if (n0 + n1 > 32) {
      c1 = n1;   // the touching pairs first, then the rest in one batch
    } else if (n0 + n1 > 0) {
      c0 = n0;
      c1 = n1;
    } else {
      break;
    }
    // lanes [0, c0) take ring 0 from its head, lanes [c0, c0 + c1) ring 1
    if (lane < c0 + c1) {
      const int qi = lane < c0 ? 0 : 1;
      const int e = qi ? (h1 + lane - c0) & (kQ - 1) : (h0 + lane) & (kQ - 1);
      const int v = qE[qi][warp][e];
      item(v & 31, v >> 5);
    }
    __syncwarp();
    h0 = (h0 + c0) & (kQ - 1);
    n0 -= c0;
    h1 = (h1 + c1) & (kQ - 1);
    n1 -= c1;
  }
  __syncwarp();
  if (FRIC && active) A.cmsk[cur][p] = sM[tid];
  if (SAMPLE) {
    // the block's sums in a fixed order: a shuffle tree in each warp, then
    // the warps in index order
    const int warp = tid >> 5;
    for (int c2 = 0; c2 < kPartialLen; ++c2) {
      double x = sVir[c2 * kBlock + tid];
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) x += __shfl_down_sync(0xffffffffu, x, o2);
      if (lane == 0) smem[warp * kPartialLen + c2] = x;
    }
    __syncthreads();
    for (int c2 = tid; c2 < kPartialLen; c2 += kBlock) {
      double sum = 0.0;
      for (int w2 = 0; w2 < kBlock / 32; ++w2) sum += smem[w2 * kPartialLen + c2];
      A.pair_partial[(int64_t)b * kPartialLen + c2] = sum;
    }
  }
}

// dynamic shared memory of a sampled launch: the per-thread virial sums
constexpr int kVirSmem = kPartialLen * kBlock * (int)sizeof(double);

template <bool NOISE, bool FRIC, bool DET>
static void launch_sample(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                          cudaStream_t st) {
  if (s.sample)
    k_pair_fp64<NOISE, FRIC, true, DET><<<bm.nblocks, kBlock, kVirSmem, st>>>(A, bm, s);
  else
    k_pair_fp64<NOISE, FRIC, false, DET><<<bm.nblocks, kBlock, 0, st>>>(A, bm, s);
}

template <bool DET>
static void launch_det(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                       cudaStream_t st) {
  const bool noise = s.noise != 0;
  const bool fric = s.friction != 0;
  if (noise && fric) launch_sample<true, true, DET>(A, bm, s, st);
  else if (noise) launch_sample<true, false, DET>(A, bm, s, st);
  else if (fric) launch_sample<false, true, DET>(A, bm, s, st);
  else launch_sample<false, false, DET>(A, bm, s, st);
}

// The sampled launches use more dynamic shared memory than the 48 KB
// default; the limit is raised per function on the current device (before
// any stream capture: the handle's allocation calls this).
int prepare_pair_fp64() {
  cudaError_t e = cudaSuccess;
  const auto raise = [&](const void* f) {
    const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               kVirSmem);
    if (r != cudaSuccess) e = r;
  };
  raise((const void*)k_pair_fp64<true, true, true, false>);
  raise((const void*)k_pair_fp64<true, false, true, false>);
  raise((const void*)k_pair_fp64<false, true, true, false>);
  raise((const void*)k_pair_fp64<false, false, true, false>);
  raise((const void*)k_pair_fp64<true, true, true, true>);
  raise((const void*)k_pair_fp64<true, false, true, true>);
  raise((const void*)k_pair_fp64<false, true, true, true>);
  raise((const void*)k_pair_fp64<false, false, true, true>);
  return e == cudaSuccess ? 0 : (int)e;
}

void launch_pair_fp64(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                      int tpp, cudaStream_t st) {
  (void)tpp;
  if (A.det) {
    launch_det<true>(A, bm, s, st);
    launch_det_gather(A, st);
  } else {
    launch_det<false>(A, bm, s, st);
  }
}

}  // namespace susp
