// k_pair_mixed.cu -- per-timestep pair force evaluation, mixed precision.
//
// The same physics as the FP64 kernel (Sec. II.A-II.C: regularised
// lubrication, pair Brownian force and torques, contact with Coulomb-capped
// tangential history, one-body drag and noise, pair virials) in single
// precision on the mirrors written by the integrator, with no FP64-pipe
// instruction on the per-pair path:
//   - Work mapping: each warp owns 32 consecutive spheres of the sorted
//     order and flattens their half-list rows into one work list (a warp
//     prefix sum of the row lengths); lane l takes items l, l+32, ...  Rows
//     of uneven length therefore cost no idle lanes.
//   - Geometry: r = (posm_q - posm_p) + H(t) dc / nc with the home-cell
//     difference dc in {-1, 0, 1}^3 taken from the top bits of the list
//     entry (the stencil offset the list build found the partner at); pairs
//     beyond the lubrication cutoff are rejected on |r|^2 before any square
//     root.
//   - Accumulation: the owner's share goes to shared-memory float
//     accumulators (one vector reduction per sphere at the end), the
//     partner's share straight to its float4 accumulator with one
//     red.global.add.v4.f32 for the force and one for the torque.
//   - Tangential history: double-float (hi, lo) per component in one
//     32-byte record per list slot (a touching pair reads and writes one
//     sector), updated with error-free FP32 transformations (dfloat.cuh), so
//     it accumulates with a 48-bit significand.
//   - Stresses: single-precision virials summed over the warp batch by batch
//     (a reduce-scatter leaves entry l in lane l); the warp sums are folded
//     into the block partial in double, and the sums over blocks, replicas
//     and time are double as well.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "reduce.cuh"
#include "dfloat.cuh"
#include "philox.cuh"
#include "susp_internal.h"

namespace susp {

// Scalar resistances of Eqs. 9-12 and 15-18 in a reciprocal form
// (beta = a_j/a_i, r = 1/(1+beta), 1/(1+1/beta) = beta r):
//   XA11 = 6 pi eta a_i r^3 (2 beta^2 / xi + beta (1 + 7 beta + beta^2)/5 L)
//   YA11 = 6 pi eta a_i r^3 (4 beta (2 + beta + 2 beta^2)/15) L
//   YB11 = -4 pi eta a_i^2 r^2 (beta (4 + beta)/5) L
//   YB21 = -4 pi eta a_j^2 r^2 ((4 beta + 1)/5) L
//   YC11 = 8 pi eta a_i^3 r (2 beta/5) L,   YC12 = 8 pi eta a_i^3 r (beta^2/10) L
//   YC22 = 8 pi eta a_j^3 r (2/5) L,        YC21 = 8 pi eta a_j^3 r (1/(10 beta)) L
// with L = ln(1/xi_e).
__device__ __forceinline__ Res8<float> resistances_f(float eta, float ai, float aj,
                                                     float ixi, float L) {
  const float pi = 3.14159265358979f;
  const float iai = 1.0f / ai;
  const float beta = aj * iai;
  const float r = 1.0f / (1.0f + beta);
  const float r2 = r * r, r3 = r2 * r;
  const float b2 = beta * beta;
  const float ta = 6.0f * pi * eta * ai * r3;
  Res8<float> R;
  R.XA11 = ta * (2.0f * b2 * ixi + 0.2f * beta * (1.0f + 7.0f * beta + b2) * L);
  R.YA11 = ta * (4.0f / 15.0f) * beta * (2.0f + beta + 2.0f * b2) * L;
  const float tb = -4.0f * pi * eta * r2 * 0.2f * L;
  R.YB11 = tb * ai * ai * beta * (4.0f + beta);
  R.YB21 = tb * aj * aj * (4.0f * beta + 1.0f);
  const float tc = 8.0f * pi * eta * r * L;
  const float ai3 = ai * ai * ai, aj3 = aj * aj * aj;
  R.YC11 = tc * ai3 * 0.4f * beta;
  R.YC12 = tc * ai3 * 0.1f * b2;
  R.YC22 = tc * aj3 * 0.4f;
  R.YC21 = tc * aj3 * 0.1f / beta;
  return R;
}

// Tangential history update in double-float (reading of Sec. II.A): rotate
// into the current tangent plane keeping the length, add v_t dt, cap at
// mu kn delta / kt.  Over one step the rotation and the increment are small
// against the stored displacement, so their sum is formed in single
// precision and added to each double-float component once.
__device__ __forceinline__ void history_update_df(float* xh, float* xl, const float* n,
                                                  const float* v, float dt, float kt,
                                                  float fmax) {
  const float nv = n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
  float c[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) c[q] = (v[q] - n[q] * nv) * dt;
  const float len0sq = xh[0] * xh[0] + xh[1] * xh[1] + xh[2] * xh[2];
  if (len0sq > 0.0f) {
    const float sn = n[0] * xh[0] + n[1] * xh[1] + n[2] * xh[2] +
                     (n[0] * xl[0] + n[1] * xl[1] + n[2] * xl[2]);
    const float q = sn * sn / len0sq;
    if (q < 1.0f) {
      // (x - n sn)(1 + eps) - x with 1 + eps = 1/sqrt(1 - q)
      const float eps = q < 1e-3f ? q * (0.5f + 0.375f * q) : rsqrtf(1.0f - q) - 1.0f;
      const float sc = sn * (1.0f + eps);
#pragma unroll
      for (int k = 0; k < 3; ++k) c[k] += xh[k] * eps - n[k] * sc;
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) xh[k] = xl[k] = 0.0f;
    }
  }
  df x[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) x[k] = df_add_f(df{xh[k], xl[k]}, c[k]);
  const float ft = kt * sqrtf(x[0].hi * x[0].hi + x[1].hi * x[1].hi + x[2].hi * x[2].hi);
  if (ft > fmax) {
    const float sc = fmax / ft;
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = df{x[k].hi * sc, x[k].lo * sc};
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    xh[k] = x[k].hi;
    xl[k] = x[k].lo;
  }
}

// (qh + ql) - (ph + pl) + (sh + sl) as a double-float (rh, rl): the large
// parts by two error-free sums, the small parts in single precision.
__device__ __forceinline__ void df_diff_shift(float qh, float ql, float ph, float pl, float sh,
                                              float sl, float& rh, float& rl) {
  float s1, e1, s2, e2;
  two_sum(qh, -ph, s1, e1);
  two_sum(s1, sh, s2, e2);
  const float lo = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fsub_rn(ql, pl), sl));
  fast_two_sum(s2, lo, rh, rl);
}

// Packed single-precision pairs (two lanes of one FP32 instruction on
// sm_100 and later), used where the operands come in natural pairs: the x
// and y components of the gap, and the (x, y) rows of the virial products.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  e = sub2(b, sub2(s, a));
}

__device__ __forceinline__ float2 dup2(float s) { return make_float2(s, s); }

// Sums v[0..31] over the 32 lanes of a warp and leaves the total of
// component l in lane l: five halving stages, in each of which a lane keeps
// one half of its components and adds the partner's copy of that half
// (lane ^ offset).  31 shuffles per lane instead of 5 per component.
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = up ? v[i] : v[i + off];
      const float keep = up ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

// resident blocks per SM the register allocation targets (4 measured
// fastest at N = 1M: 64 registers without spills; 3 blocks at 80 registers
// took 0.214 ms against 0.201 ms)
#ifndef SUSP_PAIR_MINBLOCKS
#define SUSP_PAIR_MINBLOCKS 4
#endif

// EXTRA: the optional repulsion (Eq. 34) and structural sums (Eq. 26) are
// compiled in; without them the kernel keeps the smaller body
template <bool NOISE, bool FRIC, bool SAMPLE, bool EXTRA>
__global__ void __launch_bounds__(kBlock, SUSP_PAIR_MINBLOCKS)
k_pair_mixed(Arrays A, BlockMap bm, StepArgs s) {
  constexpr unsigned kFull = 0xffffffffu;
  __shared__ float4 sF[kBlock];
  __shared__ float4 sT[kBlock];
  __shared__ unsigned long long sM[kBlock];
  __shared__ float sW[(kBlock / 32) * kPartialLen];
  __shared__ float2 sShx[9];    // x shift dcx w_x + dcy tilt/ncy, double-float
  __shared__ float sA[kBlock];  // radius (high word) of each owner sphere
  __shared__ int sArrive;
  const int b = blockIdx.x;
  // the integrator that follows may start its blocks (which wait for this
  // grid before reading forces) once every block of this grid has started
  asm volatile("griddepcontrol.launch_dependents;");
  // the previous sampled step's stress: block ch < nchunk reduces chunk ch
  // of it before its own spheres, and the last chunk of a replica sums the
  // replica (its pair partials are in the other buffer)
  if (s.fuse_red && b < A.nchunk)
    reduce_chunk_then_replica(A, b, A.pair_partial_w + (int64_t)(s.ppar ^ 1) * gridDim.x * kPartialLen,
                              1, 1);
  const int r = bm.rep[b];
  const Replica& RP = A.repl[r];
  if (threadIdx.x == 0) sArrive = 0;
  // per-warp block-partial slots; the repulsion and structural parts are
  // accumulated into them while the warp works
  for (int i = threadIdx.x; i < (kBlock / 32) * kPartialLen; i += kBlock) sW[i] = 0.0f;
  if (threadIdx.x < 9) {
    const float fx = (float)((int)threadIdx.x / 3 - 1), fy = (float)((int)threadIdx.x % 3 - 1);
    const df v = df_add(df{RP.cw_hi[0] * fx, RP.cw_lo[0] * fx}, df{RP.ct_hi * fy, RP.ct_lo * fy});
    sShx[threadIdx.x] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  const int pb = bm.start[b], pe = bm.end[b];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int p = pb + tid;
  const bool active = p < pe;
  const Ctl* ctl = A.ctl;
  const int cur = ctl->cur;
  const long long k = ctl->k;
  const float rate = RP.rate_f, eta = RP.eta_f, kn = RP.kn_f, kt = RP.kt_f, mu = RP.mu_f;
  const float c = RP.noise_cf;
  const float cwx = RP.cwf[0], cwy = RP.cwf[1], cwz = RP.cwf[2], ctilt = RP.ctilt_f;
  const float cw1h = RP.cw_hi[1], cw1l = RP.cw_lo[1], cw2h = RP.cw_hi[2], cw2l = RP.cw_lo[2];
  const uint32_t key0 = RP.key0, key1 = RP.key1;
  const int t0 = (int)RP.p0;
  const int64_t Np = A.Npad;
  const float xi_min = s.xi_min_f, xi_max = s.xi_max_f;
  // optional terms: repulsion (Eq. 34) of this replica, structural sums
  // (Eq. 26) on sampled steps; rcf and shf widen the single-precision range
  // test to the widest interaction range in use
  const bool rep_on = EXTRA && s.rep_on && RP.rep_A_f > 0.0f;
  const float repA = RP.rep_A_f, rep_hc = s.rep_hc_f;
  const bool strc = EXTRA && SAMPLE && s.structural;
  const float shf = strc ? s.shell_f : 0.0f;
  const float rcf = rep_on ? fmaxf(1.0f + 0.5f * xi_max, s.rep_fac_f) : 1.0f + 0.5f * xi_max;
  const float tsign = s.tsign_f;
  const float dtf = s.dt_f;
  const float pi = 3.14159265358979f;
  float4* __restrict__ F4 = reinterpret_cast<float4*>(A.frc[cur]);
  float4* __restrict__ T4 = reinterpret_cast<float4*>(A.trq[cur]);
  const float4* __restrict__ PM = A.posm;
  const float4* __restrict__ VM = A.velm;
  // spins: the high halves of the double-float records (a normalised
  // double-float's high word is its value rounded to single precision)
  const float4* __restrict__ OMD = reinterpret_cast<const float4*>(A.omg[cur]);
  const int* __restrict__ nbr = A.nbr[cur];
  // tangential history: one 32-byte record per list slot,
  // (x_hi, x_lo, y_hi, y_lo), (z_hi, z_lo, -, -)
  float4* __restrict__ hist = reinterpret_cast<float4*>(A.hist[cur]);

  // ---- own sphere: one-body drag and noise (Eqs. 5-6, 20-21) -------------
  int nn = 0;
  unsigned long long cm_own = 0ull;
  {
    float4 f = make_float4(0.f, 0.f, 0.f, 0.f), t = f;
    if (active) {
      nn = A.nnb[cur][p];
      if (FRIC) cm_own = A.cmsk[cur][p];
      if (s.onebody) {
        const float4 P = PM[2 * p], V = VM[p], W = OMD[2 * p];
        const float a = P.w;
        const float gt = 6.0f * pi * eta * a;
        const float gr = 8.0f * pi * eta * a * a * a;
        f = make_float4(-gt * V.x, -gt * V.y, -gt * V.z, 0.f);
        t = make_float4(-gr * W.x, -gr * W.y, gr * (-0.5f * rate - W.z), 0.f);
        if (NOISE) {
          float g[6];
          const uint32_t lt = (uint32_t)(__float_as_int(V.w) - t0);
          gauss6_f32(key0, key1, k, lt, lt, g);
          const float ct = c * sqrtf(gt), cr = c * sqrtf(gr);
          f.x += ct * g[0]; f.y += ct * g[1]; f.z += ct * g[2];
          t.x += cr * g[3]; t.y += cr * g[4]; t.z += cr * g[5];
        }
      }
    }
    sF[tid] = f;
    sA[tid] = active ? PM[2 * p].w : 0.0f;
    sT[tid] = t;
    sM[tid] = 0ull;
  }
  // ---- flatten the warp's rows ---------------------------------------------
  int incl = nn;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  const int excl = incl - nn;
  __syncwarp();

  // pair virials C, HL, BL (27 entries): each batch's 32 pairs are summed
  // over the warp as they are formed, and lane l keeps the running warp
  // total of entry l
  float vacc = 0.0f;

  // Pairs within the cutoff are queued per warp in shared memory, touching
  // pairs (queue 1) apart from the others (queue 0), and the pair physics
  // runs on full 32-lane batches of one queue: lanes beyond the cutoff do
  // not idle through it and only touching pairs run the contact branch.
  constexpr int kQ = 64;
  __shared__ int qQ[2][kBlock / 32][kQ];
  __shared__ int qM[2][kBlock / 32][kQ];        // owner lane | slot << 5 | had contact << 12
  // r_x, r_y, r_z, h; the pair kernel forms S = a_p + a_q from the radii, so
  // that four blocks fit the 164 KB shared-memory carve-out (92 KB of L1)
  __shared__ float qG[2][kBlock / 32][4][kQ];
  int qn0 = 0, qn1 = 0;

  // Pair e of queue qi (1: touching pairs): partner's share by vector
  // reductions, owner's share returned in v (force, torque) with its contact
  // bit; returns the owner.  qi is warp-uniform.
  auto physics = [&](int qi, int e, float* v, unsigned long long& mbit, float* FR,
                     float* rro, float* vp) -> int {
    const int q = qQ[qi][warp][e];
    const int meta = qM[qi][warp][e];
    const int o = meta & 31, sl = (meta >> 5) & 127;
    const float rpq[3] = {qG[qi][warp][0][e], qG[qi][warp][1][e], qG[qi][warp][2][e]};
    const float h = qG[qi][warp][3][e];
    const int po = pb + warp * 32 + o;
    const float ap = sA[tid - lane + o];
    const float aq = __ldg(PM + 2 * q).w;
    const float S = ap + aq;
    const float d = S + h;
    const float xi = 2.0f * h / S;
    const float4 WPo = __ldg(OMD + 2 * po), WQ = __ldg(OMD + 2 * q);
    const float4 VPo = __ldg(VM + po), VQ = __ldg(VM + q);
    const int tp = __float_as_int(VPo.w), tq = __float_as_int(VQ.w);
    const bool p_is_i = tp < tq;
    const float sg = p_is_i ? 1.0f : -1.0f;
    const float id = 1.0f / d;
    const float rr[3] = {sg * rpq[0], sg * rpq[1], sg * rpq[2]};
    const float n[3] = {rr[0] * id, rr[1] * id, rr[2] * id};
    const float ai = p_is_i ? ap : aq, aj = p_is_i ? aq : ap;
    const float4 Vi = p_is_i ? VPo : VQ, Vj = p_is_i ? VQ : VPo;
    const float4 Wi4 = p_is_i ? WPo : WQ, Wj4 = p_is_i ? WQ : WPo;
    const float Wi[3] = {Wi4.x, Wi4.y, Wi4.z}, Wj[3] = {Wj4.x, Wj4.y, Wj4.z};
    // relative velocity of the image of j: peculiar difference + rate r_y x
    const float dU[3] = {Vj.x - Vi.x + rate * rr[1], Vj.y - Vi.y, Vj.z - Vi.z};

    PairOut<float> ou;
    // repulsion, Eq. 34 read as the force on j: -(A/kappa) exp(-h/kappa) n on i
    FR[0] = FR[1] = FR[2] = 0.0f;
    if (rep_on) {
      const float kap = 0.01f * S;
      if (h <= rep_hc * S) {
        const float f = repA / kap * __expf(-h / kap);
        FR[0] = -f * n[0]; FR[1] = -f * n[1]; FR[2] = -f * n[2];
      }
    }
    rro[0] = rr[0]; rro[1] = rr[1]; rro[2] = rr[2];
    // queued pairs beyond the lubrication cutoff exist only with repulsion
    if (s.lubrication && (!EXTRA || xi <= xi_max)) {
      const float xi_e = fmaxf(xi, xi_min);
      const float ixi = 1.0f / xi_e;
      const float L = __logf(ixi);
      const Res8<float> R = resistances_f(eta, ai, aj, ixi, L);
      float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (NOISE) {
        const uint32_t li = (uint32_t)((p_is_i ? tp : tq) - t0);
        const uint32_t lj = (uint32_t)((p_is_i ? tq : tp) - t0);
        gauss6_f32(key0, key1, k, li, lj, g);
      }
      lub_brownian<float, NOISE>(R, n, dU, Wi, Wj, g, g + 3, c, tsign, ou);
    } else {
#pragma unroll
      for (int q3 = 0; q3 < 3; ++q3) ou.FL[q3] = ou.FB[q3] = ou.Ti[q3] = ou.Tj[q3] = 0.f;
    }
    float FC[3] = {0.f, 0.f, 0.f}, TCi[3] = {0.f, 0.f, 0.f}, TCj[3] = {0.f, 0.f, 0.f};
    mbit = 0ull;
    if (qi == 1) {
      const float delta = -h;
      float Ft[3] = {0.f, 0.f, 0.f};
      if (FRIC && mu > 0.0f) {
        float xh[3] = {0.f, 0.f, 0.f}, xl[3] = {0.f, 0.f, 0.f};
        const int64_t hi = (int64_t)sl * Np + po;
        if ((meta >> 12) & 1) {
          const float4 r0 = hist[2 * hi], r1 = hist[2 * hi + 1];
          xh[0] = r0.x; xl[0] = r0.y; xh[1] = r0.z; xl[1] = r0.w;
          xh[2] = r1.x; xl[2] = r1.y;
        }
        if (s.advance) {
          const float ww[3] = {ai * Wi[0] + aj * Wj[0], ai * Wi[1] + aj * Wj[1],
                               ai * Wi[2] + aj * Wj[2]};
          float wxn[3];
          cross3(ww, n, wxn);
          const float vt[3] = {dU[0] - wxn[0], dU[1] - wxn[1], dU[2] - wxn[2]};
          history_update_df(xh, xl, n, vt, dtf, kt, mu * kn * delta);
        }
        hist[2 * hi] = make_float4(xh[0], xl[0], xh[1], xl[1]);
        hist[2 * hi + 1] = make_float4(xh[2], xl[2], 0.f, 0.f);
        mbit = 1ull << sl;
        Ft[0] = kt * xh[0]; Ft[1] = kt * xh[1]; Ft[2] = kt * xh[2];
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
      Fi[q3] = FC[q3] + ou.FL[q3] + ou.FB[q3] + FR[q3];
      Ti_[q3] = TCi[q3] + ou.Ti[q3];
      Tj_[q3] = TCj[q3] + ou.Tj[q3];
    }
    const float* To = p_is_i ? Ti_ : Tj_;
    const float* Tq = p_is_i ? Tj_ : Ti_;
    v[0] = sg * Fi[0]; v[1] = sg * Fi[1]; v[2] = sg * Fi[2];
    v[3] = To[0]; v[4] = To[1]; v[5] = To[2];
    red_add_v4(F4 + q, -sg * Fi[0], -sg * Fi[1], -sg * Fi[2], 0.f);
    red_add_v4(T4 + q, Tq[0], Tq[1], Tq[2], 0.f);
    if (SAMPLE) {
#pragma unroll
      for (int be = 0; be < 3; ++be) {
        const float2 rb = dup2(rr[be]);
        const float2 c2 = mul2(make_float2(FC[0], FC[1]), rb);
        const float2 l2 = mul2(make_float2(ou.FL[0], ou.FL[1]), rb);
        const float2 b2 = mul2(make_float2(ou.FB[0], ou.FB[1]), rb);
        vp[be] = c2.x; vp[3 + be] = c2.y; vp[6 + be] = FC[2] * rr[be];
        vp[9 + be] = l2.x; vp[12 + be] = l2.y; vp[15 + be] = ou.FL[2] * rr[be];
        vp[18 + be] = b2.x; vp[21 + be] = b2.y; vp[24 + be] = ou.FB[2] * rr[be];
      }
    }
    return o;
  };

  // One batch: lanes [0, n0) take entries first0.. of queue 0, lanes
  // [n0, n0 + n1) entries first1.. of queue 1 (n0 + n1 <= 32, warp-uniform;
  // a full batch comes from one queue, the last batch of a warp may hold
  // both).  Queue entries are in row order, so the keys own + 32 * queue
  // along a batch are non-decreasing: the owner's shares are summed over
  // each run of equal keys by shuffles, and the run's first lane adds the
  // sums to the owner's shared-memory accumulators -- the queue-0 runs
  // first, then the queue-1 runs, so an owner with a run in each part has
  // one writer at a time.
  auto batch = [&](int n0, int first0, int n1, int first1) {
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    unsigned long long mb = 0ull;
    int own = 64;  // idle lanes: past every key
    float FR[3] = {0.f, 0.f, 0.f}, rro[3] = {0.f, 0.f, 0.f};
    float vp[32];
#pragma unroll
    for (int cc = 0; cc < 32; ++cc) vp[cc] = 0.0f;
    const int qi = lane < n0 ? 0 : 1;
    if (lane < n0 + n1)
      own = physics(qi, qi ? first1 + lane - n0 : first0 + lane, v, mb, FR, rro, vp) +
            32 * qi;
    if (SAMPLE) vacc += warp_reduce_scatter32(vp, lane);
    if (SAMPLE && rep_on) {
      // repulsion virial F^R (x) r summed over the warp into its slots
#pragma unroll
      for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) {
          float x = FR[al] * rro[be];
#pragma unroll
          for (int o2 = 16; o2 > 0; o2 >>= 1) x += __shfl_down_sync(kFull, x, o2);
          if (lane == 0) sW[warp * kPartialLen + kRepOff + 3 * al + be] += x;
        }
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int oo = __shfl_down_sync(kFull, own, off);
      const bool same = lane + off < 32 && oo == own && own < 64;
      if (!__any_sync(kFull, same)) break;  // every run is at most off long
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) {
        const float x = __shfl_down_sync(kFull, v[cc], off);
        if (same) v[cc] += x;
      }
      if (FRIC && n1 > 0) {
        const unsigned long long x = __shfl_down_sync(kFull, mb, off);
        if (same) mb |= x;
      }
    }
    const int prev = __shfl_up_sync(kFull, own, 1);
    const bool head = own < 64 && (lane == 0 || prev != own);
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      if (head && (own >> 5) == part) {
        const int o = own & 31;
        float4* so = &sF[warp * 32 + o];
        float4* st = &sT[warp * 32 + o];
        float4 f = *so, t = *st;
        f.x += v[0]; f.y += v[1]; f.z += v[2];
        t.x += v[3]; t.y += v[4]; t.z += v[5];
        *so = f;
        *st = t;
        if (FRIC && part == 1) sM[warp * 32 + o] |= mb;
      }
      __syncwarp();
    }
  };

  // Work loop of the warp, all decisions warp-uniform: flush a queue that
  // holds a full batch, else scan the next 32 list items into the queues,
  // else drain what is left.  Phase A and the pair physics each have a
  // single call site, so the kernel body stays small in instruction cache.
  // list entry of this lane's item in the next phase-A pass, fetched one
  // pass ahead so that its latency overlaps the current pass and batches
  int o_n = 0, sl_n = 0, q_n = 0;
  auto locate = [&](int b0) {
    const int t = b0 + lane;
    int o = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int v = __shfl_sync(kFull, incl, o + step - 1);
      if (v <= t) o += step;
    }
    o_n = o;
    sl_n = t - __shfl_sync(kFull, excl, o);
    q_n = t < total ? __ldg(nbr + (int64_t)sl_n * Np + pb + warp * 32 + o) : 0;
  };
  if (total > 0) locate(0);
  int base = 0;
  while (true) {
    int n0 = 0, f0 = 0, n1 = 0, f1 = 0;
    if (qn0 >= 32) {
      n0 = 32; f0 = qn0 - 32;
    } else if (qn1 >= 32) {
      n1 = 32; f1 = qn1 - 32;
    } else if (base < total) {
      const int t = base + lane;
      const int o = o_n, sl = sl_n, qe = q_n;
      const unsigned long long ocm = FRIC ? __shfl_sync(kFull, cm_own, o) : 0ull;
      if (base + 32 < total) locate(base + 32);
      bool keep = false, touch = false;
      float wst = 0.0f, dst = 1.0f, rst[3] = {0.f, 0.f, 0.f};
      float gq[4];
      if (t < total) {
        const int po = pb + warp * 32 + o;
        const int q = qe & kNbrIndexMask;
        const float4 P = __ldg(PM + 2 * po), Q = __ldg(PM + 2 * q);
        const float4 Pl = __ldg(PM + 2 * po + 1), Ql = __ldg(PM + 2 * q + 1);
        // the partner's home cell relative to the owner's, from the entry's
        // top bits: code = 3 (dcx + 1) + (dcy + 1) + 9 (dcz + 1) < 27, split
        // by multiply-shift divisions exact on these ranges (code / 9, c9 / 3)
        const int code = (int)((unsigned)qe >> kNbrIndexBits);
        const int dz1 = (code * 57) >> 9, c9 = code - 9 * dz1, dx1 = (c9 * 11) >> 5;
        const int dcx = dx1 - 1, dcy = c9 - 3 * dx1 - 1, dcz = dz1 - 1;
        const float r0 = (Q.x - P.x) + (cwx * (float)dcx + ctilt * (float)dcy);
        const float r1 = (Q.y - P.y) + cwy * (float)dcy;
        const float r2 = (Q.z - P.z) + cwz * (float)dcz;
        const float d2f = r0 * r0 + r1 * r1 + r2 * r2;
        const float rc = EXTRA ? fmaf(shf, fmaxf(P.w, Q.w), (P.w + Q.w) * rcf)
                               : (P.w + Q.w) * rcf;
        // beyond the lubrication cutoff (with a margin for single-precision
        // rounding; the exact test follows): no force, no contact
        if (d2f <= rc * rc * 1.00001f) {
          // separation in double-float from the cell-relative offsets, then
          // d^2 - S^2 with the cancelling squares summed error-free, and the
          // gap h = (d^2 - S^2) / (d + S)
          const float2 shx = sShx[c9];
          const float fy = (float)dcy, fz = (float)dcz;
          float rh[3], rl[3];
          {
            // x and y as packed pairs, z alone
            float2 s1, e1, s2, e2, h2, l2;
            two_sum2(make_float2(Q.x, Q.y), make_float2(-P.x, -P.y), s1, e1);
            two_sum2(s1, make_float2(shx.x, cw1h * fy), s2, e2);
            const float2 dl = sub2(make_float2(Ql.x, Ql.y), make_float2(Pl.x, Pl.y));
            const float2 lo = add2(add2(e1, e2), add2(dl, make_float2(shx.y, cw1l * fy)));
            fast_two_sum2(s2, lo, h2, l2);
            rh[0] = h2.x; rh[1] = h2.y; rl[0] = l2.x; rl[1] = l2.y;
          }
          df_diff_shift(Q.z, Ql.z, P.z, Pl.z, cw2h * fz, cw2l * fz, rh[2], rl[2]);
          float Sh, Sl;
          {
            float s0, e0;
            two_sum(P.w, Q.w, s0, e0);
            fast_two_sum(s0, __fadd_rn(e0, __fadd_rn(Pl.w, Ql.w)), Sh, Sl);
          }
          float pk[3], ek[3];
          {
            const float2 r2 = make_float2(rh[0], rh[1]);
            const float2 p2 = mul2(r2, r2);
            const float2 e2 = fma2(r2, r2, neg2(p2));
            pk[0] = p2.x; pk[1] = p2.y; ek[0] = e2.x; ek[1] = e2.y;
            pk[2] = __fmul_rn(rh[2], rh[2]);
            ek[2] = __fmaf_rn(rh[2], rh[2], -pk[2]);
          }
          const float pS = __fmul_rn(Sh, Sh);
          const float eS = __fmaf_rn(Sh, Sh, -pS);
          float t1, u1, t2, u2, t3, u3;
          two_sum(pk[0], pk[1], t1, u1);
          two_sum(t1, pk[2], t2, u2);
          two_sum(t2, -pS, t3, u3);
          const float small = ((u1 + u2) + u3) + ((ek[0] + ek[1]) + (ek[2] - eS)) +
                              2.0f * ((rh[0] * rl[0] + rh[1] * rl[1]) + (rh[2] * rl[2] - Sh * Sl));
          const float D = __fadd_rn(t3, small);
          const float d = sqrtf(t2);
          const float h = D / (d + Sh);
          if (strc) {
            // shells h <= shell a of the two spheres (Eq. 26)
            wst = (h <= shf * P.w ? 1.0f : 0.0f) + (h <= shf * Q.w ? 1.0f : 0.0f);
            rst[0] = rh[0]; rst[1] = rh[1]; rst[2] = rh[2];
            dst = d;
          }
          if (2.0f * h / Sh <= xi_max || (rep_on && h <= rep_hc * Sh)) {
            keep = true;
            touch = s.contact && h < 0.0f;
            gq[0] = rh[0]; gq[1] = rh[1]; gq[2] = rh[2];
            gq[3] = h;
          }
        }
      }
      if (strc) {
        // structural sums w n n of these 32 items (6 distinct entries)
        const float id2 = wst / (dst * dst);
        const float e6[6] = {rst[0] * rst[0] * id2, rst[0] * rst[1] * id2, rst[0] * rst[2] * id2,
                             rst[1] * rst[1] * id2, rst[1] * rst[2] * id2, rst[2] * rst[2] * id2};
#pragma unroll
        for (int c6 = 0; c6 < 6; ++c6) {
          float x = e6[c6];
#pragma unroll
          for (int o2 = 16; o2 > 0; o2 >>= 1) x += __shfl_down_sync(kFull, x, o2);
          if (lane == 0) sW[warp * kPartialLen + kStrOff + c6] += x;
        }
      }
      const unsigned m0 = __ballot_sync(kFull, keep && !touch);
      const unsigned m1 = __ballot_sync(kFull, touch);
      if (keep) {
        const unsigned below = (1u << lane) - 1u;
        const int qk = touch ? 1 : 0;
        const int e = touch ? qn1 + __popc(m1 & below) : qn0 + __popc(m0 & below);
        qQ[qk][warp][e] = qe & kNbrIndexMask;
        qM[qk][warp][e] = o | (sl << 5) | ((FRIC && ((ocm >> sl) & 1ull)) ? (1 << 12) : 0);
#pragma unroll
        for (int c6 = 0; c6 < 4; ++c6) qG[qk][warp][c6][e] = gq[c6];
      }
      qn0 += __popc(m0);
      qn1 += __popc(m1);
      __syncwarp();
      base += 32;
      continue;
    } else if (qn0 + qn1 > 32) {
      // what is left does not fit one batch: the touching pairs first
      n1 = qn1;
    } else if (qn0 + qn1 > 0) {
      // the warp's last batch: both queues' remainders together
      n0 = qn0; n1 = qn1;
    } else {
      break;
    }
    batch(n0, f0, n1, f1);
    qn0 -= n0;
    qn1 -= n1;
  }
  // the warp's own accumulators are complete once its batches are done
  if (active) {
    const float4 f = sF[tid], t = sT[tid];
    red_add_v4(F4 + p, f.x, f.y, f.z, 0.f);
    red_add_v4(T4 + p, t.x, t.y, t.z, 0.f);
    if (FRIC) A.cmsk[cur][p] = sM[tid];
  }
  if (SAMPLE) {
    // single-precision warp sums into shared memory; the last warp of the
    // block to arrive folds the eight warp sums (in warp order, in double)
    // into the block partial, so no warp waits at a block-wide barrier.
    // Blocks, replicas and time are summed in double by the next pair launch
    // (or the reduction kernels at the end of a call).
    if (lane < kVirLen) sW[warp * kPartialLen + lane] = vacc;
    __syncwarp();
    __threadfence_block();
    int arrived = 0;
    if (lane == 0) arrived = atomicAdd(&sArrive, 1);
    arrived = __shfl_sync(kFull, arrived, 0);
    if (arrived == kBlock / 32 - 1) {
      __threadfence_block();
      // the structural slots hold the 6 distinct entries of the symmetric
      // tensor: entry (a, b) of the 3x3 block is slot kSym[3a + b]
      constexpr int kSym[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
      for (int cc = lane; cc < kPartialLen; cc += 32) {
        const int src = cc < kStrOff ? cc : kStrOff + kSym[cc - kStrOff];
        double sum = 0.0;
        for (int w = 0; w < kBlock / 32; ++w)
          sum += (double)*(volatile float*)&sW[w * kPartialLen + src];
        A.pair_partial_w[((int64_t)s.ppar * gridDim.x + b) * kPartialLen + cc] = sum;
      }
    }
  }
}

template <bool NOISE, bool FRIC, bool EXTRA>
static void launch_pm(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                      cudaStream_t st) {
  if (s.sample)
    k_pair_mixed<NOISE, FRIC, true, EXTRA><<<bm.nblocks, kBlock, 0, st>>>(A, bm, s);
  else
    k_pair_mixed<NOISE, FRIC, false, EXTRA><<<bm.nblocks, kBlock, 0, st>>>(A, bm, s);
}

template <bool EXTRA>
static void launch_pm_extra(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                            cudaStream_t st) {
  const bool noise = s.noise != 0, fric = s.friction != 0;
  if (noise && fric) launch_pm<true, true, EXTRA>(A, bm, s, st);
  else if (noise) launch_pm<true, false, EXTRA>(A, bm, s, st);
  else if (fric) launch_pm<false, true, EXTRA>(A, bm, s, st);
  else launch_pm<false, false, EXTRA>(A, bm, s, st);
}

void launch_pair_mixed(const Arrays& A, const BlockMap& bm, const StepArgs& s, int tpp,
                       cudaStream_t st) {
  (void)tpp;
  if (s.rep_on || s.structural) launch_pm_extra<true>(A, bm, s, st);
  else launch_pm_extra<false>(A, bm, s, st);
}

}  // namespace susp
