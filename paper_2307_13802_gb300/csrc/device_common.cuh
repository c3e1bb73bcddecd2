// device_common.cuh -- small device helpers shared by the library kernels:
// block reductions, the pair physics of Sec. II (templated on the arithmetic
// type) and the minimum-image convention of the tilted box.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "susp_internal.h"

namespace susp {

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
// Sums `n` per-thread values over the block (fixed order: shuffle tree inside
// each warp, then warps in index order) and writes them to out[0..n) from
// thread 0.  smem must hold (blockDim/32) * n doubles.
template <int n>
__device__ __forceinline__ void block_sum_write(double (&v)[n], double* smem,
                                                double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < n; ++c) {
    double x = v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) smem[warp * n + c] = x;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += smem[w * n + c];
    out[c] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ double block_max(double v, double* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  double m = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < nw; ++w) m = fmax(m, smem[w]);
  }
  __syncthreads();
  return m;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// pair physics (Sec. II.A-II.C), arithmetic type Rl
// ---------------------------------------------------------------------------
template <typename Rl>
struct Res8 {
  Rl XA11, YA11, YB11, YB21, YC11, YC12, YC21, YC22;
};

// Scalar resistances of Eqs. 9-12 and 15-18 for the regularised gap xi_e
// (beta = a_j / a_i).
template <typename Rl>
__device__ __forceinline__ Res8<Rl> resistances(Rl eta, Rl ai, Rl aj, Rl xi_e,
                                                Rl lg) {
  const Rl pi = Rl(3.14159265358979323846);
  const Rl beta = aj / ai;
  const Rl ibeta = Rl(1) / beta;
  const Rl opb = Rl(1) + beta;
  const Rl opib = Rl(1) + ibeta;
  const Rl opb3 = opb * opb * opb;
  Res8<Rl> R;
  R.XA11 = Rl(6) * pi * eta * ai *
           (Rl(2) * beta * beta / opb3 * (Rl(1) / xi_e) +
            beta * (Rl(1) + Rl(7) * beta + beta * beta) / (Rl(5) * opb3) * lg);
  R.YA11 = Rl(6) * pi * eta * ai *
           (Rl(4) * beta * (Rl(2) + beta + Rl(2) * beta * beta) /
            (Rl(15) * opb3) * lg);
  R.YB11 = -Rl(4) * pi * eta * ai * ai *
           (beta * (Rl(4) + beta) / (Rl(5) * (opb * opb)) * lg);
  R.YB21 = -Rl(4) * pi * eta * aj * aj *
           (ibeta * (Rl(4) + ibeta) / (Rl(5) * (opib * opib)) * lg);
  R.YC11 = Rl(8) * pi * eta * ai * ai * ai * (Rl(2) * beta / (Rl(5) * opb) * lg);
  R.YC12 = Rl(8) * pi * eta * ai * ai * ai * (beta * beta / (Rl(10) * opb) * lg);
  R.YC22 = Rl(8) * pi * eta * aj * aj * aj * (Rl(2) * ibeta / (Rl(5) * opib) * lg);
  R.YC21 = Rl(8) * pi * eta * aj * aj * aj * (ibeta * ibeta / (Rl(10) * opib) * lg);
  return R;
}

// Scalar resistances of Eqs. 9-12 and 15-18 with the quotients of the
// printed forms taken as products with four reciprocals (beta = a_j/a_i,
// r = 1/(1 + beta), 1/beta, ixi = 1/xi_e); algebraically the same, and
// within a few ulps of the printed forms (1/(1 + 1/beta) = beta r):
//   XA11 = 6 pi eta a_i r^3 (2 beta^2 ixi + beta (1 + 7 beta + beta^2)/5 L)
//   YA11 = 6 pi eta a_i r^3 (4 beta (2 + beta + 2 beta^2)/15) L
//   YB11 = -4 pi eta a_i^2 r^2 (beta (4 + beta)/5) L
//   YB21 = -4 pi eta a_j^2 r^2 ((4 beta + 1)/5) L
//   YC11 = 8 pi eta a_i^3 r (2 beta/5) L,   YC12 = 8 pi eta a_i^3 r (beta^2/10) L
//   YC22 = 8 pi eta a_j^3 r (2/5) L,        YC21 = 8 pi eta a_j^3 r (1/(10 beta)) L
// with L = ln(1/xi_e).
__device__ __forceinline__ Res8<double> resistances_rcp(double eta, double ai, double aj,
                                                        double ixi, double L) {
  const double pi = 3.14159265358979323846;
  const double beta = aj / ai;
  const double ibeta = ai / aj;
  const double r = 1.0 / (1.0 + beta);
  const double r2 = r * r, r3 = r2 * r;
  const double b2 = beta * beta;
  const double ta = 6.0 * pi * eta * ai * r3;
  Res8<double> R;
  R.XA11 = ta * (2.0 * b2 * ixi + 0.2 * beta * (1.0 + 7.0 * beta + b2) * L);
  R.YA11 = ta * ((4.0 / 15.0) * beta * (2.0 + beta + 2.0 * b2) * L);
  const double tb = -4.0 * pi * eta * r2 * 0.2 * L;
  R.YB11 = tb * ai * ai * (beta * (4.0 + beta));
  R.YB21 = tb * aj * aj * (4.0 * beta + 1.0);
  const double tc = 8.0 * pi * eta * r * L;
  const double ai3 = ai * ai * ai, aj3 = aj * aj * aj;
  R.YC11 = tc * ai3 * (0.4 * beta);
  R.YC12 = tc * ai3 * (0.1 * b2);
  R.YC22 = tc * aj3 * 0.4;
  R.YC21 = tc * aj3 * (0.1 * ibeta);
  return R;
}

template <typename Rl>
__device__ __forceinline__ Rl dot3(const Rl* a, const Rl* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
template <typename Rl>
__device__ __forceinline__ void cross3(const Rl* a, const Rl* b, Rl* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename Rl>
struct PairOut {
  Rl FL[3], FB[3];        // lubrication and Brownian force on i
  Rl Ti[3], Tj[3];        // lubrication + Brownian torques on i and j
};

// Lubrication (Eqs. 8, 13, 14) and pair Brownian (Eqs. 22-24) terms of one
// pair.  n: unit vector i -> j; dU = U_j - U_i including the image velocity;
// th, chi: standard normal vectors; c = sqrt(2 kT / dt).
template <typename Rl, bool NOISE>
__device__ __forceinline__ void lub_brownian(const Res8<Rl>& R, const Rl* n,
                                             const Rl* dU, const Rl* Wi,
                                             const Rl* Wj, const Rl* th,
                                             const Rl* chi, Rl c, Rl tsign,
                                             PairOut<Rl>& o) {
  // lubrication
  const Rl nd = dot3(n, dU);
  Rl Nd[3], Td[3], win[3], wjn[3], dUn[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    Nd[q] = n[q] * nd;
    Td[q] = dU[q] - n[q] * nd;
  }
  cross3(Wi, n, win);
  cross3(Wj, n, wjn);
  cross3(dU, n, dUn);
  Rl ci[3], cj[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    ci[q] = R.YC11 * Wi[q] + R.YC12 * Wj[q];
    cj[q] = R.YC21 * Wi[q] + R.YC22 * Wj[q];
  }
  const Rl nci = dot3(n, ci), ncj = dot3(n, cj);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    o.FL[q] = R.XA11 * Nd[q] + R.YA11 * Td[q] + R.YB11 * win[q] + R.YB21 * wjn[q];
    o.Ti[q] = R.YB11 * dUn[q] - (ci[q] - n[q] * nci);
    o.Tj[q] = R.YB21 * dUn[q] - (cj[q] - n[q] * ncj);
  }
  if (NOISE) {
    const Rl sXA = sqrt(R.XA11), sYA = sqrt(R.YA11);
    const Rl nth = dot3(n, th), nchi = dot3(n, chi);
    Rl thn[3];
    cross3(th, n, thn);
    const Rl bi = R.YB11 / sYA, bj = R.YB21 / sYA;
    const Rl si = sqrt(R.YC11 - R.YB11 * R.YB11 / R.YA11);
    const Rl sj = sqrt(R.YC22 - R.YB21 * R.YB21 / R.YA11);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const Rl Nth = n[q] * nth;
      const Rl Tth = th[q] - n[q] * nth;
      const Rl Tchi = chi[q] - n[q] * nchi;
      o.FB[q] = c * (sXA * Nth + sYA * Tth);
      o.Ti[q] += c * (bi * thn[q] + si * Tchi);
      o.Tj[q] += c * (bj * thn[q] + tsign * sj * Tchi);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 3; ++q) o.FB[q] = Rl(0);
  }
}

// Tangential history update of a touching pair (Sec. II.A, with the reading
// of the update rule stated in the design notes): rotate the stored
// displacement into the current tangent plane keeping its length, add the
// tangential relative velocity of the contact points times dt, cap at
// mu kn delta / kt.  Always double precision.
__device__ __forceinline__ void history_update(double* xt, const double* n,
                                               const double* v, double dt,
                                               double kt, double fmax) {
  const double nv = n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
  double vt[3] = {v[0] - n[0] * nv, v[1] - n[1] * nv, v[2] - n[2] * nv};
  const double len0 = sqrt(xt[0] * xt[0] + xt[1] * xt[1] + xt[2] * xt[2]);
  const double nx = n[0] * xt[0] + n[1] * xt[1] + n[2] * xt[2];
  double pr[3] = {xt[0] - n[0] * nx, xt[1] - n[1] * nx, xt[2] - n[2] * nx};
  const double len1 = sqrt(pr[0] * pr[0] + pr[1] * pr[1] + pr[2] * pr[2]);
  if (len1 > 0.0) {
    const double sc = len0 / len1;
    xt[0] = pr[0] * sc; xt[1] = pr[1] * sc; xt[2] = pr[2] * sc;
  } else {
    xt[0] = xt[1] = xt[2] = 0.0;
  }
  xt[0] = xt[0] + vt[0] * dt;
  xt[1] = xt[1] + vt[1] * dt;
  xt[2] = xt[2] + vt[2] * dt;
  const double ft = kt * sqrt(xt[0] * xt[0] + xt[1] * xt[1] + xt[2] * xt[2]);
  if (ft > fmax) {
    const double sc = fmax / ft;
    xt[0] = xt[0] * sc; xt[1] = xt[1] * sc; xt[2] = xt[2] * sc;
  }
}

// Minimum image of x_q - x_p in the sliding-brick form of the tilted box:
// the y image count sy first (shifting x by sy * tilt), then x and z.  The
// image counts are rounded from products with the reciprocal edges iL
// rather than quotients: the two differ only where a coordinate difference
// is within an ulp of half an edge (plus whole edges), and a pair closer
// than a third of every edge -- every pair any kernel uses, since boxes hold
// at least three list cutoffs -- has differences at least a sixth of an edge
// away from those points, so its counts, and r, are the same either way.
__device__ __forceinline__ void min_image_f64(double dx, double dy, double dz,
                                              const double* L, const double* iL,
                                              double tilt, double* r, double* sy_out) {
  const double sy = rint(dy * iL[1]);
  dy = dy - sy * L[1];
  dx = dx - sy * tilt;
  const double sx = rint(dx * iL[0]);
  dx = dx - sx * L[0];
  const double sz = rint(dz * iL[2]);
  dz = dz - sz * L[2];
  r[0] = dx; r[1] = dy; r[2] = dz;
  *sy_out = sy;
}

__device__ __forceinline__ double atomic_add_f64(double* a, double v) {
  return atomicAdd(a, v);
}

// Layout-independent reads of the live state as doubles (x, y, z, a),
// (U, m or 1/I) and (W, I): the FP64 layout is read directly, the
// double-float halves of the mixed layout are summed.
__device__ __forceinline__ double4_32a read_rec_d(const double4_32a* base, int mixed,
                                                  int64_t p) {
  if (!mixed) return base[p];
  const float4* r = reinterpret_cast<const float4*>(base + p);
  const float4 h = r[0], l = r[1];
  return make_double4_32a((double)h.x + (double)l.x, (double)h.y + (double)l.y,
                          (double)h.z + (double)l.z, (double)h.w);
}

// Force / torque of sphere p as doubles in either layout.
__device__ __forceinline__ void read_vec3_d(const double* base, int mixed,
                                            int64_t Np, int64_t p, double* v) {
  if (!mixed) {
    v[0] = base[p]; v[1] = base[Np + p]; v[2] = base[2 * Np + p];
  } else {
    const float4 f = reinterpret_cast<const float4*>(base)[p];
    v[0] = f.x; v[1] = f.y; v[2] = f.z;
  }
}

// Vector reduction of a float4 into global memory (16-byte aligned).
__device__ __forceinline__ void red_add_v4(float4* addr, float a, float b, float c,
                                           float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a),
               "f"(b), "f"(c), "f"(d)
               : "memory");
}

}  // namespace susp
