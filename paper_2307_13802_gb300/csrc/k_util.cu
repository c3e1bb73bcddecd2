// k_util.cu -- state upload/download between the caller's tag order and the
// library's sorted order, force clearing, and the deterministic reduction of
// per-block stress and kinetic partial sums into per-replica accumulators.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "reduce.cuh"
#include "susp_internal.h"

namespace susp {

// Writes x, U, W (tag order, [N][3]) into the live copy in tag order with
// radius, mass and moment of inertia; wraps positions into the box as the
// integrator does; clears forces.  Tags become the identity order, so the
// next neighbour build sorts from scratch.
__global__ void k_load_state(Arrays A, const double* __restrict__ x,
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
    while (py >= R.L[1] && guard < 1024) { py = py - R.L[1]; px = px - R.tilt; ux = ux - dUx; ++guard; }
    while (py < 0.0 && guard < 1024) { py = py + R.L[1]; px = px + R.tilt; ux = ux + dUx; ++guard; }
    while (px >= R.L[0] && guard < 1024) { px = px - R.L[0]; ++guard; }
    while (px < 0.0 && guard < 1024) { px = px + R.L[0]; ++guard; }
    while (pz >= R.L[2] && guard < 1024) { pz = pz - R.L[2]; ++guard; }
    while (pz < 0.0 && guard < 1024) { pz = pz + R.L[2]; ++guard; }
    if (guard >= 1024) atomicOr(&A.ctl->err, kErrWrap);
  } else {
    atomicOr(&A.ctl->err, kErrNonFinite);
  }
  A.pos[cur][p] = make_double4_32a(px, py, pz, radius[p]);
  A.vel[cur][p] = make_double4_32a(ux, uy, uz, mass[p]);
  A.omg[cur][p] = make_double4_32a(wx, wy, wz, inertia[p]);
  const int64_t Np = A.Npad;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    A.frc[cur][q * Np + p] = 0.0;
    A.trq[cur][q * Np + p] = 0.0;
  }
  A.tag[cur][p] = (int)p;
  A.rep[cur][p] = r;
  A.slot_of_tag[p] = (int)p;
  A.nnb[cur][p] = 0;
  A.cmsk[cur][p] = 0ull;
}

__global__ void k_zero_forces(Arrays A) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int cur = A.ctl->cur;
  const int64_t Np = A.Npad;
  if (A.mixed) {
    reinterpret_cast<float4*>(A.frc[cur])[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    reinterpret_cast<float4*>(A.trq[cur])[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    A.frc[cur][q * Np + p] = 0.0;
    A.trq[cur][q * Np + p] = 0.0;
  }
}

// out[N][3] in tag order from the live copy: what = 0 x, 1 U, 2 W, 3 F, 4 T
__global__ void k_gather(Arrays A, int what, double* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= A.N) return;
  const int cur = A.ctl->cur;
  const int p = A.slot_of_tag[t];
  const int64_t Np = A.Npad;
  double v[3];
  if (what <= 2) {
    const double4_32a* base = what == 0 ? A.pos[cur] : (what == 1 ? A.vel[cur] : A.omg[cur]);
    const double4_32a r = read_rec_d(base, A.mixed, p);
    v[0] = r.x; v[1] = r.y; v[2] = r.z;
  } else {
    read_vec3_d(what == 3 ? A.frc[cur] : A.trq[cur], A.mixed, Np, p, v);
  }
  out[3 * t] = v[0]; out[3 * t + 1] = v[1]; out[3 * t + 2] = v[2];
}

// Pairs of the live half list as (tag_i, tag_j), tag_i < tag_j, written at
// per-sphere offsets (exclusive scan of the row lengths done on the host).
__global__ void k_list_pairs(Arrays A, const long long* __restrict__ off,
                             int* __restrict__ ij, int with_history,
                             double* __restrict__ xi_t) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int cur = A.ctl->cur;
  const int64_t Np = A.Npad;
  const int64_t hs = (int64_t)A.kmax * Np;
  const int nn = A.nnb[cur][p];
  const int tp = A.tag[cur][p];
  long long o = off[p];
  const unsigned long long cm = with_history ? A.cmsk[cur][p] : 0ull;
  for (int sl = 0; sl < nn; ++sl) {
    if (with_history && !((cm >> sl) & 1ull)) continue;
    const int q = A.nbr[cur][(int64_t)sl * Np + p] & kNbrIndexMask;
    const int tq = A.tag[cur][q];
    ij[2 * o] = tp < tq ? tp : tq;
    ij[2 * o + 1] = tp < tq ? tq : tp;
    if (with_history) {
      const int64_t h = (int64_t)sl * Np + p;
      for (int c = 0; c < 3; ++c) {
        if (A.mixed) {
          const float2 f = reinterpret_cast<const float2*>(A.hist[cur])[4 * h + c];
          xi_t[3 * o + c] = (double)f.x + (double)f.y;
        } else {
          xi_t[3 * o + c] = A.hist[cur][h + c * hs];
        }
      }
    }
    ++o;
  }
}

__global__ void k_row_counts(Arrays A, int with_history, long long* __restrict__ cnt) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int cur = A.ctl->cur;
  if (with_history) cnt[p] = __popcll(A.cmsk[cur][p]);
  else cnt[p] = A.nnb[cur][p];
}

// The two levels of the stress reduction as kernels of their own: one block
// per chunk, then one block per replica (reduce.cuh gives the order).
__global__ void __launch_bounds__(256) k_reduce_chunks(Arrays A, const double* pw,
                                                       int sample_pair, int sample_kin) {
  __shared__ double part[4][64];
  reduce_chunk(A, blockIdx.x, pw, sample_pair, sample_kin, part);
}

__global__ void __launch_bounds__(256) k_reduce_replicas(Arrays A, int sample_pair,
                                                         int sample_kin) {
  __shared__ double part[4][64];
  reduce_replica(A, blockIdx.x, sample_pair, sample_kin, part);
}

void launch_reduce_stress(const Arrays& A, const BlockMap& bm, int sample_pair,
                          int sample_kin, int ppar, cudaStream_t st) {
  if (!sample_pair && !sample_kin) return;
  const double* pw = A.pair_partial_w + (int64_t)ppar * bm.nblocks * kPartialLen;
  k_reduce_chunks<<<A.nchunk, 256, 0, st>>>(A, pw, sample_pair, sample_kin);
  k_reduce_replicas<<<A.R, 256, 0, st>>>(A, sample_pair, sample_kin);
}

// Green-Kubo autocorrelation (Eq. 33): C[m] = sum_{t < n-m} x[t+m] x[t] / (n-m),
// one block per lag, each summed in a fixed order.
__global__ void k_autocorr(const double* __restrict__ x, int64_t n, int64_t max_lag,
                           double* __restrict__ C) {
  __shared__ double smem[kBlock / 32];
  for (int64_t m = blockIdx.x; m < max_lag; m += gridDim.x) {
    const int64_t cnt = n - m;
    double acc = 0.0;
    for (int64_t t = threadIdx.x; t < cnt; t += blockDim.x) acc += x[t + m] * x[t];
    double v[1] = {acc};
    double out[1];
    block_sum_write<1>(v, smem, out);
    if (threadIdx.x == 0) C[m] = out[0] / (double)cnt;
  }
}

// Peak multiply-add rate of the arithmetic type T: every thread runs eight
// independent chains a = a * b + c (explicit fused multiply-adds), so the
// pipe stays busy; the sums go to `sink` only if they equal a value they
// cannot take, which keeps the work from being optimised away.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* sink, int iters, T b, T c) {
  T a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == (T)-12345.0) sink[threadIdx.x] = s;
}

// multiply-adds issued: blocks * 256 threads * iters * 8 chains
void launch_fma_peak(int fp64, void* sink, int blocks, int iters, cudaStream_t st) {
  if (fp64)
    k_fma_peak<double><<<blocks, 256, 0, st>>>((double*)sink, iters, 0.9999999, 1e-9);
  else
    k_fma_peak<float><<<blocks, 256, 0, st>>>((float*)sink, iters, 0.9999999f, 1e-9f);
}

void launch_autocorr(const double* x, int64_t n, int64_t max_lag, double* C, cudaStream_t st) {
  const int64_t grid = std::min<int64_t>(max_lag, 152 * 8);
  k_autocorr<<<(unsigned)grid, kBlock, 0, st>>>(x, n, max_lag, C);
}

void launch_load_state(const Arrays& A, const double* x, const double* U,
                       const double* W, const double* radius,
                       const double* mass, const double* inertia,
                       const int* rep_of, cudaStream_t st) {
  k_load_state<<<(unsigned)((A.N + kBlock - 1) / kBlock), kBlock, 0, st>>>(
      A, x, U, W, radius, mass, inertia, rep_of);
}

void launch_zero_forces(const Arrays& A, cudaStream_t st) {
  k_zero_forces<<<(unsigned)((A.N + kBlock - 1) / kBlock), kBlock, 0, st>>>(A);
}

void launch_gather(const Arrays& A, int what, double* out, cudaStream_t st) {
  k_gather<<<(unsigned)((A.N + kBlock - 1) / kBlock), kBlock, 0, st>>>(A, what, out);
}

void launch_row_counts(const Arrays& A, int with_history, long long* cnt,
                       cudaStream_t st) {
  k_row_counts<<<(unsigned)((A.N + kBlock - 1) / kBlock), kBlock, 0, st>>>(
      A, with_history, cnt);
}

void launch_list_pairs(const Arrays& A, const long long* off, int* ij,
                       int with_history, double* xi_t, cudaStream_t st) {
  k_list_pairs<<<(unsigned)((A.N + kBlock - 1) / kBlock), kBlock, 0, st>>>(
      A, off, ij, with_history, xi_t);
}

}  // namespace susp
