// k_det.cu -- the deterministic force sums of the FP64 path (parameter
// deterministic = 1).
//
// The pair kernel writes each listed pair's shares -- the force and torque on
// the row's sphere and the torque on the partner -- to the pair's own slot
// instead of adding them with atomics, and each sphere's one-body terms to
// its own record.  k_det_gather then sums, for every sphere, its one-body
// terms, its own row's slots in slot order and the slots where it is the
// partner in ascending slot order, so the sums, and every result after
// them, are the same from run to run.
//
// "Where it is the partner" is a reverse list built with every neighbour
// rebuild (after the list, before the live copy flips): partner counts, an
// exclusive scan into offsets, a fill, and a sort of each sphere's entries
// by slot index (the fill's order depends on scheduling; the sort removes
// that).  Every rebuild kernel here is gated on the rebuild flag like the
// others.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "susp_internal.h"

namespace susp {

namespace {
constexpr int kPer = 8;                   // elements per thread in the scan
constexpr int kSpan = kBlock * kPer;      // elements per scan block

__device__ __forceinline__ bool due(const Ctl* ctl) {
  return *(volatile const int*)&ctl->need_rebuild != 0;
}

unsigned grid_of(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }
}  // namespace

__global__ void k_rev_zero(Arrays A) {
  if (!due(A.ctl)) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i <= A.N) { A.rev_cnt[i] = 0; A.rev_fill[i] = 0; }
}

// partner counts of the new list
__global__ void k_rev_count(Arrays A) {
  if (!due(A.ctl)) return;
  const int nxt = A.ctl->cur ^ 1;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int nn = A.nnb[nxt][p];
  for (int sl = 0; sl < nn; ++sl) {
    const int q = A.nbr[nxt][(int64_t)sl * A.Npad + p] & kNbrIndexMask;
    atomicAdd(&A.rev_cnt[q], 1);
  }
}

// exclusive scan of rev_cnt[0..N) into rev_off, three passes
__global__ void k_rev_scan_blocks(Arrays A) {
  if (!due(A.ctl)) return;
  __shared__ int wsum[kBlock / 32];
  const int64_t base = (int64_t)blockIdx.x * kSpan + (int64_t)threadIdx.x * kPer;
  int v[kPer];
  int tsum = 0;
#pragma unroll
  for (int e = 0; e < kPer; ++e) {
    v[e] = base + e < A.N ? A.rev_cnt[base + e] : 0;
    tsum += v[e];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kBlock / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kBlock / 32) wsum[lane] = w;
  }
  __syncthreads();
  int run = x - tsum + (warp > 0 ? wsum[warp - 1] : 0);
#pragma unroll
  for (int e = 0; e < kPer; ++e) {
    if (base + e < A.N) A.rev_off[base + e] = run;
    run += v[e];
  }
  if (threadIdx.x == kBlock - 1) A.rev_part[blockIdx.x] = run;
}

// exclusive scan of the block totals (one block, in chunks of its size)
__global__ void k_rev_scan_top(Arrays A, int nparts) {
  if (!due(A.ctl)) return;
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int b0 = 0; b0 < nparts; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    const int v = i < nparts ? A.rev_part[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = lane < nw ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    const int excl = carry + x - v + (warp > 0 ? wsum[warp - 1] : 0);
    if (i < nparts) A.rev_part[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) A.rev_off[A.N] = carry;
}

__global__ void k_rev_scan_add(Arrays A) {
  if (!due(A.ctl)) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < A.N) A.rev_off[i] += A.rev_part[i / kSpan];
}

// the slots in which each sphere is the partner (slot index sl * Npad + p)
__global__ void k_rev_fill(Arrays A) {
  if (!due(A.ctl)) return;
  const int nxt = A.ctl->cur ^ 1;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int nn = A.nnb[nxt][p];
  for (int sl = 0; sl < nn; ++sl) {
    const int64_t e = (int64_t)sl * A.Npad + p;
    const int q = A.nbr[nxt][e] & kNbrIndexMask;
    const int at = A.rev_off[q] + atomicAdd(&A.rev_fill[q], 1);
    A.rev_ent[at] = (int)e;
  }
}

// each sphere's entries in ascending slot index (insertion sort: a sphere is
// the partner in a few slots)
__global__ void k_rev_sort(Arrays A) {
  if (!due(A.ctl)) return;
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= A.N) return;
  const int b0 = A.rev_off[q], b1 = A.rev_off[q + 1];
  for (int i = b0 + 1; i < b1; ++i) {
    const int x = A.rev_ent[i];
    int j = i - 1;
    while (j >= b0 && A.rev_ent[j] > x) {
      A.rev_ent[j + 1] = A.rev_ent[j];
      --j;
    }
    A.rev_ent[j + 1] = x;
  }
}

void launch_rev_build(const Arrays& A, cudaStream_t st) {
  const int nparts = (int)((A.N + kSpan - 1) / kSpan);
  k_rev_zero<<<grid_of(A.N + 1), kBlock, 0, st>>>(A);
  k_rev_count<<<grid_of(A.N), kBlock, 0, st>>>(A);
  k_rev_scan_blocks<<<nparts, kBlock, 0, st>>>(A);
  k_rev_scan_top<<<1, 1024, 0, st>>>(A, nparts);
  k_rev_scan_add<<<grid_of(A.N), kBlock, 0, st>>>(A);
  k_rev_fill<<<grid_of(A.N), kBlock, 0, st>>>(A);
  k_rev_sort<<<grid_of(A.N), kBlock, 0, st>>>(A);
}

// Per sphere, in a fixed order: its one-body terms, its own row's slots, then
// the slots where it is the partner (negated force, the partner's torque).
// det_slot holds per slot e: force on the row's sphere [0..2], torque on it
// [3..5], torque on the partner [6..8], component c at c * kmax * Npad + e.
__global__ void k_det_gather(Arrays A) {
  const int cur = A.ctl->cur;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int64_t Np = A.Npad, KN = (int64_t)A.kmax * Np;
  double F[3], T[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    F[c] = A.det_own[c * Np + p];
    T[c] = A.det_own[(3 + c) * Np + p];
  }
  const int nn = A.nnb[cur][p];
  for (int sl = 0; sl < nn; ++sl) {
    const int64_t e = (int64_t)sl * Np + p;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      F[c] = F[c] + A.det_slot[c * KN + e];
      T[c] = T[c] + A.det_slot[(3 + c) * KN + e];
    }
  }
  const int b0 = A.rev_off[p], b1 = A.rev_off[p + 1];
  for (int i = b0; i < b1; ++i) {
    const int64_t e = A.rev_ent[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      F[c] = F[c] - A.det_slot[c * KN + e];
      T[c] = T[c] + A.det_slot[(6 + c) * KN + e];
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    A.frc[cur][c * Np + p] = F[c];
    A.trq[cur][c * Np + p] = T[c];
  }
}

void launch_det_gather(const Arrays& A, cudaStream_t st) {
  k_det_gather<<<grid_of(A.N), kBlock, 0, st>>>(A);
}

}  // namespace susp
