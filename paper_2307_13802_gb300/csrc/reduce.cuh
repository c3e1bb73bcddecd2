// reduce.cuh -- the deterministic two-level reduction of per-block stress and
// kinetic partial sums into per-replica accumulators.  Both levels sum in a
// fixed order, so the result does not depend on scheduling.  They run either
// as two kernels of their own (k_util.cu) or in the first blocks of the next
// mixed pair launch, one chunk per block, where the last chunk of a replica
// to finish sums the replica (k_pair_mixed.cu); the order of the sums is the
// same either way.
#pragma once
#include <cuda_runtime.h>

#include "susp_internal.h"

namespace susp {

constexpr int kRedLen = kPartialLen + kKinLen;
static_assert(kRedLen <= 64, "one thread per component and row group");

// Level 1, chunk ch (all 256 threads of a block take part): thread (g, c) of
// the 4 x 64 layout sums component c over rows g, g + 4, ... of the chunk
// (coalesced rows of block partials), and the four row sums are added in
// order g = 0..3.  Each thread issues all its loads before the first add
// (rows past the chunk's end read as +0).  pw: the pair partials of the
// mixed path (one of the two buffers).
__device__ __forceinline__ void reduce_chunk(const Arrays& A, int ch, const double* pw,
                                             int sample_pair, int sample_kin,
                                             double (&part)[4][64]) {
  const int g = threadIdx.x >> 6, c = threadIdx.x & 63;
  const int b0 = A.chunk_b[ch], b1 = A.chunk_b[ch + 1];
  constexpr int kRows = kChunk / 4;
  double v[kRows];
  if (c < kPartialLen && sample_pair) {
    if (A.mixed) {
#pragma unroll
      for (int k = 0; k < kRows; ++k) {
        const int b = b0 + g + 4 * k;
        v[k] = b < b1 ? __ldcg(pw + (int64_t)b * kPartialLen + c) : 0.0;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kRows; ++k) {
        const int b = b0 + g + 4 * k;
        v[k] = b < b1 ? __ldcg(A.pair_partial + (int64_t)b * kPartialLen + c) : 0.0;
      }
    }
  } else if (c >= kPartialLen && c < kRedLen && sample_kin) {
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int b = b0 + g + 4 * k;
      v[k] = b < b1 ? __ldcg(A.kin_partial + (int64_t)b * kKinLen + (c - kPartialLen)) : 0.0;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kRows; ++k) v[k] = 0.0;
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kRows; ++k) s += v[k];
  part[g][c] = s;
  __syncthreads();
  if (g == 0 && c < kRedLen)
    A.chunk_partial[(int64_t)ch * kRedLen + c] = ((part[0][c] + part[1][c]) + part[2][c]) + part[3][c];
}

// Level 2, replica r (all 256 threads of a block take part): thread (g, c)
// sums component c over the replica's chunks g, g + 4, ... in order (loads
// issued eight at a time, through L2: in the fused form other blocks of the
// same launch wrote them), the four sums are added in order g = 0..3, and the
// result is added to the running accumulator.  With a series buffer, the
// structural xy component also records this sample's
// Sigma^B_xy = -kT / (shell V) sum w n_x n_y (Eq. 26).
__device__ __forceinline__ void reduce_replica(const Arrays& A, int r, int sample_pair,
                                               int sample_kin, double (&part)[4][64]) {
  const int g = threadIdx.x >> 6, c = threadIdx.x & 63;
  const bool is_pair = c < kPartialLen;
  const bool on = c < kRedLen && ((is_pair && sample_pair) || (!is_pair && sample_kin));
  double s = 0.0;
  if (on) {
    const int c1 = A.rep_cstart[r + 1];
    for (int ch0 = A.rep_cstart[r] + g; ch0 < c1; ch0 += 32) {
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int ch = ch0 + 4 * k;
        v[k] = ch < c1 ? __ldcg(A.chunk_partial + (int64_t)ch * kRedLen + c) : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) s += v[k];
    }
  }
  part[g][c] = s;
  __syncthreads();
  if (g == 0 && on) {
    const double tot = ((part[0][c] + part[1][c]) + part[2][c]) + part[3][c];
    double* acc = A.stress_acc + (int64_t)r * kAccStride;
    acc[c] += tot;
    if (c == 0) acc[kAccNp] += 1.0;
    if (c == kPartialLen) acc[kAccNk] += 1.0;
    if (c == kStrOff + 1 && A.series_cap > 0) {
      const Replica& R = A.repl[r];
      long long* cnt = A.series_n + 2 * (int64_t)r;
      if (cnt[0] < A.series_cap) {
        A.series[(int64_t)r * A.series_cap + cnt[0]] = -R.kT / A.shell * tot / R.V;
        cnt[0] += 1;
      } else {
        cnt[1] += 1;
      }
    }
  }
}

// The fused form, run by block ch of a launch (ch < nchunk; all 256 threads
// take part): level 1 for chunk ch, then an arrival on the chunk's replica
// counter.  The chunk sums are released by the barrier and thread 0's fence
// before the arrival; the last arrival fences, sums the replica and resets
// the counter for the next launch.
__device__ __forceinline__ void reduce_chunk_then_replica(const Arrays& A, int ch,
                                                          const double* pw, int sample_pair,
                                                          int sample_kin) {
  __shared__ double part[4][64];
  __shared__ unsigned int s_last;
  reduce_chunk(A, ch, pw, sample_pair, sample_kin, part);
  __syncthreads();
  const int r = A.chunk_rep[ch];
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int m = (unsigned int)(A.rep_cstart[r + 1] - A.rep_cstart[r]);
    s_last = atomicAdd(A.rep_tk + r, 1u) == m - 1u ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    reduce_replica(A, r, sample_pair, sample_kin, part);
    if (threadIdx.x == 0) A.rep_tk[r] = 0u;
  }
}

}  // namespace susp
