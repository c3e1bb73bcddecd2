// k_neighbors.cu -- cell binning, counting sort and the skin-padded half
// neighbour list (Sec. II: pairwise forces are summed over the neighbours of
// each sphere, found within the widest interaction range in use -- the
// lubrication cutoff xi <= xi_max of Sec. II.B, the repulsion range of
// Eq. 34, the structural shell of Eq. 26 -- plus a skin), with the
// tangential contact history (Sec. II.A) carried from the old list to the
// new one.
//
// Cells are laid on the tilted lattice in fractional coordinates
// s = H^-1 x (H the box matrix with the current tilt), nc cells per axis
// chosen at creation so that each cell is at least one list cutoff thick for
// any tilt |tilt| <= Lx/2; two spheres closer than the cutoff are then in the
// same or adjacent cells of the periodic 3x3x3 stencil.  Keys are
// replica base + cell index, so one sort groups replicas, then cells; ties
// inside a cell are ordered by tag, which makes the order deterministic.
//
// Every kernel here is gated on Ctl::need_rebuild, so the whole sequence can
// sit in every step of a captured graph (or under a conditional node) and
// costs one flag read when no rebuild is due.  The rebuild permutes all
// particle arrays into the spare copy and flips Ctl::cur at the end.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "susp_internal.h"

namespace susp {

constexpr int kScanPer = 8;                      // elements per thread
constexpr int kScanBlock = kBlock * kScanPer;    // elements per scan block

__device__ __forceinline__ bool gate(const Ctl* ctl) {
  return *(volatile const int*)&ctl->need_rebuild != 0;
}

__global__ void k_request(Ctl* ctl) { ctl->need_rebuild = 1; }

__global__ void k_zero_counts(Arrays A) {
  if (!gate(A.ctl)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= A.ncell;
       i += (int64_t)gridDim.x * blockDim.x)
    A.cell_count[i] = 0;
}

// Fractional coordinates by the reciprocal edges (an ulp from the quotients;
// the cells are sized with a relative guard of 1e-9 above the list cutoff,
// so the stencil still covers every pair), which keeps FP64 divisions off
// the rebuild.
__device__ __forceinline__ int cell_index(const Replica& R, double x, double y,
                                          double z, int* c3) {
  const double sy = y * R.iL[1];
  double sx = (x - R.tilt * sy) * R.iL[0];
  sx = sx - floor(sx);
  const double sz = z * R.iL[2];
  int cx = (int)(sx * R.nc[0]);
  int cy = (int)(sy * R.nc[1]);
  int cz = (int)(sz * R.nc[2]);
  cx = min(max(cx, 0), R.nc[0] - 1);
  cy = min(max(cy, 0), R.nc[1] - 1);
  cz = min(max(cz, 0), R.nc[2] - 1);
  if (c3) { c3[0] = cx; c3[1] = cy; c3[2] = cz; }
  return (cz * R.nc[1] + cy) * R.nc[0] + cx;
}

__global__ void k_cellkey(Arrays A) {
  if (!gate(A.ctl)) return;
  const int cur = A.ctl->cur;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int r = A.rep[cur][p];
  const Replica& R = A.repl[r];
  const double4_32a P = read_rec_d(A.pos[cur], A.mixed, p);
  const int key = (int)(R.cell_base + cell_index(R, P.x, P.y, P.z, nullptr));
  A.key[p] = key;
  atomicAdd(&A.cell_count[key], 1);
}

// exclusive scan of cell_count[0..ncell) -> cell_start, in three passes
__global__ void k_scan_blocks(Arrays A) {
  if (!gate(A.ctl)) return;
  __shared__ int wsum[kBlock / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanPer;
  int v[kScanPer];
  int tsum = 0;
#pragma unroll
  for (int e = 0; e < kScanPer; ++e) {
    const int64_t i = base + e;
    v[e] = i < A.ncell ? A.cell_count[i] : 0;
    tsum += v[e];
  }
  // inclusive scan of thread sums in the block
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
  const int excl = x - tsum + (warp > 0 ? wsum[warp - 1] : 0);
  int run = excl;
#pragma unroll
  for (int e = 0; e < kScanPer; ++e) {
    const int64_t i = base + e;
    if (i < A.ncell) A.cell_start[i] = run;
    run += v[e];
  }
  if (threadIdx.x == kBlock - 1) A.scan_part[blockIdx.x] = run;
}

__global__ void k_scan_top(Arrays A, int nparts) {
  if (!gate(A.ctl)) return;
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int base = 0; base < nparts; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < nparts ? A.scan_part[i] : 0;
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
    const int incl = x + (warp > 0 ? wsum[warp - 1] : 0);
    if (i < nparts) A.scan_part[i] = carry + incl - v;  // exclusive
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += incl;
    __syncthreads();
  }
}

__global__ void k_scan_add(Arrays A) {
  if (!gate(A.ctl)) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < A.ncell) {
    const int v = A.cell_start[i] + A.scan_part[i / kScanBlock];
    A.cell_start[i] = v;
    A.cell_fill[i] = v;
  }
  if (i == 0) A.cell_start[A.ncell] = (int)A.N;
}

__global__ void k_scatter(Arrays A) {
  if (!gate(A.ctl)) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int slot = atomicAdd(&A.cell_fill[A.key[p]], 1);
  A.perm[slot] = (int)p;
}

// order the few spheres of each cell by tag (insertion sort)
__global__ void k_cellsort(Arrays A) {
  if (!gate(A.ctl)) return;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= A.ncell) return;
  const int cur = A.ctl->cur;
  const int s0 = A.cell_start[c], s1 = A.cell_start[c + 1];
  const int* tag = A.tag[cur];
  for (int i = s0 + 1; i < s1; ++i) {
    const int v = A.perm[i];
    const int tv = tag[v];
    int j = i - 1;
    while (j >= s0 && tag[A.perm[j]] > tv) {
      A.perm[j + 1] = A.perm[j];
      --j;
    }
    A.perm[j + 1] = v;
  }
}

__global__ void k_permute(Arrays A) {
  if (!gate(A.ctl)) return;
  const int cur = A.ctl->cur, nxt = cur ^ 1;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int o = A.perm[p];
  const int64_t Np = A.Npad;
  A.pos[nxt][p] = A.pos[cur][o];
  A.vel[nxt][p] = A.vel[cur][o];
  A.omg[nxt][p] = A.omg[cur][o];
  if (A.mixed) {
    reinterpret_cast<float4*>(A.frc[nxt])[p] = reinterpret_cast<const float4*>(A.frc[cur])[o];
    reinterpret_cast<float4*>(A.trq[nxt])[p] = reinterpret_cast<const float4*>(A.trq[cur])[o];
  } else {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      A.frc[nxt][q * Np + p] = A.frc[cur][q * Np + o];
      A.trq[nxt][q * Np + p] = A.trq[cur][q * Np + o];
    }
  }
  const int t = A.tag[cur][o];
  A.tag[nxt][p] = t;
  const int r = A.rep[cur][o];
  A.rep[nxt][p] = r;
  // home cell coordinates packed 10 bits per axis (at most 1023 cells per
  // edge), decoded once here instead of at every step
  const Replica& R = A.repl[r];
  const int local = (int)(A.key[o] - R.cell_base);
  const int cx = local % R.nc[0], cy = (local / R.nc[0]) % R.nc[1],
            cz = local / (R.nc[0] * R.nc[1]);
  A.cell[p] = cx | (cy << 10) | (cz << 20);
  A.slot_of_tag[t] = (int)p;
}

// neighbour cell index along one axis, periodic (|d| <= 1, n >= 3)
__device__ __forceinline__ int wrap_cell(int i, int n) {
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

__global__ void __launch_bounds__(kBlock, 3) k_build_list(Arrays A, StepArgs s, double rc_fac) {
  if (!gate(A.ctl)) return;
  const int nxt = A.ctl->cur ^ 1;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int r = A.rep[nxt][p];
  const Replica& R = A.repl[r];
  const int ncx = R.nc[0], ncy = R.nc[1], ncz = R.nc[2];
  const int pk = A.cell[p];
  const int cx = pk & 1023, cy = (pk >> 10) & 1023, cz = pk >> 20;
  const int64_t Np = A.Npad;
  int* row = A.nbr[nxt] + p;
  int cnt = 0;
  const int kmax = A.kmax;
  if (A.mixed) {
    // Mixed layout: the candidates are tested in single precision on the
    // high words of the positions, against the cutoff widened by a margin
    // above the single-precision error of the test (a few ulps of the box
    // edge), so the list holds every pair the exact test would list and a
    // thin shell more; the pair kernel decides the interaction ranges
    // exactly.  This keeps the list build off the FP64 pipe.
    const float4 P = reinterpret_cast<const float4*>(A.pos[nxt])[2 * p];
    const float Lf[3] = {(float)R.L[0], (float)R.L[1], (float)R.L[2]};
    const float iLf[3] = {(float)R.iL[0], (float)R.iL[1], (float)R.iL[2]};
    const float tiltf = (float)R.tilt;
    const float margin = 1e-6f * fmaxf(Lf[0], fmaxf(Lf[1], Lf[2]));
    const float fac = (float)rc_fac, rfac = s.rep_on ? (float)s.rep_fac : 0.0f;
    const float shell = s.structural ? (float)s.shell : 0.0f, skin = (float)s.skin;
    const float4* __restrict__ PQ = reinterpret_cast<const float4*>(A.pos[nxt]);
    const int* __restrict__ cs = A.cell_start;
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = wrap_cell(cz + dz, ncz);
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = wrap_cell(cy + dy, ncy);
        const int64_t rowkey = R.cell_base + ((int64_t)zz * ncy + yy) * ncx;
        // The three cells of the stencil row are one range of the sorted
        // order unless the row wraps in x; dx of a partner is then
        // -1 + (q >= b1) + (q >= b2).  Candidates are tested four at a time,
        // their records loaded together so that the loads overlap.
        const bool merged = cx >= 1 && cx + 1 < ncx;
        for (int part = 0; part < (merged ? 1 : 3); ++part) {
          int lo, hi, dx0, b1, b2;
          if (merged) {
            const int64_t k0 = rowkey + cx - 1;
            lo = cs[k0];
            b1 = cs[k0 + 1];
            b2 = cs[k0 + 2];
            hi = cs[k0 + 3];
            dx0 = -1;
          } else {
            dx0 = part - 1;
            const int64_t k = rowkey + wrap_cell(cx + dx0, ncx);
            lo = cs[k];
            hi = cs[k + 1];
            b1 = b2 = 0x7fffffff;
          }
          // the half list: partners after p in the sorted order
          for (int q = max(lo, (int)p + 1); q < hi; q += 4) {
            float4 Qv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              Qv[u] = q + u < hi ? PQ[2 * (q + u)] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int qq = q + u;
              if (qq >= hi) break;
              const float4 Q = Qv[u];
              float ry = Q.y - P.y, rx = Q.x - P.x, rz = Q.z - P.z;
              const float sy = rintf(ry * iLf[1]);
              ry -= sy * Lf[1];
              rx -= sy * tiltf;
              rx -= rintf(rx * iLf[0]) * Lf[0];
              rz -= rintf(rz * iLf[2]) * Lf[2];
              const float S = P.w + Q.w;
              const float rc = fmaxf(fmaxf(S * fac, S * rfac), S + shell * fmaxf(P.w, Q.w)) +
                               skin + margin + 1e-5f * S;
              if (!(rx * rx + ry * ry + rz * rz < rc * rc)) continue;
              const int dx = dx0 + (qq >= b1 ? 1 : 0) + (qq >= b2 ? 1 : 0);
              const int code = (dx + 1) * 3 + (dy + 1) + 9 * (dz + 1);
              if (cnt < kmax) row[(int64_t)cnt * Np] = qq | (code << kNbrIndexBits);
              ++cnt;
            }
          }
        }
      }
    }
  } else {
    const double L[3] = {R.L[0], R.L[1], R.L[2]};
    const double iL[3] = {R.iL[0], R.iL[1], R.iL[2]};
    const double tilt = R.tilt;
    const double4_32a P = A.pos[nxt][p];
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = wrap_cell(cz + dz, ncz);
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = wrap_cell(cy + dy, ncy);
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = wrap_cell(cx + dx, ncx);
          const int64_t key = R.cell_base + ((int64_t)zz * ncy + yy) * ncx + xx;
          // the half list: partners after p in the sorted order
          const int q0 = max(A.cell_start[key], (int)p + 1), q1 = A.cell_start[key + 1];
          for (int q = q0; q < q1; ++q) {
            const double4_32a Q = A.pos[nxt][q];
            double rr[3], sy;
            min_image_f64(Q.x - P.x, Q.y - P.y, Q.z - P.z, L, iL, tilt, rr, &sy);
            const double d2 = rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2];
            // widest interaction range of the pair (lubrication cutoff,
            // repulsion range, structural shell), then the skin
            double rc = (P.w + Q.w) * rc_fac;
            if (s.rep_on) {
              const double rq = (P.w + Q.w) * s.rep_fac;
              if (rq > rc) rc = rq;
            }
            if (s.structural) {
              const double rs = (P.w + Q.w) + s.shell * (P.w > Q.w ? P.w : Q.w);
              if (rs > rc) rc = rs;
            }
            rc = rc + s.skin;
            if (!(d2 < rc * rc)) continue;
            if (cnt < kmax) row[(int64_t)cnt * Np] = q;
            ++cnt;
          }
        }
      }
    }
  }
  // the longest row and the number of pairs, summed over the warp first:
  // one atomic per warp on each counter (one per sphere serialises a
  // million updates of the same word)
  const int full = cnt;
  if (cnt > kmax) {
    atomicOr(&A.ctl->err, kErrOverflow);
    cnt = kmax;
  }
  A.nnb[nxt][p] = cnt;
  const unsigned am = __activemask();
  const int wmax = __reduce_max_sync(am, full);
  const unsigned wsum = __reduce_add_sync(am, (unsigned)cnt);
  if ((threadIdx.x & 31) == __ffs(am) - 1) {
    atomicMax(&A.ctl->max_row, wmax);
    atomicAdd((unsigned long long*)&A.ctl->npairs, (unsigned long long)wsum);
  }
}

// carry tangential history of touching pairs into the new list
__global__ void __launch_bounds__(kBlock) k_remap_history(Arrays A) {
  if (!gate(A.ctl)) return;
  const int cur = A.ctl->cur, nxt = cur ^ 1;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.N) return;
  const int64_t Np = A.Npad;
  const int64_t hs = (int64_t)A.kmax * Np;
  const int r = A.rep[nxt][p];
  const Replica& R = A.repl[r];
  const double L[3] = {R.L[0], R.L[1], R.L[2]};
  const int nn = A.nnb[nxt][p];
  const int op = A.perm[p];
  unsigned long long cm = 0ull;
  // Only touching pairs keep a history (the next evaluation erases it for
  // the others), so pairs apart are skipped before the old rows are
  // searched.  The mixed layout tests in single precision with a margin
  // above its rounding error: a pair within the margin keeps its history
  // and the evaluation, which decides contact exactly, erases it if apart.
  const float4 Pf = reinterpret_cast<const float4*>(A.pos[nxt])[2 * p];
  const float Lf[3] = {(float)L[0], (float)L[1], (float)L[2]};
  const float iLf[3] = {(float)R.iL[0], (float)R.iL[1], (float)R.iL[2]};
  const float tiltf = (float)R.tilt;
  const float margin = 1e-6f * fmaxf(Lf[0], fmaxf(Lf[1], Lf[2]));
  const double4_32a P = A.mixed ? double4_32a{} : A.pos[nxt][p];
  for (int sl = 0; sl < nn; ++sl) {
    const int q = A.nbr[nxt][(int64_t)sl * Np + p] & kNbrIndexMask;
    if (A.mixed) {
      const float4 Q = reinterpret_cast<const float4*>(A.pos[nxt])[2 * q];
      float ry = Q.y - Pf.y, rx = Q.x - Pf.x, rz = Q.z - Pf.z;
      const float sy = rintf(ry * iLf[1]);
      ry -= sy * Lf[1];
      rx -= sy * tiltf;
      rx -= rintf(rx * iLf[0]) * Lf[0];
      rz -= rintf(rz * iLf[2]) * Lf[2];
      const float S = (Pf.w + Q.w) * (1.0f + 1e-5f) + margin;
      if (!(rx * rx + ry * ry + rz * rz < S * S)) continue;
    } else {
      const double4_32a Q = A.pos[nxt][q];
      double rr[3], sy;
      min_image_f64(Q.x - P.x, Q.y - P.y, Q.z - P.z, L, R.iL, R.tilt, rr, &sy);
      const double d2 = rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2];
      if (!(sqrt(d2) < P.w + Q.w)) continue;
    }
    const int oq = A.perm[q];
    // the pair's slot in the old list: in op's row or in oq's, searched four
    // entries at a time so that their loads overlap
    int row = -1, slot = -1;
    const int n1 = A.nnb[cur][op];
    for (int t = 0; t < n1 && slot < 0; t += 4) {
      int e[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        e[u] = t + u < n1 ? (A.nbr[cur][(int64_t)(t + u) * Np + op] & kNbrIndexMask) : -1;
#pragma unroll
      for (int u = 3; u >= 0; --u)
        if (e[u] == oq) slot = t + u;
    }
    if (slot >= 0) {
      row = op;
    } else {
      const int n2 = A.nnb[cur][oq];
      for (int t = 0; t < n2 && slot < 0; t += 4) {
        int e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          e[u] = t + u < n2 ? (A.nbr[cur][(int64_t)(t + u) * Np + oq] & kNbrIndexMask) : -1;
#pragma unroll
        for (int u = 3; u >= 0; --u)
          if (e[u] == op) slot = t + u;
      }
      if (slot >= 0) row = oq;
    }
    if (row < 0) continue;
    if (!((A.cmsk[cur][row] >> slot) & 1ull)) continue;
    const int64_t src = (int64_t)slot * Np + row;
    const int64_t dst = (int64_t)sl * Np + p;
    if (A.mixed) {
      // one 32-byte record per slot
      const float4* ho = reinterpret_cast<const float4*>(A.hist[cur]);
      float4* hn = reinterpret_cast<float4*>(A.hist[nxt]);
      hn[2 * dst] = ho[2 * src];
      hn[2 * dst + 1] = ho[2 * src + 1];
    } else {
      const double* ho = A.hist[cur];
      double* hn = A.hist[nxt];
      hn[dst] = ho[src];
      hn[dst + hs] = ho[src + hs];
      hn[dst + 2 * hs] = ho[src + 2 * hs];
    }
    cm |= 1ull << sl;
  }
  A.cmsk[nxt][p] = cm;
}

__global__ void k_finish(Arrays A) {
  if (!gate(A.ctl)) return;
  Ctl* ctl = A.ctl;
  ctl->cur = ctl->cur ^ 1;
  ctl->need_rebuild = 0;
  ctl->disp_bound = 0.0;
  ctl->t_since_build = 0.0;
  ctl->steps_since_build = 0;
  ctl->nbuilds = ctl->nbuilds + 1;
}

__global__ void k_reset_counters(Arrays A) {
  if (!gate(A.ctl)) return;
  A.ctl->max_row = 0;
  A.ctl->npairs = 0;
}

static inline unsigned grid_for(int64_t n) {
  return (unsigned)((n + kBlock - 1) / kBlock);
}

void launch_request_rebuild(const Arrays& A, cudaStream_t st) {
  k_request<<<1, 1, 0, st>>>(A.ctl);
}

void launch_rebuild(const Arrays& A, const BlockMap& bm, const StepArgs& s,
                    cudaStream_t st, int mixed) {
  (void)bm;
  const int64_t nc = A.ncell;
  const int nparts = (int)((nc + kScanBlock - 1) / kScanBlock);
  k_reset_counters<<<1, 1, 0, st>>>(A);
  k_zero_counts<<<grid_for(nc + 1), kBlock, 0, st>>>(A);
  k_cellkey<<<grid_for(A.N), kBlock, 0, st>>>(A);
  k_scan_blocks<<<nparts, kBlock, 0, st>>>(A);
  k_scan_top<<<1, 1024, 0, st>>>(A, nparts);
  k_scan_add<<<grid_for(nc), kBlock, 0, st>>>(A);
  k_scatter<<<grid_for(A.N), kBlock, 0, st>>>(A);
  k_cellsort<<<grid_for(nc), kBlock, 0, st>>>(A);
  k_permute<<<grid_for(A.N), kBlock, 0, st>>>(A);
  k_build_list<<<grid_for(A.N), kBlock, 0, st>>>(A, s, 1.0 + 0.5 * s.xi_max);
  if (s.friction) k_remap_history<<<grid_for(A.N), kBlock, 0, st>>>(A);
  if (mixed) launch_mirror_gated_next(A, st);
  if (A.det) launch_rev_build(A, st);
  k_finish<<<1, 1, 0, st>>>(A);
}

}  // namespace susp
