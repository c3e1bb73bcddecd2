// noalloc.cu -- pair stresses of a caller-given pair list without any device
// allocation (susp_pair_stress_noalloc in include/susp.h).
//
// Some callers cannot allocate device memory at the point where they need
// the stress: code running inside another framework's memory arena, a host
// thread that must not touch the allocator, or a tool that only borrows
// buffers owned by someone else.  This entry point takes every input and the
// output as device pointers the caller already owns and keeps its only
// scratch -- the per-block partial sums and the last-block ticket of a
// single-launch reduction -- in the file-scope array below.  Every GPU that
// loads the library holds that array until the process exits.
//
// The arithmetic is that of the double-precision pair kernel for one
// evaluation (lubrication, pair noise and the normal contact force; the
// tangential history belongs to a handle's time integration and is taken as
// zero), one thread per listed pair; the stresses are
// (1/V) sum F_{i<-j} (x) r_ij for the contact, lubrication and pair
// Brownian parts.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/susp.h"
#include "device_common.cuh"
#include "philox.cuh"
#include "susp_internal.h"

namespace susp {

constexpr int kNoallocBlocks = SUSP_NOALLOC_MAX_PAIRS / kBlock;
// header (ticket + padding) then [kNoallocBlocks][27] block partials
constexpr int kNoallocHeader = 32;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocHeader +
                                                          kNoallocBlocks * kVirLen];

struct NoallocArgs {
  const double* x;
  const double* U;
  const double* W;
  const double* radii;
  const int32_t* ij;
  int64_t npairs;
  int64_t N;
  double L[3];
  double tilt, rate, eta, kn, noise_c, xi_min, xi_max, torque_sign, inv_V;
  uint32_t key0, key1;
  long long k;
  int noise, lubrication, contact;
};

template <bool NOISE>
__global__ void __launch_bounds__(kBlock)
k_pair_stress_noalloc(NoallocArgs a, double* scratch, double* out) {
  __shared__ double smem[(kBlock / 32) * kVirLen];
  __shared__ bool last;
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch);
  double* partial = scratch + kNoallocHeader;
  const int64_t t = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  double vir[kVirLen];
#pragma unroll
  for (int q = 0; q < kVirLen; ++q) vir[q] = 0.0;
  if (t < a.npairs) {
    // i = lower tag: the pair noise is defined for that orientation
    const int i0 = a.ij[2 * t], j0 = a.ij[2 * t + 1];
    const int i = i0 < j0 ? i0 : j0, j = i0 < j0 ? j0 : i0;
    if (i >= 0 && i < j && j < a.N) {
      const double xi_[3] = {a.x[3 * i], a.x[3 * i + 1], a.x[3 * i + 2]};
      const double xj_[3] = {a.x[3 * j], a.x[3 * j + 1], a.x[3 * j + 2]};
      double r[3], sy;
      const double iL[3] = {1.0 / a.L[0], 1.0 / a.L[1], 1.0 / a.L[2]};
      min_image_f64(xj_[0] - xi_[0], xj_[1] - xi_[1], xj_[2] - xi_[2], a.L, iL, a.tilt, r, &sy);
      const double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
      const double id = 1.0 / d;
      const double ai = a.radii[i], aj = a.radii[j];
      const double S = ai + aj;
      const double h = d - S;
      const double xi = 2.0 * h / S;
      if (xi <= a.xi_max) {
        const double n[3] = {r[0] * id, r[1] * id, r[2] * id};
        const double Ui[3] = {a.U[3 * i], a.U[3 * i + 1], a.U[3 * i + 2]};
        const double Uj[3] = {a.U[3 * j], a.U[3 * j + 1], a.U[3 * j + 2]};
        const double Wi[3] = {a.W[3 * i], a.W[3 * i + 1], a.W[3 * i + 2]};
        const double Wj[3] = {a.W[3 * j], a.W[3 * j + 1], a.W[3 * j + 2]};
        const double dU[3] = {Uj[0] - sy * a.rate * a.L[1] - Ui[0], Uj[1] - Ui[1],
                              Uj[2] - Ui[2]};
        PairOut<double> o;
        if (a.lubrication) {
          const double xi_e = xi < a.xi_min ? a.xi_min : xi;
          const double ixi = 1.0 / xi_e;
          const Res8<double> R = resistances_rcp(a.eta, ai, aj, ixi, log(ixi));
          double g[6] = {0, 0, 0, 0, 0, 0};
          // tags are the caller's indices
          if (NOISE) gauss6_f64(a.key0, a.key1, a.k, (uint32_t)i, (uint32_t)j, g);
          lub_brownian<double, NOISE>(R, n, dU, Wi, Wj, g, g + 3, a.noise_c, a.torque_sign, o);
        } else {
#pragma unroll
          for (int q = 0; q < 3; ++q) o.FL[q] = o.FB[q] = 0.0;
        }
        double FC[3] = {0.0, 0.0, 0.0};
        if (h < 0.0 && a.contact) {
#pragma unroll
          for (int q = 0; q < 3; ++q) FC[q] = -a.kn * (-h) * n[q];
        }
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
          for (int be = 0; be < 3; ++be) {
            vir[3 * al + be] += FC[al] * r[be];
            vir[9 + 3 * al + be] += o.FL[al] * r[be];
            vir[18 + 3 * al + be] += o.FB[al] * r[be];
          }
      }
    }
  }
  block_sum_write<kVirLen>(vir, smem, partial + (int64_t)blockIdx.x * kVirLen);
  __threadfence();
  if (threadIdx.x == 0) {
    const unsigned int tk = atomicAdd(ticket, 1u);
    last = (tk == gridDim.x - 1u);
  }
  __syncthreads();
  if (last) {
    // warp w sums components w, w + 8, w + 16, w + 24: its lanes stride over
    // the block partials (lane l takes blocks l, l + 32, ...), then a fixed
    // shuffle tree adds the 32 lane sums, so the order does not depend on
    // scheduling
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = warp; c < kVirLen; c += kBlock / 32) {
      double s = 0.0;
      for (unsigned int b = lane; b < gridDim.x; b += 32)
        s += *(volatile double*)&partial[(int64_t)b * kVirLen + c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) out[c] = s * a.inv_V;
    }
    if (threadIdx.x == 0) *ticket = 0u;
  }
}

namespace {
// device address of the scratch array in each CUDA context seen so far,
// keyed by the context's unique ID (never reused within a process): the
// address belongs to a context, so a call made in another context (after a
// device reset, or in a context the caller created) looks it up again
struct CtxAddr {
  unsigned long long id;
  double* ptr;
};
std::mutex g_noalloc_mutex;
CtxAddr g_noalloc_ptr[64] = {};
int g_noalloc_n = 0;
CUresult (*g_ctx_get_current)(CUcontext*) = nullptr;
CUresult (*g_ctx_get_id)(CUcontext, unsigned long long*) = nullptr;
}  // namespace

}  // namespace susp

// message of the last failing handle-less call (read with susp_create_error)
namespace susp {
void set_handleless_error(const std::string& msg);
}

static int noalloc_fail(int code, const std::string& msg) {
  susp::set_handleless_error(msg);
  return code;
}

extern "C" int susp_pair_stress_noalloc(int64_t N, const double* x, const double* U,
                                        const double* Omega, const double* radii,
                                        int64_t npairs, const int32_t* ij,
                                        const double box[3], double strain,
                                        const susp_params* p, double dt, int64_t k,
                                        double* stress_out, void* stream) {
  using namespace susp;
  set_handleless_error("");
  if (!x || !U || !Omega || !radii || !box || !p || !stress_out || N <= 0 || npairs < 0)
    return noalloc_fail(SUSP_EINVAL, "invalid argument (NULL pointer, N <= 0 or npairs < 0)");
  if (npairs > SUSP_NOALLOC_MAX_PAIRS)
    return noalloc_fail(SUSP_EINVAL,
                        "npairs exceeds SUSP_NOALLOC_MAX_PAIRS, the capacity of the "
                        "static scratch of susp_pair_stress_noalloc");
  if (npairs > 0 && !ij) return noalloc_fail(SUSP_EINVAL, "ij is NULL");
  if (!(dt > 0) || !(p->kT >= 0) || !(box[0] > 0 && box[1] > 0 && box[2] > 0))
    return noalloc_fail(SUSP_EINVAL, "need dt > 0, kT >= 0 and a positive box");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0)
    return noalloc_fail(SUSP_ENODEV, "no usable CUDA device");
  // cudaFree(0) makes the device's primary context current if no context is
  // (it frees nothing)
  if (cudaFree(nullptr) != cudaSuccess)
    return noalloc_fail(SUSP_ENODEV, "no usable CUDA context");
  double* scratch = nullptr;
  {
    // once per CUDA context, with it current: the device address of the
    // static array (its name in host code is only a host-side stand-in)
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_ctx_get_current || !g_ctx_get_id) {
      void* f1 = nullptr;
      void* f2 = nullptr;
      cudaDriverEntryPointQueryResult q1, q2;
      if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &f1, cudaEnableDefault, &q1) != cudaSuccess ||
          q1 != cudaDriverEntryPointSuccess || !f1 ||
          cudaGetDriverEntryPoint("cuCtxGetId", &f2, cudaEnableDefault, &q2) != cudaSuccess ||
          q2 != cudaDriverEntryPointSuccess || !f2)
        return noalloc_fail(SUSP_ECUDA, "cuCtxGetCurrent / cuCtxGetId are not available");
      g_ctx_get_current = reinterpret_cast<CUresult (*)(CUcontext*)>(f1);
      g_ctx_get_id = reinterpret_cast<CUresult (*)(CUcontext, unsigned long long*)>(f2);
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_get_id(ctx, &id) != CUDA_SUCCESS)
      return noalloc_fail(SUSP_ECUDA, "no current CUDA context");
    for (int c = 0; c < g_noalloc_n; ++c)
      if (g_noalloc_ptr[c].id == id) scratch = g_noalloc_ptr[c].ptr;
    if (!scratch) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr)
        return noalloc_fail(SUSP_ECUDA,
                            std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      scratch = static_cast<double*>(ptr);
      // a full table starts over (the entries are only a cache)
      if (g_noalloc_n == 64) g_noalloc_n = 0;
      g_noalloc_ptr[g_noalloc_n++] = CtxAddr{id, scratch};
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  // the ticket must start at zero (a previous call leaves it at zero, an
  // interrupted one might not)
  cudaError_t e = cudaMemsetAsync(scratch, 0, kNoallocHeader * sizeof(double), st);
  if (e != cudaSuccess)
    return noalloc_fail(SUSP_ECUDA, std::string("cudaMemsetAsync failed: ") + cudaGetErrorString(e));
  NoallocArgs a{};
  a.x = x; a.U = U; a.W = Omega; a.radii = radii; a.ij = ij;
  a.npairs = npairs; a.N = N;
  for (int d = 0; d < 3; ++d) a.L[d] = box[d];
  a.tilt = strain * box[1];
  a.rate = p->shear_rate;
  a.eta = p->eta;
  a.kn = p->kn;
  a.noise_c = std::sqrt(2.0 * p->kT / dt);
  a.xi_min = p->xi_min;
  a.xi_max = p->xi_max;
  a.torque_sign = p->torque_sign;
  a.inv_V = 1.0 / (box[0] * box[1] * box[2]);
  a.key0 = (uint32_t)(p->seed & 0xffffffffull);
  a.key1 = (uint32_t)(p->seed >> 32);
  a.k = (long long)k;
  a.noise = p->noise;
  a.lubrication = p->lubrication;
  a.contact = p->contact;
  const unsigned nb = npairs > 0 ? (unsigned)((npairs + kBlock - 1) / kBlock) : 1u;
  if (p->noise)
    k_pair_stress_noalloc<true><<<nb, kBlock, 0, st>>>(a, scratch, stress_out);
  else
    k_pair_stress_noalloc<false><<<nb, kBlock, 0, st>>>(a, scratch, stress_out);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return noalloc_fail(SUSP_ECUDA, std::string("launch failed: ") + cudaGetErrorString(e));
  return SUSP_OK;
}
