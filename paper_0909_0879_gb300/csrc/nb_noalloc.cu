// Allocation-free force + jerk entry point.
//
// Some callers cannot let a library allocate device memory: code whose
// device memory is all owned by another allocator (a framework's caching
// allocator, or a pool sized once at start-up), code that must not risk the
// device-wide synchronisation cudaMalloc / cudaFree can cause, and hosts
// that forbid allocation after initialisation.  nb_force_jerk_noalloc serves
// them: the caller passes every input and output buffer, and the only
// scratch the computation needs -- the FP64 partial sums of i-blocks whose
// j-range is split across CTAs -- lives in one file-scope __device__ array
// of fixed size that every GPU loading the library keeps until the process
// exits.
//
// The kernel is a variant of the force kernel in nb_force.cu (same pair
// arithmetic, same split-precision accumulation, same stream-K split of the
// (i-block, j-tile) space with a fixed-order fix-up) that reads the caller's
// FP64 arrays directly: each CTA stages its j-tiles by plain loads and
// converts them to FP32 or double-single records in shared memory, and
// zero-fills records past n, so no padded copy is needed.
#include "../../include/nbody.h"
#include "nb_internal.cuh"

#include <cstring>
#include <mutex>

namespace nbi {
namespace {

constexpr int kNaNT = 256;    // threads per CTA
constexpr int kNaJT = 256;    // j-records per tile
constexpr int kNaFold = 32;   // j per thread between acceleration folds
// Partial-sum scratch: 8 MiB of doubles, enough for kNaMaxCtas CTAs of
// 2 slots x 6 components x 256 i-particles.
constexpr size_t kNaScratchDoubles = size_t(1) << 20;
constexpr int kNaBI = kNaNT;  // one i-particle per thread
constexpr int kNaMaxCtas = static_cast<int>(kNaScratchDoubles / (2 * 6 * kNaBI));

static __device__ __align__(256) double g_noalloc_part[kNaScratchDoubles];

struct NaArgs {
  int64_t n;
  const double *m, *x, *v;
  const int32_t *idx;
  int64_t n_i;
  float eps2;
  double G;
  double *acc, *jerk;
  double *part;  // device address of g_noalloc_part
};

__device__ __forceinline__ void na_ds_add(float &hi, float &lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

__host__ __device__ __forceinline__ int na_owner(uint64_t u, uint64_t U, int P) {
  return static_cast<int>(((u + 1) * static_cast<uint64_t>(P) - 1) / U);
}

template <int PREC, int MASK>
__global__ void __launch_bounds__(kNaNT, 2)
    noalloc_force_kernel(const NaArgs A, const uint64_t U, const int P) {
  __shared__ float4 s_hi[kNaJT], s_lo[kNaJT], s_v[kNaJT];
  const int tid = threadIdx.x;
  const int p = blockIdx.x;
  const uint64_t u0 = U * static_cast<uint64_t>(p) / static_cast<uint64_t>(P);
  const uint64_t u1 = U * static_cast<uint64_t>(p + 1) / static_cast<uint64_t>(P);
  if (u0 >= u1) return;
  const uint64_t n_jt = static_cast<uint64_t>((A.n + kNaJT - 1) / kNaJT);
  const uint64_t ib_first = u0 / n_jt;
  const float eps2 = A.eps2;
  uint64_t u = u0;
  while (u < u1) {
    const uint64_t ib = u / n_jt;
    const uint64_t jt0 = u % n_jt;
    const uint64_t seg = (n_jt - jt0) < (u1 - u) ? (n_jt - jt0) : (u1 - u);
    const bool full = (jt0 == 0) && (seg == n_jt);
    const int64_t k = static_cast<int64_t>(ib) * kNaBI + tid;
    const int64_t i = k < A.n_i ? (A.idx ? A.idx[k] : k) : 0;
    float xh[3], xl[3], vi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double xc = A.x[3 * i + c];
      xh[c] = __double2float_rn(xc);
      xl[c] = PREC ? __double2float_rn(xc - static_cast<double>(xh[c])) : 0.f;
      vi[c] = __double2float_rn(A.v[3 * i + c]);
    }
    float ah[3] = {0, 0, 0}, al[3] = {0, 0, 0}, p1[3] = {0, 0, 0}, p2[3] = {0, 0, 0};
    float jh[3] = {0, 0, 0}, jl[3] = {0, 0, 0};
    for (uint64_t t = 0; t < seg; ++t) {
      const int64_t j = static_cast<int64_t>(jt0 + t) * kNaJT + tid;
      if (j < A.n) {
        const double x0 = A.x[3 * j], x1 = A.x[3 * j + 1], x2 = A.x[3 * j + 2];
        const float h0 = __double2float_rn(x0), h1 = __double2float_rn(x1),
                    h2 = __double2float_rn(x2);
        s_hi[tid] = make_float4(h0, h1, h2, __double2float_rn(A.m[j]));
        s_lo[tid] = make_float4(__double2float_rn(x0 - static_cast<double>(h0)),
                                __double2float_rn(x1 - static_cast<double>(h1)),
                                __double2float_rn(x2 - static_cast<double>(h2)), 0.f);
        s_v[tid] = make_float4(__double2float_rn(A.v[3 * j]), __double2float_rn(A.v[3 * j + 1]),
                               __double2float_rn(A.v[3 * j + 2]), 0.f);
      } else {
        // past the end: zero mass far away adds exactly zero
        s_hi[tid] = make_float4(1.0e15f, 1.0e15f, 1.0e15f, 0.f);
        s_lo[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_v[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncthreads();
#pragma unroll 1
      for (int c0 = 0; c0 < kNaJT; c0 += kNaFold) {
        float pa[3] = {0, 0, 0};
#pragma unroll 4
        for (int jj = c0; jj < c0 + kNaFold; ++jj) {
          const float4 hj = s_hi[jj];
          const float4 wj = s_v[jj];
          float dx, dy, dz;
          if (PREC) {
            const float4 lj = s_lo[jj];
            dx = (hj.x - xh[0]) + (lj.x - xl[0]);
            dy = (hj.y - xh[1]) + (lj.y - xl[1]);
            dz = (hj.z - xh[2]) + (lj.z - xl[2]);
          } else {
            dx = hj.x - xh[0];
            dy = hj.y - xh[1];
            dz = hj.z - xh[2];
          }
          const float ux = wj.x - vi[0], uy = wj.y - vi[1], uz = wj.z - vi[2];
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
          float rinv;
          if (MASK)
            rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
          else
            rinv = rsqrtf(r2);
          const float rinv2 = rinv * rinv;
          const float mr3 = (hj.w * rinv) * rinv2;
          const float rv = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
          const float cc = (rv * rinv2) * mr3;
          pa[0] = fmaf(mr3, dx, pa[0]);
          pa[1] = fmaf(mr3, dy, pa[1]);
          pa[2] = fmaf(mr3, dz, pa[2]);
          p1[0] = fmaf(mr3, ux, p1[0]);
          p1[1] = fmaf(mr3, uy, p1[1]);
          p1[2] = fmaf(mr3, uz, p1[2]);
          p2[0] = fmaf(cc, dx, p2[0]);
          p2[1] = fmaf(cc, dy, p2[1]);
          p2[2] = fmaf(cc, dz, p2[2]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (PREC)
            na_ds_add(ah[c], al[c], pa[c]);
          else
            ah[c] += pa[c];
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float jt = fmaf(-3.f, p2[c], p1[c]);
        p1[c] = p2[c] = 0.f;
        if (PREC)
          na_ds_add(jh[c], jl[c], jt);
        else
          jh[c] += jt;
      }
      __syncthreads();
    }
    if (k < A.n_i) {
      double o[6];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o[c] = static_cast<double>(ah[c]) + static_cast<double>(al[c]);
        o[3 + c] = static_cast<double>(jh[c]) + static_cast<double>(jl[c]);
      }
      if (full) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          A.acc[3 * k + c] = A.G * o[c];
          A.jerk[3 * k + c] = A.G * o[3 + c];
        }
      } else {
        const int slot = (ib == ib_first) ? 0 : 1;
        double *dst = A.part + static_cast<size_t>(p * 2 + slot) * 6 * kNaBI;
#pragma unroll
        for (int c = 0; c < 6; ++c) dst[static_cast<size_t>(c) * kNaBI + tid] = o[c];
      }
    }
    u += seg;
  }
}

__global__ void noalloc_fixup_kernel(const double *__restrict__ part, int64_t n_i,
                                     uint64_t n_jt, uint64_t U, int P, double G,
                                     double *__restrict__ acc, double *__restrict__ jerk) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n_i) return;
  const uint64_t ib = static_cast<uint64_t>(k) / kNaBI;
  const int kk = static_cast<int>(static_cast<uint64_t>(k) % kNaBI);
  const int plo = na_owner(ib * n_jt, U, P);
  const int phi = na_owner((ib + 1) * n_jt - 1, U, P);
  if (plo == phi) return;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int p = plo; p <= phi; ++p) {
    const uint64_t u0p = U * static_cast<uint64_t>(p) / static_cast<uint64_t>(P);
    const int slot = (u0p / n_jt == ib) ? 0 : 1;
    const double *src = part + static_cast<size_t>(p * 2 + slot) * 6 * kNaBI;
#pragma unroll
    for (int c = 0; c < 6; ++c) s[c] += src[static_cast<size_t>(c) * kNaBI + kk];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[3 * k + c] = G * s[c];
    jerk[3 * k + c] = G * s[3 + c];
  }
}

// Per-device set-up: the device address of the scratch array and the
// resident CTA count, resolved once with that device current.
struct NaDevice {
  bool ready = false;
  double *part = nullptr;
  int num_sms = 0;
  int per_sm[4] = {0, 0, 0, 0};
};
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
NaDevice g_na_dev[kNaMaxDevices];

using NaKernel = void (*)(const NaArgs, const uint64_t, const int);
NaKernel na_kernel(int prec, int mask) {
  if (prec)
    return mask ? &noalloc_force_kernel<1, 1> : &noalloc_force_kernel<1, 0>;
  return mask ? &noalloc_force_kernel<0, 1> : &noalloc_force_kernel<0, 0>;
}

int na_setup(int dev, NaDevice **out) {
  std::lock_guard<std::mutex> lk(g_na_mu);
  NaDevice &D = g_na_dev[dev];
  if (!D.ready) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_part);
    if (e != cudaSuccess)
      return set_error(NB_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed: %s",
                       cudaGetErrorString(e));
    e = cudaDeviceGetAttribute(&D.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
      return set_error(NB_ERR_CUDA, "device attribute query failed: %s", cudaGetErrorString(e));
    for (int prec = 0; prec < 2; ++prec)
      for (int mask = 0; mask < 2; ++mask) {
        int nb = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, na_kernel(prec, mask), kNaNT, 0) !=
                cudaSuccess ||
            nb < 1)
          nb = 1;
        D.per_sm[prec * 2 + mask] = nb;
      }
    D.part = static_cast<double *>(ptr);
    D.ready = true;
  }
  *out = &D;
  return NB_OK;
}

}  // namespace
}  // namespace nbi

using namespace nbi;

extern "C" nb_status nb_force_jerk_noalloc(int64_t n, const double *d_m, const double *d_x,
                                           const double *d_v, const int32_t *d_idx,
                                           int64_t n_idx, double eps, double G,
                                           int32_t precision, double *d_acc, double *d_jerk,
                                           void *stream) {
  if (n < 1 || n > INT32_MAX)
    return static_cast<nb_status>(set_error(
        NB_ERR_INVALID_ARG, "n = %lld out of range [1, 2^31 - 1]", static_cast<long long>(n)));
  if (n_idx < 0 || n_idx > INT32_MAX)
    return static_cast<nb_status>(set_error(NB_ERR_INVALID_ARG,
                                            "n_idx = %lld out of range [0, 2^31 - 1]",
                                            static_cast<long long>(n_idx)));
  if (d_idx == nullptr && n_idx > n)
    return static_cast<nb_status>(
        set_error(NB_ERR_INVALID_ARG, "without an index list n_idx must not exceed n"));
  if (!d_m || !d_x || !d_v || (n_idx > 0 && (!d_acc || !d_jerk)))
    return static_cast<nb_status>(set_error(NB_ERR_INVALID_ARG, "null device pointer"));
  if (!(eps >= 0.0) || !(G > 0.0) || (precision != NB_FP32 && precision != NB_DS))
    return static_cast<nb_status>(
        set_error(NB_ERR_INVALID_ARG, "need eps >= 0, G > 0 and precision NB_FP32 or NB_DS"));
  if (n_idx == 0) return NB_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return static_cast<nb_status>(
        set_error(NB_ERR_CUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e)));
  if (dev < 0 || dev >= kNaMaxDevices)
    return static_cast<nb_status>(set_error(NB_ERR_INVALID_ARG, "device index %d too large", dev));
  NaDevice *D = nullptr;
  int st = na_setup(dev, &D);
  if (st != NB_OK) return static_cast<nb_status>(st);
  const int mask = eps_masks(eps);
  const uint64_t n_jt = static_cast<uint64_t>((n + kNaJT - 1) / kNaJT);
  const uint64_t n_ib = static_cast<uint64_t>((n_idx + kNaBI - 1) / kNaBI);
  const uint64_t U = n_ib * n_jt;
  int64_t P = static_cast<int64_t>(D->num_sms) * D->per_sm[precision * 2 + mask];
  if (P > kNaMaxCtas) P = kNaMaxCtas;
  if (static_cast<int64_t>(U) < P) P = static_cast<int64_t>(U);
  const size_t need = static_cast<size_t>(P) * 2 * 6 * kNaBI;
  if (need > kNaScratchDoubles)
    return static_cast<nb_status>(set_error(
        NB_ERR_INVALID_ARG, "partial sums of %lld CTAs exceed the %zu-double no-alloc scratch",
        static_cast<long long>(P), kNaScratchDoubles));
  NaArgs A;
  A.n = n;
  A.m = d_m;
  A.x = d_x;
  A.v = d_v;
  A.idx = d_idx;
  A.n_i = n_idx;
  A.eps2 = eps2_f32(eps);
  A.G = G;
  A.acc = d_acc;
  A.jerk = d_jerk;
  A.part = D->part;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // An error left pending by earlier work on this thread would be returned
  // by the launch check below and blamed on this call: report it as what it
  // is (without clearing it) and launch nothing.
  e = cudaPeekAtLastError();
  if (e != cudaSuccess)
    return static_cast<nb_status>(set_error(
        NB_ERR_CUDA, "a CUDA error from earlier work is pending (left set): %s",
        cudaGetErrorString(e)));
  na_kernel(precision, mask)<<<static_cast<unsigned>(P), kNaNT, 0, s>>>(A, U,
                                                                         static_cast<int>(P));
  e = cudaGetLastError();
  if (e == cudaSuccess && !(U % static_cast<uint64_t>(P) == 0 &&
                            (U / static_cast<uint64_t>(P)) % n_jt == 0)) {
    const int64_t nb = (n_idx + 255) / 256;
    noalloc_fixup_kernel<<<static_cast<unsigned>(nb), 256, 0, s>>>(
        D->part, n_idx, n_jt, U, static_cast<int>(P), G, d_acc, d_jerk);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return static_cast<nb_status>(
        set_error(NB_ERR_CUDA, "no-alloc force launch failed: %s", cudaGetErrorString(e)));
  return NB_OK;
}
