// Differentiable leapfrog: the paper's second-order symplectic integrator
// (Sec. 3.1, kick-drift-kick form) in FP32 on the GPU, with a hand-written
// adjoint of the force sum and a checkpointed reverse pass.
//
// Force (acceleration only):  a_i = G sum_{j != i} m_j d / s^3,
//   d = x_j - x_i, s^2 = |d|^2 + eps^2.
// Adjoint of the force map for a cotangent g_i = dL/da_i, with the softened
// tidal tensor T(d) = I / s^3 - 3 d d^T / s^5 (symmetric, even in d):
//   dL/dx_k = G sum_{j != k} T(x_j - x_k) (m_k g_j - m_j g_k)
//   dL/dm_k = G sum_{i != k} g_i . (x_k - x_i) / s_ik^3
// Both sums are i-parallel: each CTA holds 32 i-particles, 8 threads per
// particle split the j-range and meet by a warp-shuffle butterfly, so the
// results do not depend on launch order.  j-tiles are staged in shared
// memory by the CTA's threads.  The i == j term is exactly zero for eps > 0
// and masked for eps == 0.
//
// Reverse of one KDK step (x, v) -> (x', v'):
//   v_h = v + A(x) dt/2, x' = x + v_h dt, v' = v_h + A(x') dt/2
//   lv_h = lv'; (lx', lm) += vjp_A(x'; lv' dt/2); lv_h += lx' dt;
//   (lx, lm) += vjp_A(x; lv_h dt/2); lx = lx', lv = lv_h
// The forward pass stores (x, v) every `ckpt_every` steps; the reverse pass
// re-runs each segment from its checkpoint, keeping the segment's positions,
// then walks it backwards.
#include "../../include/nbody.h"
#include "nb_internal.cuh"

#include <algorithm>
#include <cmath>

namespace nbi {
namespace {

constexpr int kLfT = 256;              // threads per CTA
constexpr int kLfTpi = 8;              // threads per i-particle
constexpr int kLfI = kLfT / kLfTpi;    // i-particles per CTA
constexpr int kLfJT = 256;             // j-records per shared tile

template <int MASK>
__global__ void __launch_bounds__(kLfT) lf_acc_kernel(int64_t n, const float *__restrict__ x,
                                                      const float *__restrict__ m, float eps2,
                                                      float G, float *__restrict__ acc) {
  __shared__ float4 sj[kLfJT];
  const int g = threadIdx.x / kLfTpi, r = threadIdx.x % kLfTpi;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kLfI + g;
  const int64_t ii = i < n ? i : 0;
  const float xi = x[3 * ii], yi = x[3 * ii + 1], zi = x[3 * ii + 2];
  float ax = 0.f, ay = 0.f, az = 0.f;
  for (int64_t j0 = 0; j0 < n; j0 += kLfJT) {
    const int64_t j = j0 + threadIdx.x;
    sj[threadIdx.x] = j < n ? make_float4(x[3 * j], x[3 * j + 1], x[3 * j + 2], m[j])
                            : make_float4(1.0e15f, 1.0e15f, 1.0e15f, 0.f);
    __syncthreads();
#pragma unroll 4
    for (int t = r; t < kLfJT; t += kLfTpi) {
      const float4 q = sj[t];
      const float dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
      const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
      float rinv;
      if (MASK)
        rinv = s2 > 0.f ? rsqrtf(s2) : 0.f;
      else
        rinv = rsqrtf(s2);
      const float f = (q.w * rinv) * (rinv * rinv);
      ax = fmaf(f, dx, ax);
      ay = fmaf(f, dy, ay);
      az = fmaf(f, dz, az);
    }
    __syncthreads();
  }
#pragma unroll
  for (int off = 1; off < kLfTpi; off <<= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, off);
    ay += __shfl_xor_sync(0xffffffffu, ay, off);
    az += __shfl_xor_sync(0xffffffffu, az, off);
  }
  if (r == 0 && i < n) {
    acc[3 * i] = G * ax;
    acc[3 * i + 1] = G * ay;
    acc[3 * i + 2] = G * az;
  }
}

// Wide shape for large N: each thread holds 4 i-particles, two per packed
// FP32x2 instruction (per-lane IEEE rounding), and TPI threads share an
// i-particle group, splitting every shared-memory tile's j-range (their sums
// meet by a warp-shuffle butterfly); 1,024 / TPI i-particles per CTA.  The
// next tile is read into registers while the current one is summed, and each
// tile's sum is added to the running total, so no FP32 sum runs over more
// than 256 / TPI terms plus one term per tile.
constexpr int kLfWideIpt = 4;

template <int MASK>
__device__ __forceinline__ float2 lf_rsq2(float2 s2) {
  float2 r;
  r.x = MASK ? (s2.x > 0.f ? rsqrtf(s2.x) : 0.f) : rsqrtf(s2.x);
  r.y = MASK ? (s2.y > 0.f ? rsqrtf(s2.y) : 0.f) : rsqrtf(s2.y);
  return r;
}

template <int MASK, int TPI>
__global__ void __launch_bounds__(kLfT) lf_acc_wide_kernel(int64_t n, const float *__restrict__ x,
                                                           const float *__restrict__ m,
                                                           float eps2, float G,
                                                           float *__restrict__ acc) {
  __shared__ float4 sj[kLfJT];
  constexpr int NQ = kLfWideIpt / 2;
  constexpr int NG = kLfT / TPI;            // i-particle groups per CTA
  constexpr int BI = NG * kLfWideIpt;       // i-particles per CTA
  const int tid = threadIdx.x, g = tid / TPI, r = tid % TPI;
  float2 nx[NQ], ny[NQ], nz[NQ];  // negated i-positions, two particles per pair
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * BI + g + (2 * q) * NG;
    const int64_t i1 = i0 + NG;
    const int64_t a0 = i0 < n ? i0 : 0, a1 = i1 < n ? i1 : 0;
    nx[q] = make_float2(-x[3 * a0], -x[3 * a1]);
    ny[q] = make_float2(-x[3 * a0 + 1], -x[3 * a1 + 1]);
    nz[q] = make_float2(-x[3 * a0 + 2], -x[3 * a1 + 2]);
  }
  const float2 e2 = make_float2(eps2, eps2);
  float2 tx[NQ], ty[NQ], tz[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) tx[q] = ty[q] = tz[q] = make_float2(0.f, 0.f);
  auto fetch = [&](int64_t j) {
    return j < n ? make_float4(x[3 * j], x[3 * j + 1], x[3 * j + 2], m[j])
                 : make_float4(1.0e15f, 1.0e15f, 1.0e15f, 0.f);
  };
  float4 next = fetch(tid);
  for (int64_t j0 = 0; j0 < n; j0 += kLfJT) {
    __syncthreads();  // the previous tile's readers are done
    sj[tid] = next;
    __syncthreads();
    next = fetch(j0 + kLfJT + tid);
    float2 px[NQ], py[NQ], pz[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) px[q] = py[q] = pz[q] = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int t = r; t < kLfJT; t += TPI) {
      const float4 qj = sj[t];
      const float2 xj = make_float2(qj.x, qj.x), yj = make_float2(qj.y, qj.y);
      const float2 zj = make_float2(qj.z, qj.z), mj = make_float2(qj.w, qj.w);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const float2 dx = __fadd2_rn(xj, nx[q]), dy = __fadd2_rn(yj, ny[q]);
        const float2 dz = __fadd2_rn(zj, nz[q]);
        const float2 s2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
        const float2 ri = lf_rsq2<MASK>(s2);
        const float2 f = __fmul2_rn(__fmul2_rn(mj, ri), __fmul2_rn(ri, ri));
        px[q] = __ffma2_rn(f, dx, px[q]);
        py[q] = __ffma2_rn(f, dy, py[q]);
        pz[q] = __ffma2_rn(f, dz, pz[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      tx[q] = __fadd2_rn(tx[q], px[q]);
      ty[q] = __fadd2_rn(ty[q], py[q]);
      tz[q] = __fadd2_rn(tz[q], pz[q]);
    }
  }
  if (TPI > 1) {
#pragma unroll
    for (int off = 1; off < TPI; off <<= 1)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        tx[q].x += __shfl_xor_sync(0xffffffffu, tx[q].x, off);
        tx[q].y += __shfl_xor_sync(0xffffffffu, tx[q].y, off);
        ty[q].x += __shfl_xor_sync(0xffffffffu, ty[q].x, off);
        ty[q].y += __shfl_xor_sync(0xffffffffu, ty[q].y, off);
        tz[q].x += __shfl_xor_sync(0xffffffffu, tz[q].x, off);
        tz[q].y += __shfl_xor_sync(0xffffffffu, tz[q].y, off);
      }
  }
  if (r != 0) return;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * BI + g + (2 * q) * NG;
    const int64_t i1 = i0 + NG;
    if (i0 < n) {
      acc[3 * i0] = G * tx[q].x;
      acc[3 * i0 + 1] = G * ty[q].x;
      acc[3 * i0 + 2] = G * tz[q].x;
    }
    if (i1 < n) {
      acc[3 * i1] = G * tx[q].y;
      acc[3 * i1 + 1] = G * ty[q].y;
      acc[3 * i1 + 2] = G * tz[q].y;
    }
  }
}

// lx_k += dL/dx_k and lm_k += dL/dm_k for the cotangent g = h * lv; with
// lv_out set, also lv_out_k = lv_k + dlv lx_k with the updated lx_k (the
// adjoint of the drift, as a separate elementwise launch would compute it).
template <int MASK>
__global__ void __launch_bounds__(kLfT)
    lf_vjp_kernel(int64_t n, const float *__restrict__ x, const float *__restrict__ m,
                  const float *__restrict__ lv, float h, float eps2, float G,
                  float *__restrict__ lx, float *__restrict__ lm, float *__restrict__ lv_out,
                  float dlv) {
  __shared__ float4 sx[kLfJT];
  __shared__ float4 sg[kLfJT];
  const int g = threadIdx.x / kLfTpi, r = threadIdx.x % kLfTpi;
  const int64_t k = static_cast<int64_t>(blockIdx.x) * kLfI + g;
  const int64_t kk = k < n ? k : 0;
  const float xk = x[3 * kk], yk = x[3 * kk + 1], zk = x[3 * kk + 2], mk = m[kk];
  const float gkx = h * lv[3 * kk], gky = h * lv[3 * kk + 1], gkz = h * lv[3 * kk + 2];
  float ox = 0.f, oy = 0.f, oz = 0.f, om = 0.f;
  for (int64_t j0 = 0; j0 < n; j0 += kLfJT) {
    const int64_t j = j0 + threadIdx.x;
    if (j < n) {
      sx[threadIdx.x] = make_float4(x[3 * j], x[3 * j + 1], x[3 * j + 2], m[j]);
      sg[threadIdx.x] = make_float4(h * lv[3 * j], h * lv[3 * j + 1], h * lv[3 * j + 2], 0.f);
    } else {
      sx[threadIdx.x] = make_float4(1.0e15f, 1.0e15f, 1.0e15f, 0.f);
      sg[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 2
    for (int t = r; t < kLfJT; t += kLfTpi) {
      const float4 q = sx[t];
      const float4 gj = sg[t];
      const float dx = q.x - xk, dy = q.y - yk, dz = q.z - zk;
      const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
      float rinv;
      if (MASK)
        rinv = s2 > 0.f ? rsqrtf(s2) : 0.f;
      else
        rinv = rsqrtf(s2);
      const float rinv2 = rinv * rinv;
      const float s3 = rinv * rinv2;
      const float s5 = s3 * rinv2;
      // u = m_k g_j - m_j g_k with both products rounded alike, so that the
      // i == j term is exactly zero (a fused form would leave the rounding
      // error of one product, amplified by 1/eps^3)
      const float ux = __fsub_rn(__fmul_rn(mk, gj.x), __fmul_rn(q.w, gkx));
      const float uy = __fsub_rn(__fmul_rn(mk, gj.y), __fmul_rn(q.w, gky));
      const float uz = __fsub_rn(__fmul_rn(mk, gj.z), __fmul_rn(q.w, gkz));
      const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
      const float c = 3.f * du * s5;
      ox = fmaf(ux, s3, fmaf(-c, dx, ox));
      oy = fmaf(uy, s3, fmaf(-c, dy, oy));
      oz = fmaf(uz, s3, fmaf(-c, dz, oz));
      // g_j . (x_k - x_j) / s^3 = -(g_j . d) s3
      om = fmaf(-fmaf(gj.x, dx, fmaf(gj.y, dy, gj.z * dz)), s3, om);
    }
    __syncthreads();
  }
#pragma unroll
  for (int off = 1; off < kLfTpi; off <<= 1) {
    ox += __shfl_xor_sync(0xffffffffu, ox, off);
    oy += __shfl_xor_sync(0xffffffffu, oy, off);
    oz += __shfl_xor_sync(0xffffffffu, oz, off);
    om += __shfl_xor_sync(0xffffffffu, om, off);
  }
  if (r == 0 && k < n) {
    const float o3[3] = {ox, oy, oz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float lxn = lx[3 * k + c] + G * o3[c];
      lx[3 * k + c] = lxn;
      if (lv_out) lv_out[3 * k + c] = fmaf(dlv, lxn, lv[3 * k + c]);
    }
    lm[k] += G * om;
  }
}

// v += a h; then, if drift, x += v dt.
__global__ void lf_kick_drift_kernel(int64_t n3, float *__restrict__ x, float *__restrict__ v,
                                     const float *__restrict__ a, float h, float dt, int drift) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n3) return;
  const float vn = fmaf(a[q], h, v[q]);
  v[q] = vn;
  if (drift) x[q] = fmaf(vn, dt, x[q]);
}

// One drift of a run of KDK steps with the kicks around it merged: with
// close set, the previous step's closing kick v += a h first; then, when
// ck_x is set, the checkpoint (x, v) of the step boundary; then this step's
// opening kick v += a h and the drift x_out = x_in + v dt.  The same
// per-element operations in the same order as separate kick and drift
// launches.  x_in may equal x_out.
__global__ void lf_step_kernel(int64_t n3, const float *x_in, float *x_out,
                               float *__restrict__ v, const float *__restrict__ a, float h,
                               float dt, int close, float *__restrict__ ck_x,
                               float *__restrict__ ck_v) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n3) return;
  const float aq = a[q], xq = x_in[q];
  float vq = v[q];
  if (close) vq = fmaf(aq, h, vq);
  if (ck_x) {
    ck_x[q] = xq;
    ck_v[q] = vq;
  }
  vq = fmaf(aq, h, vq);
  v[q] = vq;
  x_out[q] = fmaf(vq, dt, xq);
}

struct LfCtx {
  int64_t n;
  const float *m;
  float eps2, G;
  int mask;
  int sms;
  cudaStream_t s;
  int64_t launches;
};

// N >= kLfWideMin takes the wide shape; below it, the 8-threads-per-particle
// shape keeps enough CTAs to fill the GPU (N = 4096: 128 CTAs).
constexpr int64_t kLfWideMin = 65536;

// Threads per i-particle group of the wide shape, 4 or 8.  CTAs take the
// same time, so an SM's share is ceil(grid / SMs) CTAs run one after
// another; 8 threads halve the i-particles per CTA, and are taken where the
// grid then divides more evenly over the SMs (N = 131072 on 152 SMs: 3.4
// against 6.7 CTAs per SM).
int lf_wide_tpi(int64_t n, int sms) {
  auto balance = [&](int tpi) {
    const int64_t bi = kLfT / tpi * kLfWideIpt;
    const int64_t grid = (n + bi - 1) / bi;
    const int64_t rounds = (grid + sms - 1) / sms;
    return static_cast<double>(grid) / static_cast<double>(rounds * sms);
  };
  return balance(8) > balance(4) + 0.01 ? 8 : 4;
}

template <int TPI>
void launch_lf_wide(const LfCtx &C, const float *x, float *acc) {
  constexpr int bi = kLfT / TPI * kLfWideIpt;
  const unsigned grid = static_cast<unsigned>((C.n + bi - 1) / bi);
  if (C.mask)
    lf_acc_wide_kernel<1, TPI><<<grid, kLfT, 0, C.s>>>(C.n, x, C.m, C.eps2, C.G, acc);
  else
    lf_acc_wide_kernel<0, TPI><<<grid, kLfT, 0, C.s>>>(C.n, x, C.m, C.eps2, C.G, acc);
}

cudaError_t lf_acc(LfCtx &C, const float *x, float *acc) {
  if (C.n >= kLfWideMin) {
    if (lf_wide_tpi(C.n, C.sms) == 8)
      launch_lf_wide<8>(C, x, acc);
    else
      launch_lf_wide<4>(C, x, acc);
  } else {
    const unsigned grid = static_cast<unsigned>((C.n + kLfI - 1) / kLfI);
    if (C.mask)
      lf_acc_kernel<1><<<grid, kLfT, 0, C.s>>>(C.n, x, C.m, C.eps2, C.G, acc);
    else
      lf_acc_kernel<0><<<grid, kLfT, 0, C.s>>>(C.n, x, C.m, C.eps2, C.G, acc);
  }
  ++C.launches;
  return cudaGetLastError();
}

cudaError_t lf_vjp(LfCtx &C, const float *x, const float *lv, float h, float *lx, float *lm,
                   float *lv_out = nullptr, float dlv = 0.f) {
  const unsigned grid = static_cast<unsigned>((C.n + kLfI - 1) / kLfI);
  if (C.mask)
    lf_vjp_kernel<1><<<grid, kLfT, 0, C.s>>>(C.n, x, C.m, lv, h, C.eps2, C.G, lx, lm, lv_out,
                                             dlv);
  else
    lf_vjp_kernel<0><<<grid, kLfT, 0, C.s>>>(C.n, x, C.m, lv, h, C.eps2, C.G, lx, lm, lv_out,
                                             dlv);
  ++C.launches;
  return cudaGetLastError();
}

cudaError_t lf_kick(LfCtx &C, float *x, float *v, const float *a, float h, float dt, int drift) {
  const int64_t n3 = 3 * C.n;
  lf_kick_drift_kernel<<<static_cast<unsigned>((n3 + 255) / 256), 256, 0, C.s>>>(n3, x, v, a, h,
                                                                                  dt, drift);
  ++C.launches;
  return cudaGetLastError();
}

// The drift of one KDK step with the kicks around it (see lf_step_kernel),
// then A(x_out) into acc; the step's own closing kick is left to the next
// call (close = 1) or to a final lf_kick without drift.
cudaError_t lf_half_step(LfCtx &C, const float *x_in, float *x_out, float *v, float *acc,
                         float dt, bool close, float *ck) {
  const int64_t n3 = 3 * C.n;
  lf_step_kernel<<<static_cast<unsigned>((n3 + 255) / 256), 256, 0, C.s>>>(
      n3, x_in, x_out, v, acc, 0.5f * dt, dt, close ? 1 : 0, ck, ck ? ck + n3 : nullptr);
  ++C.launches;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = lf_acc(C, x_out, acc);
  return e;
}

nb_status lf_check(int64_t n, float eps, float G, const void *a, const void *b) {
  if (n < 1 || n > (int64_t(1) << 30))
    return static_cast<nb_status>(set_error(NB_ERR_INVALID_ARG, "n out of range [1, 2^30]"));
  if (!(eps >= 0.f) || !(G > 0.f))
    return static_cast<nb_status>(set_error(NB_ERR_INVALID_ARG, "need eps >= 0 and G > 0"));
  if (!a || !b) return static_cast<nb_status>(set_error(NB_ERR_INVALID_ARG, "null device pointer"));
  return NB_OK;
}

nb_status lf_err(cudaError_t e) {
  return static_cast<nb_status>(
      set_error(NB_ERR_CUDA, "leapfrog kernel launch failed: %s", cudaGetErrorString(e)));
}

LfCtx make_ctx(int64_t n, const float *m, float eps, float G, void *stream) {
  LfCtx C;
  C.n = n;
  C.m = m;
  // eps^2 not a normal float: the kernels zero the i == j term (and take
  // eps^2 = 0, which is what the device's flush of subnormals would make of it)
  C.mask = eps * eps < FLT_MIN ? 1 : 0;
  C.eps2 = C.mask ? 0.f : eps * eps;
  C.G = G;
  // A failed query leaves its error for the launch's error check to report.
  int dev = 0;
  C.sms = 0;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&C.sms, cudaDevAttrMultiProcessorCount, dev);
  if (C.sms < 1) C.sms = 1;
  C.s = static_cast<cudaStream_t>(stream);
  C.launches = 0;
  return C;
}

}  // namespace
}  // namespace nbi

using namespace nbi;

extern "C" {

nb_status nb_lf_acc(int64_t n, const float *d_x, const float *d_m, float eps, float G,
                    float *d_acc, void *stream) {
  nb_status s = lf_check(n, eps, G, d_x, d_m);
  if (s != NB_OK) return s;
  if (!d_acc) return static_cast<nb_status>(set_error(NB_ERR_INVALID_ARG, "null output"));
  LfCtx C = make_ctx(n, d_m, eps, G, stream);
  cudaError_t e = lf_acc(C, d_x, d_acc);
  return e == cudaSuccess ? NB_OK : lf_err(e);
}

nb_status nb_lf_acc_vjp(int64_t n, const float *d_x, const float *d_m, const float *d_g,
                        float eps, float G, float *d_gx, float *d_gm, void *stream) {
  nb_status s = lf_check(n, eps, G, d_x, d_m);
  if (s != NB_OK) return s;
  if (!d_g || !d_gx || !d_gm)
    return static_cast<nb_status>(set_error(NB_ERR_INVALID_ARG, "null device pointer"));
  LfCtx C = make_ctx(n, d_m, eps, G, stream);
  cudaError_t e = cudaMemsetAsync(d_gx, 0, 3 * n * sizeof(float), C.s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_gm, 0, n * sizeof(float), C.s);
  if (e == cudaSuccess) e = lf_vjp(C, d_x, d_g, 1.f, d_gx, d_gm);
  return e == cudaSuccess ? NB_OK : lf_err(e);
}

int64_t nb_lf_ckpt_floats(int64_t n, int64_t nsteps, int32_t ckpt_every) {
  if (n < 1 || nsteps < 0 || ckpt_every < 1) return -1;
  const int64_t K = (nsteps + ckpt_every - 1) / ckpt_every;
  return std::max<int64_t>(K, 1) * 6 * n;
}

int64_t nb_lf_work_floats(int64_t n, int32_t ckpt_every) {
  if (n < 1 || ckpt_every < 1) return -1;
  return (static_cast<int64_t>(ckpt_every) + 1) * 3 * n + 6 * n;
}

nb_status nb_lf_forward(int64_t n, const float *d_m, float *d_x, float *d_v, float *d_acc,
                        int64_t nsteps, float dt, float eps, float G, int32_t ckpt_every,
                        float *d_ckpt, void *stream) {
  nb_status s = lf_check(n, eps, G, d_m, d_x);
  if (s != NB_OK) return s;
  if (!d_v || !d_acc || nsteps < 0 || ckpt_every < 1 || !(std::isfinite(dt)))
    return static_cast<nb_status>(set_error(NB_ERR_INVALID_ARG, "bad leapfrog arguments"));
  LfCtx C = make_ctx(n, d_m, eps, G, stream);
  cudaError_t e = lf_acc(C, d_x, d_acc);
  for (int64_t st = 0; st < nsteps && e == cudaSuccess; ++st) {
    float *ck = (d_ckpt && st % ckpt_every == 0) ? d_ckpt + (st / ckpt_every) * 6 * n : nullptr;
    e = lf_half_step(C, d_x, d_x, d_v, d_acc, dt, st > 0, ck);
  }
  if (e == cudaSuccess && nsteps > 0) e = lf_kick(C, d_x, d_v, d_acc, 0.5f * dt, dt, 0);
  return e == cudaSuccess ? NB_OK : lf_err(e);
}

nb_status nb_lf_backward(int64_t n, const float *d_m, const float *d_ckpt, int64_t nsteps,
                         float dt, float eps, float G, int32_t ckpt_every, float *d_lx,
                         float *d_lv, float *d_lm, float *d_work, void *stream) {
  nb_status s = lf_check(n, eps, G, d_m, d_ckpt);
  if (s != NB_OK) return s;
  if (!d_lx || !d_lv || !d_lm || !d_work || nsteps < 0 || ckpt_every < 1)
    return static_cast<nb_status>(set_error(NB_ERR_INVALID_ARG, "bad leapfrog adjoint arguments"));
  LfCtx C = make_ctx(n, d_m, eps, G, stream);
  const size_t n3 = 3 * static_cast<size_t>(n);
  const size_t n3b = n3 * sizeof(float);
  float *xs = d_work;                               // (ckpt_every + 1) positions
  float *v = d_work + (ckpt_every + 1) * n3;        // velocity during recompute
  float *acc = v + n3;                              // acceleration during recompute
  cudaError_t e = cudaMemsetAsync(d_lm, 0, n * sizeof(float), C.s);
  const int64_t K = (nsteps + ckpt_every - 1) / ckpt_every;
  for (int64_t seg = K - 1; seg >= 0 && e == cudaSuccess; --seg) {
    const int64_t s0 = seg * ckpt_every;
    const int64_t L = std::min<int64_t>(ckpt_every, nsteps - s0);
    const float *slot = d_ckpt + seg * 6 * n;
    e = cudaMemcpyAsync(xs, slot, n3b, cudaMemcpyDeviceToDevice, C.s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v, slot + n3, n3b, cudaMemcpyDeviceToDevice, C.s);
    if (e == cudaSuccess) e = lf_acc(C, xs, acc);
    // the segment's positions again (the velocity after the last drift is
    // not needed, so the last closing kick is left out)
    for (int64_t q = 0; q < L && e == cudaSuccess; ++q)
      e = lf_half_step(C, xs + q * n3, xs + (q + 1) * n3, v, acc, dt, q > 0, nullptr);
    // the sweep: second kick, drift (fused into the second kick's launch,
    // writing the new lv to the other of d_lv and the now free velocity
    // buffer), first kick
    float *cur = d_lv, *other = v;
    for (int64_t q = L - 1; q >= 0 && e == cudaSuccess; --q) {
      const float *xa = xs + q * n3, *xb = xs + (q + 1) * n3;
      e = lf_vjp(C, xb, cur, 0.5f * dt, d_lx, d_lm, other, dt);  // second kick, drift
      std::swap(cur, other);
      if (e == cudaSuccess) e = lf_vjp(C, xa, cur, 0.5f * dt, d_lx, d_lm);  // first kick
    }
    if (e == cudaSuccess && cur != d_lv)
      e = cudaMemcpyAsync(d_lv, cur, n3b, cudaMemcpyDeviceToDevice, C.s);
  }
  return e == cudaSuccess ? NB_OK : lf_err(e);
}

}  // extern "C"
