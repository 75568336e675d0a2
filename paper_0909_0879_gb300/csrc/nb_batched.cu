// Batched form: thousands of independent small clusters advanced with the
// shared-step Hermite-4 scheme by one persistent kernel.
//
// Each CTA takes a cluster from a work queue (largest first) and advances
// it S steps without leaving the SM: the cluster's predicted j-records live
// in shared memory, every thread owns IPT i-particles, the force + jerk sum
// runs over the shared-memory records (split precision as in the main
// kernel, paper Sec. 4 software double precision), and the owning thread
// applies the FP64 corrector right after its sums are complete.  The FP64
// state is read and written in global memory (it stays in L2 for the
// workload's ~100 MB).  A sequence of such launches is captured in a CUDA
// graph and replayed.
//
// Threads per i-particle adapt to the cluster size: small clusters spread
// each i-particle's j-range over up to 32 lanes and meet by a warp-shuffle
// butterfly, so a 16-body cluster still occupies the whole CTA.
#include "../../include/nbody.h"
#include "nb_device.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <vector>

namespace nbi {
namespace {

constexpr int kBatchFold = 32;  // j per thread between acceleration folds

struct BatchArgs {
  int32_t n_items;        // clusters in this launch's queue
  const int64_t *off;     // cluster offsets (n_clusters + 1)
  const int32_t *order;   // queue -> cluster index
  int *queue;             // work counter (zeroed before the launch)
  double *x, *v, *a, *jk; // FP64 state, (N, 3)
  const double *m;
  double dt;              // shared step (a power of two)
  double idt2, idt3;      // 1 / dt^2, 1 / dt^3 (exact)
  float eps2;
  double G;
  int nsteps;             // steps per launch (>= 1)
  int cap;                // shared-memory record capacity
  int init_only;          // 1: evaluate a, j at the current state only
};

__device__ __forceinline__ void bds_add(float &hi, float &lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

__device__ __forceinline__ void bpredict(const double *x, const double *v, const double *a,
                                         const double *jk, int64_t i, double dt, double xp[3],
                                         double vp[3]) {
  const double h2 = 0.5 * dt, h3 = dt * (1.0 / 3.0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double xc = x[3 * i + c], vc = v[3 * i + c];
    const double ac = a[3 * i + c], jc = jk[3 * i + c];
    xp[c] = xc + dt * (vc + h2 * (ac + h3 * jc));
    vp[c] = vc + dt * (ac + h2 * jc);
  }
}

// The batched kernel keeps its predictor and corrector on the FP64 pipe:
// there the FP32 pipe carries the pair sums of every cluster on the same
// SM, and FP64 work runs beside it, while conversions and split-precision
// arithmetic would compete with it (measured 5-13 % slower).
//
// Coefficients of the Hermite corrector for one shared step dt (a power of
// two: every coefficient is exact).
struct BHermCoef {
  double dt, h2, h3;          // dt, dt/2, dt/3 (predictor)
  double s_da, s_j0, s_jn;    // snap = s_da da + s_j0 j0 + s_jn jn
  double c_da, c_j;           // crackle = c_da da + c_j (j0 + jn)
  double x_s, x_c, v_s, v_c;  // dt^4/24, dt^5/120, dt^3/6, dt^4/24
};

__device__ __forceinline__ BHermCoef bherm_coef(double dt, double idt2, double idt3) {
  BHermCoef K;
  const double dt2 = dt * dt, dt3 = dt2 * dt;
  const double idt = dt * idt2;  // 1/dt
  K.dt = dt;
  K.h2 = 0.5 * dt;
  K.h3 = dt * (1.0 / 3.0);
  K.s_da = -6.0 * idt2;
  K.s_j0 = -4.0 * idt;
  K.s_jn = -2.0 * idt;
  K.c_da = 12.0 * idt3;
  K.c_j = 6.0 * idt2;
  K.x_s = dt2 * dt2 * (1.0 / 24.0);
  K.x_c = dt3 * dt2 * (1.0 / 120.0);
  K.v_s = dt3 * (1.0 / 6.0);
  K.v_c = dt2 * dt2 * (1.0 / 24.0);
  return K;
}

// One component of the Hermite-4 step in FP64: the predictor, snap =
// (-6 da - dt (4 j0 + 2 jn)) / dt^2 and crackle = (12 da + 6 dt (j0 + jn)) /
// dt^3 with da = a0 - an, x1 = x_p + dt^4 snap / 24 + dt^5 crackle / 120,
// v1 = v_p + dt^3 snap / 6 + dt^4 crackle / 24.
__device__ __forceinline__ void bherm_component(const BHermCoef &K, double x0, double v0,
                                                double a0, double j0, double an, double jn,
                                                double &x1, double &v1) {
  const double xp = x0 + K.dt * (v0 + K.h2 * (a0 + K.h3 * j0));
  const double vp = v0 + K.dt * (a0 + K.h2 * j0);
  const double da = a0 - an;
  const double snap = K.s_da * da + (K.s_j0 * j0 + K.s_jn * jn);
  const double crackle = K.c_da * da + K.c_j * (j0 + jn);
  x1 = xp + (K.x_s * snap + K.x_c * crackle);
  v1 = vp + (K.v_s * snap + K.v_c * crackle);
}

template <int PREC, int IPT, int NT, int MASK, int PACK>
__global__ void __launch_bounds__(NT, 2) batched_hermite_kernel(const BatchArgs B) {
  using V = typename std::conditional<PACK != 0, float2, float>::type;
  using O = dev::VOps<V>;
  constexpr int W = O::W;
  static_assert(IPT % W == 0, "packed kernels need an even IPT");
  constexpr int NQ = IPT / W;
  constexpr int NARR = PREC ? 3 : 2;
  extern __shared__ __align__(16) float4 srec[];
  __shared__ int s_item;
  const int tid = threadIdx.x;
  const float eps2 = B.eps2;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(B.queue, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= B.n_items) return;  // uniform
    const int c = B.order[item];
    const int64_t base = B.off[c];
    const int n = static_cast<int>(B.off[c + 1] - base);
    int tpi = 1;
    while (tpi < 32 && (NT / (tpi * 2)) * IPT >= n) tpi *= 2;
    const int ng = NT / tpi;
    const int bi = ng * IPT;
    const int g = tid / tpi;
    const int r = tid % tpi;
    float4 *s_hi = srec;
    float4 *s_lo = srec + B.cap;
    float4 *s_v = srec + (NARR - 1) * B.cap;
    float2 *s_f = reinterpret_cast<float2 *>(srec + NARR * B.cap);  // bi x 6 sums
    const double dt = B.init_only ? 0.0 : B.dt;
    const int nsteps = B.init_only ? 1 : B.nsteps;
    // corrector coefficients of the shared step (dt a power of two: exact;
    // the host gives 1/dt^2, 1/dt^3)
    const BHermCoef K = bherm_coef(dt, B.idt2, B.idt3);

    for (int step = 0; step < nsteps; ++step) {
      for (int p = tid; p < n; p += NT) {
        double xp[3], vp[3];
        bpredict(B.x, B.v, B.a, B.jk, base + p, dt, xp, vp);
        // conversions on the integer pipe (bit-identical to the hardware ones)
        const float hx = dev::d2f_rn(xp[0]);
        const float hy = dev::d2f_rn(xp[1]);
        const float hz = dev::d2f_rn(xp[2]);
        s_hi[p] = make_float4(hx, hy, hz, dev::d2f_rn(B.m[base + p]));
        if (PREC)
          s_lo[p] = make_float4(dev::d2f_rn(xp[0] - dev::f2d(hx)),
                                dev::d2f_rn(xp[1] - dev::f2d(hy)),
                                dev::d2f_rn(xp[2] - dev::f2d(hz)), 0.f);
        s_v[p] = make_float4(dev::d2f_rn(vp[0]), dev::d2f_rn(vp[1]), dev::d2f_rn(vp[2]), 0.f);
      }
      __syncthreads();
      for (int i0 = 0; i0 < n; i0 += bi) {
        // i-data negated, so that every difference is an addition (a - b and
        // a + (-b) round alike); two i-particles per packed FP32x2 lane
        // pair when PACK (per-lane IEEE rounding: the same bits as scalar)
        V nxh[NQ][3], nxl[NQ][3], nvi[NQ][3];
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
          const int i = i0 + g + q * ng;
          const int ii = i < n ? i : 0;
          const float4 h = s_hi[ii];
          const float4 w = s_v[ii];
          const float4 l = PREC ? s_lo[ii] : make_float4(0.f, 0.f, 0.f, 0.f);
          const int qq = q / W, wl = q % W;
          O::set(nxh[qq][0], wl, -h.x); O::set(nxh[qq][1], wl, -h.y); O::set(nxh[qq][2], wl, -h.z);
          O::set(nxl[qq][0], wl, -l.x); O::set(nxl[qq][1], wl, -l.y); O::set(nxl[qq][2], wl, -l.z);
          O::set(nvi[qq][0], wl, -w.x); O::set(nvi[qq][1], wl, -w.y); O::set(nvi[qq][2], wl, -w.z);
        }
        float ah[IPT][3], al[IPT][3];
        V p1[NQ][3], p2[NQ][3];
#pragma unroll
        for (int q = 0; q < IPT; ++q)
#pragma unroll
          for (int k = 0; k < 3; ++k) ah[q][k] = al[q][k] = 0.f;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
          for (int k = 0; k < 3; ++k) p1[q][k] = p2[q][k] = O::bc(0.f);
        const V veps2 = O::bc(eps2);
        for (int j0 = r; j0 < n; j0 += kBatchFold * tpi) {
          const int jend = min(n, j0 + kBatchFold * tpi);
          V pa[NQ][3];
#pragma unroll
          for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int k = 0; k < 3; ++k) pa[q][k] = O::bc(0.f);
          auto pair = [&](int j) {
            const float4 hj = s_hi[j];
            const float4 wj = s_v[j];
            float4 lj = make_float4(0.f, 0.f, 0.f, 0.f);
            if (PREC) lj = s_lo[j];
            const V xj = O::bc(hj.x), yj = O::bc(hj.y), zj = O::bc(hj.z), mj = O::bc(hj.w);
            const V vxj = O::bc(wj.x), vyj = O::bc(wj.y), vzj = O::bc(wj.z);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
              V dx, dy, dz;
              if (PREC) {
                dx = O::add(O::add(xj, nxh[q][0]), O::add(O::bc(lj.x), nxl[q][0]));
                dy = O::add(O::add(yj, nxh[q][1]), O::add(O::bc(lj.y), nxl[q][1]));
                dz = O::add(O::add(zj, nxh[q][2]), O::add(O::bc(lj.z), nxl[q][2]));
              } else {
                dx = O::add(xj, nxh[q][0]);
                dy = O::add(yj, nxh[q][1]);
                dz = O::add(zj, nxh[q][2]);
              }
              const V ux = O::add(vxj, nvi[q][0]);
              const V uy = O::add(vyj, nvi[q][1]);
              const V uz = O::add(vzj, nvi[q][2]);
              const V r2 = O::fma(dx, dx, O::fma(dy, dy, O::fma(dz, dz, veps2)));
              const V rinv = O::template rsq<MASK>(r2);
              // 1/r^2 on the MUFU pipe beside the rsqrt: one FMA-pipe
              // operation less per pair (measured on the 4096-cluster
              // workload: 741 -> 753 G interactions/s in split precision,
              // 908 -> 928 in FP32); the masked (eps = 0) shapes keep
              // rinv * rinv, which is 0 for the self pair
              const V rinv2 = MASK ? O::mul(rinv, rinv) : O::rcp(r2);
              const V mr3 = O::mul(O::mul(mj, rinv), rinv2);
              const V rv = O::fma(dx, ux, O::fma(dy, uy, O::mul(dz, uz)));
              const V cc = O::mul(O::mul(rv, rinv2), mr3);
              pa[q][0] = O::fma(mr3, dx, pa[q][0]);
              pa[q][1] = O::fma(mr3, dy, pa[q][1]);
              pa[q][2] = O::fma(mr3, dz, pa[q][2]);
              p1[q][0] = O::fma(mr3, ux, p1[q][0]);
              p1[q][1] = O::fma(mr3, uy, p1[q][1]);
              p1[q][2] = O::fma(mr3, uz, p1[q][2]);
              p2[q][0] = O::fma(cc, dx, p2[q][0]);
              p2[q][1] = O::fma(cc, dy, p2[q][1]);
              p2[q][2] = O::fma(cc, dz, p2[q][2]);
            }
          };
          if (tpi == 1 && jend - j0 == kBatchFold) {
            // a whole chunk of consecutive j (the large clusters, which
            // carry most of the pairs): a fixed trip count, so the
            // shared-memory reads take immediate offsets
#pragma unroll 8
            for (int jj = 0; jj < kBatchFold; ++jj) pair(j0 + jj);
          } else {
#pragma unroll 4
            for (int j = j0; j < jend; j += tpi) pair(j);
          }
#pragma unroll
          for (int q = 0; q < IPT; ++q)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const float x = O::lane(pa[q / W][k], q % W);
              if (PREC)
                bds_add(ah[q][k], al[q][k], x);
              else
                ah[q][k] += x;
            }
        }
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
          // sums over the tpi threads of an i-particle: split-precision pairs
          // on the FP32 pipe, one FP64 conversion at the end
          float oh[6], ol[6];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            oh[k] = ah[q][k];
            ol[k] = al[q][k];
            oh[3 + k] = fmaf(-3.f, O::lane(p2[q / W][k], q % W), O::lane(p1[q / W][k], q % W));
            ol[3 + k] = 0.f;
          }
          for (int off = 1; off < tpi; off <<= 1)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              const float wh = __shfl_xor_sync(0xffffffffu, oh[k], off);
              const float wl = __shfl_xor_sync(0xffffffffu, ol[k], off);
              dev::ds_add_pair(oh[k], ol[k], wh, wl, oh[k], ol[k]);
            }
          // hand the sums to consecutive threads so that the FP64
          // corrector runs on full warps (an FP64 instruction costs the SM
          // the same whatever the number of active lanes)
          if (r == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) s_f[(g + q * ng) * 6 + k] = make_float2(oh[k], ol[k]);
          }
        }
        __syncthreads();
        for (int t = tid; t < bi; t += NT) {
          const int i = i0 + t;
          if (i >= n) break;
          const int64_t gi = base + i;
          double o[6];
#pragma unroll
          for (int k = 0; k < 6; ++k)
            o[k] = dev::f2d(s_f[t * 6 + k].x) + dev::f2d(s_f[t * 6 + k].y);
          if (B.init_only) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              B.a[3 * gi + k] = B.G * o[k];
              B.jk[3 * gi + k] = B.G * o[3 + k];
            }
          } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              double x1, v1;
              bherm_component(K, B.x[3 * gi + k], B.v[3 * gi + k], B.a[3 * gi + k],
                              B.jk[3 * gi + k], B.G * o[k], B.G * o[3 + k], x1, v1);
              B.x[3 * gi + k] = x1;
              B.v[3 * gi + k] = v1;
              B.a[3 * gi + k] = B.G * o[k];
              B.jk[3 * gi + k] = B.G * o[3 + k];
            }
          }
        }
        __syncthreads();  // s_f is reused by the next i-block
      }
      __syncthreads();
    }
  }
}

// Per-cluster FP64 energy: one CTA per cluster, fixed-order reductions.
__global__ void batched_energy_kernel(int32_t n_clusters, const int64_t *__restrict__ off,
                                      const double *__restrict__ m, const double *__restrict__ x,
                                      const double *__restrict__ v, double G, double eps2,
                                      double *__restrict__ kin, double *__restrict__ pot) {
  __shared__ double sk[256], sw[256];
  const int c = blockIdx.x;
  if (c >= n_clusters) return;
  const int64_t base = off[c];
  const int n = static_cast<int>(off[c + 1] - base);
  double k = 0.0, w = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t gi = base + i;
    const double vx = v[3 * gi], vy = v[3 * gi + 1], vz = v[3 * gi + 2];
    k += 0.5 * m[gi] * (vx * vx + vy * vy + vz * vz);
    double wi = 0.0;
    for (int j = i + 1; j < n; ++j) {
      const int64_t gj = base + j;
      const double dx = x[3 * gj] - x[3 * gi], dy = x[3 * gj + 1] - x[3 * gi + 1],
                   dz = x[3 * gj + 2] - x[3 * gi + 2];
      wi += m[gj] / sqrt(dx * dx + dy * dy + dz * dz + eps2);
    }
    w += m[gi] * wi;
  }
  sk[threadIdx.x] = k;
  sw[threadIdx.x] = w;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sk[threadIdx.x] += sk[threadIdx.x + s];
      sw[threadIdx.x] += sw[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    kin[c] = sk[0];
    pot[c] = -G * sw[0];
  }
}

using BKernel = void (*)(const BatchArgs);
struct BEntry {
  int prec, ipt, threads, mask, pack;
  BKernel fn;
};
#define NB_BV(P, I, T, M) BEntry{P, I, T, M, 0, &batched_hermite_kernel<P, I, T, M, 0>}
#define NB_BVP(P, I, T, M) BEntry{P, I, T, M, 1, &batched_hermite_kernel<P, I, T, M, 1>}
// Index order is part of the tuning interface.
const BEntry kBTable[] = {
    NB_BV(1, 2, 256, 0), NB_BV(1, 1, 256, 0), NB_BV(1, 2, 128, 0), NB_BV(1, 1, 128, 0),
    NB_BV(0, 2, 256, 0), NB_BV(0, 1, 256, 0), NB_BV(0, 2, 128, 0), NB_BV(0, 1, 128, 0),
    NB_BV(1, 2, 256, 1), NB_BV(0, 2, 256, 1),
    // two i-particles per packed FP32x2 instruction (bit-identical to the
    // scalar shape of the same IPT and threads)
    NB_BVP(1, 2, 128, 0), NB_BVP(1, 2, 256, 0), NB_BVP(1, 4, 128, 0),
    NB_BVP(0, 2, 128, 0), NB_BVP(0, 2, 256, 0), NB_BVP(0, 4, 128, 0),
};
constexpr int kNumBVariants = sizeof(kBTable) / sizeof(kBTable[0]);

}  // namespace
}  // namespace nbi

using namespace nbi;

struct nb_batch {
  int32_t n_clusters = 0;
  int64_t n = 0;
  int max_n = 0;
  nb_config cfg{};
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  double *m = nullptr, *x = nullptr, *v = nullptr, *a = nullptr, *jk = nullptr;
  int64_t *off = nullptr;
  int32_t *order = nullptr;   // largest cluster first
  int32_t *ident = nullptr;   // 0..n_clusters-1 (per-cluster launches)
  int *counters = nullptr;
  int n_counters = 0;
  double *ekin = nullptr, *epot = nullptr;
  int variant = -1, steps_per_launch = 1000, grid_cap = 0, use_graph = 1;
  int64_t launches = 0;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_steps = -1;
  int graph_key[4] = {0, 0, 0, 0};
  cudaEvent_t ev = nullptr;
  std::vector<void *> allocs;
};

namespace {

nb_status bfail(nb_status s, const char *msg, cudaError_t e = cudaSuccess) {
  if (e != cudaSuccess)
    return static_cast<nb_status>(
        set_error(e == cudaErrorMemoryAllocation ? NB_ERR_OOM : s, "%s: %s", msg,
                  cudaGetErrorString(e)));
  return static_cast<nb_status>(set_error(s, "%s", msg));
}

#define BCUDA(call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return bfail(NB_ERR_CUDA, #call, e_); \
  } while (0)

int pick_bvariant(const nb_batch *b) {
  if (b->variant >= 0) return b->variant;
  const int mask = eps_masks(b->cfg.eps);
  if (mask) return b->cfg.precision ? 8 : 9;
  return b->cfg.precision ? 0 : 4;
}

size_t bsmem(const BEntry &E, int cap) {
  return static_cast<size_t>(E.prec ? 3 : 2) * cap * sizeof(float4) +
         static_cast<size_t>(E.threads) * E.ipt * 6 * sizeof(float2);
}

int bgrid(nb_batch *b, int v) {
  const BEntry &E = kBTable[v];
  const size_t sm = bsmem(E, b->max_n);
  cudaFuncSetAttribute(E.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
  int per = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, E.fn, E.threads, sm) != cudaSuccess ||
      per < 1)
    per = 1;
  int grid = b->num_sms * per;
  if (b->grid_cap > 0 && b->grid_cap < grid) grid = b->grid_cap;
  return std::min(grid, std::max(1, b->n_clusters));
}

nb_status launch_batch(nb_batch *b, int v, int grid, int32_t n_items, const int32_t *order,
                       int *counter, int nsteps, int init_only) {
  const BEntry &E = kBTable[v];
  BatchArgs A;
  A.n_items = n_items;
  A.off = b->off;
  A.order = order;
  A.queue = counter;
  A.x = b->x;
  A.v = b->v;
  A.a = b->a;
  A.jk = b->jk;
  A.m = b->m;
  A.dt = std::ldexp(1.0, -b->cfg.lev_shared);
  A.idt2 = std::ldexp(1.0, 2 * b->cfg.lev_shared);
  A.idt3 = std::ldexp(1.0, 3 * b->cfg.lev_shared);
  A.eps2 = eps2_f32(b->cfg.eps);
  A.G = b->cfg.G;
  A.nsteps = nsteps;
  A.cap = b->max_n;
  A.init_only = init_only;
  E.fn<<<grid, E.threads, bsmem(E, b->max_n), b->stream>>>(A);
  BCUDA(cudaGetLastError());
  b->launches += 1;
  return NB_OK;
}

nb_status bsync(nb_batch *b) {
  BCUDA(cudaEventRecord(b->ev, b->stream));
  BCUDA(cudaEventSynchronize(b->ev));
  return NB_OK;
}

// Queue the persistent launches for nsteps steps on the stream (variant v
// on `grid` CTAs, both chosen before any stream capture begins).
nb_status queue_persistent(nb_batch *b, int64_t nsteps, int v, int grid) {
  const int S = std::max(1, b->steps_per_launch);
  const int64_t nl = (nsteps + S - 1) / S;
  if (nl > b->n_counters) return bfail(NB_ERR_INVALID_ARG, "too many launches for the counter array");
  BCUDA(cudaMemsetAsync(b->counters, 0, sizeof(int) * nl, b->stream));
  for (int64_t k = 0; k < nl; ++k) {
    const int s = static_cast<int>(std::min<int64_t>(S, nsteps - k * S));
    nb_status st = launch_batch(b, v, grid, b->n_clusters, b->order, b->counters + k, s, 0);
    if (st != NB_OK) return st;
  }
  return NB_OK;
}

}  // namespace

extern "C" {

nb_status nb_batched_init(nb_batch **out, int32_t n_clusters, const int64_t *offsets,
                          const double *m, const double *x, const double *v,
                          const nb_config *cfg) {
  if (!out) return bfail(NB_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (n_clusters < 1 || !offsets || !m || !x || !v || !cfg)
    return bfail(NB_ERR_INVALID_ARG, "need n_clusters >= 1 and non-null arrays");
  if (offsets[0] != 0) return bfail(NB_ERR_INVALID_ARG, "offsets[0] must be 0");
  int max_n = 0;
  for (int32_t c = 0; c < n_clusters; ++c) {
    const int64_t nc = offsets[c + 1] - offsets[c];
    if (nc < 1 || nc > 4096) return bfail(NB_ERR_INVALID_ARG, "cluster sizes must be in [1, 4096]");
    max_n = std::max<int>(max_n, static_cast<int>(nc));
  }
  const int64_t n = offsets[n_clusters];
  if (cfg->block_steps) return bfail(NB_ERR_INVALID_ARG, "the batched form uses a shared step (block_steps = 0)");
  if (cfg->lev_shared < 0 || cfg->lev_shared > kTicksLog2)
    return bfail(NB_ERR_INVALID_ARG, "need 0 <= lev_shared <= 20");
  if (!(std::isfinite(cfg->eps) && cfg->eps >= 0) || !(std::isfinite(cfg->G) && cfg->G > 0))
    return bfail(NB_ERR_INVALID_ARG, "bad eps or G");
  if (cfg->precision != NB_FP32 && cfg->precision != NB_DS)
    return bfail(NB_ERR_INVALID_ARG, "precision must be NB_FP32 or NB_DS");
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(x[i]) || !std::isfinite(v[i]))
      return bfail(NB_ERR_INVALID_ARG, "non-finite position or velocity");
  for (int64_t i = 0; i < n; ++i)
    if (!(m[i] >= 0)) return bfail(NB_ERR_INVALID_ARG, "negative or non-finite mass");

  nb_batch *b = new (std::nothrow) nb_batch();
  if (!b) return bfail(NB_ERR_OOM, "host memory for the batch");
  b->n_clusters = n_clusters;
  b->n = n;
  b->max_n = max_n;
  b->cfg = *cfg;
  b->stream = static_cast<cudaStream_t>(cfg->stream);
  int dev = 0;
  auto cleanup = [&](nb_status s) {
    nb_batched_destroy(b);
    return s;
  };
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cleanup(bfail(NB_ERR_CUDA, "no CUDA device"));
  auto alloc = [&](void **p, size_t bytes) -> nb_status {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      *p = nullptr;
      return bfail(NB_ERR_CUDA, "cudaMalloc", e);
    }
    try {
      b->allocs.push_back(*p);
    } catch (...) {  // no C++ exception leaves the library
      cudaFree(*p);
      *p = nullptr;
      return bfail(NB_ERR_OOM, "host memory for the allocation list");
    }
    return NB_OK;
  };
  const size_t n3 = 3 * static_cast<size_t>(n) * sizeof(double);
  b->n_counters = std::max(1024, n_clusters);
  nb_status st = NB_OK;
  if ((st = alloc(reinterpret_cast<void **>(&b->m), n * sizeof(double))) ||
      (st = alloc(reinterpret_cast<void **>(&b->x), n3)) ||
      (st = alloc(reinterpret_cast<void **>(&b->v), n3)) ||
      (st = alloc(reinterpret_cast<void **>(&b->a), n3)) ||
      (st = alloc(reinterpret_cast<void **>(&b->jk), n3)) ||
      (st = alloc(reinterpret_cast<void **>(&b->off), (n_clusters + 1) * sizeof(int64_t))) ||
      (st = alloc(reinterpret_cast<void **>(&b->order), n_clusters * sizeof(int32_t))) ||
      (st = alloc(reinterpret_cast<void **>(&b->ident), n_clusters * sizeof(int32_t))) ||
      (st = alloc(reinterpret_cast<void **>(&b->counters), b->n_counters * sizeof(int))) ||
      (st = alloc(reinterpret_cast<void **>(&b->ekin), n_clusters * sizeof(double))) ||
      (st = alloc(reinterpret_cast<void **>(&b->epot), n_clusters * sizeof(double))))
    return cleanup(st);
  if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(bfail(NB_ERR_CUDA, "event creation failed"));
  // processing order: largest cost (n^2) first, ties by index
  std::vector<int32_t> order, ident;
  try {
    order.resize(n_clusters);
    ident.resize(n_clusters);
  } catch (...) {
    return cleanup(bfail(NB_ERR_OOM, "host memory for the processing order"));
  }
  std::iota(order.begin(), order.end(), 0);
  std::iota(ident.begin(), ident.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t p, int32_t q) {
    return (offsets[p + 1] - offsets[p]) > (offsets[q + 1] - offsets[q]);
  });
  cudaStream_t s = b->stream;
  if (cudaMemcpyAsync(b->m, m, n * sizeof(double), cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(b->x, x, n3, cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(b->v, v, n3, cudaMemcpyHostToDevice, s) ||
      cudaMemsetAsync(b->a, 0, n3, s) || cudaMemsetAsync(b->jk, 0, n3, s) ||
      cudaMemcpyAsync(b->off, offsets, (n_clusters + 1) * sizeof(int64_t),
                      cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(b->order, order.data(), n_clusters * sizeof(int32_t),
                      cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(b->ident, ident.data(), n_clusters * sizeof(int32_t),
                      cudaMemcpyHostToDevice, s) ||
      cudaMemsetAsync(b->counters, 0, b->n_counters * sizeof(int), s))
    return cleanup(bfail(NB_ERR_CUDA, "initial copies failed"));
  const int vv = pick_bvariant(b);
  st = launch_batch(b, vv, bgrid(b, vv), n_clusters, b->order, b->counters, 1, 1);
  if (st != NB_OK) return cleanup(st);
  st = bsync(b);
  if (st != NB_OK) return cleanup(st);
  *out = b;
  return NB_OK;
}

void nb_batched_destroy(nb_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void *p : b->allocs)
    if (p) cudaFree(p);
  if (b->ev) cudaEventDestroy(b->ev);
  delete b;
}

nb_status nb_batched_set_tuning(nb_batch *b, int32_t variant, int32_t steps_per_launch,
                                int32_t grid_ctas, int32_t use_graph) {
  if (!b) return bfail(NB_ERR_INVALID_ARG, "null batch");
  if (variant >= kNumBVariants || variant < -1)
    return bfail(NB_ERR_INVALID_ARG, "unknown batched variant");
  if (variant >= 0) {
    const BEntry &E = kBTable[variant];
    if (E.prec != b->cfg.precision || E.mask != eps_masks(b->cfg.eps))
      return bfail(NB_ERR_INVALID_ARG, "variant precision or eps == 0 masking differs from the batch");
  }
  if (steps_per_launch < 1) return bfail(NB_ERR_INVALID_ARG, "steps_per_launch must be >= 1");
  b->variant = variant;
  b->steps_per_launch = steps_per_launch;
  b->grid_cap = grid_ctas > 0 ? grid_ctas : 0;
  b->use_graph = use_graph ? 1 : 0;
  return NB_OK;
}

nb_status nb_batched_variant_info(int32_t v, int32_t *precision, int32_t *ipt, int32_t *threads,
                                  int32_t *packed) {
  if (v < 0 || v >= kNumBVariants) return bfail(NB_ERR_INVALID_ARG, "unknown batched variant");
  if (precision) *precision = kBTable[v].prec;
  if (ipt) *ipt = kBTable[v].ipt;
  if (threads) *threads = kBTable[v].threads;
  if (packed) *packed = kBTable[v].pack;
  return NB_OK;
}

nb_status nb_batched_run(nb_batch *b, int64_t nsteps) {
  if (!b) return bfail(NB_ERR_INVALID_ARG, "null batch");
  if (nsteps < 0) return bfail(NB_ERR_INVALID_ARG, "negative step count");
  if (nsteps == 0) return NB_OK;
  const int v = pick_bvariant(b);
  const int grid = bgrid(b, v);
  if (!b->use_graph) return queue_persistent(b, nsteps, v, grid);
  const int key[4] = {v, b->steps_per_launch, b->grid_cap, grid};
  if (!b->graph || b->graph_steps != nsteps || std::memcmp(key, b->graph_key, sizeof(key)) != 0) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    // Capture on a private stream so that capture never interferes with
    // work another caller queued on the context stream.
    cudaStream_t cs;
    BCUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = b->stream;
    b->stream = cs;
    const int64_t l0 = b->launches;
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    nb_status st = e == cudaSuccess ? queue_persistent(b, nsteps, v, grid) : NB_ERR_CUDA;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    b->stream = saved;
    b->launches = l0;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || e2 != cudaSuccess || st != NB_OK)
      return bfail(NB_ERR_CUDA, "graph capture failed", e != cudaSuccess ? e : e2);
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(NB_ERR_CUDA, "graph instantiation failed", e);
    b->graph_steps = nsteps;
    std::memcpy(b->graph_key, key, sizeof(key));
  }
  BCUDA(cudaGraphLaunch(b->graph, b->stream));
  b->launches += (nsteps + b->steps_per_launch - 1) / b->steps_per_launch;
  return NB_OK;
}

nb_status nb_batched_run_per_cluster(nb_batch *b, int64_t nsteps) {
  if (!b) return bfail(NB_ERR_INVALID_ARG, "null batch");
  if (nsteps < 0) return bfail(NB_ERR_INVALID_ARG, "negative step count");
  const int v = pick_bvariant(b);
  (void)bgrid(b, v);  // sets the kernel's shared-memory attribute
  const int S = std::max(1, b->steps_per_launch);
  for (int64_t k = 0; k * S < nsteps; ++k) {
    const int s = static_cast<int>(std::min<int64_t>(S, nsteps - k * S));
    BCUDA(cudaMemsetAsync(b->counters, 0, sizeof(int) * b->n_clusters, b->stream));
    for (int32_t c = 0; c < b->n_clusters; ++c) {
      nb_status st = launch_batch(b, v, 1, 1, b->ident + c, b->counters + c, s, 0);
      if (st != NB_OK) return st;
    }
  }
  return NB_OK;
}

nb_status nb_batched_energy(nb_batch *b, double *kin, double *pot) {
  if (!b) return bfail(NB_ERR_INVALID_ARG, "null batch");
  batched_energy_kernel<<<b->n_clusters, 256, 0, b->stream>>>(
      b->n_clusters, b->off, b->m, b->x, b->v, b->cfg.G, b->cfg.eps * b->cfg.eps, b->ekin,
      b->epot);
  BCUDA(cudaGetLastError());
  b->launches += 1;
  if (kin)
    BCUDA(cudaMemcpyAsync(kin, b->ekin, b->n_clusters * sizeof(double), cudaMemcpyDeviceToHost,
                          b->stream));
  if (pot)
    BCUDA(cudaMemcpyAsync(pot, b->epot, b->n_clusters * sizeof(double), cudaMemcpyDeviceToHost,
                          b->stream));
  return bsync(b);
}

nb_status nb_batched_get_state(nb_batch *b, double *x, double *v, double *a, double *jerk) {
  if (!b) return bfail(NB_ERR_INVALID_ARG, "null batch");
  const size_t n3 = 3 * static_cast<size_t>(b->n) * sizeof(double);
  if (x) BCUDA(cudaMemcpyAsync(x, b->x, n3, cudaMemcpyDeviceToHost, b->stream));
  if (v) BCUDA(cudaMemcpyAsync(v, b->v, n3, cudaMemcpyDeviceToHost, b->stream));
  if (a) BCUDA(cudaMemcpyAsync(a, b->a, n3, cudaMemcpyDeviceToHost, b->stream));
  if (jerk) BCUDA(cudaMemcpyAsync(jerk, b->jk, n3, cudaMemcpyDeviceToHost, b->stream));
  return bsync(b);
}

nb_status nb_batched_sync(nb_batch *b) {
  if (!b) return bfail(NB_ERR_INVALID_ARG, "null batch");
  return bsync(b);
}

int64_t nb_batched_launch_count(const nb_batch *b) { return b ? b->launches : -1; }

}  // extern "C"
