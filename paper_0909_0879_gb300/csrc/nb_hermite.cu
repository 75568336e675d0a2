// O(N) kernels of the Hermite-4 block-step integrator on the GPU: predictor
// of the j-records (split precision on the FP32 pipe), FP64 corrector
// with the Aarseth step criterion and power-of-two block quantisation,
// block scheduling (minimum next time and ordered compaction of the active
// list), and the FP64 energy diagnostic.
//
// Sources: predictor / corrector after Makino & Aarseth (1992); time-step
// criterion Aarseth (1985), cited in the paper's Sec. 2; individual (block)
// time steps, paper Sec. 2, strategy (ii).  None of these formulas is
// printed in the paper; they are written out from the standard literature.
#include "nb_device.cuh"

#include <cfloat>

namespace nbi {

namespace {

using dev::kTick;

__global__ void predict_kernel(int64_t n, int64_t t_next, const double *__restrict__ x,
                               const double *__restrict__ v, const double *__restrict__ a,
                               const double *__restrict__ jk, const double *__restrict__ m,
                               const int64_t *__restrict__ t_tick, int prec,
                               float4 *__restrict__ jhi, float4 *__restrict__ jlo,
                               float4 *__restrict__ jvel, const int64_t *ctl) {
  if (ctl) {
    t_next = ctl[kCtlTnext];
    if (t_next < 0) return;
  }
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float dt = static_cast<float>(t_next - t_tick[i]) * static_cast<float>(kTick);
    float xh[3], xl[3], vp[3];
    dev::predict_ds(x, v, a, jk, i, dt, xh, xl, vp);
    float4 lo;
    dev::store_records_ds(i, xh, xl, vp, m[i], prec, jhi, jlo, jvel, &lo);
  }
}

// Padding records: zero mass far away, so they add exactly zero to every sum.
__global__ void pad_kernel(int64_t n, int64_t n_pad, float4 *jhi, float4 *jlo,
                           float4 *jvel) {
  const int64_t i = n + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  const float far = 1.0e15f;
  jhi[i] = make_float4(far, far, far, 0.f);
  if (jlo) jlo[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  jvel[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// One CTA per tile of kJT records.
__global__ void __launch_bounds__(kJT)
    tile_info_kernel(int64_t n, const float4 *__restrict__ jhi, const float4 *__restrict__ jlo,
                     float4 *__restrict__ jrel, float4 *__restrict__ tinfo,
                     const int64_t *ctl) {
  if (ctl && ctl[kCtlTnext] < 0) return;
  const int64_t j = static_cast<int64_t>(blockIdx.x) * kJT + threadIdx.x;
  const bool real = j < n;
  const float4 h = jhi[j];
  const float4 l = real ? jlo[j] : make_float4(0.f, 0.f, 0.f, 0.f);
  dev::tile_frame(blockIdx.x, j, real, h, l, jrel, tinfo);
}

__global__ void correct_kernel(int64_t n_act, const int32_t *__restrict__ act, int64_t t_next,
                               double *__restrict__ x, double *__restrict__ v,
                               double *__restrict__ a, double *__restrict__ jk,
                               int64_t *__restrict__ t_tick, int32_t *__restrict__ lev,
                               const double *__restrict__ a1, const double *__restrict__ j1,
                               double eta, int lev_min, int lev_max, int block_steps,
                               unsigned long long *n_clamped, const ExtField E,
                               const int64_t *ctl) {
  if (ctl) {
    t_next = ctl[kCtlTnext];
    n_act = ctl[kCtlNact];
    if (t_next < 0) return;
  }
  for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n_act;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dev::correct_one(k, act, t_next, x, v, a, jk, t_tick, lev, a1, j1, eta, lev_min, lev_max,
                     block_steps, n_clamped, nullptr, &E);
}

// a += sign a_ext(x), jk += sign jerk_ext(x, v) for every particle at its
// own stored position and velocity.
__global__ void ext_adjust_kernel(int64_t n, const ExtField E, double sign,
                                  const double *__restrict__ x, const double *__restrict__ v,
                                  double *__restrict__ a, double *__restrict__ jk) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xv[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  const double vv[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
  double ea[3] = {0.0, 0.0, 0.0}, ej[3] = {0.0, 0.0, 0.0};
  dev::ext_field(E, xv, vv, ea, ej, nullptr);
  for (int c = 0; c < 3; ++c) {
    a[3 * i + c] += sign * ea[c];
    jk[3 * i + c] += sign * ej[c];
  }
}

__global__ void init_levels_kernel(int64_t n, const double *__restrict__ a,
                                   const double *__restrict__ jk, double eta_start,
                                   int lev_min, int lev_max, int block_steps, int lev_shared,
                                   int32_t *__restrict__ lev, int64_t *__restrict__ t_tick) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  t_tick[i] = 0;
  if (!block_steps) {
    lev[i] = lev_shared;
    return;
  }
  const double av[3] = {a[3 * i], a[3 * i + 1], a[3 * i + 2]};
  const double jv[3] = {jk[3 * i], jk[3 * i + 1], jk[3 * i + 2]};
  const double dt0 = eta_start * dev::norm3(av) / dev::norm3(jv);
  int cl = 0;
  lev[i] = dev::level_from_dt(dt0, lev_min, lev_max, &cl);
}

// ---- block scheduling -----------------------------------------------------

constexpr int kSchedThreads = 256;
constexpr int kSchedPerThread = 4;
constexpr int kSchedChunk = kSchedThreads * kSchedPerThread;

__device__ __forceinline__ int64_t due_of(const int64_t *t_tick, const int32_t *lev,
                                          int64_t i) {
  return t_tick[i] + (static_cast<int64_t>(1) << (kTicksLog2 - lev[i]));
}

__global__ void due_min_kernel(int64_t n, const int64_t *__restrict__ t_tick,
                               const int32_t *__restrict__ lev, int64_t *d_scal) {
  __shared__ unsigned long long red[kSchedThreads / 32];
  unsigned long long mn = ~0ull;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long d = static_cast<unsigned long long>(due_of(t_tick, lev, i));
    mn = d < mn ? d : mn;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, mn, off);
    mn = o < mn ? o : mn;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kSchedThreads / 32; ++w) mn = red[w] < mn ? red[w] : mn;
    atomicMin(reinterpret_cast<unsigned long long *>(d_scal), mn);
  }
}

__global__ void due_count_kernel(int64_t n, const int64_t *__restrict__ t_tick,
                                 const int32_t *__restrict__ lev, const int64_t *d_scal,
                                 int32_t *__restrict__ blk_count) {
  __shared__ int red[kSchedThreads / 32];
  const int64_t t_next = d_scal[0];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kSchedChunk;
  int cnt = 0;
  for (int q = 0; q < kSchedPerThread; ++q) {
    const int64_t i = base + q * kSchedThreads + threadIdx.x;
    if (i < n && due_of(t_tick, lev, i) == t_next) ++cnt;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kSchedThreads / 32; ++w) s += red[w];
    blk_count[blockIdx.x] = s;
  }
}

// Exclusive scan of the per-chunk counts in one CTA; total -> d_scal[1].
__global__ void count_scan_kernel(int64_t nblk, int32_t *__restrict__ blk_count,
                                  int64_t *d_scal, int64_t n_total) {
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < nblk; base += blockDim.x) {
    const int64_t b = base + threadIdx.x;
    const int64_t c = b < nblk ? blk_count[b] : 0;
    int64_t incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int64_t o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const int nw = blockDim.x / 32;
      int64_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int64_t o = __shfl_up_sync(0xffffffffu, t, off);
        if (lane >= off) t += o;
      }
      if (lane < nw) warp_tot[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    const int64_t warp_off = wid > 0 ? warp_tot[wid - 1] : 0;
    const int64_t excl = carry + warp_off + incl - c;
    if (b < nblk) blk_count[b] = static_cast<int32_t>(excl);
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + c;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int64_t t_next = d_scal[kCtlTnext];
    if (t_next > d_scal[kCtlTend] || d_scal[kCtlBlocks] >= d_scal[kCtlMaxBlk]) {
      // stop: nothing is due before the end time (or the step budget is
      // spent); the scatter and every later kernel of the step do nothing
      d_scal[kCtlTnext] = -1;
      d_scal[kCtlNact] = 0;
    } else {
      d_scal[kCtlNact] = carry;
      d_scal[kCtlBlocks] += 1;
      d_scal[kCtlInter] += carry * n_total;
      d_scal[kCtlLastT] = t_next;
    }
  }
}

// Ordered compaction: chunk b writes its due indices, ascending, from the
// offset the scan left in blk_count[b].
__global__ void due_scatter_kernel(int64_t n, const int64_t *__restrict__ t_tick,
                                   const int32_t *__restrict__ lev, const int64_t *d_scal,
                                   const int32_t *__restrict__ blk_off,
                                   int32_t *__restrict__ act) {
  __shared__ int wcount[kSchedThreads / 32];
  __shared__ int wbase[kSchedThreads / 32];
  __shared__ int running;
  const int64_t t_next = d_scal[0];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kSchedChunk;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) running = blk_off[blockIdx.x];
  __syncthreads();
  for (int q = 0; q < kSchedPerThread; ++q) {
    const int64_t i = base + q * kSchedThreads + threadIdx.x;
    const bool due = i < n && due_of(t_tick, lev, i) == t_next;
    const unsigned bal = __ballot_sync(0xffffffffu, due);
    if (lane == 0) wcount[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int s = running;
      for (int w = 0; w < kSchedThreads / 32; ++w) {
        wbase[w] = s;
        s += wcount[w];
      }
      running = s;
    }
    __syncthreads();
    if (due) act[wbase[wid] + __popc(bal & ((1u << lane) - 1u))] = static_cast<int32_t>(i);
    __syncthreads();
  }
}

// ---- energy ---------------------------------------------------------------

constexpr int kEnThreads = 256;

// Fixed-order block reduction of one double per thread.
__device__ __forceinline__ double block_sum(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void kinetic_kernel(int64_t n, const double *__restrict__ m,
                               const double *__restrict__ v, double *__restrict__ part) {
  __shared__ double sh[kEnThreads];
  double s = 0.0;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    const double vx = v[3 * i], vy = v[3 * i + 1], vz = v[3 * i + 2];
    s = 0.5 * m[i] * (vx * vx + vy * vy + vz * vz);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// w_i = m_i sum_{j > i} m_j / sqrt(r^2 + eps^2), FP64, j staged in tiles
// from the CTA's own diagonal tile on (each pair once); the block's sum of
// w_i goes to part[blockIdx.x].
__global__ void potential_kernel(int64_t n, const double *__restrict__ m,
                                 const double *__restrict__ x, double eps2,
                                 double *__restrict__ part) {
  __shared__ double sx[kEnThreads], sy[kEnThreads], sz[kEnThreads], sm[kEnThreads];
  __shared__ double sh[kEnThreads];
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * blockDim.x;
  const int64_t i = i0 + threadIdx.x;
  const bool valid = i < n;
  const double xi = valid ? x[3 * i] : 0.0;
  const double yi = valid ? x[3 * i + 1] : 0.0;
  const double zi = valid ? x[3 * i + 2] : 0.0;
  double w = 0.0;
  for (int64_t j0 = i0; j0 < n; j0 += kEnThreads) {
    const int64_t jl = j0 + threadIdx.x;
    if (jl < n) {
      sx[threadIdx.x] = x[3 * jl];
      sy[threadIdx.x] = x[3 * jl + 1];
      sz[threadIdx.x] = x[3 * jl + 2];
      sm[threadIdx.x] = m[jl];
    }
    __syncthreads();
    const int cnt = (n - j0) < kEnThreads ? static_cast<int>(n - j0) : kEnThreads;
    // on the diagonal tile only j > i counts
    const int t0 = (j0 == i0) ? static_cast<int>(threadIdx.x) + 1 : 0;
    for (int t = t0; t < cnt; ++t) {
      const double dx = sx[t] - xi, dy = sy[t] - yi, dz = sz[t] - zi;
      const double s2 = dx * dx + dy * dy + dz * dz + eps2;
      w += sm[t] * rsqrt(s2);
    }
    __syncthreads();
  }
  const double wi = valid ? m[i] * w : 0.0;
  const double s = block_sum(wi, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// One CTA sums part[0..cnt) in a fixed order and writes out[slot].
// e_i = m_i Phi_ext(x_i); the block's sum goes to part[blockIdx.x].
__global__ void ext_potential_kernel(int64_t n, const ExtField E, const double *__restrict__ m,
                                     const double *__restrict__ x, double *__restrict__ part) {
  __shared__ double sh[kEnThreads];
  double s = 0.0;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    const double xv[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    double av[3] = {0.0, 0.0, 0.0}, phi = 0.0;
    dev::ext_field(E, xv, nullptr, av, nullptr, &phi);
    s = m[i] * phi;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void final_sum_kernel(int64_t cnt, const double *__restrict__ part, double scale,
                                 double *__restrict__ out, int slot) {
  __shared__ double sh[kEnThreads];
  double s = 0.0;
  for (int64_t b = threadIdx.x; b < cnt; b += blockDim.x) s += part[b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[slot] = scale * s;
}

}  // namespace

cudaError_t launch_predict(int64_t n, int64_t t_next, const double *x, const double *v,
                           const double *a, const double *jk, const double *m,
                           const int64_t *t_tick, int prec, float4 *jhi, float4 *jlo,
                           float4 *jvel, cudaStream_t s, const int64_t *ctl) {
  const int tb = 256;
  int64_t nb = (n + tb - 1) / tb;
  if (nb > 65535 * 16) nb = 65535 * 16;
  predict_kernel<<<static_cast<unsigned>(nb), tb, 0, s>>>(n, t_next, x, v, a, jk, m, t_tick,
                                                          prec, jhi, jlo, jvel, ctl);
  return cudaGetLastError();
}

cudaError_t launch_tile_info(int64_t n, int64_t n_jt, const float4 *jhi, const float4 *jlo,
                             float4 *jrel, float4 *tinfo, cudaStream_t s, const int64_t *ctl) {
  tile_info_kernel<<<static_cast<unsigned>(n_jt), kJT, 0, s>>>(n, jhi, jlo, jrel, tinfo, ctl);
  return cudaGetLastError();
}

cudaError_t launch_pad_records(int64_t n, int64_t n_pad, float4 *jhi, float4 *jlo,
                               float4 *jvel, cudaStream_t s) {
  if (n_pad <= n) return cudaSuccess;
  const int tb = 256;
  const int64_t nb = (n_pad - n + tb - 1) / tb;
  pad_kernel<<<static_cast<unsigned>(nb), tb, 0, s>>>(n, n_pad, jhi, jlo, jvel);
  return cudaGetLastError();
}

cudaError_t launch_correct(int64_t n_act, const int32_t *act, int64_t t_next, double *x,
                           double *v, double *a, double *jk, int64_t *t_tick, int32_t *lev,
                           const double *a1, const double *j1, double eta, int lev_min,
                           int lev_max, int block_steps, unsigned long long *n_clamped,
                           const ExtField &E, cudaStream_t s, const int64_t *ctl) {
  if (n_act <= 0) return cudaSuccess;
  const int tb = 128;
  int64_t nb = (n_act + tb - 1) / tb;
  if (ctl && nb > 1216) nb = 1216;  // grid-stride over a bound on the count
  correct_kernel<<<static_cast<unsigned>(nb), tb, 0, s>>>(
      n_act, act, t_next, x, v, a, jk, t_tick, lev, a1, j1, eta, lev_min, lev_max,
      block_steps, n_clamped, E, ctl);
  return cudaGetLastError();
}

cudaError_t launch_ext_adjust(int64_t n, const ExtField &E, double sign, const double *x,
                              const double *v, double *a, double *jk, cudaStream_t s) {
  if (n <= 0 || !E.on) return cudaSuccess;
  ext_adjust_kernel<<<static_cast<unsigned>((n + 127) / 128), 128, 0, s>>>(n, E, sign, x, v,
                                                                          a, jk);
  return cudaGetLastError();
}

cudaError_t launch_init_levels(int64_t n, const double *a, const double *jk,
                               double eta_start, int lev_min, int lev_max, int block_steps,
                               int lev_shared, int32_t *lev, int64_t *t_tick,
                               cudaStream_t s) {
  const int tb = 256;
  const int64_t nb = (n + tb - 1) / tb;
  init_levels_kernel<<<static_cast<unsigned>(nb), tb, 0, s>>>(
      n, a, jk, eta_start, lev_min, lev_max, block_steps, lev_shared, lev, t_tick);
  return cudaGetLastError();
}

int64_t next_block_scratch_ints(int64_t n) { return (n + kSchedChunk - 1) / kSchedChunk; }

cudaError_t launch_next_block(int64_t n, const int64_t *t_tick, const int32_t *lev,
                              int32_t *act, int32_t *blk_count, int64_t *d_scal,
                              cudaStream_t s, int *launches) {
  cudaError_t e = cudaMemsetAsync(d_scal, 0xff, sizeof(int64_t), s);
  if (e != cudaSuccess) return e;
  const int64_t nblk = next_block_scratch_ints(n);
  int64_t nb_min = (n + kSchedThreads - 1) / kSchedThreads;
  if (nb_min > 4096) nb_min = 4096;
  due_min_kernel<<<static_cast<unsigned>(nb_min), kSchedThreads, 0, s>>>(n, t_tick, lev,
                                                                          d_scal);
  due_count_kernel<<<static_cast<unsigned>(nblk), kSchedThreads, 0, s>>>(n, t_tick, lev,
                                                                          d_scal, blk_count);
  count_scan_kernel<<<1, 1024, 0, s>>>(nblk, blk_count, d_scal, n);
  due_scatter_kernel<<<static_cast<unsigned>(nblk), kSchedThreads, 0, s>>>(
      n, t_tick, lev, d_scal, blk_count, act);
  if (launches) *launches += 4;
  return cudaGetLastError();
}

int64_t energy_scratch_doubles(int64_t n) { return 3 * ((n + kEnThreads - 1) / kEnThreads) + 3; }

cudaError_t launch_energy(int64_t n, const double *m, const double *x, const double *v,
                          double G, double eps, const ExtField &E, double *red, double *d_out,
                          cudaStream_t s, int *launches) {
  const int64_t nb = (n + kEnThreads - 1) / kEnThreads;
  double *pk = red;
  double *pw = red + nb;
  double *pe = red + 2 * nb;
  kinetic_kernel<<<static_cast<unsigned>(nb), kEnThreads, 0, s>>>(n, m, v, pk);
  potential_kernel<<<static_cast<unsigned>(nb), kEnThreads, 0, s>>>(n, m, x, eps * eps, pw);
  if (E.on) ext_potential_kernel<<<static_cast<unsigned>(nb), kEnThreads, 0, s>>>(n, E, m, x, pe);
  final_sum_kernel<<<1, kEnThreads, 0, s>>>(nb, pk, 1.0, d_out, 0);
  final_sum_kernel<<<1, kEnThreads, 0, s>>>(nb, pw, -G, d_out, 1);
  final_sum_kernel<<<1, kEnThreads, 0, s>>>(E.on ? nb : 0, pe, 1.0, d_out, 2);
  if (launches) *launches += E.on ? 6 : 5;
  return cudaGetLastError();
}

}  // namespace nbi
