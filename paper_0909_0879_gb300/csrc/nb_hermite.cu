// O(N) kernels of the Hermite-4 block-step integrator, in FP64 on the GPU:
// predictor (and the j-records it writes for the force kernels), corrector
// with the Aarseth step criterion and power-of-two block quantisation,
// block scheduling (minimum next time and ordered compaction of the active
// list), and the FP64 energy diagnostic.
//
// Sources: predictor / corrector after Makino & Aarseth (1992); time-step
// criterion Aarseth (1985), cited in the paper's Sec. 2; individual (block)
// time steps, paper Sec. 2, strategy (ii).  None of these formulas is
// printed in the paper; they are written out from the standard literature.
#include "nb_internal.cuh"

#include <cfloat>

namespace nbi {

namespace {

constexpr double kTick = 1.0 / static_cast<double>(1 << kTicksLog2);

__device__ __forceinline__ void predict_pos_vel(const double *x, const double *v,
                                                const double *a, const double *jk,
                                                int64_t i, double dt, double xp[3],
                                                double vp[3]) {
  const double h2 = 0.5 * dt, h3 = dt * (1.0 / 3.0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double xc = x[3 * i + c], vc = v[3 * i + c];
    const double ac = a[3 * i + c], jc = jk[3 * i + c];
    // x + dt (v + dt/2 (a + dt/3 j)),  v + dt (a + dt/2 j)
    xp[c] = xc + dt * (vc + h2 * (ac + h3 * jc));
    vp[c] = vc + dt * (ac + h2 * jc);
  }
}

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
    const double dt = static_cast<double>(t_next - t_tick[i]) * kTick;
    double xp[3], vp[3];
    predict_pos_vel(x, v, a, jk, i, dt, xp, vp);
    const float hx = __double2float_rn(xp[0]);
    const float hy = __double2float_rn(xp[1]);
    const float hz = __double2float_rn(xp[2]);
    jhi[i] = make_float4(hx, hy, hz, __double2float_rn(m[i]));
    if (prec)
      jlo[i] = make_float4(__double2float_rn(xp[0] - static_cast<double>(hx)),
                           __double2float_rn(xp[1] - static_cast<double>(hy)),
                           __double2float_rn(xp[2] - static_cast<double>(hz)), 0.f);
    jvel[i] = make_float4(__double2float_rn(vp[0]), __double2float_rn(vp[1]),
                          __double2float_rn(vp[2]), 0.f);
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
  __shared__ float smn[3][kJT / 32], smx[3][kJT / 32];
  __shared__ float4 s_o;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t j = static_cast<int64_t>(blockIdx.x) * kJT + tid;
  const bool real = j < n;
  const float4 h = jhi[j];
  float mn[3], mx[3];
  const float hv[3] = {h.x, h.y, h.z};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    mn[c] = real ? hv[c] : 3.0e38f;
    mx[c] = real ? hv[c] : -3.0e38f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], off));
      mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], off));
    }
    if (lane == 0) {
      smn[c][wid] = mn[c];
      smx[c][wid] = mx[c];
    }
  }
  __syncthreads();
  if (tid == 0) {
    float o[3], hw[3];
    float r2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float a = smn[c][0], b = smx[c][0];
      for (int w = 1; w < kJT / 32; ++w) {
        a = fminf(a, smn[c][w]);
        b = fmaxf(b, smx[c][w]);
      }
      o[c] = 0.5f * a + 0.5f * b;
      // half-width covering [a, b] about o, the low words (below half an
      // ulp of the high word) and the rounding of o
      const float big = fmaxf(fabsf(a), fabsf(b));
      hw[c] = fmaxf(o[c] - a, b - o[c]) * (1.0f + 1.0e-6f) + big * 1.2e-7f;
      r2 = fmaf(hw[c], hw[c], r2);
    }
    const float R = sqrtf(r2) * (1.0f + 1.0e-6f);
    tinfo[2 * blockIdx.x] = make_float4(o[0], o[1], o[2], R);
    tinfo[2 * blockIdx.x + 1] = make_float4(hw[0], hw[1], hw[2], 0.f);
    s_o = make_float4(o[0], o[1], o[2], 0.f);
  }
  __syncthreads();
  if (real) {
    const float4 l = jlo[j];
    const float4 o = s_o;
    jrel[j] = make_float4((h.x - o.x) + l.x, (h.y - o.y) + l.y, (h.z - o.z) + l.z, h.w);
  } else {
    jrel[j] = make_float4(1.0e15f, 1.0e15f, 1.0e15f, 0.f);
  }
}

__device__ __forceinline__ double norm3(const double u[3]) {
  return sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

// Largest power of two 2^-lev <= dt (frexp is exact), clamped.
__device__ __forceinline__ int level_from_dt(double dt, int lev_min, int lev_max,
                                             int *clamped) {
  if (!(dt > 0.0)) {
    *clamped = 1;
    return lev_max;
  }
  if (isinf(dt)) return lev_min;
  int e;
  frexp(dt, &e);
  int lev = 1 - e;
  if (lev > lev_max) {
    *clamped = 1;
    lev = lev_max;
  }
  if (lev < lev_min) lev = lev_min;
  return lev;
}

// Hermite corrector, step criterion and new level of active particle k.
__device__ __forceinline__ void correct_one(
    int64_t k, const int32_t *__restrict__ act, int64_t t_next, double *__restrict__ x,
    double *__restrict__ v, double *__restrict__ a, double *__restrict__ jk,
    int64_t *__restrict__ t_tick, int32_t *__restrict__ lev, const double *__restrict__ a1,
    const double *__restrict__ j1, double eta, int lev_min, int lev_max, int block_steps,
    unsigned long long *n_clamped) {
  const int64_t i = act[k];
  const double dt = static_cast<double>(t_next - t_tick[i]) * kTick;
  double xp[3], vp[3];
  predict_pos_vel(x, v, a, jk, i, dt, xp, vp);
  const double dt2 = dt * dt, dt3 = dt2 * dt;
  // every step is a power of two, so these reciprocals are exact and the
  // products below equal the quotients bit for bit
  const double idt2 = 1.0 / dt2, idt3 = 1.0 / dt3;
  double a1v[3], j1v[3], a2e[3], a3e[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double a0 = a[3 * i + c], j0 = jk[3 * i + c];
    const double an = a1[3 * k + c], jn = j1[3 * k + c];
    const double da = a0 - an;
    // second and third derivatives of a at the start of the step
    const double snap = (-6.0 * da - dt * (4.0 * j0 + 2.0 * jn)) * idt2;
    const double crackle = (12.0 * da + 6.0 * dt * (j0 + jn)) * idt3;
    x[3 * i + c] = xp[c] + dt2 * dt2 * (snap * (1.0 / 24.0) + dt * crackle * (1.0 / 120.0));
    v[3 * i + c] = vp[c] + dt3 * (snap * (1.0 / 6.0) + dt * crackle * (1.0 / 24.0));
    a[3 * i + c] = an;
    jk[3 * i + c] = jn;
    a1v[c] = an;
    j1v[c] = jn;
    a2e[c] = snap + crackle * dt;
    a3e[c] = crackle;
  }
  t_tick[i] = t_next;
  if (block_steps) {
    const double na = norm3(a1v), nj = norm3(j1v), n2 = norm3(a2e), n3 = norm3(a3e);
    const double dtc = sqrt(eta * (na * n2 + nj * nj) / (nj * n3 + n2 * n2));
    int cl = 0;
    const int want = level_from_dt(dtc, lev_min, lev_max, &cl);
    if (cl) atomicAdd(n_clamped, 1ull);
    const int old = lev[i];
    int nl = old;
    if (want >= old) {
      nl = want;
    } else if (old - 1 >= lev_min) {
      const int64_t period = static_cast<int64_t>(1) << (kTicksLog2 - (old - 1));
      if (t_next % period == 0) nl = old - 1;
    }
    lev[i] = nl;
  }
}

__global__ void correct_kernel(int64_t n_act, const int32_t *__restrict__ act, int64_t t_next,
                               double *__restrict__ x, double *__restrict__ v,
                               double *__restrict__ a, double *__restrict__ jk,
                               int64_t *__restrict__ t_tick, int32_t *__restrict__ lev,
                               const double *__restrict__ a1, const double *__restrict__ j1,
                               double eta, int lev_min, int lev_max, int block_steps,
                               unsigned long long *n_clamped, const int64_t *ctl) {
  if (ctl) {
    t_next = ctl[kCtlTnext];
    n_act = ctl[kCtlNact];
    if (t_next < 0) return;
  }
  for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n_act;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    correct_one(k, act, t_next, x, v, a, jk, t_tick, lev, a1, j1, eta, lev_min, lev_max,
                block_steps, n_clamped);
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
  const double dt0 = eta_start * norm3(av) / norm3(jv);
  int cl = 0;
  lev[i] = level_from_dt(dt0, lev_min, lev_max, &cl);
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
                           cudaStream_t s, const int64_t *ctl) {
  if (n_act <= 0) return cudaSuccess;
  const int tb = 128;
  int64_t nb = (n_act + tb - 1) / tb;
  if (ctl && nb > 1216) nb = 1216;  // grid-stride over a bound on the count
  correct_kernel<<<static_cast<unsigned>(nb), tb, 0, s>>>(
      n_act, act, t_next, x, v, a, jk, t_tick, lev, a1, j1, eta, lev_min, lev_max,
      block_steps, n_clamped, ctl);
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

int64_t energy_scratch_doubles(int64_t n) { return 2 * ((n + kEnThreads - 1) / kEnThreads) + 2; }

cudaError_t launch_energy(int64_t n, const double *m, const double *x, const double *v,
                          double G, double eps, double *red, double *d_out, cudaStream_t s,
                          int *launches) {
  const int64_t nb = (n + kEnThreads - 1) / kEnThreads;
  double *pk = red;
  double *pw = red + nb;
  kinetic_kernel<<<static_cast<unsigned>(nb), kEnThreads, 0, s>>>(n, m, v, pk);
  potential_kernel<<<static_cast<unsigned>(nb), kEnThreads, 0, s>>>(n, m, x, eps * eps, pw);
  final_sum_kernel<<<1, kEnThreads, 0, s>>>(nb, pk, 1.0, d_out, 0);
  final_sum_kernel<<<1, kEnThreads, 0, s>>>(nb, pw, -G, d_out, 1);
  if (launches) *launches += 4;
  return cudaGetLastError();
}

}  // namespace nbi
