// Force + jerk kernels for sm_103a.
//
// What is computed (paper eq. 1, Sec. 2, with the Plummer softening of
// Sec. 3, and its time derivative):
//   a_i = G sum_j m_j d / s^3,  j_i = G sum_j m_j (w / s^3 - 3 (d.w) d / s^5)
//   d = x_j - x_i, w = v_j - v_i, s^2 = |d|^2 + eps^2
// for an active list of i against every j-record.  The i == j term is
// evaluated and is exactly zero when eps > 0 (d = w = 0); the eps == 0
// variants zero it explicitly.
//
// Design (GB300, not the paper's GT200 kernel):
//  * Pair arithmetic on the FP32 pipe with one MUFU reciprocal square root
//    per pair; no tensor cores (the pair sum is not a dense contraction).
//  * Each thread keeps IPT i-particles in registers; every j-record read from
//    shared memory (a broadcast) is reused IPT times.
//  * j-tiles of 256 records are staged in shared memory by the bulk-copy
//    (TMA) engine, cp.async.bulk + mbarrier, three stages deep, one thread
//    issuing.  No cluster multicast.
//  * Split precision ("double-single", after Gaburov, Harfst & Portegies
//    Zwart 2009, cited in the paper's Sec. 4): positions are hi + lo FP32
//    pairs and d = (x_j.hi - x_i.hi) + (x_j.lo - x_i.lo); FP32 partial sums
//    over runs of j (32 per thread for the acceleration in near tiles, a
//    256-record tile for the acceleration in far tiles and for the jerk) are
//    folded into hi + lo accumulators with an error-free two-sum, so the
//    split-precision overhead is per run, not per pair, except for the
//    three extra subtractions per coordinate in near tiles.
//  * Work decomposition: the (i-block, j-tile) space is cut into equal
//    contiguous ranges, one per persistent CTA (a "stream-K" split), so every
//    active-list length fills the GPU evenly.  An i-block whose j-range spans
//    several CTAs gets split-precision (hi, lo) partial sums that a fix-up
//    adds in a fixed order on the FP32 pipe: results are deterministic.
//  * Several threads per i-particle (TPI > 1) split a tile's j-range inside
//    the CTA for short active lists; their split-precision sums meet by a
//    warp-shuffle butterfly (commutative pair additions, identical on every
//    lane).
//  * FP64 only where a value leaves the kernel (the FP64 pipe of this part
//    retires one warp instruction per ~68 cycles per scheduler).
#include "nb_device.cuh"

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <utility>

namespace nbi {

namespace {

// j-records per thread between two folds of the acceleration sums into the
// split-precision accumulators.
constexpr int kFoldChunk = 32;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// 1-D bulk copy global -> shared through the TMA engine; completion is
// signalled on the mbarrier as transaction bytes.  dst, src 16-byte aligned
// and bytes a multiple of 16 (always kJT * 16 here).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src,
                                         uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait: false after kWaitLimit unsuccessful polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase) {
  for (uint32_t it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

// Error-free addition of x into the unevaluated sum hi + lo (two-sum).
__device__ __forceinline__ void ds_add(float &hi, float &lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

using dev::VOps;

// Split-precision accumulators of IPT i-particles: acceleration and jerk,
// high and low words.  In registers, or (SMEM) in shared memory at a
// per-thread slot so that wide IPT shapes keep registers for the pair
// arithmetic; the slots are touched only at folds.
template <int IPT, int NT, bool SMEM>
struct DsAcc;
template <int IPT, int NT>
struct DsAcc<IPT, NT, false> {
  float ah[IPT][3], al[IPT][3], jh[IPT][3], jl[IPT][3];
  __device__ __forceinline__ void init(float *, int) {
#pragma unroll
    for (int q = 0; q < IPT; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) ah[q][c] = al[q][c] = jh[q][c] = jl[q][c] = 0.f;
  }
  __device__ __forceinline__ float &AH(int q, int c) { return ah[q][c]; }
  __device__ __forceinline__ float &AL(int q, int c) { return al[q][c]; }
  __device__ __forceinline__ float &JH(int q, int c) { return jh[q][c]; }
  __device__ __forceinline__ float &JL(int q, int c) { return jl[q][c]; }
};
template <int IPT, int NT>
struct DsAcc<IPT, NT, true> {
  float *b;
  __device__ __forceinline__ void init(float *smem, int tid) {
    b = smem + tid;
#pragma unroll
    for (int k = 0; k < 12 * IPT; ++k) b[k * NT] = 0.f;
  }
  __device__ __forceinline__ float &AH(int q, int c) { return b[(12 * q + c) * NT]; }
  __device__ __forceinline__ float &AL(int q, int c) { return b[(12 * q + 3 + c) * NT]; }
  __device__ __forceinline__ float &JH(int q, int c) { return b[(12 * q + 6 + c) * NT]; }
  __device__ __forceinline__ float &JL(int q, int c) { return b[(12 * q + 9 + c) * NT]; }
};

using dev::owner_of;

// JRK = 0: acceleration only (no velocity records, no jerk sums).
template <int PREC, int IPT, int TPI, int NT, int MASK, int PACK, int SACC, int REL, int JRK>
__global__ void __launch_bounds__(NT, 1)
    force_jerk_kernel(const ForceArgs A, uint64_t U, int P) {
  using V = typename std::conditional<PACK != 0, float2, float>::type;
  using O = VOps<V>;
  constexpr int W = O::W;         // i-particles per packed lane group
  static_assert(IPT % W == 0, "packed kernels need an even IPT");
  constexpr int NQ = IPT / W;     // packed i-groups per thread
  constexpr int NG = NT / TPI;    // i-slots per CTA (per q)
  constexpr int BI = NG * IPT;    // i-particles per i-block
  static_assert(!REL || PREC, "tile-relative coordinates only help the split-precision kernel");
  constexpr int NARR = PREC ? (REL ? 4 : 3) : 2;  // hi, lo, vel, rel
  constexpr int kOffV = PREC ? 2 : 1;             // velocity array within a stage
  constexpr uint32_t kTileBytes = kJT * 16;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4 *sbase = reinterpret_cast<float4 *>(smem_raw);
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ uint32_t s_tile[kStages];  // j-tile in each stage

  const int tid = threadIdx.x;
  const int g = tid / TPI;
  const int r = tid % TPI;
  const int p = blockIdx.x;
  const uint64_t n_jt = static_cast<uint64_t>(A.n_jt);
  int64_t n_i = A.n_i;
  if (A.ctl) {
    // device-resident block step: size the split from the device's count
    n_i = A.ctl[kCtlNact];
    if (n_i < A.lo || n_i >= A.hi || n_i <= 0) return;
    U = dev::udiv(static_cast<uint64_t>(n_i + BI - 1), BI) * n_jt;
    constexpr uint64_t MU = min_units(TPI);
    const uint64_t pmax = (U + MU - 1) / MU;
    P = static_cast<int>(pmax < gridDim.x ? pmax : gridDim.x);
    if (p >= P) return;
  }
  const uint64_t u0 = dev::udiv(U * static_cast<uint64_t>(p), static_cast<uint64_t>(P));
  const uint64_t u1 = dev::udiv(U * static_cast<uint64_t>(p + 1), static_cast<uint64_t>(P));
  if (u0 >= u1) return;  // uniform over the CTA
  const uint64_t nunits = u1 - u0;
  const float eps2 = A.eps2;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();

  // Thread 0 issues the copies of the CTA's s-th unit's j-tile and notes
  // the tile for the other threads, which read it after their wait on the
  // stage's barrier (the arrival below releases the note) instead of each
  // recomputing it (measured at N = 1M: 860 -> 853 ms per evaluation).
  auto issue = [&](uint64_t s_idx) {
    const int st = static_cast<int>(s_idx % kStages);
    const uint64_t jt = dev::umod(u0 + s_idx, n_jt);
    s_tile[st] = static_cast<uint32_t>(jt);
    float4 *dst = sbase + static_cast<size_t>(st) * NARR * kJT;
    mbar_expect_tx(&bars[st], kTileBytes * (JRK ? NARR : NARR - 1));
    bulk_g2s(dst, A.jhi + jt * kJT, kTileBytes, &bars[st]);
    if (PREC) bulk_g2s(dst + kJT, A.jlo + jt * kJT, kTileBytes, &bars[st]);
    if (JRK) bulk_g2s(dst + kOffV * kJT, A.jvel + jt * kJT, kTileBytes, &bars[st]);
    if (REL) bulk_g2s(dst + 3 * kJT, A.jrel + jt * kJT, kTileBytes, &bars[st]);
  };
  if (tid == 0) {
    const uint64_t pre = nunits < kStages ? nunits : kStages;
    for (uint64_t s = 0; s < pre; ++s) issue(s);
  }

  const uint64_t ib_first = dev::udiv(u0, n_jt);
  uint64_t s_idx = 0;
  uint64_t u = u0;
  while (u < u1) {
    const uint64_t ib = dev::udiv(u, n_jt);
    const uint64_t jt0 = u - ib * n_jt;
    const uint64_t seg = (n_jt - jt0) < (u1 - u) ? (n_jt - jt0) : (u1 - u);
    const bool full = (jt0 == 0) && (seg == n_jt);

    // i-particle data, negated so that every difference is an addition
    V nxh[NQ][3], nxl[NQ][3], nvi[NQ][3];
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int64_t k = static_cast<int64_t>(ib) * BI + g + q * NG;
      int64_t i = 0;
      if (k < n_i) i = A.idx ? A.idx[k] : k;
      const float4 h = A.jhi[i];
      const float4 w = JRK ? A.jvel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      float4 l = make_float4(0.f, 0.f, 0.f, 0.f);
      if (PREC) l = A.jlo[i];
      const int qq = q / W, wl = q % W;
      O::set(nxh[qq][0], wl, -h.x); O::set(nxh[qq][1], wl, -h.y); O::set(nxh[qq][2], wl, -h.z);
      O::set(nxl[qq][0], wl, -l.x); O::set(nxl[qq][1], wl, -l.y); O::set(nxl[qq][2], wl, -l.z);
      O::set(nvi[qq][0], wl, -w.x); O::set(nvi[qq][1], wl, -w.y); O::set(nvi[qq][2], wl, -w.z);
    }
    const V veps2 = O::bc(eps2);
    // bounding box of the i-block (tile-relative far-field test)
    float bc_i[3] = {0.f, 0.f, 0.f}, bh_i[3] = {0.f, 0.f, 0.f};
    if (REL) {
      __shared__ float s_mn[3][NT / 32], s_mx[3][NT / 32];
      float mn[3] = {3.0e38f, 3.0e38f, 3.0e38f}, mx[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        const int64_t k = static_cast<int64_t>(ib) * BI + g + q * NG;
        if (k < n_i) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float xv = -O::lane(nxh[q / W][c], q % W);
            mn[c] = fminf(mn[c], xv);
            mx[c] = fmaxf(mx[c], xv);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], off));
          mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], off));
        }
      }
      __syncthreads();  // the previous segment's readers are done
      if ((tid & 31) == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          s_mn[c][tid >> 5] = mn[c];
          s_mx[c][tid >> 5] = mx[c];
        }
      }
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float a = s_mn[c][0], b = s_mx[c][0];
        for (int w = 1; w < NT / 32; ++w) {
          a = fminf(a, s_mn[c][w]);
          b = fmaxf(b, s_mx[c][w]);
        }
        bc_i[c] = 0.5f * a + 0.5f * b;
        const float big = fmaxf(fabsf(a), fabsf(b));
        bh_i[c] = fmaxf(bc_i[c] - a, b - bc_i[c]) * (1.0f + 1.0e-6f) + big * 1.2e-7f;
      }
    }
    DsAcc<IPT, NT, SACC != 0> D;
    D.init(reinterpret_cast<float *>(sbase + static_cast<size_t>(kStages) * NARR * kJT), tid);

    for (uint64_t t = 0; t < seg; ++t, ++s_idx) {
      const int st = static_cast<int>(s_idx % kStages);
      const uint32_t ph = static_cast<uint32_t>((s_idx / kStages) & 1);
      const bool ok = mbar_wait(&bars[st], ph);
      const float4 *sh = sbase + static_cast<size_t>(st) * NARR * kJT;
      const float4 *sl = sh + kJT;
      const float4 *sv = sh + kOffV * kJT;
      const float4 *sr = sh + 3 * kJT;
      // far tile: pair differences from tile-relative FP32 coordinates
      bool fast = false;
      V ndx[NQ][3];
      if (REL) {
        const uint64_t jt = s_tile[st];
        const float4 to = __ldg(&A.tinfo[2 * jt]);
        const float4 th = __ldg(&A.tinfo[2 * jt + 1]);
        const float ox[3] = {to.x, to.y, to.z}, hw[3] = {th.x, th.y, th.z};
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float d = fmaxf(0.f, fabsf(bc_i[c] - ox[c]) - (bh_i[c] + hw[c]));
          d2 = fmaf(d, d, d2);
        }
        const float lim = kRelKappa * to.w * (1.0f + 1.0e-5f);
        fast = d2 >= lim * lim;
        if (fast) {
#pragma unroll
          for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              ndx[q][c] = O::add(O::add(nxh[q][c], O::bc(ox[c])), nxl[q][c]);
        }
      }

      V p1[NQ][3], p2[NQ][3];
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) p1[q][c] = p2[q][c] = O::bc(0.f);

      // The tile is walked in chunks of CHW j-records per thread; the
      // acceleration's FP32 chunk sums are folded into the accumulators after
      // every chunk, the jerk's once per tile (its tolerance is ten times
      // looser).  Near tiles fold every kFoldChunk j: a large close-pair term
      // then only inflates the rounding of the few additions that follow it
      // in its chunk.  A far tile (every pair at least kRelKappa tile radii
      // away) has no such terms and folds once per tile (measured at N = 1M:
      // 881 -> 866 ms per evaluation with the 16-deep unroll, the same
      // sampled errors).
      constexpr int CH = (PREC && kFoldChunk < kJT / TPI) ? kFoldChunk : kJT / TPI;
      // j-loop unroll: 8 for the tile-relative kernel (measured at N = 1M:
      // 848 ms against 851 with 16 and 850 with 32), 4 elsewhere (8 is 3 %
      // slower for the FP32 IPT = 4 shape)
      constexpr int UNR = REL ? 8 : 4;
      auto walk_tile = [&](auto far_tag) {
        constexpr bool FAR = decltype(far_tag)::value;
        constexpr int CHW = FAR ? kJT / TPI : CH;
#pragma unroll 1
      for (int c0 = r; c0 < kJT; c0 += CHW * TPI) {
        V pa[NQ][3];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
          for (int c = 0; c < 3; ++c) pa[q][c] = O::bc(0.f);
#pragma unroll(UNR)
        for (int jj = c0; jj < c0 + CHW * TPI; jj += TPI) {
          float4 hj, lj;
          V vxj, vyj, vzj;
          if (JRK) {
            const float4 wj = sv[jj];
            vxj = O::bc(wj.x);
            vyj = O::bc(wj.y);
            vzj = O::bc(wj.z);
          }
          if (FAR) {
            hj = sr[jj];
          } else {
            hj = sh[jj];
            if (PREC) lj = sl[jj];
          }
          const V xj = O::bc(hj.x), yj = O::bc(hj.y), zj = O::bc(hj.z), mj = O::bc(hj.w);
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            V dx, dy, dz;
            if (FAR) {
              dx = O::add(xj, ndx[q][0]);
              dy = O::add(yj, ndx[q][1]);
              dz = O::add(zj, ndx[q][2]);
            } else if (PREC) {
              dx = O::add(O::add(xj, nxh[q][0]), O::add(O::bc(lj.x), nxl[q][0]));
              dy = O::add(O::add(yj, nxh[q][1]), O::add(O::bc(lj.y), nxl[q][1]));
              dz = O::add(O::add(zj, nxh[q][2]), O::add(O::bc(lj.z), nxl[q][2]));
            } else {
              dx = O::add(xj, nxh[q][0]);
              dy = O::add(yj, nxh[q][1]);
              dz = O::add(zj, nxh[q][2]);
            }
            V ux, uy, uz;
            if (JRK) {
              ux = O::add(vxj, nvi[q][0]);
              uy = O::add(vyj, nvi[q][1]);
              uz = O::add(vzj, nvi[q][2]);
            }
            const V r2 = O::fma(dx, dx, O::fma(dy, dy, O::fma(dz, dz, veps2)));
            const V rinv = O::template rsq<MASK>(r2);
            const V rinv2 = O::mul(rinv, rinv);
            const V mr3 = O::mul(O::mul(mj, rinv), rinv2);
            V cc;
            if (JRK) {
              const V rv = O::fma(dx, ux, O::fma(dy, uy, O::mul(dz, uz)));
              cc = O::mul(O::mul(rv, rinv2), mr3);
            }
            pa[q][0] = O::fma(mr3, dx, pa[q][0]);
            pa[q][1] = O::fma(mr3, dy, pa[q][1]);
            pa[q][2] = O::fma(mr3, dz, pa[q][2]);
            if (JRK) {
              p1[q][0] = O::fma(mr3, ux, p1[q][0]);
              p1[q][1] = O::fma(mr3, uy, p1[q][1]);
              p1[q][2] = O::fma(mr3, uz, p1[q][2]);
              p2[q][0] = O::fma(cc, dx, p2[q][0]);
              p2[q][1] = O::fma(cc, dy, p2[q][1]);
              p2[q][2] = O::fma(cc, dz, p2[q][2]);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < IPT; ++q)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float x = O::lane(pa[q / W][c], q % W);
            if (PREC)
              ds_add(D.AH(q, c), D.AL(q, c), x);
            else
              D.AH(q, c) += x;
          }
      }
      };
      if (REL && fast)
        walk_tile(std::true_type{});
      else
        walk_tile(std::false_type{});
      // fold the tile's jerk partial sums (jerk = p1 - 3 p2)
#pragma unroll
      for (int q = 0; q < (JRK ? IPT : 0); ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float jt =
              fmaf(-3.f, O::lane(p2[q / W][c], q % W), O::lane(p1[q / W][c], q % W));
          if (PREC)
            ds_add(D.JH(q, c), D.JL(q, c), jt);
          else
            D.JH(q, c) += jt;
        }
      if (__syncthreads_or(!ok)) {
        // A copy never arrived: record it, wait (bounded) for the copies
        // still in flight so none lands after exit, and leave.
        if (tid == 0) {
          atomicOr(A.err, kErrWaitTimeout);
          const uint64_t last = (s_idx + kStages < nunits) ? s_idx + kStages : nunits;
          for (uint64_t s2 = s_idx; s2 < last; ++s2)
            (void)mbar_wait(&bars[s2 % kStages], static_cast<uint32_t>((s2 / kStages) & 1));
        }
        return;
      }
      if (tid == 0 && s_idx + kStages < nunits) issue(s_idx + kStages);
    }

    // epilogue: the segment's sums, reduced over the TPI threads of each
    // i-particle in split precision on the FP32 pipe; FP64 results for a
    // whole i-block, split-precision partials otherwise
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      float oh[6], ol[6];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        oh[c] = D.AH(q, c);
        ol[c] = D.AL(q, c);
        oh[3 + c] = JRK ? D.JH(q, c) : 0.f;
        ol[3 + c] = JRK ? D.JL(q, c) : 0.f;
      }
      if (TPI > 1) {
#pragma unroll
        for (int off = 1; off < TPI; off <<= 1)
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const float wh = __shfl_xor_sync(0xffffffffu, oh[c], off);
            const float wl = __shfl_xor_sync(0xffffffffu, ol[c], off);
            dev::ds_add_pair(oh[c], ol[c], wh, wl, oh[c], ol[c]);
          }
      }
      const int kk = g + q * NG;
      const int64_t k = static_cast<int64_t>(ib) * BI + kk;
      if (TPI >= 4 && full) {
        // every thread of the i-particle holds the sums: thread r converts
        // components r, r + TPI, ..., so the FP64 work (whose warp
        // instructions cost the same however few lanes are active) takes
        // one or two rounds instead of six
        if (k < n_i) {
#pragma unroll
          for (int base = 0; base < (JRK ? 6 : 3); base += TPI) {
            const int c = base + r;
            if (c < (JRK ? 6 : 3)) {
              float hh = oh[0], ll = ol[0];
#pragma unroll
              for (int cc = 1; cc < 6; ++cc)
                if (c == cc) {
                  hh = oh[cc];
                  ll = ol[cc];
                }
              const double val = dev::ds_to_double(hh, ll, A.G);
              if (c < 3)
                A.acc[3 * k + c] = val;
              else
                A.jerk[3 * k + c - 3] = val;
            }
          }
        }
      } else if (r == 0 && k < n_i) {
        if (full) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            A.acc[3 * k + c] = dev::ds_to_double(oh[c], ol[c], A.G);
            if (JRK) A.jerk[3 * k + c] = dev::ds_to_double(oh[3 + c], ol[3 + c], A.G);
          }
        } else {
          const int slot = (ib == ib_first) ? 0 : 1;
          float2 *dst = A.part + static_cast<size_t>(p * 2 + slot) * 6 * BI;
#pragma unroll
          for (int c = 0; c < 6; ++c)
            dst[static_cast<size_t>(c) * BI + kk] = make_float2(oh[c], ol[c]);
        }
      }
    }
    u += seg;
  }
}

// Sum the partial segments of every split i-block: one warp per
// i-particle, lanes stride over the CTAs that hold a partial (ascending
// within a lane) and meet by a butterfly; the order is fixed for a given
// grid, so results are deterministic.  jerk may be null (acceleration only).
__global__ void force_fixup_kernel(const float2 *__restrict__ part, int64_t n_i,
                                   uint64_t n_jt, uint64_t U, int P, int BI,
                                   double G, double *__restrict__ acc,
                                   double *__restrict__ jerk, const int64_t *ctl,
                                   int64_t lo, int64_t hi, int mu) {
  const int lane = threadIdx.x & 31;
  const int64_t k = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (ctl) {
    // P arrives as the force kernel's grid; derive the split as it did
    n_i = ctl[kCtlNact];
    if (n_i < lo || n_i >= hi || n_i <= 0) return;
    U = dev::udiv(static_cast<uint64_t>(n_i + BI - 1), BI) * n_jt;
    const uint64_t pmax = (U + mu - 1) / mu;
    if (pmax < static_cast<uint64_t>(P)) P = static_cast<int>(pmax);
  }
  if (k >= n_i) return;  // uniform per warp
  const uint64_t ib = dev::udiv(static_cast<uint64_t>(k), BI);
  const int kk = static_cast<int>(static_cast<uint64_t>(k) - ib * BI);
  const int plo = owner_of(ib * n_jt, U, P);
  const int phi = owner_of((ib + 1) * n_jt - 1, U, P);
  if (plo == phi) return;  // written directly by its only CTA
  float h[6], l[6];
  dev::fixup_warp(part, ib, kk, plo, phi, U, P, n_jt, BI, lane, h, l);
  // Every lane holds the six sums: lane c converts component c, so the
  // warp issues one round of FP64 work instead of six (an FP64 warp
  // instruction costs the same however few lanes are active).
  const int nc = jerk ? 6 : 3;
  if (lane < nc) {
    float hh = h[0], ll = l[0];
#pragma unroll
    for (int c = 1; c < 6; ++c)
      if (lane == c) {
        hh = h[c];
        ll = l[c];
      }
    const double val = dev::ds_to_double(hh, ll, G);
    if (lane < 3)
      acc[3 * k + lane] = val;
    else
      jerk[3 * k + lane - 3] = val;
  }
}

using KernelFn = void (*)(const ForceArgs, uint64_t, int);

// fn: acceleration + jerk; acc_fn: acceleration only (compiled for the
// built-in shapes, null elsewhere).
struct Entry {
  Variant V;
  KernelFn fn;
  KernelFn acc_fn;
};

#define NB_V(PREC, IPT, TPI, NT, MASK, PACK)                 \
  Entry{Variant{PREC, IPT, TPI, NT, MASK, PACK, 0, 0},        \
        &force_jerk_kernel<PREC, IPT, TPI, NT, MASK, PACK, 0, 0, 1>, nullptr}
#define NB_VA(PREC, IPT, TPI, NT, MASK, PACK)                \
  Entry{Variant{PREC, IPT, TPI, NT, MASK, PACK, 0, 0},        \
        &force_jerk_kernel<PREC, IPT, TPI, NT, MASK, PACK, 0, 0, 1>, \
        &force_jerk_kernel<PREC, IPT, TPI, NT, MASK, PACK, 0, 0, 0>}
#define NB_VS(PREC, IPT, TPI, NT, MASK, PACK)                \
  Entry{Variant{PREC, IPT, TPI, NT, MASK, PACK, 1, 0},        \
        &force_jerk_kernel<PREC, IPT, TPI, NT, MASK, PACK, 1, 0, 1>, nullptr}
#define NB_VR(PREC, IPT, TPI, NT, MASK, PACK)                \
  Entry{Variant{PREC, IPT, TPI, NT, MASK, PACK, 0, 1},        \
        &force_jerk_kernel<PREC, IPT, TPI, NT, MASK, PACK, 0, 1, 1>, nullptr}
#define NB_VRA(PREC, IPT, TPI, NT, MASK, PACK)               \
  Entry{Variant{PREC, IPT, TPI, NT, MASK, PACK, 0, 1},        \
        &force_jerk_kernel<PREC, IPT, TPI, NT, MASK, PACK, 0, 1, 1>, \
        &force_jerk_kernel<PREC, IPT, TPI, NT, MASK, PACK, 0, 1, 0>}

// The compiled shape table.  Index order is part of the tuning interface.
const Entry kTable[] = {
    NB_V(1, 4, 1, 256, 0, 0),   // 0  DS, long lists
    NB_V(1, 2, 1, 256, 0, 0),   // 1
    NB_V(1, 1, 1, 256, 0, 0),   // 2
    NB_V(1, 1, 4, 256, 0, 0),   // 3  DS, short lists
    NB_VA(1, 1, 16, 256, 0, 0), // 4
    NB_V(0, 4, 1, 256, 0, 0),   // 5  FP32, long lists
    NB_V(0, 2, 1, 256, 0, 0),   // 6
    NB_V(0, 1, 1, 256, 0, 0),   // 7
    NB_VA(0, 1, 4, 256, 0, 0),  // 8  FP32, short lists
    NB_VA(0, 1, 16, 256, 0, 0), // 9
    NB_VA(1, 1, 1, 256, 1, 0),  // 10 DS, eps == 0
    NB_VA(0, 1, 1, 256, 1, 0),  // 11 FP32, eps == 0
    NB_V(1, 4, 1, 256, 0, 1),   // 12 DS, packed pairs of i
    NB_V(1, 2, 1, 256, 0, 1),   // 13
    NB_VA(0, 4, 1, 256, 0, 1),  // 14 FP32, packed pairs of i
    NB_V(0, 2, 1, 256, 0, 1),   // 15
    NB_VA(1, 2, 4, 256, 0, 1),  // 16 DS, packed, short lists
    NB_V(1, 2, 1, 128, 0, 1),   // 17 DS, packed, 128 threads
    NB_V(1, 4, 1, 384, 0, 1),   // 18 DS, packed, 12 warps per CTA
    NB_V(1, 4, 2, 384, 0, 1),   // 19
    NB_V(0, 4, 1, 384, 0, 1),   // 20 FP32, packed, 12 warps per CTA
    NB_V(0, 4, 2, 384, 0, 1),   // 21
    NB_VS(1, 4, 1, 256, 0, 1),  // 22 DS, packed, accumulators in shared memory
    NB_VS(1, 8, 1, 256, 0, 1),  // 23 DS, packed, 8 i-particles per thread
    NB_VS(1, 6, 1, 256, 0, 1),  // 24
    NB_VS(0, 8, 1, 256, 0, 1),  // 25 FP32, packed, 8 i-particles per thread
    NB_VRA(1, 4, 1, 256, 0, 1), // 26 DS, packed, far tiles tile-relative
    NB_VR(1, 2, 1, 256, 0, 1),  // 27
    NB_VR(1, 2, 4, 256, 0, 1),  // 28
    NB_VA(0, 8, 1, 256, 0, 1),  // 29 FP32, packed, 8 i-particles per thread
    NB_VA(1, 1, 32, 512, 0, 0), // 30 DS, short lists, a warp per i-particle
    NB_VA(0, 1, 32, 512, 0, 0), // 31 FP32, short lists, a warp per i-particle
};
constexpr int kNumVariants = sizeof(kTable) / sizeof(kTable[0]);

size_t smem_bytes(const Variant &V) {
  return static_cast<size_t>(kStages) * (V.prec ? (V.rel ? 4 : 3) : 2) * kJT * sizeof(float4) +
         (V.sacc ? static_cast<size_t>(12) * V.ipt * V.threads * sizeof(float) : 0);
}

std::mutex g_occ_mu;
int g_occ[kNumVariants] = {0};
bool g_acc_attr[kNumVariants] = {false};

}  // namespace

int num_variants() { return kNumVariants; }
const Variant &variant_at(int v) { return kTable[v].V; }
int block_i(const Variant &V) { return V.threads / V.tpi * V.ipt; }

ShapeBuckets shape_buckets(int prec, int mask, int64_t n_jt, int num_sms) {
  // Built-in choice from timings on a GB300 (N = 1M King, every shape):
  // packed FP32x2 variants for long lists (split precision with the
  // tile-relative far field, which costs ~1% when particles are not stored
  // in a spatial order and gains ~4-8% when they are; FP32 with IPT = 4,
  // 3-4% faster than IPT = 2 at every active fraction from 2^-10 to 1),
  // more threads per i-particle as the list shortens (the shortest lists a
  // warp per i-particle in 512-thread CTAs: twice the warps of the
  // 256-thread, 16-per-particle shape on the same 16-particle i-blocks,
  // N = 65,536 block steps 136.4 -> 141.0 G interactions/s in FP32 and
  // N = 1024 shared steps 50.3 -> 53.8 in DS).  The host-driven and
  // the device-resident steps use the same buckets.  nb_set_force_table
  // overrides the choice per workload.
  ShapeBuckets b{};
  if (mask) {
    b.nbk = 1;
    b.lo[0] = 1;
    b.v[0] = prec ? 10 : 11;
    return b;
  }
  const int vs[3] = {prec ? 30 : 31, prec ? 16 : 8, prec ? 26 : 14};
  const int64_t base[3] = {1, kBucketMid, kBucketLong};
  // i-blocks a shape needs so that every SM gets min_units units (a small
  // N has few j-tiles: N = 1024 is 4, and one 1024-particle i-block would
  // then run on a single CTA)
  b.nbk = 3;
  for (int k = 0; k < 3; ++k) {
    const int64_t need = min_units(kTable[vs[k]].V.tpi) * static_cast<int64_t>(num_sms);
    const int64_t blocks = (need + n_jt - 1) / n_jt;
    const int64_t fill = (blocks - 1) * block_i(kTable[vs[k]].V) + 1;
    b.lo[k] = k == 0 ? 1 : std::max(base[k], fill);
    if (k > 0 && b.lo[k] < b.lo[k - 1]) b.lo[k] = b.lo[k - 1];
    b.v[k] = vs[k];
  }
  return b;
}

int choose_variant(int prec, int mask, int64_t n_i, int64_t n_jt, int num_sms) {
  const ShapeBuckets b = shape_buckets(prec, mask, n_jt, num_sms);
  int v = b.v[0];
  for (int k = 0; k < b.nbk; ++k)
    if (n_i >= b.lo[k]) v = b.v[k];
  return v;
}

int ctas_per_sm(int v) {
  std::lock_guard<std::mutex> lk(g_occ_mu);
  if (g_occ[v] == 0) {
    int nb = 0;
    const Variant &V = kTable[v].V;
    cudaFuncSetAttribute(kTable[v].fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem_bytes(V)));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, kTable[v].fn, V.threads, smem_bytes(V)) != cudaSuccess ||
        nb < 1)
      nb = 1;
    g_occ[v] = nb;
  }
  return g_occ[v];
}

size_t part_bytes(int v, int grid) {
  return static_cast<size_t>(grid) * 2 * 6 * block_i(kTable[v].V) * sizeof(float2);
}

int force_grid(int v, int64_t n_i, int64_t n_jt, int num_sms, int grid_cap) {
  const Variant &V = kTable[v].V;
  const int64_t BI = block_i(V);
  const int64_t n_ib = (n_i + BI - 1) / BI;
  const int64_t U = n_ib * n_jt;
  int64_t P = static_cast<int64_t>(num_sms) * ctas_per_sm(v);
  if (grid_cap > 0 && grid_cap < P) P = grid_cap;
  // at least min_units j-tiles per CTA
  const int64_t mu = min_units(V.tpi);
  if ((U + mu - 1) / mu < P) P = (U + mu - 1) / mu;
  return static_cast<int>(P < 1 ? 1 : P);
}

cudaError_t launch_force_dev(int v, const ForceArgs &A, int grid, int64_t n_max,
                             cudaStream_t s, int *launches, bool with_fixup) {
  const Entry &E = kTable[v];
  const int BI = block_i(E.V);
  E.fn<<<grid, E.V.threads, smem_bytes(E.V), s>>>(A, 0, grid);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!with_fixup) {
    if (launches) *launches += 1;
    return cudaSuccess;
  }
  const int64_t cap = A.hi < n_max ? A.hi : n_max;
  const int64_t nb = (cap + 7) / 8;
  force_fixup_kernel<<<static_cast<unsigned>(nb > 0 ? nb : 1), 256, 0, s>>>(
      A.part, 0, static_cast<uint64_t>(A.n_jt), 0, grid, BI, A.G, A.acc, A.jerk, A.ctl, A.lo,
      A.hi, static_cast<int>(min_units(E.V.tpi)));
  if (launches) *launches += 2;
  return cudaGetLastError();
}

bool has_acc_only(int v) { return kTable[v].acc_fn != nullptr; }

// Without the jerk the FP32 long-list shape has registers for 8 i-particles
// per thread, which measured 6-7 % faster than 4 (uniform sphere, N =
// 65,536 and 262,144: 1.575 / 24.19 ms per evaluation against 1.680 /
// 25.86); in split precision 8 was 2 % faster in generation order and 2-4 %
// slower in a spatial order, so those keep the jerk kernel's shape.
int acc_shape(int v) { return v == 14 ? 29 : v; }

cudaError_t launch_force(int v, const ForceArgs &A, int grid, cudaStream_t s,
                         int *launches) {
  const Entry &E = kTable[v];
  const KernelFn fn = A.jerk ? E.fn : E.acc_fn;
  if (!fn) return cudaErrorInvalidValue;
  const int BI = block_i(E.V);
  const uint64_t n_ib = static_cast<uint64_t>((A.n_i + BI - 1) / BI);
  const uint64_t U = n_ib * static_cast<uint64_t>(A.n_jt);
  if (!A.jerk) {
    // same shared-memory layout as the jerk kernel (the velocity stage is
    // left unused); the attribute is set once, at the first launch
    std::lock_guard<std::mutex> lk(g_occ_mu);
    if (!g_acc_attr[v]) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem_bytes(E.V)));
      if (e != cudaSuccess) return e;
      g_acc_attr[v] = true;
    }
  }
  fn<<<grid, E.V.threads, smem_bytes(E.V), s>>>(A, U, grid);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int nl = 1;
  // Split i-blocks exist unless every CTA range is whole i-blocks.
  if (!(U % static_cast<uint64_t>(grid) == 0 &&
        (U / grid) % static_cast<uint64_t>(A.n_jt) == 0)) {
    const int tb = 256;  // 8 warps, one i-particle each
    const int64_t nb = (A.n_i + 7) / 8;
    force_fixup_kernel<<<static_cast<unsigned>(nb), tb, 0, s>>>(
        A.part, A.n_i, static_cast<uint64_t>(A.n_jt), U, grid, BI, A.G, A.acc,
        A.jerk, nullptr, 0, 0, 4);
    e = cudaGetLastError();
    ++nl;
  }
  if (launches) *launches += nl;
  return e;
}

}  // namespace nbi
