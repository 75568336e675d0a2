// Fused device-resident block steps: one block step of the Hermite-4
// integrator with individual power-of-two steps (paper Sec. 2, strategy
// (ii); predictor / corrector after Makino & Aarseth 1992) in three kinds of
// launch instead of a dozen:
//
//   block_begin  scheduling (next block time, ordered active list) and the
//                predictor of every particle's j-records (split precision on
//                the FP32 pipe), with the j-tile frames;
//   force        the force + jerk kernels of nb_force.cu, one launch per
//                active-count bucket (the others return at once);
//   block_end    the fix-up of split i-blocks and the corrector.
//
// Scheduling without a pass over the particles.  The integrator keeps every
// particle's time t_i a multiple of its step dt_i = 2^-lev_i and its next
// time t_i + dt_i after the current block time t (a step shrinks freely and
// grows only when t is a multiple of the doubled step).  Then t_i + dt_i is
// the first multiple of dt_i after t, so the next block time is the first
// multiple of the smallest occupied step after t, and a particle is due
// exactly when its step divides that time: the active set is every particle
// whose level is at least a threshold given by the trailing zeros of t_next.
// The per-level counts live in the control slots, kept up to date by the
// corrector; a check kernel rebuilds them, and verifies the property, before
// device-resident steps start (a state set by the caller that lacks it runs
// the general scheduler instead).
//
// The ordered compaction is a single pass: CTAs take tickets in the order
// they start, publish their tile's active count at once, predict their
// tile, then read the counts before them with a decoupled look-back over
// windows of 256 tiles (bounded waits; a CTA only waits on CTAs that
// started earlier and published before predicting, so every wait ends).
#include "nb_device.cuh"

namespace nbi {

namespace {

using dev::kTick;

// Look-back word: epoch (24 bits) | flag (2 bits) | value (38 bits).
constexpr int kValBits = 38;
constexpr uint64_t kValMask = (uint64_t(1) << kValBits) - 1;
constexpr uint64_t kFlagAgg = 1;  // value = this tile's active count
constexpr uint64_t kFlagPre = 2;  // value = active count of tiles 0..this one
constexpr int64_t kEpochMod = (int64_t(1) << 24) - 1;

__device__ __forceinline__ uint64_t ld_relaxed(const unsigned long long *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t lb_word(uint64_t epoch, uint64_t flag, uint64_t val) {
  return (epoch << 40) | (flag << kValBits) | (val & kValMask);
}

// Exclusive prefix of the active counts of the tiles before `vid`, by the
// whole CTA: each thread reads one predecessor's word of the current window
// of kJT tiles (waiting, bounded, until it is published in this epoch); the
// window's counts are added up to the nearest inclusive prefix, where the
// scan stops, or the next window further back is read.  A window covers
// 256 tiles, so up to N = 65,536 one round of reads suffices.  Returns false
// (on every thread) if a wait ran out.  Called by all threads of the CTA.
__device__ __forceinline__ bool look_back_cta(const unsigned long long *status, int64_t vid,
                                              uint64_t epoch, uint32_t limit,
                                              int64_t *excl_out) {
  __shared__ int64_t s_sum[kJT / 32];
  __shared__ int s_near[kJT / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int64_t excl = 0;
  for (int64_t top = vid - 1; top >= 0; top -= kJT) {
    const int64_t j = top - tid;  // thread 0 reads the nearest predecessor
    uint64_t w = 0;
    bool ready = true;
    if (j >= 0) {
      ready = false;
      for (uint32_t it = 0; it < limit; ++it) {
        w = ld_relaxed(status + j);
        if ((w >> 40) == epoch) {
          ready = true;
          break;
        }
      }
    }
    if (__syncthreads_or(!ready)) return false;
    // nearest inclusive prefix of the window: the smallest such thread
    const bool pre = j >= 0 && ((w >> kValBits) & 3) == kFlagPre;
    const unsigned pm = __ballot_sync(0xffffffffu, pre);
    if (lane == 0) s_near[wid] = pm ? wid * 32 + __ffs(pm) - 1 : kJT;
    __syncthreads();
    int near = kJT;
#pragma unroll
    for (int q = 0; q < kJT / 32; ++q) near = s_near[q] < near ? s_near[q] : near;
    int64_t val = (j >= 0 && tid <= near) ? static_cast<int64_t>(w & kValMask) : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
    if (lane == 0) s_sum[wid] = val;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kJT / 32; ++q) excl += s_sum[q];
    __syncthreads();  // s_sum and s_near are read before the next window
    if (near < kJT) break;
  }
  *excl_out = excl;
  return true;
}

__global__ void __launch_bounds__(kJT, 2) block_begin_kernel(const BeginArgs B) {
  __shared__ unsigned s_vid;
  __shared__ int s_lmax;
  __shared__ int64_t s_ctl[4];  // t_cur, blocks, max blocks, t_end
  __shared__ int64_t s_cnt[kTicksLog2 + 1];
  __shared__ int s_wcnt[kJT / 32];
  __shared__ int64_t s_excl;
  __shared__ int s_agg, s_fail;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int64_t *ctl = B.ctl;
  // Control values that no CTA of this launch writes, so that every CTA
  // takes the same decision; the per-level counts are read a lane each.
  if (wid == 0) {
    const int64_t c = lane <= kTicksLog2 ? ctl[kCtlLevCnt + lane] : 0;
    const unsigned occ = __ballot_sync(0xffffffffu, c > 0);
    if (lane <= kTicksLog2) s_cnt[lane] = c;
    if (lane == 0) {
      s_lmax = occ ? 31 - __clz(occ) : -1;
      s_vid = static_cast<unsigned>(
          atomicAdd(reinterpret_cast<unsigned long long *>(ctl + kCtlTicket), 1ull) %
          gridDim.x);
      s_ctl[0] = ctl[kCtlLastT];
      s_ctl[1] = ctl[kCtlBlocks];
      s_ctl[2] = ctl[kCtlMaxBlk];
      s_ctl[3] = ctl[kCtlTend];
    }
  }
  __syncthreads();
  const int lmax = s_lmax;
  const int64_t blocks = s_ctl[1];
  int64_t t_next = -1;
  bool stop = lmax < 0 || blocks >= s_ctl[2];
  if (!stop) {
    const int64_t step = int64_t(1) << (kTicksLog2 - lmax);
    t_next = (s_ctl[0] / step + 1) * step;
    stop = t_next > s_ctl[3];
  }
  const unsigned vid = s_vid;
  if (stop) {
    if (vid == 0 && tid == 0) {
      ctl[kCtlTnext] = -1;
      ctl[kCtlNact] = 0;
    }
    return;
  }
  // due <=> dt_i divides t_next <=> lev_i >= l_thr
  const int tz = __ffsll(static_cast<long long>(t_next)) - 1;
  const int l_thr = kTicksLog2 - (tz < kTicksLog2 ? tz : kTicksLog2);
  const int64_t i = static_cast<int64_t>(vid) * kJT + tid;
  const bool real = i < B.n;
  // the predictor's inputs, loaded before the ballot and the barrier so
  // that their round trip overlaps the level's
  dev::PSplit S;
  int64_t ti = 0;
  double mi = 0.0;
  if (real) {
    dev::load_split(i, B.sp4, B.sp2, S);
    ti = B.t_tick[i];
    mi = B.m[i];
  }
  const bool due = real && B.lev[i] >= l_thr;
  const unsigned bal = __ballot_sync(0xffffffffu, due);
  if (lane == 0) s_wcnt[wid] = __popc(bal);
  __syncthreads();
  const uint64_t epoch = static_cast<uint64_t>(blocks % kEpochMod) + 1;
  int agg = 0;
  for (int w = 0; w < kJT / 32; ++w) agg += s_wcnt[w];
  // publish this tile's count at once, so that no later CTA waits for it
  if (tid == 0)
    st_relaxed(B.status + vid,
               lb_word(epoch, vid == 0 ? kFlagPre : kFlagAgg, static_cast<uint64_t>(agg)));

  // predictor of this tile's particles (split precision, FP32 pipe, from
  // the state's FP32 split)
  float4 h = make_float4(0.f, 0.f, 0.f, 0.f), lo = h;
  if (real) {
    const float dt = static_cast<float>(t_next - ti) * static_cast<float>(kTick);
    float xh[3], xl[3], vp[3];
    dev::predict_split(S, dt, xh, xl, vp);
    h = dev::store_records_ds(i, xh, xl, vp, mi, B.prec, B.jhi, B.jlo, B.jvel, &lo);
  }
  // Tile frames only for steps whose force shape takes the far field (the
  // active count is the sum of the due levels' counts).
  int64_t n_due = 0;
  for (int l = l_thr; l <= kTicksLog2; ++l) n_due += s_cnt[l];
  if (B.jrel && n_due >= B.rel_lo)
    dev::tile_frame(vid, i, real, h, lo, B.jrel, B.tinfo);  // synchronises the CTA
  else
    __syncthreads();

  // the predecessors' counts were published while this CTA predicted
  int64_t excl = 0;
  const bool ok = look_back_cta(B.status, vid, epoch + B.lb_epoch_skew, B.lb_wait_limit, &excl);
  if (tid == 0) {
    if (!ok)
      atomicOr(reinterpret_cast<int *>(ctl + kCtlErr), kErrScanTimeout);
    else if (vid > 0)
      st_relaxed(B.status + vid, lb_word(epoch, kFlagPre, static_cast<uint64_t>(excl + agg)));
    s_excl = excl;
    s_agg = agg;
    s_fail = ok ? 0 : 1;
  }
  __syncthreads();
  if (!s_fail && due) {
    int base = 0;
    for (int w = 0; w < wid; ++w) base += s_wcnt[w];
    const int64_t pos = s_excl + base + __popc(bal & ((1u << lane) - 1u));
    if (pos < B.n) B.act[pos] = static_cast<int32_t>(i);
  }
  if (tid == 0) {
    if (vid == gridDim.x - 1) ctl[kCtlNact] = s_fail ? 0 : s_excl + s_agg;
    if (vid == 0) ctl[kCtlTnext] = t_next;
  }
}

// Sum of the split partial segments of NQ entries of one warp at once
// (entry e of ib[e], kk[e], held by CTAs plo[e]..phi[e]; use[e] false
// skips it), with the per-entry order of dev::fixup_warp: lanes stride over
// the CTAs in ascending order, then the same butterfly.  Warp-uniform.
template <int NQ>
__device__ __forceinline__ void fixup_warp_n(const float2 *__restrict__ part,
                                             const uint64_t *ib, const int *kk,
                                             const int *plo, const int *phi, const bool *use,
                                             uint64_t U, int P, uint64_t n_jt, int BI,
                                             int lane, float h[][6], float l[][6]) {
  int span = 0;
#pragma unroll
  for (int e = 0; e < NQ; ++e) {
#pragma unroll
    for (int c = 0; c < 6; ++c) h[e][c] = l[e][c] = 0.f;
    if (use[e] && phi[e] - plo[e] + 1 > span) span = phi[e] - plo[e] + 1;
  }
  // A CTA's partial of i-block ib sits in its slot 0 (its first segment)
  // unless ib is the CTA's second segment, which only the first CTA of the
  // i-block can have (every later one starts inside ib): one division per
  // entry instead of two per partial.
  int slot0[NQ];
#pragma unroll
  for (int e = 0; e < NQ; ++e) {
    const uint64_t u0p =
        dev::udiv(U * static_cast<uint64_t>(plo[e]), static_cast<uint64_t>(P));
    slot0[e] = (u0p == ib[e] * n_jt) ? 0 : 1;
  }
  // a single entry loads NB of its lane's partials before adding them (in
  // the same ascending order), so their round trips overlap
  constexpr int NB = NQ == 1 ? 4 : 1;
  for (int o0 = lane; o0 < span; o0 += 32 * NB) {
#pragma unroll
    for (int e = 0; e < NQ; ++e) {
      float2 w[NB][6];
      bool have[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int p = plo[e] + o0 + 32 * b;
        have[b] = use[e] && p <= phi[e];
        if (have[b]) {
          const int slot = p == plo[e] ? slot0[e] : 0;
          const float2 *src = part + static_cast<size_t>(p * 2 + slot) * 6 * BI;
#pragma unroll
          for (int c = 0; c < 6; ++c) w[b][c] = src[static_cast<size_t>(c) * BI + kk[e]];
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (have[b]) {
#pragma unroll
          for (int c = 0; c < 6; ++c)
            dev::ds_add_pair(h[e][c], l[e][c], w[b][c].x, w[b][c].y, h[e][c], l[e][c]);
        }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int e = 0; e < NQ; ++e)
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const float oh = __shfl_xor_sync(0xffffffffu, h[e][c], off);
        const float ol = __shfl_xor_sync(0xffffffffu, l[e][c], off);
        dev::ds_add_pair(h[e][c], l[e][c], oh, ol, h[e][c], l[e][c]);
      }
}

constexpr int kEndWarps = kEndThreads / 32;

// New force of one round's entry as block_end stages it: the fix-up sum of a
// split i-block (converted to FP64 by the fix-up warp's lanes 0..5) or
// nothing (its only CTA wrote the FP64 value to a1, j1).
struct EndStage {
  double f[4 * kEndWarps][6];
  int split[4 * kEndWarps];
};

// One round of block_end over the entries k0 .. k0 + NQ * kEndWarps - 1:
// the warps add the split partial sums of NQ entries each, then warp 0
// corrects the round's entries, a lane each.
template <int NQ>
__device__ __forceinline__ void end_round(const EndArgs &E, int64_t k0, int64_t n_act,
                                          int64_t t_next, int BI, uint64_t U, int P,
                                          EndStage &sg) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t n_jt = static_cast<uint64_t>(E.n_jt);
  uint64_t ib[NQ];
  int kk[NQ], plo[NQ], phi[NQ];
  bool valid[NQ], split[NQ];
#pragma unroll
  for (int e = 0; e < NQ; ++e) {
    const int64_t k = k0 + wid + kEndWarps * e;
    valid[e] = k < n_act;
    const uint64_t kc = valid[e] ? static_cast<uint64_t>(k) : 0;
    ib[e] = dev::udiv(kc, BI);
    kk[e] = static_cast<int>(kc - ib[e] * BI);
    plo[e] = dev::owner_of(ib[e] * n_jt, U, P);
    phi[e] = dev::owner_of((ib[e] + 1) * n_jt - 1, U, P);
    split[e] = valid[e] && plo[e] != phi[e];
  }
  // The corrector runs on three lanes per entry (one per component, ten
  // entries per warp): these lanes load its inputs while the warps add
  // the partial sums.
  constexpr int kRound = NQ * kEndWarps;
  const int eq = lane < 30 ? wid * 10 + lane / 3 : kRound;  // this lane's entry
  const int cq = lane % 3;
  dev::PState st;
  int64_t ci = -1;
  if (eq < kRound && k0 + eq < n_act) {
    ci = E.act[k0 + eq];
    dev::load_state(ci, E.x, E.v, E.a, E.jk, E.t_tick, E.lev, st);
  }
  float h[NQ][6], l[NQ][6];
  fixup_warp_n<NQ>(E.part, ib, kk, plo, phi, split, U, P, n_jt, BI, lane, h, l);
  // every lane holds the sums: lane c converts component c, so the FP64
  // work (whose warp instructions cost the same however few lanes are
  // active) is one round per warp instead of six on the corrector lane
#pragma unroll
  for (int e = 0; e < NQ; ++e) {
    const int q = wid + kEndWarps * e;
    if (lane == 0) sg.split[q] = split[e] ? 1 : 0;
    if (split[e] && lane < 6) {
      float hh = h[e][0], ll = l[e][0];
#pragma unroll
      for (int c = 1; c < 6; ++c)
        if (lane == c) {
          hh = h[e][c];
          ll = l[e][c];
        }
      sg.f[q][lane] = dev::ds_to_double(hh, ll, E.G);
    }
  }
  __syncthreads();
  if (ci >= 0) {
    const int64_t k = k0 + eq;
    double an[3], jn[3];
    if (sg.split[eq]) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        an[c] = sg.f[eq][c];
        jn[c] = sg.f[eq][3 + c];
      }
      E.a1[3 * k + cq] = dev::sel3(an, cq);
      E.j1[3 * k + cq] = dev::sel3(jn, cq);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        an[c] = E.a1[3 * k + c];
        jn[c] = E.j1[3 * k + c];
      }
    }
    // the warp's corrector lanes: whole triples of its valid entries
    int64_t nv = n_act - k0 - static_cast<int64_t>(wid) * 10;
    const int64_t cap = kRound - wid * 10;
    nv = nv < cap ? nv : cap;
    nv = nv < 10 ? nv : 10;
    const unsigned mask = nv >= 10 ? 0x3fffffffu : ((1u << (3 * nv)) - 1u);
    dev::correct_vals3(cq, mask, lane - cq, ci, st, an, jn, t_next, E.x, E.v, E.a, E.jk,
                       E.t_tick, E.lev, E.eta, E.lev_min, E.lev_max, E.block_steps,
                       E.n_clamped, E.ctl + kCtlLevCnt, &E.ext, E.sp4, E.sp2);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kEndThreads) block_end_kernel(const EndArgs E) {
  __shared__ EndStage sg;
  const int64_t t_next = E.ctl[kCtlTnext];
  if (t_next < 0) return;
  const int64_t n_act = E.ctl[kCtlNact];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // reductions without a return value: the thread does not wait for a
    // round trip before its CTA's corrector work
    atomicAdd(reinterpret_cast<unsigned long long *>(E.ctl + kCtlBlocks), 1ull);
    atomicAdd(reinterpret_cast<unsigned long long *>(E.ctl + kCtlInter),
              static_cast<unsigned long long>(n_act * E.n));
    E.ctl[kCtlLastT] = t_next;
  }
  int b = -1;
  for (int q = 0; q < E.nbk; ++q)
    if (n_act >= E.lo[q] && n_act < E.hi[q]) b = q;
  if (b < 0) return;
  // the split the force launch of this bucket derived from the same count
  const int BI = E.bi[b];
  const uint64_t U = dev::udiv(static_cast<uint64_t>(n_act + BI - 1), BI) *
                     static_cast<uint64_t>(E.n_jt);
  const uint64_t mu = static_cast<uint64_t>(E.mu[b]);
  const uint64_t pm = (U + mu - 1) / mu;
  const int P = static_cast<int>(pm < static_cast<uint64_t>(E.pmax[b]) ? pm : E.pmax[b]);
  // short lists: one entry per warp per round (the fix-ups in parallel);
  // long lists: four, so that the corrector warp runs 32 lanes
  if (n_act <= static_cast<int64_t>(kEndWarps) * gridDim.x) {
    for (int64_t k0 = static_cast<int64_t>(blockIdx.x) * kEndWarps; k0 < n_act;
         k0 += static_cast<int64_t>(gridDim.x) * kEndWarps)
      end_round<1>(E, k0, n_act, t_next, BI, U, P, sg);
  } else {
    for (int64_t k0 = static_cast<int64_t>(blockIdx.x) * 4 * kEndWarps; k0 < n_act;
         k0 += static_cast<int64_t>(gridDim.x) * 4 * kEndWarps)
      end_round<4>(E, k0, n_act, t_next, BI, U, P, sg);
  }
}

// ---- check of the level structure ----------------------------------------

constexpr int kChkThreads = 256;

__global__ void __launch_bounds__(kChkThreads)
    sched_levels_kernel(int64_t n, const int64_t *__restrict__ t_tick,
                        const int32_t *__restrict__ lev, int64_t *ctl) {
  __shared__ int cnt[kTicksLog2 + 1];
  __shared__ unsigned long long tmax_w[kChkThreads / 32];
  if (threadIdx.x <= kTicksLog2) cnt[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long tmax = 0;
  int bad = 0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int l = lev[i];
    const int64_t t = t_tick[i];
    if (l < 0 || l > kTicksLog2 || t < 0) {
      bad = 1;
      continue;
    }
    if (t % (int64_t(1) << (kTicksLog2 - l)) != 0) bad = 1;
    atomicAdd(&cnt[l], 1);
    const unsigned long long tu = static_cast<unsigned long long>(t);
    tmax = tu > tmax ? tu : tmax;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, tmax, off);
    tmax = o > tmax ? o : tmax;
  }
  if ((threadIdx.x & 31) == 0) tmax_w[threadIdx.x >> 5] = tmax;
  if (__syncthreads_or(bad) && threadIdx.x == 0)
    atomicOr(reinterpret_cast<unsigned long long *>(ctl + kCtlBad), 1ull);
  if (threadIdx.x == 0) {
    for (int w = 1; w < kChkThreads / 32; ++w) tmax = tmax_w[w] > tmax ? tmax_w[w] : tmax;
    atomicMax(reinterpret_cast<unsigned long long *>(ctl + kCtlTcur), tmax);
  }
  if (threadIdx.x <= kTicksLog2 && cnt[threadIdx.x] > 0)
    atomicAdd(reinterpret_cast<unsigned long long *>(ctl + kCtlLevCnt + threadIdx.x),
              static_cast<unsigned long long>(cnt[threadIdx.x]));
}

// Every particle's next time must lie after the latest particle time.
__global__ void __launch_bounds__(kChkThreads)
    sched_due_kernel(int64_t n, const int64_t *__restrict__ t_tick,
                     const int32_t *__restrict__ lev, int64_t *ctl) {
  const int64_t t_cur = ctl[kCtlTcur];
  int bad = 0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int l = lev[i];
    if (l < 0 || l > kTicksLog2) continue;  // flagged by the level pass
    if (t_tick[i] + (int64_t(1) << (kTicksLog2 - l)) <= t_cur) bad = 1;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0)
    atomicOr(reinterpret_cast<unsigned long long *>(ctl + kCtlBad), 2ull);
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl[kCtlLastT] = t_cur;
}

// The predictor's FP32 split of every particle's state.
__global__ void __launch_bounds__(kChkThreads)
    split_refresh_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ v,
                         const double *__restrict__ a, const double *__restrict__ jk,
                         float4 *__restrict__ sp4, float2 *__restrict__ sp2) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double xs[3], vs[3], as[3], js[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    xs[c] = x[3 * i + c];
    vs[c] = v[3 * i + c];
    as[c] = a[3 * i + c];
    js[c] = jk[3 * i + c];
  }
  dev::PSplit S;
  dev::split_state(xs, vs, as, js, S);
  dev::store_split(i, S, sp4, sp2);
}

}  // namespace

cudaError_t launch_split_refresh(int64_t n, const double *x, const double *v, const double *a,
                                 const double *jk, float4 *sp4, float2 *sp2, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = (n + kChkThreads - 1) / kChkThreads;
  split_refresh_kernel<<<static_cast<unsigned>(nb), kChkThreads, 0, s>>>(n, x, v, a, jk, sp4,
                                                                          sp2);
  return cudaGetLastError();
}

cudaError_t launch_schedule_check(int64_t n, const int64_t *t_tick, const int32_t *lev,
                                  int64_t *ctl, cudaStream_t s, int *launches) {
  int64_t nb = (n + kChkThreads - 1) / kChkThreads;
  if (nb > 1024) nb = 1024;
  sched_levels_kernel<<<static_cast<unsigned>(nb), kChkThreads, 0, s>>>(n, t_tick, lev, ctl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sched_due_kernel<<<static_cast<unsigned>(nb), kChkThreads, 0, s>>>(n, t_tick, lev, ctl);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_block_begin(const BeginArgs &B, cudaStream_t s) {
  block_begin_kernel<<<static_cast<unsigned>(B.n_jt), kJT, 0, s>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_block_end(const EndArgs &E, int grid, cudaStream_t s) {
  block_end_kernel<<<static_cast<unsigned>(grid), kEndThreads, 0, s>>>(E);
  return cudaGetLastError();
}

}  // namespace nbi
