// C ABI of libnbody (declared in include/nbody.h): context, validation,
// device memory, stream ordering, the host watchdog and error reporting.
// Every step of the computation runs in the kernels of nb_force.cu and
// nb_hermite.cu; this file only marshals.
#include "../../include/nbody.h"
#include "nb_internal.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <numeric>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

using namespace nbi;

namespace {

thread_local char g_err[512] = "";
std::atomic<int> g_inject_oom{0};

// NVTX range for one phase of a block step (visible in Nsight timelines;
// a no-op when no tool is attached).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

nb_status fail(nb_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

}  // namespace

int nbi::set_error(int status, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return status;
}

namespace {

#define NB_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA, \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,   \
                  __LINE__);                                                 \
  } while (0)

// True when no value is an infinity or a NaN (exponent field all ones),
// checked on the bit patterns in blocks so that the loop vectorises.
bool finite_all(const double *p, int64_t cnt) {
  constexpr uint64_t kExp = 0x7ff0000000000000ull;
  for (int64_t b = 0; b < cnt; b += 4096) {
    const int64_t e = b + 4096 < cnt ? b + 4096 : cnt;
    uint64_t bad = 0;
    for (int64_t i = b; i < e; ++i) {
      uint64_t u;
      std::memcpy(&u, p + i, sizeof u);
      bad |= static_cast<uint64_t>((u & kExp) == kExp);
    }
    if (bad) return false;
  }
  return true;
}

// Particles [b, e) of a state nb_set_state takes: the first particle with
// a non-finite value (*nonfinite set) or an invalid level or tick, else e.
int64_t first_bad_particle(const double *x, const double *v, const double *a,
                           const double *jerk, const int64_t *t_tick, const int32_t *lev,
                           int64_t b, int64_t e, bool *nonfinite) {
  constexpr int64_t kBlk = 1024;
  for (int64_t i0 = b; i0 < e; i0 += kBlk) {
    const int64_t i1 = i0 + kBlk < e ? i0 + kBlk : e;
    const int64_t m = 3 * (i1 - i0);
    if (!finite_all(x + 3 * i0, m) || !finite_all(v + 3 * i0, m) ||
        !finite_all(a + 3 * i0, m) || !finite_all(jerk + 3 * i0, m)) {
      // the exact particle, for the message
      for (int64_t i = i0; i < i1; ++i)
        if (!finite_all(x + 3 * i, 3) || !finite_all(v + 3 * i, 3) ||
            !finite_all(a + 3 * i, 3) || !finite_all(jerk + 3 * i, 3)) {
          *nonfinite = true;
          return i;
        }
    }
    for (int64_t i = i0; i < i1; ++i)
      if (lev[i] < 0 || lev[i] > kTicksLog2 || t_tick[i] < 0 ||
          (t_tick[i] & ((int64_t(1) << (kTicksLog2 - lev[i])) - 1)) != 0) {
        *nonfinite = false;
        return i;
      }
  }
  return e;
}

// The same over all n particles on up to 16 of the host's cores (one pass:
// contiguous ranges, the caller's thread takes the last): the first bad
// particle in index order, or n.
int64_t first_bad_particle_par(int64_t n, const double *x, const double *v, const double *a,
                               const double *jerk, const int64_t *t_tick, const int32_t *lev,
                               bool *nonfinite) {
  const unsigned hw = std::thread::hardware_concurrency();
  int T = hw ? static_cast<int>(hw) : 1;
  if (T > 16) T = 16;
  if (n < (int64_t(1) << 16) || T < 2)
    return first_bad_particle(x, v, a, jerk, t_tick, lev, 0, n, nonfinite);
  const int64_t chunk = (n + T - 1) / T;
  std::vector<int64_t> bad(T, n);
  std::vector<char> nf(T, 0);
  std::vector<std::thread> th;
  int spawned = 0;
  auto run = [&](int k) {
    const int64_t b = k * chunk, e = b + chunk < n ? b + chunk : n;
    if (b >= e) return;
    bool f = false;
    const int64_t r = first_bad_particle(x, v, a, jerk, t_tick, lev, b, e, &f);
    if (r < e) {
      bad[k] = r;
      nf[k] = f ? 1 : 0;
    }
  };
  try {
    th.reserve(T - 1);
    for (int k = 0; k < T - 1; ++k) {
      th.emplace_back(run, k);
      ++spawned;
    }
  } catch (...) {
  }
  for (int k = spawned; k < T; ++k) run(k);
  for (auto &t : th) t.join();
  for (int k = 0; k < T; ++k)
    if (bad[k] < n) {
      *nonfinite = nf[k] != 0;
      return bad[k];
    }
  return n;
}

// finite_all over large arrays on the host's cores: contiguous chunks on
// up to 16 threads (the caller's thread takes the last); a thread that
// cannot be created leaves its chunk to the caller.
bool finite_all_par(const double *p, int64_t cnt) {
  constexpr int64_t kMinPar = int64_t(1) << 20;
  if (cnt < kMinPar) return finite_all(p, cnt);
  const unsigned hw = std::thread::hardware_concurrency();
  int T = hw ? static_cast<int>(hw) : 1;
  if (T > 16) T = 16;
  if (T < 2) return finite_all(p, cnt);
  const int64_t chunk = (cnt + T - 1) / T;
  std::vector<std::thread> th;
  std::vector<char> ok(T, 1);
  int spawned = 0;
  try {
    th.reserve(T - 1);
    for (int k = 0; k < T - 1; ++k) {
      const int64_t b = k * chunk, e = b + chunk < cnt ? b + chunk : cnt;
      th.emplace_back([p, b, e, k, &ok] { ok[k] = finite_all(p + b, e - b) ? 1 : 0; });
      ++spawned;
    }
  } catch (...) {
  }
  bool good = true;
  for (int k = spawned; k < T; ++k) {
    const int64_t b = k * chunk;
    if (b >= cnt) break;
    const int64_t e = b + chunk < cnt ? b + chunk : cnt;
    good = finite_all(p + b, e - b) && good;
  }
  for (auto &t : th) t.join();
  for (int k = 0; k < spawned; ++k) good = good && ok[k];
  return good;
}

int64_t tick_of(double t, bool *ok) {
  const double s = std::ldexp(t, kTicksLog2);
  *ok = std::isfinite(t) && s >= 0.0 && s < 9.0e18 && std::floor(s) == s;
  return *ok ? static_cast<int64_t>(s) : 0;
}

}  // namespace


namespace {

// Balanced recursive bisection: split [lo, hi) of perm at a multiple of
// `leaf` particles along the longest side of its bounding box (ties broken
// by index, so the order is fully determined), recurse on both halves.
// Levels of the bisection that may split off a thread: up to ~16 workers.
int kd_threads() {
  const unsigned hw = std::thread::hardware_concurrency();
  int lv = 0;
  while (lv < 4 && (2u << lv) <= (hw ? hw : 1u)) ++lv;
  return lv;
}

// Balanced bisection of perm[lo, hi) along the widest axis of its box, down
// to leaves of `leaf` records.  With par > 0 the left half of a split runs
// on another thread (par - 1 levels deeper may split again); the halves are
// disjoint and the comparator is a total order, so the result does not
// depend on the threads.
void kd_split(const double *x, int64_t *perm, int64_t lo, int64_t hi, int64_t leaf,
              int par = 0) {
  std::vector<std::thread> workers;
  while (hi - lo > leaf) {
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t k = lo; k < hi; ++k)
      for (int c = 0; c < 3; ++c) {
        const double v = x[3 * perm[k] + c];
        mn[c] = v < mn[c] ? v : mn[c];
        mx[c] = v > mx[c] ? v : mx[c];
      }
    int ax = 0;
    for (int c = 1; c < 3; ++c)
      if (mx[c] - mn[c] > mx[ax] - mn[ax]) ax = c;
    const int64_t leaves = (hi - lo + leaf - 1) / leaf;
    const int64_t mid = lo + leaf * ((leaves + 1) / 2);
    std::nth_element(perm + lo, perm + mid, perm + hi, [&](int64_t a, int64_t b) {
      const double va = x[3 * a + ax], vb = x[3 * b + ax];
      return va < vb || (va == vb && a < b);
    });
    bool spawned = false;
    if (par > 0 && mid - lo > (int64_t(1) << 12)) {
      try {
        workers.emplace_back(kd_split, x, perm, lo, mid, leaf, par - 1);
        spawned = true;
        --par;
      } catch (...) {  // no thread to be had: this one does the half
      }
    }
    if (!spawned) kd_split(x, perm, lo, mid, leaf, 0);
    lo = mid;  // tail loop on the right half
  }
  for (auto &w : workers) w.join();
}

}  // namespace

extern "C" nb_status nb_spatial_order(int64_t n, const double *x, int64_t leaf,
                                      int64_t *perm) {
  if (n < 0 || !x || !perm || leaf < 1)
    return fail(NB_ERR_INVALID_ARG, "need n >= 0, leaf >= 1 and non-null arrays");
  if (!finite_all(x, 3 * n)) return fail(NB_ERR_INVALID_ARG, "non-finite position");
  std::iota(perm, perm + n, int64_t(0));
  try {
    kd_split(x, perm, 0, n, leaf, kd_threads());
  } catch (...) {
    return fail(NB_ERR_OOM, "host memory for the bisection");
  }
  return NB_OK;
}

struct nb_ctx {
  int64_t n = 0, n_pad = 0, n_jt = 0;
  nb_config cfg{};
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  // device state, (n,3) row-major vectors
  double *m = nullptr, *x = nullptr, *v = nullptr, *a = nullptr, *jk = nullptr;
  double *a1 = nullptr, *j1 = nullptr;  // force output of the active list
  int64_t *t_tick = nullptr;
  int32_t *lev = nullptr;
  float4 *jhi = nullptr, *jlo = nullptr, *jvel = nullptr;  // j-records
  float4 *jrel = nullptr, *tinfo = nullptr;  // tile-relative records, tile boxes (DS)
  float4 *sp4 = nullptr;  // the predictor's FP32 split of the state (fused block steps)
  float2 *sp2 = nullptr;
  int32_t *act = nullptr;       // active list
  int32_t *blk = nullptr;       // scheduling scratch
  int64_t *scal = nullptr;      // [0] t_next ticks, [1] n_act
  double *part = nullptr;       // force partial sums
  size_t part_cap = 0;
  double *red = nullptr;        // energy scratch
  int *err = nullptr;           // device error word
  unsigned long long *clamped = nullptr;
  int32_t *qidx = nullptr;      // staged host index lists
  int64_t qidx_cap = 0;
  double *qout = nullptr;       // staged outputs for host queries
  int64_t qout_cap = 0;
  // pinned host mirror of small values
  int64_t *h_scal = nullptr;    // [0] t_next [1] n_act [2] err [3] clamped
  double *h_energy = nullptr;
  cudaEvent_t ev = nullptr;
  // host-side protocol state
  int64_t t_pred = -1;          // tick of the last prediction
  int64_t t_block = -1;         // t_next of the current block
  int64_t n_act = 0;
  bool have_block = false;
  bool force_done = false;
  int variant_override = -1;
  int table_count = 0;
  int64_t table_min[32];
  int32_t table_var[32];
  int32_t table_grid[32];  // persistent-grid cap of each entry (0: full grid)
  int grid_cap = 0;
  int64_t launches = 0, n_blocks = 0, interactions = 0;
  bool inject_timeout = false;
  bool inject_lookback = false;  // fused look-back waits run out (test injection)
  cudaGraphExec_t blk_graph = nullptr;  // device-resident block steps, general scheduler
  double *blk_graph_part = nullptr;
  cudaGraphExec_t fus_graph = nullptr;  // device-resident block steps, fused kernels
  double *fus_graph_part = nullptr;
  unsigned long long *lb_status = nullptr;  // look-back words of the fused compaction
  int block_mode = 0;                   // 0: fused when the schedule allows, 1: general
  int last_fused = 0;                   // the last nb_run_blocks ran the fused steps
  int64_t graph_launches = 0, fus_graph_launches = 0;  // kernels per replay
  // fixed-step symplectic integration: one step's graph for (order, dt)
  cudaGraphExec_t sym_graph = nullptr;
  double *sym_graph_part = nullptr;
  int sym_order = 0;
  double sym_dt = 0.0;
  int64_t sym_graph_launches = 0;
  bool sym_graph_stale = false;  // the field changed since the capture
  const double *sym_graph_x = nullptr;  // the position array the graph steps
  // spatial layout of the symplectic steps: the state gathered into a
  // bisection order, stepped there and scattered back
  int sym_layout = 0;            // NB_LAYOUT_AUTO / AS_GIVEN / SPATIAL
  int last_sym_spatial = 0;
  double *lx = nullptr, *lv = nullptr, *la = nullptr, *lm = nullptr;
  int64_t *lperm = nullptr;
  bool fresh = true;             // every particle still at t = 0 from nb_init
  // nb_symplectic moved x and v: the Hermite fields (jerk, times, levels)
  // no longer belong to them until nb_set_state
  bool sym_moved = false;
  ExtField ext;  // external Galactic field (symplectic integrators, energy)
  // i-split shard (nb_shard_set): this context owns particles
  // [sh.b[sh_rank], sh.b[sh_rank + 1]) of sh.p shards; own_lo..own_hi is its
  // slice of the current block's active list (the whole list unsharded)
  ShardBounds sh{1, {0}};
  int sh_rank = 0;
  int64_t *d_sh_off = nullptr;  // device: sh.p + 1 slice offsets
  int64_t *h_sh_off = nullptr;  // pinned mirror
  int64_t own_lo = 0, own_hi = 0;
  bool sh_corrected = false;    // own slice corrected, other shards' records not yet imported
  bool sh_off_valid = false;    // h_sh_off holds the last block's offsets
  int64_t sh_nact = 0;          // active count of that block
  // storage order (nb_relayout): slot s holds the particle the caller
  // knows as perm[s]; the identity until the first relayout
  bool permuted = false;
  int32_t *d_perm = nullptr;    // slot -> caller's index
  int32_t *d_slot = nullptr;    // caller's index -> slot
  int64_t *d_q = nullptr;       // a relayout's gather order (old slots)
  double *lay_buf = nullptr;    // 3n doubles: staging of the reordering copies
  std::vector<int32_t> h_perm;  // host copy of d_perm
  int64_t relayout_every = 0;   // automatic relayout after this many block steps (0: off)
  int64_t layout_blocks = 0;    // n_blocks at the last relayout
  int64_t relayouts = 0;
  std::vector<void *> allocs;
};

namespace {

nb_status dev_alloc(nb_ctx *c, void **p, size_t bytes) {
  if (g_inject_oom.exchange(0)) return fail(NB_ERR_OOM, "injected allocation failure");
  const char *cap = std::getenv("NB_TEST_MAX_BYTES");
  if (cap) {
    if (bytes > static_cast<size_t>(std::strtoull(cap, nullptr, 10)))
      return fail(NB_ERR_OOM, "allocation of %zu bytes exceeds NB_TEST_MAX_BYTES", bytes);
  }
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA,
                "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  try {
    c->allocs.push_back(*p);
  } catch (...) {  // no C++ exception leaves the library
    cudaFree(*p);
    *p = nullptr;
    return fail(NB_ERR_OOM, "host memory for the allocation list");
  }
  return NB_OK;
}

template <class T>
nb_status dev_alloc_t(nb_ctx *c, T **p, size_t count) {
  return dev_alloc(c, reinterpret_cast<void **>(p), count * sizeof(T));
}

// Wait for the stream with a host watchdog, then read the device error word
// and the small scalars into pinned memory.
nb_status sync_ctx(nb_ctx *c) {
  // the control slots (t_next, n_act, error word, clamps, device counters)
  // are contiguous: one copy back
  NB_CUDA(cudaMemcpyAsync(c->h_scal, c->scal, kCtlSlots * sizeof(int64_t),
                          cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(cudaEventRecord(c->ev, c->stream));
  if (c->inject_timeout) {
    c->inject_timeout = false;
    cudaEventSynchronize(c->ev);
    return fail(NB_ERR_TIMEOUT, "injected watchdog timeout");
  }
  const int ms = c->cfg.sync_timeout_ms > 0 ? c->cfg.sync_timeout_ms : 600000;
  const auto t0 = std::chrono::steady_clock::now();
  for (int64_t polls = 0;; ++polls) {
    cudaError_t e = cudaEventQuery(c->ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady)
      return fail(NB_ERR_CUDA, "stream execution failed: %s", cudaGetErrorString(e));
    const auto el = std::chrono::steady_clock::now() - t0;
    const auto us = std::chrono::duration_cast<std::chrono::microseconds>(el).count();
    if (us > static_cast<int64_t>(ms) * 1000)
      return fail(NB_ERR_TIMEOUT, "GPU work did not finish within %d ms", ms);
    // spin for the first 2 ms (block steps wait microseconds), then yield
    if (us > 2000) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  const int err = static_cast<int>(c->h_scal[kCtlErr] & 0xffffffff);
  if (err != 0) {
    // reported once: clear the word (stream-ordered) so that the context
    // can go on after the caller restores a state
    c->h_scal[kCtlErr] = 0;
    cudaMemsetAsync(c->scal + kCtlErr, 0, sizeof(int64_t), c->stream);
    return fail(NB_ERR_DEVICE, "a bounded device-side wait ran out: %s%s(device error word 0x%x)",
                (err & kErrWaitTimeout) ? "force kernel shared-memory tile; " : "",
                (err & kErrScanTimeout) ? "active-list look-back; " : "", err);
  }
  return NB_OK;
}

nb_status check_ctx(nb_ctx *c) {
  if (!c) return fail(NB_ERR_INVALID_ARG, "null context");
  return NB_OK;
}

// Hermite calls need the jerk, times and levels of the current x and v.
nb_status check_hermite(nb_ctx *c) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (c->sym_moved)
    return fail(NB_ERR_STATE, "nb_symplectic moved the particles; nb_set_state must give the "
                              "Hermite state (jerk, times, levels) before Hermite steps");
  return NB_OK;
}

// Force shape for n_i active particles, and the cap of its persistent grid
// (which sets the stream-K j-split) through *grid_cap.
int pick_variant(nb_ctx *c, int64_t n_i, int *grid_cap) {
  *grid_cap = c->grid_cap;
  if (c->variant_override >= 0) return c->variant_override;
  for (int k = 0; k < c->table_count; ++k)
    if (n_i >= c->table_min[k]) {
      if (c->table_grid[k] > 0) *grid_cap = c->table_grid[k];
      return c->table_var[k];
    }
  return choose_variant(c->cfg.precision, eps_masks(c->cfg.eps), n_i, c->n_jt, c->num_sms);
}

nb_status ensure_part(nb_ctx *c, size_t bytes) {
  if (bytes <= c->part_cap) return NB_OK;
  // Grows only when a tuning override asks for a larger grid than the one
  // sized at init; never on the default path.
  if (c->part) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->part);
    for (auto &p : c->allocs)
      if (p == c->part) p = nullptr;
    c->part = nullptr;
  }
  nb_status s = dev_alloc(c, reinterpret_cast<void **>(&c->part), bytes);
  if (s != NB_OK) return s;
  c->part_cap = bytes;
  return NB_OK;
}

// Queue one force evaluation of n_i i-particles (d_idx may be null for the
// identity list) into d_acc / d_jerk.
nb_status queue_force(nb_ctx *c, const int32_t *d_idx, int64_t n_i, double *d_acc,
                      double *d_jerk) {
  if (n_i == 0) return NB_OK;
  int cap = 0;
  const int v = pick_variant(c, n_i, &cap);
  const int grid = force_grid(v, n_i, c->n_jt, c->num_sms, cap);
  nb_status s = ensure_part(c, part_bytes(v, grid));
  if (s != NB_OK) return s;
  ForceArgs A;
  A.jhi = c->jhi;
  A.jlo = c->jlo;
  A.jvel = c->jvel;
  A.jrel = c->jrel;
  A.tinfo = c->tinfo;
  A.n_jt = c->n_jt;
  A.idx = d_idx;
  A.n_i = n_i;
  A.eps2 = eps2_f32(c->cfg.eps);
  A.G = c->cfg.G;
  A.acc = d_acc;
  A.jerk = d_jerk;
  A.part = reinterpret_cast<float2 *>(c->part);
  A.err = c->err;
  int nl = 0;
  NB_CUDA(launch_force(v, A, grid, c->stream, &nl));
  c->launches += nl;
  c->interactions += n_i * c->n;
  return NB_OK;
}

nb_status queue_predict(nb_ctx *c, int64_t tick) {
  NB_CUDA(launch_predict(c->n, tick, c->x, c->v, c->a, c->jk, c->m, c->t_tick,
                         c->cfg.precision, c->jhi, c->jlo, c->jvel, c->stream));
  c->launches += 1;
  if (c->jrel) {
    NB_CUDA(launch_tile_info(c->n, c->n_jt, c->jhi, c->jlo, c->jrel, c->tinfo, c->stream));
    c->launches += 1;
  }
  c->t_pred = tick;
  return NB_OK;
}

nb_status validate_config(const nb_config *cfg) {
  if (!cfg) return fail(NB_ERR_INVALID_ARG, "null config");
  if (!(std::isfinite(cfg->G) && cfg->G > 0))
    return fail(NB_ERR_INVALID_ARG, "G must be finite and > 0");
  if (!(std::isfinite(cfg->eps) && cfg->eps >= 0))
    return fail(NB_ERR_INVALID_ARG, "eps must be finite and >= 0");
  if (cfg->precision != NB_FP32 && cfg->precision != NB_DS)
    return fail(NB_ERR_INVALID_ARG, "precision must be NB_FP32 or NB_DS");
  if (cfg->lev_min < 0 || cfg->lev_max > kTicksLog2 || cfg->lev_min > cfg->lev_max)
    return fail(NB_ERR_INVALID_ARG, "need 0 <= lev_min <= lev_max <= 20");
  if (cfg->block_steps) {
    if (!(std::isfinite(cfg->eta) && cfg->eta > 0) ||
        !(std::isfinite(cfg->eta_start) && cfg->eta_start > 0))
      return fail(NB_ERR_INVALID_ARG, "eta and eta_start must be finite and > 0");
  } else if (cfg->lev_shared < 0 || cfg->lev_shared > kTicksLog2) {
    return fail(NB_ERR_INVALID_ARG, "need 0 <= lev_shared <= 20");
  }
  return NB_OK;
}

// storage order (defined with the spatial layout below)
nb_status relayout(nb_ctx *c);
nb_status relayout_if_due(nb_ctx *c);
nb_status ensure_qidx(nb_ctx *c, int64_t n_idx);

}  // namespace

extern "C" {

void nb_default_config(nb_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->G = 1.0;
  cfg->eps = 1e-3;
  cfg->eta = 0.01;
  cfg->eta_start = 0.01;
  cfg->lev_min = 3;
  cfg->lev_max = 20;
  cfg->precision = NB_DS;
  cfg->block_steps = 1;
  cfg->lev_shared = 8;
  cfg->sync_timeout_ms = 600000;
  cfg->stream = nullptr;
}

const char *nb_status_string(nb_status s) {
  switch (s) {
    case NB_OK: return "ok";
    case NB_ERR_INVALID_ARG: return "invalid argument";
    case NB_ERR_STATE: return "call out of order";
    case NB_ERR_CUDA: return "CUDA error";
    case NB_ERR_OOM: return "out of device memory";
    case NB_ERR_NUMERIC: return "non-finite result";
    case NB_ERR_TIMEOUT: return "watchdog timeout";
    case NB_ERR_DEVICE: return "device-side error";
  }
  return "unknown status";
}

const char *nb_last_error(void) { return g_err; }

void nb_destroy(nb_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (void *p : c->allocs)
    if (p) cudaFree(p);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  if (c->h_energy) cudaFreeHost(c->h_energy);
  if (c->h_sh_off) cudaFreeHost(c->h_sh_off);
  if (c->ev) cudaEventDestroy(c->ev);
  if (c->blk_graph) cudaGraphExecDestroy(c->blk_graph);
  if (c->fus_graph) cudaGraphExecDestroy(c->fus_graph);
  if (c->sym_graph) cudaGraphExecDestroy(c->sym_graph);
  delete c;
}

nb_status nb_init(nb_ctx **out, int64_t n, const double *m, const double *x,
                  const double *v, const nb_config *cfg) {
  if (!out) return fail(NB_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (n < 1 || n > (int64_t(1) << 30))
    return fail(NB_ERR_INVALID_ARG, "n = %lld out of range [1, 2^30]", (long long)n);
  if (!m || !x || !v) return fail(NB_ERR_INVALID_ARG, "null input array");
  nb_status s = validate_config(cfg);
  if (s != NB_OK) return s;
  if (!finite_all_par(m, n) || !finite_all_par(x, 3 * n) || !finite_all_par(v, 3 * n))
    return fail(NB_ERR_INVALID_ARG, "non-finite mass, position or velocity");
  for (int64_t i = 0; i < n; ++i)
    if (m[i] < 0) return fail(NB_ERR_INVALID_ARG, "negative mass at %lld", (long long)i);

  nb_ctx *c = new (std::nothrow) nb_ctx();
  if (!c) return fail(NB_ERR_OOM, "host memory for the context");
  c->cfg = *cfg;
  c->n = n;
  c->n_jt = (n + kJT - 1) / kJT;
  c->n_pad = c->n_jt * kJT;
  c->stream = static_cast<cudaStream_t>(cfg->stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    nb_destroy(c);
    return fail(NB_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
#define TRY(expr)          \
  do {                     \
    nb_status s_ = (expr); \
    if (s_ != NB_OK) {     \
      nb_destroy(c);       \
      return s_;           \
    }                      \
  } while (0)
  const size_t n3 = 3 * static_cast<size_t>(n);
  TRY(dev_alloc_t(c, &c->m, n));
  TRY(dev_alloc_t(c, &c->x, n3));
  TRY(dev_alloc_t(c, &c->v, n3));
  TRY(dev_alloc_t(c, &c->a, n3));
  TRY(dev_alloc_t(c, &c->jk, n3));
  TRY(dev_alloc_t(c, &c->a1, n3));
  TRY(dev_alloc_t(c, &c->j1, n3));
  TRY(dev_alloc_t(c, &c->t_tick, n));
  TRY(dev_alloc_t(c, &c->lev, n));
  TRY(dev_alloc_t(c, &c->jhi, c->n_pad));
  if (cfg->precision == NB_DS) {
    TRY(dev_alloc_t(c, &c->jlo, c->n_pad));
    TRY(dev_alloc_t(c, &c->jrel, c->n_pad));
    TRY(dev_alloc_t(c, &c->tinfo, 2 * c->n_jt));
  }
  TRY(dev_alloc_t(c, &c->jvel, c->n_pad));
  TRY(dev_alloc_t(c, &c->act, n));
  TRY(dev_alloc_t(c, &c->blk, next_block_scratch_ints(n) + 1));
  TRY(dev_alloc_t(c, &c->scal, kCtlSlots));
  TRY(dev_alloc_t(c, &c->lb_status, c->n_jt));
  TRY(dev_alloc_t(c, &c->sp4, 4 * static_cast<size_t>(n)));
  TRY(dev_alloc_t(c, &c->sp2, n));
  // the device error word and the clamp counter live in scal[2] and scal[3]
  c->err = reinterpret_cast<int *>(c->scal + kCtlErr);
  c->clamped = reinterpret_cast<unsigned long long *>(c->scal + kCtlClamped);
  TRY(dev_alloc_t(c, &c->red, energy_scratch_doubles(n)));
  // Partial-sum scratch for the largest built-in grid of every variant of
  // this precision, so the default path never allocates after init.
  size_t pb = 0;
  for (int vv = 0; vv < num_variants(); ++vv) {
    const Variant &V = variant_at(vv);
    if (V.prec != cfg->precision) continue;
    const size_t b = part_bytes(vv, c->num_sms * ctas_per_sm(vv));
    pb = b > pb ? b : pb;
  }
  TRY(dev_alloc(c, reinterpret_cast<void **>(&c->part), pb));
  c->part_cap = pb;
  if (cudaMallocHost(reinterpret_cast<void **>(&c->h_scal), 2 * kCtlSlots * sizeof(int64_t)) !=
          cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void **>(&c->h_energy), 4 * sizeof(double)) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess) {
    nb_destroy(c);
    return fail(NB_ERR_CUDA, "pinned host buffers / event creation failed");
  }
  std::memset(c->h_scal, 0, 2 * kCtlSlots * sizeof(int64_t));
#define TRYC(call)                                                                  \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      nb_destroy(c);                                                                \
      return fail(NB_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));            \
    }                                                                               \
  } while (0)
  cudaStream_t st = c->stream;
  TRYC(cudaMemcpyAsync(c->m, m, n * sizeof(double), cudaMemcpyHostToDevice, st));
  TRYC(cudaMemcpyAsync(c->x, x, n3 * sizeof(double), cudaMemcpyHostToDevice, st));
  TRYC(cudaMemcpyAsync(c->v, v, n3 * sizeof(double), cudaMemcpyHostToDevice, st));
  TRYC(cudaMemsetAsync(c->a, 0, n3 * sizeof(double), st));
  TRYC(cudaMemsetAsync(c->jk, 0, n3 * sizeof(double), st));
  TRYC(cudaMemsetAsync(c->t_tick, 0, n * sizeof(int64_t), st));
  TRYC(cudaMemsetAsync(c->scal, 0, kCtlSlots * sizeof(int64_t), st));
  TRYC(cudaMemsetAsync(c->lb_status, 0, c->n_jt * sizeof(unsigned long long), st));
  // no end time and no block budget unless nb_run_blocks sets them
  c->h_scal[kCtlSlots + 0] = INT64_MAX;
  c->h_scal[kCtlSlots + 1] = INT64_MAX;
  TRYC(cudaMemcpyAsync(c->scal + kCtlTend, c->h_scal + kCtlSlots, 2 * sizeof(int64_t),
                       cudaMemcpyHostToDevice, st));
  TRYC(launch_pad_records(n, c->n_pad, c->jhi, c->jlo, c->jvel, st));
  c->launches += 1;
  TRY(queue_predict(c, 0));
  TRY(queue_force(c, nullptr, n, c->a, c->jk));
  TRYC(launch_init_levels(n, c->a, c->jk, cfg->eta_start, cfg->lev_min, cfg->lev_max,
                          cfg->block_steps, cfg->lev_shared, c->lev, c->t_tick, st));
  c->launches += 1;
  TRY(sync_ctx(c));
  // initial force must be finite
  {
    std::vector<double> probe;
    try {
      probe.resize(n3);
    } catch (...) {
      nb_destroy(c);
      return fail(NB_ERR_OOM, "host memory for the initial-force check");
    }
    TRYC(cudaMemcpy(probe.data(), c->a, n3 * sizeof(double), cudaMemcpyDeviceToHost));
    if (!finite_all(probe.data(), static_cast<int64_t>(n3))) {
      nb_destroy(c);
      return fail(NB_ERR_NUMERIC, "initial acceleration is not finite (coincident particles with eps = 0?)");
    }
  }
  c->have_block = false;
  c->force_done = false;
  *out = c;
  return NB_OK;
#undef TRY
#undef TRYC
}

nb_status nb_next_block(nb_ctx *c, double *t_next, int64_t *n_active) {
  Range r("nb_next_block");
  nb_status s = check_hermite(c);
  if (s != NB_OK) return s;
  if (c->sh_corrected)
    return fail(NB_ERR_STATE, "shard: nb_shard_import of the last block's records comes first");
  s = relayout_if_due(c);
  if (s != NB_OK) return s;
  int nl = 0;
  NB_CUDA(launch_next_block(c->n, c->t_tick, c->lev, c->act, c->blk, c->scal, c->stream, &nl));
  c->launches += nl;
  if (c->sh.p > 1) {
    NB_CUDA(launch_shard_offsets(c->act, c->scal, c->sh, c->d_sh_off, c->stream));
    NB_CUDA(cudaMemcpyAsync(c->h_sh_off, c->d_sh_off, (c->sh.p + 1) * sizeof(int64_t),
                            cudaMemcpyDeviceToHost, c->stream));
    c->launches += 1;
  }
  s = sync_ctx(c);
  if (s != NB_OK) return s;
  c->t_block = c->h_scal[kCtlTnext];
  c->n_act = c->h_scal[kCtlNact];
  c->sh_off_valid = true;
  c->own_lo = c->sh.p > 1 ? c->h_sh_off[c->sh_rank] : 0;
  c->own_hi = c->sh.p > 1 ? c->h_sh_off[c->sh_rank + 1] : c->n_act;
  c->have_block = true;
  c->fresh = false;
  c->force_done = false;
  c->n_blocks += 1;
  if (t_next) *t_next = std::ldexp(static_cast<double>(c->t_block), -kTicksLog2);
  if (n_active) *n_active = c->n_act;
  return NB_OK;
}

nb_status nb_predict(nb_ctx *c, double t) {
  Range r("nb_predict");
  nb_status s = check_hermite(c);
  if (s != NB_OK) return s;
  bool ok;
  const int64_t tick = tick_of(t, &ok);
  if (!ok) return fail(NB_ERR_INVALID_ARG, "time %.17g is not a non-negative multiple of 2^-20", t);
  s = queue_predict(c, tick);
  if (s != NB_OK) return s;
  c->force_done = false;
  return NB_OK;
}

nb_status nb_force_jerk_dev(nb_ctx *c, const int32_t *d_idx, int64_t n_idx, double *d_acc,
                            double *d_jerk) {
  Range r("nb_force_jerk");
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (c->t_pred < 0) return fail(NB_ERR_STATE, "nb_predict must come first");
  if (d_idx == nullptr) {
    if (!c->have_block) return fail(NB_ERR_STATE, "no active list: call nb_next_block first");
    if (n_idx >= 0 && n_idx != c->n_act)
      return fail(NB_ERR_INVALID_ARG, "n_idx %lld != active count %lld", (long long)n_idx,
                  (long long)c->n_act);
    if (c->t_pred != c->t_block)
      return fail(NB_ERR_STATE, "prediction time differs from the block time");
    // a shard evaluates its own slice of the active list
    const int64_t lo = c->own_lo, cnt = c->own_hi - c->own_lo;
    s = queue_force(c, c->act + lo, cnt, c->a1 + 3 * lo, c->j1 + 3 * lo);
    if (s != NB_OK) return s;
    if (d_acc && cnt)
      NB_CUDA(cudaMemcpyAsync(d_acc, c->a1 + 3 * lo, 3 * cnt * sizeof(double),
                              cudaMemcpyDeviceToDevice, c->stream));
    if (d_jerk && cnt)
      NB_CUDA(cudaMemcpyAsync(d_jerk, c->j1 + 3 * lo, 3 * cnt * sizeof(double),
                              cudaMemcpyDeviceToDevice, c->stream));
    c->force_done = true;
    return NB_OK;
  }
  if (n_idx < 0) return fail(NB_ERR_INVALID_ARG, "negative n_idx");
  if (n_idx > 0 && (!d_acc || !d_jerk))
    return fail(NB_ERR_INVALID_ARG, "d_acc and d_jerk are required with an explicit index list");
  if (c->permuted && n_idx > 0) {
    // the caller's indices to storage slots
    s = ensure_qidx(c, n_idx);
    if (s != NB_OK) return s;
    NB_CUDA(launch_map_index(n_idx, d_idx, c->d_slot, c->n, c->qidx, c->stream));
    c->launches += 1;
    d_idx = c->qidx;
  }
  return queue_force(c, d_idx, n_idx, d_acc, d_jerk);
}

nb_status nb_force_jerk(nb_ctx *c, const int32_t *idx, int64_t n_idx, double *acc, double *jerk) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (c->t_pred < 0) return fail(NB_ERR_STATE, "nb_predict must come first");
  const double *src_a = nullptr, *src_j = nullptr;
  int64_t cnt = 0;
  if (idx == nullptr) {
    s = nb_force_jerk_dev(c, nullptr, n_idx, nullptr, nullptr);
    if (s != NB_OK) return s;
    src_a = c->a1 + 3 * c->own_lo;
    src_j = c->j1 + 3 * c->own_lo;
    cnt = c->own_hi - c->own_lo;
  } else {
    if (n_idx < 0) return fail(NB_ERR_INVALID_ARG, "negative n_idx");
    for (int64_t k = 0; k < n_idx; ++k)
      if (idx[k] < 0 || idx[k] >= c->n)
        return fail(NB_ERR_INVALID_ARG, "index %lld at position %lld out of range [0, %lld)",
                    (long long)idx[k], (long long)k, (long long)c->n);
    s = ensure_qidx(c, n_idx);
    if (s != NB_OK) return s;
    if (6 * n_idx > c->qout_cap) {
      if (c->qout) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->qout);
        for (auto &p : c->allocs)
          if (p == c->qout) p = nullptr;
        c->qout = nullptr;
      }
      s = dev_alloc_t(c, &c->qout, 6 * n_idx);
      if (s != NB_OK) return s;
      c->qout_cap = 6 * n_idx;
    }
    if (n_idx > 0)
      NB_CUDA(cudaMemcpyAsync(c->qidx, idx, n_idx * sizeof(int32_t), cudaMemcpyHostToDevice,
                              c->stream));
    if (c->permuted && n_idx > 0) {
      NB_CUDA(launch_map_index(n_idx, c->qidx, c->d_slot, c->n, c->qidx, c->stream));
      c->launches += 1;
    }
    s = queue_force(c, c->qidx, n_idx, c->qout, c->qout + 3 * n_idx);
    if (s != NB_OK) return s;
    src_a = c->qout;
    src_j = c->qout + 3 * n_idx;
    cnt = n_idx;
  }
  if (acc && cnt)
    NB_CUDA(cudaMemcpyAsync(acc, src_a, 3 * cnt * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
  if (jerk && cnt)
    NB_CUDA(cudaMemcpyAsync(jerk, src_j, 3 * cnt * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
  s = sync_ctx(c);
  if (s != NB_OK) return s;
  if ((acc && !finite_all_par(acc, 3 * cnt)) || (jerk && !finite_all_par(jerk, 3 * cnt)))
    return fail(NB_ERR_NUMERIC, "non-finite acceleration or jerk");
  return NB_OK;
}

nb_status nb_correct(nb_ctx *c, double t) {
  Range r("nb_correct");
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  bool ok;
  const int64_t tick = tick_of(t, &ok);
  if (!ok) return fail(NB_ERR_INVALID_ARG, "time %.17g is not a non-negative multiple of 2^-20", t);
  if (!c->have_block || !c->force_done || tick != c->t_block)
    return fail(NB_ERR_STATE, "nb_correct needs nb_next_block, nb_predict and nb_force_jerk "
                              "of the active list at the same time first");
  const int64_t lo = c->own_lo;
  NB_CUDA(launch_correct(c->own_hi - lo, c->act + lo, c->t_block, c->x, c->v, c->a, c->jk,
                         c->t_tick, c->lev, c->a1 + 3 * lo, c->j1 + 3 * lo, c->cfg.eta,
                         c->cfg.lev_min, c->cfg.lev_max, c->cfg.block_steps, c->clamped,
                         c->ext, c->stream));
  c->launches += 1;
  c->force_done = false;
  c->have_block = false;
  if (c->sh.p > 1) {
    c->sh_corrected = true;
    c->sh_nact = c->n_act;
  }
  return NB_OK;
}

nb_status nb_step(nb_ctx *c, double *t_next, int64_t *n_active) {
  double tn;
  int64_t na;
  nb_status s = nb_next_block(c, &tn, &na);
  if (s != NB_OK) return s;
  s = nb_predict(c, tn);
  if (s != NB_OK) return s;
  s = nb_force_jerk_dev(c, nullptr, na, nullptr, nullptr);
  if (s != NB_OK) return s;
  s = nb_correct(c, tn);
  if (s != NB_OK) return s;
  if (t_next) *t_next = tn;
  if (n_active) *n_active = na;
  return NB_OK;
}

}  // extern "C"

namespace {

constexpr int kGraphSteps = 32;  // block steps per graph replay

// Force shapes of the device-resident steps: the built-in choice per
// active-count bucket (the same shapes nb_step runs).
struct Bucket {
  int64_t lo, hi;
  int v;
};

int step_buckets(const nb_ctx *c, Bucket *b) {
  const ShapeBuckets sb = shape_buckets(c->cfg.precision, eps_masks(c->cfg.eps), c->n_jt,
                                        c->num_sms);
  // buckets no active count can reach (or empty ones) are left out
  int k = 0;
  for (int q = 0; q < sb.nbk; ++q) {
    const int64_t hi = q + 1 < sb.nbk ? sb.lo[q + 1] : INT64_MAX;
    if (sb.lo[q] <= c->n && sb.lo[q] < hi) b[k++] = {sb.lo[q], hi, sb.v[q]};
  }
  return k;
}

ForceArgs device_force_args(const nb_ctx *c, const Bucket &b) {
  ForceArgs A;
  A.jhi = c->jhi;
  A.jlo = c->jlo;
  A.jvel = c->jvel;
  A.jrel = c->jrel;
  A.tinfo = c->tinfo;
  A.n_jt = c->n_jt;
  A.idx = c->act;
  A.n_i = 0;
  A.eps2 = eps2_f32(c->cfg.eps);
  A.G = c->cfg.G;
  A.acc = c->a1;
  A.jerk = c->j1;
  A.part = reinterpret_cast<float2 *>(c->part);
  A.err = c->err;
  A.ctl = c->scal;
  A.lo = b.lo;
  A.hi = b.hi;
  return A;
}

// Queue kGraphSteps device-resident block steps on stream s with the
// general scheduler (any state); *launches counts the kernels.
nb_status queue_device_blocks(nb_ctx *c, cudaStream_t s, int64_t *launches) {
  Bucket b[3];
  const int nbk = step_buckets(c, b);
  const int prec = c->cfg.precision;
  for (int step = 0; step < kGraphSteps; ++step) {
    int nl = 0;
    NB_CUDA(launch_next_block(c->n, c->t_tick, c->lev, c->act, c->blk, c->scal, s, &nl));
    NB_CUDA(launch_predict(c->n, 0, c->x, c->v, c->a, c->jk, c->m, c->t_tick, prec, c->jhi,
                           c->jlo, c->jvel, s, c->scal));
    ++nl;
    if (c->jrel) {
      NB_CUDA(launch_tile_info(c->n, c->n_jt, c->jhi, c->jlo, c->jrel, c->tinfo, s, c->scal));
      ++nl;
    }
    for (int k = 0; k < nbk; ++k) {
      const int grid = c->num_sms * ctas_per_sm(b[k].v);
      NB_CUDA(launch_force_dev(b[k].v, device_force_args(c, b[k]), grid, c->n, s, &nl));
    }
    NB_CUDA(launch_correct(c->n, c->act, 0, c->x, c->v, c->a, c->jk, c->t_tick, c->lev, c->a1,
                           c->j1, c->cfg.eta, c->cfg.lev_min, c->cfg.lev_max,
                           c->cfg.block_steps, c->clamped, c->ext, s, c->scal));
    ++nl;
    *launches += nl;
  }
  return NB_OK;
}

// The fused form for a level-structured schedule: block_begin (scheduling
// from the per-level counts + predictor + tile frames), the force launch of
// every active-count bucket (the ones outside their range return at once),
// block_end (fix-up + corrector).
nb_status queue_fused_blocks(nb_ctx *c, cudaStream_t s, int64_t *launches) {
  Bucket b[3];
  const int nbk = step_buckets(c, b);
  BeginArgs B;
  B.n = c->n;
  B.n_jt = c->n_jt;
  B.x = c->x;
  B.v = c->v;
  B.a = c->a;
  B.jk = c->jk;
  B.m = c->m;
  B.t_tick = c->t_tick;
  B.lev = c->lev;
  B.sp4 = c->sp4;
  B.sp2 = c->sp2;
  B.prec = c->cfg.precision;
  B.jhi = c->jhi;
  B.jlo = c->jlo;
  B.jvel = c->jvel;
  B.jrel = c->jrel;
  B.tinfo = c->tinfo;
  // the smallest active count whose force shape takes the far field
  B.rel_lo = INT64_MAX;
  for (int k = 0; k < nbk; ++k)
    if (variant_at(b[k].v).rel && b[k].lo < B.rel_lo) B.rel_lo = b[k].lo;
  B.act = c->act;
  B.ctl = c->scal;
  B.status = c->lb_status;
  if (c->inject_lookback) {
    // test injection: a few polls for an epoch no CTA ever publishes
    B.lb_wait_limit = 256;
    B.lb_epoch_skew = uint64_t(1) << 24;
  }
  EndArgs E;
  E.n = c->n;
  E.n_jt = c->n_jt;
  E.nbk = nbk;
  for (int k = 0; k < nbk; ++k) {
    E.lo[k] = b[k].lo;
    E.hi[k] = b[k].hi;
    E.bi[k] = block_i(variant_at(b[k].v));
    E.pmax[k] = c->num_sms * ctas_per_sm(b[k].v);
    E.mu[k] = static_cast<int>(min_units(variant_at(b[k].v).tpi));
  }
  E.part = reinterpret_cast<const float2 *>(c->part);
  E.G = c->cfg.G;
  E.a1 = c->a1;
  E.j1 = c->j1;
  E.act = c->act;
  E.x = c->x;
  E.v = c->v;
  E.a = c->a;
  E.jk = c->jk;
  E.t_tick = c->t_tick;
  E.lev = c->lev;
  E.eta = c->cfg.eta;
  E.lev_min = c->cfg.lev_min;
  E.lev_max = c->cfg.lev_max;
  E.block_steps = c->cfg.block_steps;
  E.n_clamped = c->clamped;
  E.ctl = c->scal;
  E.ext = c->ext;
  E.sp4 = c->sp4;
  E.sp2 = c->sp2;
  const int end_grid = c->num_sms * 2;
  // The bucket launches are independent graph branches (fork after
  // block_begin, join before block_end), so the ones outside their range
  // return while the selected one runs instead of after it.
  cudaStream_t bs[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[3] = {nullptr, nullptr, nullptr};
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int k = 0; k < nbk && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&bs[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming);
  }
  for (int step = 0; step < kGraphSteps && e == cudaSuccess; ++step) {
    int nl = 0;
    e = launch_block_begin(B, s);
    if (e == cudaSuccess) e = cudaEventRecord(fork, s);
    for (int k = 0; k < nbk && e == cudaSuccess; ++k) {
      e = cudaStreamWaitEvent(bs[k], fork, 0);
      if (e == cudaSuccess)
        e = launch_force_dev(b[k].v, device_force_args(c, b[k]), E.pmax[k], c->n, bs[k], &nl,
                             false);
      if (e == cudaSuccess) e = cudaEventRecord(join[k], bs[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, join[k], 0);
    }
    if (e == cudaSuccess) e = launch_block_end(E, end_grid, s);
    *launches += 2 + nl;
  }
  for (int k = 0; k < nbk; ++k) {
    if (bs[k]) cudaStreamDestroy(bs[k]);
    if (join[k]) cudaEventDestroy(join[k]);
  }
  if (fork) cudaEventDestroy(fork);
  if (e != cudaSuccess)
    return fail(NB_ERR_CUDA, "fused block-step capture: %s", cudaGetErrorString(e));
  return NB_OK;
}

// Capture kGraphSteps block steps into an executable graph (on a private
// stream; the occupancy cache and shared-memory attributes are warm).
nb_status capture_blocks(nb_ctx *c, bool fused, cudaGraphExec_t *out, int64_t *launches) {
  cudaStream_t cs;
  NB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  *launches = 0;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  nb_status qs = NB_ERR_CUDA;
  if (e == cudaSuccess)
    qs = fused ? queue_fused_blocks(c, cs, launches) : queue_device_blocks(c, cs, launches);
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess || e2 != cudaSuccess || qs != NB_OK)
    return fail(NB_ERR_CUDA, "capture of the block-step graph failed: %s",
                cudaGetErrorString(e != cudaSuccess ? e : e2));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess)
    return fail(NB_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  return NB_OK;
}

// ---- fixed-step symplectic integration

// The arrays a symplectic run steps: the context's own, or the
// spatially ordered copies.
struct SymArrays {
  double *x, *v, *a;
  const double *m;
};

// Acceleration of every particle into S.a (acceleration-only kernel of the
// built-in shape for n, or its acceleration-only counterpart).
nb_status queue_acc_all(nb_ctx *c, const SymArrays &S, cudaStream_t s, int64_t *launches) {
  const int v = acc_shape(choose_variant(c->cfg.precision, eps_masks(c->cfg.eps), c->n,
                                         c->n_jt, c->num_sms));
  if (!has_acc_only(v)) return fail(NB_ERR_STATE, "force shape %d has no acceleration-only kernel", v);
  const int grid = force_grid(v, c->n, c->n_jt, c->num_sms, 0);
  if (part_bytes(v, grid) > c->part_cap)
    return fail(NB_ERR_STATE, "partial-sum scratch too small for shape %d", v);
  ForceArgs A;
  A.jhi = c->jhi;
  A.jlo = c->jlo;
  A.jvel = c->jvel;
  A.jrel = c->jrel;
  A.tinfo = c->tinfo;
  A.n_jt = c->n_jt;
  A.idx = nullptr;
  A.n_i = c->n;
  A.eps2 = eps2_f32(c->cfg.eps);
  A.G = c->cfg.G;
  A.acc = S.a;
  A.jerk = nullptr;
  A.part = reinterpret_cast<float2 *>(c->part);
  A.err = c->err;
  int nl = 0;
  NB_CUDA(launch_force(v, A, grid, s, &nl));
  *launches += nl;
  return NB_OK;
}

nb_status queue_kick_drift(nb_ctx *c, const SymArrays &S, cudaStream_t s, double h, double d,
                           bool rec, int64_t *launches) {
  NB_CUDA(launch_kick_drift(c->n, c->n_jt, h, d, rec, c->ext, S.a, S.v, S.x, S.m,
                            c->cfg.precision, c->jhi, c->jlo, c->jvel, c->jrel, c->tinfo, s));
  *launches += 1;
  return NB_OK;
}

// One step: the stages' kick-drift + force with the kicks between two
// drifts merged, then the closing half kick.
nb_status queue_symplectic_step(nb_ctx *c, const SymArrays &A, cudaStream_t s, const double *w,
                                int S, double dt, int64_t *launches) {
  for (int k = 0; k < S; ++k) {
    const double h = 0.5 * dt * ((k > 0 ? w[k - 1] : 0.0) + w[k]);
    nb_status st = queue_kick_drift(c, A, s, h, w[k] * dt, true, launches);
    if (st == NB_OK) st = queue_acc_all(c, A, s, launches);
    if (st != NB_OK) return st;
  }
  return queue_kick_drift(c, A, s, 0.5 * dt * w[S - 1], 0.0, false, launches);
}

nb_status capture_symplectic(nb_ctx *c, const SymArrays &A, const double *w, int S, double dt) {
  if (c->sym_graph) {
    cudaGraphExecDestroy(c->sym_graph);
    c->sym_graph = nullptr;
  }
  cudaStream_t cs;
  NB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  int64_t nl = 0;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  nb_status qs = NB_ERR_CUDA;
  if (e == cudaSuccess) qs = queue_symplectic_step(c, A, cs, w, S, dt, &nl);
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (qs != NB_OK && qs != NB_ERR_CUDA) {
    if (e2 == cudaSuccess) cudaGraphDestroy(g);
    return qs;
  }
  if (e != cudaSuccess || e2 != cudaSuccess || qs != NB_OK)
    return fail(NB_ERR_CUDA, "capture of the symplectic step failed: %s",
                cudaGetErrorString(e != cudaSuccess ? e : e2));
  e = cudaGraphInstantiate(&c->sym_graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess)
    return fail(NB_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  c->sym_graph_launches = nl;
  return NB_OK;
}

// Whether a run takes the spatial layout.  Automatic: split precision (the
// far field is what the layout buys), N >= 131,072 (on a uniform sphere in
// random order the layout measured 26-30 % faster per evaluation from N =
// 262,144 up, but only 8 % at 65,536 and nothing on a concentrated
// Plummer cluster there), and an estimated saving, a quarter of the run's
// force time at ~2e12 interactions/s, above 1.5 times the layout's cost
// (the bisection on the host cores, ~8 ns per particle and level, and the
// copies).
bool symplectic_spatial(const nb_ctx *c, int S, int64_t nsteps) {
  if (c->sym_layout == NB_LAYOUT_AS_GIVEN || nsteps == 0) return false;
  if (c->sym_layout == NB_LAYOUT_SPATIAL) return true;
  if (c->cfg.precision != NB_DS || c->n < 131072) return false;
  const double n = static_cast<double>(c->n);
  const double run_s = static_cast<double>(nsteps) * S * n * n / 2e12;
  const double layout_s = n * std::log2(n) * 8e-9 + n * 2e-8;
  return 0.25 * run_s > 1.5 * layout_s;
}

// Gather x, v, m into a bisection order of the current positions.
nb_status spatial_gather(nb_ctx *c, SymArrays *A) {
  const int64_t n = c->n;
  const size_t n3 = 3 * static_cast<size_t>(n);
  if (!c->lx) {
    nb_status s = dev_alloc_t(c, &c->lx, n3);
    if (s == NB_OK) s = dev_alloc_t(c, &c->lv, n3);
    if (s == NB_OK) s = dev_alloc_t(c, &c->la, n3);
    if (s == NB_OK) s = dev_alloc_t(c, &c->lm, n);
    if (s == NB_OK) s = dev_alloc_t(c, &c->lperm, n);
    if (s != NB_OK) return s;
  }
  std::vector<double> hx;
  std::vector<int64_t> perm;
  try {
    hx.resize(n3);
    perm.resize(n);
  } catch (...) {
    return fail(NB_ERR_OOM, "host memory for the spatial layout");
  }
  NB_CUDA(cudaMemcpyAsync(hx.data(), c->x, n3 * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
  nb_status s = sync_ctx(c);
  if (s != NB_OK) return s;
  std::iota(perm.begin(), perm.end(), int64_t(0));
  try {
    kd_split(hx.data(), perm.data(), 0, n, kJT, kd_threads());
  } catch (...) {
    return fail(NB_ERR_OOM, "host memory for the bisection");
  }
  NB_CUDA(cudaMemcpyAsync(c->lperm, perm.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice,
                          c->stream));
  NB_CUDA(launch_permute(n, c->lperm, c->x, c->lx, 3, false, c->stream));
  NB_CUDA(launch_permute(n, c->lperm, c->v, c->lv, 3, false, c->stream));
  NB_CUDA(launch_permute(n, c->lperm, c->m, c->lm, 1, false, c->stream));
  c->launches += 3;
  // the host arrays go out of scope: the copy from them must be done first
  s = sync_ctx(c);
  if (s != NB_OK) return s;
  *A = SymArrays{c->lx, c->lv, c->la, c->lm};
  return NB_OK;
}

// Re-store every per-particle array in a balanced-bisection order of the
// current positions (leaves of one 256-record tile).  The new slot s holds
// the particle of old slot q[s]; the caller's index of slot s becomes
// perm_old[q[s]].  Each array is gathered into the staging buffer and
// copied back, so the arrays keep their addresses (captured CUDA graphs
// stay valid).  The j-records, the active list and the fused steps' split
// state belong to the old order: the protocol restarts at nb_next_block
// and nb_run_blocks rebuilds the split at its start.
nb_status relayout(nb_ctx *c) {
  const int64_t n = c->n;
  const size_t n3 = 3 * static_cast<size_t>(n);
  if (!c->lay_buf) {
    nb_status s = dev_alloc_t(c, &c->lay_buf, n3);
    if (s == NB_OK) s = dev_alloc_t(c, &c->d_perm, n);
    if (s == NB_OK) s = dev_alloc_t(c, &c->d_slot, n);
    if (s == NB_OK) s = dev_alloc_t(c, &c->d_q, n);
    if (s != NB_OK) return s;
  }
  std::vector<double> hx;
  std::vector<int64_t> q;
  std::vector<int32_t> perm_new;
  try {
    hx.resize(n3);
    q.resize(n);
    perm_new.resize(n);
    if (!c->permuted) {
      c->h_perm.resize(n);
      std::iota(c->h_perm.begin(), c->h_perm.end(), int32_t(0));
    }
  } catch (...) {
    return fail(NB_ERR_OOM, "host memory for the relayout");
  }
  NB_CUDA(cudaMemcpyAsync(hx.data(), c->x, n3 * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
  nb_status s = sync_ctx(c);
  if (s != NB_OK) return s;
  if (!finite_all_par(hx.data(), static_cast<int64_t>(n3)))
    return fail(NB_ERR_NUMERIC, "non-finite position: no relayout");
  std::iota(q.begin(), q.end(), int64_t(0));
  try {
    kd_split(hx.data(), q.data(), 0, n, kJT, kd_threads());
  } catch (...) {
    return fail(NB_ERR_OOM, "host memory for the bisection");
  }
  for (int64_t k = 0; k < n; ++k) perm_new[k] = c->h_perm[q[k]];
  NB_CUDA(cudaMemcpyAsync(c->d_q, q.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice,
                          c->stream));
  double *const vec3[] = {c->x, c->v, c->a, c->jk};
  for (double *p : vec3) {
    NB_CUDA((launch_gather_rows<double, int64_t>(n, c->d_q, p, c->lay_buf, 3, c->stream)));
    NB_CUDA(cudaMemcpyAsync(p, c->lay_buf, n3 * sizeof(double), cudaMemcpyDeviceToDevice,
                            c->stream));
  }
  NB_CUDA((launch_gather_rows<double, int64_t>(n, c->d_q, c->m, c->lay_buf, 1, c->stream)));
  NB_CUDA(cudaMemcpyAsync(c->m, c->lay_buf, n * sizeof(double), cudaMemcpyDeviceToDevice,
                          c->stream));
  int64_t *ti = reinterpret_cast<int64_t *>(c->lay_buf);
  NB_CUDA((launch_gather_rows<int64_t, int64_t>(n, c->d_q, c->t_tick, ti, 1, c->stream)));
  NB_CUDA(cudaMemcpyAsync(c->t_tick, ti, n * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                          c->stream));
  int32_t *li = reinterpret_cast<int32_t *>(c->lay_buf);
  NB_CUDA((launch_gather_rows<int32_t, int64_t>(n, c->d_q, c->lev, li, 1, c->stream)));
  NB_CUDA(cudaMemcpyAsync(c->lev, li, n * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                          c->stream));
  NB_CUDA(cudaMemcpyAsync(c->d_perm, perm_new.data(), n * sizeof(int32_t),
                          cudaMemcpyHostToDevice, c->stream));
  NB_CUDA(launch_invert(n, c->d_perm, c->d_slot, c->stream));
  c->launches += 8;
  // the new order is queued on the stream: the host side follows it before
  // the wait, so the mapping matches the arrays even if the wait reports an
  // error (the copies from the host vectors were staged when queued)
  c->h_perm.swap(perm_new);
  c->permuted = true;
  c->have_block = false;
  c->force_done = false;
  c->t_pred = -1;
  c->layout_blocks = c->n_blocks;
  c->relayouts += 1;
  return sync_ctx(c);
}

// The automatic relayout of nb_set_relayout_every, when it is due.
nb_status relayout_if_due(nb_ctx *c) {
  if (c->relayout_every <= 0 || c->sh.p > 1) return NB_OK;
  if (c->n_blocks - c->layout_blocks < c->relayout_every) return NB_OK;
  return relayout(c);
}

// Room for n_idx staged indices.
nb_status ensure_qidx(nb_ctx *c, int64_t n_idx) {
  if (n_idx <= c->qidx_cap) return NB_OK;
  if (c->qidx) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->qidx);
    for (auto &p : c->allocs)
      if (p == c->qidx) p = nullptr;
    c->qidx = nullptr;
  }
  nb_status s = dev_alloc_t(c, &c->qidx, n_idx);
  if (s != NB_OK) return s;
  c->qidx_cap = n_idx;
  return NB_OK;
}

}  // namespace

extern "C" void nb_external_allen_santillan(nb_external *e) {
  if (!e) return;
  // Allen & Santillan (1991): length 1 kpc, mass 2.32e7 solar masses,
  // velocity 10 km/s, G = 1
  e->G = 1.0;
  e->center[0] = e->center[1] = e->center[2] = 0.0;
  e->m_bulge = 606.0;
  e->b_bulge = 0.3873;
  e->m_disk = 3690.0;
  e->a_disk = 5.3178;
  e->b_disk = 0.25;
  e->m_halo = 4615.0;
  e->a_halo = 12.0;
  e->gamma_halo = 2.02;
  e->r_cut = 100.0;
}

extern "C" nb_status nb_set_external(nb_ctx *c, const nb_external *e) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  ExtField f;
  if (e) {
    const double vals[] = {e->G,      e->center[0], e->center[1], e->center[2],
                           e->m_bulge, e->b_bulge,  e->m_disk,    e->a_disk,
                           e->b_disk,  e->m_halo,   e->a_halo,    e->gamma_halo,
                           e->r_cut};
    if (!finite_all(vals, static_cast<int64_t>(sizeof(vals) / sizeof(vals[0]))))
      return fail(NB_ERR_INVALID_ARG, "non-finite external-field parameter");
    if (e->G < 0 || e->m_bulge < 0 || e->m_disk < 0 || e->m_halo < 0 || e->a_disk < 0)
      return fail(NB_ERR_INVALID_ARG, "negative G, mass or disk scale length");
    if (!(e->b_bulge > 0) || !(e->b_disk > 0) || !(e->a_halo > 0) || !(e->r_cut > 0) ||
        !(e->gamma_halo > 1))
      return fail(NB_ERR_INVALID_ARG,
                  "b_bulge, b_disk, a_halo and r_cut must be positive and gamma_halo > 1");
    f.on = 1;
    f.G = e->G;
    for (int k = 0; k < 3; ++k) f.c[k] = e->center[k];
    f.mb = e->m_bulge;
    f.bb = e->b_bulge;
    f.md = e->m_disk;
    f.ad = e->a_disk;
    f.bd = e->b_disk;
    f.mh = e->m_halo;
    f.ah = e->a_halo;
    f.gam = e->gamma_halo;
    f.rcut = e->r_cut;
  }
  // the stored a and jerk of every particle carry the field: take the old
  // one out and put the new one in at each particle's own state; a state
  // fresh from nb_init also gets its initial levels from the new totals
  NB_CUDA(launch_ext_adjust(c->n, c->ext, -1.0, c->x, c->v, c->a, c->jk, c->stream));
  NB_CUDA(launch_ext_adjust(c->n, f, 1.0, c->x, c->v, c->a, c->jk, c->stream));
  c->launches += (c->ext.on ? 1 : 0) + (f.on ? 1 : 0);
  if (c->fresh) {
    NB_CUDA(launch_init_levels(c->n, c->a, c->jk, c->cfg.eta_start, c->cfg.lev_min,
                               c->cfg.lev_max, c->cfg.block_steps, c->cfg.lev_shared, c->lev,
                               c->t_tick, c->stream));
    c->launches += 1;
  }
  c->ext = f;
  c->sym_graph_stale = true;
  // the block-step graphs hold the field in their kernels' arguments
  if (c->blk_graph) {
    cudaGraphExecDestroy(c->blk_graph);
    c->blk_graph = nullptr;
  }
  if (c->fus_graph) {
    cudaGraphExecDestroy(c->fus_graph);
    c->fus_graph = nullptr;
  }
  c->have_block = false;
  c->force_done = false;
  c->t_pred = -1;
  return sync_ctx(c);
}

extern "C" nb_status nb_symplectic(nb_ctx *c, int32_t order, double dt, int64_t nsteps) {
  Range r("nb_symplectic");
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (c->sh.p > 1) return fail(NB_ERR_STATE, "the symplectic integrators run unsharded contexts only");
  double w[7];
  const int S = symplectic_stages(order, w);
  if (S == 0) return fail(NB_ERR_INVALID_ARG, "symplectic order %d is not 2 or 6", order);
  if (!std::isfinite(dt)) return fail(NB_ERR_INVALID_ARG, "non-finite time step");
  if (nsteps < 0) return fail(NB_ERR_INVALID_ARG, "negative step count");
  SymArrays A{c->x, c->v, c->a, c->m};
  const bool spatial = symplectic_spatial(c, S, nsteps);
  if (spatial) {
    s = spatial_gather(c, &A);
    if (s != NB_OK) return s;
  }
  c->last_sym_spatial = spatial ? 1 : 0;
  // the acceleration at the current positions, then nsteps replays of one
  // step's graph
  int64_t nl = 0;
  s = queue_kick_drift(c, A, c->stream, 0.0, 0.0, true, &nl);
  if (s == NB_OK) s = queue_acc_all(c, A, c->stream, &nl);
  if (s != NB_OK) return s;
  c->launches += nl;
  c->interactions += c->n * c->n;
  c->sym_moved = true;
  c->fresh = false;
  c->have_block = false;
  c->force_done = false;
  c->t_pred = -1;
  if (nsteps > 0) {
    if (!c->sym_graph || c->sym_order != order || c->sym_dt != dt ||
        c->sym_graph_part != c->part || c->sym_graph_stale || c->sym_graph_x != A.x) {
      s = capture_symplectic(c, A, w, S, dt);
      if (s != NB_OK) return s;
      c->sym_order = order;
      c->sym_dt = dt;
      c->sym_graph_part = c->part;
      c->sym_graph_stale = false;
      c->sym_graph_x = A.x;
    }
    for (int64_t k = 0; k < nsteps; ++k) NB_CUDA(cudaGraphLaunch(c->sym_graph, c->stream));
    c->launches += nsteps * c->sym_graph_launches;
    c->interactions += nsteps * S * c->n * c->n;
  }
  // the acceleration left in the state is the total one at the final x
  if (c->ext.on) {
    NB_CUDA(launch_ext_add(c->n, c->ext, A.x, A.a, c->stream));
    c->launches += 1;
  }
  if (spatial) {
    NB_CUDA(launch_permute(c->n, c->lperm, c->lx, c->x, 3, true, c->stream));
    NB_CUDA(launch_permute(c->n, c->lperm, c->lv, c->v, 3, true, c->stream));
    NB_CUDA(launch_permute(c->n, c->lperm, c->la, c->a, 3, true, c->stream));
    c->launches += 3;
  }
  return sync_ctx(c);
}

extern "C" nb_status nb_set_symplectic_layout(nb_ctx *c, int32_t mode) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (mode != NB_LAYOUT_AUTO && mode != NB_LAYOUT_AS_GIVEN && mode != NB_LAYOUT_SPATIAL)
    return fail(NB_ERR_INVALID_ARG, "unknown symplectic layout %d", mode);
  c->sym_layout = mode;
  return NB_OK;
}

extern "C" nb_status nb_last_symplectic_layout(nb_ctx *c, int32_t *spatial) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (!spatial) return fail(NB_ERR_INVALID_ARG, "null output pointer");
  *spatial = c->last_sym_spatial;
  return NB_OK;
}

extern "C" nb_status nb_run_blocks(nb_ctx *c, double t_end, int64_t max_blocks,
                                   int64_t *blocks_done, double *t_last) {
  Range r("nb_run_blocks");
  nb_status s = check_hermite(c);
  if (s != NB_OK) return s;
  if (c->sh.p > 1)
    return fail(NB_ERR_STATE, "device-resident block steps run unsharded contexts only");
  bool ok;
  const int64_t tend = tick_of(t_end, &ok);
  if (!ok) return fail(NB_ERR_INVALID_ARG, "t_end %.17g is not a non-negative multiple of 2^-20",
                       t_end);
  if (max_blocks < 0) return fail(NB_ERR_INVALID_ARG, "negative block budget");
  s = relayout_if_due(c);
  if (s != NB_OK) return s;
  // partial-sum scratch for every shape the device-resident steps may run
  size_t pb = 0;
  {
    const ShapeBuckets sb = shape_buckets(c->cfg.precision, eps_masks(c->cfg.eps),
                                          c->n_jt, c->num_sms);
    for (int q = 0; q < sb.nbk; ++q) {
      const size_t bytes = part_bytes(sb.v[q], c->num_sms * ctas_per_sm(sb.v[q]));
      pb = bytes > pb ? bytes : pb;
    }
  }
  s = ensure_part(c, pb);
  if (s != NB_OK) return s;
  if (c->block_mode == 0) {
    // per-level counts and the level-structure check for the fused steps
    NB_CUDA(cudaMemsetAsync(c->scal + kCtlTicket, 0,
                            (kCtlLevCnt + kTicksLog2 + 1 - kCtlTicket) * sizeof(int64_t),
                            c->stream));
    int nl = 0;
    NB_CUDA(launch_schedule_check(c->n, c->t_tick, c->lev, c->scal, c->stream, &nl));
    // the predictor's FP32 split of the state, kept current by the fused
    // corrector from here on
    NB_CUDA(launch_split_refresh(c->n, c->x, c->v, c->a, c->jk, c->sp4, c->sp2, c->stream));
    c->launches += nl + 1;
  }
  s = sync_ctx(c);
  if (s != NB_OK) return s;
  const bool fused = c->block_mode == 0 && c->h_scal[kCtlBad] == 0;
  const int64_t b0 = c->h_scal[kCtlBlocks];
  const int64_t i0 = c->h_scal[kCtlInter];
  c->h_scal[kCtlSlots + 0] = tend;
  c->h_scal[kCtlSlots + 1] = max_blocks > 0 ? b0 + max_blocks : INT64_MAX;
  NB_CUDA(cudaMemcpyAsync(c->scal + kCtlTend, c->h_scal + kCtlSlots, 2 * sizeof(int64_t),
                          cudaMemcpyHostToDevice, c->stream));
  cudaGraphExec_t &graph = fused ? c->fus_graph : c->blk_graph;
  double *&graph_part = fused ? c->fus_graph_part : c->blk_graph_part;
  int64_t &per_replay = fused ? c->fus_graph_launches : c->graph_launches;
  if (!graph || graph_part != c->part) {
    if (graph) {
      cudaGraphExecDestroy(graph);
      graph = nullptr;
    }
    s = capture_blocks(c, fused, &graph, &per_replay);
    if (s != NB_OK) return s;
    graph_part = c->part;
  }
  int64_t last_blocks = b0;
  for (;;) {
    NB_CUDA(cudaGraphLaunch(graph, c->stream));
    c->launches += per_replay;
    s = sync_ctx(c);
    if (s != NB_OK) return s;
    const int64_t nb = c->h_scal[kCtlBlocks];
    if (c->h_scal[kCtlTnext] < 0 || nb == last_blocks) break;
    last_blocks = nb;
  }
  c->h_scal[kCtlSlots + 0] = INT64_MAX;
  c->h_scal[kCtlSlots + 1] = INT64_MAX;
  NB_CUDA(cudaMemcpyAsync(c->scal + kCtlTend, c->h_scal + kCtlSlots, 2 * sizeof(int64_t),
                          cudaMemcpyHostToDevice, c->stream));
  s = sync_ctx(c);
  if (s != NB_OK) return s;
  const int64_t done = c->h_scal[kCtlBlocks] - b0;
  c->n_blocks += done;
  if (done > 0) c->fresh = false;
  c->interactions += c->h_scal[kCtlInter] - i0;
  c->have_block = false;
  c->force_done = false;
  c->t_pred = -1;
  c->last_fused = fused ? 1 : 0;
  if (blocks_done) *blocks_done = done;
  if (t_last) *t_last = std::ldexp(static_cast<double>(c->h_scal[kCtlLastT]), -kTicksLog2);
  return NB_OK;
}

extern "C" nb_status nb_set_block_mode(nb_ctx *c, int32_t mode) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (mode != NB_BLOCKS_AUTO && mode != NB_BLOCKS_GENERAL)
    return fail(NB_ERR_INVALID_ARG, "unknown block-step mode %d", mode);
  c->block_mode = mode;
  return NB_OK;
}

extern "C" nb_status nb_last_block_path(nb_ctx *c, int32_t *fused) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (!fused) return fail(NB_ERR_INVALID_ARG, "null output pointer");
  *fused = c->last_fused;
  return NB_OK;
}

extern "C" {

nb_status nb_energy(nb_ctx *c, double *kin, double *pot, double *tot) {
  Range r("nb_energy");
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  int nl = 0;
  double *d_out = c->red + energy_scratch_doubles(c->n) - 3;
  NB_CUDA(launch_energy(c->n, c->m, c->x, c->v, c->cfg.G, c->cfg.eps, c->ext, c->red, d_out,
                        c->stream, &nl));
  c->launches += nl;
  NB_CUDA(cudaMemcpyAsync(c->h_energy, d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
  s = sync_ctx(c);
  if (s != NB_OK) return s;
  const double w = c->h_energy[1] + c->h_energy[2];
  if (kin) *kin = c->h_energy[0];
  if (pot) *pot = w;
  if (tot) *tot = c->h_energy[0] + w;
  if (!std::isfinite(c->h_energy[0]) || !std::isfinite(w))
    return fail(NB_ERR_NUMERIC, "non-finite energy");
  return NB_OK;
}

nb_status nb_get_state(nb_ctx *c, double *x, double *v, double *a, double *jerk,
                       int64_t *t_tick, int32_t *lev) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  const size_t n3 = 3 * static_cast<size_t>(c->n) * sizeof(double);
  if (c->permuted) {
    // gathered into the caller's order (slot of caller index u: d_slot[u]),
    // one array at a time through the staging buffer
    const int64_t n = c->n;
    double *const src3[] = {c->x, c->v, c->a, c->jk};
    double *const dst3[] = {x, v, a, jerk};
    for (int k = 0; k < 4; ++k) {
      if (!dst3[k]) continue;
      NB_CUDA((launch_gather_rows<double, int32_t>(n, c->d_slot, src3[k], c->lay_buf, 3,
                                                  c->stream)));
      NB_CUDA(cudaMemcpyAsync(dst3[k], c->lay_buf, n3, cudaMemcpyDeviceToHost, c->stream));
      c->launches += 1;
    }
    if (t_tick) {
      int64_t *ti = reinterpret_cast<int64_t *>(c->lay_buf);
      NB_CUDA((launch_gather_rows<int64_t, int32_t>(n, c->d_slot, c->t_tick, ti, 1, c->stream)));
      NB_CUDA(cudaMemcpyAsync(t_tick, ti, n * sizeof(int64_t), cudaMemcpyDeviceToHost,
                              c->stream));
      c->launches += 1;
    }
    if (lev) {
      int32_t *li = reinterpret_cast<int32_t *>(c->lay_buf);
      NB_CUDA((launch_gather_rows<int32_t, int32_t>(n, c->d_slot, c->lev, li, 1, c->stream)));
      NB_CUDA(cudaMemcpyAsync(lev, li, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
      c->launches += 1;
    }
    return sync_ctx(c);
  }
  if (x) NB_CUDA(cudaMemcpyAsync(x, c->x, n3, cudaMemcpyDeviceToHost, c->stream));
  if (v) NB_CUDA(cudaMemcpyAsync(v, c->v, n3, cudaMemcpyDeviceToHost, c->stream));
  if (a) NB_CUDA(cudaMemcpyAsync(a, c->a, n3, cudaMemcpyDeviceToHost, c->stream));
  if (jerk) NB_CUDA(cudaMemcpyAsync(jerk, c->jk, n3, cudaMemcpyDeviceToHost, c->stream));
  if (t_tick)
    NB_CUDA(cudaMemcpyAsync(t_tick, c->t_tick, c->n * sizeof(int64_t), cudaMemcpyDeviceToHost,
                            c->stream));
  if (lev)
    NB_CUDA(cudaMemcpyAsync(lev, c->lev, c->n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            c->stream));
  return sync_ctx(c);
}

nb_status nb_set_state(nb_ctx *c, const double *x, const double *v, const double *a,
                       const double *jerk, const int64_t *t_tick, const int32_t *lev) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (!x || !v || !a || !jerk || !t_tick || !lev)
    return fail(NB_ERR_INVALID_ARG, "nb_set_state needs all six arrays");
  const int64_t n = c->n;
  // one pass over the six arrays on the host's cores before any copy, so a
  // rejected state leaves the context's state as it was
  bool nonfinite = false;
  const int64_t bad = first_bad_particle_par(n, x, v, a, jerk, t_tick, lev, &nonfinite);
  if (bad < n) {
    if (nonfinite) return fail(NB_ERR_INVALID_ARG, "non-finite state (particle %lld)",
                               (long long)bad);
    return fail(NB_ERR_INVALID_ARG, "particle %lld: level or tick invalid", (long long)bad);
  }
  const size_t n3 = 3 * static_cast<size_t>(n) * sizeof(double);
  if (c->permuted) {
    // uploaded in the caller's order, then gathered into the storage order
    // (slot s holds the caller's particle d_perm[s])
    double *const dst3[] = {c->x, c->v, c->a, c->jk};
    const double *const src3[] = {x, v, a, jerk};
    for (int k = 0; k < 4; ++k) {
      NB_CUDA(cudaMemcpyAsync(c->lay_buf, src3[k], n3, cudaMemcpyHostToDevice, c->stream));
      NB_CUDA((launch_gather_rows<double, int32_t>(n, c->d_perm, c->lay_buf, dst3[k], 3,
                                                  c->stream)));
    }
    int64_t *ti = reinterpret_cast<int64_t *>(c->lay_buf);
    NB_CUDA(cudaMemcpyAsync(ti, t_tick, n * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    NB_CUDA((launch_gather_rows<int64_t, int32_t>(n, c->d_perm, ti, c->t_tick, 1, c->stream)));
    int32_t *li = reinterpret_cast<int32_t *>(c->lay_buf);
    NB_CUDA(cudaMemcpyAsync(li, lev, n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    NB_CUDA((launch_gather_rows<int32_t, int32_t>(n, c->d_perm, li, c->lev, 1, c->stream)));
    c->launches += 6;
  } else {
    NB_CUDA(cudaMemcpyAsync(c->x, x, n3, cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(cudaMemcpyAsync(c->v, v, n3, cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(cudaMemcpyAsync(c->a, a, n3, cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(cudaMemcpyAsync(c->jk, jerk, n3, cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(cudaMemcpyAsync(c->t_tick, t_tick, n * sizeof(int64_t), cudaMemcpyHostToDevice,
                            c->stream));
    NB_CUDA(cudaMemcpyAsync(c->lev, lev, n * sizeof(int32_t), cudaMemcpyHostToDevice,
                            c->stream));
  }
  c->have_block = false;
  c->force_done = false;
  c->t_pred = -1;
  c->sym_moved = false;
  c->fresh = false;
  c->sh_corrected = false;
  c->sh_off_valid = false;
  return sync_ctx(c);
}

nb_status nb_get_active(nb_ctx *c, int32_t *idx, int64_t cap, int64_t *n_active) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (!c->have_block) return fail(NB_ERR_STATE, "no active list: call nb_next_block first");
  if (n_active) *n_active = c->n_act;
  if (idx) {
    if (cap < c->n_act) return fail(NB_ERR_INVALID_ARG, "capacity %lld < active count %lld",
                                    (long long)cap, (long long)c->n_act);
    if (c->n_act)
      NB_CUDA(cudaMemcpyAsync(idx, c->act, c->n_act * sizeof(int32_t), cudaMemcpyDeviceToHost,
                              c->stream));
  }
  s = sync_ctx(c);
  if (s != NB_OK) return s;
  if (idx && c->permuted)  // storage slots to the caller's indices
    for (int64_t k = 0; k < c->n_act; ++k) idx[k] = c->h_perm[idx[k]];
  return NB_OK;
}

nb_status nb_relayout(nb_ctx *c) {
  Range r("nb_relayout");
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (c->sh.p > 1)
    return fail(NB_ERR_STATE, "a shard exchanges records in its peers' order: no relayout");
  return relayout(c);
}

nb_status nb_set_relayout_every(nb_ctx *c, int64_t block_steps) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (block_steps < 0) return fail(NB_ERR_INVALID_ARG, "negative relayout interval");
  c->relayout_every = block_steps;
  c->layout_blocks = c->n_blocks;
  return NB_OK;
}

nb_status nb_get_storage_order(nb_ctx *c, int32_t *perm, int64_t *relayouts) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (perm) {
    if (c->permuted)
      std::copy(c->h_perm.begin(), c->h_perm.end(), perm);
    else
      std::iota(perm, perm + c->n, int32_t(0));
  }
  if (relayouts) *relayouts = c->relayouts;
  return NB_OK;
}

nb_status nb_get_counters(nb_ctx *c, int64_t *n_blocks, int64_t *n_interactions,
                          int64_t *n_clamped) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  s = sync_ctx(c);
  if (s != NB_OK) return s;
  if (n_blocks) *n_blocks = c->n_blocks;
  if (n_interactions) *n_interactions = c->interactions;
  if (n_clamped) *n_clamped = c->h_scal[kCtlClamped];
  return NB_OK;
}

nb_status nb_sync(nb_ctx *c) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  return sync_ctx(c);
}

int64_t nb_launch_count(const nb_ctx *c) { return c ? c->launches : -1; }

nb_status nb_set_force_variant(nb_ctx *c, int32_t variant, int32_t grid_ctas) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (variant >= num_variants() || variant < -1)
    return fail(NB_ERR_INVALID_ARG, "unknown force variant %d", variant);
  if (variant >= 0) {
    const Variant &V = variant_at(variant);
    if (V.prec != c->cfg.precision)
      return fail(NB_ERR_INVALID_ARG, "variant %d has the other precision", variant);
    if (V.mask != eps_masks(c->cfg.eps))
      return fail(NB_ERR_INVALID_ARG, "variant %d does not match the self-pair masking of this eps", variant);
  }
  c->variant_override = variant;
  c->grid_cap = grid_ctas > 0 ? grid_ctas : 0;
  return NB_OK;
}

nb_status nb_set_force_table(nb_ctx *c, int32_t count, const int64_t *min_n,
                             const int32_t *variant, const int32_t *grid_ctas) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (count < 0 || count > 32) return fail(NB_ERR_INVALID_ARG, "table holds 0..32 entries");
  if (count > 0 && (!min_n || !variant)) return fail(NB_ERR_INVALID_ARG, "null table arrays");
  for (int k = 0; k < count; ++k) {
    if (variant[k] < 0 || variant[k] >= num_variants())
      return fail(NB_ERR_INVALID_ARG, "unknown force variant %d", variant[k]);
    const Variant &V = variant_at(variant[k]);
    if (V.prec != c->cfg.precision || V.mask != eps_masks(c->cfg.eps))
      return fail(NB_ERR_INVALID_ARG, "variant %d does not match the context", variant[k]);
    if (grid_ctas && grid_ctas[k] < 0)
      return fail(NB_ERR_INVALID_ARG, "negative grid cap %d", grid_ctas[k]);
  }
  // partial-sum scratch for the largest grid any table entry can use
  size_t pb = 0;
  for (int k = 0; k < count; ++k) {
    const size_t b = part_bytes(variant[k], c->num_sms * ctas_per_sm(variant[k]));
    pb = b > pb ? b : pb;
  }
  s = ensure_part(c, pb);
  if (s != NB_OK) return s;
  c->table_count = count;
  for (int k = 0; k < count; ++k) {
    c->table_min[k] = min_n[k];
    c->table_var[k] = variant[k];
    c->table_grid[k] = grid_ctas ? grid_ctas[k] : 0;
  }
  return NB_OK;
}

nb_status nb_variant_info(int32_t v, int32_t *precision, int32_t *ipt, int32_t *tpi,
                          int32_t *threads, int32_t *packed) {
  if (v < 0 || v >= num_variants()) return fail(NB_ERR_INVALID_ARG, "unknown variant %d", v);
  const Variant &V = variant_at(v);
  if (precision) *precision = V.prec;
  if (ipt) *ipt = V.ipt;
  if (tpi) *tpi = V.tpi;
  if (threads) *threads = V.threads;
  if (packed) *packed = V.pack;
  return NB_OK;
}

nb_status nb_debug_inject(nb_ctx *c, int32_t kind) {
  if (kind == 1) {
    g_inject_oom.store(1);
    return NB_OK;
  }
  if (kind == 2) {
    if (!c) return fail(NB_ERR_INVALID_ARG, "timeout injection needs a context");
    c->inject_timeout = true;
    return NB_OK;
  }
  if (kind == 3 || kind == 0) {
    if (!c) return fail(NB_ERR_INVALID_ARG, "this injection needs a context");
    const bool want = kind == 3;
    if (kind == 0) c->inject_timeout = false;
    if (c->inject_lookback != want) {
      // the fused block-step graph holds the waits' arguments: capture anew
      cudaStreamSynchronize(c->stream);
      if (c->fus_graph) cudaGraphExecDestroy(c->fus_graph);
      c->fus_graph = nullptr;
      c->inject_lookback = want;
    }
    return NB_OK;
  }
  return fail(NB_ERR_INVALID_ARG, "unknown injection kind %d", kind);
}

nb_status nb_shard_set(nb_ctx *c, int32_t nranks, int32_t rank, const int64_t *bounds) {
  nb_status s = check_hermite(c);
  if (s != NB_OK) return s;
  if (nranks < 1 || nranks > kMaxShards || rank < 0 || rank >= nranks)
    return fail(NB_ERR_INVALID_ARG, "need 1 <= nranks <= %d and 0 <= rank < nranks", kMaxShards);
  if (nranks > 1 && !bounds) return fail(NB_ERR_INVALID_ARG, "null shard bounds");
  if (nranks > 1) {
    if (bounds[0] != 0 || bounds[nranks] != c->n)
      return fail(NB_ERR_INVALID_ARG, "shard bounds must run from 0 to n");
    for (int r = 0; r < nranks; ++r)
      if (bounds[r + 1] < bounds[r])
        return fail(NB_ERR_INVALID_ARG, "shard bounds must not decrease");
  }
  if (c->have_block || c->sh_corrected)
    return fail(NB_ERR_STATE, "change the sharding between block steps only");
  if (nranks > 1 && c->permuted)
    return fail(NB_ERR_STATE, "shards need the caller's particle order: this context was "
                              "re-stored by nb_relayout");
  if (nranks > 1 && !c->d_sh_off) {
    s = dev_alloc_t(c, &c->d_sh_off, kMaxShards + 1);
    if (s != NB_OK) return s;
    if (cudaMallocHost(reinterpret_cast<void **>(&c->h_sh_off),
                       (kMaxShards + 1) * sizeof(int64_t)) != cudaSuccess) {
      c->h_sh_off = nullptr;
      return fail(NB_ERR_CUDA, "pinned host buffer for the shard offsets");
    }
  }
  c->sh.p = nranks;
  c->sh_rank = nranks > 1 ? rank : 0;
  for (int r = 0; r <= kMaxShards; ++r) c->sh.b[r] = 0;
  if (nranks > 1)
    for (int r = 0; r <= nranks; ++r) c->sh.b[r] = bounds[r];
  c->sh_corrected = false;
  c->sh_off_valid = false;
  return NB_OK;
}

nb_status nb_shard_offsets(nb_ctx *c, int64_t *offsets) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (!offsets) return fail(NB_ERR_INVALID_ARG, "null output");
  if (!c->sh_off_valid)
    return fail(NB_ERR_STATE, "no block yet: call nb_next_block first");
  if (c->sh.p == 1) {
    offsets[0] = 0;
    offsets[1] = c->n_act;
    return NB_OK;
  }
  for (int r = 0; r <= c->sh.p; ++r) offsets[r] = c->h_sh_off[r];
  return NB_OK;
}

nb_status nb_shard_export(nb_ctx *c, double *d_rec, int64_t *count) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (c->sh.p == 1 || !c->sh_corrected)
    return fail(NB_ERR_STATE, "nb_shard_export follows nb_correct on a shard");
  const int64_t cnt = c->own_hi - c->own_lo;
  if (cnt > 0 && !d_rec) return fail(NB_ERR_INVALID_ARG, "null record buffer");
  NB_CUDA(launch_shard_export(c->own_lo, c->own_hi, c->act, c->x, c->v, c->a, c->jk, c->t_tick,
                              c->lev, d_rec, c->stream));
  if (cnt > 0) c->launches += 1;
  if (count) *count = cnt;
  return NB_OK;
}

nb_status nb_shard_import(nb_ctx *c, const double *d_rec, int64_t n_rec) {
  nb_status s = check_ctx(c);
  if (s != NB_OK) return s;
  if (c->sh.p == 1 || !c->sh_corrected)
    return fail(NB_ERR_STATE, "nb_shard_import follows nb_correct on a shard");
  if (n_rec != c->sh_nact)
    return fail(NB_ERR_INVALID_ARG, "%lld records for an active list of %lld",
                (long long)n_rec, (long long)c->sh_nact);
  if (n_rec > 0 && !d_rec) return fail(NB_ERR_INVALID_ARG, "null record buffer");
  NB_CUDA(launch_shard_import(n_rec, c->own_lo, c->own_hi, c->act, d_rec, c->x, c->v, c->a,
                              c->jk, c->t_tick, c->lev, c->stream));
  if (n_rec > 0) c->launches += 1;
  c->sh_corrected = false;
  return NB_OK;
}

}  // extern "C"
