// Internal declarations shared by the CUDA translation units of libnbody.
// Not part of the public C ABI (see include/nbody.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cfloat>

namespace nbi {

// Time is an integer count of 2^-20 ticks.
constexpr int kTicksLog2 = 20;

// j-records per shared-memory tile and pipeline depth of the force kernels.
constexpr int kJT = 256;
constexpr int kStages = 3;

// Bound on the polls of any device-side wait; past it the kernel records an
// error in the context's error word and returns instead of hanging.
constexpr uint32_t kWaitLimit = 1u << 24;

// Device error-word bits.
constexpr int kErrWaitTimeout = 1;

// Whether the kernels must zero the i == j pair term explicitly: eps^2 in
// FP32 is not a normal number (eps == 0, or so small that the device, which
// flushes subnormals to zero, would see eps^2 = 0 and evaluate the self
// pair as 0 * rsqrt(0) = NaN).
inline int eps_masks(double eps) {
  return static_cast<float>(eps * eps) < FLT_MIN ? 1 : 0;
}
// eps^2 as the FP32 kernels take it: 0 when the masked kernels run.
inline float eps2_f32(double eps) {
  return eps_masks(eps) ? 0.f : static_cast<float>(eps * eps);
}

// One force + jerk evaluation: active i-list against all (padded) j-records.
struct ForceArgs {
  const float4 *jhi;   // (x, y, z, m): FP32 values, or the high words (DS)
  const float4 *jlo;   // (x_lo, y_lo, z_lo, 0): low words (DS only)
  const float4 *jvel;  // (vx, vy, vz, 0)
  const float4 *jrel;  // (x - O_t, m): position relative to its tile's origin
  const float4 *tinfo; // per tile: (O_t, R_t), (half-widths of the box, 0)
  int64_t n_jt;        // j-tiles; records are padded to n_jt * kJT
  const int32_t *idx;  // i-list (n_i entries); nullptr = 0..n_i-1
  int64_t n_i;
  float eps2;
  double G;
  double *acc;         // (n_i, 3)
  double *jerk;        // (n_i, 3); null: acceleration only (launch_force)
  float2 *part;        // partial sums of split i-blocks (hi, lo pairs)
  int *err;            // device error word
  // Device-resident mode (block steps replayed from a CUDA graph): when ctl
  // is set the active count is ctl[kCtlNact]; a launch does nothing unless
  // it lies in [lo, hi), and the stream-K split is derived on the device.
  const int64_t *ctl = nullptr;
  int64_t lo = 0, hi = 0;
};

// External Galactic field (Allen & Santillan 1991; parameters as in
// nb_external of include/nbody.h).  on = 0: no field.
struct ExtField {
  int on = 0;
  double G = 0.0, c[3] = {0.0, 0.0, 0.0};
  double mb = 0.0, bb = 0.0;            // bulge
  double md = 0.0, ad = 0.0, bd = 0.0;  // disk
  double mh = 0.0, ah = 1.0, gam = 2.0, rcut = 1.0;  // halo
};
// Layout of the context's small device control array (int64 slots).
constexpr int kCtlTnext = 0;    // t_next of the current block (ticks); -1 = stop
constexpr int kCtlNact = 1;     // active count of the current block
constexpr int kCtlErr = 2;      // device error word (low 32 bits)
constexpr int kCtlClamped = 3;  // step-criterion clamps
constexpr int kCtlBlocks = 4;   // block steps taken on the device
constexpr int kCtlTend = 5;     // stop when the next block would pass this tick
constexpr int kCtlMaxBlk = 6;   // ... or when kCtlBlocks reaches this count
constexpr int kCtlInter = 7;    // interactions evaluated on the device
constexpr int kCtlLastT = 8;    // t of the last block taken on the device
constexpr int kCtlTicket = 9;   // CTA tickets of the fused block-begin kernel
constexpr int kCtlBad = 10;     // nonzero: the schedule is not level-structured
constexpr int kCtlTcur = 11;    // latest particle time (ticks), from the check
constexpr int kCtlLevCnt = 16;  // kTicksLog2 + 1 slots: particles per level
constexpr int kCtlSlots = 40;

// Device error-word bit of a timed-out look-back in the fused compaction.
constexpr int kErrScanTimeout = 2;

// Minimum j-tiles per CTA of the stream-K split, by the shape's threads
// per i-particle: 2 for the short-list shapes (16 or more; their lists are
// latency-bound and the CTA with the most tiles sets the time), 4
// otherwise (fewer split segments keep the fix-up short).
__host__ __device__ constexpr int64_t min_units(int tpi) { return tpi >= 16 ? 2 : 4; }

// Active-list lengths where the built-in force shape changes.
constexpr int64_t kBucketMid = 64;
constexpr int64_t kBucketLong = 1024;

// Records the per-thread error message returned by nb_last_error() and
// returns status unchanged (defined in nb_api.cu, shared by every C-ABI file).
int set_error(int status, const char *fmt, ...);

// Bytes of one j-record set per particle: FP32 (hi, vel) or DS (hi, lo, vel).
inline int record_bytes(int prec) { return prec ? 48 : 32; }

struct Variant {
  int prec;     // 0 = FP32, 1 = double-single
  int ipt;      // i-particles per thread
  int tpi;      // threads per i-particle (j split inside the CTA)
  int threads;  // threads per CTA
  int mask;     // 1: zero the i == j term (eps == 0)
  int pack;     // 1: two i-particles per packed FP32x2 instruction
  int sacc;     // 1: split-precision accumulators in shared memory
  int rel;      // 1: far tiles in tile-relative FP32 coordinates (DS only)
};

// A tile is "far" from an i-block when the distance between their bounding
// boxes is at least kRelKappa times the tile's radius; then positions
// relative to the tile's origin carry a relative error of at most
// 2^-23 (1.5 + 2 / kRelKappa) = 3.5 * 2^-23 in every pair difference
// (below the 1e-6 force tolerance with FP32 pair arithmetic on top).
// Measured on the N = 1M King cluster: kappa 3 / 2 / 1.5 / 1 give 919 /
// 905 / 891 / 881 ms per evaluation (with the 8-deep j unroll).
constexpr float kRelKappa = 1.0f;

int num_variants();
const Variant &variant_at(int v);
int block_i(const Variant &V);  // i-particles per i-block
// Built-in force shapes by active-list length: bucket k (lo[k] <= n_i <
// lo[k+1]) runs variant v[k].  A bucket's lower edge is raised above its
// nominal length (kBucketMid, kBucketLong) until its shape has enough
// (i-block, j-tile) units to give every SM min_units of them.
struct ShapeBuckets {
  int nbk;
  int64_t lo[3];
  int v[3];
};
ShapeBuckets shape_buckets(int prec, int mask, int64_t n_jt, int num_sms);
// The variant of n_i's bucket.
int choose_variant(int prec, int mask, int64_t n_i, int64_t n_jt, int num_sms);
// Resident CTAs per SM of a variant (occupancy query, cached).
int ctas_per_sm(int v);
// Bytes of partial-sum scratch a launch of variant v on `grid` CTAs needs.
size_t part_bytes(int v, int grid);
// Persistent grid for a variant, an active-list length and an optional cap.
int force_grid(int v, int64_t n_i, int64_t n_jt, int num_sms, int grid_cap);
// The variant has an acceleration-only kernel (the built-in shapes).
bool has_acc_only(int v);
// The shape the acceleration-only evaluation takes for built-in shape v.
int acc_shape(int v);
// Queue the force kernel (and its fix-up when i-blocks are split) on `s`.
// With A.jerk null the acceleration-only kernel runs (cudaErrorInvalidValue
// when the variant has none).  Returns the number of kernel launches
// through *launches.
cudaError_t launch_force(int v, const ForceArgs &A, int grid, cudaStream_t s,
                         int *launches);
// Device-resident form: A.ctl, A.lo, A.hi set; `grid` is the largest
// persistent grid of the variant and n_max bounds the active count.
// Without with_fixup the split i-blocks' partial sums are left in A.part
// for the fused block-end kernel.
cudaError_t launch_force_dev(int v, const ForceArgs &A, int grid, int64_t n_max,
                             cudaStream_t s, int *launches, bool with_fixup = true);

// --- Hermite and bookkeeping kernels (nb_hermite.cu) ---
// With ctl set, t_next is read from ctl[kCtlTnext] (negative: no-op).
cudaError_t launch_predict(int64_t n, int64_t t_next, const double *x,
                           const double *v, const double *a, const double *jk,
                           const double *m, const int64_t *t_tick, int prec,
                           float4 *jhi, float4 *jlo, float4 *jvel,
                           cudaStream_t s, const int64_t *ctl = nullptr);
cudaError_t launch_pad_records(int64_t n, int64_t n_pad, float4 *jhi,
                               float4 *jlo, float4 *jvel, cudaStream_t s);
// Per 256-record tile: bounding box, origin O_t (FP32 box centre), radius
// R_t, and every record's position relative to O_t.  With ctl set, a
// negative ctl[kCtlTnext] makes it a no-op.
cudaError_t launch_tile_info(int64_t n, int64_t n_jt, const float4 *jhi,
                             const float4 *jlo, float4 *jrel, float4 *tinfo,
                             cudaStream_t s, const int64_t *ctl = nullptr);
// With ctl set, n_act and t_next come from ctl (n_act is then a bound).
cudaError_t launch_correct(int64_t n_act, const int32_t *act, int64_t t_next,
                           double *x, double *v, double *a, double *jk,
                           int64_t *t_tick, int32_t *lev, const double *a1,
                           const double *j1, double eta, int lev_min,
                           int lev_max, int block_steps,
                           unsigned long long *n_clamped, const ExtField &E,
                           cudaStream_t s, const int64_t *ctl = nullptr);
// a += sign a_ext(x), jk += sign jerk_ext(x, v) for every particle (its own
// stored state); a no-op unless E.on.
cudaError_t launch_ext_adjust(int64_t n, const ExtField &E, double sign, const double *x,
                              const double *v, double *a, double *jk, cudaStream_t s);
cudaError_t launch_init_levels(int64_t n, const double *a, const double *jk,
                               double eta_start, int lev_min, int lev_max,
                               int block_steps, int lev_shared, int32_t *lev,
                               int64_t *t_tick, cudaStream_t s);
// Writes t_next (ticks) and n_act to d_scal[kCtlTnext], d_scal[kCtlNact]
// and the active list to act.  When the next block would pass
// d_scal[kCtlTend] or d_scal[kCtlBlocks] has reached d_scal[kCtlMaxBlk],
// t_next is set to -1 and n_act to 0 (everything after it is a no-op);
// otherwise kCtlBlocks, kCtlInter (n_act * n) and kCtlLastT advance.
// Returns the number of launches through *launches.
cudaError_t launch_next_block(int64_t n, const int64_t *t_tick,
                              const int32_t *lev, int32_t *act,
                              int32_t *blk_count, int64_t *d_scal,
                              cudaStream_t s, int *launches);
int64_t next_block_scratch_ints(int64_t n);
// Kinetic and softened potential energy in FP64 into d_out[0..1], and the
// external field's potential energy sum_i m_i Phi(x_i) into d_out[2] (0
// when E.on is 0).
cudaError_t launch_energy(int64_t n, const double *m, const double *x,
                          const double *v, double G, double eps, const ExtField &E,
                          double *red, double *d_out, cudaStream_t s, int *launches);
int64_t energy_scratch_doubles(int64_t n);

// --- Fused device-resident block steps (nb_blockstep.cu) ---
// Per-level counts, latest particle time and the level-structure check of
// the schedule (every particle's next time is the first multiple of its
// step after the latest particle time) into the control slots; the caller
// zeroes slots kCtlTicket..kCtlLevCnt + kTicksLog2 first.
cudaError_t launch_schedule_check(int64_t n, const int64_t *t_tick, const int32_t *lev,
                                  int64_t *ctl, cudaStream_t s, int *launches);

// Scheduling + prediction of one block step, one CTA per j-tile.
struct BeginArgs {
  int64_t n, n_jt;
  const double *x, *v, *a, *jk, *m;
  const int64_t *t_tick;
  const int32_t *lev;
  const float4 *sp4;                 // the predictor's FP32 split of the state
  const float2 *sp2;
  int prec;
  float4 *jhi, *jlo, *jvel;
  float4 *jrel, *tinfo;              // DS only (tile frames), else null
  int64_t rel_lo;                    // tile frames only from this active count on
  int32_t *act;
  int64_t *ctl;
  unsigned long long *status;        // n_jt look-back words
  // Look-back waits: polls before giving up, and an offset added to the
  // epoch the waits look for (nonzero only for the test injection that
  // makes every wait run out: no CTA publishes that epoch).
  uint32_t lb_wait_limit = kWaitLimit;
  uint64_t lb_epoch_skew = 0;
};
cudaError_t launch_block_begin(const BeginArgs &B, cudaStream_t s);

// Fix-up of the split i-blocks + corrector of one block step.
struct EndArgs {
  int64_t n, n_jt;
  int nbk;                           // force-shape buckets of the step
  int64_t lo[3], hi[3];              // active-count range of each bucket
  int bi[3], pmax[3];                // i-block size and persistent grid
  int mu[3];                         // minimum j-tiles per CTA (min_units)
  const float2 *part;                // partial sums of split i-blocks (hi, lo pairs)
  double G;
  double *a1, *j1;
  const int32_t *act;
  double *x, *v, *a, *jk;
  int64_t *t_tick;
  int32_t *lev;
  double eta;
  int lev_min, lev_max, block_steps;
  unsigned long long *n_clamped;
  int64_t *ctl;
  ExtField ext;                      // external field (on = 0: none)
  float4 *sp4;                       // the predictor's FP32 split, kept current
  float2 *sp2;
};
// The predictor's FP32 split of every particle's state into sp4, sp2.
cudaError_t launch_split_refresh(int64_t n, const double *x, const double *v, const double *a,
                                 const double *jk, float4 *sp4, float2 *sp2, cudaStream_t s);
cudaError_t launch_block_end(const EndArgs &E, int grid, cudaStream_t s);
constexpr int kEndThreads = 256;

// --- i-split shards (nb_shard.cu) ---
constexpr int kMaxShards = 64;
constexpr int kShardRecDoubles = 14;  // x, v, a, jerk (3 each), t_tick, lev (bit copies)
// Contiguous index ranges [b[r], b[r+1]) of the p shards.
struct ShardBounds {
  int p;
  int64_t b[kMaxShards + 1];
};
// off[r] (r = 0..p): first entry of the active list (ctl[kCtlNact] entries,
// ascending) at or above b[r].
cudaError_t launch_shard_offsets(const int32_t *act, const int64_t *ctl, const ShardBounds &B,
                                 int64_t *off, cudaStream_t s);
// rec[k - lo] = record of particle act[k] for k in [lo, hi).
cudaError_t launch_shard_export(int64_t lo, int64_t hi, const int32_t *act, const double *x,
                                const double *v, const double *a, const double *jk,
                                const int64_t *t_tick, const int32_t *lev, double *rec,
                                cudaStream_t s);
// State of particle act[k] = rec[k] for k in [0, n_act) outside [lo, hi).
cudaError_t launch_shard_import(int64_t n_act, int64_t lo, int64_t hi, const int32_t *act,
                                const double *rec, double *x, double *v, double *a, double *jk,
                                int64_t *t_tick, int32_t *lev, cudaStream_t s);

// --- Fixed-step symplectic integration (nb_symplectic.cu) ---
// Stage weights of the scheme of the given order into w (at most 7);
// returns the stage count (1 for order 2, 7 for order 6, 0 otherwise).
int symplectic_stages(int order, double *w);
// v += h (a + a_ext(x)), x += d v for every particle (a factor of 0 skips
// its update; a_ext only when E.on); with rec set also the j-records and,
// when jrel is set, the tile frames.
cudaError_t launch_kick_drift(int64_t n, int64_t n_jt, double h, double d, bool rec,
                              const ExtField &E, const double *a, double *v, double *x,
                              const double *m, int prec, float4 *jhi, float4 *jlo,
                              float4 *jvel, float4 *jrel, float4 *tinfo, cudaStream_t s);
// Rows of w doubles: dst[k] = src[perm[k]], or with scatter dst[perm[k]] =
// src[k].
cudaError_t launch_permute(int64_t n, const int64_t *perm, const double *src, double *dst,
                           int w, bool scatter, cudaStream_t s);
// a += a_ext(x) for every particle.
cudaError_t launch_ext_add(int64_t n, const ExtField &E, const double *x, double *a,
                           cudaStream_t s);

// --- Storage order (nb_layout.cu) ---
// Rows of w elements: dst[k] = src[idx[k]], k < n (T: double, int64_t,
// int32_t; I: int32_t, int64_t).
template <class T, class I>
cudaError_t launch_gather_rows(int64_t n, const I *idx, const T *src, T *dst, int w,
                               cudaStream_t s);
// inv[perm[k]] = k for a permutation of [0, n).
cudaError_t launch_invert(int64_t n, const int32_t *perm, int32_t *inv, cudaStream_t s);
// out[k] = slot[in[k]] for indices in [0, n); others are left as they are.
cudaError_t launch_map_index(int64_t n_idx, const int32_t *in, const int32_t *slot, int64_t n,
                             int32_t *out, cudaStream_t s);
}  // namespace nbi
