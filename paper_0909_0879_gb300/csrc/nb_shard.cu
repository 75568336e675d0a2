// i-split shards of the Hermite block-step integrator.
//
// The paper's two-GPU version of its code (Sec. 4, version E) divides the
// particles whose forces are computed among the GPUs, every GPU holding all
// the particles as sources.  Here a context can be one shard of P: it keeps
// the whole state (so it predicts every particle and sees the whole active
// list), owns the particles of one contiguous index range, evaluates the
// force and runs the corrector only for its slice of the active list, and
// exchanges the corrected records of the block with the other shards.
// Because the active list is in ascending index order and the ranges are
// contiguous and ascending, the slices of ranks 0..P-1 are consecutive
// pieces of it: concatenating the shards' records in rank order gives the
// records of the whole active list in its own order, with no counts to
// exchange (every shard finds every rank's slice in its own copy of the
// list).  These are the kernels; the bookkeeping is in nb_api.cu.
#include "nb_device.cuh"

namespace nbi {

namespace {

// Offsets of every rank's slice in the ascending active list: thread r
// finds the first entry k with act[k] >= bounds[r] (binary search).
__global__ void shard_offsets_kernel(const int32_t *__restrict__ act,
                                     const int64_t *__restrict__ ctl, const ShardBounds B,
                                     int64_t *__restrict__ off) {
  const int r = threadIdx.x;
  if (r > B.p) return;
  const int64_t n_act = ctl[kCtlNact];
  const int64_t key = B.b[r];
  int64_t lo = 0, hi = n_act;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (static_cast<int64_t>(act[mid]) < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  off[r] = lo;
}

// Records of active entries lo..hi-1 (the shard's slice), in list order.
__global__ void shard_export_kernel(int64_t lo, int64_t hi, const int32_t *__restrict__ act,
                                    const double *__restrict__ x, const double *__restrict__ v,
                                    const double *__restrict__ a, const double *__restrict__ jk,
                                    const int64_t *__restrict__ t_tick,
                                    const int32_t *__restrict__ lev, double *__restrict__ rec) {
  const int64_t k = lo + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= hi) return;
  const int64_t i = act[k];
  double *r = rec + (k - lo) * kShardRecDoubles;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    r[c] = x[3 * i + c];
    r[3 + c] = v[3 * i + c];
    r[6 + c] = a[3 * i + c];
    r[9 + c] = jk[3 * i + c];
  }
  r[12] = __longlong_as_double(static_cast<long long>(t_tick[i]));
  r[13] = __longlong_as_double(static_cast<long long>(lev[i]));
}

// The whole active list's records (n_act, list order) into the state,
// except the shard's own slice lo..hi-1, which its corrector wrote.
__global__ void shard_import_kernel(int64_t n_act, int64_t lo, int64_t hi,
                                    const int32_t *__restrict__ act,
                                    const double *__restrict__ rec, double *__restrict__ x,
                                    double *__restrict__ v, double *__restrict__ a,
                                    double *__restrict__ jk, int64_t *__restrict__ t_tick,
                                    int32_t *__restrict__ lev) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n_act || (k >= lo && k < hi)) return;
  const int64_t i = act[k];
  const double *r = rec + k * kShardRecDoubles;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    x[3 * i + c] = r[c];
    v[3 * i + c] = r[3 + c];
    a[3 * i + c] = r[6 + c];
    jk[3 * i + c] = r[9 + c];
  }
  t_tick[i] = static_cast<int64_t>(__double_as_longlong(r[12]));
  lev[i] = static_cast<int32_t>(__double_as_longlong(r[13]));
}

}  // namespace

cudaError_t launch_shard_offsets(const int32_t *act, const int64_t *ctl, const ShardBounds &B,
                                 int64_t *off, cudaStream_t s) {
  shard_offsets_kernel<<<1, 96, 0, s>>>(act, ctl, B, off);
  return cudaGetLastError();
}

cudaError_t launch_shard_export(int64_t lo, int64_t hi, const int32_t *act, const double *x,
                                const double *v, const double *a, const double *jk,
                                const int64_t *t_tick, const int32_t *lev, double *rec,
                                cudaStream_t s) {
  if (hi <= lo) return cudaSuccess;
  const int64_t nb = (hi - lo + 127) / 128;
  shard_export_kernel<<<static_cast<unsigned>(nb), 128, 0, s>>>(lo, hi, act, x, v, a, jk,
                                                                t_tick, lev, rec);
  return cudaGetLastError();
}

cudaError_t launch_shard_import(int64_t n_act, int64_t lo, int64_t hi, const int32_t *act,
                                const double *rec, double *x, double *v, double *a, double *jk,
                                int64_t *t_tick, int32_t *lev, cudaStream_t s) {
  if (n_act <= 0) return cudaSuccess;
  const int64_t nb = (n_act + 127) / 128;
  shard_import_kernel<<<static_cast<unsigned>(nb), 128, 0, s>>>(n_act, lo, hi, act, rec, x, v,
                                                                a, jk, t_tick, lev);
  return cudaGetLastError();
}

}  // namespace nbi
