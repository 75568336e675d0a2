// Storage order of a context's particles (nb_relayout).  The force kernel's
// tile-relative far field needs every 256-record tile and every i-block to
// be compact in space; particles stored in a bisection order of their
// positions give that, and as they move the tiles spread.  Re-storing the
// state in a fresh order brings the compact tiles back; these kernels move
// the per-particle arrays between the caller's order and the storage
// order.  Pure data movement: no arithmetic on the values.
#include "nb_internal.cuh"

namespace nbi {
namespace {

// dst[k] = src[idx[k]] for rows of w elements.
template <class T, class I>
__global__ void gather_rows_kernel(int64_t n, const I *__restrict__ idx,
                                   const T *__restrict__ src, T *__restrict__ dst, int w) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t from = static_cast<int64_t>(idx[k]);
  for (int c = 0; c < w; ++c) dst[w * k + c] = src[w * from + c];
}

// inv[perm[k]] = k.
__global__ void invert_kernel(int64_t n, const int32_t *__restrict__ perm,
                              int32_t *__restrict__ inv) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  inv[perm[k]] = static_cast<int32_t>(k);
}

// out[k] = slot[in[k]] for in[k] in [0, n); an index outside stays as it
// is (the force call's contract leaves such an index undefined, and this
// kernel reads nothing out of range).  in and out may be the same array.
__global__ void map_index_kernel(int64_t n_idx, const int32_t *in, const int32_t *slot, int64_t n,
                                 int32_t *out) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n_idx) return;
  const int32_t u = in[k];
  out[k] = (u >= 0 && u < n) ? slot[u] : u;
}

inline unsigned blocks_for(int64_t n) { return static_cast<unsigned>((n + 255) / 256); }

}  // namespace

template <class T, class I>
cudaError_t launch_gather_rows(int64_t n, const I *idx, const T *src, T *dst, int w,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  gather_rows_kernel<T, I><<<blocks_for(n), 256, 0, s>>>(n, idx, src, dst, w);
  return cudaGetLastError();
}

template cudaError_t launch_gather_rows<double, int32_t>(int64_t, const int32_t *,
                                                         const double *, double *, int,
                                                         cudaStream_t);
template cudaError_t launch_gather_rows<double, int64_t>(int64_t, const int64_t *,
                                                         const double *, double *, int,
                                                         cudaStream_t);
template cudaError_t launch_gather_rows<int64_t, int32_t>(int64_t, const int32_t *,
                                                          const int64_t *, int64_t *, int,
                                                          cudaStream_t);
template cudaError_t launch_gather_rows<int64_t, int64_t>(int64_t, const int64_t *,
                                                          const int64_t *, int64_t *, int,
                                                          cudaStream_t);
template cudaError_t launch_gather_rows<int32_t, int32_t>(int64_t, const int32_t *,
                                                          const int32_t *, int32_t *, int,
                                                          cudaStream_t);
template cudaError_t launch_gather_rows<int32_t, int64_t>(int64_t, const int64_t *,
                                                          const int32_t *, int32_t *, int,
                                                          cudaStream_t);

cudaError_t launch_invert(int64_t n, const int32_t *perm, int32_t *inv, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  invert_kernel<<<blocks_for(n), 256, 0, s>>>(n, perm, inv);
  return cudaGetLastError();
}

cudaError_t launch_map_index(int64_t n_idx, const int32_t *in, const int32_t *slot, int64_t n,
                             int32_t *out, cudaStream_t s) {
  if (n_idx <= 0) return cudaSuccess;
  map_index_kernel<<<blocks_for(n_idx), 256, 0, s>>>(n_idx, in, slot, n, out);
  return cudaGetLastError();
}

}  // namespace nbi
