// Fixed-step symplectic integration (Sec. 2.2) of every particle on the
// device-resident FP64 state: the kick-drift-kick leapfrog (second order)
// and the sixth-order scheme, a symmetric composition of seven leapfrog
// steps of lengths w_k dt.  The forces come from the acceleration-only form
// of the force kernel (nb_force.cu) in the context's precision, plus, when
// the context has one, the external Galactic field of Sec. 2.1 (FP64, in
// the kick).
//
// One step of S stages with weights w_0..w_{S-1} runs, with the kicks
// between two drifts merged into one:
//   for k: v += (w_{k-1} + w_k) dt/2 a   (w_{-1} = 0; a = pair sum + field)
//          x += w_k dt v, j-records, tile frames
//          a = A(x)
//   v += w_{S-1} dt/2 a
// so a step takes S force evaluations and leaves x, v at the same instant.
#include "nb_device.cuh"

namespace nbi {
namespace {

// Yoshida (1990, Phys. Lett. A 150, 262), solution A: the first of the
// three sixth-order weight sets of Kinoshita, Yoshida & Nakai (1991,
// Table 1), the one Sec. 2.2 takes.  w0 = 1 - 2 (w1 + w2 + w3); the stages
// run w3 w2 w1 w0 w1 w2 w3.
constexpr double kY6W1 = -1.17767998417887100695;
constexpr double kY6W2 = 0.235573213359358133684;
constexpr double kY6W3 = 0.784513610477557263820;

// One CTA per 256-record tile, thread t on record j = tile * kJT + t:
// v += h (a + a_ext(x)) and x += d v in FP64 (each skipped when its factor
// is 0; a_ext only with the field on), then, with rec set, the particle's
// j-records and (split precision) the tile's frame for the far-field test
// of the force kernel.
__global__ void __launch_bounds__(kJT)
    kick_drift_kernel(int64_t n, double h, double d, int rec, const ExtField E,
                      const double *__restrict__ a, double *__restrict__ v,
                      double *__restrict__ x,
                      const double *__restrict__ m, int prec, float4 *__restrict__ jhi,
                      float4 *__restrict__ jlo, float4 *__restrict__ jvel,
                      float4 *__restrict__ jrel, float4 *__restrict__ tinfo) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * kJT + threadIdx.x;
  const bool real = j < n;
  float4 hr = make_float4(0.f, 0.f, 0.f, 0.f), lr = hr;
  if (real) {
    double xv[3], vv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      vv[c] = v[3 * j + c];
      xv[c] = x[3 * j + c];
    }
    if (h != 0.0) {
      double at[3] = {a[3 * j], a[3 * j + 1], a[3 * j + 2]};
      if (E.on) dev::ext_field(E, xv, nullptr, at, nullptr, nullptr);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        vv[c] = fma(h, at[c], vv[c]);
        v[3 * j + c] = vv[c];
      }
    }
    if (d != 0.0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        xv[c] = fma(d, vv[c], xv[c]);
        x[3 * j + c] = xv[c];
      }
    }
    if (rec) hr = dev::store_records(j, xv, vv, m[j], prec, jhi, jlo, jvel, &lr);
  } else if (rec) {
    hr = jhi[j];  // padding record (zero mass, far away)
  }
  if (rec && jrel) dev::tile_frame(blockIdx.x, j, real, hr, lr, jrel, tinfo);
}

__global__ void ext_add_kernel(int64_t n, const ExtField E, const double *__restrict__ x,
                               double *__restrict__ a) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xv[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  double av[3] = {a[3 * i], a[3 * i + 1], a[3 * i + 2]};
  dev::ext_field(E, xv, nullptr, av, nullptr, nullptr);
  for (int c = 0; c < 3; ++c) a[3 * i + c] = av[c];
}

// dst[k] = src[perm[k]] (gather) or dst[perm[k]] = src[k] (scatter) for
// rows of w doubles.
__global__ void permute_kernel(int64_t n, const int64_t *__restrict__ perm,
                               const double *__restrict__ src, double *__restrict__ dst, int w,
                               int scatter) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t p = perm[k];
  const int64_t from = scatter ? k : p, to = scatter ? p : k;
  for (int c = 0; c < w; ++c) dst[w * to + c] = src[w * from + c];
}

}  // namespace

cudaError_t launch_permute(int64_t n, const int64_t *perm, const double *src, double *dst,
                           int w, bool scatter, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  permute_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(n, perm, src, dst, w,
                                                                       scatter ? 1 : 0);
  return cudaGetLastError();
}

int symplectic_stages(int order, double *w) {
  if (order == 2) {
    w[0] = 1.0;
    return 1;
  }
  if (order == 6) {
    const double w0 = 1.0 - 2.0 * (kY6W1 + kY6W2 + kY6W3);
    const double s[7] = {kY6W3, kY6W2, kY6W1, w0, kY6W1, kY6W2, kY6W3};
    for (int k = 0; k < 7; ++k) w[k] = s[k];
    return 7;
  }
  return 0;
}

cudaError_t launch_kick_drift(int64_t n, int64_t n_jt, double h, double d, bool rec,
                              const ExtField &E, const double *a, double *v, double *x,
                              const double *m, int prec, float4 *jhi, float4 *jlo,
                              float4 *jvel, float4 *jrel, float4 *tinfo, cudaStream_t s) {
  if (n_jt <= 0) return cudaSuccess;
  kick_drift_kernel<<<static_cast<unsigned>(n_jt), kJT, 0, s>>>(
      n, h, d, rec ? 1 : 0, E, a, v, x, m, prec, jhi, jlo, jvel, jrel, tinfo);
  return cudaGetLastError();
}

cudaError_t launch_ext_add(int64_t n, const ExtField &E, const double *x, double *a,
                           cudaStream_t s) {
  if (n <= 0 || !E.on) return cudaSuccess;
  ext_add_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(n, E, x, a);
  return cudaGetLastError();
}

}  // namespace nbi
