// Device functions shared by the host-driven kernels (one kernel per
// operation) and the fused device-resident block-step kernels, so that both
// paths perform the same arithmetic in the same order and give the same bits.
//
// Predictor / corrector after Makino & Aarseth (1992); time-step criterion
// Aarseth (1985), cited in the paper's Sec. 2; block (individual) time steps,
// paper Sec. 2, strategy (ii).  Not part of the public C ABI.
#pragma once

#include "nb_internal.cuh"

namespace nbi {
namespace dev {

constexpr double kTick = 1.0 / static_cast<double>(1 << kTicksLog2);

// Taylor predictor to dt: x + dt (v + dt/2 (a + dt/3 j)),  v + dt (a + dt/2 j).
__device__ __forceinline__ void predict_pos_vel(const double *x, const double *v,
                                                const double *a, const double *jk,
                                                int64_t i, double dt, double xp[3],
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

// Scalar and packed (two lanes per instruction, sm_100+ f32x2) FP32 ops
// with identical per-lane IEEE round-to-nearest results, so the scalar and
// packed kernels give bit-identical sums.
template <class V>
struct VOps;
template <>
struct VOps<float> {
  static constexpr int W = 1;
  static __device__ __forceinline__ float bc(float s) { return s; }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
  template <int MASK>
  static __device__ __forceinline__ float rsq(float r2) {
    if (MASK) return r2 > 0.f ? rsqrtf(r2) : 0.f;
    return rsqrtf(r2);
  }
  // 1/r2 from the MUFU pipe (PTX rcp.approx.ftz.f32, the hardware's
  // approximate reciprocal) instead of rinv * rinv on the FMA pipe
  static __device__ __forceinline__ float rcp(float r2) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
    return y;
  }
  static __device__ __forceinline__ float lane(float a, int) { return a; }
  static __device__ __forceinline__ void set(float &a, int, float s) { a = s; }
};
template <>
struct VOps<float2> {
  static constexpr int W = 2;
  static __device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
  }
  template <int MASK>
  static __device__ __forceinline__ float2 rsq(float2 r2) {
    return make_float2(VOps<float>::rsq<MASK>(r2.x), VOps<float>::rsq<MASK>(r2.y));
  }
  static __device__ __forceinline__ float2 rcp(float2 r2) {
    return make_float2(VOps<float>::rcp(r2.x), VOps<float>::rcp(r2.y));
  }
  static __device__ __forceinline__ float lane(float2 a, int w) { return w ? a.y : a.x; }
  static __device__ __forceinline__ void set(float2 &a, int w, float s) {
    if (w)
      a.y = s;
    else
      a.x = s;
  }
};

// FP64 <-> FP32 conversions on the integer pipe.  This part's FP64 pipe
// retires one warp instruction per ~68 cycles per scheduler and a
// conversion occupies it like an FMA, while these are a dozen integer
// operations.  Both are bit-identical to the hardware conversions; values
// whose result would not be a normal number take the hardware path.
//
// Round-to-nearest-even double -> float (IEEE 754 binary64 -> binary32).
__device__ __forceinline__ float d2f_rn(double d) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  const int e = static_cast<int>((b >> 52) & 0x7ff) - 1023 + 127;
  if (e < 1 || e > 254) return __double2float_rn(d);  // zero, subnormal, out of range
  const unsigned long long m = b & ((1ull << 52) - 1);
  const unsigned long long rem = m & ((1ull << 29) - 1);  // the 29 dropped bits
  unsigned int bits = (static_cast<unsigned int>(e) << 23) | static_cast<unsigned int>(m >> 29);
  // round half to even; a carry out of the mantissa steps the exponent,
  // as it should (up to infinity past the largest float)
  if (rem > (1ull << 28) || (rem == (1ull << 28) && (bits & 1u))) bits += 1u;
  bits |= static_cast<unsigned int>(b >> 32) & 0x80000000u;
  return __uint_as_float(bits);
}

// Exact float -> double.
__device__ __forceinline__ double f2d(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xffu;
  if (e == 0u || e == 255u) return static_cast<double>(f);  // zero, subnormal, inf, NaN
  const unsigned long long b = (static_cast<unsigned long long>(u & 0x80000000u) << 32) |
                               (static_cast<unsigned long long>(e - 127u + 1023u) << 52) |
                               (static_cast<unsigned long long>(u & 0x7fffffu) << 29);
  return __longlong_as_double(static_cast<long long>(b));
}

// j-records of particle i at the predicted (xp, vp): FP32 position (the
// high word in DS) + mass, DS low words, FP32 velocity.  Returns the first
// and the low words through *lo (zero in FP32).
__device__ __forceinline__ float4 store_records(int64_t i, const double xp[3],
                                                const double vp[3], double m, int prec,
                                                float4 *__restrict__ jhi,
                                                float4 *__restrict__ jlo,
                                                float4 *__restrict__ jvel, float4 *lo) {
  const float hx = d2f_rn(xp[0]);
  const float hy = d2f_rn(xp[1]);
  const float hz = d2f_rn(xp[2]);
  const float4 h = make_float4(hx, hy, hz, d2f_rn(m));
  jhi[i] = h;
  float4 l = make_float4(0.f, 0.f, 0.f, 0.f);
  if (prec) {
    l = make_float4(d2f_rn(xp[0] - f2d(hx)), d2f_rn(xp[1] - f2d(hy)), d2f_rn(xp[2] - f2d(hz)),
                    0.f);
    jlo[i] = l;
  }
  jvel[i] = make_float4(d2f_rn(vp[0]), d2f_rn(vp[1]), d2f_rn(vp[2]), 0.f);
  *lo = l;
  return h;
}

// Frame of one tile of kJT records (called by all kJT threads of a CTA,
// thread t holding record j = tile * kJT + t): the bounding box of the
// high words, its FP32 centre O_t, half-widths and radius R_t into
// tinfo[2 tile], tinfo[2 tile + 1], and every record's position relative
// to O_t into jrel.  The half-widths cover the box about O_t, the low
// words (below half an ulp of the high word) and the rounding of O_t.
__device__ __forceinline__ void tile_frame(int64_t tile, int64_t j, bool real, float4 h,
                                           float4 l, float4 *__restrict__ jrel,
                                           float4 *__restrict__ tinfo) {
  __shared__ float smn[3][kJT / 32], smx[3][kJT / 32];
  __shared__ float4 s_o;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
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
      const float big = fmaxf(fabsf(a), fabsf(b));
      hw[c] = fmaxf(o[c] - a, b - o[c]) * (1.0f + 1.0e-6f) + big * 1.2e-7f;
      r2 = fmaf(hw[c], hw[c], r2);
    }
    const float R = sqrtf(r2) * (1.0f + 1.0e-6f);
    tinfo[2 * tile] = make_float4(o[0], o[1], o[2], R);
    tinfo[2 * tile + 1] = make_float4(hw[0], hw[1], hw[2], 0.f);
    s_o = make_float4(o[0], o[1], o[2], 0.f);
  }
  __syncthreads();
  if (real) {
    const float4 o = s_o;
    jrel[j] = make_float4((h.x - o.x) + l.x, (h.y - o.y) + l.y, (h.z - o.z) + l.z, h.w);
  } else {
    jrel[j] = make_float4(1.0e15f, 1.0e15f, 1.0e15f, 0.f);
  }
}

// Unsigned division and remainder, in 32 bits when both operands fit (a
// 64-bit division is a long instruction sequence; the result is the same).
__host__ __device__ __forceinline__ uint64_t udiv(uint64_t a, uint64_t b) {
  if (((a | b) >> 32) == 0) return static_cast<uint32_t>(a) / static_cast<uint32_t>(b);
  return a / b;
}
__host__ __device__ __forceinline__ uint64_t umod(uint64_t a, uint64_t b) {
  if (((a | b) >> 32) == 0) return static_cast<uint32_t>(a) % static_cast<uint32_t>(b);
  return a % b;
}

// CTA owning unit u of U units split over P CTAs (ranges [U p / P, U (p+1) / P)).
__host__ __device__ __forceinline__ int owner_of(uint64_t u, uint64_t U, int P) {
  return static_cast<int>(udiv((u + 1) * static_cast<uint64_t>(P) - 1, U));
}

// Split-precision ("double-single") arithmetic on the FP32 pipe: a value
// is the unevaluated sum hi + lo of two floats.  The partial sums of split
// i-blocks and their reductions use it instead of FP64, whose pipe retires
// only ~1.6 lane-operations per SM clock on this part.
//
// Exact sum of two floats: s + e == a + b (Knuth's two-sum; the error is the
// same whichever operand comes first, so the pair sum below is commutative
// and a butterfly leaves the same total on every lane).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

// (ah + al) + (bh + bl) as a normalised pair (h, l).
__device__ __forceinline__ void ds_add_pair(float ah, float al, float bh, float bl, float &h,
                                            float &l) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// Particle i predicted by dt (ticks times 2^-20, exact in FP32), on the
// FP32 pipe in split precision, for its j-records:
//   x_p = x + dt v + dt^2 (a/2 + dt j/6),   v_p = v + dt a + dt^2 j/2.
// x and v are split into FP32 pairs hi + lo (the FP64 subtraction of the
// rounded high word is exact); dt v_hi is formed exactly as the FP32
// product plus its FMA rounding error; the low words and the a and j terms,
// smaller than dt v by about dt over the particle's dynamical time, are
// summed in FP32; a two-sum adds the increment to the position pair.  The
// position error is a few ulps of the a and j terms (~2^-24 |dt^2 a|),
// far below the FP32 rounding of a pair difference; the velocity is
// rounded to FP32 as the records store it.
// The predictor takes the state as its FP32 split (PSplit): per component
// the high and low words of x and v and a, j rounded to FP32.  The fused
// block steps keep this split beside the FP64 state (the corrector writes
// it), so that predicting all N particles each step is FP32 work only.
struct PSplit {
  float x0[3], x1[3], v0[3], v1[3], a[3], j[3];
};

__device__ __forceinline__ void split_state(const double xs[3], const double vs[3],
                                            const double as[3], const double js[3],
                                            PSplit &S) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    S.x0[c] = d2f_rn(xs[c]);
    S.x1[c] = d2f_rn(xs[c] - f2d(S.x0[c]));
    S.v0[c] = d2f_rn(vs[c]);
    S.v1[c] = d2f_rn(vs[c] - f2d(S.v0[c]));
    S.a[c] = d2f_rn(as[c]);
    S.j[c] = d2f_rn(js[c]);
  }
}

// Storage of the split: four float4 (sp4[4 i .. 4 i + 3]) and one float2
// (sp2[i]) per particle, in the order x0, x1, v0, v1, a, j.
__device__ __forceinline__ void store_split(int64_t i, const PSplit &S, float4 *sp4,
                                            float2 *sp2) {
  sp4[4 * i + 0] = make_float4(S.x0[0], S.x0[1], S.x0[2], S.x1[0]);
  sp4[4 * i + 1] = make_float4(S.x1[1], S.x1[2], S.v0[0], S.v0[1]);
  sp4[4 * i + 2] = make_float4(S.v0[2], S.v1[0], S.v1[1], S.v1[2]);
  sp4[4 * i + 3] = make_float4(S.a[0], S.a[1], S.a[2], S.j[0]);
  sp2[i] = make_float2(S.j[1], S.j[2]);
}

__device__ __forceinline__ void load_split(int64_t i, const float4 *__restrict__ sp4,
                                           const float2 *__restrict__ sp2, PSplit &S) {
  const float4 q0 = sp4[4 * i + 0];
  const float4 q1 = sp4[4 * i + 1];
  const float4 q2 = sp4[4 * i + 2];
  const float4 q3 = sp4[4 * i + 3];
  const float2 q4 = sp2[i];
  S.x0[0] = q0.x; S.x0[1] = q0.y; S.x0[2] = q0.z; S.x1[0] = q0.w;
  S.x1[1] = q1.x; S.x1[2] = q1.y; S.v0[0] = q1.z; S.v0[1] = q1.w;
  S.v0[2] = q2.x; S.v1[0] = q2.y; S.v1[1] = q2.z; S.v1[2] = q2.w;
  S.a[0] = q3.x; S.a[1] = q3.y; S.a[2] = q3.z; S.j[0] = q3.w;
  S.j[1] = q4.x; S.j[2] = q4.y;
}

__device__ __forceinline__ void predict_split(const PSplit &S, float dt, float xh[3],
                                              float xl[3], float vp[3]) {
  const float h2 = 0.5f * dt, h3 = dt * (1.0f / 3.0f);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float x0 = S.x0[c], x1 = S.x1[c];
    const float v0 = S.v0[c], v1 = S.v1[c];
    const float ac = S.a[c], jc = S.j[c];
    const float p = dt * v0;
    const float pe = fmaf(dt, v0, -p);  // dt v0 = p + pe exactly
    const float q = fmaf(dt, v1, pe) + dt * (h2 * fmaf(h3, jc, ac));
    float s, e;
    two_sum(x0, p, s, e);
    e = __fadd_rn(e, __fadd_rn(x1, q));
    const float hh = __fadd_rn(s, e);
    xh[c] = hh;
    xl[c] = __fsub_rn(e, __fsub_rn(hh, s));
    vp[c] = v0 + (v1 + dt * fmaf(h2, jc, ac));
  }
}

// (predict_ds_vals takes the particle's loaded state, predict_ds loads it.)
__device__ __forceinline__ void predict_ds_vals(const double xs[3], const double vs[3],
                                                const double as[3], const double js[3],
                                                float dt, float xh[3], float xl[3],
                                                float vp[3]) {
  PSplit S;
  split_state(xs, vs, as, js, S);
  predict_split(S, dt, xh, xl, vp);
}

__device__ __forceinline__ void predict_ds(const double *__restrict__ x,
                                           const double *__restrict__ v,
                                           const double *__restrict__ a,
                                           const double *__restrict__ jk, int64_t i, float dt,
                                           float xh[3], float xl[3], float vp[3]) {
  double xs[3], vs[3], as[3], js[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    xs[c] = x[3 * i + c];
    vs[c] = v[3 * i + c];
    as[c] = a[3 * i + c];
    js[c] = jk[3 * i + c];
  }
  predict_ds_vals(xs, vs, as, js, dt, xh, xl, vp);
}

// j-records of particle i from a split-precision prediction: high words and
// mass, low words (DS only), FP32 velocity.  Returns the first and the low
// words through *lo (zero in FP32).
__device__ __forceinline__ float4 store_records_ds(int64_t i, const float xh[3],
                                                   const float xl[3], const float vp[3],
                                                   double m, int prec,
                                                   float4 *__restrict__ jhi,
                                                   float4 *__restrict__ jlo,
                                                   float4 *__restrict__ jvel, float4 *lo) {
  const float4 h = make_float4(xh[0], xh[1], xh[2], d2f_rn(m));
  jhi[i] = h;
  float4 l = make_float4(0.f, 0.f, 0.f, 0.f);
  if (prec) {
    l = make_float4(xl[0], xl[1], xl[2], 0.f);
    jlo[i] = l;
  }
  jvel[i] = make_float4(vp[0], vp[1], vp[2], 0.f);
  *lo = l;
  return h;
}

// The pair (h, l) times G in FP64.
__device__ __forceinline__ double ds_to_double(float h, float l, double G) {
  return G * (f2d(h) + f2d(l));
}

// Sum of the split-precision partial segments (float2 hi, lo) of entry kk
// of split i-block ib, held by CTAs plo..phi: lanes stride over the CTAs
// (ascending within a lane) and meet by a butterfly, so every lane returns
// the same total, in an order fixed by the split.  Called by a full warp.
__device__ __forceinline__ void fixup_warp(const float2 *__restrict__ part, uint64_t ib,
                                           int kk, int plo, int phi, uint64_t U, int P,
                                           uint64_t n_jt, int BI, int lane, float h[6],
                                           float l[6]) {
#pragma unroll
  for (int c = 0; c < 6; ++c) h[c] = l[c] = 0.f;
  // slot 1 (a CTA's second segment) only for the first CTA, and only when
  // its range starts before the i-block
  const int slot0 =
      udiv(U * static_cast<uint64_t>(plo), static_cast<uint64_t>(P)) == ib * n_jt ? 0 : 1;
  for (int p = plo + lane; p <= phi; p += 32) {
    const int slot = p == plo ? slot0 : 0;
    const float2 *src = part + static_cast<size_t>(p * 2 + slot) * 6 * BI;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float2 w = src[static_cast<size_t>(c) * BI + kk];
      ds_add_pair(h[c], l[c], w.x, w.y, h[c], l[c]);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float oh = __shfl_xor_sync(0xffffffffu, h[c], off);
      const float ol = __shfl_xor_sync(0xffffffffu, l[c], off);
      ds_add_pair(h[c], l[c], oh, ol, h[c], l[c]);
    }
}

__device__ __forceinline__ double dot3(const double u[3]) {
  return u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
}

__device__ __forceinline__ double norm3(const double u[3]) { return sqrt(dot3(u)); }

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

// Level of the Aarseth step dt = sqrt(q), q = N / D >= 0, without forming
// q or dt: floor(log2 q) = e_N - e_D - [f_N < f_D] exactly (N = f_N 2^e_N,
// D = f_D 2^e_D, f in [1, 2)), and the largest 2^-lev <= dt has
// lev = -floor(floor(log2 q) / 2).  N and D are FP32 (subnormals are flushed
// to zero); special values: q = 0 or undefined, and an overflowed N, give
// lev_max and a clamp; D = 0 (q = inf) gives lev_min.
__device__ __forceinline__ int level_from_ratio_f(float N, float D, int lev_min, int lev_max,
                                                  int *clamped) {
  if (isnan(N) || isnan(D) || !(N > 0.f) || isinf(D)) {  // q = 0 or undefined
    *clamped = 1;
    return lev_max;
  }
  if (isinf(N)) {  // an FP32 overflow of the numerator: take the smallest step
    *clamped = 1;
    return lev_max;
  }
  if (!(D > 0.f)) return lev_min;  // q = inf
  const int bN = __float_as_int(N), bD = __float_as_int(D);
  const int F = ((bN >> 23) & 0xff) - ((bD >> 23) & 0xff) -
                ((bN & 0x7fffff) < (bD & 0x7fffff) ? 1 : 0);
  int lev = -(F >> 1);
  if (lev > lev_max) {
    *clamped = 1;
    lev = lev_max;
  }
  if (lev < lev_min) lev = lev_min;
  return lev;
}

// 2^k as a float, |k| <= 126 (exact).
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// |u| in FP32 without overflow or underflow of the squares: the components
// are scaled by a power of two near 1 / max|u_c| first (exact).
__device__ __forceinline__ float norm3f(const float u[3]) {
  const float m = fmaxf(fabsf(u[0]), fmaxf(fabsf(u[1]), fabsf(u[2])));
  if (isnan(u[0] + u[1] + u[2])) return u[0] + u[1] + u[2];
  if (!(m > 0.f) || isinf(m)) return m;
  int e = ((__float_as_int(m) >> 23) & 0xff) - 127;
  e = e < -125 ? -125 : (e > 125 ? 125 : e);
  const float sc = pow2f(-e);
  const float x = u[0] * sc, y = u[1] * sc, z = u[2] * sc;
  return sqrtf(fmaf(x, x, fmaf(y, y, z * z))) * pow2f(e);
}

// Coefficients of the Hermite corrector for one step dt on the FP32 pipe
// (the FP64 pipe of this part retires one warp instruction per ~68 cycles
// per scheduler).  dt is a power of two of ticks (2^-20 .. 2^0), so 1/dt is
// exact and so is every coefficient.
struct HermCoefF {
  float dt;
  float s_da, s_j0, s_jn;  // snap = s_da da + s_j0 j0 + s_jn jn
  float c_da, c_j;         // crackle = c_da da + c_j (j0 + jn)
};

__device__ __forceinline__ HermCoefF herm_coef_f(float dt, float idt) {
  HermCoefF K;
  const float idt2 = idt * idt;
  K.dt = dt;
  K.s_da = -6.f * idt2;
  K.s_j0 = -4.f * idt;
  K.s_jn = -2.f * idt;
  K.c_da = 12.f * idt2 * idt;
  K.c_j = 6.f * idt2;
  return K;
}

// One component of the Hermite-4 step from (x0, v0, a0, j0) with the new
// force (an, jn): the second and third derivatives of a at the start of the
// step,
//   snap = (-6 da - dt (4 j0 + 2 jn)) / dt^2,
//   crackle = (12 da + 6 dt (j0 + jn)) / dt^3,   da = a0 - an,
// the corrected
//   x1 = x0 + dt (v0 + dt (a0/2 + dt (j0/6 + dt (snap/24 + dt crackle/120)))),
//   v1 = v0 + dt (a0 + dt (j0/2 + dt (snap/6 + dt crackle/24))),
// and the derivatives at the end of the step for the step criterion,
// a2 = snap + dt crackle, a3 = crackle.  (This is the predictor's Taylor
// polynomial plus the dt^4 and dt^5 terms.)  The terms of x0, v0, a0 and
// the difference da are FP64, so that a smooth external field, which can
// dominate a, keeps full precision; the terms of j0, snap and crackle,
// smaller than the a0 term by about dt over the dynamical time, are
// evaluated on the FP32 pipe (6 FP64 instructions per component instead
// of 17: the FP64 pipe of this part retires one warp instruction per ~68
// cycles per scheduler).
__device__ __forceinline__ void herm_component_f(const HermCoefF &K, double dtd, double x0,
                                                 double v0, double a0, float j0, double an,
                                                 float jn, double &x1, double &v1, float &a2,
                                                 float &a3) {
  const float dt = K.dt;
  const float da = d2f_rn(a0 - an);
  const float snap = fmaf(K.s_da, da, fmaf(K.s_j0, j0, K.s_jn * jn));
  const float crackle = fmaf(K.c_da, da, K.c_j * (j0 + jn));
  const float qx =
      dt * fmaf(dt, fmaf(dt, crackle * (1.f / 120.f), snap * (1.f / 24.f)), j0 * (1.f / 6.f));
  const float qv = dt * fmaf(dt, fmaf(dt, crackle * (1.f / 24.f), snap * (1.f / 6.f)), 0.5f * j0);
  x1 = fma(dtd, fma(dtd, fma(0.5, a0, f2d(qx)), v0), x0);
  v1 = fma(dtd, a0 + f2d(qv), v0);
  a2 = fmaf(crackle, dt, snap);
  a3 = crackle;
}

// External Galactic field of Allen & Santillan (1991) at position x, FP64:
// acceleration added into a, and, when v and jk are set, its time
// derivative along v (the jerk) added into jk; the potential into *phi when
// phi is set.  With d = x - centre, r = |d|, R^2 = d_x^2 + d_y^2, z = d_z:
//   bulge (Plummer)          Phi = -G M_b / sqrt(r^2 + b_b^2)
//   disk (Miyamoto-Nagai)    Phi = -G M_d / D, D^2 = R^2 + (a_d + zeta)^2,
//                            zeta = sqrt(z^2 + b_d^2)
//   halo                     M(r) = M_h q^gamma / (1 + q^(gamma-1)), q = r / a_h,
//                            held at M(r_cut) beyond r_cut; force -G M(r) d / r^3;
//                            Phi = -G M(r) / r - G M_h / ((gamma-1) a_h) (F(q_cut) - F(q))
//                            inside the cut, F(q) = ln(1 + q^(gamma-1))
//                            - (gamma-1) / (1 + q^(gamma-1)); -G M(r_cut) / r beyond.
// Jerk terms: bulge -G M_b (v / s^3 - 3 (d.v) d / s^5), s^2 = r^2 + b_b^2;
// disk -G M_d ((v_x, v_y, g') / D^3 - 3 D' (d_x, d_y, g) / D^4) with
// g = z (a_d + zeta) / zeta, g' = v_z (1 + a_d b_d^2 / zeta^3),
// D' = (d_x v_x + d_y v_y + (a_d + zeta) z v_z / zeta) / D; halo
// -G (M v / r^3 + (M' - 3 M / r) (d.v) d / r^4), M' = dM/dr (0 beyond the cut).
__device__ __forceinline__ void ext_field(const ExtField &E, const double x[3],
                                          const double *v, double a[3], double *jk,
                                          double *phi) {
  const double dx = x[0] - E.c[0], dy = x[1] - E.c[1], dz = x[2] - E.c[2];
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double r = sqrt(r2);
  const bool wj = v != nullptr && jk != nullptr;
  const double vx = wj ? v[0] : 0.0, vy = wj ? v[1] : 0.0, vz = wj ? v[2] : 0.0;
  const double dv = dx * vx + dy * vy + dz * vz;
  double ph = 0.0;
  {
    const double s2 = r2 + E.bb * E.bb;
    const double s = sqrt(s2);
    const double f = E.G * E.mb / (s2 * s);
    a[0] -= f * dx;
    a[1] -= f * dy;
    a[2] -= f * dz;
    ph -= E.G * E.mb / s;
    if (wj) {
      const double c = 3.0 * dv / s2;
      jk[0] -= f * (vx - c * dx);
      jk[1] -= f * (vy - c * dy);
      jk[2] -= f * (vz - c * dz);
    }
  }
  {
    const double zeta = sqrt(dz * dz + E.bd * E.bd);
    const double w = E.ad + zeta;
    const double D2 = dx * dx + dy * dy + w * w;
    const double D = sqrt(D2);
    const double f = E.G * E.md / (D2 * D);
    const double g = dz * w / zeta;
    a[0] -= f * dx;
    a[1] -= f * dy;
    a[2] -= f * g;
    ph -= E.G * E.md / D;
    if (wj) {
      const double Ddot = (dx * vx + dy * vy + w * dz * vz / zeta) / D;
      const double gdot = vz * (1.0 + E.ad * E.bd * E.bd / (zeta * zeta * zeta));
      const double c = 3.0 * Ddot / D;
      jk[0] -= f * (vx - c * dx);
      jk[1] -= f * (vy - c * dy);
      jk[2] -= f * (gdot - c * g);
    }
  }
  {
    const double rr = r < E.rcut ? r : E.rcut;
    const double q = rr / E.ah;
    const double u = pow(q, E.gam - 1.0);
    const double Mr = E.mh * q * u / (1.0 + u);
    if (r > 0.0) {
      const double f = E.G * Mr / (r2 * r);
      a[0] -= f * dx;
      a[1] -= f * dy;
      a[2] -= f * dz;
      if (wj) {
        const double Mp = r < E.rcut ? E.mh * u * (E.gam + u) / ((1.0 + u) * (1.0 + u) * E.ah)
                                     : 0.0;
        const double c = E.G * (Mp - 3.0 * Mr / r) * dv / (r2 * r2);
        jk[0] -= f * vx + c * dx;
        jk[1] -= f * vy + c * dy;
        jk[2] -= f * vz + c * dz;
      }
    }
    if (phi) {
      if (r < E.rcut) {
        const double uc = pow(E.rcut / E.ah, E.gam - 1.0);
        const double Fc = log(1.0 + uc) - (E.gam - 1.0) / (1.0 + uc);
        const double Fq = log(1.0 + u) - (E.gam - 1.0) / (1.0 + u);
        ph += (r > 0.0 ? -E.G * Mr / r : 0.0) - E.G * E.mh / ((E.gam - 1.0) * E.ah) * (Fc - Fq);
      } else {
        ph -= E.G * Mr / r;
      }
      *phi = ph;
    }
  }
}

// State of one particle as the corrector reads it (loaded ahead of the
// corrector so that the loads overlap other work).
struct PState {
  double x[3], v[3], a[3], j[3];
  int64_t t;
  int lev;
};

__device__ __forceinline__ void load_state(int64_t i, const double *__restrict__ x,
                                           const double *__restrict__ v,
                                           const double *__restrict__ a,
                                           const double *__restrict__ jk,
                                           const int64_t *__restrict__ t_tick,
                                           const int32_t *__restrict__ lev, PState &st) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    st.x[c] = x[3 * i + c];
    st.v[c] = v[3 * i + c];
    st.a[c] = a[3 * i + c];
    st.j[c] = jk[3 * i + c];
  }
  st.t = t_tick[i];
  st.lev = lev[i];
}

// The field's acceleration and jerk at the predictor's position and
// velocity (the expression of predict_pos_vel) added into an, jn.  Not
// inlined: the corrector kernels keep their registers when no field is set.
static __device__ __noinline__ void ext_at_prediction(const ExtField &E, const PState &st,
                                                      double dt, double h2, double h3,
                                                      double an[3], double jn[3]) {
  double xp[3], vp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    xp[c] = st.x[c] + dt * (st.v[c] + h2 * (st.a[c] + h3 * st.j[c]));
    vp[c] = st.v[c] + dt * (st.a[c] + h2 * st.j[c]);
  }
  ext_field(E, xp, vp, an, jn, nullptr);
}

// Hermite corrector, step criterion and new level of particle i (state st)
// with its new pair force an, jn at t_next, plus, when ext is on, the
// external field's acceleration and jerk at the predicted position and
// velocity.  With lev_cnt set, a change of level moves the particle between
// the per-level counts.
__device__ __forceinline__ void correct_vals(
    int64_t i, const PState &st, const double an_pair[3], const double jn_pair[3],
    int64_t t_next, double *__restrict__ x, double *__restrict__ v, double *__restrict__ a,
    double *__restrict__ jk, int64_t *__restrict__ t_tick, int32_t *__restrict__ lev,
    double eta, int lev_min, int lev_max, int block_steps, unsigned long long *n_clamped,
    int64_t *lev_cnt, const ExtField *ext = nullptr, float4 *sp4 = nullptr,
    float2 *sp2 = nullptr) {
  const int64_t dtk = t_next - st.t;
  const double dt = static_cast<double>(dtk) * kTick;
  const double h2 = 0.5 * dt, h3 = dt * (1.0 / 3.0);
  double an3[3] = {an_pair[0], an_pair[1], an_pair[2]};
  double jn3[3] = {jn_pair[0], jn_pair[1], jn_pair[2]};
  if (ext && ext->on) ext_at_prediction(*ext, st, dt, h2, h3, an3, jn3);
  // A due particle's step is a power of two of ticks, so 1/dt is a power
  // of two, built exactly from the exponent (no division).
  const float dtf = static_cast<float>(dtk) * static_cast<float>(kTick);
  const float idt = (dtk > 0 && (dtk & (dtk - 1)) == 0)
                        ? pow2f(kTicksLog2 - (63 - __clzll(dtk)))
                        : 1.f / dtf;
  const HermCoefF K = herm_coef_f(dtf, idt);
  float anf[3], jnf[3], a2e[3], a3e[3];
  double xn[3], vn[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    anf[c] = d2f_rn(an3[c]);
    jnf[c] = d2f_rn(jn3[c]);
    herm_component_f(K, dt, st.x[c], st.v[c], st.a[c], d2f_rn(st.j[c]), an3[c], jnf[c], xn[c],
                     vn[c], a2e[c], a3e[c]);
    x[3 * i + c] = xn[c];
    v[3 * i + c] = vn[c];
    a[3 * i + c] = an3[c];
    jk[3 * i + c] = jn3[c];
  }
  t_tick[i] = t_next;
  if (sp4) {
    // the predictor's FP32 split of the new state (a, j: the values above)
    PSplit S;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      S.x0[c] = d2f_rn(xn[c]);
      S.x1[c] = d2f_rn(xn[c] - f2d(S.x0[c]));
      S.v0[c] = d2f_rn(vn[c]);
      S.v1[c] = d2f_rn(vn[c] - f2d(S.v0[c]));
      S.a[c] = anf[c];
      S.j[c] = jnf[c];
    }
    store_split(i, S, sp4, sp2);
  }
  if (block_steps) {
    // Aarseth's criterion dt^2 = eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2)
    // in FP32, as numerator and denominator; the level comes from their
    // exponents (it only has to place dt between powers of two)
    const float na = norm3f(anf), nj = norm3f(jnf), n2 = norm3f(a2e), n3 = norm3f(a3e);
    const float N = static_cast<float>(eta) * fmaf(na, n2, nj * nj);
    const float D = fmaf(nj, n3, n2 * n2);
    int cl = 0;
    const int want = level_from_ratio_f(N, D, lev_min, lev_max, &cl);
    if (cl) atomicAdd(n_clamped, 1ull);
    const int old = st.lev;
    int nl = old;
    if (want >= old) {
      nl = want;
    } else if (old - 1 >= lev_min) {
      const int64_t period = static_cast<int64_t>(1) << (kTicksLog2 - (old - 1));
      if (t_next % period == 0) nl = old - 1;
    }
    lev[i] = nl;
    if (lev_cnt && nl != old) {
      atomicAdd(reinterpret_cast<unsigned long long *>(lev_cnt + old),
                static_cast<unsigned long long>(-1ll));
      atomicAdd(reinterpret_cast<unsigned long long *>(lev_cnt + nl), 1ull);
    }
  }
}

template <typename T>
__device__ __forceinline__ T sel3(const T u[3], int c) {
  return c == 0 ? u[0] : (c == 1 ? u[1] : u[2]);
}

// correct_vals on three lanes of a warp, lane base + c taking component c
// of the Hermite update (the same arithmetic per component): every lane of
// the triple holds the particle's whole state and new pair force, the
// derivatives at the end of the step and the split words meet by shuffles,
// and lane base writes the time, the step criterion's level and the split.
// The FP64 and integer-pipe work per warp is a third of one lane's doing
// all three components.  mask: the lanes of the warp that call it (whole
// triples).
__device__ __forceinline__ void correct_vals3(
    int c, unsigned mask, int base, int64_t i, const PState &st, const double an_pair[3],
    const double jn_pair[3], int64_t t_next, double *__restrict__ x, double *__restrict__ v,
    double *__restrict__ a, double *__restrict__ jk, int64_t *__restrict__ t_tick,
    int32_t *__restrict__ lev, double eta, int lev_min, int lev_max, int block_steps,
    unsigned long long *n_clamped, int64_t *lev_cnt, const ExtField *ext, float4 *sp4,
    float2 *sp2) {
  const int64_t dtk = t_next - st.t;
  const double dt = static_cast<double>(dtk) * kTick;
  const double h2 = 0.5 * dt, h3 = dt * (1.0 / 3.0);
  double an3[3] = {an_pair[0], an_pair[1], an_pair[2]};
  double jn3[3] = {jn_pair[0], jn_pair[1], jn_pair[2]};
  if (ext && ext->on) ext_at_prediction(*ext, st, dt, h2, h3, an3, jn3);
  const float dtf = static_cast<float>(dtk) * static_cast<float>(kTick);
  const float idt = (dtk > 0 && (dtk & (dtk - 1)) == 0)
                        ? pow2f(kTicksLog2 - (63 - __clzll(dtk)))
                        : 1.f / dtf;
  const HermCoefF K = herm_coef_f(dtf, idt);
  const double anc = sel3(an3, c), jnc = sel3(jn3, c);
  const float jncf = d2f_rn(jnc);
  double xn, vn;
  float a2c, a3c;
  herm_component_f(K, dt, sel3(st.x, c), sel3(st.v, c), sel3(st.a, c), d2f_rn(sel3(st.j, c)),
                   anc, jncf, xn, vn, a2c, a3c);
  x[3 * i + c] = xn;
  v[3 * i + c] = vn;
  a[3 * i + c] = anc;
  jk[3 * i + c] = jnc;
  const float x0 = d2f_rn(xn), x1 = d2f_rn(xn - f2d(x0));
  const float v0 = d2f_rn(vn), v1 = d2f_rn(vn - f2d(v0));
  const float ancf = d2f_rn(anc);
  float anf[3], jnf[3], a2e[3], a3e[3], sx0[3], sx1[3], sv0[3], sv1[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    anf[q] = __shfl_sync(mask, ancf, base + q);
    jnf[q] = __shfl_sync(mask, jncf, base + q);
    a2e[q] = __shfl_sync(mask, a2c, base + q);
    a3e[q] = __shfl_sync(mask, a3c, base + q);
    sx0[q] = __shfl_sync(mask, x0, base + q);
    sx1[q] = __shfl_sync(mask, x1, base + q);
    sv0[q] = __shfl_sync(mask, v0, base + q);
    sv1[q] = __shfl_sync(mask, v1, base + q);
  }
  if (c != 0) return;
  t_tick[i] = t_next;
  if (sp4) {
    PSplit S;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      S.x0[q] = sx0[q];
      S.x1[q] = sx1[q];
      S.v0[q] = sv0[q];
      S.v1[q] = sv1[q];
      S.a[q] = anf[q];
      S.j[q] = jnf[q];
    }
    store_split(i, S, sp4, sp2);
  }
  if (block_steps) {
    const float na = norm3f(anf), nj = norm3f(jnf), n2 = norm3f(a2e), n3 = norm3f(a3e);
    const float N = static_cast<float>(eta) * fmaf(na, n2, nj * nj);
    const float D = fmaf(nj, n3, n2 * n2);
    int cl = 0;
    const int want = level_from_ratio_f(N, D, lev_min, lev_max, &cl);
    if (cl) atomicAdd(n_clamped, 1ull);
    const int old = st.lev;
    int nl = old;
    if (want >= old) {
      nl = want;
    } else if (old - 1 >= lev_min) {
      const int64_t period = static_cast<int64_t>(1) << (kTicksLog2 - (old - 1));
      if (t_next % period == 0) nl = old - 1;
    }
    lev[i] = nl;
    if (lev_cnt && nl != old) {
      atomicAdd(reinterpret_cast<unsigned long long *>(lev_cnt + old),
                static_cast<unsigned long long>(-1ll));
      atomicAdd(reinterpret_cast<unsigned long long *>(lev_cnt + nl), 1ull);
    }
  }
}

// The corrector of active entry k (particle act[k]) with its new force in
// a1, j1 (entry-indexed).
__device__ __forceinline__ void correct_one(
    int64_t k, const int32_t *__restrict__ act, int64_t t_next, double *__restrict__ x,
    double *__restrict__ v, double *__restrict__ a, double *__restrict__ jk,
    int64_t *__restrict__ t_tick, int32_t *__restrict__ lev, const double *__restrict__ a1,
    const double *__restrict__ j1, double eta, int lev_min, int lev_max, int block_steps,
    unsigned long long *n_clamped, int64_t *lev_cnt, const ExtField *ext = nullptr) {
  const int64_t i = act[k];
  PState st;
  load_state(i, x, v, a, jk, t_tick, lev, st);
  const double an[3] = {a1[3 * k], a1[3 * k + 1], a1[3 * k + 2]};
  const double jn[3] = {j1[3 * k], j1[3 * k + 1], j1[3 * k + 2]};
  correct_vals(i, st, an, jn, t_next, x, v, a, jk, t_tick, lev, eta, lev_min, lev_max,
               block_steps, n_clamped, lev_cnt, ext);
}

}  // namespace dev
}  // namespace nbi
