// mcx_tracer.cuh -- the fused per-ray tracer (device code).
//
// One thread carries one ray from the source through every component of the
// instrument with the whole ray state in registers (McXtrace's sequential
// component model, arXiv 2410.08747 Sec. 1 and Sec. 2.2.2).  The component
// table sits in shared memory; the loop over components is uniform across a
// warp, so the per-component branch never diverges, only the alive predicate
// does.  Monitors are updated with global atomics (the race-free monitor
// update the paper's port needed, Sec. 2.2.2); per-component loss tallies are
// reduced per warp before touching shared memory.
//
// Two forms share this file:
//   plain (MODE 0)  every quantity in binary64;
//   mixed (MODE 1)  the ray is sampled and propagated in binary32 inside each
//                   component frame; the lab position, lab-to-local
//                   translations/rotations and monitor sums stay binary64.
// On GB300 a binary64 warp instruction occupies the FP64 pipe for ~64
// scheduler cycles, so the mixed form keeps binary64 arithmetic to the frame
// transforms themselves: conversions between the two formats on the ray's
// path are done exactly with integer bit operations, tallies are summed in
// compensated binary32, and a monitor hit's weight is widened once.
//
// Translation units that include this file are compiled with -fmad=false:
// every decision that sets a count (clip, bin, table cell) must round exactly
// as the operation sequence of the draw-and-arithmetic contract says, so
// nothing may be contracted into a fused multiply-add.  Explicit fma() appears
// only where a weight, never a count, depends on the result.
#pragma once

#ifdef __CUDACC_RTC__
// Compiled at run time for one instrument (mcx_jit.cu): no host headers.
#define CUDART_INF __longlong_as_double(0x7ff0000000000000LL)
#define CUDART_INF_F __int_as_float(0x7f800000)
#else
#include <cfloat>
#include <cmath>

#include <math_constants.h>
#endif

#include "mcx_internal.h"

namespace mcx {

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): per round (hi0, lo0) = M0 * c0,
// (hi1, lo1) = M1 * c2, c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), then
// the key advances by the Weyl constants.
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t& o0,
                                              uint32_t& o1, uint32_t& o2, uint32_t& o3) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // each 32 x 32 -> 64-bit product in one wide multiply
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  o0 = c0; o1 = c1; o2 = c2; o3 = c3;
}

// The random stream of one ray: counter (id lo, id hi, block, instrument),
// key (seed lo, seed hi); words are consumed in order, four per block.
struct RayStream {
  uint32_t c0, c1, c3, k0, k1, blk, left;
  uint32_t w0, w1, w2, w3;

  __device__ __forceinline__ void init(uint64_t id, uint32_t instr, uint64_t seed) {
    c0 = (uint32_t)id; c1 = (uint32_t)(id >> 32); c3 = instr;
    k0 = (uint32_t)seed; k1 = (uint32_t)(seed >> 32);
    blk = 0; left = 0;
  }
  __device__ __forceinline__ uint32_t next() {
    if (left == 0) {
      philox4x32_10(c0, c1, blk, c3, k0, k1, w0, w1, w2, w3);
      ++blk;
      left = 4;
    }
    const uint32_t r = w0;
    w0 = w1; w1 = w2; w2 = w3;
    --left;
    return r;
  }
};

// binary64 draw: top 53 bits of (hi << 32 | lo) from two consecutive words;
// binary32 draw: top 24 bits of one word.  Both exact, in [0, 1).
template <typename R> struct Uniform;
template <> struct Uniform<double> {
  __device__ __forceinline__ static double draw(RayStream& s) {
    const uint32_t lo = s.next();
    const uint32_t hi = s.next();
    const uint64_t v = ((uint64_t)hi << 32) | (uint64_t)lo;
    return (double)(v >> 11) * 0x1.0p-53;
  }
};
// The binary32 value (x >> 8) 2^-24 is built without a conversion instruction
// (those share GB300's slow FP64-class pipe): its top 23 bits become the
// significand of 1.f, from which 1 is subtracted exactly, and the 24th bit
// adds 2^-24 exactly.
template <> struct Uniform<float> {
  __device__ __forceinline__ static float draw(RayStream& s) {
    const uint32_t x = s.next();
    const float hi = __uint_as_float(0x3f800000u | (x >> 9)) - 1.0f;
    return hi + __uint_as_float(((x >> 8) & 1u) * 0x33800000u);
  }
};

// floor of a binary32 value in [0, 2^23) without a conversion instruction:
// adding 2^23 with rounding toward zero leaves the integer part in the
// significand's low bits.
__device__ __forceinline__ int trunc_small(float f) {
  return __float_as_int(__fadd_rz(f, 8388608.0f)) - 0x4b000000;
}
// The same floor as a binary32 value (FADD only).
__device__ __forceinline__ float floor_small(float f) {
  return __fadd_rz(f, 8388608.0f) - 8388608.0f;
}

// ------------------------------------------------------------------ math helpers
template <typename T> __device__ __forceinline__ T sqrt_rn(T x);
template <> __device__ __forceinline__ double sqrt_rn<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float sqrt_rn<float>(float x) { return sqrtf(x); }

// ------------------------------------------------------------------ Gaussian deviates
// The natural logarithm from IEEE operations in a fixed order, so that the
// Gaussian source's count-deciding draws are the same in every
// implementation of the contract (the device's own log is not correctly
// rounded): x = m 2^e with m in [sqrt(1/2), sqrt(2)] (exponent and
// significand from the bits, then one exact halving), f = (m - 1)/(m + 1),
// ln m = 2 f (1 + f^2/3 + f^4/5 + ...) by Horner to f^20 (binary64) or f^10
// (binary32), ln x = e ln 2 + ln m.  x must be positive and normal.
template <typename R>
__device__ __forceinline__ R ln_series(R x) {
  int e;
  R m;
  int K;
  if constexpr (sizeof(R) == 8) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    e = (int)((b >> 52) & 0x7ffull) - 1023;
    m = __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
    K = 10;
  } else {
    const unsigned b = __float_as_uint(x);
    e = (int)((b >> 23) & 0xffu) - 127;
    m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
    K = 5;
  }
  if (m > (R)1.4142135623730951) { m = m * (R)0.5; e += 1; }
  const R f = (m - (R)1) / (m + (R)1);
  const R f2 = f * f;
  R p = (R)1 / (R)(2 * K + 1);
  for (int k = K - 1; k >= 0; --k) p = p * f2 + (R)1 / (R)(2 * k + 1);
  return (R)e * (R)0.6931471805599453 + (R)2 * f * p;
}

// A pair of standard normal deviates by Marsaglia's polar method: pairs
// (a, b) = (2u - 1, 2u' - 1) of the ray's next draws until 0 < s = a a + b b
// < 1 (16 pairs at most, else (0, 0)), then (a, b) sqrt(-2 ln s / s).
template <typename R>
__device__ __forceinline__ void gauss_pair(RayStream& rs, R& z1, R& z2) {
  z1 = (R)0;
  z2 = (R)0;
  for (int t = 0; t < 16; ++t) {
    const R a = (R)2 * Uniform<R>::draw(rs) - (R)1;
    const R b = (R)2 * Uniform<R>::draw(rs) - (R)1;
    const R s = a * a + b * b;
    if (s < (R)1 && s > (R)0) {
      const R g = sqrt_rn<R>(((R)-2 * ln_series<R>(s)) / s);
      z1 = a * g;
      z2 = b * g;
      return;
    }
  }
}

// Weight-only arithmetic.  A path length through an analytic solid, a
// spectral weight or an attenuation factor never decides a count (clip, bin,
// table cell), so the binary32 form takes the hardware approximations here:
// division as a * (approximate 1/b) (__fdividef, 2 ulp), square root as an
// approximate hardware root, exp via exp2 (__expf); each is within a few
// 1e-7 relative of the correctly rounded value, two orders below the binary32
// tolerance stated for the mixed form.  The binary64 form keeps IEEE
// operations, and every count-deciding operation keeps them in both forms.
__device__ __forceinline__ double wdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float wdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double wsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float wsqrt(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double wexp(double x) { return exp(x); }
__device__ __forceinline__ float wexp(float x) { return __expf(x); }

template <typename T> __device__ __forceinline__ T inf_of();
template <> __device__ __forceinline__ double inf_of<double>() { return CUDART_INF; }
template <> __device__ __forceinline__ float inf_of<float>() { return CUDART_INF_F; }
template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// Exact binary32 -> binary64 with integer operations: the 8-bit exponent is
// rebiased by +896 into the 11-bit field and the significand widened by 29
// bits (high word (a >> 3) + (896 << 20), low word a << 29).  Zeros and normal
// numbers take the integer path; denormals, infinities and NaNs use the
// hardware conversion.
// The rare cases sit behind non-inlined calls: an inlined conversion would be
// if-converted and issued (predicated) on every call, occupying the FP64 pipe.
static __device__ __noinline__ double f2d_slow(float f) { return (double)f; }
static __device__ __noinline__ float d2f_slow(double d) { return (float)d; }

__device__ __forceinline__ double f2d(float f) {
  const uint32_t b = __float_as_uint(f), a = b & 0x7fffffffu;
  if (a != 0u && a - 0x00800000u >= 0x7f000000u) return f2d_slow(f);
  const uint32_t hi = a ? (a >> 3) + (896u << 20) : 0u;
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)(a << 29));
}

// binary64 -> binary32 rounded to nearest, ties to even, with integer
// operations (the same result as a conversion instruction).  Zeros and
// results in the normal binary32 range take the integer path.
__device__ __forceinline__ float d2f(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t ah = hi & 0x7fffffffu;
  if ((ah | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
  if (ah - (897u << 20) >= (254u << 20)) return d2f_slow(d);
  uint32_t t = ((ah << 3) | (lo >> 29)) - (896u << 23);
  const uint32_t rem = lo & 0x1fffffffu;
  t += (rem > 0x10000000u || (rem == 0x10000000u && (t & 1u))) ? 1u : 0u;
  return __uint_as_float(t | (hi & 0x80000000u));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-thread running sums: binary64 for the plain form, compensated binary32
// (Neumaier) for the mixed form.
struct AccD {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
struct AccF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  __device__ __forceinline__ double value() const { return f2d(s) + f2d(c); }
};

// precision of a trace: R decides counts (sampling, clips, bins, cells),
// W carries the weight and the volume geometry.
template <int MODE> struct Prec;
template <> struct Prec<0> { using R = double; using W = double; using Acc = AccD; };
template <> struct Prec<1> { using R = float; using W = float; using Acc = AccF; };

// Parameters in the decision type (binary32 copies are rounded on the host).
template <typename R> __device__ __forceinline__ R par(const DevComp& C, int i);
template <> __device__ __forceinline__ double par<double>(const DevComp& C, int i) { return C.p[i]; }
template <> __device__ __forceinline__ float par<float>(const DevComp& C, int i) { return C.pf[i]; }
template <typename R> __device__ __forceinline__ R inv_of(const DevComp& C, int i);
template <> __device__ __forceinline__ double inv_of<double>(const DevComp& C, int i) { return C.inv[i]; }
template <> __device__ __forceinline__ float inv_of<float>(const DevComp& C, int i) { return C.invf[i]; }
template <typename R> __device__ __forceinline__ R aux_of(const DevComp& C, int i);
template <> __device__ __forceinline__ double aux_of<double>(const DevComp& C, int i) { return C.aux[i]; }
template <> __device__ __forceinline__ float aux_of<float>(const DevComp& C, int i) { return C.auxf[i]; }

// ------------------------------------------------------------------ frames (binary64)
__device__ __forceinline__ void to_local(const DevComp& C, const double X[3], const double K[3],
                                         double x[3], double k[3]) {
  const double d0 = X[0] - C.o[0], d1 = X[1] - C.o[1], d2 = X[2] - C.o[2];
  if (C.identity) {
    x[0] = d0; x[1] = d1; x[2] = d2;
    k[0] = K[0]; k[1] = K[1]; k[2] = K[2];
    return;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    x[i] = (C.R[i] * d0 + C.R[3 + i] * d1) + C.R[6 + i] * d2;
    k[i] = (C.R[i] * K[0] + C.R[3 + i] * K[1]) + C.R[6 + i] * K[2];
  }
}

__device__ __forceinline__ void to_lab(const DevComp& C, const double p[3], double X[3]) {
  if (C.identity) {
    X[0] = C.o[0] + p[0]; X[1] = C.o[1] + p[1]; X[2] = C.o[2] + p[2];
    return;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    X[i] = C.o[i] + ((C.R[3 * i] * p[0] + C.R[3 * i + 1] * p[1]) + C.R[3 * i + 2] * p[2]);
}

__device__ __forceinline__ void dir_to_lab(const DevComp& C, const double k[3], double K[3]) {
  if (C.identity) { K[0] = k[0]; K[1] = k[1]; K[2] = k[2]; return; }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    K[i] = (C.R[3 * i] * k[0] + C.R[3 * i + 1] * k[1]) + C.R[3 * i + 2] * k[2];
}

// Identity-frame translations X - o and o + p.  Components on the optical
// axis (origin x = y = 0, the usual placement) take straight-line code with a
// single binary64 add on z (x - 0 and 0 + x are exact, so skipping them leaves
// the result unchanged); any other origin goes through an out-of-line call,
// so the common path never issues the extra binary64 adds, even predicated.
struct D3 {
  double x, y, z;
};
static __device__ __noinline__ D3 sub_o_general(double o0, double o1, double o2, double X0, double X1,
                                                double X2) {
  return D3{X0 - o0, X1 - o1, X2 - o2};
}
static __device__ __noinline__ D3 add_o_general(double o0, double o1, double o2, double p0, double p1,
                                                double p2) {
  return D3{o0 + p0, o1 + p1, o2 + p2};
}
__device__ __forceinline__ void sub_origin(const DevComp& C, const double X[3], double x[3]) {
  if ((C.zo & 3) == 3) {
    x[0] = X[0];
    x[1] = X[1];
    x[2] = X[2] - C.o[2];
  } else {
    const D3 r = sub_o_general(C.o[0], C.o[1], C.o[2], X[0], X[1], X[2]);
    x[0] = r.x; x[1] = r.y; x[2] = r.z;
  }
}
// X = o + (p0, p1, 0): on the axis the z sum is o_z exactly
__device__ __forceinline__ void add_origin(const DevComp& C, double p0, double p1, double X[3]) {
  if ((C.zo & 3) == 3) {
    X[0] = p0;
    X[1] = p1;
    X[2] = C.o[2];
  } else {
    const D3 r = add_o_general(C.o[0], C.o[1], C.o[2], p0, p1, 0.0);
    X[0] = r.x; X[1] = r.y; X[2] = r.z;
  }
}

// ------------------------------------------------------------------ chords
// [lo, hi] intersected with {t : |x + t k| <= h}; false when empty.  Used
// for the chords of analytic solids only (weight-only: wdiv).
template <typename T>
__device__ __forceinline__ bool clip_slab(T x, T k, T h, T& lo, T& hi) {
  if (k != (T)0) {
    T t1, t2;
    if constexpr (sizeof(T) == 4) {
      const float r = wdiv(1.f, k);
      t1 = (-h - x) * r;
      t2 = (h - x) * r;
    } else {
      t1 = (-h - x) / k;
      t2 = (h - x) / k;
    }
    lo = tmax(lo, tmin(t1, t2));
    hi = tmin(hi, tmax(t1, t2));
  } else if (x < -h || x > h) {
    return false;
  }
  return hi > lo;
}

// [lo, hi] intersected with {t : a <= x + t k <= b}; false when empty (with
// a = -h, b = h the same operations as clip_slab).
template <typename T>
__device__ __forceinline__ bool clip_range(T x, T k, T a, T b, T& lo, T& hi) {
  if (k != (T)0) {
    const T t1 = (a - x) / k;
    const T t2 = (b - x) / k;
    lo = tmax(lo, tmin(t1, t2));
    hi = tmin(hi, tmax(t1, t2));
  } else if (x < a || x > b) {
    return false;
  }
  return hi > lo;
}

// roots of a t^2 + 2 b t + c = 0 without cancellation (chords only:
// weight-only arithmetic)
template <typename T>
__device__ __forceinline__ bool quad_roots(T a, T b, T c, T& t1, T& t2) {
  T disc;
  if constexpr (sizeof(T) == 4) disc = fmaf(b, b, -(a * c));
  else disc = b * b - a * c;
  if (!(disc > (T)0)) return false;
  const T sq = wsqrt(disc);
  const T q = (b >= (T)0) ? -(b + sq) : -(b - sq);
  const T r1 = wdiv(q, a), r2 = wdiv(c, q);
  t1 = tmin(r1, r2);
  t2 = tmax(r1, r2);
  return true;
}

template <typename T>
__device__ T chord_box(const T x[3], const T k[3], T wx, T wy, T wz, T t_lo) {
  T lo = t_lo, hi = inf_of<T>();
  if (!clip_slab<T>(x[0], k[0], (T)0.5 * wx, lo, hi)) return (T)0;
  if (!clip_slab<T>(x[1], k[1], (T)0.5 * wy, lo, hi)) return (T)0;
  if (!clip_slab<T>(x[2], k[2], (T)0.5 * wz, lo, hi)) return (T)0;
  return hi - lo;
}

template <typename T>
__device__ T chord_cyl(const T x[3], const T k[3], T radius, T height, T t_lo) {
  T lo = t_lo, hi = inf_of<T>();
  T a, c, b;
  if constexpr (sizeof(T) == 4) {
    a = fmaf(k[0], k[0], k[2] * k[2]);
    c = fmaf(x[0], x[0], fmaf(x[2], x[2], -(radius * radius)));
    b = fmaf(x[0], k[0], x[2] * k[2]);
  } else {
    a = k[0] * k[0] + k[2] * k[2];
    c = x[0] * x[0] + x[2] * x[2] - radius * radius;
    b = x[0] * k[0] + x[2] * k[2];
  }
  if (a > (T)0) {
    T t1, t2;
    if (!quad_roots<T>(a, b, c, t1, t2)) return (T)0;
    lo = tmax(lo, t1);
    hi = tmin(hi, t2);
  } else if (c > (T)0) {
    return (T)0;
  }
  if (!clip_slab<T>(x[1], k[1], (T)0.5 * height, lo, hi)) return (T)0;
  return hi > lo ? hi - lo : (T)0;
}

template <typename T>
__device__ T chord_sphere(const T x[3], const T k[3], T radius, T t_lo) {
  T a, b, c;
  if constexpr (sizeof(T) == 4) {
    a = fmaf(k[0], k[0], fmaf(k[1], k[1], k[2] * k[2]));
    b = fmaf(x[0], k[0], fmaf(x[1], k[1], x[2] * k[2]));
    c = fmaf(x[0], x[0], fmaf(x[1], x[1], fmaf(x[2], x[2], -(radius * radius))));
  } else {
    a = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    b = x[0] * k[0] + x[1] * k[1] + x[2] * k[2];
    c = x[0] * x[0] + x[1] * x[1] + x[2] * x[2] - radius * radius;
  }
  T t1, t2;
  if (!(a > (T)0) || !quad_roots<T>(a, b, c, t1, t2)) return (T)0;
  const T lo = tmax(t_lo, t1), hi = t2;
  return hi > lo ? hi - lo : (T)0;
}

template <typename T>
__device__ __forceinline__ T chord_of(const DevComp& C, const T x[3], const T k[3], T t_lo) {
  if (C.type == T_ABS_BOX)
    return chord_box<T>(x, k, par<T>(C, 0), par<T>(C, 1), par<T>(C, 2), t_lo);
  if (C.type == T_ABS_CYL) return chord_cyl<T>(x, k, par<T>(C, 0), par<T>(C, 1), t_lo);
  return chord_sphere<T>(x, k, par<T>(C, 0), t_lo);
}

// ------------------------------------------------------------------ mu(E)
// Cell j = floor((E - e_min) * cell_inv) decided in R, clamped to the table.
template <int MODE, class Tbl>
__device__ __forceinline__ int cell_of(const Tbl& I, typename Prec<MODE>::R E) {
  using R = typename Prec<MODE>::R;
  R v;
  if constexpr (MODE == 0) v = (E - I.e_min) * I.cell_inv;
  else v = (E - I.e_min_f) * I.cell_inv_f;
  int j;
  if constexpr (MODE == 0) {
    if (!(v >= 0.0)) j = 0;
    else if (v >= (double)I.n_cell) j = I.n_cell - 1;
    else j = (int)v;
  } else {
    // same decision as above without conversions: v >= n iff floor(v) >= n
    if (!(v >= 0.f)) j = 0;
    else if (!(v < 8388608.f)) j = I.n_cell - 1;
    else j = min(trunc_small(v), I.n_cell - 1);
  }
  return j;
}

template <int MODE, class Tbl>
__device__ __forceinline__ typename Prec<MODE>::W mu_of(const Tbl& I, int m, typename Prec<MODE>::R E) {
  const size_t at = (size_t)m * (size_t)I.n_cell + (size_t)cell_of<MODE>(I, E);
  if constexpr (MODE == 0) {
    const double2 c = __ldg(I.mu64 + at);
    return c.x + c.y * E;
  } else {
    const float2 c = __ldg(I.mu32 + at);
    return c.x + c.y * E;
  }
}

// The mu tables alone, by value (for out-of-line callers).
struct MuTab {
  const double2* mu64;
  const float2* mu32;
  int32_t n_mat, n_cell;
  double e_min, cell_inv;
  float e_min_f, cell_inv_f;
};
__device__ __forceinline__ MuTab mu_tab(const DevInstrument& I) {
  return MuTab{I.mu64, I.mu32, I.n_mat, I.n_cell, I.e_min, I.cell_inv, I.e_min_f, I.cell_inv_f};
}

// Scattering coefficient of material m at E, kind 0 Rayleigh or 1 Compton,
// from the per-cell tables sc = [kind][n_mat][n_cell] (c0, c1) in the
// decision type R: c0 + c1 E on E's cell (the scattering depth decides
// whether a ray scatters, so it is formed in R).
template <int MODE>
__device__ __forceinline__ typename Prec<MODE>::R sc_of(const MuTab& T,
                                                        const typename Prec<MODE>::R* __restrict__ sc,
                                                        int kind, int m, typename Prec<MODE>::R E) {
  const size_t at = 2 * (((size_t)kind * (size_t)T.n_mat + (size_t)m) * (size_t)T.n_cell +
                         (size_t)cell_of<MODE>(T, E));
  return __ldg(sc + at) + __ldg(sc + at + 1) * E;
}

// ------------------------------------------------------------------ 3D-DDA
// Line integral of mu over the centred voxel grid by incremental voxel
// walking (Amanatides & Woo, Eurographics 1987).
//
// The walk is parametrised from the grid entry point.  Per axis, the entry
// point is split (in binary64) into an integer voxel index and a fractional
// offset d0 in [0, 1] voxel to the first plane ahead; the k-th later plane
// on that axis then lies at t = d0 v/|k_axis| + k v/|k_axis| past the entry.
// No position is ever rounded to T, so a ray that grazes a family of planes
// (small |k_axis|) does not amplify coordinate rounding into its crossing
// parameters, and no error accumulates along long paths.  `a_in`/`a_out` are
// the entry/exit parameters on the binary64 local line x + t k.  `mu` points
// at this thread's column of per-material attenuations (stride `ms`).
#ifndef MCX_DDA_CHUNK
#define MCX_DDA_CHUNK 4
#endif
#ifndef MCX_VOX_MIN_BLOCKS
#define MCX_VOX_MIN_BLOCKS 3
#endif
#ifndef MCX_VOX_MIN_BLOCKS_MIXED
#define MCX_VOX_MIN_BLOCKS_MIXED 5
#endif
#ifndef MCX_VOX_MIN_BLOCKS_MIXED_GENERIC
#define MCX_VOX_MIN_BLOCKS_MIXED_GENERIC 4
#endif
#ifndef MCX_WALK_WORD
#define MCX_WALK_WORD 8
#endif
constexpr int kDdaChunk = MCX_DDA_CHUNK;   // crossings walked ahead of their loads
constexpr int kWalkWord = MCX_WALK_WORD;   // bytes per voxel load of the fused kernels' walk
// Resident 256-thread blocks per SM the phantom kernels are compiled for.
// Binary64 form: 3 (its FP64 pipe, not latency, bounds it: 1.15e8 rays/s on
// the 256^3 CT projection against 9.6e7 with 5).  Mixed form, kernels
// compiled for an instrument: 5 (2.43e9 against 2.29e9 with 3 on the CT
// projection, 2.13e9 against 1.97e9 on the EDXCT block, 1.81e8 against
// 1.43e8 with scattering); generic kernels, whose table reads need more
// registers: 4 (2.25e9 on the CT projection, 1.99e9 with 5, 2.17e9 with 3).
constexpr int kVoxMinBlocks = MCX_VOX_MIN_BLOCKS;
constexpr int kVoxMinBlocksMixed = MCX_VOX_MIN_BLOCKS_MIXED;
constexpr int kVoxMinBlocksMixedGeneric = MCX_VOX_MIN_BLOCKS_MIXED_GENERIC;
// the generic kernels' value
template <int MODE>
__host__ __device__ constexpr int vox_min_blocks() {
  return MODE == 1 ? kVoxMinBlocksMixedGeneric : kVoxMinBlocks;
}
// Resident 256-thread blocks per SM a compiled kernel without a phantom is
// built for.
#ifndef MCX_SPEC_MIN_BLOCKS
#define MCX_SPEC_MIN_BLOCKS 6   // measured: 5.74e10 rays/s against 5.58e10 with 5 (absorption)
#endif
constexpr int kSpecMinBlocks = MCX_SPEC_MIN_BLOCKS;
// Resident 256-thread blocks per SM of the generic kernels without a phantom
// (measured: 3.28e10 rays/s on the absorption instrument against 3.06e10
// with 5 and 2.85e10 with 6; the compiled kernels' 6 blocks, tried with 7
// and 8, lost 8 %).
#ifndef MCX_GENERIC_MIN_BLOCKS
#define MCX_GENERIC_MIN_BLOCKS 4
#endif
constexpr int kGenericMinBlocks = MCX_GENERIC_MIN_BLOCKS;
// Resident 256-thread blocks per SM of a batch kernel compiled by families
// without a phantom (measured on the 376-instrument batch: 3.64e10 rays/s
// against 3.39e10 with 5 and 3.14e10 with 6: its detectors' traffic, not
// issue, bounds it).
#ifndef MCX_FAMILY_MIN_BLOCKS
#define MCX_FAMILY_MIN_BLOCKS 4
#endif
constexpr int kFamilyMinBlocks = MCX_FAMILY_MIN_BLOCKS;

// The binary32 walk can read the phantom a word at a time.  Its device
// layout makes the axis that faces the source contiguous, so most crossings
// step to the next byte: a lane keeps the aligned WORD-byte word holding its
// current voxel and loads a new one only when a crossing leaves it (fewer L1
// accesses per crossing; each lane's load is a separate sector access, since
// the walk's rays are unrelated).  The device phantom is padded to whole
// 16-byte words, so a word load never leaves the allocation.
template <int WORD> struct VoxWordT {
  uint32_t w[WORD < 4 ? 1 : WORD / 4];
};
template <int WORD>
__device__ __forceinline__ VoxWordT<WORD> load_word(const uint8_t* __restrict__ vox, int key) {
  VoxWordT<WORD> r;
  if constexpr (WORD == 1) {
    r.w[0] = __ldg(vox + key);
  } else if constexpr (WORD == 4) {
    r.w[0] = __ldg(reinterpret_cast<const unsigned*>(vox) + key);
  } else if constexpr (WORD == 8) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(vox) + key);
    r.w[0] = v.x; r.w[1] = v.y;
  } else {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(vox) + key);
    r.w[0] = v.x; r.w[1] = v.y; r.w[2] = v.z; r.w[3] = v.w;
  }
  return r;
}
// byte `lin` of the word that holds it
template <int WORD>
__device__ __forceinline__ unsigned word_byte(const VoxWordT<WORD>& v, int lin) {
  if constexpr (WORD == 1) return v.w[0];
  if constexpr (WORD == 4) return __byte_perm(v.w[0], 0u, (unsigned)(lin & 3)) & 0xffu;
  // one byte permute over the 8-byte pair (w1:w0) picks byte lin mod 8
  if constexpr (WORD == 8) return __byte_perm(v.w[0], v.w[1], (unsigned)(lin & 7)) & 0xffu;
  const bool hi = ((lin >> 3) & 1) != 0;
  return __byte_perm(hi ? v.w[2] : v.w[0], hi ? v.w[3] : v.w[1], (unsigned)(lin & 7)) & 0xffu;
}

// binary64 form: the sequential walk over [a_in, a_out] of the local line.
static __device__ double dda_tau64(const double xl[3], const double kl[3], double a_in, double a_out,
                           const DevComp& C, const uint8_t* __restrict__ vox,
                           const double* __restrict__ mu, int ms) {
  using T = double;
  const int n[3] = {C.n[0], C.n[1], C.n[2]};
  const double iv = C.inv[0];
  const T v = par<T>(C, 0);
  const T INF = inf_of<T>();
  int idx[3], stp[3];
  T base[3], tdel[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double e = (xl[i] + a_in * kl[i] + C.aux[i]) * iv;   // voxel units from the corner
    int j = __double2int_rd(e);
    j = j < 0 ? 0 : (j >= n[i] ? n[i] - 1 : j);
    idx[i] = j;
    // an axis whose direction component rounds to 0 in T is not stepped
    const T ak = (T)fabs(kl[i]);
    stp[i] = ak > (T)0 ? (kl[i] > 0.0 ? 1 : -1) : 0;
    if (stp[i] != 0) {
      double d0 = stp[i] > 0 ? (double)(j + 1) - e : e - (double)j;
      d0 = d0 < 0.0 ? 0.0 : d0;
      tdel[i] = v / ak;
      base[i] = (T)d0 * tdel[i];
    } else {
      tdel[i] = (T)0;
      base[i] = INF;
    }
  }
  T cnt[3] = {(T)1, (T)1, (T)1};
  const T L = (T)(a_out - a_in);
  // device layout: voxel (x, y, z) at x vstride[0] + y vstride[1] + z vstride[2]
  const int dx = stp[0] * C.vstride[0], dy = stp[1] * C.vstride[1], dz = stp[2] * C.vstride[2];
  int ix = idx[0], iy = idx[1], iz = idx[2];
  int lin = ix * C.vstride[0] + iy * C.vstride[1] + iz * C.vstride[2];
  T tx = base[0], ty = base[1], tz = base[2];
  T t = (T)0, tau = (T)0;
  const int guard = n[0] + n[1] + n[2] + 2;
  {
    // binary64: a plain sequential walk.  Its compares run on the slow FP64
    // pipe, which bounds this form, so nothing is evaluated ahead.
    for (int step = 0; step < guard; ++step) {
      const T tn = tmin(tmin(tx, ty), tmin(tz, L));
      const unsigned m = __ldg(vox + lin);
      tau += mu[m * ms] * tmax(tn - t, (T)0);
      if (tn >= L) break;
      t = tn;
      if (tx <= ty && tx <= tz) {
        ix += stp[0];
        if ((unsigned)ix >= (unsigned)n[0]) break;
        lin += dx;
        tx = fma(cnt[0], tdel[0], base[0]);
        cnt[0] += (T)1;
      } else if (ty <= tz) {
        iy += stp[1];
        if ((unsigned)iy >= (unsigned)n[1]) break;
        lin += dy;
        ty = fma(cnt[1], tdel[1], base[1]);
        cnt[1] += (T)1;
      } else {
        iz += stp[2];
        if ((unsigned)iz >= (unsigned)n[2]) break;
        lin += dz;
        tz = fma(cnt[2], tdel[2], base[2]);
        cnt[2] += (T)1;
      }
    }
  }
  return tau;
}

// binary32: a counted walk.  The walk ends at E = min(L, the first plane on
// any axis whose crossing would leave the grid); on each axis it crosses
// exactly the planes with fma(k, tdel, base) < E (the parameter formula of the
// steps themselves, so the counts agree with the step-by-step comparisons),
// and those planes all lie inside the grid.  With the counts known, a step is
// an unconditional argmin-and-advance on one running byte offset, with no
// bounds or exit tests; the segments, their order and the final one (to E)
// are those of the sequential walk, so tau is the same bit for bit.  The
// voxel addresses do not depend on the loaded bytes, so the walk runs
// kDdaChunk crossings ahead of its loads.
struct Walk32 {
  int lin;          // byte offset of the entry voxel in the device layout
  int steps;        // crossings inside the walk
  int d[3];         // signed byte stride of a crossing along x, y, z
  float base[3];    // parameter of the first crossing per axis (infinite: not stepped)
  float tdel[3];    // parameter between crossings per axis
  float E;          // end of the walk
};

// The walk of the binary64 local line x + t k over [a_in, a_out] (grid
// entry and exit): entry voxel and offsets in binary64, the rest binary32.
__device__ __forceinline__ Walk32 dda_setup32(const double xl[3], const double kl[3], double a_in,
                                               double a_out, const DevComp& C) {
  Walk32 w;
  const double iv = C.inv[0];
  const float v = C.pf[0];
  int idx[3], stp[3], lim[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int n = C.n[i];
    const double e = (xl[i] + a_in * kl[i] + C.aux[i]) * iv;   // voxel units from the corner
    int j = __double2int_rd(e);
    j = j < 0 ? 0 : (j >= n ? n - 1 : j);
    idx[i] = j;
    // an axis whose direction component rounds to 0 in binary32 is not stepped
    const float ak = (float)fabs(kl[i]);
    stp[i] = ak > 0.f ? (kl[i] > 0.0 ? 1 : -1) : 0;
    if (stp[i] != 0) {
      double d0 = stp[i] > 0 ? (double)(j + 1) - e : e - (double)j;
      d0 = d0 < 0.0 ? 0.0 : d0;
      w.tdel[i] = v / ak;
      w.base[i] = (float)d0 * w.tdel[i];
    } else {
      w.tdel[i] = 0.f;
      w.base[i] = CUDART_INF_F;
    }
    w.d[i] = stp[i] * C.vstride[i];
    lim[i] = stp[i] > 0 ? n - 1 - j : (stp[i] < 0 ? j : 0);   // planes inside the grid
  }
  w.lin = idx[0] * C.vstride[0] + idx[1] * C.vstride[1] + idx[2] * C.vstride[2];
  float E = (float)(a_out - a_in);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (stp[i] != 0) E = tmin(E, fma((float)lim[i], w.tdel[i], w.base[i]));
  w.E = E;
  int steps = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    int c = 0;
    if (stp[i] != 0) {
      const float rd = 1.f / w.tdel[i];
      const float q = tmin(tmax((E - w.base[i]) * rd, 0.f), (float)(lim[i] + 1));
      const float fl = floor_small(q);
      c = trunc_small(fl < q ? fl + 1.f : fl);          // ceil(q): planes with base + k tdel < E
      c = min(c, lim[i]);
      if (c > 0 && fma((float)(c - 1), w.tdel[i], w.base[i]) >= E) --c;
      if (c < lim[i] && fma((float)c, w.tdel[i], w.base[i]) < E) ++c;
    }
    steps += c;
  }
  w.steps = steps;
  return w;
}

// One crossing to the nearest of the three next planes tn (ties go to x,
// then y, as in the sequential walk): only that axis advances its byte
// offset, its next plane and its count.  Written as predicated instructions,
// so that a crossing is straight-line code (two compares, two predicate
// operations and nine predicated updates), never a branch.
__device__ __forceinline__ void dda_advance(float tn, float& tx, float& ty, float& tz, float& c0,
                                            float& c1, float& c2, int& lin, const Walk32& w) {
  asm("{\n\t.reg .pred px, py, pz;\n\t"
      "setp.eq.f32 px, %0, %7;\n\t"
      "setp.eq.and.f32 py, %1, %7, !px;\n\t"
      "or.pred pz, px, py;\n\t"
      "not.pred pz, pz;\n\t"
      "@px add.s32 %6, %6, %8;\n\t"
      "@py add.s32 %6, %6, %9;\n\t"
      "@pz add.s32 %6, %6, %10;\n\t"
      "@px fma.rn.f32 %0, %3, %11, %14;\n\t"
      "@py fma.rn.f32 %1, %4, %12, %15;\n\t"
      "@pz fma.rn.f32 %2, %5, %13, %16;\n\t"
      "@px add.rn.f32 %3, %3, 0f3F800000;\n\t"
      "@py add.rn.f32 %4, %4, 0f3F800000;\n\t"
      "@pz add.rn.f32 %5, %5, 0f3F800000;\n\t}"
      : "+f"(tx), "+f"(ty), "+f"(tz), "+f"(c0), "+f"(c1), "+f"(c2), "+r"(lin)
      : "f"(tn), "r"(w.d[0]), "r"(w.d[1]), "r"(w.d[2]), "f"(w.tdel[0]), "f"(w.tdel[1]),
        "f"(w.tdel[2]), "f"(w.base[0]), "f"(w.base[1]), "f"(w.base[2]));
}

// Optical depth along a set-up walk: sum of mu[material] x segment, with
// `mu` this thread's column of attenuations (stride ms).  WORD = bytes per
// voxel load (1: one byte per crossing; 4, 8, 16: see VoxWordT).
template <int WORD>
__device__ __forceinline__ float dda_walk32(const Walk32& w, const uint8_t* __restrict__ vox,
                                            const float* __restrict__ mu, int ms) {
  constexpr int shift = WORD == 1 ? 0 : (WORD == 4 ? 2 : (WORD == 8 ? 3 : 4));
  int lin = w.lin;
  float tx = w.base[0], ty = w.base[1], tz = w.base[2];
  float c0 = 1.f, c1 = 1.f, c2 = 1.f;
  float t = 0.f, tau = 0.f;
  const int steps = w.steps;
  int done = 0;
  if constexpr (WORD == 1) {
    // whole chunks: every crossing is inside the count, so nothing is
    // predicated on it; a lane whose count is spent leaves the loop
    for (; done + kDdaChunk <= steps; done += kDdaChunk) {
      int at[kDdaChunk];
      float seg[kDdaChunk];
#pragma unroll
      for (int s = 0; s < kDdaChunk; ++s) {
        const float tn = tmin(tmin(tx, ty), tz);
        at[s] = lin;
        seg[s] = tn - t;
        t = tn;
        dda_advance(tn, tx, ty, tz, c0, c1, c2, lin, w);
      }
      unsigned m[kDdaChunk];
#pragma unroll
      for (int s = 0; s < kDdaChunk; ++s) m[s] = __ldg(vox + at[s]);
#pragma unroll
      for (int s = 0; s < kDdaChunk; ++s) tau += mu[m[s] * ms] * seg[s];
    }
    // the last crossings (fewer than a chunk), one at a time
    for (; done < steps; ++done) {
      const float tn = tmin(tmin(tx, ty), tz);
      const unsigned m = __ldg(vox + lin);
      tau += mu[m * ms] * (tn - t);
      t = tn;
      dda_advance(tn, tx, ty, tz, c0, c1, c2, lin, w);
    }
    tau += mu[__ldg(vox + lin) * ms] * tmax(w.E - t, 0.f);
    return tau;
  } else {
    // the word of the voxel the walk is in (key = its index)
    int ckey = lin >> shift;
    VoxWordT<WORD> cw = load_word<WORD>(vox, ckey);
    for (; done + kDdaChunk <= steps; done += kDdaChunk) {
      int at[kDdaChunk];
      float seg[kDdaChunk];
#pragma unroll
      for (int s = 0; s < kDdaChunk; ++s) {
        const float tn = tmin(tmin(tx, ty), tz);
        at[s] = lin;
        seg[s] = tn - t;
        t = tn;
        dda_advance(tn, tx, ty, tz, c0, c1, c2, lin, w);
      }
      // the chunk's new words are all requested before any is used
      VoxWordT<WORD> nw[kDdaChunk];
      bool need[kDdaChunk];
#pragma unroll
      for (int s = 0; s < kDdaChunk; ++s) {
        const int key = at[s] >> shift;
        need[s] = key != (s == 0 ? ckey : (at[s - 1] >> shift));
        if (need[s]) nw[s] = load_word<WORD>(vox, key);
      }
#pragma unroll
      for (int s = 0; s < kDdaChunk; ++s) {
        if (need[s]) cw = nw[s];
        tau += mu[word_byte<WORD>(cw, at[s]) * ms] * seg[s];
      }
      ckey = at[kDdaChunk - 1] >> shift;
    }
    for (; done < steps; ++done) {
      const float tn = tmin(tmin(tx, ty), tz);
      const int key = lin >> shift;
      if (key != ckey) { cw = load_word<WORD>(vox, key); ckey = key; }
      tau += mu[word_byte<WORD>(cw, lin) * ms] * (tn - t);
      t = tn;
      dda_advance(tn, tx, ty, tz, c0, c1, c2, lin, w);
    }
    if ((lin >> shift) != ckey) cw = load_word<WORD>(vox, lin >> shift);
    tau += mu[word_byte<WORD>(cw, lin) * ms] * tmax(w.E - t, 0.f);
    return tau;
  }
}

// ------------------------------------------------------------------ fixed-step traversal
// The paper's own voxel traversal (Sec. 3.3), selected by a phantom's p1 =
// s > 0: from the entry into the whole grid, steps of h = voxel / s along the
// line, each weighted by the material of the voxel that holds its end point
// (clamped to the grid); the last step ends at the grid exit.  Positions are
// 32.32 fixed-point voxel coordinates: the entry point and the step vector
// are rounded to that lattice once, in binary64, and each step is an exact
// integer addition, so every form samples the same voxels.  The entry, the
// exit and the rounding follow the binary64 local line in both forms.
//
// Kernels are built for a set of traversals (their VOX parameter): the
// exact walk, the march, or both (a batch whose instruments differ), so a
// kernel of one kind carries no registers for the other.  In the generic
// kernels the march is an out-of-line call, so that its loop gets the
// kernel's whole register budget (inlined there it spilled); kernels
// compiled for one instrument or family inline it, with the grid's sizes,
// strides and step as constants.  Its operands are passed by value (the
// line, the grid's half extents, 1/voxel, the step, the step bound, the
// sizes and strides).
template <typename A, int WORD>
__device__ __forceinline__ A march_tau(double x0, double x1, double x2, double k0, double k1,
                                           double k2, double h0, double h1, double h2, double iv,
                                           double step, double cap, int n0, int n1, int n2, int v0,
                                           int v1, int v2, const uint8_t* __restrict__ vox,
                                           const A* __restrict__ mu, int ms) {
  const double x[3] = {x0, x1, x2}, k[3] = {k0, k1, k2}, hf[3] = {h0, h1, h2};
  double a_in = 0.0, a_out = CUDART_INF;
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (!clip_range<double>(x[i], k[i], -hf[i], hf[i], a_in, a_out)) return (A)0;
  const double L = a_out - a_in, scale = 4294967296.0;   // 2^32
  long long P[3], D[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    P[i] = __double2ll_rn(((x[i] + a_in * k[i]) + hf[i]) * iv * scale);
    D[i] = __double2ll_rn((step * k[i]) * iv * scale);
  }
  const long long n = (long long)ceil(L / step);
  const long long steps = n < (long long)cap ? n : (long long)cap;   // cap: any chord of the grid
  const double last = L - (double)(n - 1) * step;
  if (steps <= 0) return (A)0;
  // byte offset of the voxel holding the current position (clamped)
  auto voxel = [&]() {
    const int i0 = min(max((int)(P[0] >> 32), 0), n0 - 1);
    const int i1 = min(max((int)(P[1] >> 32), 0), n1 - 1);
    const int i2 = min(max((int)(P[2] >> 32), 0), n2 - 1);
    return i0 * v0 + i1 * v1 + i2 * v2;
  };
  constexpr int shift = WORD == 1 ? 0 : (WORD == 4 ? 2 : (WORD == 8 ? 3 : 4));
  const long long body = steps - 1;
  // mu summed per chunk of steps, the chunks' sums into `sum`: a path of N
  // steps carries the rounding of N / kDdaChunk running additions rather
  // than of N (a single running binary32 sum of the ~750 equal steps through
  // 250 mm of water drifts by ~3e-5 in tau)
  A sum = (A)0;
  long long done = 0;
  int ckey = -1;
  VoxWordT<WORD> cw{};
  for (; done + kDdaChunk <= body; done += kDdaChunk) {
    int at[kDdaChunk];
#pragma unroll
    for (int s = 0; s < kDdaChunk; ++s) {
      P[0] += D[0]; P[1] += D[1]; P[2] += D[2];
      at[s] = voxel();
    }
    if constexpr (WORD == 1) {
      unsigned b[kDdaChunk];
#pragma unroll
      for (int s = 0; s < kDdaChunk; ++s) b[s] = __ldg(vox + at[s]);
      A cs = mu[b[0] * ms];
#pragma unroll
      for (int s = 1; s < kDdaChunk; ++s) cs += mu[b[s] * ms];
      sum += cs;
    } else {
      VoxWordT<WORD> nw[kDdaChunk];
      bool need[kDdaChunk];
#pragma unroll
      for (int s = 0; s < kDdaChunk; ++s) {
        const int key = at[s] >> shift;
        need[s] = key != (s == 0 ? ckey : (at[s - 1] >> shift));
        if (need[s]) nw[s] = load_word<WORD>(vox, key);
      }
      A cs = (A)0;
#pragma unroll
      for (int s = 0; s < kDdaChunk; ++s) {
        if (need[s]) cw = nw[s];
        cs += mu[word_byte<WORD>(cw, at[s]) * ms];
      }
      sum += cs;
      ckey = at[kDdaChunk - 1] >> shift;
    }
  }
  for (; done < body; ++done) {
    P[0] += D[0]; P[1] += D[1]; P[2] += D[2];
    sum += mu[__ldg(vox + voxel()) * ms];
  }
  P[0] += D[0]; P[1] += D[1]; P[2] += D[2];
  return (A)step * sum + (A)last * mu[__ldg(vox + voxel()) * ms];
}

// out of line: generic kernels (the loop gets the whole register budget)
template <typename A, int WORD>
static __device__ __noinline__ A march_call(double x0, double x1, double x2, double k0, double k1,
                                            double k2, double h0, double h1, double h2, double iv,
                                            double step, double cap, int n0, int n1, int n2, int v0,
                                            int v1, int v2, const uint8_t* __restrict__ vox,
                                            const A* __restrict__ mu, int ms) {
  return march_tau<A, WORD>(x0, x1, x2, k0, k1, k2, h0, h1, h2, iv, step, cap, n0, n1, n2, v0, v1, v2,
                            vox, mu, ms);
}

// INL: inlined into kernels compiled for one instrument or family, whose
// grid sizes, strides and step are constants there
template <typename A, int WORD, bool INL>
__device__ __forceinline__ A march_of(const DevComp& C, const double xl[3], const double kl[3],
                                      const uint8_t* vox, const A* mu, int ms) {
  if constexpr (INL)
    return march_tau<A, WORD>(xl[0], xl[1], xl[2], kl[0], kl[1], kl[2], C.aux[0], C.aux[1], C.aux[2],
                              C.inv[0], C.p[2], C.p[3], C.n[0], C.n[1], C.n[2], C.vstride[0],
                              C.vstride[1], C.vstride[2], vox, mu, ms);
  else
    return march_call<A, WORD>(xl[0], xl[1], xl[2], kl[0], kl[1], kl[2], C.aux[0], C.aux[1], C.aux[2],
                               C.inv[0], C.p[2], C.p[3], C.n[0], C.n[1], C.n[2], C.vstride[0],
                               C.vstride[1], C.vstride[2], vox, mu, ms);
}

// ------------------------------------------------------------------ scattering phantom
// One scattering event in the decision type R: Compton when a draw falls
// below mc / (mr + mc) of the voxel's material, else Rayleigh; the polar
// angle by rejection, mu = 2u - 1 accepted when 2u' falls below the law
// (Thomson 1 + mu^2; Klein-Nishina e^2 (e + 1/e - (1 - mu^2)) with
// e = 1 / (1 + (E / m_e c^2)(1 - mu)); both at most 2), 16 pairs at most,
// else forward; the azimuth from a point (a, b) of the unit disc,
// cos phi = (a a - b b)/s, sin phi = 2ab/s; the new direction by the usual
// rotation of the old one (the z-axis formula when |k_z| >= 0.99999).
// Compton lowers E to e E.  Every step is one IEEE operation in this order.
template <typename R>
__device__ __forceinline__ void scatter_dir(RayStream& rs, R mr, R mc, R k[3], R& E) {
  const R uc = Uniform<R>::draw(rs);
  const bool compton = mc > (R)0 && uc < mc / (mr + mc);
  const R kk = E / (R)510.99895;
  R mu = (R)1, eps = (R)1;
  for (int t = 0; t < 16; ++t) {
    const R m = (R)2 * Uniform<R>::draw(rs) - (R)1;
    const R u = Uniform<R>::draw(rs);
    R f, e = (R)1;
    if (compton) {
      e = (R)1 / ((R)1 + kk * ((R)1 - m));
      f = e * e * ((e + (R)1 / e) - ((R)1 - m * m));
    } else {
      f = (R)1 + m * m;
    }
    if ((R)2 * u < f) { mu = m; eps = e; break; }
  }
  R cp = (R)1, sp = (R)0;
  for (int t = 0; t < 16; ++t) {
    const R a = (R)2 * Uniform<R>::draw(rs) - (R)1;
    const R b = (R)2 * Uniform<R>::draw(rs) - (R)1;
    const R s = a * a + b * b;
    if (s < (R)1 && s > (R)0) { cp = (a * a - b * b) / s; sp = ((R)2 * a * b) / s; break; }
  }
  const R st = sqrt_rn<R>((R)1 - mu * mu);
  const R kx = k[0], ky = k[1], kz = k[2];
  if (kz < (R)0.99999 && kz > (R)-0.99999) {
    const R tt = sqrt_rn<R>((R)1 - kz * kz);
    k[0] = st * (kx * kz * cp - ky * sp) / tt + kx * mu;
    k[1] = st * (ky * kz * cp + kx * sp) / tt + ky * mu;
    k[2] = -(st * cp * tt) + kz * mu;
  } else {
    k[0] = st * cp;
    k[1] = st * sp;
    k[2] = kz > (R)0 ? mu : -mu;
  }
  if (compton) E = E * eps;
}

// The fixed-step march with scattering (Sec. 3.3: a step updates the weight
// and may change the direction).  Per step the scattering depth
// (mu_R + mu_C)[m](E) len is added up in the decision type R; when it reaches
// tau* = -ln(1 - u) (drawn at the grid entry and after each scattering) the
// ray scatters at the step's end point: that point in binary64 from the
// fixed-point position, an event of scatter_dir (a Compton event lowers E
// and absorption and scattering ahead are looked up at the new energy), a new
// leg from there (the position continues exactly, the step vector is rounded
// anew); at most 8 scatterings, so at most 9 legs.  The absorption depth
// mu[m] len of every step accumulates in `tau` (weight only), summed in two
// levels: blocks of 32 steps, then the blocks, so a path of N steps carries
// the rounding of 32 + N/32 additions rather than of N (one running binary32
// sum drifts by ~3e-5 in tau over the ~750 equal steps through 250 mm of
// water at 1/3 mm; the lanes of a warp flush their blocks at different
// steps, so the flush stays in A: a binary64 add there would issue on most
// steps).  sc holds the coefficient tables of sc_of; the thread's column mu
// holds n_mat absorption coefficients, then n_mat scattering sums
// mu_R + mu_C at the ray's energy (stride ms).
//
// The march is written as resumable pieces: march_begin (grid entry, first
// leg), march_run (up to a budget of steps, stopping at a scattering or at
// the leg's end), march_event (the scattering and the next leg) and
// march_end.  march_scatter runs them to the end for one ray; the refilling
// trace (trace_refill) runs a few steps of every lane's ray at a time.  Both
// take the same operations in the same order.
//
// The state of a leg (kept in registers by the refilling trace) ...
template <int MODE>
struct MarchLeg {
  using R = typename Prec<MODE>::R;
  using A = typename Prec<MODE>::W;
  long long P[3];   // 32.32 fixed-point position in voxel units
  long long D[3];   // the leg's step vector, same units
  long long s;      // steps taken in this leg
  long long steps;  // steps of this leg
  A last;           // the leg's last step length
  R lastR;          // the same in the decision type
  R acc;            // scattering depth since the last draw
  R tstar;          // the depth at which the ray scatters next
  A tau_b;          // absorption depth of the finished 32-step blocks
  A part;           // absorption depth of the open block
  int nsc;          // scatterings so far
};
// ... and its line (binary64): the leg's start point and direction in the
// phantom's frame and the parameter where the leg leaves the grid.
struct MarchLine {
  double xs[3];
  double ks[3];
  double a_out;
};

// Step vector, step count and last step of a leg of length L along ks.
template <int MODE>
__device__ __forceinline__ void march_leg(const DevComp& C, const double ks[3], double L, MarchLeg<MODE>& st) {
  using R = typename Prec<MODE>::R;
  using A = typename Prec<MODE>::W;
  const double step = C.p[2], iv = C.inv[0], scale = 4294967296.0;
  const long long cap = (long long)C.p[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) st.D[i] = __double2ll_rn((step * ks[i]) * iv * scale);
  const long long n = (long long)ceil(L / step);
  st.steps = n < cap ? n : cap;
  const double last = L - (double)(n - 1) * step;
  st.lastR = (R)last;
  st.last = (A)last;
  st.s = 0;
}

// Grid entry of the local line (x, k): false when the line misses the grid.
// Fills the scattering sums of the column at E and draws the first tau*.
template <int MODE>
__device__ __forceinline__ bool march_begin(const DevComp& C, const double x[3], const double k[3],
                                            RayStream& rs, typename Prec<MODE>::W* mu, int ms,
                                            const typename Prec<MODE>::R* __restrict__ sc, const MuTab& T,
                                            typename Prec<MODE>::R E, MarchLeg<MODE>& st, MarchLine& ln) {
  using R = typename Prec<MODE>::R;
  using A = typename Prec<MODE>::W;
  const int nm = T.n_mat;
  const double iv = C.inv[0], scale = 4294967296.0;
  double a_in = 0.0, a_out = CUDART_INF;
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (!clip_range<double>(x[i], k[i], -C.aux[i], C.aux[i], a_in, a_out)) return false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ln.xs[i] = x[i];
    ln.ks[i] = k[i];
    st.P[i] = __double2ll_rn(((x[i] + a_in * k[i]) + C.aux[i]) * iv * scale);
  }
  A* smu = mu + nm * ms;   // the scattering sums, after the absorption column
  for (int mm = 0; mm < nm; ++mm) smu[mm * ms] = sc_of<MODE>(T, sc, 0, mm, E) + sc_of<MODE>(T, sc, 1, mm, E);
  st.tstar = -ln_series<R>((R)1 - Uniform<R>::draw(rs));
  st.acc = (R)0;
  st.tau_b = (A)0;
  st.part = (A)0;
  st.nsc = 0;
  ln.a_out = a_out;
  march_leg<MODE>(C, k, a_out - a_in, st);
  return true;
}

// At most `limit` (<= kMarchAhead) steps of the current leg.  Returns 1 when
// the ray scatters at the end of the step just taken (m_out: that voxel's
// material; *taken: the steps taken), 2 when the leg has ended without a
// scattering, 0 when the steps ran out first.  The voxels of the next
// kMarchAhead steps are requested before the first of them is used (their
// addresses do not depend on the loaded bytes, and every address is clamped
// into the grid, so a request past the leg's end or past a scattering is
// harmless and its byte is never used).
#ifndef MCX_MARCH_AHEAD
#define MCX_MARCH_AHEAD 4
#endif
constexpr int kMarchAhead = MCX_MARCH_AHEAD;
template <int MODE>
__device__ __forceinline__ int march_chunk(const DevComp& C, const uint8_t* __restrict__ vox,
                                           const typename Prec<MODE>::W* mu, int ms, int nm,
                                           MarchLeg<MODE>& st, int limit, int& taken, unsigned& m_out) {
  using R = typename Prec<MODE>::R;
  using A = typename Prec<MODE>::W;
  const double step = C.p[2];
  const R hR = (R)step;
  const A* smu = mu + nm * ms;
  taken = 0;
  if (st.s >= st.steps) return 2;
  const long long rest = st.steps - st.s;
  const int n = rest < (long long)limit ? (int)rest : limit;
  unsigned mv[kMarchAhead];
  {
    long long Q[3] = {st.P[0], st.P[1], st.P[2]};
#pragma unroll
    for (int j = 0; j < kMarchAhead; ++j) {
      int lin = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        Q[i] += st.D[i];
        lin += min(max((int)(Q[i] >> 32), 0), C.n[i] - 1) * C.vstride[i];
      }
      mv[j] = __ldg(vox + lin);
    }
  }
#pragma unroll
  for (int j = 0; j < kMarchAhead; ++j) {
    if (j >= n) break;
#pragma unroll
    for (int i = 0; i < 3; ++i) st.P[i] += st.D[i];
    const long long s = ++st.s;
    const unsigned m = mv[j];
    st.part += mu[m * ms] * (s < st.steps ? (A)step : st.last);
    if ((s & 31) == 0) {
      st.tau_b += st.part;
      st.part = (A)0;
    }
    if (st.nsc < 8) {
      st.acc = st.acc + smu[m * ms] * (s < st.steps ? hR : st.lastR);
      if (st.acc >= st.tstar) {
        m_out = m;
        taken = j + 1;
        return 1;
      }
    }
  }
  taken = n;
  return st.s >= st.steps ? 2 : 0;
}

// Up to `budget` steps of the current leg (the steps taken are subtracted
// from it), chunk after chunk; returns as march_chunk does.
template <int MODE>
__device__ __forceinline__ int march_run(const DevComp& C, const uint8_t* __restrict__ vox,
                                         const typename Prec<MODE>::W* mu, int ms, int nm,
                                         MarchLeg<MODE>& st, long long& budget, unsigned& m_out) {
  while (budget > 0) {
    int taken = 0;
    const int r = march_chunk<MODE>(C, vox, mu, ms, nm, st, budget < kMarchAhead ? (int)budget : kMarchAhead,
                                    taken, m_out);
    budget -= taken;
    if (r != 0) return r;
  }
  return st.s >= st.steps ? 2 : 0;
}

// The scattering at the end of the step just taken (material m): the
// point, the new direction (and energy), the next tau*, and the next leg.
// Returns false when the scattering point lies past the grid (the last step
// ends outside it): the ray then leaves from that point along ln.ks.
template <int MODE>
__device__ __forceinline__ bool march_event(const DevComp& C, RayStream& rs, typename Prec<MODE>::W* mu, int ms,
                                            const typename Prec<MODE>::R* __restrict__ sc, const MuTab& T,
                                            typename Prec<MODE>::R& E, unsigned m, MarchLeg<MODE>& st,
                                            MarchLine& ln) {
  using R = typename Prec<MODE>::R;
  using A = typename Prec<MODE>::W;
  const int nm = T.n_mat;
  const double v = C.p[0], iv = C.inv[0], scale = 4294967296.0;
  ++st.nsc;
#pragma unroll
  for (int i = 0; i < 3; ++i) ln.xs[i] = ((double)st.P[i] * 0x1p-32) * v - C.aux[i];
  R kr[3] = {(R)ln.ks[0], (R)ln.ks[1], (R)ln.ks[2]};
  const R e0 = E;
  scatter_dir<R>(rs, sc_of<MODE>(T, sc, 0, (int)m, E), sc_of<MODE>(T, sc, 1, (int)m, E), kr, E);
#pragma unroll
  for (int i = 0; i < 3; ++i) ln.ks[i] = (double)kr[i];
  if (E != e0) {   // Compton: absorption and scattering ahead at the new energy
    A* smu = mu + nm * ms;
    for (int mm = 0; mm < nm; ++mm) {
      mu[mm * ms] = mu_of<MODE>(T, mm, E);
      smu[mm * ms] = sc_of<MODE>(T, sc, 0, mm, E) + sc_of<MODE>(T, sc, 1, mm, E);
    }
  }
  st.tstar = -ln_series<R>((R)1 - Uniform<R>::draw(rs));
  st.acc = (R)0;
  double a_in = 0.0, a_out = CUDART_INF;
  bool inside = true;
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (inside && !clip_range<double>(ln.xs[i], ln.ks[i], -C.aux[i], C.aux[i], a_in, a_out)) inside = false;
  if (!inside) return false;
  if (a_in > 0.0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) st.P[i] = __double2ll_rn(((ln.xs[i] + a_in * ln.ks[i]) + C.aux[i]) * iv * scale);
  }
  ln.a_out = a_out;
  march_leg<MODE>(C, ln.ks, a_out - a_in, st);
  return true;
}

// Runs the march of the local line (x, k) to its end.  Returns the number of
// scatterings; when > 0, x and k become the line leaving the grid (exit
// point, last direction); tau receives the absorption depth.
template <int MODE>
__device__ __forceinline__ int march_scatter(const DevComp& C, double x[3], double k[3], RayStream& rs,
                                             const uint8_t* __restrict__ vox,
                                             typename Prec<MODE>::W* mu, int ms,
                                             const typename Prec<MODE>::R* __restrict__ sc,
                                             const MuTab& T, typename Prec<MODE>::R& E,
                                             typename Prec<MODE>::W& tau) {
  using A = typename Prec<MODE>::W;
  MarchLeg<MODE> st;
  MarchLine ln;
  tau = (A)0;
  if (!march_begin<MODE>(C, x, k, rs, mu, ms, sc, T, E, st, ln)) return 0;
  for (;;) {
    unsigned m = 0;
    long long budget = 0x7fffffffffffffffLL;
    if (march_run<MODE>(C, vox, mu, ms, T.n_mat, st, budget, m) == 2) {
      tau = st.tau_b + st.part;
      if (st.nsc > 0) {
#pragma unroll
        for (int i = 0; i < 3; ++i) { x[i] = ln.xs[i] + ln.a_out * ln.ks[i]; k[i] = ln.ks[i]; }
      }
      return st.nsc;
    }
    if (!march_event<MODE>(C, rs, mu, ms, sc, T, E, m, st, ln)) {   // a last step past the grid
      tau = st.tau_b + st.part;
#pragma unroll
      for (int i = 0; i < 3; ++i) { x[i] = ln.xs[i]; k[i] = ln.ks[i]; }
      return st.nsc;
    }
  }
}

// Generic kernels call the scattering march out of line, on copies of the
// line, the stream and the energy; kernels compiled for an instrument
// inline it.
template <int MODE>
static __device__ __noinline__ int scatter_call(const DevComp& C, double* x, double* k, RayStream* rs,
                                                const uint8_t* vox, typename Prec<MODE>::W* mu, int ms,
                                                const typename Prec<MODE>::R* sc, MuTab T,
                                                typename Prec<MODE>::R* E, typename Prec<MODE>::W* tau) {
  return march_scatter<MODE>(C, x, k, *rs, vox, mu, ms, sc, T, *E, *tau);
}
template <int MODE, bool INL>
__device__ __forceinline__ int scatter_of(const DevComp& C, double x[3], double k[3], RayStream& rs,
                                          const uint8_t* vox, typename Prec<MODE>::W* mu, int ms,
                                          const typename Prec<MODE>::R* sc, const MuTab& T,
                                          typename Prec<MODE>::R& E, typename Prec<MODE>::W& tau) {
  if constexpr (INL) {
    return march_scatter<MODE>(C, x, k, rs, vox, mu, ms, sc, T, E, tau);
  } else {
    double lx[3] = {x[0], x[1], x[2]}, lk[3] = {k[0], k[1], k[2]};
    RayStream c = rs;
    typename Prec<MODE>::R e = E;
    typename Prec<MODE>::W t;
    const int r = scatter_call<MODE>(C, lx, lk, &c, vox, mu, ms, sc, T, &e, &t);
    rs = c;
    E = e;
    tau = t;
#pragma unroll
    for (int i = 0; i < 3; ++i) { x[i] = lx[i]; k[i] = lk[i]; }
    return r;
  }
}

// ------------------------------------------------------------------ absorbers
// Optical depth of one ray through an absorber, plain form: the binary64
// local line as is (the same chord formulas as the oracle's).
template <int VOX, bool INL>
__device__ double absorber_tau_plain(const DevInstrument& I, const DevComp& C, const double xl[3],
                                     const double kl[3], double E, double* mu_col, int ms) {
  if ((VOX & kVoxMask) && C.type == T_PHANTOM) {
    if ((VOX & kVoxMask) == kVoxMarch || ((VOX & kVoxMask) == kVoxBoth && C.p[1] > 0.0)) {
      for (int m = 0; m < I.n_mat; ++m) mu_col[m * ms] = mu_of<0>(I, m, E);
      return march_of<double, 1, INL>(C, xl, kl, I.vox, mu_col, ms);
    }
    if constexpr ((VOX & kVoxWalk) == 0) return 0.0;
    double a_in = 0.0, a_out = CUDART_INF;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (!clip_range<double>(xl[i], kl[i], C.p[6 + 2 * i], C.p[7 + 2 * i], a_in, a_out)) return 0.0;
    for (int m = 0; m < I.n_mat; ++m) mu_col[m * ms] = mu_of<0>(I, m, E);
    return dda_tau64(xl, kl, a_in, a_out, C, I.vox, mu_col, ms);
  }
  const double L = chord_of<double>(C, xl, kl, 0.0);
  return L > 0.0 ? mu_of<0>(I, C.material, E) * L : 0.0;
}

// Mixed form: the line's origin moves to (near) its closest approach to the
// component origin, p = x + s k with s from binary32 and the move itself in
// binary64, so that binary32 only sees small coordinates; the phantom's entry
// and exit parameters found in binary32 are carried back to the binary64 line.
template <int VOX, bool INL>
__device__ float absorber_tau_mixed(const DevInstrument& I, const DevComp& C, const double xl[3],
                                    const double kl[3], const float xf[3], const float kf[3],
                                    float E, float* mu_col, int ms) {
  if ((VOX & kVoxMask) && C.type == T_PHANTOM && ((VOX & kVoxMask) == kVoxMarch || ((VOX & kVoxMask) == kVoxBoth && C.p[1] > 0.0))) {
    for (int m = 0; m < I.n_mat; ++m) mu_col[m * ms] = mu_of<1>(I, m, E);
    return march_of<float, kWalkWord, INL>(C, xl, kl, I.vox, mu_col, ms);
  }
  const float s = -((xf[0] * kf[0] + xf[1] * kf[1]) + xf[2] * kf[2]);
  const double sd = f2d(s);
  float p[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) p[i] = d2f(fma(sd, kl[i], xl[i]));
  const float t_lo = -s;
  if ((VOX & kVoxMask) && C.type == T_PHANTOM) {
    if constexpr ((VOX & kVoxWalk) == 0) return 0.f;
    float a_in = t_lo, a_out = CUDART_INF_F;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (!clip_range<float>(p[i], kf[i], C.pf[6 + 2 * i], C.pf[7 + 2 * i], a_in, a_out)) return 0.f;
    for (int m = 0; m < I.n_mat; ++m) mu_col[m * ms] = mu_of<1>(I, m, E);
    return dda_walk32<kWalkWord>(dda_setup32(xl, kl, sd + f2d(a_in), sd + f2d(a_out), C), I.vox, mu_col, ms);
  }
  const float L = chord_of<float>(C, p, kf, t_lo);
  return L > 0.f ? mu_of<1>(I, C.material, E) * L : 0.f;
}

// Mixed form, analytic solids: the re-origin is done in the lab frame, where
// it needs no rotation: d = X - o (binary64), s ~ -(d . K), p = d + s K.  p
// is small (the line's closest approach to the solid's centre), so the
// rotation into the solid's frame is exact enough in binary32.  Only the
// weight depends on this chord, never a count.
//
// p is rounded to binary32 once.  When d and K are themselves binary32
// values (K is, whenever the source frame is the identity; d is, for the
// usual placements on the optical axis), d + s K is formed and rounded in a
// single binary32 fused multiply-add.  Otherwise it is formed in binary64
// and then rounded, out of line so that the common path issues no binary64
// instruction.  The two roundings of the rare path can differ from the single
// one by one binary32 ulp of p, far inside the mixed form's tolerance.
struct F3 {
  float x, y, z;
};
static __device__ __noinline__ F3 reorigin64(double d0, double d1, double d2, double K0, double K1, double K2,
                                             float s) {
  const double sd = f2d(s);
  return F3{d2f(fma(sd, K0, d0)), d2f(fma(sd, K1, d1)), d2f(fma(sd, K2, d2))};
}

__device__ __forceinline__ float solid_tau_mixed(const DevInstrument& I, const DevComp& C, const double X[3],
                                                 const double K[3], const float kf[3], bool k_exact, float E) {
  double d[3];
  float df[3];
  sub_origin(C, X, d);
  bool exact = k_exact;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    df[i] = d2f(d[i]);
    exact = exact && __double_as_longlong(f2d(df[i])) == __double_as_longlong(d[i]);
  }
  const float s = -fmaf(df[0], kf[0], fmaf(df[1], kf[1], df[2] * kf[2]));
  float pl[3];
  if (exact) {
#pragma unroll
    for (int i = 0; i < 3; ++i) pl[i] = fmaf(s, kf[i], df[i]);
  } else {
    const F3 r = reorigin64(d[0], d[1], d[2], K[0], K[1], K[2], s);
    pl[0] = r.x; pl[1] = r.y; pl[2] = r.z;
  }
  float p[3], q[3];
  if (C.identity) {
#pragma unroll
    for (int i = 0; i < 3; ++i) { p[i] = pl[i]; q[i] = kf[i]; }
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      p[i] = fmaf(C.Rf[i], pl[0], fmaf(C.Rf[3 + i], pl[1], C.Rf[6 + i] * pl[2]));
      q[i] = fmaf(C.Rf[i], kf[0], fmaf(C.Rf[3 + i], kf[1], C.Rf[6 + i] * kf[2]));
    }
  }
  const float L = chord_of<float>(C, p, q, -s);
  return L > 0.f ? mu_of<1>(I, C.material, E) * L : 0.f;
}

// ------------------------------------------------------------------ monitors
template <typename R>
__device__ __forceinline__ int bin_of(R v, R lo, R inv, int n) {
  const R f = (v - lo) * inv;
  if (!(f >= (R)0) || !(f < (R)n)) return -1;
  return (int)f;
}
// binary32 form: for f >= 0, f < n holds exactly when floor(f) < n, so the
// bound is checked on the integer and no conversion is issued.
template <>
__device__ __forceinline__ int bin_of<float>(float v, float lo, float inv, int n) {
  const float f = (v - lo) * inv;
  if (!(f >= 0.f) || !(f < 8388608.f)) return -1;
  const int i = trunc_small(f);
  return i < n ? i : -1;
}

// A hit's three updates of a monitor bin in global memory.  With `keep`
// (a monitor's l2keep: its instrument's global monitors fit well inside the
// L2; a compile-time constant in compiled tables) they carry an
// L2 evict-last cache hint, so that the randomly updated bins stay in the L2
// instead of being written back and fetched again during the launch; a
// monitor larger than the L2 would only push other data (a phantom) out, so
// it is updated without the hint.  The sums are the same either way.
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bin_add(MonBin* b, double w, bool keep) {
  if (keep) {
    const uint64_t pol = l2_keep_policy();
    asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" :: "l"(&b->N), "l"(1ull), "l"(pol) : "memory");
    asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" :: "l"(&b->sw), "d"(w), "l"(pol) : "memory");
    asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" :: "l"(&b->sw2), "d"(w * w), "l"(pol) : "memory");
  } else {
    atomicAdd(&b->N, 1ull);
    atomicAdd(&b->sw, w);
    atomicAdd(&b->sw2, w * w);
  }
}
__device__ __forceinline__ void score(MonBin* __restrict__ bins, int64_t at, double w, bool keep) {
  bin_add(bins + at, w, keep);
}
// The mixed form widens a hit's weight with the hardware conversion and
// squares it in binary64 (exact: a 24-bit significand squared fits): two
// instructions on the FP64 pipe, which this form otherwise leaves nearly
// idle, in place of two integer-built widenings.
__device__ __forceinline__ void score(MonBin* __restrict__ bins, int64_t at, float w, bool keep) {
  bin_add(bins + at, (double)w, keep);
}

// A block's private copies of its instrument's small monitors (shared
// memory; null pointers: every monitor is scored with global atomics).  A
// monitor whose bins are hit by most rays would otherwise queue thousands of
// atomics on the same few L2 sectors; here they land in shared memory and
// reach HBM once per block (flush_private).
struct PrivBins {
  double* sw;
  double* sw2;
  unsigned* N;
};

__device__ __forceinline__ double widen(double w) { return w; }
__device__ __forceinline__ double widen(float w) { return f2d(w); }

// Scores weight w into bin b of monitor C.
template <typename W>
__device__ __forceinline__ void score_bin(const DevInstrument& I, const DevComp& C, const PrivBins& pv,
                                          int64_t b, W w) {
  if (C.priv >= 0 && pv.N) {
    const int at = C.priv + (int)b;
    atomicAdd(pv.N + at, 1u);
    const double wd = (double)w;
    atomicAdd(pv.sw + at, wd);
    atomicAdd(pv.sw2 + at, wd * wd);
  } else {
    score(I.bins, C.mon_offset + b, w, C.l2keep != 0);
  }
}

// Number of bins of monitor C.
__device__ __forceinline__ int64_t mon_bins_of(const DevComp& C) {
  if (C.type == T_MON_PSD) return (int64_t)C.n[0] * C.n[1];
  if (C.type == T_MON_EPSD) return (int64_t)C.n[0] * C.n[1] * C.n[2];
  return C.n[0];
}

// ------------------------------------------------------------------ source
// Source point (sx, sy) in the source frame, unit direction k towards a
// uniform point of the target rectangle, energy E: the draw contract.
template <typename R>
__device__ __forceinline__ void direction_from(const DevComp& S, R sx, R sy, R tx, R ty, R k[3]) {
  const R dx = tx - sx, dy = ty - sy, dz = par<R>(S, 5);
  const R len = sqrt_rn<R>(dx * dx + dy * dy + dz * dz);
  const R il = (R)1 / len;   // one division, then three products
  k[0] = dx * il;
  k[1] = dy * il;
  k[2] = dz * il;
}

// Source point and aim point in the source frame plus energy (the draw
// contract's steps 1-2).
template <typename R, bool OPT = true>
__device__ __forceinline__ void sample_start(const DevComp& S, RayStream& rs, R& sx, R& sy, R& tx,
                                             R& ty, R& E) {
  sx = (R)0;
  sy = (R)0;
  if (S.shape == SHAPE_DISK) {
    const R r = par<R>(S, 0);
    const R rr = r * r;
    for (int attempt = 0; attempt < 64; ++attempt) {
      const R u1 = Uniform<R>::draw(rs);
      const R u2 = Uniform<R>::draw(rs);
      const R x = r * ((R)2 * u1 - (R)1);
      const R y = r * ((R)2 * u2 - (R)1);
      if (x * x + y * y <= rr) { sx = x; sy = y; break; }
    }
  } else if (S.shape == SHAPE_RECT) {
    const R u1 = Uniform<R>::draw(rs);
    const R u2 = Uniform<R>::draw(rs);
    sx = par<R>(S, 0) * (u1 - (R)0.5);
    sy = par<R>(S, 1) * (u2 - (R)0.5);
  } else if (OPT && S.shape == SHAPE_GAUSS) {
    R z1, z2;
    gauss_pair<R>(rs, z1, z2);
    sx = par<R>(S, 0) * z1;
    sy = par<R>(S, 1) * z2;
  }
  const R u3 = Uniform<R>::draw(rs);
  const R u4 = Uniform<R>::draw(rs);
  tx = par<R>(S, 6) * (u3 - (R)0.5);
  ty = par<R>(S, 7) * (u4 - (R)0.5);
  if (OPT && S.spectrum == SPEC_GAUSS) {
    R z1, z2;
    gauss_pair<R>(rs, z1, z2);
    E = par<R>(S, 4) + par<R>(S, 8) * z1;
  } else {
    const R u5 = Uniform<R>::draw(rs);
    const R emin = par<R>(S, 2), emax = par<R>(S, 3);
    E = emin + (emax - emin) * u5;
  }
}

// A start's weight (weight only, never a count): the Kramers factor
// f(E)/mean(f) (1 for a flat or Gaussian spectrum) times a Gaussian source's
// divergence weight exp(-(ax^2 + ay^2)/2), a = (aim - source point) /
// (D sigma') per axis (inv0, inv1 = 1/(D sigma'), 0 for none).
template <typename R, bool OPT = true>
__device__ __forceinline__ R source_weight(const DevComp& S, R sx, R sy, R tx, R ty, R E) {
  R w = (R)1;
  if constexpr (sizeof(R) == 8) {
    if (S.spectrum == SPEC_KRAMERS) w = ((S.p[4] - E) / E) / S.aux[1];
    if (OPT && S.shape == SHAPE_GAUSS) {
      const double ax = (tx - sx) * S.inv[0], ay = (ty - sy) * S.inv[1];
      w *= exp(-0.5 * (ax * ax + ay * ay));
    }
  } else {
    if (S.spectrum == SPEC_KRAMERS) w = wdiv(S.pf[4] - E, E) * S.auxf[0];
    if (OPT && S.shape == SHAPE_GAUSS) {
      const float ax = (tx - sx) * S.invf[0], ay = (ty - sy) * S.invf[1];
      w *= wexp(-0.5f * (ax * ax + ay * ay));
    }
  }
  return w;
}

template <typename R, bool OPT = true>
__device__ __forceinline__ void sample_source(const DevComp& S, RayStream& rs, R& sx, R& sy,
                                              R k[3], R& E, R& w) {
  R tx, ty;
  sample_start<R, OPT>(S, rs, sx, sy, tx, ty, E);
  direction_from<R>(S, sx, sy, tx, ty, k);
  w = source_weight<R, OPT>(S, sx, sy, tx, ty, E);
}

// ------------------------------------------------------------------ compound refractive lens
// Refraction at a surface of unit normal m (along the ray, m.k > 0) with
// eta = n1/n2 given as em1 = eta - 1 and ee = eta^2 - 1, both formed from
// delta so that eta's tiny departure from 1 keeps its digits:
// cos_t^2 = cos_i^2 - ee (1 - cos_i^2), k' = eta k - (ee / (eta cos_i + cos_t)) m
// (the vector Snell law with eta cos_i - cos_t = ee / (eta cos_i + cos_t)).
// Count-deciding: IEEE operations in this order.  False on total reflection.
template <typename R>
__device__ __forceinline__ bool refract(R k[3], const R m[3], R em1, R ee) {
  const R ci = (k[0] * m[0] + k[1] * m[1]) + k[2] * m[2];
  const R ct2 = ci * ci - ee * ((R)1 - ci * ci);
  if (!(ct2 >= (R)0)) return false;
  const R ct = sqrt_rn<R>(ct2);
  const R g = ee / ((ci + em1 * ci) + ct);
#pragma unroll
  for (int i = 0; i < 3; ++i) k[i] = (k[i] + em1 * k[i]) - g * m[i];
  return true;
}

// The smaller root of a s^2 + b s + c = 0 (b > 0) without cancellation:
// -2c / (b + sqrt(b^2 - 4ac)); false if there is none.
template <typename R>
__device__ __forceinline__ bool near_root(R a, R b, R c, R& s) {
  const R disc = b * b - (R)4 * a * c;
  if (!(disc >= (R)0) || !(b > (R)0)) return false;
  s = ((R)-2 * c) / (b + sqrt_rn<R>(disc));
  return true;
}

// One ray through the lens stack in its frame (Sec. 3.2): for lens j at
// z_j = (j - (N-1)/2) pitch, the front surface z = z_j - d/2 - h r^2
// (h = 1/(2R)), a refraction into the material (index 1 - delta), the back
// surface z = z_j + d/2 + h r^2 and a refraction out.  A ray outside the
// aperture at a surface, or unable to reach the next surface, is absorbed
// (false).  `path` receives the length inside the material (weight only).
template <typename R, typename A>
__device__ __forceinline__ bool lens_stack(const DevComp& C, R x[3], R k[3], R E, A& path) {
  const R invR = inv_of<R>(C, 0);
  const R h = invR * (R)0.5;
  const R hd = aux_of<R>(C, 0);
  const R ra = par<R>(C, 2);
  const R rr = ra * ra;
  const int N = C.n[0];
  const R hN = ((R)N - (R)1) * (R)0.5;
  const R pitch = par<R>(C, 6);
  const R q = par<R>(C, 5) / E;
  const R delta = par<R>(C, 4) * (q * q);
  const R om = (R)1 - delta;
  const R em1_in = delta / om;
  const R ee_in = (delta * ((R)2 - delta)) / (om * om);
  const R em1_out = -delta;
  const R ee_out = -(delta * ((R)2 - delta));
  path = (A)0;
  for (int j = 0; j < N; ++j) {
    const R zc = ((R)j - hN) * pitch;
    R s, m[3];
    {  // front surface: h (x^2 + y^2) + z - (zc - hd) = 0
      const R a = h * (k[0] * k[0] + k[1] * k[1]);
      const R b = (R)2 * h * (x[0] * k[0] + x[1] * k[1]) + k[2];
      const R c = h * (x[0] * x[0] + x[1] * x[1]) + (x[2] - (zc - hd));
      if (!near_root<R>(a, b, c, s) || !(s >= (R)0)) return false;
#pragma unroll
      for (int i = 0; i < 3; ++i) x[i] = x[i] + s * k[i];
      if (x[0] * x[0] + x[1] * x[1] > rr) return false;
      const R g0 = x[0] * invR, g1 = x[1] * invR;
      const R gl = sqrt_rn<R>((g0 * g0 + g1 * g1) + (R)1);
      m[0] = g0 / gl; m[1] = g1 / gl; m[2] = (R)1 / gl;
      if (!refract<R>(k, m, em1_in, ee_in)) return false;
    }
    {  // back surface: -h (x^2 + y^2) + z - (zc + hd) = 0
      const R a = -(h * (k[0] * k[0] + k[1] * k[1]));
      const R b = k[2] - (R)2 * h * (x[0] * k[0] + x[1] * k[1]);
      const R c = (x[2] - (zc + hd)) - h * (x[0] * x[0] + x[1] * x[1]);
      if (!near_root<R>(a, b, c, s) || !(s >= (R)0)) return false;
#pragma unroll
      for (int i = 0; i < 3; ++i) x[i] = x[i] + s * k[i];
      path += (A)s;
      if (x[0] * x[0] + x[1] * x[1] > rr) return false;
      const R g0 = x[0] * invR, g1 = x[1] * invR;
      const R gl = sqrt_rn<R>((g0 * g0 + g1 * g1) + (R)1);
      m[0] = -(g0 / gl); m[1] = -(g1 / gl); m[2] = (R)1 / gl;
      if (!refract<R>(k, m, em1_out, ee_out)) return false;
    }
  }
  return true;
}

// ------------------------------------------------------------------ planar components
// Moves the ray to the component's local z = 0 plane and applies it (clip or
// score).  Returns false if the ray is absorbed there; `x`, `y` become the
// in-plane position.
template <typename R, typename W>
__device__ __forceinline__ bool planar(const DevInstrument& I, const DevComp& C, const PrivBins& pv,
                                       R& x, R& y, R z, R qx, R qy, R qz, R E, W w, bool& scored) {
  // a restoring monitor lets a ray that cannot reach its plane pass unscored
  if (qz == (R)0) return C.restore != 0;
  const R t = -z / qz;
  if (t < (R)0) return C.restore != 0;
  x = x + t * qx;
  y = y + t * qy;
  switch (C.type) {
    case T_SLIT_RECT:
      return x >= par<R>(C, 0) && x <= par<R>(C, 1) && y >= par<R>(C, 2) && y <= par<R>(C, 3);
    case T_SLIT_CIRC: {
      const R r = par<R>(C, 0);
      return x * x + y * y <= r * r;
    }
    case T_MON_PSD: {
      const int ix = bin_of<R>(x, par<R>(C, 0), inv_of<R>(C, 0), C.n[0]);
      const int iy = bin_of<R>(y, par<R>(C, 2), inv_of<R>(C, 1), C.n[1]);
      if (ix >= 0 && iy >= 0) {
        score_bin(I, C, pv, (int64_t)iy * C.n[0] + ix, w);
        scored = true;
      }
      return true;
    }
    case T_MON_E:
      if (x >= par<R>(C, 0) && x < par<R>(C, 1) && y >= par<R>(C, 2) && y < par<R>(C, 3)) {
        const int ie = bin_of<R>(E, par<R>(C, 4), inv_of<R>(C, 2), C.n[0]);
        if (ie >= 0) {
          score_bin(I, C, pv, ie, w);
          scored = true;
        }
      }
      return true;
    case T_MON_L:
      if (x >= par<R>(C, 0) && x < par<R>(C, 1) && y >= par<R>(C, 2) && y < par<R>(C, 3)) {
        const R lam = (R)kHcKevAngstrom / E;
        const int il = bin_of<R>(lam, par<R>(C, 4), inv_of<R>(C, 2), C.n[0]);
        if (il >= 0) {
          score_bin(I, C, pv, il, w);
          scored = true;
        }
      }
      return true;
    case T_MON_EPSD: {
      const int ix = bin_of<R>(x, par<R>(C, 0), inv_of<R>(C, 0), C.n[0]);
      const int iy = bin_of<R>(y, par<R>(C, 2), inv_of<R>(C, 1), C.n[1]);
      const int ie = bin_of<R>(E, par<R>(C, 4), inv_of<R>(C, 2), C.n[2]);
      if (ix >= 0 && iy >= 0 && ie >= 0) {
        score_bin(I, C, pv, ((int64_t)iy * C.n[0] + ix) * C.n[2] + ie, w);
        scored = true;
      }
      return true;
    }
    default:
      return true;
  }
}

// ------------------------------------------------------------------ component tables
// The component list as the ray loop sees it.  SmemTable: any instrument,
// copied into shared memory by each block, count known at run time.  A
// specialised kernel (mcx_jit.cu) supplies its own table type whose entries
// are compile-time constants (kStatic): the loop over components is unrolled
// and every parameter folds into the instructions that use it.
struct SmemTable {
  static constexpr bool kStatic = false;
  static constexpr int kN = kMaxComps;
  const DevComp* c;
  int n;
  __device__ __forceinline__ const DevComp& operator[](int i) const { return c[i]; }
  __device__ __forceinline__ int size() const { return n; }
};

// Calls body(c) for c = 1 .. size-1 in order (unrolled for a static table).
template <class Tab, class F>
__device__ __forceinline__ void for_each_component(const Tab& tab, F&& body) {
  if constexpr (Tab::kStatic) {
#pragma unroll
    for (int c = 1; c < Tab::kN; ++c) body(c);
  } else {
    for (int c = 1; c < tab.size(); ++c) body(c);
  }
}

// ------------------------------------------------------------------ loss tallies
// Weight removed at each component (absorbed at a clip, attenuated in an
// absorber).  Every lane of the warp calls add() for every component.
//
// WarpLoss: a run-time component table.  The warp's losses at a component
// are summed with shuffles and added to the warp's row in shared memory.
template <int MODE>
struct WarpLoss {
  double* row;
  __device__ __forceinline__ void add(int c, typename Prec<MODE>::W v) {
    if (__any_sync(0xffffffffu, v != (typename Prec<MODE>::W)0)) {
      const typename Prec<MODE>::W s = warp_sum(v);
      if ((threadIdx.x & 31u) == 0) row[c] += widen(s);
    }
  }
  __device__ __forceinline__ void flush() {}
};

// ThreadLoss: a compiled table, whose component indices are constants.  Each
// thread keeps one running sum per component in registers (binary64 for the
// plain form, compensated binary32 for the mixed form); the warp sums them
// into its shared-memory row once, after its last ray.
template <int MODE, int N>
struct ThreadLoss {
  double* row;
  typename Prec<MODE>::Acc acc[N];
  __device__ __forceinline__ void add(int c, typename Prec<MODE>::W v) {
    if (__any_sync(0xffffffffu, v != (typename Prec<MODE>::W)0)) acc[c].add(v);
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int c = 1; c < N; ++c) {
      const double s = warp_sum(acc[c].value());
      if ((threadIdx.x & 31u) == 0) row[c] += s;
    }
  }
};

template <bool B, class T, class F> struct Pick { using type = T; };
template <class T, class F> struct Pick<false, T, F> { using type = F; };

// ------------------------------------------------------------------ one ray
// Traces ray `id` (if `valid`) through the instrument.  Every lane of the
// warp must call these together: the loss tallies use warp votes and
// shuffles.  `loss` receives the weight removed per component; `mu_col` is
// this thread's column of per-material attenuations.
template <int VOX, class Tab, class Loss>
__device__ __forceinline__ void trace_ray_plain(const DevInstrument& I, const Tab& comp,
                                                const PrivBins& pv, Loss& loss,
                                                double* mu_col, int ms,
                                                uint64_t id, uint64_t seed, bool valid, AccD& acc_w0,
                                                AccD& acc_wend) {
  const DevComp& S = comp[0];
  double E = 0.0, w = 0.0;
  bool alive = valid;
  double X[3] = {0.0, 0.0, 0.0}, K[3] = {0.0, 0.0, 1.0};
  RayStream rs;   // the ray's stream; a scattering phantom draws on from it
  if (valid) {
    rs.init(id, (uint32_t)I.instr_id, seed);
    double sx, sy, k[3];
    sample_source<double, (VOX & kOptics) != 0>(S, rs, sx, sy, k, E, w);
    acc_w0.add(w);
    const double sl[3] = {sx, sy, 0.0};
    to_lab(S, sl, X);
    dir_to_lab(S, k, K);
  }
  for_each_component(comp, [&](int c) {
    const DevComp& C = comp[c];
    double lost = 0.0;
    if (alive) {
      double xl[3], kl[3];
      to_local(C, X, K, xl, kl);
      if ((VOX & kVoxMarch) && C.type == T_PHANTOM && C.p[4] != 0.0 && C.p[1] > 0.0) {
        // a scattering phantom: the line may leave changed
        for (int m = 0; m < I.n_mat; ++m) mu_col[m * ms] = mu_of<0>(I, m, E);
        double tau;
        const int nsc = scatter_of<0, Tab::kStatic>(C, xl, kl, rs, I.vox, mu_col, ms, I.sc64, mu_tab(I),
                                                     E, tau);
        if (tau > 0.0) {
          const double wn = w * exp(-tau);
          lost = w - wn;
          w = wn;
        }
        if (nsc > 0) {
          to_lab(C, xl, X);
          dir_to_lab(C, kl, K);
        }
      } else if (C.type >= T_ABS_BOX && C.type <= T_PHANTOM) {
        const double tau = absorber_tau_plain<VOX, Tab::kStatic>(I, C, xl, kl, E, mu_col, ms);
        if (tau > 0.0) {
          const double wn = w * exp(-tau);
          lost = w - wn;
          w = wn;
        }
      } else if ((VOX & kOptics) && C.type == T_LENS) {
        double path;
        if (!lens_stack<double, double>(C, xl, kl, E, path)) {
          lost = w;
          alive = false;
        } else {
          const double tau = mu_of<0>(I, C.material, E) * path;
          if (tau > 0.0) {
            const double wn = w * exp(-tau);
            lost = w - wn;
            w = wn;
          }
          to_lab(C, xl, X);
          dir_to_lab(C, kl, K);
        }
      } else {
        double x = xl[0], y = xl[1];
        bool scored = false;
        if (!planar<double, double>(I, C, pv, x, y, xl[2], kl[0], kl[1], kl[2], E, w, scored)) {
          lost = w;
          alive = false;
        } else if (!C.restore) {
          const double p[3] = {x, y, 0.0};
          to_lab(C, p, X);
        }
      }
    }
    loss.add(c, lost);
  });
  if (alive) acc_wend.add(w);
}

// The mixed form's ray between components: the line in the lab frame
// (binary64) with its binary32 direction, energy, weight and stream.
struct RayMixed {
  double X[3], K[3];
  float kf[3];            // binary32 rounding of K
  float E, w;
  float det;              // weight scored at the last monitor (ray-start mode)
  bool alive;
  bool k_exact_turned;    // K is exactly kf after a lens or a scattering turned the ray
  RayStream rs;           // the ray's stream; a scattering phantom draws on from it
};

// The ray's start: its source draws (or a given start), weight and line.
template <int VOX>
__device__ __forceinline__ void ray_begin_mixed(const DevInstrument& I, const DevComp& S, uint64_t id,
                                                uint64_t seed, bool valid, RayMixed& r, AccF& acc_w0) {
  r.E = 0.f;
  r.w = 0.f;
  r.alive = valid;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r.X[i] = 0.0;
    r.K[i] = i == 2 ? 1.0 : 0.0;
    r.kf[i] = i == 2 ? 1.f : 0.f;
  }
  r.k_exact_turned = S.identity != 0;   // K is exactly kf (identity source frame)
  r.det = 0.f;
  if (valid) {
    float sx, sy, k[3];
    if (I.ext) {
      // given start: source point, aim point, energy and initial weight
      const uint64_t q = id - I.ext_base, n = I.ext_n;
      sx = I.ext[q];
      sy = I.ext[n + q];
      r.E = I.ext[2 * n + q];
      direction_from<float>(S, sx, sy, I.ext[3 * n + q], I.ext[4 * n + q], k);
      r.w = I.ext[5 * n + q];
      r.alive = r.w != 0.f;   // a zero-weight start is emitted but not traced
    } else {
      r.rs.init(id, (uint32_t)I.instr_id, seed);
      sample_source<float, (VOX & kOptics) != 0>(S, r.rs, sx, sy, k, r.E, r.w);
    }
    acc_w0.add(r.w);
    if (S.identity) {
      add_origin(S, f2d(sx), f2d(sy), r.X);
#pragma unroll
      for (int i = 0; i < 3; ++i) { r.kf[i] = k[i]; r.K[i] = f2d(k[i]); }
    } else {
      const double sl[3] = {f2d(sx), f2d(sy), 0.0};
      const double kl[3] = {f2d(k[0]), f2d(k[1]), f2d(k[2])};
      to_lab(S, sl, r.X);
      dir_to_lab(S, kl, r.K);
#pragma unroll
      for (int i = 0; i < 3; ++i) r.kf[i] = d2f(r.K[i]);
    }
  }
}

// The ray's line in component C's frame (binary64) and its binary32 copy.
__device__ __forceinline__ void local_line_mixed(const DevComp& C, const RayMixed& r, double xl[3], double kl[3],
                                                 float xf[3], float qf[3]) {
  if (C.identity) {
    sub_origin(C, r.X, xl);
#pragma unroll
    for (int i = 0; i < 3; ++i) { kl[i] = r.K[i]; qf[i] = r.kf[i]; }
  } else {
    to_local(C, r.X, r.K, xl, kl);
#pragma unroll
    for (int i = 0; i < 3; ++i) qf[i] = d2f(kl[i]);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) xf[i] = d2f(xl[i]);
}

// A scattering phantom's result on the ray: the absorption depth tau, and
// when it scattered (nsc > 0) the new local line (xl, kl).  Returns the
// weight removed.
__device__ __forceinline__ float scatter_result_mixed(const DevComp& C, RayMixed& r, float tau, int nsc,
                                                      const double xl[3], const double kl[3]) {
  float lost = 0.f;
  if (tau > 0.f) {
    const float wn = r.w * wexp(-tau);
    lost = r.w - wn;
    r.w = wn;
  }
  if (nsc > 0) {
    // the new line: binary64 position, binary32-exact direction
    to_lab(C, xl, r.X);
    dir_to_lab(C, kl, r.K);
    if (C.identity) {
#pragma unroll
      for (int i = 0; i < 3; ++i) r.kf[i] = (float)kl[i];
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) r.kf[i] = d2f(r.K[i]);
    }
    r.k_exact_turned = C.identity != 0;
  }
  return lost;
}

// Component C applied to the ray: returns the weight it removes.  k_exact0:
// the source frame is the identity (K is exactly kf until something turns
// the ray).
template <int VOX, class Tab>
__device__ __forceinline__ float component_mixed(const DevInstrument& I, const DevComp& C, const PrivBins& pv,
                                                 float* mu_col, int ms, bool k_exact0, RayMixed& r) {
  float lost = 0.f;
  if (!r.alive) return lost;
  if (C.type >= T_ABS_BOX && C.type <= T_ABS_SPHERE) {
    const float tau = solid_tau_mixed(I, C, r.X, r.K, r.kf, (VOX & (kOptics | kVoxMarch)) ? r.k_exact_turned : k_exact0, r.E);
    if (tau > 0.f) {
      const float wn = r.w * wexp(-tau);
      lost = r.w - wn;
      r.w = wn;
    }
    return lost;
  }
  double xl[3], kl[3];
  float xf[3], qf[3];
  local_line_mixed(C, r, xl, kl, xf, qf);
  if ((VOX & kVoxMarch) && C.type == T_PHANTOM && C.p[4] != 0.0 && C.p[1] > 0.0) {
    // a scattering phantom: the line may leave changed
    for (int m = 0; m < I.n_mat; ++m) mu_col[m * ms] = mu_of<1>(I, m, r.E);
    float tau;
    const int nsc = scatter_of<1, Tab::kStatic>(C, xl, kl, r.rs, I.vox, mu_col, ms, I.sc32, mu_tab(I),
                                                 r.E, tau);
    lost = scatter_result_mixed(C, r, tau, nsc, xl, kl);
  } else if ((VOX & kVoxMask) && C.type == T_PHANTOM) {
    const float tau = absorber_tau_mixed<VOX, Tab::kStatic>(I, C, xl, kl, xf, qf, r.E, mu_col, ms);
    if (tau > 0.f) {
      const float wn = r.w * wexp(-tau);
      lost = r.w - wn;
      r.w = wn;
    }
  } else if ((VOX & kOptics) && C.type == T_LENS) {
    float path;
    if (!lens_stack<float, float>(C, xf, qf, r.E, path)) {
      lost = r.w;
      r.alive = false;
    } else {
      const float tau = mu_of<1>(I, C.material, r.E) * path;
      if (tau > 0.f) {
        const float wn = r.w * wexp(-tau);
        lost = r.w - wn;
        r.w = wn;
      }
      // the new line in the lab frame: binary64 from the binary32 ray
      const double p[3] = {f2d(xf[0]), f2d(xf[1]), f2d(xf[2])};
      const double q[3] = {f2d(qf[0]), f2d(qf[1]), f2d(qf[2])};
      to_lab(C, p, r.X);
      dir_to_lab(C, q, r.K);
      if (C.identity) {
#pragma unroll
        for (int i = 0; i < 3; ++i) r.kf[i] = qf[i];
      } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) r.kf[i] = d2f(r.K[i]);
      }
      r.k_exact_turned = C.identity != 0;
    }
  } else {
    float x = xf[0], y = xf[1];
    bool scored = false;
    const bool ok = planar<float, float>(I, C, pv, x, y, xf[2], qf[0], qf[1], qf[2], r.E, r.w, scored);
    if (C.last && scored) r.det = r.w;
    if (!ok) {
      lost = r.w;
      r.alive = false;
    } else if (!C.last && !C.restore) {
      if (C.identity) {
        add_origin(C, f2d(x), f2d(y), r.X);
      } else {
        const double p[3] = {f2d(x), f2d(y), 0.0};
        to_lab(C, p, r.X);
      }
    }
  }
  return lost;
}

template <int VOX, class Tab, class Loss>
__device__ __forceinline__ void trace_ray_mixed(const DevInstrument& I, const Tab& comp,
                                                const PrivBins& pv, Loss& loss,
                                                float* mu_col, int ms,
                                                uint64_t id, uint64_t seed, bool valid, AccF& acc_w0,
                                                AccF& acc_wend) {
  RayMixed r;
  ray_begin_mixed<VOX>(I, comp[0], id, seed, valid, r, acc_w0);
  const bool k_exact0 = comp[0].identity != 0;
  for_each_component(comp, [&](int c) {
    loss.add(c, component_mixed<VOX, Tab>(I, comp[c], pv, mu_col, ms, k_exact0, r));
  });
  if (r.alive) acc_wend.add(r.w);
  if (I.det_w && valid) I.det_w[id - I.ext_base] = r.det;
}

template <int MODE, int VOX, class Tab, class Loss>
__device__ __forceinline__ void trace_ray(const DevInstrument& I, const Tab& comp,
                                          const PrivBins& pv, Loss& loss,
                                          typename Prec<MODE>::W* mu_col, int ms, uint64_t id,
                                          uint64_t seed, bool valid,
                                          typename Prec<MODE>::Acc& acc_w0,
                                          typename Prec<MODE>::Acc& acc_wend) {
  if constexpr (MODE == 0)
    trace_ray_plain<VOX, Tab>(I, comp, pv, loss, mu_col, ms, id, seed, valid, acc_w0, acc_wend);
  else
    trace_ray_mixed<VOX, Tab>(I, comp, pv, loss, mu_col, ms, id, seed, valid, acc_w0, acc_wend);
}

// ------------------------------------------------------------------ block plumbing
// Dynamic shared memory of a tracing block: component table, per-warp loss
// rows, per-thread attenuation columns.
template <int MODE>
struct BlockSmem {
  DevComp* comp;
  double* lost;
  PrivBins priv;
  typename Prec<MODE>::W* mu;

  // with_table = false: a specialised kernel keeps its table in constants.
  // n_priv: bins of the block-private monitor copies (0: none).
  __device__ __forceinline__ void carve(unsigned char* base, int n_warps, bool with_table = true,
                                        int n_priv = 0) {
    comp = reinterpret_cast<DevComp*>(base);
    lost = reinterpret_cast<double*>(comp + (with_table ? kMaxComps : 0));
    double* p = lost + n_warps * kMaxComps;
    if (n_priv > 0) {
      priv.sw = p;
      priv.sw2 = p + n_priv;
      priv.N = reinterpret_cast<unsigned*>(p + 2 * n_priv);
      p += 2 * n_priv + (n_priv + 1) / 2;   // N rounded up to whole doubles
    } else {
      priv = PrivBins{nullptr, nullptr, nullptr};
    }
    mu = reinterpret_cast<typename Prec<MODE>::W*>(p);
  }
};

__device__ __forceinline__ void load_comps(DevComp* dst, const DevComp* src, int n_comp) {
  const int n16 = n_comp * (int)(sizeof(DevComp) / 16);
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  for (int i = threadIdx.x; i < n16; i += blockDim.x) d[i] = s[i];
}

// Adds the block's tallies into the instrument's global tallies.  Must be
// called by every thread of the block after its last ray.
__device__ __forceinline__ void flush_tallies(const DevInstrument& I, double* lost, int n_warps,
                                              double acc_w0, double acc_wend, double* red) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  acc_w0 = warp_sum(acc_w0);
  acc_wend = warp_sum(acc_wend);
  if (lane == 0) { red[warp] = acc_w0; red[32 + warp] = acc_wend; }
  __syncthreads();
  if ((int)threadIdx.x < I.n_comp) {
    double s = 0.0;
    for (int wv = 0; wv < n_warps; ++wv) s += lost[wv * kMaxComps + threadIdx.x];
    if (s != 0.0) atomicAdd(&I.tallies[threadIdx.x], s);
  }
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int wv = 0; wv < n_warps; ++wv) { a += red[wv]; b += red[32 + wv]; }
    atomicAdd(&I.tallies[I.n_comp], a);
    atomicAdd(&I.tallies[I.n_comp + 1], b);
  }
}

__host__ __device__ inline size_t block_smem_bytes(int n_mat, int block, int precision,
                                                   bool with_table = true, int n_priv = 0) {
  const size_t w = precision == 0 ? sizeof(double) : sizeof(float);
  const size_t priv = n_priv > 0 ? sizeof(double) * (2 * (size_t)n_priv + (n_priv + 1) / 2) : 0;
  return (with_table ? sizeof(DevComp) * kMaxComps : 0) +
         sizeof(double) * (size_t)(block / kWarp) * kMaxComps + priv +
         w * (size_t)n_mat * (size_t)block;
}

// Adds the block's private monitor copies into the instrument's monitors.
// Called by every thread of the block after its last ray.
template <class Tab>
__device__ __forceinline__ void flush_private(const Tab& tab, const DevInstrument& I, const PrivBins& pv) {
  if (!pv.N) return;
  __syncthreads();
  for_each_component(tab, [&](int c) {
    const DevComp& C = tab[c];
    if (C.priv < 0 || C.type < T_MON_PSD || C.type > T_MON_EPSD) return;
    const int nb = (int)mon_bins_of(C);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const unsigned n = pv.N[C.priv + b];
      if (n == 0) continue;
      MonBin* g = I.bins + C.mon_offset + b;
      atomicAdd(&g->N, (unsigned long long)n);
      atomicAdd(&g->sw, pv.sw[C.priv + b]);
      atomicAdd(&g->sw2, pv.sw2[C.priv + b]);
    }
  });
}

// ------------------------------------------------------------------ batches
// A batch's instrument families (mcx_batch.cu, mcx_jit.cu): with_table calls
// f(table) with the table type of an instrument's family, given its table in
// shared memory.  GenericFamilies: one family, every field read from shared
// memory.  A batch compiled by families supplies its own, whose tables hold
// the fields its members share as compile-time constants.
struct GenericFamilies {
  template <class F>
  __device__ __forceinline__ static void with_table(int family, const DevComp* table, int n, const F& f) {
    (void)family;
    f(SmemTable{table, n});
  }
};

// One work item's rays traced with the table of the instrument's family.
// A compiled family table keeps the removed weight in per-thread sums over
// the item (ThreadLoss), added to the warp's row at the item's end.
template <int MODE, int VOX>
struct BatchItem {
  const DevInstrument& I;
  const BlockSmem<MODE>& sm;
  const WorkItem& wi;
  uint64_t seed;
  typename Prec<MODE>::Acc& acc_w0;
  typename Prec<MODE>::Acc& acc_wend;
  template <class Tab>
  __device__ __forceinline__ void operator()(const Tab& tab) const {
    const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    using Loss = typename Pick<Tab::kStatic, ThreadLoss<MODE, Tab::kN>, WarpLoss<MODE>>::type;
    Loss loss{sm.lost + warp * kMaxComps};
    for (uint64_t base = wi.begin + warp * 32u; base < wi.end; base += blockDim.x) {
      const uint64_t id = base + lane;
      trace_ray<MODE, VOX>(I, tab, PrivBins{}, loss, sm.mu + threadIdx.x, blockDim.x, id, seed,
                           id < wi.end, acc_w0, acc_wend);
    }
    loss.flush();
  }
};

// The persistent batch kernel's body: resident blocks take work items from
// `ticket` (one atomic per item and block) until the list is exhausted;
// nothing waits on another block.  When the instrument changes the block
// flushes its tallies for the previous one and loads the new component
// table into shared memory.
template <int MODE, int VOX, class Fams>
__device__ __forceinline__ void batch_rays(const DevInstrument* __restrict__ insts,
                                           const WorkItem* __restrict__ items, uint32_t n_items,
                                           unsigned int* __restrict__ ticket, uint64_t seed,
                                           unsigned char* smem, double* red) {
  __shared__ DevInstrument s_inst;
  __shared__ unsigned int s_item;
  const int n_warps = blockDim.x >> 5;
  BlockSmem<MODE> sm;
  sm.carve(smem, n_warps);
  for (int i = threadIdx.x; i < n_warps * kMaxComps; i += blockDim.x) sm.lost[i] = 0.0;
  typename Prec<MODE>::Acc acc_w0, acc_wend;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(ticket, 1u);
    __syncthreads();
    const unsigned item = s_item;
    if (item >= n_items) break;
    const WorkItem wi = items[item];
    if ((int)wi.inst != cur) {
      if (cur >= 0) {
        flush_tallies(s_inst, sm.lost, n_warps, acc_w0.value(), acc_wend.value(), red);
        __syncthreads();
        for (int i = threadIdx.x; i < n_warps * kMaxComps; i += blockDim.x) sm.lost[i] = 0.0;
        acc_w0 = typename Prec<MODE>::Acc();
        acc_wend = typename Prec<MODE>::Acc();
      }
      if (threadIdx.x == 0) s_inst = insts[wi.inst];
      __syncthreads();
      load_comps(sm.comp, s_inst.comps, s_inst.n_comp);
      cur = (int)wi.inst;
    }
    __syncthreads();
    Fams::with_table(s_inst.family, sm.comp, s_inst.n_comp,
                     BatchItem<MODE, VOX>{s_inst, sm, wi, seed, acc_w0, acc_wend});
    __syncthreads();  // s_item and s_inst are rewritten by the next item
  }
  if (cur >= 0) flush_tallies(s_inst, sm.lost, n_warps, acc_w0.value(), acc_wend.value(), red);
}

// ------------------------------------------------------------------ ray order (voxel phantoms)
// Rays with consecutive ids aim at unrelated points of the target.  A warp
// walks a phantom for as long as its longest ray, so the step counts of its
// rays spread widely (about 60 % of the lanes busy on the 256^3 CT
// projection); and an SM's rays cross unrelated parts of the phantom, so its
// L1 keeps few of their voxels (16 % hits).  Two orderings address this;
// each id is still traced exactly as before, only which lane traces it
// changes (and with it the order of the floating-point monitor and tally
// sums).
//  * Across the GPU (launch_ray_order, id_at): a phantom trace's ids are
//    counting-sorted by the tile of their aim point, chunk by chunk, and a
//    block takes kWarpBatch ids per warp at a time from a ticket, so that it
//    walks one small patch of the target (L1 hits 16 % -> 70 %) while the
//    blocks share the work evenly.
//  * Within a warp (mixed form): each warp estimates every id's number of
//    voxel crossings in its batch, orders the batch by that estimate with a
//    counting sort in its own slice of shared memory and traces the ids 32
//    at a time in that order (about 97 % of the lanes busy); warps never
//    wait for one another.  The binary64 walk, bound by the FP64 pipe, is
//    faster without it (1.17e8 against 8.6e7 rays/s).
//   MCX_RAY_ORDER 0: ids in order; 1: ordered by estimated walk (default).
//   MCX_WARP_BATCH: ids per warp batch.  128 (measured on the 256^3
//   projection, mixed, compiled: 2.60e9 rays/s at 64 or 128, 2.56e9 at 256,
//   2.45e9 at 512): the batch's key and order arrays are static shared
//   memory of every resident block, and the unified L1 that keeps the
//   phantom's voxels gets what shared memory does not take.
#ifndef MCX_RAY_ORDER
#define MCX_RAY_ORDER 1
#endif
#ifndef MCX_WARP_BATCH
#define MCX_WARP_BATCH 128
#endif
constexpr int kRayOrder = MCX_RAY_ORDER;
constexpr int kWarpBatch = MCX_WARP_BATCH;    // ids per warp batch, at most (a multiple of 32)
constexpr int kSortMaxWarps = 8;              // warps of the largest tracing block (256 threads)
constexpr int kKeyBins = 256;                 // key = estimated crossings / 4, clamped
static_assert(kWarpBatch % 32 == 0 && kWarpBatch <= 65536, "warp batch");

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(double x) { return d2f(x); }

// Source point and aim point of ray `id` in the source frame, as the tracer
// draws them (or reads them from a given start), rounded to binary32.
template <int MODE>
__device__ __forceinline__ void start_of(const DevInstrument& I, const DevComp& S, uint64_t id,
                                         uint64_t seed, float& sx, float& sy, float& tx, float& ty) {
  using R = typename Prec<MODE>::R;
  if constexpr (MODE == 1) {
    if (I.ext) {
      const uint64_t r = id - I.ext_base, n = I.ext_n;
      sx = I.ext[r];
      sy = I.ext[n + r];
      tx = I.ext[3 * n + r];
      ty = I.ext[4 * n + r];
      return;
    }
  }
  RayStream rs;
  rs.init(id, (uint32_t)I.instr_id, seed);
  R a, b, c, d, E;
  sample_start<R>(S, rs, a, b, c, d, E);
  sx = to_f(a); sy = to_f(b); tx = to_f(c); ty = to_f(d);
}

// The ordering key of ray `id`: its estimated voxel crossings / 4 in
// [0, kKeyBins), from the chord of its undeflected line through the first
// phantom's attenuating box times (|kx| + |ky| + |kz|) / voxel (binary32,
// approximate: the key only groups rays).
template <int MODE, class Tab>
__device__ __forceinline__ unsigned order_key(const DevInstrument& I, const Tab& tab, uint64_t id,
                                              uint64_t seed) {
  const DevComp& S = tab[0];
  float sx, sy, tx, ty;
  start_of<MODE>(I, S, id, seed, sx, sy, tx, ty);
  const float d0 = tx - sx, d1 = ty - sy, d2 = S.pf[5];
  float P[3], K[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    P[i] = to_f(S.o[i]) + (S.Rf[3 * i] * sx + S.Rf[3 * i + 1] * sy);
    K[i] = (S.Rf[3 * i] * d0 + S.Rf[3 * i + 1] * d1) + S.Rf[3 * i + 2] * d2;
  }
  float steps = 0.f;
  bool found = false;
  for_each_component(tab, [&](int c) {
    const DevComp& C = tab[c];
    if (found || C.type != T_PHANTOM) return;
    found = true;
    float q[3], k[3];
    const float e0 = P[0] - to_f(C.o[0]), e1 = P[1] - to_f(C.o[1]), e2 = P[2] - to_f(C.o[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      q[i] = (C.Rf[i] * e0 + C.Rf[3 + i] * e1) + C.Rf[6 + i] * e2;
      k[i] = (C.Rf[i] * K[0] + C.Rf[3 + i] * K[1]) + C.Rf[6 + i] * K[2];
    }
    float lo = 0.f, hi = CUDART_INF_F;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (k[i] != 0.f) {
        const float r = wdiv(1.f, k[i]);
        const float t1 = (C.pf[6 + 2 * i] - q[i]) * r, t2 = (C.pf[7 + 2 * i] - q[i]) * r;
        lo = fmaxf(lo, fminf(t1, t2));
        hi = fminf(hi, fmaxf(t1, t2));
      } else if (q[i] < C.pf[6 + 2 * i] || q[i] > C.pf[7 + 2 * i]) {
        hi = -1.f;
      }
    }
    if (hi > lo) steps = wdiv((hi - lo) * ((fabsf(k[0]) + fabsf(k[1])) + fabsf(k[2])), 4.f * C.pf[0]);
  });
  return (unsigned)trunc_small(fminf(fmaxf(steps, 0.f), (float)(kKeyBins - 1)));
}

// bit i of x (x < 2^8) to bit 2i
__device__ __forceinline__ unsigned spread_bits(unsigned x) {
  x = (x | (x << 4)) & 0x0F0Fu;
  x = (x | (x << 2)) & 0x3333u;
  x = (x | (x << 1)) & 0x5555u;
  return x;
}

// The tile of ray `id`'s aim point on the source's target rectangle, in
// Morton order (kTileBits bits per axis): rays of one tile cross the phantom
// side by side, so a block that traces them finds their voxels in its L1.
template <int MODE>
__device__ __forceinline__ unsigned aim_tile(const DevInstrument& I, const DevComp& S, uint64_t id,
                                             uint64_t seed) {
  float sx, sy, tx, ty;
  start_of<MODE>(I, S, id, seed, sx, sy, tx, ty);
  const float side = (float)(1 << kTileBits), cap = side - 1.f;
  const float fu = fminf(fmaxf((wdiv(tx, S.pf[6]) + 0.5f) * side, 0.f), cap);
  const float fv = fminf(fmaxf((wdiv(ty, S.pf[7]) + 0.5f) * side, 0.f), cap);
  return spread_bits((unsigned)trunc_small(fu)) | (spread_bits((unsigned)trunc_small(fv)) << 1);
}

// Ray id traced at position p of a phantom trace's range (the ray order).
__device__ __forceinline__ uint64_t id_at(const DevInstrument& I, uint64_t p) {
  return I.perm ? I.perm_base + I.perm[p - I.perm_base] : p;
}

// Rays [begin, end) in ordered warp batches.  A batch holds the warp's share
// of the range (rounded up to 32), at most kWarpBatch ids, so that small
// ranges still reach every warp.  Every lane of the warp calls this.
template <int MODE, int VOX, class Tab, class Loss>
__device__ __forceinline__ void trace_sorted(const DevInstrument& I, const Tab& tab, const BlockSmem<MODE>& sm,
                                             Loss& loss, uint64_t begin, uint64_t end, uint64_t seed,
                                             typename Prec<MODE>::Acc& acc_w0,
                                             typename Prec<MODE>::Acc& acc_wend) {
  __shared__ unsigned char s_key[kSortMaxWarps][kWarpBatch];
  __shared__ unsigned short s_order[kSortMaxWarps][kWarpBatch];
  __shared__ unsigned s_bin[kSortMaxWarps][kKeyBins];
  const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  unsigned char* key = s_key[warp];
  unsigned short* order = s_order[warp];
  unsigned* bin = s_bin[warp];
  // one warp batch: ids at positions [b0, b0 + n) ordered by walk length
  auto batch = [&](uint64_t b0, int n) {
    for (int i = lane; i < kKeyBins; i += 32) bin[i] = 0u;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const unsigned k = order_key<MODE>(I, tab, id_at(I, b0 + (uint64_t)i), seed);
      key[i] = (unsigned char)k;
      atomicAdd(&bin[k], 1u);
    }
    __syncwarp();
    // exclusive prefix sum of the bins, kKeyBins / 32 per lane
    constexpr int per = kKeyBins / 32;
    unsigned own = 0u;
#pragma unroll
    for (int j = 0; j < per; ++j) own += bin[lane * per + j];
    unsigned x = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (unsigned)o) x += y;
    }
    unsigned run = x - own;
#pragma unroll
    for (int j = 0; j < per; ++j) {
      const unsigned c = bin[lane * per + j];
      bin[lane * per + j] = run;
      run += c;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) order[atomicAdd(&bin[key[i]], 1u)] = (unsigned short)i;
    __syncwarp();
    for (int g = 0; g < n; g += 32) {
      const int k = g + (int)lane;
      const bool valid = k < n;
      const uint64_t id = id_at(I, b0 + (uint64_t)(valid ? order[k] : 0));
      trace_ray<MODE, VOX, Tab>(I, tab, sm.priv, loss, sm.mu + threadIdx.x, blockDim.x, id, seed, valid,
                                acc_w0, acc_wend);
    }
    __syncwarp();   // the next batch rewrites the keys and the order
  };
  if (I.perm) {
    // ids grouped by aim-point tile: a block takes kWarpBatch ids per warp
    // at a time from a ticket, so that it walks one small patch of the
    // target (whose voxels its L1 keeps) while the blocks share the work
    // evenly whatever each patch costs
    __shared__ uint64_t s_b0;
    const uint64_t span = (uint64_t)(blockDim.x >> 5) * kWarpBatch;
    for (;;) {
      if (threadIdx.x == 0) s_b0 = begin + (uint64_t)atomicAdd(I.ticket, 1u) * span;
      __syncthreads();
      const uint64_t bb = s_b0;
      __syncthreads();
      if (bb >= end) break;
      const uint64_t b0 = bb + (uint64_t)warp * kWarpBatch;
      if (b0 < end) batch(b0, (int)((end - b0) < (uint64_t)kWarpBatch ? (end - b0) : (uint64_t)kWarpBatch));
    }
    return;
  }
  const uint64_t n_warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const uint64_t share = ((end - begin + n_warps - 1) / n_warps + 31) & ~(uint64_t)31;
  const int nb = (int)(share < (uint64_t)kWarpBatch ? share : (uint64_t)kWarpBatch);
  for (uint64_t b0 = begin + gw * nb; b0 < end; b0 += n_warps * nb)
    batch(b0, (int)((end - b0) < (uint64_t)nb ? (end - b0) : (uint64_t)nb));
}

// ------------------------------------------------------------------ refilled lanes
// A phantom that scatters gives its rays very different numbers of steps (a
// ray may scatter up to eight times, and every leg has its own length), so
// lanes that each trace one ray from start to end leave most of the warp
// idle while its longest ray marches.  Here each lane carries its own ray
// through the march and the warp refills lanes whose ray is done.
// * A round gives every marching lane kRefillSteps steps, as chunks of
//   kMarchAhead with the same trip count on every lane (no lane runs a step
//   loop of its own, which would split the warp into groups that step
//   apart).  A lane whose ray scatters stops; once kEventAt lanes have
//   stopped so (or no lane marches on), their scatterings run at once.
// * A ray whose march has ended waits.  Once kRefillAt lanes wait (or no ray
//   id is left), the waiting lanes together apply the march's result, run
//   the components after the phantom and end their rays, then take the next
//   positions of the warp's batch (kWarpBatch positions, from the ordered
//   launch's ticket or in grid-stride order) and together run the source,
//   the components before the phantom and the grid entry.
// Batching the events, the exits and the starts keeps their divergent and
// binary64 work on many lanes at once instead of one lane at a time.  Each
// ray takes the operations of trace_ray_mixed in the same order; only the
// order in which the rays add to the monitors and tallies changes.  The
// removed weight goes to the warp's loss row by shared-memory atomics, since
// the lanes reach a component at different times.
// Steps per round, lanes waiting before a refill, lanes stopped at a
// scattering before the events run, and resident 256-thread blocks per SM
// (compiled kernel, generic kernel).  Measured on the EDXCT block scattering
// by water (5e7 mixed rays, compiled / generic kernel, rays/s): one ray per
// lane 1.93e8 / 1.34e8; rounds of 32 steps, refills at 8, events at once
// 1.43e8 / 1.13e8; refills at 16 2.12e8; refills at 16, events at 12,
// 64-step rounds 2.52e8, with 2 blocks per SM for the generic kernel
// (which spills at 4) 1.61e8; 128-step rounds 2.37e8; 16-step 2.42e8;
// refills at 24 and events at 20 1.89e8.
#ifndef MCX_REFILL_STEPS
#define MCX_REFILL_STEPS 64
#endif
#ifndef MCX_REFILL_AT
#define MCX_REFILL_AT 16
#endif
#ifndef MCX_EVENT_AT
#define MCX_EVENT_AT 12
#endif
#ifndef MCX_SCATTER_MIN_BLOCKS
#define MCX_SCATTER_MIN_BLOCKS 4
#endif
#ifndef MCX_SCATTER_MIN_BLOCKS_GENERIC
#define MCX_SCATTER_MIN_BLOCKS_GENERIC 2
#endif
constexpr int kRefillSteps = MCX_REFILL_STEPS;
constexpr int kRefillAt = MCX_REFILL_AT;
constexpr int kEventAt = MCX_EVENT_AT;
constexpr int kScatterMinBlocks = MCX_SCATTER_MIN_BLOCKS;
constexpr int kScatterMinBlocksGeneric = MCX_SCATTER_MIN_BLOCKS_GENERIC;
static_assert(kRefillSteps % kMarchAhead == 0, "a round is whole chunks");

__device__ __forceinline__ bool scatters(const DevComp& C) {
  return C.type == T_PHANTOM && C.p[4] != 0.0 && C.p[1] > 0.0;
}

// f(component cp), cp a scattering phantom's index (or -1: nothing): a
// compiled table folds the index and the component's fields into
// constants; a run-time table reads its entry.
template <class Tab, class F>
__device__ __forceinline__ void at_component(const Tab& tab, int cp, const F& f) {
  if constexpr (Tab::kStatic) {
    for_each_component(tab, [&](int c) {
      if (scatters(tab[c]) && c == cp) f(tab[c]);
    });
  } else {
    if (cp >= 0) f(tab[cp]);
  }
}

template <int VOX, class Tab>
__device__ __forceinline__ void trace_refill(const DevInstrument& I, const Tab& tab, const BlockSmem<1>& sm,
                                             uint64_t begin, uint64_t end, uint64_t seed, AccF& acc_w0,
                                             AccF& acc_wend) {
  __shared__ MarchLine s_line[kSortMaxWarps * 32];   // each lane's march line (used at events only)
  const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  double* row = sm.lost + warp * kMaxComps;
  float* mu_col = sm.mu + threadIdx.x;
  const int ms = blockDim.x;
  MarchLine& ln = s_line[threadIdx.x];
  const bool k_exact0 = tab[0].identity != 0;
  int cp = -1;   // the scattering phantom (none: every ray is traced straight through)
  for_each_component(tab, [&](int c) {
    if (cp < 0 && scatters(tab[c])) cp = c;
  });
  auto remove = [&](int c, float v) {
    if (v != 0.f) atomicAdd(&row[c], (double)v);
  };
  RayMixed r;
  MarchLeg<1> st;
  uint64_t id = 0;
  unsigned m_ev = 0u;     // material of the voxel where the pending scattering happens
  bool busy = false;      // this lane's ray is in the march
  bool event = false;     // it scattered in this round; the event is still to run
  bool waiting = false;   // its ray is done marching (or never marched); the rest is still to run
  bool marched = false;   // ... after a march, whose result is still to apply
  bool past = false;      // ... that ended at a scattering point past the grid
  // the warp's batch of positions [b_next, b_end), and whether ids are left
  // (all warp-uniform)
  uint64_t b_next = 0, b_end = 0, round = 0;
  bool more = true;
  const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const uint64_t n_w = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (;;) {
    const unsigned idle = __ballot_sync(0xffffffffu, !busy);
    if (idle == 0xffffffffu || (more ? __popc(idle) >= kRefillAt : __any_sync(0xffffffffu, waiting))) {
      // the waiting rays end: the march's result, the components after the
      // phantom, the tallies
      if (waiting) {
        if (marched) at_component(tab, cp, [&](const DevComp& C) {
          double xl[3], kl[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            xl[i] = past ? ln.xs[i] : ln.xs[i] + ln.a_out * ln.ks[i];
            kl[i] = ln.ks[i];
          }
          remove(cp, scatter_result_mixed(C, r, st.tau_b + st.part, st.nsc, xl, kl));
        });
        for_each_component(tab, [&](int c) {
          if (c > cp) remove(c, component_mixed<VOX, Tab>(I, tab[c], sm.priv, mu_col, ms, k_exact0, r));
        });
        if (r.alive) acc_wend.add(r.w);
        if (I.det_w) I.det_w[id - I.ext_base] = r.det;
        waiting = false;
      }
      // positions of the warp's batch for the idle lanes (warp-uniform)
      bool got = false;
      uint64_t pos = 0;
      if (more) {
        if (b_next >= b_end) {
          uint64_t b;
          if (I.ticket) {
            unsigned t = 0u;
            if (lane == 0u) t = atomicAdd(I.ticket, 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            b = begin + (uint64_t)t * kWarpBatch;
          } else {
            b = begin + (gw + round * n_w) * kWarpBatch;
            ++round;
          }
          if (b >= end) {
            more = false;
          } else {
            b_next = b;
            b_end = end - b < (uint64_t)kWarpBatch ? end : b + kWarpBatch;
          }
        }
        if (more) {
          const unsigned rank = __popc(idle & ((1u << lane) - 1u));
          if (!busy && b_next + rank < b_end) {
            pos = b_next + rank;
            got = true;
          }
          const uint64_t nb = b_next + (uint64_t)__popc(idle);
          b_next = nb < b_end ? nb : b_end;
        }
      }
      // the new rays: source, the components before the phantom, the entry
      if (got) {
        id = id_at(I, pos);
        ray_begin_mixed<VOX>(I, tab[0], id, seed, true, r, acc_w0);
        for_each_component(tab, [&](int c) {
          if (c < cp) remove(c, component_mixed<VOX, Tab>(I, tab[c], sm.priv, mu_col, ms, k_exact0, r));
        });
        if (r.alive) at_component(tab, cp, [&](const DevComp& C) {
          double xl[3], kl[3];
          float xf[3], qf[3];
          local_line_mixed(C, r, xl, kl, xf, qf);
          for (int m = 0; m < I.n_mat; ++m) mu_col[m * ms] = mu_of<1>(I, m, r.E);
          // a line that misses the grid goes on unchanged, nothing removed
          busy = march_begin<1>(C, xl, kl, r.rs, mu_col, ms, I.sc32, mu_tab(I), r.E, st, ln);
        });
        marched = busy;
        past = false;
        waiting = !busy;   // stopped before the phantom or missed its grid
      }
    }
    if (!more && !__any_sync(0xffffffffu, busy || waiting)) break;
    // the round: kRefillSteps / kMarchAhead chunks with the same trip count
    // on every lane, so the warp reconverges after every chunk.  A lane whose
    // ray scatters stops until the events run and a lane whose last leg ends
    // waits for the next refill: that work runs after a round (events) and
    // at a refill (the exit), on all such lanes at once.
    for (int k = 0; k < kRefillSteps / kMarchAhead; ++k) {
      if (busy && !event) {
        at_component(tab, cp, [&](const DevComp& C) {
          int taken = 0;
          const int run = march_chunk<1>(C, I.vox, mu_col, ms, I.n_mat, st, kMarchAhead, taken, m_ev);
          if (run == 1) {
            event = true;
          } else if (run == 2) {   // the last leg ended inside the grid's bounds
            busy = false;
            waiting = true;
          }
        });
      }
      __syncwarp();
    }
    // the scatterings, once kEventAt lanes have one or no lane marches on
    const unsigned ev = __ballot_sync(0xffffffffu, event);
    if (__popc(ev) >= kEventAt || (ev != 0u && !__any_sync(0xffffffffu, busy && !event))) {
      if (event) {
        at_component(tab, cp, [&](const DevComp& C) {
          if (!march_event<1>(C, r.rs, mu_col, ms, I.sc32, mu_tab(I), r.E, m_ev, st, ln)) {
            busy = false;   // a scattering point past the grid: the ray leaves from there
            waiting = true;
            past = true;
          }
        });
        event = false;
      }
    }
  }
}

// The body of a single-instrument tracing kernel: grid-stride over warps of
// 32 consecutive ray ids, or over ordered batches when a phantom is walked
// (every lane of a warp runs the same number of iterations, ids past the end
// are traced as invalid, so the warp-level tally reductions always see all
// 32 lanes), then the block's tallies are flushed.
// With a SmemTable the block first copies the instrument's table into shared
// memory.
template <int MODE, int VOX, class Tab>
__device__ __forceinline__ void trace_rays(const DevInstrument& I, uint64_t begin, uint64_t end,
                                           uint64_t seed, unsigned char* smem, double* red) {
  const int n_warps = blockDim.x >> 5;
  BlockSmem<MODE> sm;
  sm.carve(smem, n_warps, !Tab::kStatic, I.n_priv);
  Tab tab{};
  if constexpr (!Tab::kStatic) {
    load_comps(sm.comp, I.comps, I.n_comp);
    tab = Tab{sm.comp, I.n_comp};
  }
  for (int i = threadIdx.x; i < n_warps * kMaxComps; i += blockDim.x) sm.lost[i] = 0.0;
  for (int i = threadIdx.x; i < I.n_priv; i += blockDim.x) {
    sm.priv.sw[i] = 0.0;
    sm.priv.sw2[i] = 0.0;
    sm.priv.N[i] = 0u;
  }
  __syncthreads();

  const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  typename Prec<MODE>::Acc acc_w0, acc_wend;
  using Loss = typename Pick<Tab::kStatic, ThreadLoss<MODE, Tab::kN>, WarpLoss<MODE>>::type;
  Loss loss{sm.lost + warp * kMaxComps};
  // the per-warp walk ordering pays for the binary32 walk; the binary64
  // walk (bound by its FP64 pipe) runs faster without it
  if constexpr (MODE == 1 && (VOX & kScatter) != 0) {
    trace_refill<VOX, Tab>(I, tab, sm, begin, end, seed, acc_w0, acc_wend);
  } else if constexpr ((VOX & kVoxMask) && kRayOrder != 0 && MODE == 1) {
    trace_sorted<MODE, VOX, Tab>(I, tab, sm, loss, begin, end, seed, acc_w0, acc_wend);
  } else {
    for (uint64_t base = begin + (uint64_t)blockIdx.x * blockDim.x + warp * 32u; base < end;
         base += stride) {
      const uint64_t p = base + lane;
      trace_ray<MODE, VOX, Tab>(I, tab, sm.priv, loss, sm.mu + threadIdx.x, blockDim.x,
                                (VOX & kVoxMask) && p < end ? id_at(I, p) : p, seed, p < end, acc_w0, acc_wend);
    }
  }
  loss.flush();
  flush_private(tab, I, sm.priv);
  flush_tallies(I, sm.lost, n_warps, acc_w0.value(), acc_wend.value(), red);
}

}  // namespace mcx
