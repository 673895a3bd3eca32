// dg_device.cuh -- device-side building blocks of the fused DGSEM stage kernels.
//
// Arithmetic traits for the two precisions, FP64 <-> FP32 conversions done in integer
// arithmetic, the element geometry of a tensor-product GLL element, and the Euler fluxes
// of Sec. 2 / Sec. 3.1.1 / App. A (point flux, Ranocha two-point flux, Rusanov, HLL,
// HLLC), all templated on the flux arithmetic type R (double or float).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dg {

// ---------------------------------------------------------------------------------------
// FP64 <-> FP32 conversion in integer arithmetic.
// On sm_103a the hardware double->float conversion issues at under one result per clock
// per SM (slower than an FP64 FMA), so the mixed-precision path converts the FP64 state
// with integer instructions instead, written from the IEEE-754 binary64/binary32
// encodings: round-to-nearest-even on the 29 discarded mantissa bits; results below the
// smallest normal float flush to a signed zero; overflow gives infinity; NaN stays NaN.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float d2f_rn(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x);
  const uint32_t lo = (uint32_t)__double2loint(x);
  const uint32_t ah = hi & 0x7fffffffu;
  // (ah << 3) | (lo >> 29): the low 9 exponent bits over the top 23 mantissa bits.
  // Subtracting 384 (= 896 mod 512) in that 9-bit field rebiases 1023 -> 127 for every
  // exponent that has a normal float image (the field result is then 1..254).
  uint32_t b = __funnelshift_l(lo, ah, 3) - 0xC0000000u;
  const uint32_t rest = lo & 0x1fffffffu;                        // 29 discarded bits
  b += (rest > 0x10000000u) | ((rest == 0x10000000u) & b);      // nearest, ties to even
  if (ah < 0x38100000u) b = 0u;                                  // below FLT_MIN: flush to zero
  if (ah >= 0x47f00000u)                                         // overflow, inf, nan
    b = 0x7f800000u | ((ah > 0x7ff00000u || (ah == 0x7ff00000u && lo)) ? 0x400000u : 0u);
  return __uint_as_float(b | (hi & 0x80000000u));
}

// FP64 -> FP32 rounding toward zero: the same rebiasing as d2f_rn without the rounding and
// overflow handling (six integer operations instead of about fourteen).  For finite values
// below FLT_MAX, which the state and the quantities derived from it are; magnitudes below
// FLT_MIN flush to a signed zero.  Relative error below 2^-23.
__device__ __forceinline__ float d2f_rz(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x);
  const uint32_t lo = (uint32_t)__double2loint(x);
  const uint32_t ah = hi & 0x7fffffffu;
  uint32_t b = __funnelshift_l(lo, ah, 3) - 0xC0000000u;
  b = ah < 0x38100000u ? 0u : b;
  return __uint_as_float(b | (hi & 0x80000000u));
}

__device__ __forceinline__ double f2d(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t sign = b & 0x80000000u;
  const uint32_t ex = (b >> 23) & 0xffu;
  const uint32_t man = b & 0x7fffffu;
  uint32_t hi, lo;
  if (ex == 0u) {  // zero (float subnormals flush to zero; the kernels never produce them)
    hi = sign;
    lo = 0u;
  } else if (ex == 255u) {
    hi = sign | 0x7ff00000u | (man >> 3);
    lo = man << 29;
  } else {
    hi = sign | ((ex + 896u) << 20) | (man >> 3);
    lo = man << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// FP32 -> FP64 widening of the flux-precision results (the residual and its increments):
// normal floats are exact; zero and subnormals give a signed zero, infinities and NaN a NaN
// (so that a non-finite result stays non-finite).  Nine integer operations.
__device__ __forceinline__ double f2d_w(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t a = b & 0x7fffffffu;
  uint32_t hi = (a >> 3) + 0x38000000u;   // rebias the exponent 127 -> 1023
  hi = a < 0x00800000u ? 0u : hi;
  hi = a >= 0x7f800000u ? 0x7ff80000u : hi;
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)(b << 29));
}

// The same widening for a float known to be finite (the caller checks): normal floats exact,
// zero a signed zero, subnormals a double of the same sign below 2^-126.  Seven integer
// operations.
__device__ __forceinline__ double f2d_fin(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t a = b & 0x7fffffffu;
  const uint32_t hi = a ? (a >> 3) + 0x38000000u : 0u;
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)(b << 29));
}

// 1/x in FP64 for |x| between 2^-125 and 2^125: an FP32 reciprocal seed (relative error
// below 2^-21) refined by two Newton-Raphson steps y <- y + y (1 - x y), each of which
// squares the error, so the result is within an ulp or two of the quotient.  Four FP64
// operations instead of a full division (which issues at about a ninth of the FP64 FMA
// rate on sm_103a); other x, zero, infinities and NaN take the division.
__device__ __forceinline__ double rcp64(double x) {
  const uint32_t ah = (uint32_t)__double2hiint(x) & 0x7fffffffu;
  if (ah - 0x38200000u >= 0x47c00000u - 0x38200000u) return 1.0 / x;
  double y = f2d(__fdividef(1.0f, d2f_rz(x)));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// Finite test on the exponent bits only (integer pipe).
__device__ __forceinline__ bool finite64(double x) {
  return (((uint32_t)__double2hiint(x)) & 0x7ff00000u) != 0x7ff00000u;
}

// ---------------------------------------------------------------------------------------
// Signal-speed reductions (the Eq. dt_hyp bound) over 64-bit patterns.  A node contributes
// its speed |u| + a >= 0 as a bit pattern, a quiet NaN if one of its inputs is not finite, or
// +infinity if it has rho <= 0 or p <= 0.  Non-negative doubles order like their unsigned bit
// patterns and the quiet NaN lies above +infinity, so one unsigned maximum keeps the worst
// case of a whole state: non-finite > non-positive > the largest speed (a floating-point
// maximum would drop the NaN and return a finite bound for a broken state).
// ---------------------------------------------------------------------------------------
constexpr unsigned long long kSpeedNonFinite = 0x7ff8000000000000ull;
constexpr unsigned long long kSpeedNonPositive = 0x7ff0000000000000ull;

__device__ __forceinline__ unsigned long long speed_bits(double sp, bool finite_in, bool positive) {
  if (!finite_in) return kSpeedNonFinite;
  if (!positive) return kSpeedNonPositive;
  return (unsigned long long)__double_as_longlong(sp);
}

// unsigned maximum over a block (blockDim.x a multiple of 32, at most 1024); the result is
// valid in thread 0
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long x) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  __shared__ unsigned long long red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    x = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
      x = y > x ? y : x;
    }
  }
  return x;
}

// the Euler signal speed of one node (FP64), as a reduction code
template <int DIM>
__device__ __forceinline__ unsigned long long euler_speed_bits(const double* U, long long stride, long long i,
                                                               double gamma) {
  const double rho = U[i];
  bool fin = isfinite(rho);
  double m2 = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const double m = U[(1 + d) * stride + i];
    fin = fin && isfinite(m);
    m2 += m * m;
  }
  const double E = U[(DIM + 1) * stride + i];
  fin = fin && isfinite(E);
  const double p = (gamma - 1.0) * (E - 0.5 * m2 / rho);
  const bool pos = rho > 0.0 && p > 0.0;
  return speed_bits(pos ? sqrt(m2) / rho + sqrt(gamma * p / rho) : 0.0, fin, pos);
}

// ---------------------------------------------------------------------------------------
// Arithmetic traits.  FP32 uses the fast reciprocal/rsqrt unit (a few ulp); FP64 uses
// Newton-refined reciprocals (within two ulp) and the correctly rounded sqrt.
// ---------------------------------------------------------------------------------------
template <class R> struct Ar;

template <> struct Ar<double> {
  static __device__ __forceinline__ double load(double x) { return x; }
  static __device__ __forceinline__ double widen(double x) { return x; }
  static __device__ __forceinline__ double rcp(double x) { return rcp64(x); }
  static __device__ __forceinline__ double div(double a, double b) { return a * rcp64(b); }
  static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  static __device__ __forceinline__ double log(double x) { return ::log(x); }
  static __device__ __forceinline__ double fmax(double a, double b) { return ::fmax(a, b); }
  static __device__ __forceinline__ double fmin(double a, double b) { return ::fmin(a, b); }
  static __device__ __forceinline__ double abs(double a) { return ::fabs(a); }
  // |f|^2 below this uses the series of the log mean (error ~ 0.02 u^5 < 1e-16)
  static constexpr double kLogMeanSeries = 1e-3;
};

template <> struct Ar<float> {
  static __device__ __forceinline__ float load(double x) { return d2f_rz(x); }
  static __device__ __forceinline__ double widen(float x) { return f2d_w(x); }
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float sqrt(float x) { return x * rsqrtf(x); }
  static __device__ __forceinline__ float log(float x) { return logf(x); }
  static __device__ __forceinline__ float fmax(float a, float b) { return fmaxf(a, b); }
  static __device__ __forceinline__ float fmin(float a, float b) { return fminf(a, b); }
  static __device__ __forceinline__ float abs(float a) { return fabsf(a); }
  // |f|^2 below this uses the series (error ~ 0.02 u^5 ~ 2e-12, below FP32 rounding)
  static constexpr float kLogMeanSeries = 1e-2f;
};

// ---------------------------------------------------------------------------------------
// Tensor-product element geometry.
// ---------------------------------------------------------------------------------------
template <int DIM, int N> struct Geo {
  static constexpr int N1 = N + 1;
  static constexpr int NP = (DIM == 2) ? N1 * N1 : N1 * N1 * N1;  // nodes per element
  static constexpr int NFN = (DIM == 2) ? N1 : N1 * N1;            // nodes per face
  static constexpr int NLINE = NP / N1;                            // lines per direction
  static constexpr int NPAIR = N * N1 / 2;                         // pairs a<b per line
  static constexpr int NV = DIM + 2;                               // conserved variables
  // elements per group: enough that the per-node and per-face-node roles fill ~128 threads
  static constexpr int W = (NP > 2 * DIM * NFN) ? NP : 2 * DIM * NFN;
  static constexpr int EPB = (W >= 96) ? 1 : (128 / W);
  // stride of direction l in the node index (i fastest)
  static __host__ __device__ constexpr int stride(int l) { return l == 0 ? 1 : (l == 1 ? N1 : N1 * N1); }
  // node index of the m-th point on line q of direction l
  static __device__ __forceinline__ int line_node(int l, int q, int m) {
    const int S = stride(l);
    return (q % S) + m * S + (q / S) * S * N1;
  }
  // line index and position along direction l of node nd
  static __device__ __forceinline__ int node_line(int l, int nd) {
    const int S = stride(l);
    return (nd % S) + (nd / (S * N1)) * S;
  }
  static __device__ __forceinline__ int node_pos(int l, int nd) { return (nd / stride(l)) % N1; }
};

// ---------------------------------------------------------------------------------------
// Euler physics (Sec. 2).  u: conserved (rho, m_1..m_DIM, E).
//
// Pressure enters the fluxes as the deviation pd = p - p_ref from a global constant p_ref:
// the momentum fluxes use pd, everything else p = pd + p_ref.  A constant added to the
// momentum flux leaves the discrete operator unchanged in exact arithmetic (the rows of D
// sum to zero, and F* - F(U_own) is invariant), and at low Mach number it keeps the
// pressure gradient out of FP32 cancellation.  pd is taken from the FP64 total energy (the
// ideal-gas closure of Sec. 2), pd = g - (gamma-1)/2 |m|^2/rho with g = (gamma-1) E - p_ref:
// g is one FP64 fused multiply-add (the only FP64 operation of a node's primitives), then
// rounded to R; the kinetic part, which carries no cancellation, is formed in R.  Explicit
// rounding intrinsics make every call site produce the same bits, so the two elements
// sharing a face see the same pd.  irho = 1/rho is passed in (Ar<R>::rcp(u[0]) at every
// call site), so that one reciprocal serves pd and the velocities.
// ---------------------------------------------------------------------------------------
// hgm1 = (gamma-1)/2 in R (host-precomputed).
template <int DIM>
__device__ __forceinline__ float pdev_i(const double* u64, const float* u, float irho, double gm1,
                                        double p_ref, float hgm1) {
  float m2 = __fmul_rn(u[1], u[1]);
#pragma unroll
  for (int d = 1; d < DIM; ++d) m2 = __fmaf_rn(u[1 + d], u[1 + d], m2);
  const float g = d2f_rz(__fma_rn(gm1, u64[DIM + 1], -p_ref));
  return __fmaf_rn(-hgm1, __fmul_rn(m2, irho), g);
}

template <int DIM>
__device__ __forceinline__ double pdev_i(const double* u64, const double* u, double irho, double gm1,
                                         double p_ref, double hgm1) {
  (void)u64;
  double m2 = __dmul_rn(u[1], u[1]);
#pragma unroll
  for (int d = 1; d < DIM; ++d) m2 = __fma_rn(u[1 + d], u[1 + d], m2);
  const double g = __fma_rn(gm1, u[DIM + 1], -p_ref);
  return __fma_rn(-hgm1, __dmul_rn(m2, irho), g);
}

// pd of a node from its FP64 state u64 and its flux-precision copy u
template <int DIM, class R>
__device__ __forceinline__ R pdev(const double* u64, const R* u, double gm1, double p_ref, R hgm1) {
  return pdev_i<DIM>(u64, u, Ar<R>::rcp(u[0]), gm1, p_ref, hgm1);
}

// Positivity of a node's state, rho > 0 and p > 0 (equivalently rho e > 0), decided on the
// FP64 values.  FP32: the pressure pd + p_ref formed in FP32 is accepted when it exceeds a
// margin of 2^-18 ((gamma-1)|E| + |p_ref|), which bounds its rounding error; below the
// margin (near vacuum, never in smooth flow) the decision is taken again in FP64 from the
// FP64 state.  FP64: the sign of pd + p_ref.  A NaN density passes (the finite checks of
// the stage outputs catch it).
template <int DIM>
__device__ __forceinline__ bool positive(const double* u64, const float* u, float pd, float p_ref,
                                         float margin_e, float margin_0, double gm1) {
  if (__double2hiint(u64[0]) <= 0) return false;
  if (pd + p_ref > __fmaf_rn(margin_e, fabsf(u[DIM + 1]), margin_0)) return true;
  double m2 = u64[1] * u64[1];
#pragma unroll
  for (int d = 1; d < DIM; ++d) m2 = fma(u64[1 + d], u64[1 + d], m2);
  return gm1 * (u64[DIM + 1] - 0.5 * m2 / u64[0]) > 0.0;
}
template <int DIM>
__device__ __forceinline__ bool positive(const double* u64, const double* u, double pd, double p_ref,
                                         double, double, double) {
  (void)u;
  return __double2hiint(u64[0]) > 0 && pd + p_ref > 0.0;
}

template <int DIM, class R> struct Prim {
  R rho, irho, v[DIM], p, pd;
};

template <int DIM, class R>
__device__ __forceinline__ Prim<DIM, R> prims_i(const R* u, R irho, R pd, R p_ref) {
  Prim<DIM, R> q;
  q.rho = u[0];
  q.irho = irho;
#pragma unroll
  for (int d = 0; d < DIM; ++d) q.v[d] = u[1 + d] * q.irho;
  q.pd = pd;
  q.p = pd + p_ref;
  return q;
}

template <int DIM, class R>
__device__ __forceinline__ Prim<DIM, R> prims(const R* u, R pd, R p_ref) {
  return prims_i<DIM>(u, Ar<R>::rcp(u[0]), pd, p_ref);
}

// The trace of a node as the Riemann fluxes see it: the momentum rebuilt as rho v from the
// primitives.  Every kernel that evaluates a face flux forms its inputs this one way, from
// values each side derives identically from the FP64 state, so that F* gets the same bits
// wherever it is evaluated (both elements of a face, the shock-capturing blend).
template <int DIM, class R>
__device__ __forceinline__ void trace_momentum(const Prim<DIM, R>& q, R* u) {
#pragma unroll
  for (int d = 0; d < DIM; ++d) u[1 + d] = q.rho * q.v[d];
}

// Cartesian flux F^L(U) in direction L (compile-time); momentum carries pd.
template <int DIM, int L, class R>
__device__ __forceinline__ void point_flux(const R* u, const Prim<DIM, R>& q, R* F) {
  const R mn = u[1 + L];
  F[0] = mn;
#pragma unroll
  for (int d = 0; d < DIM; ++d) F[1 + d] = mn * q.v[d] + (d == L ? q.pd : R(0));
  F[DIM + 1] = (u[DIM + 1] + q.p) * q.v[L];
}

// Four flux-precision values loaded or stored as one 16-byte (FP32) shared-memory access.
template <class R>
struct alignas(4 * sizeof(R)) Q4 {
  R x, y, z, w;
};

// Per-node records of Ranocha's two-point flux (App. A), built once per node:
//   A = (rho, beta = rho/p, 2 ln rho, ln beta)      (FP64: the logarithms are not used)
//   B = (v_1, v_2, v_3 (0 in 2D), pd = p - p_ref)
template <int DIM, class R>
__device__ __forceinline__ void ec_records(const Prim<DIM, R>& q, Q4<R>& A, Q4<R>& B) {
  const R beta = q.rho * Ar<R>::rcp(q.p);
  if constexpr (sizeof(R) == 4) A = Q4<R>{q.rho, beta, R(2) * Ar<R>::log(q.rho), Ar<R>::log(beta)};
  else A = Q4<R>{q.rho, beta, R(0), R(0)};
  B = Q4<R>{q.v[0], q.v[1], DIM == 3 ? q.v[DIM - 1] : R(0), q.pd};
}

// Ranocha's EC two-point flux in direction L from two records (App. A; energy component in
// the published consistent form
//   f_rho = rho^ln {{v_L}},  f_m = f_rho {{v}} + {{p}} e_L,
//   f_E = f_rho (1/((gamma-1) beta^ln) + v_a.v_b/2) + (p_a v_b,L + p_b v_a,L)/2,
// where beta = rho/p and {{.}} is the arithmetic mean; {{p}} e_L is carried by pd).
// Logarithmic means: with s = a + b, f = (a - b)/s, u = f^2, a^ln = (s/2)/Fs(u) where
// Fs(u) = atanh(f)/f = 1 + u/3 + u^2/5 + u^3/7 + ... .  For small u (the Ismail-Roe idea of
// a series near a = b) rho^ln/2 = (s/4) G(u), G = 1/Fs = 1 - u/3 - 4u^2/45 - 44u^3/945 -
// c4 u^4, and 1/beta^ln = 2 Fs(u)/s, so that beta^ln is never inverted; otherwise
// rho^ln/2 = (a - b)/(2 ln a - 2 ln b) and 1/beta^ln = (ln a - ln b)/(a - b).  FP32 takes
// the per-node logarithms of the records and evaluates both forms, then selects (no
// divergent branch); the two means share one reciprocal of s_rho s_beta and run as packed
// FP32x2 operations.  FP64 branches and takes the logarithm of the ratio only on the (rare,
// in smooth regions) log branch.  The energy pressure term is split as
// (pd_a v_b,L + pd_b v_a,L)/2 + p_ref {{v_L}}.
// a - b on both lanes (packed FP32x2)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  ra = (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
  rb = (unsigned long long)__float_as_uint(b.x) | ((unsigned long long)__float_as_uint(b.y) << 32);
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  return make_float2(__uint_as_float((unsigned)rd), __uint_as_float((unsigned)(rd >> 32)));
}

// The FP32 flux in three parts, so that a caller may evaluate several pairs under one warp
// vote: the two logarithmic means by their series (ec_log_means), the quotient form where a
// lane needs it (ec_log_means_fix, under the caller's vote), the flux from the means
// (ec_flux_assemble).  ec_flux_rec runs the three for one pair.
struct EcMeans {
  float2 s, d, u;  // sums, differences and squared relative differences of (rho, beta)
  float hr, ib;    // rho^ln / 2 and 1 / beta^ln
  bool lg;         // this lane needs the quotient form for one of the two
};
__device__ __forceinline__ EcMeans ec_log_means(const Q4<float>& a, const Q4<float>& b) {
  EcMeans m;
  const float2 ra = make_float2(a.x, a.y), rb = make_float2(b.x, b.y);  // (rho, beta)
  m.s = __fadd2_rn(ra, rb);
  m.d = sub2(ra, rb);
  float inv;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(m.s.x * m.s.y));
  const float2 is = make_float2(m.s.y * inv, m.s.x * inv);                // (1/s_rho, 1/s_beta)
  const float2 f = __fmul2_rn(m.d, is);
  m.u = __fmul2_rn(f, f);
  // G/4 and 2 Fs by Horner's rule (immediate coefficients)
  float G = __fmaf_rn(-0.25f * 0.030194003527336861f, m.u.x, -0.25f * 44.0f / 945.0f);
  G = __fmaf_rn(G, m.u.x, -0.25f * 4.0f / 45.0f);
  G = __fmaf_rn(G, m.u.x, -0.25f / 3.0f);
  G = __fmaf_rn(G, m.u.x, 0.25f);
  float Fs = __fmaf_rn(2.0f / 9.0f, m.u.y, 2.0f / 7.0f);
  Fs = __fmaf_rn(Fs, m.u.y, 2.0f / 5.0f);
  Fs = __fmaf_rn(Fs, m.u.y, 2.0f / 3.0f);
  Fs = __fmaf_rn(Fs, m.u.y, 2.0f);
  m.hr = m.s.x * G;
  m.ib = is.y * Fs;
  m.lg = !(m.u.x < Ar<float>::kLogMeanSeries) || !(m.u.y < Ar<float>::kLogMeanSeries);
  return m;
}
__device__ __forceinline__ void ec_log_means_fix(const Q4<float>& a, const Q4<float>& b, EcMeans& m) {
  const float2 dl = sub2(make_float2(a.z, a.w), make_float2(b.z, b.w));
  float r0, r1;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(dl.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(m.d.y));
  m.hr = m.u.x < Ar<float>::kLogMeanSeries ? m.hr : m.d.x * r0;
  m.ib = m.u.y < Ar<float>::kLogMeanSeries ? m.ib : dl.y * r1;
}
template <int DIM, int L>
__device__ __forceinline__ void ec_flux_assemble(const Q4<float>& av, const Q4<float>& bv, const EcMeans& m,
                                                 float igm1, float p_ref, float* F) {
  const float hr = m.hr, ib = m.ib;
  const float2 vs01 = __fadd2_rn(make_float2(av.x, av.y), make_float2(bv.x, bv.y));
  const float vs2 = av.z + bv.z;
  const float2 pv = __fmul2_rn(make_float2(av.x, av.y), make_float2(bv.x, bv.y));
  const float vab = __fmaf_rn(av.z, bv.z, pv.x + pv.y);
  const float vsl = L == 0 ? vs01.x : (L == 1 ? vs01.y : vs2);
  const float val = L == 0 ? av.x : (L == 1 ? av.y : av.z);
  const float vbl = L == 0 ? bv.x : (L == 1 ? bv.y : bv.z);
  const float frho = hr * vsl;
  const float hf = 0.5f * frho;
  F[0] = frho;
  const float2 fm = __fmul2_rn(make_float2(hf, hf), vs01);
  F[1] = fm.x;
  F[2] = fm.y;
  if constexpr (DIM == 3) F[3] = hf * vs2;
  F[1 + L] = __fmaf_rn(0.5f, av.w + bv.w, F[1 + L]);
  const float e1 = frho * __fmaf_rn(0.5f, vab, igm1 * ib);
  const float pt = __fmaf_rn(av.w, vbl, bv.w * val);
  F[DIM + 1] = __fmaf_rn(0.5f, __fmaf_rn(p_ref, vsl, pt), e1);
}

template <int DIM, int L>
__device__ __forceinline__ void ec_flux_rec(const Q4<float>& a, const Q4<float>& av, const Q4<float>& b,
                                            const Q4<float>& bv, float igm1, float p_ref, float* F) {
  EcMeans m = ec_log_means(a, b);
  if (__any_sync(__activemask(), m.lg)) ec_log_means_fix(a, b, m);
  ec_flux_assemble<DIM, L>(av, bv, m, igm1, p_ref, F);
}

template <int DIM, int L>
__device__ __forceinline__ void ec_flux_rec(const Q4<double>& a, const Q4<double>& av, const Q4<double>& b,
                                            const Q4<double>& bv, double igm1, double p_ref, double* F) {
  const double sr = a.x + b.x, sb = a.y + b.y, dr = a.x - b.x, db = a.y - b.y;
  const double inv = rcp64(sr * sb);
  const double isr = sb * inv, isb = sr * inv;
  const double fr = dr * isr, fb = db * isb;
  const double ur = fr * fr, ub = fb * fb;
  double hr, ib;
  if (ur < Ar<double>::kLogMeanSeries) {
    const double G = 0.25 + ur * (-0.25 / 3.0 + ur * (-0.25 * 4.0 / 45.0 + ur * (-0.25 * 44.0 / 945.0 +
                                                                                 ur * (-0.25 * 0.030194003527336861))));
    hr = sr * G;
  } else {
    hr = 0.5 * dr * rcp64(::log(a.x * rcp64(b.x)));
  }
  if (ub < Ar<double>::kLogMeanSeries) {
    const double Fs = 2.0 + ub * (2.0 / 3.0 + ub * (2.0 / 5.0 + ub * (2.0 / 7.0 + ub * (2.0 / 9.0))));
    ib = isb * Fs;
  } else {
    ib = ::log(a.y * rcp64(b.y)) * rcp64(db);
  }
  const double vs[3] = {av.x + bv.x, av.y + bv.y, av.z + bv.z};
  const double vab = av.x * bv.x + av.y * bv.y + av.z * bv.z;
  const double va[3] = {av.x, av.y, av.z}, vb[3] = {bv.x, bv.y, bv.z};
  const double frho = hr * vs[L];
  const double hf = 0.5 * frho;
  F[0] = frho;
#pragma unroll
  for (int dd = 0; dd < DIM; ++dd) F[1 + dd] = hf * vs[dd];
  F[1 + L] += 0.5 * (av.w + bv.w);
  F[DIM + 1] = frho * (igm1 * ib + 0.5 * vab) + 0.5 * (av.w * vb[L] + bv.w * va[L] + p_ref * vs[L]);
}

// Log mean a^ln with its series branch (the curved kernel's contracted flux below): with
// s = a+b, f = (a-b)/s, u = f^2, a^ln = (s/2) G(u), G = 1/Fs as above; otherwise
// (a-b)/ln(a/b).  FP32 takes the logarithms la, lb computed once per node and evaluates both
// forms, then selects; FP64 branches.  Arguments: a, b; d = a - b, la, lb (FP32 only),
// s = a + b, f = d / s.
template <class R>
__device__ __forceinline__ R log_mean_from(R a, R b, R d, R la, R lb, R s, R f) {
  const R u = f * f;
  if constexpr (sizeof(R) == 4) {
    const R G = R(1) - u * (R(1.0 / 3.0) + u * (R(4.0 / 45.0) + u * (R(44.0 / 945.0) +
                                                                      u * R(0.030194003527336861))));
    const R lg = d * Ar<R>::rcp(la - lb);
    return u < R(Ar<R>::kLogMeanSeries) ? (R(0.5) * s) * G : lg;
  } else {
    if (u < R(Ar<R>::kLogMeanSeries)) {
      const R G = R(1) - u * (R(1.0 / 3.0) + u * (R(4.0 / 45.0) + u * (R(44.0 / 945.0) +
                                                                        u * R(0.030194003527336861))));
      return (R(0.5) * s) * G;
    }
    return Ar<R>::div(d, Ar<R>::log(Ar<R>::div(a, b)));
  }
}

// The same two-point flux contracted with a direction n, sum_d n_d F#_d (curved elements:
// the contravariant volume flux with the metric terms averaged over the pair, Sec. 3.1.1
// Eq. vol_split with Ja^l): the log means and the velocity products do not depend on the
// direction, so one evaluation replaces DIM of them.
template <int DIM, class R>
__device__ __forceinline__ void ec_flux_prims_n(R rL, const R* vL, R pdL, R bL, R lrL, R lbL, R rR,
                                                const R* vR, R pdR, R bR, R lrR, R lbR, R igm1,
                                                R p_ref, const R* n, R* F) {
  const R sr = rL + rR, sb = bL + bR, dr = rL - rR, db = bL - bR;
  const R inv = Ar<R>::rcp(sr * sb);
  const R fr = dr * (sb * inv);
  const R fb = db * (sr * inv);
  const R rho_ln = log_mean_from(rL, rR, dr, lrL, lrR, sr, fr);
  const R beta_ln = log_mean_from(bL, bR, db, lbL, lbR, sb, fb);
  R vs[DIM];
  R vLvR = R(0), vsn = R(0), vLn = R(0), vRn = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    vs[d] = vL[d] + vR[d];
    vLvR += vL[d] * vR[d];
    vsn += n[d] * vs[d];
    vLn += n[d] * vL[d];
    vRn += n[d] * vR[d];
  }
  const R frho = (R(0.5) * rho_ln) * vsn;
  const R hf = R(0.5) * frho;
  const R pa = R(0.5) * (pdL + pdR);
  F[0] = frho;
#pragma unroll
  for (int d = 0; d < DIM; ++d) F[1 + d] = hf * vs[d] + pa * n[d];
  F[DIM + 1] = frho * (igm1 * Ar<R>::rcp(beta_ln) + R(0.5) * vLvR) +
               R(0.5) * ((pdL + p_ref) * vRn + (pdR + p_ref) * vLn);
}

template <int DIM, int L, class R>
__device__ __forceinline__ void ec_flux(const Prim<DIM, R>& a, const Prim<DIM, R>& b, R igm1,
                                        R p_ref, R* F) {
  Q4<R> aA, aB, bA, bB;
  ec_records<DIM>(a, aA, aB);
  ec_records<DIM>(b, bA, bB);
  ec_flux_rec<DIM, L>(aA, aB, bA, bB, igm1, p_ref, F);
}

// Local Lax-Friedrichs (Rusanov): F* = (F_L + F_R)/2 - lambda/2 (U_R - U_L),
// lambda = max(|u_L| + a_L, |u_R| + a_R) along L (Sec. 3.1.1 "Lax-Friedrichs").
template <int DIM, int L, class R>
__device__ __forceinline__ void rusanov(const R* uL, const Prim<DIM, R>& a, const R* uR,
                                        const Prim<DIM, R>& b, R gamma, R* F) {
  const R cL = Ar<R>::sqrt(gamma * a.p * a.irho), cR = Ar<R>::sqrt(gamma * b.p * b.irho);
  const R lam = Ar<R>::fmax(Ar<R>::abs(a.v[L]) + cL, Ar<R>::abs(b.v[L]) + cR);
  R FL[DIM + 2], FR[DIM + 2];
  point_flux<DIM, L>(uL, a, FL);
  point_flux<DIM, L>(uR, b, FR);
#pragma unroll
  for (int v = 0; v < DIM + 2; ++v) F[v] = R(0.5) * (FL[v] + FR[v]) - R(0.5) * lam * (uR[v] - uL[v]);
}

// Davis/Einfeldt wave-speed estimates with Roe averages (for HLL and HLLC).
template <int DIM, int L, class R>
__device__ __forceinline__ void wave_speeds(const R* uL, const R* uR, const Prim<DIM, R>& a,
                                            const Prim<DIM, R>& b, R gamma, R& SL, R& SR) {
  const R sL = Ar<R>::sqrt(a.rho), sR = Ar<R>::sqrt(b.rho);
  const R iw = Ar<R>::rcp(sL + sR);
  R v2 = R(0), vtL = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const R vt = (sL * a.v[d] + sR * b.v[d]) * iw;
    v2 += vt * vt;
    if (d == L) vtL = vt;
  }
  const R HL = (uL[DIM + 1] + a.p) * a.irho, HR = (uR[DIM + 1] + b.p) * b.irho;
  const R Ht = (sL * HL + sR * HR) * iw;
  const R at = Ar<R>::sqrt((gamma - R(1)) * (Ht - R(0.5) * v2));
  const R cL = Ar<R>::sqrt(gamma * a.p * a.irho), cR = Ar<R>::sqrt(gamma * b.p * b.irho);
  SL = Ar<R>::fmin(a.v[L] - cL, vtL - at);
  SR = Ar<R>::fmax(b.v[L] + cR, vtL + at);
}

template <int DIM, int L, class R>
__device__ __forceinline__ void hll(const R* uL, const Prim<DIM, R>& a, const R* uR,
                                    const Prim<DIM, R>& b, R gamma, R* F) {
  R SL, SR;
  wave_speeds<DIM, L>(uL, uR, a, b, gamma, SL, SR);
  R FL[DIM + 2], FR[DIM + 2];
  point_flux<DIM, L>(uL, a, FL);
  point_flux<DIM, L>(uR, b, FR);
  if (SL >= R(0)) {
#pragma unroll
    for (int v = 0; v < DIM + 2; ++v) F[v] = FL[v];
  } else if (SR <= R(0)) {
#pragma unroll
    for (int v = 0; v < DIM + 2; ++v) F[v] = FR[v];
  } else {
    const R iS = Ar<R>::rcp(SR - SL);
#pragma unroll
    for (int v = 0; v < DIM + 2; ++v) F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (uR[v] - uL[v])) * iS;
  }
}

// HLLC (Toro, Spruce and Speares): S_L >= 0 -> F_L; S* >= 0 -> F*_L; S_R > 0 -> F*_R; else
// F_R (the star flux is always formed and the upwind cases select over it, without a
// branch).  Star state U*_K = rho_K (S_K - u_K)/(S_K - S*) (1, S* e_L + tangential,
// E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))); p_R - p_L is taken as pd_R - pd_L.
// Written in jump form, identical in exact arithmetic: with m_K = rho_K (S_K - u_K),
//   S* - u_L = (dp - m_R du)/(m_L - m_R),  S* - u_R = (dp - m_L du)/(m_L - m_R),
// dp = p_R - p_L, du = u_R - u_L, and delta = (S* - u_K)/(S_K - S*),
//   F*_K = F_K + S_K delta (rho_K, rho_K S_K e_L + rho_K tangential, E_K + p_K + m_K S*).
// The star correction U*_K - U_K is formed from the jumps instead of as a difference of two
// full states, which for the small jumps of smooth flow keeps its FP32 rounding down to that
// of the jumps.
template <int DIM, int L, class R>
__device__ __forceinline__ void hllc(const R* uL, const Prim<DIM, R>& a, const R* uR,
                                     const Prim<DIM, R>& b, R gamma, R* F) {
  R SL, SR;
  wave_speeds<DIM, L>(uL, uR, a, b, gamma, SL, SR);
  R FL[DIM + 2], FR[DIM + 2];
  point_flux<DIM, L>(uL, a, FL);
  point_flux<DIM, L>(uR, b, FR);
  const R mL = a.rho * (SL - a.v[L]), mR = b.rho * (SR - b.v[L]);
  const R dp = b.pd - a.pd, du = b.v[L] - a.v[L];
  const R iden = Ar<R>::rcp(mL - mR);
  const R dL = (dp - mR * du) * iden;  // S* - u_L
  const R Ss = a.v[L] + dL;
  const bool upl = SL >= R(0), upr = SR <= R(0) && Ss < R(0);
  {
    // one star state: left if S* >= 0, else right (selects, not pointers, keep it in
    // registers); the upwind cases select F_L or F_R over it, without a branch
    const bool left = (Ss >= R(0));
    const R SK = left ? SL : SR;
    const R mK = left ? mL : mR;
    const R rK = left ? a.rho : b.rho;
    const R pK = left ? a.p : b.p;
    const R dK = left ? dL : (dp - mL * du) * iden;  // S* - u_K
    const R sK = SK - (left ? a.v[L] : b.v[L]);      // S_K - u_K
    const R sd = SK * Ar<R>::div(dK, sK - dK);       // S_K delta
    const R rs = rK * sd;
    const R EK = left ? uL[DIM + 1] : uR[DIM + 1];
#pragma unroll
    for (int v = 0; v < DIM + 2; ++v) {
      const R FKv = left ? FL[v] : FR[v];
      R w;
      if (v == 0) w = rs;
      else if (v == DIM + 1) w = sd * (EK + pK + mK * Ss);
      else if (v == 1 + L) w = rs * SK;
      else w = rs * (left ? a.v[v - 1] : b.v[v - 1]);
      F[v] = upl ? FL[v] : (upr ? FR[v] : FKv + w);
    }
  }
}

}  // namespace dg
