// Device helpers and cross-file kernel wrappers of liblsmskubo.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "internal.h"

namespace lsms {

extern std::atomic<long long> g_launches;

// Optional per-launch CUDA-event timers (off by default), recorded on the
// launch stream around each kernel; read back by lsms_kernel_timer_report.
extern std::atomic<bool> g_timer_on;
void timer_begin(const char* name, cudaStream_t st);
void timer_end(cudaStream_t st);

#define LSMS_CUDA_TRY(expr)                                                              \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      return ::lsms::fail(LSMS_ERR_CUDA, "%s failed: %s (%s:%d)", #expr,                 \
                          cudaGetErrorString(_e), __FILE__, __LINE__);                   \
  } while (0)

// Every kernel launch goes through this: it counts launches and reports a bad
// launch configuration at once.
#define LSMS_LAUNCH(kernel, grid, block, smem, stream, ...)                             \
  do {                                                                                   \
    const bool _tm = ::lsms::g_timer_on.load(std::memory_order_relaxed);                 \
    if (_tm) ::lsms::timer_begin(#kernel, (stream));                                     \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                         \
    if (_tm) ::lsms::timer_end((stream));                                                \
    ::lsms::g_launches.fetch_add(1, std::memory_order_relaxed);                          \
    cudaError_t _e = cudaGetLastError();                                                 \
    if (_e != cudaSuccess)                                                               \
      return ::lsms::fail(LSMS_ERR_CUDA, "launch of %s failed: %s", #kernel,             \
                          cudaGetErrorString(_e));                                       \
  } while (0)

constexpr int kMaxEnergies = 64;
struct EnergyTable {
  double2 z[kMaxEnergies];
};

// ------------------------------------------------------------------ complex
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

template <typename R> struct CxT;
template <> struct CxT<double> { using T = double2; };
template <> struct CxT<float> { using T = float2; };
template <typename R> using Cx = typename CxT<R>::T;

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a*b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc - a*b
template <typename C> __device__ __forceinline__ C cfms(C a, C b, C acc) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
// acc + a^T-free conj(a)*b is not needed; real scale:
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return mk(a.x * s, a.y * s); }

__device__ __forceinline__ double2 crcp(double2 a) {
  const double d = a.x * a.x + a.y * a.y;
  return make_double2(a.x / d, -a.y / d);
}
__device__ __forceinline__ float2 crcp(float2 a) {
  const float d = a.x * a.x + a.y * a.y;
  return make_float2(a.x / d, -a.y / d);
}
__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ float cabs1(float2 a) { return fabsf(a.x) + fabsf(a.y); }

__device__ __forceinline__ float2 to32(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to64(float2 a) { return make_double2((double)a.x, (double)a.y); }
__device__ __forceinline__ double2 to64(double2 a) { return a; }
template <typename C> __device__ __forceinline__ C cvt(double2 a);
template <> __device__ __forceinline__ double2 cvt<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 cvt<float2>(double2 a) { return to32(a); }

__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }
__device__ __forceinline__ bool finite2(float2 a) { return isfinite(a.x) && isfinite(a.y); }

// ------------------------------------------------------------------ double-float
// A real number held as hi + lo in two floats (unit roundoff about 2^-48), for
// FP64-accurate arithmetic on the FP32 pipes: products by the FMA two-product,
// sums by two-sum.  Complex values are float4 (re.hi, re.lo, im.hi, im.lo).

// (s, t) += p with the rounding error of s + p kept exactly (two-sum).
__device__ __forceinline__ void df_add(float& s, float& t, float p) {
  const float a = s + p;
  const float bb = a - s;
  t += (s - (a - bb)) + (p - bb);
  s = a;
}

// (s, t) += (ah + al)(bh + bl): exact ah*bh (FMA two-product) plus the cross terms.
__device__ __forceinline__ void df_mac(float& s, float& t, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  df_add(s, t, p);
  t += e;
}

__device__ __forceinline__ float4 df_split(double2 a) {
  const float rh = (float)a.x, ih = (float)a.y;
  return make_float4(rh, (float)(a.x - (double)rh), ih, (float)(a.y - (double)ih));
}

__device__ __forceinline__ double2 df_join(float4 a) {
  return make_double2((double)a.x + (double)a.y, (double)a.z + (double)a.w);
}

// Packed forms on float2 (the paired FP32 instructions of sm_100 and later: two
// lanes of arithmetic per instruction).  A complex accumulator is s = (re, im)
// high parts and t = (re, im) low parts; a complex product m x splits as
// m.re (x.re, x.im) + m.im (-x.im, x.re), each a real value times a pair.
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

// (s, t) += (ah + al)(bh + bl) lane-wise: exact ah bh (two-product), the cross
// terms, and the two-sum's rounding error into t.  BLO = false: bl is zero (b is
// a float) and its cross term is left out.
template <bool BLO = true>
__device__ __forceinline__ void df2_mac(float2& s, float2& t, float2 ah, float2 al, float2 bh, float2 bl) {
  const float2 p = __fmul2_rn(ah, bh);
  float2 e = __ffma2_rn(ah, bh, f2neg(p));
  if constexpr (BLO) e = __ffma2_rn(ah, bl, e);
  e = __ffma2_rn(al, bh, e);
  const float2 a = __fadd2_rn(s, p);
  const float2 bb = __fadd2_rn(a, f2neg(s));
  const float2 err = __fadd2_rn(__fadd2_rn(s, f2neg(__fadd2_rn(a, f2neg(bb)))), __fadd2_rn(p, f2neg(bb)));
  t = __fadd2_rn(t, __fadd2_rn(err, e));
  s = a;
}

// complex accumulator: re = s.x + t.x, im = s.y + t.y
struct DfAcc {
  float2 s, t;
};
__device__ __forceinline__ DfAcc df_zero() { return DfAcc{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

// acc += a * b (complex, double-float; a, b as (re.hi, re.lo, im.hi, im.lo)).
// Scalar instructions: in the 16 x 16 products that use it, pairing the operands
// for the paired instructions cost more than it saved.
__device__ __forceinline__ void dfc_mac(DfAcc& acc, float4 a, float4 b) {
  df_mac(acc.s.x, acc.t.x, a.x, a.y, b.x, b.y);
  df_mac(acc.s.x, acc.t.x, -a.z, -a.w, b.z, b.w);
  df_mac(acc.s.y, acc.t.y, a.x, a.y, b.z, b.w);
  df_mac(acc.s.y, acc.t.y, a.z, a.w, b.x, b.y);
}

// acc += c * w, c real (hi, lo), w complex (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ void dfr_mac(DfAcc& acc, float2 c, float4 w) {
  df2_mac(acc.s, acc.t, make_float2(c.x, c.x), make_float2(c.y, c.y), make_float2(w.x, w.z), make_float2(w.y, w.w));
}

// normalised (hi, lo) pairs of an accumulator
__device__ __forceinline__ float4 df_value(const DfAcc& a) {
  const float rh = a.s.x + a.t.x, ih = a.s.y + a.t.y;
  return make_float4(rh, a.t.x - (rh - a.s.x), ih, a.t.y - (ih - a.s.y));
}

// Real double-float values (hi, lo) as float2, normalised (|lo| <= ulp(hi) / 2).
__device__ __forceinline__ float2 dd_from(double a) {
  const float h = (float)a;
  return make_float2(h, (float)(a - (double)h));
}
__device__ __forceinline__ float2 dd_norm(float s, float t) {  // fast two-sum, |s| >= |t|
  const float h = s + t;
  return make_float2(h, t - (h - s));
}
__device__ __forceinline__ float2 dd_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bb = s - a.x;
  const float e = (a.x - (s - bb)) + (b.x - bb) + a.y + b.y;
  return dd_norm(s, e);
}
__device__ __forceinline__ float2 dd_sub(float2 a, float2 b) { return dd_add(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 dd_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return dd_norm(p, e);
}
// a * f with f a float (exact small integers in the recurrences)
__device__ __forceinline__ float2 dd_mulf(float2 a, float f) {
  const float p = a.x * f;
  float e = fmaf(a.x, f, -p);
  e = fmaf(a.y, f, e);
  return dd_norm(p, e);
}
// complex double-float as float4 (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ float4 ddc(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }
__device__ __forceinline__ float2 ddc_re(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 ddc_im(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 ddc_mul(float4 a, float4 b) {
  return ddc(dd_sub(dd_mul(ddc_re(a), ddc_re(b)), dd_mul(ddc_im(a), ddc_im(b))),
             dd_add(dd_mul(ddc_re(a), ddc_im(b)), dd_mul(ddc_im(a), ddc_re(b))));
}
__device__ __forceinline__ float4 ddc_sub(float4 a, float4 b) {
  return ddc(dd_sub(ddc_re(a), ddc_re(b)), dd_sub(ddc_im(a), ddc_im(b)));
}
__device__ __forceinline__ float4 ddc_scale(float4 a, float2 s) { return ddc(dd_mul(ddc_re(a), s), dd_mul(ddc_im(a), s)); }
__device__ __forceinline__ float4 ddc_scalef(float4 a, float f) { return ddc(dd_mulf(ddc_re(a), f), dd_mulf(ddc_im(a), f)); }

// ------------------------------------------------------------------ wrappers (lu.cu)
// Blocked right-looking LU with partial pivoting of every unit of a chunk, in
// place in the factor arrays (column-major, ld = n).  Complex128: pivots are
// applied to the panel and the trailing columns only ("progressive" form; the
// solve applies them block by block).  Complex64: afterwards L is put in the row
// order of the final permutation and the pivots are replaced by it (k_lapack_rows).
template <typename R>
int lu_factor_chunk(const Unit* d_units, int n_units, int n_max, char* fac_base,
                    int32_t* stat, cudaStream_t st);
// Solve L U X = P B in place for the n x nrhs column-major block at
// ws + unit.<field> (complex<R>), skipping units whose done flag is set.
template <typename R>
int lu_solve_chunk(const Unit* d_units, int n_units, int n_max, const char* fac_base, char* ws,
                   int which_rhs, int nrhs, const int32_t* done, int32_t* stat, cudaStream_t st);

enum RhsField { RHS_X = 0, RHS_X32 = 1 };

// Refinement residual X32 = B - M X of the mixed form on the tensor cores, bf16
// fixed-point digits with exact FP32 accumulation (resid_tc.cu).
int residual_tc_chunk(const Unit* d_units, int n_units, int n_max, const char* fac_base, char* ws, int K, int nrhs,
                      bool explicit_b, const int32_t* done, int32_t* stat, cudaStream_t st);
int opt_residual_tc();
int opt_solve_cols();
int opt_solve_regs();
int opt_solve_steps();

// One block step of the complex64 triangular solves on the tensor cores (tc_gemm.cu):
// forward X[rows >= 32 (s + 1)] -= L[., block s] X[block s], backward
// X[rows < 32 s] -= U[., block s] X[block s], on the X32 field, nrhs <= 32.
int step_tc_chunk(const Unit* d_units, int n_units, int n_max, const char* fac_base, char* ws, int nrhs,
                  const int32_t* done, int32_t* stat, int s, bool forward, cudaStream_t st);
// Trailing update A22 -= L21 U12 of the complex64 LU on the tensor cores (tc_gemm.cu).
int gemm_tc_chunk(const Unit* d_units, int n_units, int n_max, int k, char* fac_base, int32_t* stat,
                  cudaStream_t st);

int existing_device_data(lsms_liz* liz, DeviceData** out);

// Process-wide options (lsms_set_option).
double opt_growth_limit();
int opt_fallback_slots();
int opt_ir_max_sweeps();

// Index checks of the LSMS_DEBUG_BOUNDS build (python -m paper_2311_12134_gb300.build
// --debug-bounds): a value outside [lo, hi) flags the unit LSMS_UNIT_BAD_INPUT
// and the caller skips the access; no trap.  In normal builds every check is
// the constant true and compiles away.
#ifdef LSMS_DEBUG_BOUNDS
constexpr bool kDebugBounds = true;
#else
constexpr bool kDebugBounds = false;
#endif
__device__ __forceinline__ bool dbg_in(long long v, long long lo, long long hi, int32_t* stat_word) {
  if (!kDebugBounds || (v >= lo && v < hi)) return true;
  atomicOr(stat_word, LSMS_UNIT_BAD_INPUT);
  return false;
}

// Non-negative float maximum into a global word (the bit patterns of
// non-negative floats order like their values); NaN is stored as +inf.
__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
  v += 0.0f;  // -0 -> +0
  if (!(v <= 3.4e38f)) v = __int_as_float(0x7f800000);
  atomicMax(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}
// Warp maximum of non-negative floats (NaN as +inf).
__device__ __forceinline__ float warp_max_nonneg(float v) {
  v += 0.0f;
  if (!(v <= 3.4e38f)) v = __int_as_float(0x7f800000);
  return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
}

}  // namespace lsms
