// Refinement residual R = B - M X of the mixed form on the 5th-generation
// tensor cores (tcgen05, sm_103a), to double-float accuracy (about 2^-48 of
// |M| |X|), by exact fixed-point splitting into bf16 digits (the Ozaki scheme).
//
// Row r of M is scaled by 2^-E_r (2^E_r: the smallest power of two above the
// row's largest |Re| or |Im|, recorded by the assembly), column c of X by
// 2^-F_c (recorded by k_widen / k_ir_update).  Each scaled real value, held as a
// double-float pair, becomes six balanced base-256 digits
//   v 2^7 = sum_{s=1..6} a_s 2^{8 (1 - s)} + rest,  a_s integers, |a_s| <= 129,
//   |rest| <= 2^-41 (2^-48 of the scale),
// all exact in bf16.  A digit product a_s b_t is an integer of at most 129^2 and
// belongs to weight class g = s + t; the 21 pairs with g <= 7 run as bf16
// tcgen05.mma with FP32 accumulation in tensor memory, one accumulator per class.
// Per real K a class sum grows by at most 6 * 129^2 < 2^17, so 128 real K
// accumulate exactly in FP32 (below 2^24): every 4 chunks of 32 real K the
// accumulators are read with tcgen05.ld and added, scaled by 2^{-8 (g - 2)},
// into double-float registers.  The dropped classes (g >= 8) and the digit
// rests stay below 2^-48 of the scales.  The complex product is the real
// embedding
//   [Re MX | Im MX] = [Re M | Im M] x [[Re X, Im X], [-Im X, Re X]].
//
// CTA: 128 rows of one unit (TMEM lanes), 16 complex right-hand-side columns
// (blockIdx.z picks the slice), 8 warps.  Per chunk of 16 complex columns of M:
//   all threads  split 8 elements of M (two threads per row, loaded during the
//                previous chunk's products) into the six digit planes of A and
//                one element of X into the six planes of B (no-swizzle K-major
//                core-matrix layout in shared memory), real and imaginary
//                parts in the two lanes of the paired FP32 instructions;
//   one thread   issues the 42 tcgen05.mma (M = 128, N = 32, K = 16) of the
//                chunk and commits them to an mbarrier (bounded waits, polled
//                by one warp);
//   every 4th    warps 0-3 add the real outputs of their TMEM lanes, warps 4-7
//                the imaginary ones.
#include <cstdint>

#include <cuda_bf16.h>

#include "common.cuh"

namespace lsms {

namespace rtc {

constexpr int ND = 6;        // digits per operand
constexpr int NG = 6;        // weight classes g = 2..7 (index s + t - 2 of digits s, t >= 1)
constexpr int KCC = 16;      // complex columns of M per chunk (32 real K)
constexpr int NC = 16;       // complex right-hand-side columns per CTA
constexpr int TM = 128;      // rows per CTA (TMEM lanes)
constexpr int NT = 256;      // threads: two per row (column halves)
constexpr int NOUT = 2 * NC; // real accumulator columns per class: [Re | Im]
constexpr int LBO = 128;     // bytes between core matrices (8 rows x 16 bytes) adjacent in K
constexpr int SBO = 512;     // bytes between 8-row groups (the 4 core matrices of 32 K)
constexpr int PLANE_A = TM / 8 * SBO;    // 8 KB
constexpr int PLANE_B = NOUT / 8 * SBO;  // 2 KB
constexpr int SMEM_USED = ND * PLANE_A + ND * PLANE_B + 64;
// requested per CTA so that at most two CTAs share an SM (two TMEM allocations of 256 columns)
constexpr int SMEM_LAUNCH = 80 * 1024;
constexpr uint32_t TMEM_COLS = 256;      // NG * NOUT = 192, rounded up to a power of two
constexpr int FLUSH = 4;                 // chunks per exact accumulation window (128 real K)
constexpr long long kWaitLimit = 1ll << 24;
static_assert(SMEM_USED <= SMEM_LAUNCH, "shared memory");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of the 16-byte core-matrix row (row, K unit of 8 elements) in a plane.
__device__ __forceinline__ uint32_t core_off(int row, int kunit) {
  return (uint32_t)((row >> 3) * SBO + kunit * LBO + (row & 7) * 16);
}

// Shared-memory matrix descriptor, K-major, no swizzle: leading byte offset =
// distance between core matrices adjacent in K, stride byte offset = distance
// between 8-row groups; version bits 46-47 = 1.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(LBO >> 4) << 16;
  d |= (uint64_t)(SBO >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16 with bf16 A and B: D f32, both K-major, N and M.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4)                 // D format f32
         | (1u << 7)               // A format bf16
         | (1u << 10)              // B format bf16
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(mbar), "r"(phase)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Exponent E with 0 <= m < 2^E (E = 0 for m = 0): the scale of a row or column.
__device__ __forceinline__ int scale_exp(float m) {
  const int b = (int)((__float_as_uint(m) >> 23) & 0xff);
  return m > 0.f ? (b == 0 ? -126 : b - 126) : 0;
}
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }

// Round to the nearest integer (ties to even) for |x| < 2^22: adding and
// removing 1.5 * 2^23 leaves no fraction bits.
__device__ __forceinline__ float2 rint2(float2 x) {
  const float2 big = make_float2(12582912.f, 12582912.f), nbig = make_float2(-12582912.f, -12582912.f);
  return __fadd2_rn(__fadd2_rn(x, big), nbig);
}

// (r, c) <- (r + c, rounding error) exactly (two-sum), lane-wise.
__device__ __forceinline__ void two_sum2(float2& r, float2& c) {
  const float2 a = __fadd2_rn(r, c);
  const float2 bb = __fadd2_rn(a, make_float2(-r.x, -r.y));
  const float2 e = __fadd2_rn(__fadd2_rn(r, make_float2(bb.x - a.x, bb.y - a.y)), __fadd2_rn(c, make_float2(-bb.x, -bb.y)));
  r = a;
  c = e;
}

// The six digits of the double-float value (h + l) 2^7 / 2^E, sc = 2^{7 - E},
// two values at once (lanes).  With r the remainder in units of the next digit:
// d = rint(r), r = 256 (r - d) (exact); the low part c (|c| <= 2^-17 at the
// start) is folded in exactly (two-sum) before digits 3 and 5, when two steps of
// 256 have made it as large as half a unit, so every digit satisfies |d| <= 129.
__device__ __forceinline__ void digits6x2(float2 h, float2 l, float2 sc, float2* d) {
  const float2 k256 = make_float2(256.f, 256.f), nk256 = make_float2(-256.f, -256.f);
  const float2 k64k = make_float2(65536.f, 65536.f);
  float2 r = __fmul2_rn(h, sc), c = __fmul2_rn(l, sc);
#pragma unroll
  for (int s = 0; s < ND; ++s) {
    if (s == 2 || s == 4) {
      c = __fmul2_rn(c, k64k);
      two_sum2(r, c);
    }
    const float2 q = rint2(r);
    d[s] = q;
    if (s + 1 < ND) r = __ffma2_rn(q, nk256, __fmul2_rn(r, k256));  // 256 r - 256 q: exact
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // digits are small integers: exact
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ unsigned short bf16_bits(float x) {
  const __nv_bfloat16 v = __float2bfloat16_rn(x);
  return *reinterpret_cast<const unsigned short*>(&v);
}

}  // namespace rtc

// grid (ceil(n_max / 128), n_units, ceil(nrhs / 16)), block 256, dynamic smem
// rtc::SMEM_LAUNCH.  X32 = B - M X (rounded to complex64) for the unit's rows of
// this tile and the 16 columns of this slice.  Every wait on the tensor core is
// bounded; on a timeout the unit is flagged LSMS_UNIT_TIMEOUT (and re-solved by
// the FP64 fallback) and the CTA returns after a second bounded wait.
__global__ void __launch_bounds__(256, 2) k_residual_tc(const Unit* __restrict__ units, const char* fac_base, char* ws,
                                                     int K, int nrhs, bool explicit_b, const int32_t* __restrict__ done,
                                                     int32_t* stat) {
  using namespace rtc;
  const Unit u = units[blockIdx.y];
  if (done[u.stat_off]) return;
  const int n = u.n;
  const int row0 = blockIdx.x * TM;
  if (row0 >= n) return;
  const int col0 = blockIdx.z * NC;
  if (col0 >= nrhs) return;
  const float4* M = reinterpret_cast<const float4*>(fac_base + u.m64_off);  // (re.hi, im.hi, re.lo, im.lo)
  const float* rowmax = reinterpret_cast<const float*>(fac_base + u.m64_off + rowmax_rel_off(n));
  const float4* Xdf = reinterpret_cast<const float4*>(ws + u.xdf_off);      // (re.hi, re.lo, im.hi, im.lo)
  const float* colmax = reinterpret_cast<const float*>(ws + u.xdf_off + colmax_rel_off(n, nrhs));

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;                          // ND planes of PLANE_A
  uint8_t* sB = smem + ND * PLANE_A;           // ND planes of PLANE_B
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + ND * PLANE_A + ND * PLANE_B);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + ND * PLANE_A + ND * PLANE_B + 16);
  __shared__ int s_cexp[NC];

  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (tid < NC) s_cexp[tid] = col0 + tid < nrhs ? scale_exp(colmax[col0 + tid]) : 0;
  // epilogue: TMEM lane (warp % 4) * 32 + lane = row rl; warps 0-3 the real outputs, 4-7 the imaginary ones
  const int rl = (warp & 3) * 32 + (tid & 31), half = warp >> 2;
  const int row = row0 + rl;
  const bool live = row < n;
  const int E = live ? scale_exp(rowmax[row]) : 0;
  // A: warp w splits rows 16 w .. 16 w + 15, two lanes per row; lane parity p takes the complex
  // columns 4p .. 4p + 3 and 8 + 4p .. 8 + 4p + 3 of each chunk, so that a warp's 8-byte stores
  // fill two whole core matrices (conflict-free)
  const int arow_l = warp * 16 + ((tid & 31) >> 1), aq0 = (tid & 1) * 4;
  const int arow = row0 + arow_l;
  const bool alive = arow < n;
  const int EA = alive ? scale_exp(rowmax[arow]) : 0;
  const float2 rsc = make_float2(pow2f(7 - EA), pow2f(7 - EA));
  // B: element (row j, column cc) of the chunk's 16 x 16 block of X
  const int bcc = tid & 15, bj = tid >> 4;
  const int bcol = col0 + bcc;
  const int F_b = bcol < nrhs ? scale_exp(colmax[bcol]) : 0;
  const float2 csc = make_float2(pow2f(7 - F_b), pow2f(7 - F_b));
  // epilogue: warps 0-3 the real outputs, warps 4-7 the imaginary ones, of row rl
  float accs[NC], acct[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) accs[c] = acct[c] = 0.f;

  auto load_chunk = [&](int c0, float4* mv, float4& xv) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {  // q < 4: columns aq0 + q; q >= 4: 8 + aq0 + q - 4
      const int col = c0 + (q >> 2) * 8 + aq0 + (q & 3);
      mv[q] = (alive && col < n) ? M[(size_t)col * n + arow] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int j = c0 + bj;
    xv = (bcol < nrhs && j < n) ? Xdf[(size_t)bcol * n + j] : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  // warp 0 polls the mbarrier (bounded) while the others wait at the barrier, leaving the
  // issue slots to the SM's other CTA
  auto wait_mma = [&](int j) -> bool {
    bool ok = true;
    if (warp == 0) {
      ok = false;
      const uint32_t mb = smem_u32(mbar);
      for (long long it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(mb, (uint32_t)(j & 1))) {
          ok = true;
          break;
        }
    }
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return ok;
  };
  auto flush = [&](uint32_t tmem) {
    const uint32_t base = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(half * NC);
#pragma unroll 1
    for (int g = 0; g < NG; ++g) {
      float v[16];
      tmem_ld16(base + (uint32_t)(g * NOUT), v);
      const float w = pow2f(-8 * g);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float x = v[c] * w;  // an integer times a power of two: exact
        const float a = accs[c] + x;
        const float bb = a - accs[c];
        acct[c] += (accs[c] - (a - bb)) + (x - bb);
        accs[c] = a;
      }
    }
  };

  const int nchunks = (n + KCC - 1) / KCC;
  float4 mv[8], xv;
  load_chunk(0, mv, xv);
  uint32_t tmem = 0;
  bool ok = true;
  int issued = -1;
  for (int ch = 0; ch < nchunks; ++ch) {
    if (ch > 0) {
      if (!(ok = wait_mma(ch - 1))) break;          // planes free again, accumulators current
      if (ch % FLUSH == 0) flush(tmem);
    }
    // ---- A planes: this thread's 8 elements (4 in each column half); real parts -> K unit hh,
    // imaginary parts -> K unit 2 + hh, at element offset aq0 within the 8-element unit
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const uint32_t o_re = core_off(arow_l, hh) + aq0 * 2, o_im = core_off(arow_l, 2 + hh) + aq0 * 2;
      float2 d[4][ND];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 v = mv[hh * 4 + q];
        rtc::digits6x2(make_float2(v.x, v.y), make_float2(v.z, v.w), rsc, d[q]);
      }
#pragma unroll
      for (int s = 0; s < ND; ++s) {
        uint2 pr, pi;
        pr.x = rtc::pack_bf16(d[0][s].x, d[1][s].x);
        pr.y = rtc::pack_bf16(d[2][s].x, d[3][s].x);
        pi.x = rtc::pack_bf16(d[0][s].y, d[1][s].y);
        pi.y = rtc::pack_bf16(d[2][s].y, d[3][s].y);
        *reinterpret_cast<uint2*>(sA + s * PLANE_A + o_re) = pr;
        *reinterpret_cast<uint2*>(sA + s * PLANE_A + o_im) = pi;
      }
    }
    // ---- B planes: one element of X; output row bcc (Re): K bj -> Re X, K 16 + bj -> -Im X;
    // output row NC + bcc (Im): K bj -> Im X, K 16 + bj -> Re X
    {
      float2 d[ND];
      rtc::digits6x2(make_float2(xv.x, xv.z), make_float2(xv.y, xv.w), csc, d);
      const uint32_t kb = (uint32_t)((bj & 7) * 2);
      const uint32_t o_re = core_off(bcc, bj >> 3) + kb, o_ren = core_off(bcc, 2 + (bj >> 3)) + kb;
      const uint32_t o_im = core_off(NC + bcc, bj >> 3) + kb, o_imr = core_off(NC + bcc, 2 + (bj >> 3)) + kb;
#pragma unroll
      for (int s = 0; s < ND; ++s) {
        uint8_t* plane = sB + s * PLANE_B;
        const unsigned short re = rtc::bf16_bits(d[s].x), im = rtc::bf16_bits(d[s].y);
        *reinterpret_cast<unsigned short*>(plane + o_re) = re;
        *reinterpret_cast<unsigned short*>(plane + o_ren) = (unsigned short)(im ^ 0x8000u);  // -Im X
        *reinterpret_cast<unsigned short*>(plane + o_im) = im;
        *reinterpret_cast<unsigned short*>(plane + o_imr) = re;
      }
    }
    // the next chunk's elements are loaded while this chunk's products run
    if (ch + 1 < nchunks) load_chunk((ch + 1) * KCC, mv, xv);
    // generic-proxy stores visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem = *tslot;
    if (tid == 0) {
      const uint32_t idesc = make_idesc(TM, NOUT);
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      // first chunk of a window: each class starts from zero with its first product, which in
      // this order (A digit s outer, B digit t inner) is the pair (s = 0, t = g), K step 0
      const bool fresh = (ch % FLUSH) == 0;
#pragma unroll
      for (int s = 0; s < ND; ++s) {
#pragma unroll
        for (int t = 0; t < ND - s; ++t) {
          const int g = s + t;  // weight class of digits (s + 1, t + 1)
#pragma unroll
          for (int ks = 0; ks < 2; ++ks)
            mma_bf16(tmem + (uint32_t)(g * NOUT), make_desc(a0 + s * PLANE_A + ks * 2 * LBO),
                     make_desc(b0 + t * PLANE_B + ks * 2 * LBO), idesc, (fresh && ks == 0 && s == 0) ? 0u : 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(mbar))
                   : "memory");
    }
    issued = ch;
  }
  if (ok && issued >= 0) {
    if ((ok = wait_mma(issued))) flush(tmem);
  }
  if (ok && live) {
    // MX = U 2^{E + F - 14}; this thread holds the real (half 0) or imaginary (half 1) parts
    const double2* B = reinterpret_cast<const double2*>(ws + u.r_off);
    float* X32 = reinterpret_cast<float*>(ws + u.x32_off);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int col = col0 + c;
      if (col >= nrhs) continue;
      const double mx = ldexp((double)accs[c] + (double)acct[c], E + s_cexp[c] - 14);
      double b;
      if (explicit_b) {
        const double2 bb = B[(size_t)col * n + row];
        b = half ? bb.y : bb.x;
      } else {
        b = (half == 0 && row == col && col < K) ? 1.0 : 0.0;
      }
      X32[2 * ((size_t)col * n + row) + half] = (float)(b - mx);
    }
  }
  if (!ok) {
    if (tid == 0) {
      atomicOr(&stat[u.stat_off], LSMS_UNIT_TIMEOUT);
      const uint32_t mb = smem_u32(mbar);
      for (long long it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(mb, (uint32_t)(issued & 1))) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(TMEM_COLS));
  }
}

int residual_tc_chunk(const Unit* d_units, int n_units, int n_max, const char* fac_base, char* ws, int K, int nrhs,
                      bool explicit_b, const int32_t* done, int32_t* stat, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    LSMS_CUDA_TRY(cudaFuncSetAttribute(k_residual_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       rtc::SMEM_LAUNCH));
    attr_set = true;
  }
  const dim3 grid((n_max + rtc::TM - 1) / rtc::TM, n_units, (nrhs + rtc::NC - 1) / rtc::NC);
  LSMS_LAUNCH(k_residual_tc, grid, dim3(rtc::NT), rtc::SMEM_LAUNCH, st, d_units, fac_base, ws, K, nrhs, explicit_b,
              done, stat);
  return LSMS_OK;
}

}  // namespace lsms
