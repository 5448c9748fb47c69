// Refinement residual R = B - M X of the mixed form on the 5th-generation
// tensor cores (tcgen05, sm_103a), to double-float accuracy (about 2^-48 of
// |M| |X|), by exact fixed-point splitting into bf16 digits (the Ozaki scheme).
//
// Row r of M is scaled by 2^-E_r (2^E_r: the smallest power of two above the
// row's largest |Re| or |Im|, recorded by the assembly), column c of X by
// 2^-F_c (recorded by k_widen / k_ir_update).  Each scaled real value, held as a
// double-float pair, becomes six balanced base-256 digits
//   v 2^8 = sum_{s=1..6} a_s 2^{8 (1 - s)} + rest,  a_s integers,
//   |a_1| <= 256, |a_s| <= 128 for s > 1, |rest| <= 2^-41 (2^-49 of the scale),
// all exact in bf16.  A digit product a_s b_t is an integer below 2^16 and
// belongs to weight class g = s + t; the 21 pairs with g <= 7 run as bf16
// tcgen05.mma with FP32 accumulation in tensor memory, one accumulator per class.
// Per real K a class sum grows by at most 2^17 (at most 6 pairs, first digits up
// to 256), so 128 real K accumulate exactly in FP32 (below 2^24): every 4 chunks
// of 32 real K the accumulators are read with tcgen05.ld and added, scaled by
// 2^{-8 (g - 2)}, into double-float registers.  The dropped classes (g >= 8) and
// the digit rests stay below 2^-48 of the scales.  The complex product is the
// real embedding
//   [Re MX | Im MX] = [Re M | Im M] x [[Re X, Im X], [-Im X, Re X]].
//
// CTA: 128 rows of one unit (TMEM lanes), 16 complex right-hand-side columns
// (blockIdx.z picks the slice), 4 warps.  Per chunk of 16 complex columns of M:
//   all threads  split their row's 32 real values into the six digit planes of
//                A (no-swizzle K-major core-matrix layout in shared memory),
//   warp 0       splits the 16 x 16 block of X into the six planes of B,
//   one thread   issues the 42 tcgen05.mma (M = 128, N = 32, K = 16) of the
//                chunk and commits them to an mbarrier (bounded waits).
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

// Byte offset of element (row, k) in a plane: 8 x 8 core matrices of 16-byte rows.
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

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Exponent E with 0 <= m < 2^E (E = 0 for m = 0): the scale of a row or column.
__device__ __forceinline__ int scale_exp(float m) {
  const int b = (int)((__float_as_uint(m) >> 23) & 0xff);
  return m > 0.f ? (b == 0 ? -126 : b - 126) : 0;
}
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }

// The six digits of the double-float value (h + l) 2^8 / 2^E (scale = 2^{8 - E}):
// d = rint(r), r = (r - d) exact, (r, c) renormalised exactly by two-sum, both
// times 256 (exact).
__device__ __forceinline__ void digits6(float h, float l, float scale, float* d) {
  float r = h * scale, c = l * scale;
#pragma unroll
  for (int s = 0; s < ND; ++s) {
    const float q = rintf(r);
    d[s] = q;
    r -= q;
    const float a = r + c;
    const float bb = a - r;
    const float e = (r - (a - bb)) + (c - bb);
    r = a * 256.f;
    c = e * 256.f;
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // digits are small integers: exact
  return *reinterpret_cast<const uint32_t*>(&v);
}

}  // namespace rtc

// grid (ceil(n_max / 128), n_units, ceil(nrhs / 16)), block 128, dynamic smem
// rtc::SMEM_LAUNCH.  X32 = B - M X (rounded to complex64) for the unit's rows of
// this tile and the 16 columns of this slice.  Every wait on the tensor core is
// bounded; on a timeout the unit is flagged LSMS_UNIT_TIMEOUT (and re-solved by
// the FP64 fallback) and the CTA returns after a second bounded wait.
__global__ void __launch_bounds__(128) k_residual_tc(const Unit* __restrict__ units, const char* fac_base, char* ws,
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
  __shared__ float s_cscale[NC];
  __shared__ int s_cexp[NC];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (tid < NC) {
    const int col = col0 + tid;
    const int F = col < nrhs ? scale_exp(colmax[col]) : 0;
    s_cexp[tid] = F;
    s_cscale[tid] = pow2f(8 - F);
  }
  const int row = row0 + tid;
  const bool live = row < n;
  const int E = live ? scale_exp(rowmax[row]) : 0;
  const float rscale = pow2f(8 - E);

  // double-float accumulators of sum_g acc_g 2^{-8 g}: [Re outputs 0..15 | Im outputs 0..15]
  float accs[NOUT], acct[NOUT];
#pragma unroll
  for (int c = 0; c < NOUT; ++c) accs[c] = acct[c] = 0.f;

  auto wait_mma = [&](int j) -> bool {
    bool ok = false;
    const uint32_t mb = smem_u32(mbar);
    for (long long it = 0; it < kWaitLimit; ++it)
      if (mbar_try_wait(mb, (uint32_t)(j & 1))) {
        ok = true;
        break;
      }
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return ok;
  };
  auto flush = [&](uint32_t tmem) {
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int g = 0; g < NG; ++g) {
      float v[32];
      tmem_ld32(lane_base + (uint32_t)(g * NOUT), v);
      const float w = pow2f(-8 * g);
#pragma unroll
      for (int c = 0; c < NOUT; ++c) {
        const float x = v[c] * w;  // an integer times a power of two: exact
        const float a = accs[c] + x;
        const float bb = a - accs[c];
        acct[c] += (accs[c] - (a - bb)) + (x - bb);
        accs[c] = a;
      }
    }
  };

  const int nchunks = (n + KCC - 1) / KCC;
  uint32_t tmem = 0;
  bool ok = true;
  int issued = -1;
  for (int ch = 0; ch < nchunks; ++ch) {
    if (ch > 0) {
      if (!(ok = wait_mma(ch - 1))) break;          // planes free again, accumulators current
      if (ch % FLUSH == 0) flush(tmem);
    }
    const int c0 = ch * KCC;
    // ---- A planes: this thread's row, 16 complex columns -> 32 real K
    {
      float4 mv[KCC];
#pragma unroll
      for (int jj = 0; jj < KCC; ++jj)
        mv[jj] = (live && c0 + jj < n) ? M[(size_t)(c0 + jj) * n + row] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int part = 0; part < 2; ++part) {    // 0: Re (K 0..15), 1: Im (K 16..31)
#pragma unroll
        for (int half = 0; half < 2; ++half) {  // 8 columns per core-matrix row
          float d[8][ND];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 v = mv[half * 8 + q];
            digits6(part ? v.y : v.x, part ? v.w : v.z, rscale, d[q]);
          }
          const uint32_t off = core_off(tid, part * 2 + half);
#pragma unroll
          for (int s = 0; s < ND; ++s) {
            uint4 pk;
            pk.x = rtc::pack_bf16(d[0][s], d[1][s]);
            pk.y = rtc::pack_bf16(d[2][s], d[3][s]);
            pk.z = rtc::pack_bf16(d[4][s], d[5][s]);
            pk.w = rtc::pack_bf16(d[6][s], d[7][s]);
            *reinterpret_cast<uint4*>(sA + s * PLANE_A + off) = pk;
          }
        }
      }
    }
    // ---- B planes (warp 0): item = (complex column cc, 8 rows jg) of X
    if (warp == 0) {
      const int cc = lane & 15, jg = lane >> 4;
      const int col = col0 + cc;
      const float cs = s_cscale[cc];
      float dr[8][ND], di[8][ND];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = c0 + jg * 8 + q;
        const float4 v = (col < nrhs && j < n) ? Xdf[(size_t)col * n + j] : make_float4(0.f, 0.f, 0.f, 0.f);
        digits6(v.x, v.y, cs, dr[q]);
        digits6(v.z, v.w, cs, di[q]);
      }
      // output row cc (Re): K jg -> Re X, K 2 + jg -> -Im X; output row NC + cc (Im): K jg -> Im X, K 2 + jg -> Re X
      const uint32_t o_re = core_off(cc, 0), o_im = core_off(NC + cc, 0);
#pragma unroll
      for (int s = 0; s < ND; ++s) {
        uint4 pr, pi, pn;
        pr.x = rtc::pack_bf16(dr[0][s], dr[1][s]);
        pr.y = rtc::pack_bf16(dr[2][s], dr[3][s]);
        pr.z = rtc::pack_bf16(dr[4][s], dr[5][s]);
        pr.w = rtc::pack_bf16(dr[6][s], dr[7][s]);
        pi.x = rtc::pack_bf16(di[0][s], di[1][s]);
        pi.y = rtc::pack_bf16(di[2][s], di[3][s]);
        pi.z = rtc::pack_bf16(di[4][s], di[5][s]);
        pi.w = rtc::pack_bf16(di[6][s], di[7][s]);
        pn.x = pi.x ^ 0x80008000u;  // -Im X: flip both bf16 sign bits
        pn.y = pi.y ^ 0x80008000u;
        pn.z = pi.z ^ 0x80008000u;
        pn.w = pi.w ^ 0x80008000u;
        uint8_t* plane = sB + s * PLANE_B;
        *reinterpret_cast<uint4*>(plane + o_re + jg * LBO) = pr;
        *reinterpret_cast<uint4*>(plane + o_re + (2 + jg) * LBO) = pn;
        *reinterpret_cast<uint4*>(plane + o_im + jg * LBO) = pi;
        *reinterpret_cast<uint4*>(plane + o_im + (2 + jg) * LBO) = pr;
      }
    }
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
    const double2* B = reinterpret_cast<const double2*>(ws + u.r_off);
    float2* X32 = reinterpret_cast<float2*>(ws + u.x32_off);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int col = col0 + c;
      if (col >= nrhs) continue;
      const int sh = E + s_cexp[c] - 16;
      const double re = ldexp((double)accs[c] + (double)acct[c], sh);
      const double im = ldexp((double)accs[NC + c] + (double)acct[NC + c], sh);
      double2 b;
      if (explicit_b) b = B[(size_t)col * n + row];
      else b = (row == col && col < K) ? mk(1.0, 0.0) : mk(0.0, 0.0);
      X32[(size_t)col * n + row] = make_float2((float)(b.x - re), (float)(b.y - im));
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
  LSMS_LAUNCH(k_residual_tc, grid, dim3(128), rtc::SMEM_LAUNCH, st, d_units, fac_base, ws, K, nrhs, explicit_b, done,
              stat);
  return LSMS_OK;
}

}  // namespace lsms
