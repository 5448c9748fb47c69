// Trailing update of the complex64 LU on the 5th-generation tensor cores
// (tcgen05, sm_103a): A22 -= L21 U12 for every unit of a chunk.
//
// The complex product is written as one real GEMM (real embedding):
//   [C_re | C_im] -= [L_re  L_im] x [ U_re  U_im ]
//                                   [-U_im  U_re ]
// i.e. A^ = [L_re, L_im] (128 rows x 2 NB), B^ = the 2 NB x 2 N block above.
// Each fp32 operand is split into TF32 hi + lo parts and the product is formed
// as hi*hi + hi*lo + lo*hi ("3xTF32"), accumulated in FP32 in tensor memory,
// which keeps complex64 accuracy for the refinement that follows.
//
// One CTA (4 warps) per 128-row block, walking its 128 x 32 complex output tiles:
//   all threads  load L21 (128 x 32, once) and U12 (32 x 32, per tile), split
//                hi/lo, and store them K-major into shared memory with the
//                128-byte swizzle,
//   one thread   issues 24 tcgen05.mma (M = 128, N = 64, K = 8, kind::tf32)
//                into one of two 64-column TMEM accumulators and commits to
//                that accumulator's mbarrier,
//   all threads  wait (bounded), read the accumulator with tcgen05.ld
//                (warp w owns TMEM lanes 32w..32w+31) and update C in place,
//                one tile behind the products.
#include <cstdint>

#include "common.cuh"

namespace lsms {

namespace tc {

constexpr int NB = 32;            // complex panel width (K of the complex product)
constexpr int TM = 128;           // tile rows (TMEM lanes)
constexpr int TNC = 32;           // complex columns per tile
constexpr int TN = 2 * TNC;       // real accumulator columns: [re | im]
constexpr int CHUNK_A = TM * 128;           // one 128-byte-wide K chunk of A (bytes)
constexpr int CHUNK_B = TN * 128;           // one K chunk of B
constexpr int OP_A = 2 * CHUNK_A;           // real K = 2 NB = 64 tf32 = two chunks
constexpr int OP_B = 2 * CHUNK_B;
constexpr int SMEM_BYTES = 2 * OP_A + 2 * OP_B + 64;  // hi/lo of A and B + barrier + TMEM slot
constexpr uint32_t TMEM_COLS = 64;
constexpr int kPrefetchTiles = 1;            // C tiles requested into L2 ahead of their loads
constexpr long long kWaitLimit = 1ll << 24;  // bounded mbarrier wait (polls)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, k) of a K-major operand with 128-byte swizzle:
// rows are 128 B apart inside a 16 KB K chunk (32 fp32 of K); the 16-byte unit
// index inside a row is XOR-ed with the row index modulo 8.
__device__ __forceinline__ uint32_t swz(int row, int k, int chunk_bytes) {
  const int kc = k >> 5, kb = (k & 31) * 4;
  return (uint32_t)(kc * chunk_bytes + row * 128 + ((((kb >> 4) ^ (row & 7))) << 4) + (kb & 15));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart (stride byte offset), version bits 46-47 = 1.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::tf32: D f32, A/B tf32, both K-major, N and M.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4)                 // D format f32
         | (2u << 7)               // A format tf32
         | (2u << 10)              // B format tf32
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
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

}  // namespace tc

// grid (row tiles, n_units), block 128, dynamic smem tc::SMEM_BYTES.  One CTA
// per 128-row block of a unit's trailing matrix, walking the block's 32-column
// tiles: L21's hi/lo split is staged once, and for tile j the CTA overlaps
//   the tensor-core product of tile j (TMEM accumulator j % 2),
//   the loads of U12 for tile j + 1 and of C for tile j (into registers),
//   the epilogue of tile j - 1 (tcgen05.ld, C - product, store).
// Every wait on the tensor core is bounded; on a timeout the unit is flagged
// LSMS_UNIT_TIMEOUT, the walk stops, and the CTA waits (bounded) for its last
// issued product before freeing the accumulators.
__global__ void __launch_bounds__(128) k_gemm_tc(const Unit* __restrict__ units, char* fac_base, int k,
                                                 int32_t* stat) {
  using namespace tc;
  const Unit u = units[blockIdx.y];
  const int n = u.n;
  const int t0 = k + NB;
  const int mt = n - t0;
  if (mt <= 0) return;
  const int ti = blockIdx.x;
  if (ti * TM >= mt) return;
  const int tn = (mt + TNC - 1) / TNC;
  const int row0 = t0 + ti * TM;
  float2* A = reinterpret_cast<float2*>(fac_base + u.fac_off);

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAh = smem;
  uint8_t* sAl = smem + OP_A;
  uint8_t* sBh = smem + 2 * OP_A;
  uint8_t* sBl = smem + 2 * OP_A + OP_B;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * OP_A + 2 * OP_B);  // [2], one per accumulator
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 2 * OP_A + 2 * OP_B + 16);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // two TMEM accumulators of 64 columns (warp 0 allocates; the address lands in shared memory)
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(2 * TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }

  // hi (TF32-rounded) and lo parts of four values, stored at K offset kk of row rr
  auto put = [](uint8_t* sh, uint8_t* sl, int rr, int kk, int chunk, float a0, float a1, float a2, float a3) {
    float4 h, l;
    h.x = tf32_hi(a0); h.y = tf32_hi(a1); h.z = tf32_hi(a2); h.w = tf32_hi(a3);
    l.x = a0 - h.x; l.y = a1 - h.y; l.z = a2 - h.z; l.w = a3 - h.w;
    *reinterpret_cast<float4*>(sh + swz(rr, kk, chunk)) = h;
    *reinterpret_cast<float4*>(sl + swz(rr, kk, chunk)) = l;
  };

  // U12 columns of tile j: thread loads column bc = tid / 4, rows j0 .. j0 + 7
  // (64 contiguous bytes; 16-byte loads when n is even)
  const int bc = tid >> 2, j0 = (tid & 3) * 8;
  float2 w[8];
  auto load_b = [&](int j) {
    const int col = t0 + j * TNC + bc;
    const float2* src = A + (size_t)col * n + k + j0;
    if (col >= n) {
#pragma unroll
      for (int q = 0; q < 8; ++q) w[q] = make_float2(0.f, 0.f);
    } else if ((n & 1) == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 t4 = __ldg(reinterpret_cast<const float4*>(src) + q);
        w[2 * q] = make_float2(t4.x, t4.y);
        w[2 * q + 1] = make_float2(t4.z, t4.w);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) w[q] = __ldg(src + q);
    }
  };
  // B^ row bc (output column bc, real part):      [U_re(., bc) | -U_im(., bc)]
  // B^ row bc + 32 (output column bc, imaginary): [U_im(., bc) |  U_re(., bc)]
  auto store_b = [&]() {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float2* x = w + 4 * h;
      const int kk = j0 + 4 * h;
      put(sBh, sBl, bc, kk, CHUNK_B, x[0].x, x[1].x, x[2].x, x[3].x);
      put(sBh, sBl, bc, NB + kk, CHUNK_B, -x[0].y, -x[1].y, -x[2].y, -x[3].y);
      put(sBh, sBl, bc + TNC, kk, CHUNK_B, x[0].y, x[1].y, x[2].y, x[3].y);
      put(sBh, sBl, bc + TNC, NB + kk, CHUNK_B, x[0].x, x[1].x, x[2].x, x[3].x);
    }
  };
  // C tile j, this thread's row (32 complex entries)
  const int crow = row0 + warp * 32 + lane;
  float2 cv[TNC];
  auto load_c = [&](int j) {
    const int c0 = t0 + j * TNC;
#pragma unroll
    for (int c = 0; c < TNC; ++c)
      cv[c] = (crow < n && c0 + c < n) ? A[(size_t)(c0 + c) * n + crow] : make_float2(0.f, 0.f);
  };

  // C tile j requested into L2 ahead of its loads: the tile's 32 column segments
  // of 128 rows are 256 lines of 128 bytes, two per thread (column tid / 4)
  auto prefetch_c = [&](int j) {
    const int col = t0 + j * TNC + (tid >> 2);
    if (col >= n) return;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = row0 + ((tid & 3) * 2 + h) * 16;
      if (row < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(A + (size_t)col * n + row));
    }
  };
  for (int j = 0; j < kPrefetchTiles && j < tn; ++j) prefetch_c(j);

  // A^ row r = [L_re(r, 0..31) | L_im(r, 0..31)]: thread r, one coalesced load per column
  {
    const int row = row0 + tid;
    const bool ok = row < n;
    float2 v[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) v[j] = ok ? __ldg(&A[(size_t)(k + j) * n + row]) : make_float2(0.f, 0.f);
    load_b(0);
#pragma unroll
    for (int q = 0; q < NB / 4; ++q) {
      put(sAh, sAl, tid, 4 * q, CHUNK_A, v[4 * q].x, v[4 * q + 1].x, v[4 * q + 2].x, v[4 * q + 3].x);
      put(sAh, sAl, tid, NB + 4 * q, CHUNK_A, v[4 * q].y, v[4 * q + 1].y, v[4 * q + 2].y, v[4 * q + 3].y);
    }
  }

  // bounded wait, CTA-uniform outcome (tcgen05.ld is warp-collective)
  auto wait_mma = [&](int j) -> bool {
    bool ok = false;
    const uint32_t mb = smem_u32(mbar + (j & 1));
    const uint32_t parity = (uint32_t)((j >> 1) & 1);
    for (long long it = 0; it < kWaitLimit; ++it)
      if (tc::mbar_try_wait(mb, parity)) {
        ok = true;
        break;
      }
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return ok;
  };
  auto epilogue = [&](int j, uint32_t tmem) {
    const uint32_t lane_base = tmem + (uint32_t)((j & 1) * TMEM_COLS) + ((uint32_t)(warp * 32) << 16);
    float dre[32], dim[32];
    tc::tmem_ld32(lane_base + 0, dre);   // columns 0..31: real parts
    tc::tmem_ld32(lane_base + 32, dim);  // columns 32..63: imaginary parts
    const int c0 = t0 + j * TNC;
    if (crow < n) {
#pragma unroll
      for (int c = 0; c < TNC; ++c)
        if (c0 + c < n) A[(size_t)(c0 + c) * n + crow] = make_float2(cv[c].x - dre[c], cv[c].y - dim[c]);
    }
  };

  uint32_t tmem = 0;
  int issued = -1;  // last tile whose product was issued
  bool ok = true;
  for (int j = 0; j < tn; ++j) {
    if (j > 0 && !(ok = wait_mma(j - 1))) break;  // product j - 1 done: B stage free, accumulator ready
    store_b();
    // make the generic-proxy stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem = *tslot;
    if (tid == 0) {
      const uint32_t idesc = make_idesc(TM, TN);
      const uint32_t d = tmem + (uint32_t)((j & 1) * TMEM_COLS);
      const uint32_t a_hi = smem_u32(sAh), a_lo = smem_u32(sAl), b_hi = smem_u32(sBh), b_lo = smem_u32(sBl);
      uint32_t acc = 0;
      // hi*hi, hi*lo, lo*hi
      for (int s = 0; s < 3; ++s) {
        const uint32_t ab = (s == 2) ? a_lo : a_hi;
        const uint32_t bb = (s == 1) ? b_lo : b_hi;
#pragma unroll
        for (int kc = 0; kc < 2; ++kc)
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) {
            mma_tf32(d, make_desc(ab + kc * CHUNK_A + k4 * 32), make_desc(bb + kc * CHUNK_B + k4 * 32), idesc, acc);
            acc = 1;
          }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(mbar + (j & 1)))
                   : "memory");
    }
    issued = j;
    if (j + 1 < tn) load_b(j + 1);
    if (j + kPrefetchTiles < tn) prefetch_c(j + kPrefetchTiles);
    if (j > 0) epilogue(j - 1, tmem);
    load_c(j);
  }
  if (ok && issued >= 0) {
    if ((ok = wait_mma(issued))) epilogue(issued, tmem);
  }
  if (!ok) {
    if (tid == 0) {
      atomicOr(&stat[u.stat_off], LSMS_UNIT_TIMEOUT);
      // give the tensor core a second bounded window before the accumulators are freed
      const uint32_t mb = smem_u32(mbar + (issued & 1));
      for (long long it = 0; it < kWaitLimit; ++it)
        if (tc::mbar_try_wait(mb, (uint32_t)((issued >> 1) & 1))) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(2 * TMEM_COLS));
  }
}

int gemm_tc_chunk(const Unit* d_units, int n_units, int n_max, int k, char* fac_base, int32_t* stat,
                  cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    LSMS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
    attr_set = true;
  }
  const int mt = n_max - k - tc::NB;
  if (mt <= 0) return LSMS_OK;
  const int tm = (mt + tc::TM - 1) / tc::TM;
  LSMS_LAUNCH(k_gemm_tc, dim3(tm, n_units), dim3(128), tc::SMEM_BYTES, st, d_units, fac_base, k, stat);
  return LSMS_OK;
}

}  // namespace lsms

namespace lsms {

// One block step of the complex64 triangular solves on the tensor cores, the
// same 3xTF32 real-embedding product as k_gemm_tc with the solved block as B:
//   forward (L y = P b):  X[r] -= L[r, 32 s .. 32 s + 31] y_s  for r >= 32 (s + 1),
//   backward (U x = y):   X[r] -= U[r, 32 s .. 32 s + nbp - 1] x_s  for r < 32 s,
// y_s / x_s = the rows 32 s .. of X (final before the launch), X = the unit's
// n x nrhs complex64 right-hand-side block (nrhs <= 32: one 32-column tile, the
// columns beyond nrhs zero); the tile that holds the next block (s + 1 forward,
// s - 1 backward) then multiplies it by the stored inverse of its diagonal block.
// grid (row tiles of 128, n_units), block 128, dynamic smem tc::SMEM_BYTES (so at
// most two CTAs per SM); one 64-column TMEM accumulator; the wait on the tensor
// core is bounded (LSMS_UNIT_TIMEOUT).
__global__ void __launch_bounds__(128) k_step_tc(const Unit* __restrict__ units, const char* fac_base, char* ws,
                                                 int nrhs, const int32_t* __restrict__ done, int32_t* stat, int s,
                                                 int forward) {
  using namespace tc;
  const Unit u = units[blockIdx.y];
  if (done && done[u.stat_off]) return;
  const int n = u.n, nb = (n + NB - 1) / NB;
  const int kc = NB * s;
  int r_begin, r_end;
  if (forward) {
    if (s < 0 || s + 1 >= nb) return;
    r_begin = kc + NB;
    r_end = n;
  } else {
    if (s >= nb || s < 1) return;
    r_begin = 0;
    r_end = kc;
  }
  const int row0 = r_begin + blockIdx.x * TM;
  if (row0 >= r_end) return;
  const int nbp = min(NB, n - kc);
  const float2* F = reinterpret_cast<const float2*>(fac_base + u.fac_off);
  float2* X = reinterpret_cast<float2*>(ws + u.x32_off);

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAh = smem;
  uint8_t* sAl = smem + OP_A;
  uint8_t* sBh = smem + 2 * OP_A;
  uint8_t* sBl = smem + 2 * OP_A + OP_B;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * OP_A + 2 * OP_B);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 2 * OP_A + 2 * OP_B + 16);
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
  auto put = [](uint8_t* sh, uint8_t* sl, int rr, int kk, int chunk, float a0, float a1, float a2, float a3) {
    float4 h, l;
    h.x = tf32_hi(a0); h.y = tf32_hi(a1); h.z = tf32_hi(a2); h.w = tf32_hi(a3);
    l.x = a0 - h.x; l.y = a1 - h.y; l.z = a2 - h.z; l.w = a3 - h.w;
    *reinterpret_cast<float4*>(sh + swz(rr, kk, chunk)) = h;
    *reinterpret_cast<float4*>(sl + swz(rr, kk, chunk)) = l;
  };
  // B^ from the solved block: output column bc = tid / 4, block rows j0 .. j0 + 7
  {
    const int bc = tid >> 2, j0 = (tid & 3) * 8;
    float2 w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      w[q] = (bc < nrhs && j0 + q < nbp) ? X[(size_t)bc * n + kc + j0 + q] : make_float2(0.f, 0.f);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float2* x = w + 4 * h;
      const int kk = j0 + 4 * h;
      put(sBh, sBl, bc, kk, CHUNK_B, x[0].x, x[1].x, x[2].x, x[3].x);
      put(sBh, sBl, bc, NB + kk, CHUNK_B, -x[0].y, -x[1].y, -x[2].y, -x[3].y);
      put(sBh, sBl, bc + TNC, kk, CHUNK_B, x[0].y, x[1].y, x[2].y, x[3].y);
      put(sBh, sBl, bc + TNC, NB + kk, CHUNK_B, x[0].x, x[1].x, x[2].x, x[3].x);
    }
  }
  // A^ row r = [F_re(r, kc ..) | F_im(r, kc ..)]: thread r, one coalesced load per column
  {
    const int row = row0 + tid;
    const bool ok = row < r_end;
    float2 v[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
      v[j] = (ok && j < nbp) ? __ldg(&F[(size_t)(kc + j) * n + row]) : make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NB / 4; ++q) {
      put(sAh, sAl, tid, 4 * q, CHUNK_A, v[4 * q].x, v[4 * q + 1].x, v[4 * q + 2].x, v[4 * q + 3].x);
      put(sAh, sAl, tid, NB + 4 * q, CHUNK_A, v[4 * q].y, v[4 * q + 1].y, v[4 * q + 2].y, v[4 * q + 3].y);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    const uint32_t idesc = make_idesc(TM, TN);
    const uint32_t a_hi = smem_u32(sAh), a_lo = smem_u32(sAl), b_hi = smem_u32(sBh), b_lo = smem_u32(sBl);
    uint32_t acc = 0;
    for (int p = 0; p < 3; ++p) {  // hi*hi, hi*lo, lo*hi
      const uint32_t ab = (p == 2) ? a_lo : a_hi;
      const uint32_t bb = (p == 1) ? b_lo : b_hi;
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          mma_tf32(tmem, make_desc(ab + c2 * CHUNK_A + k4 * 32), make_desc(bb + c2 * CHUNK_B + k4 * 32), idesc, acc);
          acc = 1;
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
  }
  // this thread's row of X while the products run
  const int crow = row0 + warp * 32 + lane;
  const bool live = crow < r_end;
  float2 cv[TNC];
#pragma unroll
  for (int c = 0; c < TNC; ++c) cv[c] = (live && c < nrhs) ? X[(size_t)c * n + crow] : make_float2(0.f, 0.f);
  bool ok = false;
  for (long long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(smem_u32(mbar), 0u)) {
      ok = true;
      break;
    }
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    float dre[32], dim[32];
    tmem_ld32(lane_base + 0, dre);
    tmem_ld32(lane_base + 32, dim);
    if (live) {
#pragma unroll
      for (int c = 0; c < TNC; ++c)
        if (c < nrhs) X[(size_t)c * n + crow] = make_float2(cv[c].x - dre[c], cv[c].y - dim[c]);
    }
  } else if (tid == 0) {
    atomicOr(&stat[u.stat_off], LSMS_UNIT_TIMEOUT);
    for (long long it = 0; it < kWaitLimit; ++it)
      if (mbar_try_wait(smem_u32(mbar), 0u)) break;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(TMEM_COLS));
  }
  // the tile that holds the next block finalizes it after its own update:
  // y = T^{-1} X[block] with the stored inverse of the diagonal block (L forward,
  // U backward); the operand planes are free again (the products completed)
  int fb = -1;
  if (forward) {
    if (blockIdx.x == 0 && s + 1 < nb) fb = s + 1;
  } else if (s >= 1 && (int)blockIdx.x == (NB * (s - 1)) / TM) {
    fb = s - 1;
  }
  if (fb >= 0 && ok) {
    float2(*sT)[NB + 1] = reinterpret_cast<float2(*)[NB + 1]>(smem);
    float2(*sIn)[NB + 1] = reinterpret_cast<float2(*)[NB + 1]>(smem + NB * (NB + 1) * sizeof(float2));
    const float2* D = reinterpret_cast<const float2*>(fac_base + u.m64_off + diag_inv_rel_off(n)) +
                      (size_t)fb * 2 * NB * NB + (forward ? 0 : NB * NB);
    const int k0 = NB * fb, fbp = min(NB, n - k0);
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
      const int i = idx % NB, c = idx / NB;
      sT[i][c] = D[idx];
      sIn[i][c] = (c < nrhs && i < fbp) ? X[(size_t)c * n + k0 + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
      const int i = idx % NB, c = idx / NB;
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < NB; j += 2) {
        a0 = cfma(sT[i][j], sIn[j][c], a0);
        a1 = cfma(sT[i][j + 1], sIn[j + 1][c], a1);
      }
      if (i < fbp && c < nrhs) X[(size_t)c * n + k0 + i] = make_float2(a0.x + a1.x, a0.y + a1.y);
    }
  }
}

int step_tc_chunk(const Unit* d_units, int n_units, int n_max, const char* fac_base, char* ws, int nrhs,
                  const int32_t* done, int32_t* stat, int s, bool forward, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    LSMS_CUDA_TRY(cudaFuncSetAttribute(k_step_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
    attr_set = true;
  }
  if (nrhs < 1 || nrhs > tc::TNC) return fail(LSMS_ERR_ARG, "internal: step_tc_chunk nrhs %d", nrhs);
  const int rows = forward ? n_max - tc::NB * (s + 1) : tc::NB * s;
  if (rows <= 0) return LSMS_OK;
  LSMS_LAUNCH(k_step_tc, dim3((rows + tc::TM - 1) / tc::TM, n_units), dim3(128), tc::SMEM_BYTES, st, d_units,
              fac_base, ws, nrhs, done, stat, s, forward ? 1 : 0);
  return LSMS_OK;
}

}  // namespace lsms
