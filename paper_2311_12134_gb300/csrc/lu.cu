// Batched blocked LU with partial pivoting and the block solves for the tau
// column blocks.
//
// Eq. (tau-inverse) needs [T^{-1} - g]^{-1}; for each (atom, energy) unit the
// LIZ matrix M (n = K S, column-major, ld = n) is factored P M = L U in place.
// Pivoting: the row with the largest |Re| + |Im| in the column, the lowest row
// on ties.  Right-looking, panel width NB:
//   k_panel      factor the n-k x NB panel (pivot search by warp shuffles),
//   k_swap_trsm  apply the panel's row swaps to the columns right of it and
//                form U12 = L11^{-1} A12 (one warp per column); columns left
//                of the panel are not swapped (L is kept as computed, LINPACK
//                style),
//   k_gemm       A22 -= L21 U12: register-tiled complex GEMM on the FP64 pipe
//                (FP64 form); the complex64 form uses k_gemm_tc (tc_gemm.cu),
//                the same update on the tensor cores.
// Units of a chunk are sorted by n (largest first); each launch covers every
// unit and units already finished return at once.  k_solve (FP64) and
// k_solve_c64 (complex64) then run blocked forward/backward substitution; the
// forward sweep applies each panel's row swaps to the right-hand sides just
// before that panel's block of L, so the right-hand sides come in unpermuted.
#include <algorithm>
#include <type_traits>

#include <cooperative_groups.h>

#include "common.cuh"

namespace lsms {

template <typename R> struct LuCfg { static constexpr int NB = 32; };

__device__ __forceinline__ double2 shfl2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// The row interchanges of one factor panel (rows k + j <-> sp[j], j = 0..31 in
// order; sp[j] = k + j for no interchange) applied to one column by one warp.
// Lane j holds row k + j of the column in x on entry and exit; rows below the
// panel that the interchanges reach are read and written in place.  When those
// rows are all distinct (the usual case) each is read once up front and written
// once at the end and the sequence runs in registers; repeated targets take the
// sequential path through memory.
template <typename C>
__device__ __forceinline__ C panel_swaps(C x, C* col, const int* sp, int k, int lane) {
  constexpr int NB = 32;
  const int pj = sp[lane];
  const bool outj = pj >= k + NB;
  const unsigned same = __match_any_sync(0xffffffffu, outj ? pj : -1 - lane);
  const bool fast = !__any_sync(0xffffffffu, outj && __popc(same) > 1);
  if (fast) {
    C y = outj ? col[pj] : x;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int p = sp[j];
      if (p == k + j) continue;
      if (p < k + NB) {
        const int b = p - k;
        const C va = shfl2(x, j);
        const C vb = shfl2(x, b);
        if (lane == j) x = vb;
        if (lane == b) x = va;
      } else if (lane == j) {
        const C t = y;
        y = x;
        x = t;
      }
    }
    if (outj) col[pj] = y;
  } else {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int p = sp[j];
      if (p == k + j) continue;
      if (p < k + NB) {
        const int b = p - k;
        const C va = shfl2(x, j);
        const C vb = shfl2(x, b);
        if (lane == j) x = vb;
        if (lane == b) x = va;
      } else {
        if (lane == j) {
          const C t = col[p];
          col[p] = x;
          x = t;
        }
        __syncwarp();
      }
    }
  }
  return x;
}

// Asynchronous global -> shared copy of one complex element (cp.async: 8 bytes
// for complex64, 16 for complex128); completed by cp.async.wait_all.
__device__ __forceinline__ void cp_async_elem(float2* dst, const float2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2* dst, const double2* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

// ------------------------------------------------------------------ panel
template <typename R, int NB>
__global__ void __launch_bounds__(1024) k_panel(const Unit* __restrict__ units, char* fac_base, int k,
                                               int32_t* stat, int max_rows) {
  using C = Cx<R>;
  const Unit u = units[blockIdx.x];
  const int n = u.n;
  if (k >= n || n - k <= max_rows) return;  // k_panel_smem factors those
  C* A = reinterpret_cast<C*>(fac_base + u.fac_off);
  int32_t* piv = reinterpret_cast<int32_t*>(fac_base + u.piv_off);
  const int nbp = min(NB, n - k);
  __shared__ R s_val[32];
  __shared__ int s_idx[32];
  __shared__ C s_row[NB];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  int flags = 0;
  float umax = 0.f;  // complex64: largest |U| entry of the panel rows this thread saw (column k + tid)
  for (int j = 0; j < nbp; ++j) {
    const int col = k + j;
    const C* Ac = A + (size_t)col * n;
    R best = R(-1);
    int bidx = n;
    for (int i = col + tid; i < n; i += blockDim.x) {
      const R v = cabs1(Ac[i]);
      if (v > best) { best = v; bidx = i; }  // strict: first (lowest) row kept; NaN never wins
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const R ov = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
      if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
    }
    if (lane == 0) { s_val[warp] = best; s_idx[warp] = bidx; }
    __syncthreads();
    if (warp == 0) {
      best = lane < nwarps ? s_val[lane] : R(-1);
      bidx = lane < nwarps ? s_idx[lane] : n;
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        const R ov = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
        if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
      }
      if (lane == 0) s_piv = (bidx < n) ? bidx : col;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != col) {
      for (int c = tid; c < nbp; c += blockDim.x) {
        C* a = A + (size_t)(k + c) * n;
        const C t = a[col];
        a[col] = a[p];
        a[p] = t;
      }
    }
    if (tid == 0) piv[col] = p;
    __syncthreads();
    for (int c = tid; c < nbp; c += blockDim.x) s_row[c] = A[(size_t)(k + c) * n + col];
    __syncthreads();
    if constexpr (std::is_same<R, float>::value) {
      if (tid >= j && tid < nbp) umax = fmaxf(umax, cabs1(s_row[tid]));  // row col of U
    }
    const C pv = s_row[j];
    const bool zero = (pv.x == R(0) && pv.y == R(0));
    if (zero) flags |= LSMS_UNIT_ZERO_PIVOT;
    if (!finite2(pv)) flags |= LSMS_UNIT_NONFINITE;
    const C r = zero ? mk(R(0), R(0)) : crcp(pv);
    for (int i = col + 1 + tid; i < n; i += blockDim.x) {
      C* ai = A + (size_t)col * n + i;
      const C l = cmul(*ai, r);
      if (!zero) *ai = l;
      for (int c = j + 1; c < nbp; ++c) {
        C* a = A + (size_t)(k + c) * n + i;
        *a = cfms(l, s_row[c], *a);
      }
    }
    __syncthreads();
  }
  if (tid == 0 && flags) atomicOr(&stat[u.stat_off], flags);
  if constexpr (std::is_same<R, float>::value) {
    if (warp == 0) {
      const float wm = warp_max_nonneg(umax);
      if (lane == 0) atomic_max_nonneg(reinterpret_cast<float*>(fac_base + u.m64_off + growth_rel_off(n)) + 1, wm);
    }
  }
}

// Panel factorization held in shared memory: the m = n - k rows x NB columns of
// the panel are read once (cp.async), factored column by column in shared
// memory, and written back once.  Units whose panel does not fit (m > max_rows)
// are left to k_panel, which works in global memory.
// One thread per physical row (the launch takes the tallest panel of its units
// rounded up to a warp, at most 1024 threads, so short panels leave room for more
// CTAs per SM).  Rows never move in
// shared memory: each thread keeps the logical (pivoted) number of its row in a
// register, so a row interchange is two register updates.  The pivot search
// for column j + 1 runs inside the update of column j (on the values just
// written), which leaves one block barrier per column.  Same arithmetic and pivot
// choices as the row-swapping form (largest |Re| + |Im|, lowest logical row on
// ties, NaN never chosen unless the whole column is NaN).
constexpr int kPanelThreads = 1024;

template <typename R, int NB>
__global__ void __launch_bounds__(kPanelThreads) k_panel_smem(const Unit* __restrict__ units, char* fac_base, int k,
                                                              int32_t* stat, int max_rows) {
  using C = Cx<R>;
  constexpr int NT = kPanelThreads, NW = NT / 32;
  static_assert(NW <= 32, "one warp reduces the warp results");
  const Unit u = units[blockIdx.x];
  const int n = u.n;
  if (k >= n) return;
  const int m = n - k;
  const int nw = blockDim.x >> 5;  // warps launched: ceil(rows / 32), at most NW
  if (m > max_rows || m > (int)blockDim.x) return;
  extern __shared__ __align__(16) unsigned char panel_raw[];
  C* sP = reinterpret_cast<C*>(panel_raw);  // [NB][m], column-major, physical rows
  C* A = reinterpret_cast<C*>(fac_base + u.fac_off);
  int32_t* piv = reinterpret_cast<int32_t*>(fac_base + u.piv_off);
  const int nbp = min(NB, m);
  __shared__ R s_val[2][NW];
  __shared__ int s_lg[2][NW], s_ph[2][NW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool own = tid < m;  // this thread's physical row is tid
  if (own)
    for (int c = 0; c < nbp; ++c) cp_async_elem(&sP[c * m + tid], &A[(size_t)(k + c) * n + k + tid]);
  asm volatile("cp.async.wait_all;" ::: "memory");
  int lg = tid;  // logical row of physical row tid
  // warp-level best (value, logical row, physical row); lowest logical row on ties
  auto warp_best = [&](R& best, int& bl, int& bp) {
    if constexpr (std::is_same<R, float>::value) {
      // single-instruction warp reductions: the magnitude as an order-preserving
      // key (non-negative floats order like their bit patterns; NaN and
      // non-candidates (best < 0) get key 0), then the lowest logical row among
      // the lanes holding the largest key
      const unsigned key = best >= 0.f ? __float_as_uint(best) + 1u : 0u;
      const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
      const unsigned lmin = __reduce_min_sync(0xffffffffu, key == kmax ? (unsigned)bl : 0xffffffffu);
      const unsigned win = __ballot_sync(0xffffffffu, key == kmax && (unsigned)bl == lmin);
      const int src = __ffs(win) - 1;
      best = __shfl_sync(0xffffffffu, best, src);
      bp = __shfl_sync(0xffffffffu, bp, src);
      bl = (int)lmin;
    } else {
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        const R ov = __shfl_xor_sync(0xffffffffu, best, off);
        const int ol = __shfl_xor_sync(0xffffffffu, bl, off);
        const int op = __shfl_xor_sync(0xffffffffu, bp, off);
        if (ov > best || (ov == best && ol < bl)) { best = ov; bl = ol; bp = op; }
      }
    }
  };
  auto mag = [](C v) -> R {  // |Re| + |Im|; NaN below every number
    const R a = cabs1(v);
    return a >= R(0) ? a : R(-0.5);
  };
  {
    R best = own ? mag(sP[tid]) : R(-1);
    int bl = own ? tid : m, bp = tid;
    warp_best(best, bl, bp);
    if (lane == 0) { s_val[0][warp] = best; s_lg[0][warp] = bl; s_ph[0][warp] = bp; }
  }
  __syncthreads();
  int flags = 0;
  // Rolled: the fully unrolled loop (both precisions) gives the same factors
  // and is no faster.  Invariants the loop rests on: thread t alone writes
  // physical row t; the pivot row's thread has logical row j during step j and
  // does not write, so its values read by the others are those of step j - 1;
  // the warp results of step j + 1 go to the other parity buffer than those
  // read in step j, and the step's barrier separates both from step j + 2.
  bool dead = false;  // LSMS_DEBUG_BOUNDS: a pivot index out of range stops the panel (CTA-uniform)
#pragma unroll 1
  for (int j = 0; j < NB; ++j) {
    if (j < nbp && !dead) {
      const int par = j & 1;
      R best = lane < nw ? s_val[par][lane] : R(-1);  // nw <= 32 warp results
      int bl = lane < nw ? s_lg[par][lane] : m, bp = lane < nw ? s_ph[par][lane] : 0;
      warp_best(best, bl, bp);
      const int p = bl, pph = bp;
      if (kDebugBounds) {
        int32_t* sw = &stat[u.stat_off];
        if (!(dbg_in(p, j, m, sw) & dbg_in(pph, 0, m, sw))) {
          if (tid == 0)
            for (int jj = j; jj < nbp; ++jj) piv[k + jj] = k + jj;
          dead = true;
          continue;
        }
      }
      if (tid == 0) piv[k + j] = k + p;
      lg = lg == j ? p : (lg == p ? j : lg);  // interchange logical rows j and p
      const C pv = sP[j * m + pph];
      const bool zero = (pv.x == R(0) && pv.y == R(0));
      if (zero) flags |= LSMS_UNIT_ZERO_PIVOT;
      if (!finite2(pv)) flags |= LSMS_UNIT_NONFINITE;
      const C rcp = zero ? mk(R(0), R(0)) : crcp(pv);
      best = R(-1);
      bl = m;
      bp = tid;
      if (own && lg > j) {
        const C l = cmul(sP[j * m + tid], rcp);
        if (!zero) sP[j * m + tid] = l;
#pragma unroll
        for (int c = j + 1; c < NB; ++c) {
          if (c < nbp) {
            const C v = cfms(l, sP[c * m + pph], sP[c * m + tid]);
            sP[c * m + tid] = v;
            if (c == j + 1) {
              best = mag(v);
              bl = lg;
            }
          }
        }
      }
      if (j + 1 < nbp) {
        warp_best(best, bl, bp);
        if (lane == 0) { s_val[par ^ 1][warp] = best; s_lg[par ^ 1][warp] = bl; s_ph[par ^ 1][warp] = bp; }
      }
      __syncthreads();
    }
  }
  // write back in logical order
  if (own && dbg_in(lg, 0, m, &stat[u.stat_off]))
    for (int c = 0; c < nbp; ++c) A[(size_t)(k + c) * n + k + lg] = sP[c * m + tid];
  if (tid == 0 && flags) atomicOr(&stat[u.stat_off], flags);
  if constexpr (std::is_same<R, float>::value) {
    // pivot growth: rows that became rows of U (logical row < nbp), columns right of the diagonal
    float umax = 0.f;
    if (own && lg < nbp)
      for (int c = lg; c < nbp; ++c) umax = fmaxf(umax, cabs1(sP[c * m + tid]));
    const float wm = warp_max_nonneg(umax);
    if (lane == 0) atomic_max_nonneg(reinterpret_cast<float*>(fac_base + u.m64_off + growth_rel_off(n)) + 1, wm);
  }
}

// ------------------------------------------------------------------ tall panels on a cluster
// Panels taller than shared memory holds (m = n - k above max_rows) on a
// cluster of kPanelCluster CTAs per unit (thread-block cluster, distributed
// shared memory): CTA r owns the physical rows [r R, (r + 1) R) of the panel,
// R = ceil(m / kPanelCluster), up to kClusterRows per thread, kept in global
// memory (the panel is L2-resident: 32 columns).  As in k_panel_smem, rows do not
// move during the panel: each thread keeps the logical number of each of its
// rows, a pivot exchanges two logical numbers, and the pivot search of column
// j + 1 runs inside the update of column j.  Per column one cluster barrier:
// every CTA publishes its best candidate (|Re| + |Im|, lowest logical row on
// ties, NaN only if the whole column is NaN) in a parity slot of its shared
// memory and, after the barrier, reads all kPanelCluster slots through
// distributed shared memory, so all CTAs take the same pivot; the barrier's
// release/acquire also orders the row updates of one column before the next
// column's reads (those go to L2, ld.global.cg).  At the end, the at most 64 rows
// whose logical and physical numbers differ are read into shared memory,
// a cluster barrier, and written to their logical positions.  Same pivots and
// arithmetic as the single-CTA panels.
constexpr int kPanelCluster = 8;
constexpr int kClusterThreads = 1024;
constexpr int kClusterRows = 3;  // rows per thread: m <= 8 x 1024 x 3 = 24,576

template <typename R, int NB>
__global__ void __cluster_dims__(kPanelCluster, 1, 1) __launch_bounds__(kClusterThreads, 1)
    k_panel_cluster(const Unit* __restrict__ units, char* fac_base, int k, int32_t* stat, int max_rows) {
  using C = Cx<R>;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const Unit u = units[blockIdx.y];
  const int n = u.n;
  if (k >= n || n - k <= max_rows) return;  // the same for every CTA of the cluster (one unit)
  const int m = n - k, nbp = min(NB, m);
  const int per = (m + kPanelCluster - 1) / kPanelCluster;
  if (per > kClusterRows * kClusterThreads) return;  // the host launches k_panel instead
  C* A = reinterpret_cast<C*>(fac_base + u.fac_off);
  int32_t* piv = reinterpret_cast<int32_t*>(fac_base + u.piv_off);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rbeg = rank * per, rend = min(m, rbeg + per);
  __shared__ R c_val[2];  // this CTA's candidate per parity (read by the cluster)
  __shared__ int c_lg[2], c_ph[2];
  __shared__ R w_val[32];
  __shared__ int w_lg[32], w_ph[32];
  __shared__ int s_p, s_pph;
  __shared__ C s_prow[NB];
  __shared__ C s_move[64][NB];  // rows whose logical and physical numbers differ
  __shared__ int s_mtgt[64], s_nmove;
  auto at = [&](int i, int c) -> C* { return A + (size_t)(k + c) * n + k + i; };
  auto warp_best = [](R& best, int& bl, int& bp) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const R ov = __shfl_xor_sync(0xffffffffu, best, off);
      const int ol = __shfl_xor_sync(0xffffffffu, bl, off);
      const int op = __shfl_xor_sync(0xffffffffu, bp, off);
      if (ov > best || (ov == best && ol < bl)) { best = ov; bl = ol; bp = op; }
    }
  };
  auto mag = [](C v) -> R {  // |Re| + |Im|; NaN below every number
    const R a = cabs1(v);
    return a >= R(0) ? a : R(-0.5);
  };
  // the CTA's best (value, logical, physical) into its parity slot
  auto publish = [&](R best, int bl, int bp, int par) {
    warp_best(best, bl, bp);
    if (lane == 0) { w_val[warp] = best; w_lg[warp] = bl; w_ph[warp] = bp; }
    __syncthreads();
    if (warp == 0) {
      best = w_val[lane];
      bl = w_lg[lane];
      bp = w_ph[lane];
      warp_best(best, bl, bp);
      if (lane == 0) { c_val[par] = best; c_lg[par] = bl; c_ph[par] = bp; }
    }
  };
  int lg[kClusterRows];
#pragma unroll
  for (int t = 0; t < kClusterRows; ++t) lg[t] = rbeg + tid + t * kClusterThreads;
  auto own = [&](int t) { return rbeg + tid + t * kClusterThreads < rend; };
  {
    R best = R(-1);
    int bl = m, bp = 0;
#pragma unroll
    for (int t = 0; t < kClusterRows; ++t)
      if (own(t)) {
        const R v = mag(__ldcg(at(lg[t], 0)));
        if (v > best || (v == best && lg[t] < bl)) { best = v; bl = lg[t]; bp = lg[t]; }
      }
    publish(best, bl, bp, 0);
  }
  cluster.sync();
  int flags = 0;
  for (int j = 0; j < nbp; ++j) {
    const int par = j & 1;
    if (warp == 0) {  // every CTA reduces the cluster's candidates itself: the same pivot everywhere
      R best = R(-1);
      int bl = m, bp = 0;
      if (lane < kPanelCluster) {
        best = *cluster.map_shared_rank(&c_val[par], lane);
        bl = *cluster.map_shared_rank(&c_lg[par], lane);
        bp = *cluster.map_shared_rank(&c_ph[par], lane);
      }
      warp_best(best, bl, bp);
      if (lane == 0) { s_p = bl; s_pph = bp; }
    }
    __syncthreads();
    const int p = s_p, pph = s_pph;
    if (rank == 0 && tid == 0) piv[k + j] = k + p;
#pragma unroll
    for (int t = 0; t < kClusterRows; ++t) lg[t] = lg[t] == j ? p : (lg[t] == p ? j : lg[t]);
    // the pivot row (physical pph, logical j now) was last written in column j - 1 by its owner
    if (tid < nbp - j) s_prow[j + tid] = __ldcg(at(pph, j + tid));
    __syncthreads();
    const C pv = s_prow[j];
    const bool zero = (pv.x == R(0) && pv.y == R(0));
    if (zero) flags |= LSMS_UNIT_ZERO_PIVOT;
    if (!finite2(pv)) flags |= LSMS_UNIT_NONFINITE;
    const C rcp = zero ? mk(R(0), R(0)) : crcp(pv);
    R best = R(-1);
    int bl = m, bp = 0;
#pragma unroll
    for (int t = 0; t < kClusterRows; ++t) {
      const int i = rbeg + tid + t * kClusterThreads;
      if (i < rend && lg[t] > j) {
        const C l = cmul(__ldcg(at(i, j)), rcp);
        if (!zero) *at(i, j) = l;
        for (int c = j + 1; c < nbp; ++c) {
          const C v = cfms(l, s_prow[c], __ldcg(at(i, c)));
          *at(i, c) = v;
          if (c == j + 1) {
            const R a = mag(v);
            if (a > best || (a == best && lg[t] < bl)) { best = a; bl = lg[t]; bp = i; }
          }
        }
      }
    }
    if (j + 1 < nbp) publish(best, bl, bp, par ^ 1);
    cluster.sync();  // candidates and this column's row updates visible to the cluster
  }
  // rows out of place: read them, then (after every CTA has read its own) write them
  if (tid == 0) s_nmove = 0;
  __syncthreads();
  float umax = 0.f;
#pragma unroll
  for (int t = 0; t < kClusterRows; ++t) {
    const int i = rbeg + tid + t * kClusterThreads;
    if (i >= rend) continue;
    if constexpr (std::is_same<R, float>::value) {
      if (lg[t] < nbp)  // a row of U: columns from its diagonal
        for (int c = lg[t]; c < nbp; ++c) umax = fmaxf(umax, cabs1(__ldcg(at(i, c))));
    }
    if (lg[t] != i) {
      const int slot = atomicAdd(&s_nmove, 1);  // at most 64 rows leave their place in a panel
      if (slot < 64) {
        s_mtgt[slot] = lg[t];
        for (int c = 0; c < nbp; ++c) s_move[slot][c] = __ldcg(at(i, c));
      }
    }
  }
  cluster.sync();
  const int nmove = min(s_nmove, 64);
  for (int x = tid; x < nmove * nbp; x += blockDim.x) {
    const int slot = x / nbp, c = x % nbp;
    *at(s_mtgt[slot], c) = s_move[slot][c];
  }
  if (rank == 0 && tid == 0 && flags) atomicOr(&stat[u.stat_off], flags);
  if constexpr (std::is_same<R, float>::value) {
    const float wm = warp_max_nonneg(umax);
    if (lane == 0 && wm > 0.f)
      atomic_max_nonneg(reinterpret_cast<float*>(fac_base + u.m64_off + growth_rel_off(n)) + 1, wm);
  }
  cluster.sync();  // no CTA leaves while others may still read its shared memory
}

// ------------------------------------------------------------------ swap + trsm
// Columns right of the panel, one thread per column (256 columns per CTA): the
// panel's row interchanges, then U12 = L11^{-1} A12.  The 32 interchanges are
// the same for every column, so the CTA composes them once into a permutation
// of the panel rows and the rows below the panel they reach: each thread then
// loads its column's 32 panel rows already permuted (gathers), writes the rows
// below the panel (their new values always come from panel rows), solves the
// unit-lower triangle in registers with L11 read as shared-memory broadcasts,
// and stores the 32 rows.  One broadcast of L11 serves 32 columns, where a
// warp per column needed a shuffle or shared-memory access per step and
// column.  Columns left of the panel keep their row order (L is stored as
// computed, LINPACK style): the forward solve applies each panel's
// interchanges to the right-hand sides before that panel's columns of L are used.
// The 32 interchanges of panel k (row k + j with row piv[k + j], j = 0..nbp-1,
// applied in order) composed into one gather, by one warp: panel row k + i takes
// the value of row src[i]; the distinct rows below the panel that the
// interchanges reach, tgt[q] (q < *nt), take the value of row tgt_src[q] (always
// a panel row).  Read every source before writing any target.
__device__ __noinline__ void compose_panel_swaps(const int32_t* piv, int k, int nbp, int lane, int* step,
                                                    int* tgt, int* src, int* tgt_src, int* nt) {
  constexpr int NB = 32;
  const int p = lane < nbp ? piv[k + lane] : k + lane;
  const bool out = p >= k + NB;
  // distinct rows below the panel: each gets a slot 32 + t, t = rank of its first occurrence
  const unsigned same = __match_any_sync(0xffffffffu, out ? p : -1 - lane);
  const int first = __ffs(same) - 1;
  const unsigned firsts = __ballot_sync(0xffffffffu, out && first == lane);
  const int t = __popc(firsts & ((1u << first) - 1u));
  step[lane] = p == k + lane ? -1 : (out ? NB + t : p - k);  // slot exchanged with slot lane
  if (out && first == lane) tgt[t] = p;
  const int n_tgt = __popc(firsts);
  if (lane == 0) *nt = n_tgt;
  __syncwarp();
  // the slot whose starting value ends in slot s: the interchanges undone in reverse order
  auto origin = [&](int s) {
    for (int j = NB - 1; j >= 0; --j) {
      const int o = step[j];
      if (o < 0) continue;
      if (s == j) s = o;
      else if (s == o) s = j;
    }
    return s;
  };
  auto row_of = [&](int s) { return s < NB ? k + s : tgt[s - NB]; };
  src[lane] = row_of(origin(lane));
  if (lane < n_tgt) tgt_src[lane] = row_of(origin(NB + lane));
  __syncwarp();
}

constexpr int kSwapCols = 256;  // columns per CTA of k_swap_trsm
constexpr int kSwapTileBytes = 32 * (kSwapCols + 1) * 8;  // complex64 panel-row tile of k_swap_trsm

// Complex64 body of k_swap_trsm: the panel rows k .. k + 31 of the CTA's columns
// move between global and shared memory as coalesced 32-row column segments (a
// warp per column, lane = row); each thread then gathers its column's
// interchanged rows from the tile, solves in registers and puts them back.
// Rows below the panel that the interchanges reach are read and written directly.
template <int NB>
__device__ __forceinline__ void k_swap_trsm_staged(float2* A, int n, int k, int c0, const float2 (*sL)[NB + 1],
                                                   const int* sTgtRow, const int* sSrcRow, const int* sTgtSrc,
                                                   const int* sNt, float* growth_u) {
  extern __shared__ float2 sTile[];  // [NB][kSwapCols + 1]
  constexpr int LD = kSwapCols + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ncols = min(kSwapCols, n - c0);
  // the tile's 256-byte column segments requested into L2 at once (two lines per thread), so
  // the warps' loads below find them there
  for (int x = tid; x < 2 * ncols; x += blockDim.x)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(A + (size_t)(c0 + (x >> 1)) * n + k + 16 * (x & 1)));
  for (int cc = warp; cc < ncols; cc += 8) sTile[lane * LD + cc] = A[(size_t)(c0 + cc) * n + k + lane];
  __syncthreads();
  float umax = 0.f;  // pivot growth: largest |U12| entry of this column
  if (tid < ncols) {
    float2* Ac = A + (size_t)(c0 + tid) * n;
    float2 x[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {  // gathered: the interchanged panel rows
      const int r = sSrcRow[i];
      x[i] = r < k + NB ? sTile[(r - k) * LD + tid] : Ac[r];
    }
    // rows below the panel: new values from panel rows (in the tile)
    const int nt = *sNt;
    for (int q = 0; q < nt; ++q) Ac[sTgtRow[q]] = sTile[(sTgtSrc[q] - k) * LD + tid];
    // U12 = L11^{-1} A12 (unit lower), by rows
#pragma unroll
    for (int i = 1; i < NB; ++i) {
      float2 a0 = x[i], a1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < i; j += 2) {
        a0 = cfms(sL[i][j], x[j], a0);
        if (j + 1 < i) a1 = cfms(sL[i][j + 1], x[j + 1], a1);
      }
      x[i] = make_float2(a0.x + a1.x, a0.y + a1.y);
    }
    // the column's tile entries were read above by this thread only
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      sTile[i * LD + tid] = x[i];
      umax = fmaxf(umax, cabs1(x[i]));
    }
  }
  {
    const float wm = warp_max_nonneg(umax);
    if (lane == 0) atomic_max_nonneg(growth_u, wm);
  }
  __syncthreads();
  for (int cc = warp; cc < ncols; cc += 8) A[(size_t)(c0 + cc) * n + k + lane] = sTile[lane * LD + cc];
}

template <typename R, int NB>
__global__ void __launch_bounds__(256) k_swap_trsm(const Unit* __restrict__ units, char* fac_base, int k,
                                                   int32_t* stat) {
  using C = Cx<R>;
  static_assert(NB == 32, "one warp of interchanges");
  const Unit u = units[blockIdx.y];
  const int n = u.n;
  const int c0 = k + NB + blockIdx.x * kSwapCols;
  if (c0 >= n) return;  // columns right of the panel exist only when the panel is full
  C* A = reinterpret_cast<C*>(fac_base + u.fac_off);
  const int32_t* piv = reinterpret_cast<const int32_t*>(fac_base + u.piv_off);
  if (kDebugBounds) {  // the panel's pivots must lie in [k + j, n)
    const bool bad = threadIdx.x < NB && !dbg_in(piv[k + threadIdx.x], k + threadIdx.x, n, &stat[u.stat_off]);
    if (__syncthreads_or(bad)) return;
  }
  __shared__ C sL[NB][NB + 1];
  __shared__ int sStep[NB];       // slot exchanged with slot j at interchange j (-1: none)
  __shared__ int sTgtRow[NB];     // row of target slot 32 + t
  __shared__ int sSrcRow[NB];     // panel row i takes the value of row sSrcRow[i]
  __shared__ int sTgtSrc[NB];     // target row t takes the value of (panel) row sTgtSrc[t]
  __shared__ int sNt;             // number of distinct rows below the panel
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx % NB, j = idx / NB;
    sL[i][j] = A[(size_t)(k + j) * n + k + i];
  }
  if (tid < 32) compose_panel_swaps(piv, k, NB, tid, sStep, sTgtRow, sSrcRow, sTgtSrc, &sNt);
  if constexpr (sizeof(C) == 8) {
    k_swap_trsm_staged<NB>(A, n, k, c0, sL, sTgtRow, sSrcRow, sTgtSrc, &sNt,
                           reinterpret_cast<float*>(fac_base + u.m64_off + growth_rel_off(n)) + 1);
    return;
  }
  __syncthreads();
  const int c = c0 + tid;
  if (c >= n) return;
  C* Ac = A + (size_t)c * n;
  C x[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) x[i] = Ac[sSrcRow[i]];  // gathered: the interchanged panel rows
  // rows below the panel: new values from panel rows, which are written only at the end
  const int nt = sNt;
  for (int q0 = 0; q0 < nt; q0 += 8) {
    C tv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) tv[q] = q0 + q < nt ? Ac[sTgtSrc[q0 + q]] : mk(R(0), R(0));
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q0 + q < nt) Ac[sTgtRow[q0 + q]] = tv[q];
  }
  // U12 = L11^{-1} A12 (unit lower), by rows
#pragma unroll
  for (int i = 1; i < NB; ++i) {
    C a0 = x[i], a1 = mk(R(0), R(0));
#pragma unroll
    for (int j = 0; j < i; j += 2) {
      a0 = cfms(sL[i][j], x[j], a0);
      if (j + 1 < i) a1 = cfms(sL[i][j + 1], x[j + 1], a1);
    }
    x[i] = mk(a0.x + a1.x, a0.y + a1.y);
  }
#pragma unroll
  for (int i = 0; i < NB; ++i) Ac[k + i] = x[i];
}

// ------------------------------------------------------------------ trailing GEMM (SIMT)
// Tile 64 x 64, K slices of 16; thread (ty, tx) owns rows ty + 16 r, columns tx + 16 c.
template <typename R, int NB>
__global__ void __launch_bounds__(256) k_gemm(const Unit* __restrict__ units, char* fac_base, int k,
                                              int tiles_max) {
  using C = Cx<R>;
  const Unit u = units[blockIdx.y];
  const int n = u.n;
  const int t0 = k + NB;
  const int mt = n - t0;
  if (mt <= 0) return;
  const int tiles = (mt + 63) >> 6;
  const int ti = blockIdx.x / tiles_max, tj = blockIdx.x % tiles_max;
  if (ti >= tiles || tj >= tiles) return;
  C* A = reinterpret_cast<C*>(fac_base + u.fac_off);
  const int row0 = t0 + 64 * ti, col0 = t0 + 64 * tj;
  __shared__ C sA[16][64];
  __shared__ C sB[16][65];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  C acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = mk(R(0), R(0));
  for (int ks = 0; ks < NB; ks += 16) {
    for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
      const int i = idx & 63, kk = idx >> 6;
      const int row = row0 + i;
      sA[kk][i] = row < n ? A[(size_t)(k + ks + kk) * n + row] : mk(R(0), R(0));
      const int kk2 = idx & 15, j = idx >> 4;
      const int col = col0 + j;
      sB[kk2][j] = col < n ? A[(size_t)col * n + k + ks + kk2] : mk(R(0), R(0));
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      C a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = sA[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = sB[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = cfma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int col = col0 + tx + 16 * c;
    if (col >= n) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int row = row0 + ty + 16 * r;
      if (row < n) {
        C* a = A + (size_t)col * n + row;
        *a = csub(*a, acc[r][c]);
      }
    }
  }
}

// ------------------------------------------------------------------ solve
// X[i][c] -= sum_j A[i][k + j] sX[j][c] for rows i in [r0, r1): one thread per
// (row, group of 4 right-hand sides); the NB column entries of A are loaded 8 at
// a time before use so that the loads overlap.
template <typename R, int NB>
__device__ __forceinline__ void update_rows(const Cx<R>* __restrict__ A, Cx<R>* X, const Cx<R> (*sX)[33], int n, int k,
                                            int nbp, int r0, int r1, int nrhs, int tid, int nthr) {
  using C = Cx<R>;
  constexpr int G = 4;  // right-hand sides per thread
  const int rows = r1 - r0;
  if (rows <= 0) return;
  const int ngrp = (nrhs + G - 1) / G;
  for (int idx = tid; idx < rows * ngrp; idx += nthr) {
    const int i = r0 + idx % rows, g = (idx / rows) * G;
    C acc[G];
#pragma unroll
    for (int c = 0; c < G; ++c) acc[c] = (g + c < nrhs) ? X[(size_t)(g + c) * n + i] : mk(R(0), R(0));
    for (int j0 = 0; j0 < nbp; j0 += 8) {
      C l[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) l[jj] = (j0 + jj < nbp) ? A[(size_t)(k + j0 + jj) * n + i] : mk(R(0), R(0));
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
#pragma unroll
        for (int c = 0; c < G; ++c) acc[c] = cfms(l[jj], sX[j0 + jj][(g + c < nrhs) ? g + c : 0], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < G; ++c)
      if (g + c < nrhs) X[(size_t)(g + c) * n + i] = acc[c];
  }
}

// One CTA of 512 threads per unit: L y = P b (unit lower, each panel's swaps
// applied just before its block), then U x = y, on the n x nrhs column-major
// block X.  The NB x NB triangles are solved by warps taking columns in turn (lane = row, values
// passed by shuffles); the rows below/above are updated by the whole CTA.
template <typename R, int NB>
__global__ void __launch_bounds__(512, 2) k_solve(const Unit* __restrict__ units, const char* fac_base, char* ws,
                                                int which, int nrhs, const int32_t* done) {
  using C = Cx<R>;
  static_assert(NB == 32, "one lane per row of the diagonal block");
  const Unit u = units[blockIdx.x];
  if (done && done[u.stat_off]) return;
  const int n = u.n;
  if (n == 0) return;  // an unused FP64 fallback slot
  const C* A = reinterpret_cast<const C*>(fac_base + u.fac_off);
  C* X = reinterpret_cast<C*>(ws + (which == RHS_X ? u.x_off : u.x32_off));
  const int32_t* piv = reinterpret_cast<const int32_t*>(fac_base + u.piv_off);
  __shared__ C sT[NB][NB + 1];
  __shared__ C sX[NB][33];
  __shared__ int sp[NB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x;
  // forward
  for (int k = 0; k < n; k += NB) {
    const int nbp = min(NB, n - k);
    for (int idx = tid; idx < NB * NB; idx += nthr) {
      const int i = idx % NB, j = idx / NB;
      sT[i][j] = (i < nbp && j < nbp) ? A[(size_t)(k + j) * n + k + i] : mk(R(0), R(0));
    }
    if (tid < NB) sp[tid] = tid < nbp ? piv[k + tid] : k + tid;
    __syncthreads();
    for (int col = warp; col < nrhs; col += nthr >> 5) {
      C x = lane < nbp ? X[(size_t)col * n + k + lane] : mk(R(0), R(0));
      x = panel_swaps(x, X + (size_t)col * n, sp, k, lane);
      for (int j = 0; j < nbp - 1; ++j) {
        const C xj = shfl2(x, j);
        if (lane > j) x = cfms(sT[lane][j], xj, x);
      }
      if (lane < nbp) {
        X[(size_t)col * n + k + lane] = x;
        sX[lane][col] = x;
      }
    }
    __syncthreads();
    update_rows<R, NB>(A, X, sX, n, k, nbp, k + nbp, n, nrhs, tid, nthr);
    __syncthreads();
  }
  // backward
  const int last = ((n - 1) / NB) * NB;
  for (int k = last; k >= 0; k -= NB) {
    const int nbp = min(NB, n - k);
    for (int idx = tid; idx < NB * NB; idx += nthr) {
      const int i = idx % NB, j = idx / NB;
      sT[i][j] = (i < nbp && j < nbp) ? A[(size_t)(k + j) * n + k + i] : mk(R(1), R(0));
    }
    __syncthreads();
    for (int col = warp; col < nrhs; col += nthr >> 5) {
      C x = lane < nbp ? X[(size_t)col * n + k + lane] : mk(R(0), R(0));
      for (int j = nbp - 1; j >= 0; --j) {
        if (lane == j) x = cmul(x, crcp(sT[j][j]));
        const C xj = shfl2(x, j);
        if (lane < j) x = cfms(sT[lane][j], xj, x);
      }
      if (lane < nbp) {
        X[(size_t)col * n + k + lane] = x;
        sX[lane][col] = x;
      }
    }
    __syncthreads();
    update_rows<R, NB>(A, X, sX, n, k, nbp, 0, k, nrhs, tid, nthr);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ complex64 solve
// The complex64 solve of the mixed form, specialised on the padded right-hand-side
// count NCOL (columns >= nrhs are zero and never stored).  The update of the rows
// below (forward) or above (backward) a solved block gives each thread one row
// and G = min(NCOL, 8) columns: per step j one coalesced 8-byte load of the
// factor, G/2 16-byte shared-memory loads of the solved block and 4 G FMAs.
constexpr int kSolveThreads = 256;  // complex64 solve CTA

template <int NCOL, int NT>
__device__ __forceinline__ void update_rows_c64(const float2* __restrict__ A, float2* X, const float2 (*sX)[NCOL],
                                                int n, int k, int nbp, int r0, int r1, int nrhs, int tid) {
  constexpr int G = NCOL < 8 ? NCOL : 8;
  constexpr int NG = NCOL / G;
  constexpr int NB = 32;
  const int rows = r1 - r0;
  if (rows <= 0) return;
  // work item = (row, group of G columns); a warp takes 32 consecutive rows of one
  // group and the NG groups of the same rows go to consecutive warps, so the
  // factor's 32-row segments are fetched once and reused from L1 by the others
  const int chunks = (rows + 31) / 32;
  for (int idx = tid; idx < chunks * 32 * NG; idx += NT) {
    const int gi = (idx >> 5) % NG;
    const int i = r0 + ((idx >> 5) / NG) * 32 + (idx & 31);
    if (i >= r1) continue;
    const int g = gi * G;
    // the factor entries of this thread's next item (read once from DRAM) are
    // requested into L2 now, by the warps of the first column group only (with
    // 32 columns the extra L2 traffic cost more than the latency it hid)
    if constexpr (NCOL <= 16) {
      const int nidx = idx + NT;
      const int ni = r0 + ((nidx >> 5) / NG) * 32 + (nidx & 31);
      if (gi == 0 && ni < r1 && (nidx >> 5) % NG == 0) {
        const float2* An = A + (size_t)k * n + ni;
#pragma unroll 4
        for (int j = 0; j < nbp; ++j) asm volatile("prefetch.global.L2 [%0];" ::"l"(An + (size_t)j * n));
      }
    }
    float2 acc[G];
#pragma unroll
    for (int c = 0; c < G; ++c) acc[c] = (g + c < nrhs) ? X[(size_t)(g + c) * n + i] : make_float2(0.f, 0.f);
    const float2* Ai = A + (size_t)k * n + i;
    if (nbp == NB) {
#pragma unroll 1
      for (int j0 = 0; j0 < NB; j0 += 8) {
        float2 l[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) l[jj] = Ai[(size_t)(j0 + jj) * n];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
#pragma unroll
          for (int c = 0; c < G; c += 2) {
            const float4 xx = *reinterpret_cast<const float4*>(&sX[j0 + jj][g + c]);
            acc[c] = cfms(l[jj], make_float2(xx.x, xx.y), acc[c]);
            acc[c + 1] = cfms(l[jj], make_float2(xx.z, xx.w), acc[c + 1]);
          }
        }
      }
    } else {
      for (int j = 0; j < nbp; ++j) {
        const float2 l = Ai[(size_t)j * n];
#pragma unroll
        for (int c = 0; c < G; c += 2) {
          const float4 xx = *reinterpret_cast<const float4*>(&sX[j][g + c]);
          acc[c] = cfms(l, make_float2(xx.x, xx.y), acc[c]);
          acc[c + 1] = cfms(l, make_float2(xx.z, xx.w), acc[c + 1]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < G; ++c)
      if (g + c < nrhs) X[(size_t)(g + c) * n + i] = acc[c];
  }
}

// Inverses of the 32 x 32 diagonal blocks of the complex64 factors, L_bb (unit
// lower) and U_bb (upper), stored after the double-float copy of M for the
// solves.  grid (ceil(n_max / 32), n_units), block 64: warp 0 inverts L_bb,
// warp 1 U_bb, lane j forming column j by substitution; a partial last block is
// padded with the identity.
__global__ void __launch_bounds__(64) k_diag_inv(const Unit* __restrict__ units, char* fac_base) {
  constexpr int NB = kDiagNB;
  const Unit u = units[blockIdx.y];
  const int n = u.n, k = blockIdx.x * NB;
  if (k >= n) return;
  const int nbp = min(NB, n - k);
  const float2* A = reinterpret_cast<const float2*>(fac_base + u.fac_off);
  float2* D = reinterpret_cast<float2*>(fac_base + u.m64_off + diag_inv_rel_off(n)) + (size_t)blockIdx.x * 2 * NB * NB;
  __shared__ float2 sB[NB][NB + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < NB * NB; idx += 64) {
    const int i = idx % NB, j = idx / NB;
    sB[i][j] = (i < nbp && j < nbp) ? A[(size_t)(k + j) * n + k + i] : make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  float2 y[NB];
  if (warp == 0) {  // L y = e_lane, L unit lower
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      float2 a = make_float2(i == lane ? 1.f : 0.f, 0.f);
#pragma unroll
      for (int m = 0; m < i; ++m) a = cfms(sB[i][m], y[m], a);
      y[i] = a;
    }
  } else {  // U y = e_lane, U upper
#pragma unroll
    for (int i = NB - 1; i >= 0; --i) {
      float2 a = make_float2(i == lane ? 1.f : 0.f, 0.f);
#pragma unroll
      for (int m = i + 1; m < NB; ++m) a = cfms(sB[i][m], y[m], a);
      y[i] = cmul(a, crcp(sB[i][i]));
    }
  }
  float2* out = D + (size_t)warp * NB * NB + (size_t)lane * NB;  // column lane
#pragma unroll
  for (int i = 0; i < NB; ++i) out[i] = y[i];
}

// After the complex64 factorization L's columns are as computed: each panel's
// rows in the order of that panel's step (LINPACK style).  k_lapack_rows applies
// to every 32-column block of L the interchanges of all later panels, which puts
// L in the row order of one permutation (P M = L U), and replaces the pivots by
// that permutation: row r of P b is row perm[r] of b.  The solves then permute
// their right-hand sides once (k_perm_rows) and substitute without interchanges,
// so a block step of the forward substitution is the same product for every row
// below it and can be spread over many CTAs.
// A CTA walks the blocks from the last to the first with the composed
// permutation of the later panels in shared memory (idx: new row r takes old row
// idx[r]; pos: the inverse), moving the rows of its group of blocks.  Prepending an interchange (a, c) to the sequence
// exchanges the values a and c in idx.  Only the rows with idx[r] != r move; a
// pass reads all moved entries of some columns into shared memory, then writes
// them.  Dynamic shared memory: lap_smem_bytes(n_max) (14 bytes per row: the
// complex64 n <= 16,600).
constexpr int kLapCols = 32;
constexpr int kLapMaxN = 65535;  // row indices held as 16-bit values
__host__ __device__ inline size_t lap_stage_elems(int n_max) { return (size_t)(n_max > 2048 ? n_max : 2048); }
inline size_t lap_smem_bytes(int n_max) { return lap_stage_elems(n_max) * 8 + (size_t)3 * n_max * 2; }

constexpr int kLapBlocks = 8;  // 32-column blocks of L per CTA of k_lapack_rows

// grid (ceil((blocks - 1) / kLapBlocks), n_units): CTA g moves the rows of blocks
// g kLapBlocks .. g kLapBlocks + kLapBlocks - 1, after building the composition of
// the later panels' interchanges itself (the prepends are cheap; the row moves of
// the blocks run in parallel over the CTAs).
__global__ void __launch_bounds__(256) k_lapack_rows(const Unit* __restrict__ units, const char* fac_base_c,
                                                     int n_max, int32_t* stat) {
  constexpr int NB = 32;
  char* fac_base = const_cast<char*>(fac_base_c);
  const Unit u = units[blockIdx.y];
  const int n = u.n;
  const int nb = (n + NB - 1) / NB;
  const int b_lo = blockIdx.x * kLapBlocks, b_hi = min(nb - 2, b_lo + kLapBlocks - 1);
  if (b_lo > b_hi) return;
  float2* A = reinterpret_cast<float2*>(fac_base + u.fac_off);
  const int32_t* piv = reinterpret_cast<const int32_t*>(fac_base + u.piv_off);
  extern __shared__ __align__(16) unsigned char lap_raw[];
  const int cap = (int)lap_stage_elems(n_max);
  float2* stage = reinterpret_cast<float2*>(lap_raw);
  unsigned short* idx = reinterpret_cast<unsigned short*>(stage + cap);
  unsigned short* pos = idx + n_max;
  unsigned short* list = pos + n_max;
  __shared__ int s_cnt;
  const int tid = threadIdx.x;
  for (int r = tid; r < n; r += blockDim.x) idx[r] = pos[r] = (unsigned short)r;
  __syncthreads();
  for (int b = nb - 2; b >= b_lo; --b) {
    // prepend panel b + 1's interchanges, its last one first
    if (tid == 0) {
      const int r0 = NB * (b + 1), r1 = min(n, r0 + NB);
      for (int r = r1 - 1; r >= r0; --r) {
        const int a = r, c = piv[r];
        if (a != c && dbg_in(c, r, n, &stat[u.stat_off])) {
          const int ra = pos[a], rc = pos[c];
          idx[ra] = (unsigned short)c;
          idx[rc] = (unsigned short)a;
          pos[a] = (unsigned short)rc;
          pos[c] = (unsigned short)ra;
        }
      }
      s_cnt = 0;
    }
    __syncthreads();
    if (b > b_hi) continue;
    for (int r = NB * (b + 1) + tid; r < n; r += blockDim.x)
      if (idx[r] != r) list[atomicAdd(&s_cnt, 1)] = (unsigned short)r;
    __syncthreads();
    const int m = s_cnt;
    if (m == 0) continue;
    const int cpp = max(1, min(kLapCols, cap / m));  // columns per pass
    for (int c0 = NB * b; c0 < NB * b + NB; c0 += cpp) {
      const int nc = min(cpp, NB * b + NB - c0);
      for (int x = tid; x < nc * m; x += blockDim.x) {
        const int c = c0 + x / m, i = x % m;
        stage[x] = A[(size_t)c * n + idx[list[i]]];
      }
      __syncthreads();
      for (int x = tid; x < nc * m; x += blockDim.x) {
        const int c = c0 + x / m, i = x % m;
        A[(size_t)c * n + list[i]] = stage[x];
      }
      __syncthreads();
    }
  }
}

// After k_lapack_rows (which reads the pivots): the pivots replaced by the full
// permutation, the interchanges of all panels applied in order to the identity.
// One CTA per unit; dynamic shared memory 2 n_max bytes.
__global__ void __launch_bounds__(256) k_lapack_perm(const Unit* __restrict__ units, char* fac_base, int32_t* stat) {
  const Unit u = units[blockIdx.x];
  const int n = u.n;
  int32_t* piv = reinterpret_cast<int32_t*>(fac_base + u.piv_off);
  extern __shared__ unsigned short perm_raw[];
  for (int r = threadIdx.x; r < n; r += blockDim.x) perm_raw[r] = (unsigned short)r;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int r = 0; r < n; ++r) {
      const int c = piv[r];
      if (c != r && dbg_in(c, r, n, &stat[u.stat_off])) {
        const unsigned short t = perm_raw[r];
        perm_raw[r] = perm_raw[c];
        perm_raw[c] = t;
      }
    }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) piv[r] = perm_raw[r];
}

// Right-hand-side columns permuted by the factorization's row permutation:
// row r of column c takes row perm[r].  grid (nrhs, n_units), block 256,
// dynamic shared memory n_max complex64 values.
__global__ void __launch_bounds__(256) k_perm_rows(const Unit* __restrict__ units, const char* fac_base, char* ws,
                                                   int nrhs, const int32_t* done) {
  const Unit u = units[blockIdx.y];
  if (done && done[u.stat_off]) return;
  const int c = blockIdx.x;
  if (c >= nrhs) return;
  const int n = u.n;
  const int32_t* perm = reinterpret_cast<const int32_t*>(fac_base + u.piv_off);
  float2* X = reinterpret_cast<float2*>(ws + u.x32_off) + (size_t)c * n;
  extern __shared__ float2 sv[];
  for (int r = threadIdx.x; r < n; r += blockDim.x) sv[r] = X[perm[r]];
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) X[r] = sv[r];
}

// One CTA of NT threads per unit and slice of NCOL right-hand-side columns
// (blockIdx.y; several CTAs resident per SM, so one chain's block phases overlap
// the others' row updates): L y = P b (unit lower, L in the row order of P, the
// right-hand sides permuted by k_perm_rows before), then U x = y, on the
// n x nrhs column-major block X.  Each 32-row block step multiplies its rows by
// the stored inverse of the diagonal block (all threads, no serial chain) and
// updates the rows below (above, going back) with the block's 32 columns of L (U).
template <int NCOL, int NT, int MINB = 1024 / NT>
__global__ void __launch_bounds__(NT, MINB) k_solve_c64(const Unit* __restrict__ units, const char* fac_base,
                                                     char* ws, int which, int nrhs, const int32_t* done) {
  static_assert(NCOL >= 2 && NCOL % 2 == 0 && NCOL <= 32, "padded column count");
  constexpr int NB = kDiagNB;
  const Unit u = units[blockIdx.x];
  if (done && done[u.stat_off]) return;
  const int n = u.n;
  // columns [NCOL y, NCOL y + NCOL) of the right-hand sides (slice y = blockIdx.y)
  const int c_off = blockIdx.y * NCOL;
  nrhs = min(NCOL, nrhs - c_off);
  if (nrhs <= 0) return;
  const float2* A = reinterpret_cast<const float2*>(fac_base + u.fac_off);
  const float2* D = reinterpret_cast<const float2*>(fac_base + u.m64_off + diag_inv_rel_off(n));
  float2* X = reinterpret_cast<float2*>(ws + (which == RHS_X ? u.x_off : u.x32_off)) + (size_t)c_off * n;
  __shared__ float2 sT[NB][NB + 1];                 // inverse of the diagonal block
  __shared__ __align__(16) float2 sX[NB][NCOL];     // the block's solved rows
  __shared__ float2 sIn[NB][NCOL + 1];              // the block's rows before the inverse
  const int tid = threadIdx.x;
  // y = T^-1 (block rows) for every (row, column) pair of the block
  auto apply_inverse = [&](int k, int nbp) {
#pragma unroll 1
    for (int idx = tid; idx < NB * NCOL; idx += NT) {
      const int i = idx % NB, c = idx / NB;
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < NB; j += 2) {
        a0 = cfma(sT[i][j], sIn[j][c], a0);
        a1 = cfma(sT[i][j + 1], sIn[j + 1][c], a1);
      }
      const float2 y = make_float2(a0.x + a1.x, a0.y + a1.y);
      sX[i][c] = y;
      if (i < nbp && c < nrhs) X[(size_t)c * n + k + i] = y;
    }
  };
  // forward (the right-hand sides already permuted by k_perm_rows)
  for (int k = 0; k < n; k += NB) {
    const int nbp = min(NB, n - k);
    const float2* Dk = D + (size_t)(k / NB) * 2 * NB * NB;  // L^-1 block
    for (int idx = tid; idx < NB * NB; idx += NT) sT[idx % NB][idx / NB] = Dk[idx];
    for (int idx = tid; idx < NB * NCOL; idx += NT) {
      const int i = idx % NB, c = idx / NB;
      sIn[i][c] = (c < nrhs && i < nbp) ? X[(size_t)c * n + k + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    apply_inverse(k, nbp);
    __syncthreads();
    update_rows_c64<NCOL, NT>(A, X, sX, n, k, nbp, k + nbp, n, nrhs, tid);
    __syncthreads();
  }
  // backward
  const int last = ((n - 1) / NB) * NB;
  for (int k = last; k >= 0; k -= NB) {
    const int nbp = min(NB, n - k);
    const float2* Dk = D + (size_t)(k / NB) * 2 * NB * NB + NB * NB;  // U^-1 block
    for (int idx = tid; idx < NB * NB; idx += NT) sT[idx % NB][idx / NB] = Dk[idx];
    for (int idx = tid; idx < NB * NCOL; idx += NT) {
      const int i = idx % NB, c = idx / NB;
      sIn[i][c] = (c < nrhs && i < nbp) ? X[(size_t)c * n + k + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    apply_inverse(k, nbp);
    __syncthreads();
    update_rows_c64<NCOL, NT>(A, X, sX, n, k, nbp, 0, k, nrhs, tid);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ block-step solves
// The complex64 substitutions as one launch per 32-row block step over all units
// of a chunk, each step's row update spread over row tiles (many CTAs per unit):
// the chain of dependent block steps moves from inside one CTA to the launch
// sequence.  NCOL = right-hand-side columns (8, 16 or 32, padded); a tile has
// step_rows<NCOL>() rows and 256 threads, a thread one row and step_cols<NCOL>()
// columns.  Each thread requests its row's 32 factor entries and its X entries
// before the block's solved rows arrive in shared memory, so one memory latency
// covers the whole update.  The tile that holds the next block finalizes it
// after its own update: y = T^{-1} x with the stored inverse of the diagonal block.
template <int NCOL> __host__ __device__ constexpr int step_cols() { return NCOL < 16 ? NCOL : 16; }
template <int NCOL> __host__ __device__ constexpr int step_rows() { return 256 * step_cols<NCOL>() / NCOL; }

// Registers of one thread of a step update: X rows [row0, row0 + rows), its row
// r = row0 + threadIdx.x % TR and CH columns from g; the factor entries
// F[r, c0 .. c0 + nbp) (column-major, ld n; zero beyond nbp).
template <int NCOL>
struct StepRegs {
  static constexpr int CH = step_cols<NCOL>();
  float2 l[32], acc[CH];
  int r, g;
  bool live;
  __device__ __forceinline__ void load(const float2* __restrict__ F, const float2* X, int n, int c0, int nbp,
                                       int row0, int rows, int nrhs) {
    constexpr int TR = step_rows<NCOL>();
    r = row0 + threadIdx.x % TR;
    g = (threadIdx.x / TR) * CH;
    live = threadIdx.x % TR < rows;
    if (!live) return;
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = (g + c < nrhs) ? X[(size_t)(g + c) * n + r] : make_float2(0.f, 0.f);
    const float2* Fr = F + (size_t)c0 * n + r;
#pragma unroll
    for (int j = 0; j < 32; ++j) l[j] = j < nbp ? Fr[(size_t)j * n] : make_float2(0.f, 0.f);
  }
  // X[r, g ..] = acc - l y (y = sY, 32 rows, zero-padded)
  __device__ __forceinline__ void finish(float2* X, const float2 (*sY)[NCOL], int n, int nrhs) {
    if (!live) return;
#pragma unroll
    for (int j = 0; j < 32; ++j)
#pragma unroll
      for (int c = 0; c < CH; c += 2) {
        const float4 yy = *reinterpret_cast<const float4*>(&sY[j][g + c]);
        acc[c] = cfms(l[j], make_float2(yy.x, yy.y), acc[c]);
        acc[c + 1] = cfms(l[j], make_float2(yy.z, yy.w), acc[c + 1]);
      }
#pragma unroll
    for (int c = 0; c < CH; ++c)
      if (g + c < nrhs) X[(size_t)(g + c) * n + r] = acc[c];
  }
};

// Block k (nbp rows) of X := T^{-1} X[block k], T^{-1} = Dk (32 x 32 column-major,
// identity-padded).  Every thread of the CTA calls it; sIn / sT are scratch.
template <int NCOL>
__device__ __forceinline__ void step_finalize(const float2* __restrict__ Dk, float2* X, float2 (*sT)[33],
                                              float2 (*sIn)[NCOL + 1], int n, int k, int nbp, int nrhs) {
  constexpr int NB = 32;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) sT[idx % NB][idx / NB] = Dk[idx];
  for (int idx = tid; idx < NB * NCOL; idx += blockDim.x) {
    const int i = idx % NB, c = idx / NB;
    sIn[i][c] = (c < nrhs && i < nbp) ? X[(size_t)c * n + k + i] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int idx = tid; idx < NB * NCOL; idx += blockDim.x) {
    const int i = idx % NB, c = idx / NB;
    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < NB; j += 2) {
      a0 = cfma(sT[i][j], sIn[j][c], a0);
      a1 = cfma(sT[i][j + 1], sIn[j + 1][c], a1);
    }
    if (i < nbp && c < nrhs) X[(size_t)c * n + k + i] = make_float2(a0.x + a1.x, a0.y + a1.y);
  }
}

// Forward step s (L y = P b, right-hand sides permuted before): with block s
// final, the rows below it take X[r] -= L[r, block s] y_s (tile t: rows
// 32 (s + 1) + TR t ...); then tile 0, whose first 32 rows are block s + 1,
// finalizes that block with L_{s+1}^{-1}.  s = -1 only finalizes block 0.
// grid (row tiles, n_units), block 256.
template <int NCOL>
__global__ void __launch_bounds__(256, 2) k_fwd_step(const Unit* __restrict__ units, const char* fac_base, char* ws,
                                                  int nrhs, const int32_t* done, int s) {
  constexpr int NB = 32, TR = step_rows<NCOL>();
  const Unit u = units[blockIdx.y];
  if (done && done[u.stat_off]) return;
  const int n = u.n;
  const int nb = (n + NB - 1) / NB;
  if (s + 1 >= nb) return;
  const int r_begin = NB * (s + 1);
  const int row0 = r_begin + blockIdx.x * TR;
  if (row0 >= n) return;
  const float2* A = reinterpret_cast<const float2*>(fac_base + u.fac_off);
  float2* X = reinterpret_cast<float2*>(ws + u.x32_off);
  __shared__ __align__(16) float2 sY[NB][NCOL];
  __shared__ float2 sT[NB][NB + 1];
  __shared__ float2 sIn[NB][NCOL + 1];
  if (s >= 0) {
    StepRegs<NCOL> t;
    t.load(A, X, n, NB * s, NB, row0, min(TR, n - row0), nrhs);
    for (int idx = threadIdx.x; idx < NB * NCOL; idx += blockDim.x) {
      const int i = idx % NB, c = idx / NB;
      sY[i][c] = c < nrhs ? X[(size_t)c * n + NB * s + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    t.finish(X, sY, n, nrhs);
  }
  if (blockIdx.x == 0) {
    __syncthreads();  // this tile's rows of block s + 1 are updated (no other tile writes them)
    const float2* D = reinterpret_cast<const float2*>(fac_base + u.m64_off + diag_inv_rel_off(n));
    step_finalize<NCOL>(D + (size_t)(s + 1) * 2 * NB * NB, X, sT, sIn, n, r_begin, min(NB, n - r_begin), nrhs);
  }
}

// Backward step s (U x = y): with block s final, rows [0, 32 s) take
// X[r] -= U[r, block s] x_s (tile t: rows TR t ...); the tile holding block s - 1
// then finalizes it with U_{s-1}^{-1}.  For a unit with s = its block count the
// launch only finalizes its last block.  grid (row tiles, n_units), block 256.
template <int NCOL>
__global__ void __launch_bounds__(256, 2) k_bwd_step(const Unit* __restrict__ units, const char* fac_base, char* ws,
                                                  int nrhs, const int32_t* done, int s) {
  constexpr int NB = 32, TR = step_rows<NCOL>();
  const Unit u = units[blockIdx.y];
  if (done && done[u.stat_off]) return;
  const int n = u.n;
  const int nb = (n + NB - 1) / NB;
  if (s > nb || s < 1) return;
  const int fin_tile = (NB * (s - 1)) / TR;  // the tile holding block s - 1
  const float2* A = reinterpret_cast<const float2*>(fac_base + u.fac_off);
  float2* X = reinterpret_cast<float2*>(ws + u.x32_off);
  __shared__ __align__(16) float2 sY[NB][NCOL];
  __shared__ float2 sT[NB][NB + 1];
  __shared__ float2 sIn[NB][NCOL + 1];
  if (s < nb) {
    const int row0 = TR * blockIdx.x;
    if (row0 >= NB * s) return;
    const int nbp = min(NB, n - NB * s);
    StepRegs<NCOL> t;
    t.load(A, X, n, NB * s, nbp, row0, min(TR, NB * s - row0), nrhs);
    for (int idx = threadIdx.x; idx < NB * NCOL; idx += blockDim.x) {
      const int i = idx % NB, c = idx / NB;
      sY[i][c] = (c < nrhs && i < nbp) ? X[(size_t)c * n + NB * s + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    t.finish(X, sY, n, nrhs);
  }
  if (blockIdx.x == fin_tile) {
    __syncthreads();
    const float2* D = reinterpret_cast<const float2*>(fac_base + u.m64_off + diag_inv_rel_off(n));
    const int k = NB * (s - 1);
    step_finalize<NCOL>(D + (size_t)(s - 1) * 2 * NB * NB + NB * NB, X, sT, sIn, n, k, min(NB, n - k), nrhs);
  }
}

// The block finalize of the tensor-core step solves: y_b = T^{-1} X[block b] with
// the stored inverse of the diagonal block (L after forward step s: b = s + 1;
// U after backward step s: b = s - 1; s = -1: the first block forward, the
// unit's last block backward).  grid (n_units), block 256.
__global__ void __launch_bounds__(256) k_step_final(const Unit* __restrict__ units, const char* fac_base, char* ws,
                                                    int nrhs, const int32_t* done, int s, int forward) {
  constexpr int NB = 32;
  const Unit u = units[blockIdx.x];
  if (done && done[u.stat_off]) return;
  const int n = u.n, nb = (n + NB - 1) / NB;
  int b;
  if (forward) {
    b = s + 1;
    if (b > nb - 1) return;
  } else if (s < 0) {
    b = nb - 1;
  } else {
    if (s >= nb || s < 1) return;
    b = s - 1;
  }
  __shared__ float2 sT[NB][NB + 1];
  __shared__ float2 sIn[NB][NB + 1];
  float2* X = reinterpret_cast<float2*>(ws + u.x32_off);
  const float2* D = reinterpret_cast<const float2*>(fac_base + u.m64_off + diag_inv_rel_off(n));
  step_finalize<NB>(D + (size_t)b * 2 * NB * NB + (forward ? 0 : NB * NB), X, sT, sIn, n, NB * b,
                    min(NB, n - NB * b), nrhs);
}

// ------------------------------------------------------------------ wrappers
template <typename R>
int lu_factor_chunk(const Unit* d_units, int n_units, int n_max, char* fac_base, int32_t* stat,
                    cudaStream_t st) {
  constexpr int NB = LuCfg<R>::NB;
  // panels up to kPanelSmemBytes stay in shared memory; taller ones use k_panel
  constexpr int kPanelSmemBytes = 224 * 1024;
  const int max_rows = kPanelSmemBytes / (NB * (int)sizeof(Cx<R>));
  static bool attr_set = false;
  if (!attr_set) {
    LSMS_CUDA_TRY(cudaFuncSetAttribute(k_panel_smem<R, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kPanelSmemBytes));
    if (sizeof(Cx<R>) == 8)
      LSMS_CUDA_TRY(cudaFuncSetAttribute(k_swap_trsm<R, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSwapTileBytes));
    attr_set = true;
  }
  for (int k = 0; k < n_max; k += NB) {
    const int m_max = n_max - k;
    if (m_max > max_rows) {
      // taller panels on one CTA per unit, or, from 2048 rows (few units of large LIZ
      // matrices: the single CTA would leave most SMs idle), on a cluster of CTAs per unit
      if (m_max > 2048 && (m_max + kPanelCluster - 1) / kPanelCluster <= kClusterRows * kClusterThreads)
        LSMS_LAUNCH((k_panel_cluster<R, NB>), dim3(kPanelCluster, n_units), dim3(kClusterThreads), 0, st, d_units,
                    fac_base, k, stat, max_rows);
      else
        LSMS_LAUNCH((k_panel<R, NB>), dim3(n_units), dim3(1024), 0, st, d_units, fac_base, k, stat, max_rows);
    }
    const int rows_smem = std::min(m_max, max_rows);
    // one thread per row: short panels launch fewer threads, so more CTAs fit on an SM
    const int threads = std::min(kPanelThreads, (rows_smem + 31) / 32 * 32);
    LSMS_LAUNCH((k_panel_smem<R, NB>), dim3(n_units), dim3(threads), (size_t)rows_smem * NB * sizeof(Cx<R>), st,
                d_units, fac_base, k, stat, max_rows);
    const int trail = n_max - k - NB;
    if (trail <= 0) continue;
    // one warp per column right of the panel
    LSMS_LAUNCH((k_swap_trsm<R, NB>), dim3((trail + kSwapCols - 1) / kSwapCols, n_units), dim3(256),
                sizeof(Cx<R>) == 8 ? kSwapTileBytes : 0, st, d_units,
                fac_base, k, stat);
    if constexpr (std::is_same<R, float>::value) {
      // complex64: the trailing update runs on the tensor cores (3xTF32, tc_gemm.cu)
      const int rc = gemm_tc_chunk(d_units, n_units, n_max, k, fac_base, stat, st);
      if (rc) return rc;
    } else {
      const int tiles = (trail + 63) / 64;
      LSMS_LAUNCH((k_gemm<R, NB>), dim3(tiles * tiles, n_units), dim3(256), 0, st, d_units, fac_base, k, tiles);
    }
  }
  // complex64: inverses of the diagonal blocks for the solves, L in the row order
  // of the final permutation
  if constexpr (std::is_same<R, float>::value) {
    LSMS_LAUNCH(k_diag_inv, dim3((n_max + kDiagNB - 1) / kDiagNB, n_units), dim3(64), 0, st, d_units, fac_base);
    const size_t lap = lap_smem_bytes(n_max);
    if (lap > 227 * 1024 || n_max > kLapMaxN)
      return fail(LSMS_ERR_ARG, "n = %d too large for the complex64 form (at most 16,600)", n_max);
    static size_t lap_attr = 48 * 1024;
    if (lap > lap_attr) {
      LSMS_CUDA_TRY(cudaFuncSetAttribute(k_lapack_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lap));
      lap_attr = lap;
    }
    const int nb_max = (n_max + 31) / 32;
    if (nb_max > 1)
      LSMS_LAUNCH(k_lapack_rows, dim3((nb_max - 1 + kLapBlocks - 1) / kLapBlocks, n_units), dim3(256), lap, st,
                  d_units, fac_base, n_max, stat);
    LSMS_LAUNCH(k_lapack_perm, dim3(n_units), dim3(256), (size_t)n_max * 2, st, d_units, fac_base, stat);
  }
  return LSMS_OK;
}

template <int NCOL>
static int solve_steps(const Unit* d_units, int n_units, int n_max, const char* fac_base, char* ws, int nrhs,
                       const int32_t* done, cudaStream_t st) {
  constexpr int NB = 32, TR = step_rows<NCOL>();
  const int nb = (n_max + NB - 1) / NB;
  for (int s = -1; s + 1 < nb; ++s) {
    const int rows = n_max - NB * (s + 1);
    const dim3 g(s < 0 ? 1 : (rows + TR - 1) / TR, n_units);
    LSMS_LAUNCH(k_fwd_step<NCOL>, g, dim3(256), 0, st, d_units, fac_base, ws, nrhs, done, s);
  }
  for (int s = nb; s >= 1; --s) {
    const dim3 g((NB * s + TR - 1) / TR, n_units);
    LSMS_LAUNCH(k_bwd_step<NCOL>, g, dim3(256), 0, st, d_units, fac_base, ws, nrhs, done, s);
  }
  return LSMS_OK;
}

// The block steps with the row updates on the tensor cores (k_step_tc, whose
// tile holding the next block finalizes it); k_step_final takes the first block
// of each direction.
static int solve_steps_tc(const Unit* d_units, int n_units, int n_max, const char* fac_base, char* ws, int nrhs,
                          const int32_t* done, int32_t* stat, cudaStream_t st) {
  constexpr int NB = 32;
  const int nb = (n_max + NB - 1) / NB;
  int rc;
  LSMS_LAUNCH(k_step_final, dim3(n_units), dim3(256), 0, st, d_units, fac_base, ws, nrhs, done, -1, 1);
  for (int s = 0; s + 1 < nb; ++s)
    if ((rc = step_tc_chunk(d_units, n_units, n_max, fac_base, ws, nrhs, done, stat, s, true, st))) return rc;
  LSMS_LAUNCH(k_step_final, dim3(n_units), dim3(256), 0, st, d_units, fac_base, ws, nrhs, done, -1, 0);
  for (int s = nb - 1; s >= 1; --s)
    if ((rc = step_tc_chunk(d_units, n_units, n_max, fac_base, ws, nrhs, done, stat, s, false, st))) return rc;
  return LSMS_OK;
}

template <typename R>
int lu_solve_chunk(const Unit* d_units, int n_units, int n_max, const char* fac_base, char* ws, int which_rhs,
                   int nrhs, const int32_t* done, int32_t* stat, cudaStream_t st) {
  if (nrhs < 1 || nrhs > 32) return fail(LSMS_ERR_ARG, "internal: nrhs %d out of range", nrhs);
  constexpr int NB = LuCfg<R>::NB;
  if constexpr (std::is_same<R, float>::value) {
    if (which_rhs != RHS_X32) return fail(LSMS_ERR_ARG, "internal: complex64 solves work on the X32 field");
    // the right-hand sides in the row order of the factors' permutation
    const size_t pb = (size_t)n_max * sizeof(float2);
    static size_t perm_attr = 48 * 1024;
    if (pb > perm_attr) {
      if (pb > 227 * 1024) return fail(LSMS_ERR_ARG, "internal: n = %d too large for the permutation", n_max);
      LSMS_CUDA_TRY(cudaFuncSetAttribute(k_perm_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pb));
      perm_attr = pb;
    }
    LSMS_LAUNCH(k_perm_rows, dim3(nrhs, n_units), dim3(256), pb, st, d_units, fac_base, ws, nrhs, done);
    // option "solve_steps": 1 = one CTA chain per unit and column slice; 2 = block-step launches
    // (row updates on the FP32 pipes); 3 = block-step launches with the row updates on the tensor
    // cores; 0 (default) = block steps when the chains could not fill the GPU (fewer than two per
    // SM: few units of large LIZ matrices), on the tensor cores from 9 columns, else chains
    int steps = opt_solve_steps();
    if (steps == 0) {
      static int sms = 0;
      if (!sms) {
        int dev = 0;
        LSMS_CUDA_TRY(cudaGetDevice(&dev));
        LSMS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      }
      const int slices = nrhs <= 16 ? 1 : 2;
      steps = (long long)n_units * slices < 2LL * sms ? (nrhs > 8 ? 3 : 2) : 1;
    }
    if (steps == 3) return solve_steps_tc(d_units, n_units, n_max, fac_base, ws, nrhs, done, stat, st);
    if (steps == 2) {
      if (nrhs <= 8) return solve_steps<8>(d_units, n_units, n_max, fac_base, ws, nrhs, done, st);
      if (nrhs <= 16) return solve_steps<16>(d_units, n_units, n_max, fac_base, ws, nrhs, done, st);
      return solve_steps<32>(d_units, n_units, n_max, fac_base, ws, nrhs, done, st);
    }
    // more than 8 columns: column slices per CTA (option "solve_cols"; default 8
    // for up to 16 columns, 16 above), each slice a CTA with its own chain of
    // block steps; wider slices read the factors fewer times, narrower ones give
    // more concurrent chains
    const dim3 g1(n_units), b256(kSolveThreads);
    if (nrhs <= 2) LSMS_LAUNCH((k_solve_c64<2, kSolveThreads>), g1, b256, 0, st, d_units, fac_base, ws, which_rhs, nrhs, done);
    else if (nrhs <= 4) LSMS_LAUNCH((k_solve_c64<4, kSolveThreads>), g1, b256, 0, st, d_units, fac_base, ws, which_rhs, nrhs, done);
    else if (nrhs <= 8) LSMS_LAUNCH((k_solve_c64<8, kSolveThreads>), g1, b256, 0, st, d_units, fac_base, ws, which_rhs, nrhs, done);
    else {
      // option "solve_regs": 0 = 8 CTAs of 128 threads per SM (64 registers), 1 = 4 (128 registers),
      // 2 = 6 (85 registers)
      int sl = opt_solve_cols();
      if (sl <= 0) sl = nrhs <= 16 ? 8 : 16;
      if (sl == 32 && nrhs <= 16) sl = 16;  // one slice holds every column
      const int regs = opt_solve_regs();
      const dim3 gs(n_units, (nrhs + sl - 1) / sl);
#define LSMS_SOLVE(NCOL, NT, MINB) \
  LSMS_LAUNCH((k_solve_c64<NCOL, NT, MINB>), gs, dim3(NT), 0, st, d_units, fac_base, ws, which_rhs, nrhs, done)
      if (sl == 8) {
        if (regs == 2) LSMS_SOLVE(8, 128, 6);
        else if (regs) LSMS_SOLVE(8, 128, 4);
        else LSMS_SOLVE(8, 128, 8);
      } else if (sl == 16) {
        if (regs == 2) LSMS_SOLVE(16, 128, 6);
        else if (regs) LSMS_SOLVE(16, 128, 4);
        else LSMS_SOLVE(16, 128, 8);
      } else {
        LSMS_SOLVE(32, 256, 2);
      }
#undef LSMS_SOLVE
    }
  } else {
    LSMS_LAUNCH((k_solve<R, NB>), dim3(n_units), dim3(512), 0, st, d_units, fac_base, ws, which_rhs, nrhs, done);
  }
  return LSMS_OK;
}

template int lu_factor_chunk<double>(const Unit*, int, int, char*, int32_t*, cudaStream_t);
template int lu_factor_chunk<float>(const Unit*, int, int, char*, int32_t*, cudaStream_t);
template int lu_solve_chunk<double>(const Unit*, int, int, const char*, char*, int, int, const int32_t*, int32_t*,
                                    cudaStream_t);
template int lu_solve_chunk<float>(const Unit*, int, int, const char*, char*, int, int, const int32_t*, int32_t*,
                                   cudaStream_t);

}  // namespace lsms
