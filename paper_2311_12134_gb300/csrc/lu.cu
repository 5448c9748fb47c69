// Batched blocked LU with partial pivoting and the block solves for the tau
// column blocks.
//
// Eq. (tau-inverse) needs [T^{-1} - g]^{-1}; for each (atom, energy) unit the
// LIZ matrix M (n = K S, column-major, ld = n) is factored P M = L U in place.
// Pivoting: the row with the largest |Re| + |Im| in the column, the lowest row
// on ties.  Right-looking, panel width NB:
//   k_panel      factor the n-k x NB panel (pivot search by warp shuffles),
//   k_swap_trsm  apply the panel's row swaps to every other column (left ones
//                too, so L ends up in the final row order) and form
//                U12 = L11^{-1} A12 (one warp per column),
//   k_gemm       A22 -= L21 U12: register-tiled complex GEMM on the FP64 pipe
//                (FP64 form); the complex64 form uses k_gemm_tc (tc_gemm.cu),
//                the same update on the tensor cores,
//   k_perm       the permutation P as perm[i] (original row at position i) and
//                its inverse iperm.
// Units of a chunk are sorted by n (largest first); each launch covers every
// unit and units already finished return at once.  k_solve then runs plain
// forward/backward substitution on right-hand sides already permuted by P.
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace lsms {

template <typename R> struct LuCfg { static constexpr int NB = 32; };

__device__ __forceinline__ double2 shfl2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// ------------------------------------------------------------------ panel
template <typename R, int NB>
__global__ void __launch_bounds__(256) k_panel(const Unit* __restrict__ units, char* fac_base, int k,
                                               int32_t* stat, int max_rows) {
  using C = Cx<R>;
  const Unit u = units[blockIdx.x];
  const int n = u.n;
  if (k >= n || n - k <= max_rows) return;  // k_panel_smem factors those
  C* A = reinterpret_cast<C*>(fac_base + u.fac_off);
  int32_t* piv = reinterpret_cast<int32_t*>(fac_base + u.piv_off);
  const int nbp = min(NB, n - k);
  __shared__ R s_val[8];
  __shared__ int s_idx[8];
  __shared__ C s_row[NB];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  int flags = 0;
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
}

// Panel factorization held in shared memory: the m = n - k rows x NB columns of
// the panel are read once, factored column by column in shared memory (pivot
// search by warp shuffles), and written back once.  Units whose panel does not
// fit (m > max_rows) are left to k_panel, which works in global memory.
template <typename R, int NB>
__global__ void __launch_bounds__(512) k_panel_smem(const Unit* __restrict__ units, char* fac_base, int k,
                                                    int32_t* stat, int max_rows) {
  using C = Cx<R>;
  const Unit u = units[blockIdx.x];
  const int n = u.n;
  if (k >= n) return;
  const int m = n - k;
  if (m > max_rows) return;
  extern __shared__ __align__(16) unsigned char panel_raw[];
  C* sP = reinterpret_cast<C*>(panel_raw);  // [NB][m], column-major
  C* A = reinterpret_cast<C*>(fac_base + u.fac_off);
  int32_t* piv = reinterpret_cast<int32_t*>(fac_base + u.piv_off);
  const int nbp = min(NB, m);
  __shared__ R s_val[16];
  __shared__ int s_idx[16];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x, nwarps = nthr >> 5;
  for (int c = 0; c < nbp; ++c)
    for (int r = tid; r < m; r += nthr) sP[c * m + r] = A[(size_t)(k + c) * n + k + r];
  __syncthreads();
  int flags = 0;
  for (int j = 0; j < nbp; ++j) {
    C* Pj = sP + j * m;
    R best = R(-1);
    int bidx = m;
    for (int i = j + tid; i < m; i += nthr) {
      const R v = cabs1(Pj[i]);
      if (v > best) { best = v; bidx = i; }  // strict: lowest row kept; NaN never wins
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
      bidx = lane < nwarps ? s_idx[lane] : m;
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        const R ov = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
        if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
      }
      if (lane == 0) {
        const int p = (bidx < m) ? bidx : j;
        s_piv = p;
        piv[k + j] = k + p;
      }
    }
    __syncthreads();
    const int p = s_piv;
    if (p != j && tid < nbp) {
      C* col = sP + tid * m;
      const C t = col[j];
      col[j] = col[p];
      col[p] = t;
    }
    __syncthreads();
    const C pv = Pj[j];
    const bool zero = (pv.x == R(0) && pv.y == R(0));
    if (zero) flags |= LSMS_UNIT_ZERO_PIVOT;
    if (!finite2(pv)) flags |= LSMS_UNIT_NONFINITE;
    const C r = zero ? mk(R(0), R(0)) : crcp(pv);
    for (int i = j + 1 + tid; i < m; i += nthr) {
      const C l = cmul(Pj[i], r);
      if (!zero) Pj[i] = l;
      for (int c = j + 1; c < nbp; ++c) sP[c * m + i] = cfms(l, sP[c * m + j], sP[c * m + i]);
    }
    __syncthreads();
  }
  for (int c = 0; c < nbp; ++c)
    for (int r = tid; r < m; r += nthr) A[(size_t)(k + c) * n + k + r] = sP[c * m + r];
  if (tid == 0 && flags) atomicOr(&stat[u.stat_off], flags);
}

// ------------------------------------------------------------------ swap + trsm
// One warp per column outside the panel; lane i holds rows k+i (+32 r).
// Columns left of the panel only take the row swaps; columns to its right also
// get U12 = L11^{-1} A12.
constexpr int kSwapCols = 64;  // columns per CTA of k_swap_trsm (8 warps x 8)

template <typename R, int NB>
__global__ void __launch_bounds__(256) k_swap_trsm(const Unit* __restrict__ units, char* fac_base, int k) {
  using C = Cx<R>;
  constexpr int RPL = NB / 32;
  const Unit u = units[blockIdx.y];
  const int n = u.n;
  if (k >= n) return;
  const int nbp = min(NB, n - k);
  const int v0 = blockIdx.x * kSwapCols;           // virtual columns: [0, k) left, then right
  const int n_virtual = n - nbp;
  if (v0 >= n_virtual) return;
  C* A = reinterpret_cast<C*>(fac_base + u.fac_off);
  const int32_t* piv = reinterpret_cast<const int32_t*>(fac_base + u.piv_off);
  __shared__ C sL[NB][NB + 1];
  __shared__ int sp[NB];
  const bool any_right = (k + NB < n) && (v0 + kSwapCols > k);
  if (any_right) {
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
      const int i = idx % NB, j = idx / NB;
      sL[i][j] = A[(size_t)(k + j) * n + k + i];
    }
  }
  for (int j = threadIdx.x; j < NB; j += blockDim.x) sp[j] = j < nbp ? piv[k + j] : k + j;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int v = v0 + warp; v < min(v0 + kSwapCols, n_virtual); v += blockDim.x >> 5) {
  int c;
  bool right;
  if (v < k) {
    c = v;
    right = false;
  } else {
    c = v - k + k + NB;
    right = true;
  }
  C* Ac = A + (size_t)c * n;
  C x[RPL];
#pragma unroll
  for (int r = 0; r < RPL; ++r) {
    const int i = lane + 32 * r;
    x[r] = i < nbp ? Ac[k + i] : mk(R(0), R(0));
  }
  // Rows below the panel that the swaps touch: when all of them are distinct
  // (the usual case) each is read once up front and written once at the end;
  // the swap sequence then runs in registers.  Repeated targets take the
  // sequential path through memory.
  bool fast = false;
  C y = mk(R(0), R(0));
  int pj = k + lane;
  if (RPL == 1) {
    pj = sp[lane];
    const bool outj = pj >= k + NB;
    const unsigned same = __match_any_sync(0xffffffffu, outj ? pj : -1 - lane);
    fast = !__any_sync(0xffffffffu, outj && __popc(same) > 1);
    if (fast && outj) y = Ac[pj];
  }
  if (fast) {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int p = sp[j];
      if (p == k + j) continue;
      if (p < k + NB) {
        const int b = p - k;
        const C va = shfl2(x[0], j);
        const C vb = shfl2(x[0], b);
        if (lane == j) x[0] = vb;
        if (lane == b) x[0] = va;
      } else if (lane == j) {
        const C t = y;
        y = x[0];
        x[0] = t;
      }
    }
    if (pj >= k + NB) Ac[pj] = y;
  } else {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int p = sp[j];
      if (p == k + j) continue;
      if (p < k + NB) {
        const int b = p - k;
        const C va = shfl2(x[j / 32], j % 32);
        C vb = x[0];
#pragma unroll
        for (int r = 0; r < RPL; ++r)
          if (b / 32 == r) vb = shfl2(x[r], b % 32);
        if (lane == j % 32) x[j / 32] = vb;
#pragma unroll
        for (int r = 0; r < RPL; ++r)
          if (b / 32 == r && lane == b % 32) x[r] = va;
      } else {
        if (lane == j % 32) {
          const C t = Ac[p];
          Ac[p] = x[j / 32];
          x[j / 32] = t;
        }
        __syncwarp();
      }
    }
  }
  if (right) {
#pragma unroll
    for (int j = 0; j < NB - 1; ++j) {
      const C xj = shfl2(x[j / 32], j % 32);
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        if (i > j) x[r] = cfms(sL[i][j], xj, x[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RPL; ++r) {
    const int i = lane + 32 * r;
    if (i < nbp) Ac[k + i] = x[r];
  }
  }  // column loop
}

// perm[i] = original row now at position i, iperm[perm[i]] = i.  One thread per unit.
__global__ void k_perm(const Unit* __restrict__ units, int n_units, char* fac_base) {
  const int ui = blockIdx.x * blockDim.x + threadIdx.x;
  if (ui >= n_units) return;
  const Unit u = units[ui];
  const int n = u.n;
  int32_t* piv = reinterpret_cast<int32_t*>(fac_base + u.piv_off);
  int32_t* perm = piv + n;
  int32_t* iperm = piv + 2 * n;
  for (int i = 0; i < n; ++i) perm[i] = i;
  for (int i = 0; i < n; ++i) {
    const int p = piv[i];
    const int t = perm[i];
    perm[i] = perm[p];
    perm[p] = t;
  }
  for (int i = 0; i < n; ++i) iperm[perm[i]] = i;
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

// One CTA of 512 threads per unit: L y = b (unit lower), then U x = y,
// for the n x nrhs column-major block X whose rows are already permuted by P.
// The NB x NB triangles are solved by warps taking columns in turn (lane = row, values
// passed by shuffles); the rows below/above are updated by the whole CTA.
template <typename R, int NB>
__global__ void __launch_bounds__(512, 2) k_solve(const Unit* __restrict__ units, const char* fac_base, char* ws,
                                                int which, int nrhs, const int32_t* done) {
  using C = Cx<R>;
  static_assert(NB == 32, "one lane per row of the diagonal block");
  const Unit u = units[blockIdx.x];
  if (done && done[u.stat_off]) return;
  const int n = u.n;
  const C* A = reinterpret_cast<const C*>(fac_base + u.fac_off);
  C* X = reinterpret_cast<C*>(ws + (which == RHS_X ? u.x_off : u.x32_off));
  __shared__ C sT[NB][NB + 1];
  __shared__ C sX[NB][33];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x;
  // forward
  for (int k = 0; k < n; k += NB) {
    const int nbp = min(NB, n - k);
    for (int idx = tid; idx < NB * NB; idx += nthr) {
      const int i = idx % NB, j = idx / NB;
      sT[i][j] = (i < nbp && j < nbp) ? A[(size_t)(k + j) * n + k + i] : mk(R(0), R(0));
    }
    __syncthreads();
    for (int col = warp; col < nrhs; col += nthr >> 5) {
      C x = lane < nbp ? X[(size_t)col * n + k + lane] : mk(R(0), R(0));
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

// ------------------------------------------------------------------ wrappers
template <typename R>
int lu_factor_chunk(const Unit* d_units, int n_units, int n_max, char* fac_base, int32_t* stat,
                    cudaStream_t st) {
  constexpr int NB = LuCfg<R>::NB;
  // panels up to kPanelSmemBytes stay in shared memory; taller ones use k_panel
  constexpr int kPanelSmemBytes = 200 * 1024;
  const int max_rows = kPanelSmemBytes / (NB * (int)sizeof(Cx<R>));
  static bool attr_set = false;
  if (!attr_set) {
    LSMS_CUDA_TRY(cudaFuncSetAttribute(k_panel_smem<R, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kPanelSmemBytes));
    attr_set = true;
  }
  for (int k = 0; k < n_max; k += NB) {
    const int m_max = n_max - k;
    if (m_max > max_rows)
      LSMS_LAUNCH((k_panel<R, NB>), dim3(n_units), dim3(256), 0, st, d_units, fac_base, k, stat, max_rows);
    const int rows_smem = std::min(m_max, max_rows);
    LSMS_LAUNCH((k_panel_smem<R, NB>), dim3(n_units), dim3(512), (size_t)rows_smem * NB * sizeof(Cx<R>), st,
                d_units, fac_base, k, stat, max_rows);
    // one warp per column outside the panel: left ones [0, k), right ones [k + NB, n)
    LSMS_LAUNCH((k_swap_trsm<R, NB>), dim3((n_max + kSwapCols - 1) / kSwapCols, n_units), dim3(256), 0, st, d_units,
                fac_base, k);
    const int trail = n_max - k - NB;
    if (trail <= 0) continue;
    if constexpr (std::is_same<R, float>::value) {
      // complex64: the trailing update runs on the tensor cores (3xTF32, tc_gemm.cu)
      const int rc = gemm_tc_chunk(d_units, n_units, n_max, k, fac_base, stat, st);
      if (rc) return rc;
    } else {
      const int tiles = (trail + 63) / 64;
      LSMS_LAUNCH((k_gemm<R, NB>), dim3(tiles * tiles, n_units), dim3(256), 0, st, d_units, fac_base, k, tiles);
    }
  }
  LSMS_LAUNCH(k_perm, dim3((n_units + 127) / 128), dim3(128), 0, st, d_units, n_units, fac_base);
  return LSMS_OK;
}

template <typename R>
int lu_solve_chunk(const Unit* d_units, int n_units, const char* fac_base, char* ws, int which_rhs, int nrhs,
                   const int32_t* done, cudaStream_t st) {
  if (nrhs < 1 || nrhs > 32) return fail(LSMS_ERR_ARG, "internal: nrhs %d out of range", nrhs);
  constexpr int NB = LuCfg<R>::NB;
  LSMS_LAUNCH((k_solve<R, NB>), dim3(n_units), dim3(512), 0, st, d_units, fac_base, ws, which_rhs, nrhs, done);
  return LSMS_OK;
}

template int lu_factor_chunk<double>(const Unit*, int, int, char*, int32_t*, cudaStream_t);
template int lu_factor_chunk<float>(const Unit*, int, int, char*, int32_t*, cudaStream_t);
template int lu_solve_chunk<double>(const Unit*, int, const char*, char*, int, int, const int32_t*, cudaStream_t);
template int lu_solve_chunk<float>(const Unit*, int, const char*, char*, int, int, const int32_t*, cudaStream_t);

}  // namespace lsms
