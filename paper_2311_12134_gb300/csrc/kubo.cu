// Kubo-Greenwood traces, their fixed-order reduction into sigma and rho, and
// the adjoint (gradient) kernels.
//
// Eq. (lsms-conductivity-formula): for centre atom m and energy pair
// c = (z1, z2),
//   S_c[mu][nu](m) = sum_{n in LIZ_m} Tr[ J^{m mu}(z2,z1) tau^{0n}(z1) J^{n nu}(z1,z2) tau^{n0}(z2) ]
// with tau^{0n} = (tau^{n0})^T (complex-symmetric M).  Eq.
// (sigma-tilde-consolidation) then combines the four pairs at finite delta.
// FP64 arithmetic, except the mixed form's K x K products (double-float on the
// FP32 pipes, FP64-class accuracy); sums over atoms and sites run in a fixed order.
#include <cmath>
#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace lsms {

// c = 2a + b for (z1, z2) = (a, b), a/b = 0 for +, 1 for -; the swapped pair is 2b + a.
__device__ __forceinline__ int swap_combo(int c) { return ((c & 1) << 1) | (c >> 1); }

// J (per delta block d at d * J_dstride) as double-float (hi, lo) pairs, compact:
// out[d][per].  grid (ceil(per / 256), n_dj).
__global__ void k_split_j(const double2* __restrict__ J, int64_t J_dstride, int64_t per, float4* __restrict__ out) {
  const int d = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (int64_t)gridDim.x * blockDim.x)
    out[(size_t)d * per + i] = df_split(J[(size_t)d * J_dstride + i]);
}

// ------------------------------------------------------------------ forward traces
// grid (n_atoms, n_delta * 4), block 256 = 16 x 16 element threads.
// DF = false: FP64 arithmetic (FP64 form).  DF = true (mixed form): the K x K
// products and the site sum in double-float arithmetic on the FP32 pipes
// (unit roundoff about 2^-48; the last trace and everything after it in FP64).
template <bool DF>
__global__ void __launch_bounds__(256) k_kubo_partial(const int64_t* __restrict__ offsets,
                                                      const int32_t* __restrict__ site_atom,
                                                      const int32_t* __restrict__ species,
                                                      const double2* __restrict__ J, int64_t J_dstride,
                                                      const float4* __restrict__ Jdf, int64_t Jdf_dstride,
                                                      const double2* __restrict__ tau, int64_t S_total, int K,
                                                      int n_atoms, int n_species, const int32_t* __restrict__ halve,
                                                      double2* __restrict__ partial) {
  using V = typename std::conditional<DF, float4, double2>::type;
  using Acc = typename std::conditional<DF, DfAcc, double2>::type;
  const int m = blockIdx.x;
  const int d = blockIdx.y >> 2, c = blockIdx.y & 3;
  if (halve && c >= 2 && *halve) return;  // taken as the conjugate of combination 3 - c (k_kubo_reduce)
  const int a = c >> 1, b = c & 1;
  const int e1 = 2 * d + a, e2 = 2 * d + b;
  const int cb = swap_combo(c);
  const int KK = K * K;
  const double2* Jd = J + (size_t)d * J_dstride;
  const float4* Jdfd = DF ? Jdf + (size_t)d * Jdf_dstride : nullptr;  // J already split (mixed form)
  auto ldJ = [&](size_t idx) -> V {
    if constexpr (DF) return Jdfd[idx];
    else return Jd[idx];
  };
  __shared__ V sT1[16][17], sT2[16][17];
  __shared__ V sB[3][16][17];
  __shared__ V sP[3][16][17];
  auto ld = [](double2 x) -> V {
    if constexpr (DF) return df_split(x);
    else return x;
  };
  auto zero = []() -> Acc {
    if constexpr (DF) return df_zero();
    else return mk(0.0, 0.0);
  };
  auto mac = [](Acc& acc, V x, V y) {
    if constexpr (DF) dfc_mac(acc, x, y);
    else acc = cfma(x, y, acc);
  };
  auto val = [](const Acc& acc) -> V {
    if constexpr (DF) return df_value(acc);
    else return acc;
  };
  auto wide = [](V x) -> double2 {
    if constexpr (DF) return df_join(x);
    else return x;
  };
  auto nz = [](V x) -> bool {  // NaN counts as nonzero
    if constexpr (DF) return x.x != 0.f || x.z != 0.f;
    else return x.x != 0.0 || x.y != 0.0;
  };
  const int tid = threadIdx.x;
  const int i = tid >> 4, j = tid & 15, lane = tid & 31, warp = tid >> 5;
  const bool act = (i < K) && (j < K);
  const int spm = min(max(0, species[m]), n_species - 1);
  auto load_jm = [&]() {  // J^{m mu} of the swapped combination, into sB
    if (act) {
#pragma unroll
      for (int u = 0; u < 3; ++u) sB[u][i][j] = ldJ((((size_t)spm * 4 + cb) * 3 + u) * KK + i * K + j);
    }
  };
  // The trace Tr[J^{m mu} Y^nu] reads Y^nu(i, j) only where J^{m mu}(j, i) != 0
  // for some mu (the dipole J: at most 3 of 16 entries per row), so only those
  // entries of Y are accumulated, each by one thread of a compacted list.
  __shared__ int sList[256], sWarpCnt[8];
  __shared__ unsigned sJr[3][16];  // bit t of sJr[nu][x]: J^{n nu}(x, t) != 0
  load_jm();
  __syncthreads();
  int cnt = 0, my = -1;
  {
    const bool need = act && (nz(sB[0][j][i]) || nz(sB[1][j][i]) || nz(sB[2][j][i]));
    const unsigned bal = __ballot_sync(0xffffffffu, need);
    if (lane == 0) sWarpCnt[warp] = __popc(bal);
    __syncthreads();
    int base = 0;
    for (int w = 0; w < 8; ++w) {
      if (w < warp) base += sWarpCnt[w];
      cnt += sWarpCnt[w];
    }
    if (need) sList[base + __popc(bal & ((1u << lane) - 1u))] = tid;
    __syncthreads();
    if (tid < cnt) my = sList[tid];
  }
  const int yi = my >> 4, yj = my & 15;
  Acc Y[3];
#pragma unroll
  for (int v = 0; v < 3; ++v) Y[v] = zero();
  const int64_t s0 = offsets[m], s1 = offsets[m + 1];
  for (int64_t s = s0; s < s1; ++s) {
    const int sp = min(max(0, species[site_atom[s]]), n_species - 1);  // out-of-range ids never index J
    if (act) {
      sT1[i][j] = ld(tau[((size_t)e1 * S_total + s) * KK + i * K + j]);
      sT2[i][j] = ld(tau[((size_t)e2 * S_total + s) * KK + i * K + j]);
#pragma unroll
      for (int v = 0; v < 3; ++v) sB[v][i][j] = ldJ((((size_t)sp * 4 + c) * 3 + v) * KK + i * K + j);
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const unsigned br = __ballot_sync(0xffffffffu, act && nz(sB[v][i][j]));
      if (j == 0) sJr[v][i] = (br >> (lane & 16)) & 0xffffu;
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int v = 0; v < 3; ++v) {  // J^nu tau^{n0}(z2) over the nonzero entries of J's row i
        Acc acc = zero();
        for (unsigned b = sJr[v][i]; b; b &= b - 1) {
          const int q = __ffs(b) - 1;
          mac(acc, sB[v][i][q], sT2[q][j]);
        }
        sP[v][i][j] = val(acc);
      }
    }
    __syncthreads();
    if (my >= 0) {
#pragma unroll
      for (int v = 0; v < 3; ++v)
        for (int q = 0; q < K; ++q) mac(Y[v], sT1[q][yi], sP[v][q][yj]);  // tau^{0n}(z1) = tau^{n0}(z1)^T
    }
    __syncthreads();
  }
  // S[mu][nu] = Tr[J^{m mu} Y^nu] = sum_ij Jm[i][j] Y[j][i]; entries outside the list are 0
  if (act) {
#pragma unroll
    for (int v = 0; v < 3; ++v) sP[v][i][j] = V{};
  }
  load_jm();
  __syncthreads();
  if (my >= 0) {
#pragma unroll
    for (int v = 0; v < 3; ++v) sP[v][yi][yj] = val(Y[v]);
  }
  __syncthreads();
  __shared__ double2 red[9][8];
  for (int u = 0; u < 3; ++u)
    for (int v = 0; v < 3; ++v) {
      double2 t = act ? cmul(wide(sB[u][i][j]), wide(sP[v][j][i])) : mk(0.0, 0.0);
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
        t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
      }
      if (lane == 0) red[u * 3 + v][warp] = t;
    }
  __syncthreads();
  if (tid < 9) {
    double2 t = mk(0.0, 0.0);
    for (int w = 0; w < 8; ++w) t = cadd(t, red[tid][w]);
    partial[((size_t)(d * 4 + c) * n_atoms + m) * 9 + tid] = t;
  }
}

// grid (n_delta * 4 * 9), block 256: fixed-order sum over atoms.  With the halving
// flag set, combinations (-,+) and (-,-) are the conjugates of (+,-) and (+,+).
__global__ void __launch_bounds__(256) k_kubo_reduce(const double2* __restrict__ partial, int n_atoms,
                                                     const int32_t* __restrict__ halve, double2* __restrict__ S) {
  int dc = blockIdx.x / 9;
  const int e = blockIdx.x % 9;
  const int c = dc & 3;
  const bool conj_of = halve && c >= 2 && *halve;
  if (conj_of) dc = (dc & ~3) | (3 - c);
  double2 t = mk(0.0, 0.0);
  for (int m = threadIdx.x; m < n_atoms; m += blockDim.x) t = cadd(t, partial[((size_t)dc * n_atoms + m) * 9 + e]);
  __shared__ double2 sh[256];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) S[(size_t)(blockIdx.x / 9) * 9 + e] = conj_of ? mk(sh[0].x, -sh[0].y) : sh[0];
}

// Conjugate-pair mode: *flag = 1 when the current matrices allow the halving,
// J(-,-) = conj J(+,+) and J(-,+) = conj J(+,-) (to 1e-12 of the largest |J|,
// |.| = |Re| + |Im|), for every species and broadening block; else 0.  Then with
// tau(z*) = conj tau(z) the traces of (-,-) and (-,+) are the conjugates of those
// of (+,+) and (+,-).  One CTA; flag set before the traces run.
__global__ void __launch_bounds__(256) k_check_conj_j(const double2* __restrict__ J, int64_t J_dstride, int n_dj,
                                                      int64_t per_species4, int n_species, int32_t* flag) {
  // per_species4: elements of one combination block (3 K K); J[d][s][c][...]
  double dm = 0.0, am = 0.0;
  const int64_t total = (int64_t)n_dj * n_species * per_species4;
  for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
    const int64_t d = i / ((int64_t)n_species * per_species4);
    const int64_t r = i % ((int64_t)n_species * per_species4);
    const int64_t sp = r / per_species4, q = r % per_species4;
    const double2* Js = J + (size_t)d * J_dstride + (size_t)sp * 4 * per_species4;
    const double2 pp = Js[q], pm = Js[per_species4 + q], mp = Js[2 * per_species4 + q], mm = Js[3 * per_species4 + q];
    dm = fmax(dm, fmax(fabs(mm.x - pp.x) + fabs(mm.y + pp.y), fabs(mp.x - pm.x) + fabs(mp.y + pm.y)));
    am = fmax(am, fmax(fmax(cabs1(pp), cabs1(pm)), fmax(cabs1(mp), cabs1(mm))));
    if (!finite2(pp) || !finite2(pm) || !finite2(mp) || !finite2(mm)) dm = INFINITY;
  }
  __shared__ double s1[256], s2[256];
  s1[threadIdx.x] = dm;
  s2[threadIdx.x] = am;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s1[threadIdx.x] = fmax(s1[threadIdx.x], s1[threadIdx.x + w]);
      s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *flag = (s1[0] <= 1e-12 * s2[0]) ? 1 : 0;
}

// one block: sigma~ = -S/(pi V), sigma = (st0 - st1 - st2 + st3)/4, rho = (Re sigma)^{-1}
__global__ void k_kubo_finish(const double2* __restrict__ S, int n_delta, double volume,
                              double2* __restrict__ sigma_tilde, double2* __restrict__ sigma,
                              double* __restrict__ rho) {
  const double pref = -1.0 / (M_PI * volume);
  for (int d = threadIdx.x; d < n_delta; d += blockDim.x) {
    double2 sg[9];
    for (int e = 0; e < 9; ++e) {
      double2 acc = mk(0.0, 0.0);
      for (int c = 0; c < 4; ++c) {
        const double2 st = mk(pref * S[(size_t)(d * 4 + c) * 9 + e].x, pref * S[(size_t)(d * 4 + c) * 9 + e].y);
        if (sigma_tilde) sigma_tilde[(size_t)(d * 4 + c) * 9 + e] = st;
        const double sgn = (c == 0 || c == 3) ? 0.25 : -0.25;
        acc.x += sgn * st.x;
        acc.y += sgn * st.y;
      }
      sg[e] = acc;
      sigma[(size_t)d * 9 + e] = acc;
    }
    if (rho) {
      const double a0 = sg[0].x, a1 = sg[1].x, a2 = sg[2].x, a3 = sg[3].x, a4 = sg[4].x, a5 = sg[5].x,
                   a6 = sg[6].x, a7 = sg[7].x, a8 = sg[8].x;
      const double c0 = a4 * a8 - a5 * a7, c1 = a5 * a6 - a3 * a8, c2 = a3 * a7 - a4 * a6;
      const double det = a0 * c0 + a1 * c1 + a2 * c2;
      const double id = 1.0 / det;
      double* o = rho + (size_t)d * 9;
      o[0] = c0 * id;
      o[1] = (a2 * a7 - a1 * a8) * id;
      o[2] = (a1 * a5 - a2 * a4) * id;
      o[3] = c1 * id;
      o[4] = (a0 * a8 - a2 * a6) * id;
      o[5] = (a2 * a3 - a0 * a5) * id;
      o[6] = c2 * id;
      o[7] = (a1 * a6 - a0 * a7) * id;
      o[8] = (a0 * a4 - a1 * a3) * id;
    }
  }
}

// ------------------------------------------------------------------ adjoint
// f = sum conj(w) sigma.  Abar^nu_{m,d,c} = a_c sum_mu conj(w[d][mu][nu]) J^{m mu}(swap c),
// a_c = -s_c / (4 pi V).  grid (n_atoms, n_delta * 4), block 256.
__global__ void __launch_bounds__(256) k_adj_abar(const int32_t* __restrict__ species,
                                                  const double2* __restrict__ J, int64_t J_dstride,
                                                  const double2* __restrict__ w, int K, double volume,
                                                  int n_delta, int n_species, double2* __restrict__ abar,
                                                  float4* __restrict__ abar_df) {
  const int m = blockIdx.x;
  const int d = blockIdx.y >> 2, c = blockIdx.y & 3;
  const int cb = swap_combo(c);
  const int KK = K * K;
  const int tid = threadIdx.x;
  if (tid >= KK) return;
  const double2* Jd = J + (size_t)d * J_dstride;
  const int sp = min(max(0, species[m]), n_species - 1);
  const double ac = ((c == 0 || c == 3) ? -1.0 : 1.0) / (4.0 * M_PI * volume);
  for (int v = 0; v < 3; ++v) {
    double2 acc = mk(0.0, 0.0);
    for (int u = 0; u < 3; ++u) {
      const double2 wc = w[(size_t)d * 9 + u * 3 + v];
      const double2 cw = mk(ac * wc.x, -ac * wc.y);
      acc = cfma(cw, Jd[(((size_t)sp * 4 + cb) * 3 + u) * KK + tid], acc);
    }
    const size_t o = ((((size_t)m * n_delta + d) * 4 + c) * 3 + v) * KK + tid;
    abar[o] = acc;
    if (abar_df) abar_df[o] = df_split(acc);  // split once for the double-float right-hand sides
  }
}

// Right-hand sides of the adjoint solves for unit (m, e), one CTA per LIZ site n:
//   B[:, 0:K]  rows of site n = sum_{c: z1 = z_e} sum_nu J^{n nu}(c) tau^{n0}(z2) Abar^nu_c
//   B[:, K:2K] rows of site n = sum_{c: z2 = z_e} sum_nu J^{n nu}(c)^T tau^{n0}(z1) (Abar^nu_c)^T
// B is column-major n x 2K complex128 at ws + unit.r_off.  grid (S_max, n_units).
// DF: the products in double-float arithmetic on the FP32 pipes (FP64 accuracy,
// mixed form); otherwise FP64.
template <bool DF>
__global__ void __launch_bounds__(256) k_adj_rhs(const Unit* __restrict__ units, const int32_t* __restrict__ site_atom,
                                                 const int32_t* __restrict__ species, const double2* __restrict__ J,
                                                 int64_t J_dstride, const double2* __restrict__ tau, int64_t S_total,
                                                 const double2* __restrict__ abar, const float4* __restrict__ Jdf,
                                                 int64_t Jdf_dstride, const float4* __restrict__ abar_df,
                                                 int n_delta, int n_species, int K, char* ws) {
  using V = typename std::conditional<DF, float4, double2>::type;
  const Unit u = units[blockIdx.y];
  const int nsite = blockIdx.x;
  if (nsite >= u.S) return;
  const int KK = K * K;
  const int m = u.atom, e = u.energy;
  const int d = e >> 1, sgn = e & 1;
  const int64_t s = u.site_off + nsite;
  const int sp = min(max(0, species[site_atom[s]]), n_species - 1);
  const double2* Jd = J + (size_t)d * J_dstride;
  __shared__ V sT[16][17], sJ[16][17], sA[16][17], sQ[16][17];
  // nonzero patterns: bit t of r[x] = entry (x, t) nonzero, of c[x] = entry (t, x)
  __shared__ unsigned sJr[16], sJc[16], sAr[16], sAc[16];
  const int tid = threadIdx.x, i = tid >> 4, j = tid & 15, lane = tid & 31;
  const bool act = (i < K) && (j < K);
  auto load = [](double2 x) -> V {
    if constexpr (DF) return df_split(x);
    else return x;
  };
  auto nz = [](V x) -> bool {  // NaN counts as nonzero
    if constexpr (DF) return x.x != 0.f || x.z != 0.f;
    else return x.x != 0.0 || x.y != 0.0;
  };
  // the patterns of a 16 x 16 shared matrix: a warp holds rows 2w, 2w + 1 (16 lanes each)
  auto patterns = [&](const V (*M)[17], unsigned* r, unsigned* c) {
    const unsigned br = __ballot_sync(0xffffffffu, act && nz(M[i][j]));
    const unsigned bc = __ballot_sync(0xffffffffu, act && nz(M[j][i]));
    if (j == 0) {
      r[i] = (br >> (lane & 16)) & 0xffffu;
      c[i] = (bc >> (lane & 16)) & 0xffffu;
    }
  };
  DfAcc f1 = df_zero(), f2 = df_zero();
  double2 acc1 = mk(0.0, 0.0), acc2 = mk(0.0, 0.0);
  for (int part = 0; part < 2; ++part) {
    for (int cc = 0; cc < 2; ++cc) {
      // combos with z1 = z_e (part 0) or z2 = z_e (part 1)
      int c;
      if (part == 0) c = (sgn << 1) | cc;  // a = sgn, b = cc
      else c = (cc << 1) | sgn;            // a = cc, b = sgn
      const int a = c >> 1, b = c & 1;
      const int eo = (part == 0) ? (2 * d + b) : (2 * d + a);  // the other energy's tau
      if (act) sT[i][j] = load(tau[((size_t)eo * S_total + s) * KK + i * K + j]);
      for (int v = 0; v < 3; ++v) {
        if (act) {
          const size_t jo = (((size_t)sp * 4 + c) * 3 + v) * KK + i * K + j;
          const size_t ao = ((((size_t)m * n_delta + d) * 4 + c) * 3 + v) * KK + i * K + j;
          if constexpr (DF) {  // J and Abar split once per call (k_split_j, k_adj_abar)
            sJ[i][j] = Jdf[(size_t)d * Jdf_dstride + jo];
            sA[i][j] = abar_df[ao];
          } else {
            sJ[i][j] = Jd[jo];
            sA[i][j] = abar[ao];
          }
        }
        // a zero Abar^nu_c (gradient weights without this nu) contributes nothing
        if (!__syncthreads_or(act && nz(sA[i][j]))) continue;
        // The products run over the nonzero entries only (the dipole J couples
        // l to l +- 1, m to m, m +- 1: at most 3 of 16 per row and column), in
        // ascending order: the same sums as the dense loops.
        patterns(sJ, sJr, sJc);
        patterns(sA, sAr, sAc);
        __syncthreads();
        if (act) {
          if constexpr (DF) {
            DfAcc q = df_zero();
            if (part == 0)
              for (unsigned mk_ = sJr[i]; mk_; mk_ &= mk_ - 1) {
                const int t = __ffs(mk_) - 1;
                dfc_mac(q, sJ[i][t], sT[t][j]);  // J tau
              }
            else
              for (unsigned mk_ = sJc[i]; mk_; mk_ &= mk_ - 1) {
                const int t = __ffs(mk_) - 1;
                dfc_mac(q, sJ[t][i], sT[t][j]);  // J^T tau
              }
            sQ[i][j] = df_value(q);
          } else {
            double2 q = mk(0.0, 0.0);
            if (part == 0)
              for (unsigned mk_ = sJr[i]; mk_; mk_ &= mk_ - 1) {
                const int t = __ffs(mk_) - 1;
                q = cfma(sJ[i][t], sT[t][j], q);
              }
            else
              for (unsigned mk_ = sJc[i]; mk_; mk_ &= mk_ - 1) {
                const int t = __ffs(mk_) - 1;
                q = cfma(sJ[t][i], sT[t][j], q);
              }
            sQ[i][j] = q;
          }
        }
        __syncthreads();
        if (act) {
          // part 0: (J tau) Abar over column j of Abar; part 1: (J^T tau) Abar^T over row j
          const unsigned am = part == 0 ? sAc[j] : sAr[j];
          for (unsigned mk_ = am; mk_; mk_ &= mk_ - 1) {
            const int t = __ffs(mk_) - 1;
            if constexpr (DF) {
              if (part == 0) dfc_mac(f1, sQ[i][t], sA[t][j]);
              else dfc_mac(f2, sQ[i][t], sA[j][t]);
            } else {
              if (part == 0) acc1 = cfma(sQ[i][t], sA[t][j], acc1);
              else acc2 = cfma(sQ[i][t], sA[j][t], acc2);
            }
          }
        }
        __syncthreads();
      }
    }
  }
  if (act) {
    if constexpr (DF) {
      acc1 = df_join(df_value(f1));
      acc2 = df_join(df_value(f2));
    }
    double2* B = reinterpret_cast<double2*>(ws + u.r_off);
    const int n = u.n;
    B[(size_t)j * n + K * nsite + i] = acc1;
    B[(size_t)(K + j) * n + K * nsite + i] = acc2;
  }
}

// Per-site gradient contribution for unit (m, e), site p (one CTA each):
//   D_p = - tau^{p0} (X1_p)^T - X2_p (tau^{p0})^T,  X = M^{-1} B  (n x 2K at ws + unit.x_off)
// written to G[e][s] (K x K row-major).  grid (S_max, n_units).  DF: the products
// in double-float arithmetic on the FP32 pipes (mixed form), else FP64.
template <bool DF>
__global__ void __launch_bounds__(256) k_adj_site(const Unit* __restrict__ units, const double2* __restrict__ tau,
                                                  int64_t S_total, int K, const char* ws, double2* __restrict__ G) {
  using V = typename std::conditional<DF, float4, double2>::type;
  const Unit u = units[blockIdx.y];
  const int p = blockIdx.x;
  if (p >= u.S) return;
  const int KK = K * K;
  const int e = u.energy, n = u.n;
  const int64_t s = u.site_off + p;
  const double2* X = reinterpret_cast<const double2*>(ws + u.x_off);
  __shared__ V sT[16][17], sX1[16][17], sX2[16][17];
  auto ld = [](double2 x) -> V {
    if constexpr (DF) return df_split(x);
    else return x;
  };
  const int tid = threadIdx.x, i = tid >> 4, j = tid & 15;
  const bool act = (i < K) && (j < K);
  if (act) {
    sT[i][j] = ld(tau[((size_t)e * S_total + s) * KK + i * K + j]);
    sX1[i][j] = ld(X[(size_t)j * n + K * p + i]);
    sX2[i][j] = ld(X[(size_t)(K + j) * n + K * p + i]);
  }
  __syncthreads();
  if (act) {
    double2 r;
    if constexpr (DF) {
      DfAcc acc = df_zero();
      for (int t = 0; t < K; ++t) {
        dfc_mac(acc, sT[i][t], sX1[j][t]);   // tau^{p0} X1^T
        dfc_mac(acc, sX2[i][t], sT[j][t]);   // X2 tau^{p0 T}
      }
      r = df_join(df_value(acc));
    } else {
      double2 acc = mk(0.0, 0.0);
      for (int t = 0; t < K; ++t) {
        acc = cfma(sT[i][t], sX1[j][t], acc);
        acc = cfma(sX2[i][t], sT[j][t], acc);
      }
      r = acc;
    }
    G[((size_t)e * S_total + s) * KK + i * K + j] = mk(-r.x, -r.y);
  }
}

// grad_tinv[e][i] = conj( sum over the sites of atom i, in site order ).  grid (n_atoms, n_energy).
__global__ void __launch_bounds__(256) k_adj_reduce(const int64_t* __restrict__ inv_off,
                                                    const int64_t* __restrict__ inv_sites,
                                                    const double2* __restrict__ G, int64_t S_total, int K,
                                                    int n_atoms, double2* __restrict__ grad) {
  const int a = blockIdx.x, e = blockIdx.y;
  const int KK = K * K;
  const int t = threadIdx.x;
  if (t >= KK) return;
  double2 acc = mk(0.0, 0.0);
  for (int64_t q = inv_off[a]; q < inv_off[a + 1]; ++q) acc = cadd(acc, G[((size_t)e * S_total + inv_sites[q]) * KK + t]);
  grad[((size_t)e * n_atoms + a) * KK + t] = mk(acc.x, -acc.y);
}

// grad_species[s][e] = sum over atoms of species s (atom order) of grad[e][atom].
// grid (n_species, n_energy).
__global__ void __launch_bounds__(256) k_adj_species(const int32_t* __restrict__ species,
                                                     const double2* __restrict__ grad, int K, int n_atoms,
                                                     int n_energy, double2* __restrict__ out) {
  const int s = blockIdx.x, e = blockIdx.y;
  const int KK = K * K;
  const int t = threadIdx.x;
  if (t >= KK) return;
  double2 acc = mk(0.0, 0.0);
  for (int a = 0; a < n_atoms; ++a)
    if (species[a] == s) acc = cadd(acc, grad[((size_t)e * n_atoms + a) * KK + t]);
  out[((size_t)s * n_energy + e) * KK + t] = acc;
}

// ------------------------------------------------------------------ wrappers
int kubo_forward(const int64_t* offsets, const int32_t* site_atom, const int32_t* species, int n_species,
                 const double2* J, int64_t J_dstride, const double2* tau, int64_t S_total, int K, int n_atoms, int n_delta,
                 double volume, bool df, float4* jdf, double2* partial, double2* S, double2* sigma_tilde,
                 double2* sigma, double* rho, cudaStream_t st, int32_t* halve) {
  if (halve) {
    const int n_dj = J_dstride > 0 ? n_delta : 1;
    LSMS_LAUNCH(k_check_conj_j, dim3(1), dim3(256), 0, st, J, J_dstride > 0 ? J_dstride : 0, n_dj,
                (int64_t)3 * K * K, n_species, halve);
  }
  if (df) {
    const int64_t per = (int64_t)n_species * 12 * K * K;
    const int n_dj = J_dstride > 0 ? n_delta : 1;
    LSMS_LAUNCH(k_split_j, dim3((unsigned)((per + 255) / 256), n_dj), dim3(256), 0, st, J, J_dstride, per, jdf);
    LSMS_LAUNCH(k_kubo_partial<true>, dim3(n_atoms, n_delta * 4), dim3(256), 0, st, offsets, site_atom, species, J,
                J_dstride, jdf, J_dstride > 0 ? per : 0, tau, S_total, K, n_atoms, n_species, halve, partial);
  } else {
    LSMS_LAUNCH(k_kubo_partial<false>, dim3(n_atoms, n_delta * 4), dim3(256), 0, st, offsets, site_atom, species, J,
                J_dstride, nullptr, 0, tau, S_total, K, n_atoms, n_species, halve, partial);
  }
  LSMS_LAUNCH(k_kubo_reduce, dim3(n_delta * 4 * 9), dim3(256), 0, st, partial, n_atoms, halve, S);
  LSMS_LAUNCH(k_kubo_finish, dim3(1), dim3(32), 0, st, S, n_delta, volume, sigma_tilde, sigma, rho);
  return LSMS_OK;
}

// x *= a for n complex values.
__global__ void k_cscale(double2* __restrict__ x, int64_t n, double a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = mk(a * x[i].x, a * x[i].y);
}

// The per-atom terms of Eq. (lsms-conductivity-formula) with the -1/(pi V)
// prefactor: out [n_delta][4][n_atoms][3][3].
int kubo_atoms(const int64_t* offsets, const int32_t* site_atom, const int32_t* species, int n_species,
               const double2* J, int64_t J_dstride, const double2* tau, int64_t S_total, int K, int n_atoms,
               int n_delta, double volume, bool df, float4* jdf, double2* out, cudaStream_t st) {
  if (df) {
    const int64_t per = (int64_t)n_species * 12 * K * K;
    const int n_dj = J_dstride > 0 ? n_delta : 1;
    LSMS_LAUNCH(k_split_j, dim3((unsigned)((per + 255) / 256), n_dj), dim3(256), 0, st, J, J_dstride, per, jdf);
    LSMS_LAUNCH(k_kubo_partial<true>, dim3(n_atoms, n_delta * 4), dim3(256), 0, st, offsets, site_atom, species, J,
                J_dstride, jdf, J_dstride > 0 ? per : 0, tau, S_total, K, n_atoms, n_species, nullptr, out);
  } else {
    LSMS_LAUNCH(k_kubo_partial<false>, dim3(n_atoms, n_delta * 4), dim3(256), 0, st, offsets, site_atom, species, J,
                J_dstride, nullptr, 0, tau, S_total, K, n_atoms, n_species, nullptr, out);
  }
  const int64_t cnt = (int64_t)n_delta * 4 * n_atoms * 9;
  LSMS_LAUNCH(k_cscale, dim3((unsigned)std::min<int64_t>((cnt + 255) / 256, 4096)), dim3(256), 0, st, out, cnt,
              -1.0 / (M_PI * volume));
  return LSMS_OK;
}

int adj_abar(const int32_t* species, int n_species, const double2* J, int64_t J_dstride, const double2* w, int K,
             double volume, int n_atoms, int n_delta, double2* abar, float4* abar_df, cudaStream_t st) {
  LSMS_LAUNCH(k_adj_abar, dim3(n_atoms, n_delta * 4), dim3(256), 0, st, species, J, J_dstride, w, K, volume,
              n_delta, n_species, abar, abar_df);
  return LSMS_OK;
}

int split_j(const double2* J, int64_t J_dstride, int n_species, int K, int n_delta, float4* out, int64_t* out_dstride,
            cudaStream_t st) {
  const int64_t per = (int64_t)n_species * 12 * K * K;
  const int n_dj = J_dstride > 0 ? n_delta : 1;
  LSMS_LAUNCH(k_split_j, dim3((unsigned)((per + 255) / 256), n_dj), dim3(256), 0, st, J, J_dstride, per, out);
  *out_dstride = J_dstride > 0 ? per : 0;
  return LSMS_OK;
}

int adj_rhs(const Unit* d_units, int n_units, int S_max, const int32_t* site_atom, const int32_t* species,
            int n_species, const double2* J, int64_t J_dstride, const double2* tau, int64_t S_total,
            const double2* abar, const float4* jdf, int64_t jdf_dstride, const float4* abar_df, int n_delta, int K,
            char* ws, bool df, cudaStream_t st) {
  if (df)
    LSMS_LAUNCH(k_adj_rhs<true>, dim3(S_max, n_units), dim3(256), 0, st, d_units, site_atom, species, J, J_dstride,
                tau, S_total, abar, jdf, jdf_dstride, abar_df, n_delta, n_species, K, ws);
  else
    LSMS_LAUNCH(k_adj_rhs<false>, dim3(S_max, n_units), dim3(256), 0, st, d_units, site_atom, species, J, J_dstride,
                tau, S_total, abar, nullptr, 0, nullptr, n_delta, n_species, K, ws);
  return LSMS_OK;
}

int adj_site(const Unit* d_units, int n_units, int S_max, const double2* tau, int64_t S_total, int K, const char* ws,
             double2* G, bool df, cudaStream_t st) {
  if (df) LSMS_LAUNCH(k_adj_site<true>, dim3(S_max, n_units), dim3(256), 0, st, d_units, tau, S_total, K, ws, G);
  else LSMS_LAUNCH(k_adj_site<false>, dim3(S_max, n_units), dim3(256), 0, st, d_units, tau, S_total, K, ws, G);
  return LSMS_OK;
}

int adj_reduce(const int64_t* inv_off, const int64_t* inv_sites, const double2* G, int64_t S_total, int K,
               int n_atoms, int n_energy, double2* grad, cudaStream_t st) {
  LSMS_LAUNCH(k_adj_reduce, dim3(n_atoms, n_energy), dim3(256), 0, st, inv_off, inv_sites, G, S_total, K, n_atoms,
              grad);
  return LSMS_OK;
}

int adj_species(const int32_t* species, const double2* grad, int K, int n_atoms, int n_species, int n_energy,
                double2* out, cudaStream_t st) {
  LSMS_LAUNCH(k_adj_species, dim3(n_species, n_energy), dim3(256), 0, st, species, grad, K, n_atoms, n_energy, out);
  return LSMS_OK;
}

}  // namespace lsms

// ------------------------------------------------------------------ sigma without allocation
// Scratch for lsms_kubo_sigma_noalloc: the per-atom partial traces and the
// reduced sums live in this file-scope device array instead of memory the call
// allocates.  Host code must not use its name as an address; the address is
// fetched per device with cudaGetSymbolAddress.
namespace lsms {
namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;
__device__ __align__(256) unsigned char g_sigma_scratch[kNoAllocScratchBytes];
std::mutex g_scratch_mu;
void* g_scratch_addr[64];

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

// Bytes of the double-float copy of J used by the mixed-form traces.
size_t jdf_scratch_bytes(int n_species, int K, int n_delta, int64_t J_dstride) {
  return round256((size_t)(J_dstride > 0 ? n_delta : 1) * n_species * 12 * K * K * sizeof(float4));
}

namespace {

int scratch_address(void** out) {
  int dev = 0;
  LSMS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(LSMS_ERR_CUDA, "device index %d unsupported", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sigma_scratch);
    if (e != cudaSuccess || !p)
      return fail(LSMS_ERR_CUDA, "cudaGetSymbolAddress of the sigma scratch failed: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LSMS_OK;
}
}  // namespace

}  // namespace lsms

using namespace lsms;

extern "C" int lsms_kubo_sigma_noalloc(const lsms_liz* liz_c, int lmax, const int32_t* species, int n_species,
                                       const lsms_complex* J, int64_t J_delta_stride, const lsms_complex* tau,
                                       int n_delta, double volume, int precision, lsms_complex* sigma_tilde,
                                       lsms_complex* sigma, double* rho, void* stream) {
  clear_error();
  lsms_liz* liz = const_cast<lsms_liz*>(liz_c);
  if (!liz) return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_noalloc: NULL liz");
  if (lmax < 0 || lmax > kMaxLmax) return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_noalloc: lmax must be in 0..%d", kMaxLmax);
  if (!species || n_species < 1) return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_noalloc: species required, n_species >= 1");
  if (n_delta < 1 || 2 * n_delta > kMaxEnergies || !J || !tau || !sigma)
    return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_noalloc: J, tau, sigma required, 1 <= n_delta <= %d", kMaxEnergies / 2);
  if (!(volume > 0.0) || !std::isfinite(volume)) return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_noalloc: volume must be > 0");
  if (J_delta_stride < 0) return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_noalloc: negative J stride");
  if (precision != LSMS_FP64 && precision != LSMS_MIXED)
    return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_noalloc: unknown precision %d", precision);
  const int K = (lmax + 1) * (lmax + 1);
  const size_t part_bytes = round256((size_t)n_delta * 4 * liz->n_atoms * 9 * sizeof(double2));
  const size_t s_bytes = round256((size_t)n_delta * 36 * sizeof(double2));
  const size_t jdf_bytes = precision == LSMS_MIXED ? jdf_scratch_bytes(n_species, K, n_delta, J_delta_stride) : 0;
  if (part_bytes + s_bytes + jdf_bytes > kNoAllocScratchBytes)
    return fail(LSMS_ERR_ARG,
                "lsms_kubo_sigma_noalloc: %d atoms x %d deltas need %zu bytes of scratch; the static buffer holds "
                "%zu bytes (about 29,000 atom-delta pairs); use lsms_kubo_sigma",
                liz->n_atoms, n_delta, part_bytes + s_bytes + jdf_bytes, kNoAllocScratchBytes);
  DeviceData* dd = nullptr;
  int rc = existing_device_data(liz, &dd);
  if (rc) return rc;
  void* scratch = nullptr;
  if ((rc = scratch_address(&scratch))) return rc;
  char* base = static_cast<char*>(scratch);
  // Every scratch element read by the kernels is written earlier in the same
  // call (split J by k_split_j, partial traces by k_kubo_partial, sums by
  // k_kubo_reduce), so the previous call's contents need no clearing.
  return kubo_forward(dd->offsets, dd->site_atom, species, n_species, reinterpret_cast<const double2*>(J),
                      J_delta_stride, reinterpret_cast<const double2*>(tau), liz->total_sites, K, liz->n_atoms,
                      n_delta, volume, precision == LSMS_MIXED,
                      reinterpret_cast<float4*>(base + part_bytes + s_bytes), reinterpret_cast<double2*>(base),
                      reinterpret_cast<double2*>(base + part_bytes),
                      reinterpret_cast<double2*>(sigma_tilde), reinterpret_cast<double2*>(sigma), rho,
                      reinterpret_cast<cudaStream_t>(stream), nullptr);
}
