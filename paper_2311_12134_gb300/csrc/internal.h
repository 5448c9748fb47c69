// Internal declarations shared by the host (C++) and device (CUDA) parts of
// liblsmskubo.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lsmskubo.h"

namespace lsms {

constexpr int kMaxLmax = 3;
constexpr int kMaxK = 16;                       // (kMaxLmax + 1)^2
constexpr int kMaxL3 = 2 * kMaxLmax;            // l'' range of g
constexpr int kMaxK3 = (kMaxL3 + 1) * (kMaxL3 + 1);

// Error reporting (thread-local message; returns the code for chaining).
int fail(int code, const char* fmt, ...);
void clear_error();

// Mixed form: the region at m64_off holds the double-float copy of M (n x n
// float4) and, after it, the inverses of the 32 x 32 diagonal blocks of L and U
// (complex64, column-major, block b at 2 b 1024 entries: L^-1 then U^-1).
#ifdef __CUDACC__
#define LSMS_HD __host__ __device__
#else
#define LSMS_HD
#endif
constexpr int kDiagNB = 32;
LSMS_HD inline int64_t diag_inv_rel_off(int n) { return ((int64_t)n * n * 16 + 255) / 256 * 256; }
LSMS_HD inline int64_t diag_inv_bytes(int n) {
  return ((int64_t)((n + kDiagNB - 1) / kDiagNB) * 2 * kDiagNB * kDiagNB * 8 + 255) / 256 * 256;
}
// After the diagonal-block inverses: the pivot-growth record of the unit, two
// floats (max |M| over the assembled matrix, max |U| over the complex64 factor;
// |.| = |Re| + |Im|), padded to 256 bytes.
LSMS_HD inline int64_t growth_rel_off(int n) { return diag_inv_rel_off(n) + diag_inv_bytes(n); }
constexpr int64_t kGrowthBytes = 256;
// After the growth record: the largest |Re| or |Im| of the high parts of each
// row of M (n floats), the row scales of the tensor-core refinement residual.
LSMS_HD inline int64_t rowmax_rel_off(int n) { return growth_rel_off(n) + kGrowthBytes; }
LSMS_HD inline int64_t m64_region_bytes(int n) { return rowmax_rel_off(n) + ((int64_t)n * 4 + 255) / 256 * 256; }
// The double-float copy of X (n x nrhs float4) is followed by the largest |Re|
// or |Im| of the high parts of each column (at most 32 floats), the column
// scales of the tensor-core residual.
LSMS_HD inline int64_t colmax_rel_off(int n, int nrhs) { return ((int64_t)n * nrhs * 16 + 255) / 256 * 256; }
constexpr int64_t kColmaxBytes = 256;

// One (atom, energy) LIZ problem inside a chunk of the batched solve.
struct Unit {
  int32_t atom;      // centre atom m
  int32_t energy;    // energy index e
  int32_t n;         // K * S_m
  int32_t S;         // LIZ size S_m
  int64_t site_off;  // first site of LIZ_m in the global site arrays
  int64_t fac_off;   // byte offset of the factor matrix (from fac base)
  int64_t m64_off;   // byte offset of the double-float copy of M and the diagonal-block inverses (mixed form)
  int64_t piv_off;   // byte offset of the pivots (from fac base)
  int64_t x_off;     // byte offset of the n x RHS complex128 solution block (workspace)
  int64_t r_off;     // byte offset of the n x RHS complex128 residual block (workspace)
  int64_t x32_off;   // byte offset of the n x RHS complex64 scratch (workspace)
  int64_t p_off;     // byte offset of the convergence-probe vectors (mixed form, workspace)
  int64_t xdf_off;   // byte offset of X as double-float (hi, lo) pairs (mixed form, workspace)
  int64_t stat_off;  // index into the per-unit scratch scalars
  int32_t conj;      // 1: solved with its conjugate partner's factors on conjugated right-hand sides
  int32_t pad;
};

struct Chunk {
  int u0, u1;        // unit range in the plan
  int f0, f1;        // range of the units that own factors (fac_units)
  int n_max;         // largest n in the chunk (units are sorted by n, descending)
  size_t ws_bytes;   // workspace bytes used by the chunk
};

// Work plan of one call shape.  units: every (atom, energy) system solved;
// fac_units: the ones whose matrix is assembled and factored (all of them,
// except the second energy of each conjugate pair in the conjugate-pair mode,
// which reuses its partner's factors).  Both are atom-major, atoms sorted by
// LIZ size (largest first); a chunk holds whole atoms.
struct Plan {
  int lmax = -1, n_energy = 0, precision = 0, nrhs = 0;
  bool store = false, conj = false;
  int fac_per_atom = 0;          // fac_units per atom
  size_t ws_bytes = 0;
  std::vector<Unit> units;       // host copies
  std::vector<Unit> fac_units;
  std::vector<Chunk> chunks;
  void* d_block = nullptr;       // one device allocation holding the two device copies
  Unit* d_units = nullptr;
  Unit* d_fac_units = nullptr;
};

struct DeviceData {
  void* block = nullptr;         // one device allocation holding the arrays below
  int64_t* offsets = nullptr;    // [N+1]
  int32_t* site_atom = nullptr;  // [S]
  double* disp = nullptr;        // [S][3]
  int64_t* inv_off = nullptr;    // [N+1] sites of each atom (images included)
  int64_t* inv_sites = nullptr;  // [S]
  int32_t* site_centre = nullptr;// [S] centre atom of the LIZ holding site s
  std::map<std::tuple<int, int, int, int, size_t, int>, Plan> plans;
};

}  // namespace lsms

struct lsms_liz {
  int n_atoms = 0;
  int64_t total_sites = 0;
  int max_sites = 0, min_sites = 0;
  bool periodic = false;
  std::vector<int64_t> offsets;
  std::vector<int32_t> site_atom;
  std::vector<int32_t> image;
  std::vector<double> disp;
  std::vector<int64_t> inv_off;
  std::vector<int64_t> inv_sites;
  std::vector<int32_t> site_centre;
  std::mutex mu;
  std::map<int, lsms::DeviceData> dev;  // per CUDA device
};

namespace lsms {
// Host tables (host.cpp).
// Real Gaunt C[L1][L2][L3], L1, L2 < (lmax+1)^2, L3 < (2 lmax+1)^2.
std::vector<double> gaunt_real(int lmax);
// Sparse coupling of g: for each (L, L') the list of (L'', s C_{LL'L''}),
// s = i^{l - l' - l''} = +-1 (the exponent is even whenever C != 0).
struct Coupling {
  std::vector<int32_t> start;   // [K*K + 1]
  std::vector<int32_t> lpp;     // [nnz] L''
  std::vector<double> coef;     // [nnz]
};
Coupling g_coupling(int lmax);
// Y_L normalisation N_l^|m| * (sqrt 2 for m != 0), L < (l3max+1)^2.
std::vector<double> ylm_norm(int l3max);
}  // namespace lsms
