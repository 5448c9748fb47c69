// C ABI entry points of liblsmskubo, the per-device tables and work plans, and
// the kernels that assemble the LIZ KKR matrices and refine the tau blocks.
//
// Path per call of lsms_tau_blocks (Eq. tau-inverse on every LIZ):
//   k_assemble   M = T^{-1} - g, g from Gaunt x h_l(kappa R) x Y_L(R^)
//   lu (lu.cu)   P M = L U, blocked, all units of a chunk per launch
//   k_solve      X = M^{-1} E0 -> tau^{p0}
//   mixed form:  complex64 LU/solves, then k_residual (B - M X to about
//                2^-48, double-float arithmetic on the FP32 pipes) / k_solve
//                (complex64 correction) / k_ir_update until the correction is
//                below 1e-10 of X (at most kIrMaxIter sweeps)
//   k_write_tau  scatter X into tau[e][site]
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <numeric>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace lsms {

std::atomic<long long> g_launches{0};
std::atomic<bool> g_timer_on{false};

namespace {
struct TimerRec {
  std::string name;
  int ev;  // index of the start event; the stop event is ev + 1
};
std::mutex g_timer_mu;
std::vector<cudaEvent_t> g_timer_events;
std::vector<TimerRec> g_timer_recs;
size_t g_timer_next = 0;

cudaEvent_t timer_event() {
  if (g_timer_next == g_timer_events.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_timer_events.push_back(e);
  }
  return g_timer_events[g_timer_next++];
}
}  // namespace

void timer_begin(const char* name, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_timer_mu);
  const int idx = (int)g_timer_next;
  cudaEvent_t a = timer_event();
  if (!a) return;
  cudaEventRecord(a, st);
  g_timer_recs.push_back(TimerRec{name, idx});
}

void timer_end(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_timer_mu);
  cudaEvent_t b = timer_event();
  if (!b) return;
  cudaEventRecord(b, st);
}

// kernels in kubo.cu
int kubo_forward(const int64_t* offsets, const int32_t* site_atom, const int32_t* species, int n_species,
                 const double2* J, int64_t J_dstride, const double2* tau, int64_t S_total, int K, int n_atoms, int n_delta,
                 double volume, bool df, float4* jdf, double2* partial, double2* S, double2* sigma_tilde,
                 double2* sigma, double* rho, cudaStream_t st, int32_t* halve);
size_t jdf_scratch_bytes(int n_species, int K, int n_delta, int64_t J_dstride);
int kubo_atoms(const int64_t* offsets, const int32_t* site_atom, const int32_t* species, int n_species,
               const double2* J, int64_t J_dstride, const double2* tau, int64_t S_total, int K, int n_atoms,
               int n_delta, double volume, bool df, float4* jdf, double2* out, cudaStream_t st);
int adj_abar(const int32_t* species, int n_species, const double2* J, int64_t J_dstride, const double2* w, int K,
             double volume, int n_atoms, int n_delta, double2* abar, float4* abar_df, cudaStream_t st);
int split_j(const double2* J, int64_t J_dstride, int n_species, int K, int n_delta, float4* out, int64_t* out_dstride,
            cudaStream_t st);
int adj_rhs(const Unit* d_units, int n_units, int S_max, const int32_t* site_atom, const int32_t* species,
            int n_species, const double2* J, int64_t J_dstride, const double2* tau, int64_t S_total,
            const double2* abar, const float4* jdf, int64_t jdf_dstride, const float4* abar_df, int n_delta, int K,
            char* ws, bool df, cudaStream_t st);
int adj_site(const Unit* d_units, int n_units, int S_max, const double2* tau, int64_t S_total, int K, const char* ws,
             double2* G, bool df, cudaStream_t st);
int adj_reduce(const int64_t* inv_off, const int64_t* inv_sites, const double2* G, int64_t S_total, int K,
               int n_atoms, int n_energy, double2* grad, cudaStream_t st);
int adj_species(const int32_t* species, const double2* grad, int K, int n_atoms, int n_species, int n_energy,
                double2* out, cudaStream_t st);

constexpr int kIrMaxIter = 6;
constexpr double kIrTol = 1e-10;

// Process-wide options (lsms_set_option / lsms_get_option).
static std::atomic<double> g_opt_growth_limit{1e3};
static std::atomic<int> g_opt_fallback_slots{8};
static std::atomic<int> g_opt_ir_max_sweeps{kIrMaxIter};
static std::atomic<int> g_opt_streams{0};  // 0: LSMS_STREAMS or the default
static std::atomic<int> g_opt_residual_tc{1};
static std::atomic<int> g_opt_solve_cols{0};  // 0: 8 columns per CTA up to 16 right-hand sides, else 16
static std::atomic<int> g_opt_solve_regs{0};
static std::atomic<int> g_opt_solve_steps{0};  // 0, 1: one CTA chain per unit and slice; 2: block-step launches
static std::atomic<int> g_opt_nvtx{0};

// NVTX range over one stage of a call (option "nvtx"; the header-only NVTX3
// calls cost nothing without an attached tool).  Ranges mark when the host
// enqueues a stage on its stream.
struct NvtxRange {
  bool on;
  explicit NvtxRange(const char* name) : on(g_opt_nvtx.load(std::memory_order_relaxed) != 0) {
    if (on) nvtxRangePushA(name);
  }
  ~NvtxRange() {
    if (on) nvtxRangePop();
  }
};
int opt_residual_tc() { return g_opt_residual_tc.load(); }
int opt_solve_cols() { return g_opt_solve_cols.load(); }
int opt_solve_regs() { return g_opt_solve_regs.load(); }
int opt_solve_steps() { return g_opt_solve_steps.load(); }
double opt_growth_limit() { return g_opt_growth_limit.load(); }
int opt_fallback_slots() { return g_opt_fallback_slots.load(); }
int opt_ir_max_sweeps() { return g_opt_ir_max_sweeps.load(); }
constexpr int kProbe = 2;  // random combinations of the right-hand sides in the convergence probe
constexpr size_t kAlign = 256;
static inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// ------------------------------------------------------------------ constant tables
constexpr int kCpMax = 768;  // nonzero Gaunt couplings for lmax = 3: 708
__constant__ int32_t c_cp_start[kMaxK * kMaxK + 1];
__constant__ int32_t c_cp_lpp[kCpMax];
__constant__ double c_cp_coef[kCpMax];
__constant__ double c_ylm_norm[kMaxK3];
__constant__ float2 c_ylm_norm_dd[kMaxK3];  // the same as (hi, lo) float pairs
__constant__ int32_t c_l_of[kMaxK3];

static std::mutex g_dev_mu;
static bool g_dev_init[64];

static int ensure_device_tables(int dev) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (dev < 0 || dev >= 64) return fail(LSMS_ERR_CUDA, "device index %d unsupported", dev);
  if (g_dev_init[dev]) return LSMS_OK;
  const Coupling cp = g_coupling(kMaxLmax);
  if (cp.lpp.size() > (size_t)kCpMax) return fail(LSMS_ERR_ARG, "internal: coupling table too large");
  const std::vector<double> nrm = ylm_norm(kMaxL3);
  std::vector<int32_t> lof(kMaxK3);
  for (int L = 0; L < kMaxK3; ++L) {
    int l = 0;
    while ((l + 1) * (l + 1) <= L) ++l;
    lof[L] = l;
  }
  LSMS_CUDA_TRY(cudaMemcpyToSymbol(c_cp_start, cp.start.data(), cp.start.size() * sizeof(int32_t)));
  LSMS_CUDA_TRY(cudaMemcpyToSymbol(c_cp_lpp, cp.lpp.data(), cp.lpp.size() * sizeof(int32_t)));
  LSMS_CUDA_TRY(cudaMemcpyToSymbol(c_cp_coef, cp.coef.data(), cp.coef.size() * sizeof(double)));
  LSMS_CUDA_TRY(cudaMemcpyToSymbol(c_ylm_norm, nrm.data(), nrm.size() * sizeof(double)));
  std::vector<float2> nrm_dd(nrm.size());
  for (size_t i = 0; i < nrm.size(); ++i) {
    const float h = (float)nrm[i];
    nrm_dd[i] = make_float2(h, (float)(nrm[i] - (double)h));
  }
  LSMS_CUDA_TRY(cudaMemcpyToSymbol(c_ylm_norm_dd, nrm_dd.data(), nrm_dd.size() * sizeof(float2)));
  LSMS_CUDA_TRY(cudaMemcpyToSymbol(c_l_of, lof.data(), lof.size() * sizeof(int32_t)));
  g_dev_init[dev] = true;
  return LSMS_OK;
}

// Several host arrays in one device allocation and one copy (each piece 256-byte
// aligned): a LIZ set's tables and a plan's unit lists cost one cudaMalloc, one
// cudaMemcpy and one cudaFree instead of one of each per array.
class Packed {
 public:
  template <typename T>
  size_t add(const std::vector<T>& v) {
    const size_t off = host_.size();
    const size_t bytes = v.size() * sizeof(T);
    host_.resize(off + align_up(std::max<size_t>(bytes, 1)));
    if (bytes) std::memcpy(host_.data() + off, v.data(), bytes);
    return off;
  }
  int upload(void** block) {
    LSMS_CUDA_TRY(cudaMalloc(block, std::max<size_t>(host_.size(), 1)));
    if (!host_.empty()) LSMS_CUDA_TRY(cudaMemcpy(*block, host_.data(), host_.size(), cudaMemcpyHostToDevice));
    return LSMS_OK;
  }

 private:
  std::vector<char> host_;
};
template <typename T>
static T* at(void* block, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(block) + off);
}

// Device copy of the LIZ arrays (made once per device, synchronous).
static int device_data(lsms_liz* liz, DeviceData** out) {
  int dev = 0;
  LSMS_CUDA_TRY(cudaGetDevice(&dev));
  int rc = ensure_device_tables(dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(liz->mu);
  auto it = liz->dev.find(dev);
  if (it == liz->dev.end()) {
    DeviceData dd;
    Packed pk;
    const size_t o_off = pk.add(liz->offsets), o_sa = pk.add(liz->site_atom), o_disp = pk.add(liz->disp),
                 o_ioff = pk.add(liz->inv_off), o_isites = pk.add(liz->inv_sites), o_sc = pk.add(liz->site_centre);
    if ((rc = pk.upload(&dd.block))) return rc;
    dd.offsets = at<int64_t>(dd.block, o_off);
    dd.site_atom = at<int32_t>(dd.block, o_sa);
    dd.disp = at<double>(dd.block, o_disp);
    dd.inv_off = at<int64_t>(dd.block, o_ioff);
    dd.inv_sites = at<int64_t>(dd.block, o_isites);
    dd.site_centre = at<int32_t>(dd.block, o_sc);
    it = liz->dev.emplace(dev, std::move(dd)).first;
  }
  *out = &it->second;
  return LSMS_OK;
}

// The device copy of a LIZ set if an earlier call made one on the current
// device; never allocates.
int existing_device_data(lsms_liz* liz, DeviceData** out) {
  int dev = 0;
  LSMS_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(liz->mu);
  auto it = liz->dev.find(dev);
  if (it == liz->dev.end())
    return fail(LSMS_ERR_ARG, "no device copy of this LIZ set on device %d: call lsms_tau_blocks with it first", dev);
  *out = &it->second;
  return LSMS_OK;
}

// ------------------------------------------------------------------ plans
struct UnitBytes {
  size_t fac, piv, m64, x, b, x32, probe, xdf;
};

static UnitBytes unit_bytes(int n, int precision, int nrhs, bool backward) {
  UnitBytes ub{};
  const size_t nn = (size_t)n * n;
  ub.fac = align_up(nn * (precision == LSMS_FP64 ? 16 : 8));
  ub.piv = align_up((size_t)n * 4);  // pivots (row interchanged with row i at step i)
  // double-float M + diagonal-block inverses + pivot-growth record + row maxima
  ub.m64 = precision == LSMS_FP64 ? 0 : (size_t)m64_region_bytes(n);
  ub.x = align_up((size_t)n * nrhs * 16);
  ub.b = backward ? align_up((size_t)n * nrhs * 16) : 0;
  // complex64 corrections; the convergence probe uses the first kProbe columns
  ub.x32 = precision == LSMS_FP64 ? 0 : align_up((size_t)n * std::max(nrhs, kProbe) * 8);
  ub.probe = precision == LSMS_FP64 ? 0 : align_up((size_t)n * kProbe * 2 * 16);  // y_q and (B w)_q
  // X as float4 (hi, lo) and its column maxima
  ub.xdf = precision == LSMS_FP64 ? 0 : (size_t)(colmax_rel_off(n, nrhs) + kColmaxBytes);
  return ub;
}

// Workspace bytes of a unit: the right-hand-side blocks, plus the factors,
// pivots and (mixed form) the double-float copy of M when the unit owns factors
// that live in the workspace (no factor store).
static size_t ws_unit_bytes(const UnitBytes& ub, bool factors_in_ws) {
  return (factors_in_ws ? ub.fac + ub.piv + ub.m64 : 0) + ub.x + ub.b + ub.x32 + ub.probe + ub.xdf;
}

// Energies of one atom solved by a plan, and whether each owns factors.
// conj: energies come in (z, conj z) pairs; the forward solves only the first
// of each pair, the backward solves both with the first one's factors.
static void plan_energies(int n_energy, bool conj, bool backward, std::vector<int>* es, std::vector<char>* owns) {
  es->clear();
  owns->clear();
  for (int e = 0; e < n_energy; ++e) {
    if (conj && (e & 1) && !backward) continue;
    es->push_back(e);
    owns->push_back(!(conj && (e & 1)));
  }
}

// Atoms sorted by LIZ size (largest first, then atom index); every energy of an atom is adjacent.
static std::vector<int> atom_order(const lsms_liz* liz) {
  std::vector<int> order(liz->n_atoms);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (liz->offsets[a + 1] - liz->offsets[a]) > (liz->offsets[b + 1] - liz->offsets[b]);
  });
  return order;
}

// FP64 fallback of the mixed form: `slots` FP64 re-solves, each sized for the
// largest LIZ matrix (factors, pivots, solution, and for the adjoint its
// right-hand sides), plus the slot table and the slot count.
struct FbLayout {
  int slots = 0;
  size_t fac = 0, piv = 0, x = 0, b = 0, slot = 0;
  size_t units_off = 0, count_off = 0, region_off = 0, total = 0;
};

static FbLayout fb_layout(const lsms_liz* liz, int lmax, int precision, int nrhs, bool backward) {
  FbLayout f;
  f.slots = precision == LSMS_MIXED ? std::max(opt_fallback_slots(), 0) : 0;
  if (!f.slots) return f;
  const size_t n = (size_t)(lmax + 1) * (lmax + 1) * liz->max_sites;
  f.fac = align_up(n * n * 16);
  f.piv = align_up(n * 4);
  f.x = align_up(n * nrhs * 16);
  f.b = backward ? f.x : 0;
  f.slot = f.fac + f.piv + f.x + f.b;
  f.units_off = 0;
  f.count_off = align_up((size_t)f.slots * sizeof(Unit));
  f.region_off = f.count_off + kAlign;
  f.total = f.region_off + (size_t)f.slots * f.slot;
  return f;
}

struct WsHeader {
  size_t stat, done, extra, fb, chunk;  // byte offsets
  size_t total_fixed;
};

static WsHeader ws_header(const lsms_liz* liz, int n_energy, size_t extra_bytes, size_t fb_bytes) {
  WsHeader h{};
  const size_t nu = (size_t)liz->n_atoms * n_energy;
  h.stat = 0;
  h.done = align_up(nu * 4);
  h.extra = h.done + align_up(nu * 4);
  h.fb = h.extra + align_up(extra_bytes);
  h.chunk = h.fb + align_up(fb_bytes);
  h.total_fixed = h.chunk;
  return h;
}

// Conjugate-pair mode: one flag per energy pair (t^-1 pair not conjugate).
static size_t conj_extra_bytes(int n_energy) { return align_up((size_t)(n_energy / 2 + 1) * 4); }

// abar (complex128), the per-site gradient blocks, abar as double-float pairs
static size_t backward_extra_bytes(const lsms_liz* liz, int lmax, int n_energy) {
  const size_t KK = (size_t)(lmax + 1) * (lmax + 1) * (lmax + 1) * (lmax + 1);
  const int n_delta = n_energy / 2;
  return 2 * align_up((size_t)liz->n_atoms * n_delta * 12 * KK * 16) +
         align_up((size_t)n_energy * liz->total_sites * KK * 16);
}

static int get_plan(lsms_liz* liz, DeviceData* dd, int lmax, int n_energy, int precision, int nrhs, bool backward,
                    bool store, bool conj, size_t chunk_bytes, Plan** out) {
  const auto key = std::make_tuple(lmax, n_energy, precision,
                                   nrhs * 8 + (conj ? 4 : 0) + (backward ? 2 : 0) + (store ? 1 : 0), chunk_bytes, 0);
  std::lock_guard<std::mutex> lk(liz->mu);
  auto it = dd->plans.find(key);
  if (it != dd->plans.end()) {
    *out = &it->second;
    return LSMS_OK;
  }
  const int K = (lmax + 1) * (lmax + 1);
  Plan p;
  p.lmax = lmax;
  p.n_energy = n_energy;
  p.precision = precision;
  p.nrhs = nrhs;
  p.store = store;
  p.conj = conj;
  p.ws_bytes = chunk_bytes;
  std::vector<int> es;
  std::vector<char> owns;
  plan_energies(n_energy, conj, backward, &es, &owns);
  p.fac_per_atom = (int)std::count(owns.begin(), owns.end(), 1);
  const std::vector<int> order = atom_order(liz);
  size_t store_off = 0;
  size_t cur = 0;
  Chunk ch{0, 0, 0, 0, 0, 0};
  for (int m : order) {
    const int S = (int)(liz->offsets[m + 1] - liz->offsets[m]);
    const int n = K * S;
    const UnitBytes ub = unit_bytes(n, precision, nrhs, backward);
    size_t need = 0;
    for (size_t i = 0; i < es.size(); ++i) need += ws_unit_bytes(ub, owns[i] && !store);
    if (need > chunk_bytes)
      return fail(LSMS_ERR_NOMEM, "workspace of %zu bytes cannot hold the %zu energies of one atom (%zu bytes)",
                  chunk_bytes, es.size(), need);
    if (cur + need > chunk_bytes) {  // chunks hold whole atoms (all energies)
      ch.u1 = (int)p.units.size();
      ch.f1 = (int)p.fac_units.size();
      ch.ws_bytes = cur;
      p.chunks.push_back(ch);
      ch = Chunk{(int)p.units.size(), 0, (int)p.fac_units.size(), 0, 0, 0};
      cur = 0;
    }
    Unit owner{};
    for (size_t i = 0; i < es.size(); ++i) {
      Unit u{};
      u.atom = m;
      u.energy = es[i];
      u.n = n;
      u.S = S;
      u.site_off = liz->offsets[m];
      if (owns[i]) {
        if (store) {
          u.fac_off = (int64_t)store_off;
          u.piv_off = (int64_t)(store_off + ub.fac);
          u.m64_off = (int64_t)(store_off + ub.fac + ub.piv);
          store_off += ub.fac + ub.piv + ub.m64;
        } else {
          u.fac_off = (int64_t)cur;
          u.piv_off = (int64_t)(cur + ub.fac);
          u.m64_off = (int64_t)(cur + ub.fac + ub.piv);
          cur += ub.fac + ub.piv + ub.m64;
        }
        owner = u;
      } else {  // second energy of a conjugate pair: the first one's factors (just placed)
        u.fac_off = owner.fac_off;
        u.piv_off = owner.piv_off;
        u.m64_off = owner.m64_off;
        u.conj = 1;
      }
      u.x_off = (int64_t)cur;
      cur += ub.x;
      u.r_off = (int64_t)cur;
      cur += ub.b;
      u.x32_off = (int64_t)cur;
      cur += ub.x32;
      u.p_off = (int64_t)cur;
      cur += ub.probe;
      u.xdf_off = (int64_t)cur;
      cur += ub.xdf;
      u.stat_off = (int64_t)es[i] * liz->n_atoms + m;  // index of this unit's status word
      ch.n_max = std::max(ch.n_max, n);
      p.units.push_back(u);
      if (owns[i]) p.fac_units.push_back(u);
    }
  }
  ch.u1 = (int)p.units.size();
  ch.f1 = (int)p.fac_units.size();
  ch.ws_bytes = cur;
  p.chunks.push_back(ch);
  Packed pk;
  const size_t o_u = pk.add(p.units), o_f = pk.add(p.fac_units);
  int rc = pk.upload(&p.d_block);
  if (rc) return rc;
  p.d_units = at<Unit>(p.d_block, o_u);
  p.d_fac_units = at<Unit>(p.d_block, o_f);
  it = dd->plans.emplace(key, std::move(p)).first;
  *out = &it->second;
  return LSMS_OK;
}

// ------------------------------------------------------------------ assembly
constexpr int kAsmQ = 16;  // column sites per set-up round
constexpr int kAsmE = 2;   // energies per set-up round

// Y_L(R^), l <= 6: real harmonics without the Condon-Shortley phase from the
// upward associated-Legendre recurrence for P_l^m / sin^m and (x + i y)^m.
__device__ void ylm6(double x, double y, double z, double* Y) {
  double tr = 1.0, ti = 0.0;  // (x + i y)^m
  double qmm = 1.0;           // (2m - 1)!!
#pragma unroll
  for (int m = 0; m <= kMaxL3; ++m) {
    if (m > 0) {
      const double nr = tr * x - ti * y;
      ti = tr * y + ti * x;
      tr = nr;
      qmm *= (2 * m - 1);
    }
    double q2 = 0.0, q1 = 0.0;
#pragma unroll
    for (int l = m; l <= kMaxL3; ++l) {
      double q;
      if (l == m) q = qmm;
      else if (l == m + 1) q = (2 * m + 1) * z * qmm;
      else q = ((2 * l - 1) * z * q1 - (l + m - 1) * q2) * (1.0 / (l - m));
      q2 = q1;
      q1 = q;
      const int L0 = l * l + l;
      if (m == 0) {
        Y[L0] = c_ylm_norm[L0] * q;
      } else {
        Y[L0 + m] = c_ylm_norm[L0 + m] * q * tr;
        Y[L0 - m] = c_ylm_norm[L0 - m] * q * ti;
      }
    }
  }
}

// hp[l] = mpref * h_l(kappa d), l <= 6, where mpref * sum_L'' i^{l-l'-l''} C_{LL'L''}
// h_l''(kappa d) Y_L''(R^) is the block -g: kappa = principal sqrt(z); Im z >= 0:
// h = h^(1), mpref = +4 pi i kappa; Im z < 0: h = h^(2), mpref = -4 pi i kappa (the
// decaying, advanced branch).  Upward recurrence h_{l+1} = (2l+1)/x h_l - h_{l-1}.
__device__ void hankel6(double d, double2 z, double2* hp) {
  const double r = hypot(z.x, z.y);
  const double kre = sqrt(0.5 * (r + z.x));
  double kim = sqrt(0.5 * fmax(r - z.x, 0.0));
  const bool adv = z.y < 0.0;
  if (adv) kim = -kim;
  const double four_pi = 4.0 * M_PI;
  const double2 mpref = adv ? mk(four_pi * kim, -four_pi * kre) : mk(-four_pi * kim, four_pi * kre);
  const double2 xx = mk(kre * d, kim * d);
  const double2 ix = crcp(xx);
  double sn, cs;
  sincos(xx.x, &sn, &cs);
  const double f = exp(adv ? xx.y : -xx.y);
  const double2 ex = adv ? mk(f * cs, -f * sn) : mk(f * cs, f * sn);  // e^{-+ix}
  double2 hm = cmul(ex, ix);                                             // h_{-1}
  double2 h = adv ? mk(-hm.y, hm.x) : mk(hm.y, -hm.x);                  // h_0
  hp[0] = cmul(mpref, h);
#pragma unroll
  for (int l = 0; l < kMaxL3; ++l) {
    const double2 hn = csub(cmul(mk((2.0 * l + 1.0) * ix.x, (2.0 * l + 1.0) * ix.y), h), hm);
    hm = h;
    h = hn;
    hp[l + 1] = cmul(mpref, h);
  }
}

// The same two set-ups in double-float arithmetic on the FP32 pipes (mixed form):
// only the square root, the reciprocal, sincos and exp stay in FP64.
__device__ void ylm6_df(float2 x, float2 y, float2 z, float2* Y) {
  float2 tr = make_float2(1.f, 0.f), ti = make_float2(0.f, 0.f);  // (x + i y)^m
  float qmm_f = 1.f;                                               // (2m - 1)!! (exact in float)
#pragma unroll
  for (int m = 0; m <= kMaxL3; ++m) {
    if (m > 0) {
      const float2 nr = dd_sub(dd_mul(tr, x), dd_mul(ti, y));
      ti = dd_add(dd_mul(tr, y), dd_mul(ti, x));
      tr = nr;
      qmm_f *= (float)(2 * m - 1);
    }
    const float2 qmm = make_float2(qmm_f, 0.f);
    float2 q2 = make_float2(0.f, 0.f), q1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int l = m; l <= kMaxL3; ++l) {
      float2 q;
      if (l == m) q = qmm;
      else if (l == m + 1) q = dd_mulf(dd_mul(z, qmm), (float)(2 * m + 1));
      else q = dd_mul(dd_sub(dd_mulf(dd_mul(z, q1), (float)(2 * l - 1)), dd_mulf(q2, (float)(l + m - 1))),
                      dd_from(1.0 / (l - m)));
      q2 = q1;
      q1 = q;
      const int L0 = l * l + l;
      if (m == 0) {
        Y[L0] = dd_mul(c_ylm_norm_dd[L0], q);
      } else {
        const float2 qc = dd_mul(c_ylm_norm_dd[L0 + m], q);
        Y[L0 + m] = dd_mul(qc, tr);
        Y[L0 - m] = dd_mul(qc, ti);
      }
    }
  }
}

// hp[l] = mpref h_l(kappa d) in double-float; kappa and mpref of the energy given.
__device__ void hankel6_df(double d, double2 kap, double2 mpref, bool adv, float4* hp) {
  const double2 xx = mk(kap.x * d, kap.y * d);
  const double2 ix = crcp(xx);
  double sn, cs;
  sincos(xx.x, &sn, &cs);
  const double f = exp(adv ? xx.y : -xx.y);
  const double2 ex = adv ? mk(f * cs, -f * sn) : mk(f * cs, f * sn);  // e^{-+ix}
  const double2 hm64 = cmul(ex, ix);                                   // h_{-1}
  const double2 h064 = adv ? mk(-hm64.y, hm64.x) : mk(hm64.y, -hm64.x);  // h_0
  const float4 ixd = ddc(dd_from(ix.x), dd_from(ix.y));
  const float4 mp = ddc(dd_from(mpref.x), dd_from(mpref.y));
  float4 hm = ddc(dd_from(hm64.x), dd_from(hm64.y));
  float4 h = ddc(dd_from(h064.x), dd_from(h064.y));
  hp[0] = ddc_mul(mp, h);
#pragma unroll
  for (int l = 0; l < kMaxL3; ++l) {
    const float4 hn = ddc_sub(ddc_mul(ddc_scalef(ixd, (float)(2 * l + 1)), h), hm);
    hm = h;
    h = hn;
    hp[l + 1] = ddc_mul(mp, h);
  }
}

// Tolerance of the complex-symmetry check of the t^{-1} blocks (relative to the
// block's largest entry, |.| = |Re| + |Im|).
constexpr double kSymTol = 1e-12;

// grid (S_max, atoms in the chunk), block 256: one CTA per row site p of one
// atom's LIZ, for all energies of that atom.  First, the t^{-1} block of site p
// is checked for complex symmetry at every energy (M^T = M is what makes the
// row block tau^{0n} = (tau^{n0})^T); a block that is not symmetric to kSymTol
// flags the unit LSMS_UNIT_TINV_ASYM.  Only the blocks (p, q >= p) are formed:
// off the diagonal M is complex symmetric (g_{L'L}(-R) = g_{LL'}(R), the Gaunt
// coefficients being symmetric in L, L' and Y_L(-R^) = (-1)^l Y_L(R^) with
// l + l' + l'' even), so block (q, p) is written as the transpose of (p, q).  Per
// round of 16 column sites q: 16 lanes compute Y_L(R^) once for all energies;
// then, 2 energies at a time, 32 lanes compute
// V[L''] = mpref h_l''(kappa R) Y_L''(R^) and thread (L, L') forms
// sum_L'' s C_{LL'L''} V[L''] for those blocks (diagonal blocks: t^{-1}).
// FP64 form: FP64 sums, M (complex128) written into the factor array.
// Mixed form: the sums in double-float arithmetic on the FP32 pipes (FP64
// accuracy); writes M as (hi, lo) float pairs (float4 per element, at
// fac_base + m64_off) for the refinement residual and, if write_fac, the hi part
// (complex64) as the matrix to factor; the largest |M| entry goes into the
// unit's pivot-growth record.
template <bool MIXED>
__global__ void __launch_bounds__(256, 4) k_assemble(const Unit* __restrict__ units, int nE,
                                                  const double* __restrict__ disp,
                                                  const int32_t* __restrict__ site_atom,
                                                  const int32_t* __restrict__ species,
                                                  const double2* __restrict__ tinv, int n_species, int n_energy,
                                                  EnergyTable E, int K, char* fac_base, char* ws, bool write_fac,
                                                  int32_t* stat) {
  const Unit* ua = units + (size_t)blockIdx.y * nE;
  const Unit u0 = ua[0];
  const int p = blockIdx.x;
  if (p >= u0.S) return;
  const int S = u0.S, n = u0.n;
  __shared__ __align__(16) unsigned char sYraw[kAsmQ * kMaxK3 * 8];  // FP64 or double-float Y_L
  __shared__ double sD[kAsmQ];
  __shared__ __align__(16) unsigned char sVraw[kAsmE * kAsmQ * kMaxK3 * 16];
  // Gaunt coupling table in shared memory: threads index it divergently, which
  // constant memory would serialise.
  __shared__ double s_coef[kCpMax];
  __shared__ float2 s_coef2[kCpMax];
  __shared__ int32_t s_lpp[kCpMax];
  __shared__ int32_t s_start[kMaxK * kMaxK + 1];
  const int tid = threadIdx.x;
  for (int i = tid; i < kMaxK * kMaxK + 1; i += blockDim.x) s_start[i] = c_cp_start[i];
  const int n_cp = c_cp_start[kMaxK * kMaxK];
  for (int i = tid; i < n_cp; i += blockDim.x) {
    const double c = c_cp_coef[i];
    s_coef[i] = c;
    const float ch = (float)c;
    s_coef2[i] = make_float2(ch, (float)(c - (double)ch));
    s_lpp[i] = c_cp_lpp[i];
  }
  const int L = tid & 15, Lp = tid >> 4;
  const bool act = (L < K) && (Lp < K);
  const int64_t sp0 = u0.site_off + p;
  const double px = disp[3 * sp0], py = disp[3 * sp0 + 1], pz = disp[3 * sp0 + 2];
  int spp = species[site_atom[sp0]];
  int bad = 0;
  if (spp < 0 || spp >= n_species) {  // reject without reading outside tinv
    bad = LSMS_UNIT_BAD_INPUT;
    spp = 0;
  }
  // complex symmetry of the t^{-1} block of site p, per energy of this atom
  __shared__ unsigned int s_dmax[kMaxEnergies], s_amax[kMaxEnergies];
  for (int i = tid; i < nE; i += blockDim.x) s_dmax[i] = s_amax[i] = 0u;
  __syncthreads();
  for (int ee = 0; ee < nE; ++ee) {
    float dv = 0.f, av = 0.f;
    if (act) {
      const double2* tb = tinv + (((size_t)spp * n_energy) + ua[ee].energy) * K * K;
      const double2 a = tb[L * K + Lp], b = tb[Lp * K + L];
      dv = (float)(fabs(a.x - b.x) + fabs(a.y - b.y));
      av = (float)cabs1(a);
    }
    dv = warp_max_nonneg(dv);
    av = warp_max_nonneg(av);
    if ((tid & 31) == 0) {
      atomicMax(&s_dmax[ee], __float_as_uint(dv));
      atomicMax(&s_amax[ee], __float_as_uint(av));
    }
  }
  __syncthreads();
  int t0 = 0, t1 = 0;
  if (act) {
    t0 = s_start[L * kMaxK + Lp];
    t1 = s_start[L * kMaxK + Lp + 1];
  }
  // mixed form: this thread's couplings (at most kCpPair for lmax <= 3) in registers, so a
  // Gaunt term costs one shared-memory load (V) instead of three
  constexpr int kCpPair = 7;
  float2 cpc[kCpPair];
  int cpl[kCpPair];
  const bool cp_regs = t1 - t0 <= kCpPair;
#pragma unroll
  for (int t = 0; t < kCpPair; ++t) {
    const bool in = MIXED && t0 + t < t1;
    cpc[t] = in ? s_coef2[t0 + t] : make_float2(0.f, 0.f);
    cpl[t] = in ? s_lpp[t0 + t] : 0;
  }
  // mixed form: row maxima of block row p (over the columns of blocks q >= p; the
  // CTAs of sites q < p add the rest through their transposed blocks) and the
  // largest |M| entry, per energy of the atom; NONFINITE per energy
  __shared__ unsigned int s_rmax[kMaxEnergies][kMaxK];
  __shared__ unsigned int s_mmax[kMaxEnergies];
  __shared__ int s_flags[kMaxEnergies];
  // mixed form: row maxima of the transposed blocks' rows K q + L' of one group
  __shared__ unsigned int s_tmax[kAsmE][kAsmQ][kMaxK];
  for (int x = tid; x < kAsmE * kAsmQ * kMaxK; x += blockDim.x) (&s_tmax[0][0][0])[x] = 0u;
  for (int x = tid; x < nE * kMaxK; x += blockDim.x) (&s_rmax[0][0])[x] = 0u;
  for (int x = tid; x < nE; x += blockDim.x) {
    s_mmax[x] = 0u;
    s_flags[x] = 0;
  }
  // rounds of kAsmQ column sites q >= p (block (q, p) is the transpose of (p, q));
  // the harmonics of a round serve every energy, the Hankel set-up and the Gaunt
  // sums run kAsmE energies at a time
  for (int q0 = p; q0 < S; q0 += kAsmQ) {
    const int nq = min(kAsmQ, S - q0);
    __syncthreads();
    if (tid < kAsmQ) {
      const int q = q0 + tid;
      if (tid < nq && q != p) {
        const int64_t sq = u0.site_off + q;
        const double rx = disp[3 * sq] - px, ry = disp[3 * sq + 1] - py, rz = disp[3 * sq + 2] - pz;
        const double d = sqrt(rx * rx + ry * ry + rz * rz);
        const double id = 1.0 / d;
        sD[tid] = d;
        if (MIXED)
          ylm6_df(dd_from(rx * id), dd_from(ry * id), dd_from(rz * id),
                  reinterpret_cast<float2*>(sYraw) + tid * kMaxK3);
        else
          ylm6(rx * id, ry * id, rz * id, reinterpret_cast<double*>(sYraw) + tid * kMaxK3);
      }
    }
    for (int e0 = 0; e0 < nE; e0 += kAsmE) {
      const int ne = min(kAsmE, nE - e0);
      __syncthreads();
      if (tid < kAsmE * kAsmQ) {
        const int ee = tid / kAsmQ, qq = tid % kAsmQ, q = q0 + qq;
        if (ee < ne && qq < nq && q != p) {
          const int base = (ee * kAsmQ + qq) * kMaxK3;
          if (MIXED) {
            const double2 z = E.z[ua[e0 + ee].energy];
            const double r = hypot(z.x, z.y);
            const double kre = sqrt(0.5 * (r + z.x));
            double kim = sqrt(0.5 * fmax(r - z.x, 0.0));
            const bool adv = z.y < 0.0;
            if (adv) kim = -kim;
            const double four_pi = 4.0 * M_PI;
            const double2 mpref = adv ? mk(four_pi * kim, -four_pi * kre) : mk(-four_pi * kim, four_pi * kre);
            float4 hp[kMaxL3 + 1];
            hankel6_df(sD[qq], mk(kre, kim), mpref, adv, hp);
            const float2* Yq = reinterpret_cast<const float2*>(sYraw) + qq * kMaxK3;
#pragma unroll
            for (int l = 0; l <= kMaxL3; ++l)
              for (int Lpp = l * l; Lpp < (l + 1) * (l + 1); ++Lpp)
                reinterpret_cast<float4*>(sVraw)[base + Lpp] = ddc_scale(hp[l], Yq[Lpp]);
          } else {
            double2 hp[kMaxL3 + 1];
            hankel6(sD[qq], E.z[ua[e0 + ee].energy], hp);
            const double* Yq = reinterpret_cast<const double*>(sYraw) + qq * kMaxK3;
#pragma unroll
            for (int l = 0; l <= kMaxL3; ++l)
              for (int Lpp = l * l; Lpp < (l + 1) * (l + 1); ++Lpp)
                reinterpret_cast<double2*>(sVraw)[base + Lpp] = mk(hp[l].x * Yq[Lpp], hp[l].y * Yq[Lpp]);
          }
        }
      }
      __syncthreads();
      int nf[kAsmE];
      float mmax[kAsmE];  // mixed form: largest |M| entry written, per energy
      float rmax[kAsmE];  // mixed form: largest |Re| or |Im| (high parts) in this thread's row, per energy
#pragma unroll
      for (int ee = 0; ee < kAsmE; ++ee) {
        nf[ee] = 0;
        mmax[ee] = 0.f;
        rmax[ee] = 0.f;
      }
      for (int ee = 0; ee < ne && act; ++ee) {
        const Unit& u = ua[e0 + ee];
        for (int qq = 0; qq < nq; ++qq) {
          const int q = q0 + qq;
          const size_t idx = (size_t)(K * q + Lp) * n + K * p + L;
          const int base = (ee * kAsmQ + qq) * kMaxK3;
          if (MIXED) {
            float4 v4;
            if (q == p) {
              v4 = df_split(tinv[(((size_t)spp * n_energy) + u.energy) * K * K + L * K + Lp]);
            } else {
              DfAcc acc = df_zero();
              const float4* Vq = reinterpret_cast<const float4*>(sVraw) + base;
              if (cp_regs) {
#pragma unroll
                for (int t = 0; t < kCpPair; ++t)
                  if (t0 + t < t1) dfr_mac(acc, cpc[t], Vq[cpl[t]]);
              } else {
                for (int t = t0; t < t1; ++t) dfr_mac(acc, s_coef2[t], Vq[s_lpp[t]]);
              }
              v4 = df_value(acc);
            }
            if (!(isfinite(v4.x) && isfinite(v4.z))) nf[ee] |= LSMS_UNIT_NONFINITE;
            mmax[ee] = fmaxf(mmax[ee], fabsf(v4.x) + fabsf(v4.z));
            const float vm = fmaxf(fabsf(v4.x), fabsf(v4.z));
            rmax[ee] = fmaxf(rmax[ee], vm);
            const float4 m4 = make_float4(v4.x, v4.z, v4.y, v4.w);
            reinterpret_cast<float4*>(fac_base + u.m64_off)[idx] = m4;
            if (write_fac) reinterpret_cast<float2*>(fac_base + u.fac_off)[idx] = make_float2(v4.x, v4.z);
            if (q != p) {  // M(K q + L', K p + L) = M(K p + L, K q + L')
              const size_t idt = (size_t)(K * p + L) * n + K * q + Lp;
              reinterpret_cast<float4*>(fac_base + u.m64_off)[idt] = m4;
              if (write_fac) reinterpret_cast<float2*>(fac_base + u.fac_off)[idt] = make_float2(v4.x, v4.z);
              unsigned tm = __float_as_uint(vm <= 3.4e38f ? vm : __int_as_float(0x7f800000));
              if (K == kMaxK) {  // every lane active: the 16 lanes of row K q + L' reduce in registers
#pragma unroll
                for (int off = 1; off < 16; off <<= 1) tm = max(tm, __shfl_xor_sync(0xffffffffu, tm, off));
                if (L == 0) s_tmax[ee][qq][Lp] = max(s_tmax[ee][qq][Lp], tm);
              } else {
                atomicMax(&s_tmax[ee][qq][Lp], tm);
              }
            }
          } else {
            double2 v;
            if (q == p) {
              v = tinv[(((size_t)spp * n_energy) + u.energy) * K * K + L * K + Lp];
            } else {
              v = mk(0.0, 0.0);
              const double2* Vq = reinterpret_cast<const double2*>(sVraw) + base;
              for (int t = t0; t < t1; ++t) {
                const double c = s_coef[t];
                const double2 w = Vq[s_lpp[t]];
                v.x = fma(c, w.x, v.x);
                v.y = fma(c, w.y, v.y);
              }
            }
            if (!finite2(v)) nf[ee] |= LSMS_UNIT_NONFINITE;
            reinterpret_cast<double2*>(fac_base + u.fac_off)[idx] = v;
            if (q != p) reinterpret_cast<double2*>(fac_base + u.fac_off)[(size_t)(K * p + L) * n + K * q + Lp] = v;
          }
        }
      }
      if (MIXED) {  // maxima of the transposed blocks' rows K q + L' into the units' row maxima
        __syncthreads();  // the group's transposed maxima are complete
        for (int x = tid; x < ne * nq * kMaxK; x += blockDim.x) {
          const int ee = x / (nq * kMaxK), qq = (x / kMaxK) % nq, l2 = x % kMaxK;
          const int q = q0 + qq;
          if (l2 < K && q != p) {
            const Unit& u = ua[e0 + ee];
            atomicMax(reinterpret_cast<unsigned int*>(fac_base + u.m64_off + rowmax_rel_off(u.n)) + K * q + l2,
                      s_tmax[ee][qq][l2]);
          }
          s_tmax[ee][qq][l2] = 0u;
        }
      }
      for (int ee = 0; ee < ne; ++ee) {
        if (nf[ee]) atomicOr(&s_flags[e0 + ee], nf[ee]);
        if (MIXED) {
          const float wm = warp_max_nonneg(mmax[ee]);
          if ((tid & 31) == 0) atomicMax(&s_mmax[e0 + ee], __float_as_uint(wm));
          if (act) {
            float rm = rmax[ee] + 0.0f;
            if (!(rm <= 3.4e38f)) rm = __int_as_float(0x7f800000);
            atomicMax(&s_rmax[e0 + ee][L], __float_as_uint(rm));
          }
        }
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < nE; e += blockDim.x) {
    int f = bad | s_flags[e];
    if (!(__uint_as_float(s_dmax[e]) <= (float)kSymTol * __uint_as_float(s_amax[e]))) f |= LSMS_UNIT_TINV_ASYM;
    if (f) atomicOr(&stat[ua[e].stat_off], f);
    if (MIXED) atomic_max_nonneg(reinterpret_cast<float*>(fac_base + ua[e].m64_off + growth_rel_off(ua[e].n)),
                                 __uint_as_float(s_mmax[e]));
  }
  if (MIXED) {
    for (int x = tid; x < nE * kMaxK; x += blockDim.x) {
      const int e = x / kMaxK, l2 = x % kMaxK;
      if (l2 < K)
        atomicMax(reinterpret_cast<unsigned int*>(fac_base + ua[e].m64_off + rowmax_rel_off(ua[e].n)) + K * p + l2,
                  s_rmax[e][l2]);
    }
  }
}

// Zero the pivot-growth records and the row maxima of the units (before
// k_assemble, which raises them by atomic maxima).  One CTA per unit.
__global__ void k_growth_init(const Unit* __restrict__ units, int n_units, char* fac_base) {
  const Unit u = units[blockIdx.x];
  float* g = reinterpret_cast<float*>(fac_base + u.m64_off + growth_rel_off(u.n));
  if (threadIdx.x < 2) g[threadIdx.x] = 0.f;
  float* rm = reinterpret_cast<float*>(fac_base + u.m64_off + rowmax_rel_off(u.n));
  for (int i = threadIdx.x; i < u.n; i += blockDim.x) rm[i] = 0.f;
}

// Pivot growth of the complex64 factorization: LSMS_UNIT_GROWTH when
// max |U| > limit * max |M| (|.| = |Re| + |Im|).  With partial pivoting the
// growth stays near 1 on well-posed LIZ matrices; a large value means the
// complex64 factors may be too inaccurate for the refinement to recover FP64
// accuracy, and the unit is re-solved in the FP64 form.  One thread per unit.
__global__ void k_growth_check(const Unit* __restrict__ units, int n_units, const char* fac_base, float limit,
                               int32_t* stat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_units) return;
  const Unit u = units[i];
  const float* g = reinterpret_cast<const float*>(fac_base + u.m64_off + growth_rel_off(u.n));
  // a non-finite M is flagged by the assembly; a finite M with a non-finite factor is growth
  int w = (isfinite(g[0]) && !(g[1] <= limit * g[0])) ? LSMS_UNIT_GROWTH : 0;
  // bits 24-30: the growth's binary exponent + 64 (1..127; 127 also for a non-finite ratio)
  if (isfinite(g[0]) && g[0] > 0.f) {
    const float r = g[1] / g[0];
    const int code = !isfinite(r) ? 127 : (r > 0.f ? min(127, max(1, ilogbf(r) + 64)) : 1);
    w |= code << 24;
  }
  if (w) atomicOr(&stat[u.stat_off], w);
}

// lsms_unit_stats: one CTA reduces the status words into the stats record.
__global__ void __launch_bounds__(1024) k_unit_stats(const int32_t* __restrict__ st, int64_t n, lsms_stats* out) {
  constexpr int NF = 8;
  __shared__ unsigned long long s_sum[NF + 3];  // flags, invalid, sweeps, probes
  __shared__ int s_max[3];                      // sweeps, probes, growth code
  const int tid = threadIdx.x;
  if (tid < NF + 3) s_sum[tid] = 0ull;
  if (tid < 3) s_max[tid] = 0;
  __syncthreads();
  unsigned long long f[NF] = {}, inv = 0, sw = 0, pr = 0;
  int swm = 0, prm = 0, gm = 0;
  for (int64_t i = tid; i < n; i += blockDim.x) {
    const int w = st[i];
#pragma unroll
    for (int b = 0; b < NF; ++b) f[b] += (w >> b) & 1;
    inv += (w & 0xff & ~LSMS_UNIT_FP64_FALLBACK) != 0;
    const int s = (w >> 8) & 0xff, p = (w >> 16) & 0xff, g = (w >> 24) & 0x7f;
    sw += s;
    pr += p;
    swm = max(swm, s);
    prm = max(prm, p);
    gm = max(gm, g);
  }
#pragma unroll
  for (int b = 0; b < NF; ++b) atomicAdd(&s_sum[b], f[b]);
  atomicAdd(&s_sum[NF], inv);
  atomicAdd(&s_sum[NF + 1], sw);
  atomicAdd(&s_sum[NF + 2], pr);
  atomicMax(&s_max[0], swm);
  atomicMax(&s_max[1], prm);
  atomicMax(&s_max[2], gm);
  __syncthreads();
  if (tid == 0) {
    lsms_stats r;
    r.units = n;
    for (int b = 0; b < NF; ++b) r.flag_units[b] = (int64_t)s_sum[b];
    r.invalid_units = (int64_t)s_sum[NF];
    r.sweeps_sum = (int64_t)s_sum[NF + 1];
    r.probes_sum = (int64_t)s_sum[NF + 2];
    r.sweeps_max = s_max[0];
    r.probes_max = s_max[1];
    r.growth_code_max = s_max[2];
    *out = r;
  }
}

// ------------------------------------------------------------------ RHS / refinement kernels
// Right-hand sides enter the solves in the original row order: the forward
// sweep of the solve applies the factor's row swaps panel by panel.

// X = E0 (the first K columns of the identity), complex<R>.
template <typename C>
__global__ void k_rhs_identity(const Unit* __restrict__ units, char* ws, int which, int K, int nrhs) {
  const Unit u = units[blockIdx.y];
  const int n = u.n;
  C* X = reinterpret_cast<C*>(ws + (which == RHS_X ? u.x_off : u.x32_off));
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)n * nrhs;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), c = (int)(idx / n);
    X[idx] = (i == c && c < K) ? cvt<C>(make_double2(1.0, 0.0)) : cvt<C>(make_double2(0.0, 0.0));
  }
}

// X32 = B rounded (mixed form) or X = B (FP64 form); B complex128 at r_off.
__global__ void k_copy_b(const Unit* __restrict__ units, char* ws, int nrhs, bool to_x32) {
  const Unit u = units[blockIdx.y];
  const int n = u.n;
  const double2* B = reinterpret_cast<const double2*>(ws + u.r_off);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)n * nrhs;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const double2 b = B[idx];
    if (to_x32) reinterpret_cast<float2*>(ws + u.x32_off)[idx] = to32(b);
    else reinterpret_cast<double2*>(ws + u.x_off)[idx] = b;
  }
}

// X = X32 widened, its double-float copy (lo parts zero) and the column maxima
// max_i max(|Re X_ic|, |Im X_ic|) for the tensor-core residual.  One CTA per unit.
__global__ void __launch_bounds__(256) k_widen(const Unit* __restrict__ units, char* ws, int nrhs) {
  const Unit u = units[blockIdx.x];
  const int n = u.n;
  const float2* X32 = reinterpret_cast<const float2*>(ws + u.x32_off);
  double2* X = reinterpret_cast<double2*>(ws + u.x_off);
  float4* Xdf = reinterpret_cast<float4*>(ws + u.xdf_off);
  __shared__ unsigned int s_cmax[32];
  const int tid = threadIdx.x;
  if (tid < 32) s_cmax[tid] = 0u;
  __syncthreads();
  for (int c = 0; c < nrhs; ++c) {
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
      const int i = i0 + tid;
      float m = 0.f;
      if (i < n) {
        const size_t idx = (size_t)c * n + i;
        const float2 x = X32[idx];
        X[idx] = to64(x);
        Xdf[idx] = make_float4(x.x, 0.f, x.y, 0.f);
        m = fmaxf(fabsf(x.x), fabsf(x.y));
      }
      m = warp_max_nonneg(m);
      if ((tid & 31) == 0) atomicMax(&s_cmax[c], __float_as_uint(m));
    }
  }
  __syncthreads();
  if (tid < nrhs) reinterpret_cast<float*>(ws + u.xdf_off + colmax_rel_off(n, nrhs))[tid] = __uint_as_float(s_cmax[tid]);
}

// Refinement residual, FP64-accurate, on the FP32 pipes: B - M X with M held as
// (hi, lo) float pairs and X split the same way, products by the FMA two-product
// and sums by two-sum (double-float arithmetic, unit roundoff about 2^-48), in
// paired FP32 instructions (real and imaginary lanes).  Output rounded to
// complex64 into X32 for the correction solve.  grid (ceil(n_max / 64),
// n_units), block 256: 64 rows x NRHS columns, 4 column groups of CPG = NRHS / 4
// columns per thread.  The X tile is staged in shared memory as the two pairs
// each product needs, (x.re, x.im) and (-x.im, x.re), high and low parts.
// XLO = false: X is the widened complex64 first solution (its low parts are
// zero), so the products M.hi X.lo are left out.
template <int NRHS, bool XLO>
__global__ void __launch_bounds__(256, 3) k_residual(const Unit* __restrict__ units, const char* fac_base, char* ws,
                                                     int K, bool explicit_b, const int32_t* __restrict__ done) {
  constexpr int CPG = (NRHS + 3) / 4;
  constexpr int NCOL = 4 * CPG;  // padded column count; columns >= NRHS are zero and never stored
  const Unit u = units[blockIdx.y];
  if (done[u.stat_off]) return;
  const int n = u.n;
  const int row0 = blockIdx.x * 64;
  if (row0 >= n) return;
  const float4* M = reinterpret_cast<const float4*>(fac_base + u.m64_off);  // (re.hi, im.hi, re.lo, im.lo)
  const float4* Xdf = reinterpret_cast<const float4*>(ws + u.xdf_off);       // (re.hi, re.lo, im.hi, im.lo)
  float2* X32 = reinterpret_cast<float2*>(ws + u.x32_off);
  __shared__ float4 sP[32][NCOL + 1], sQ[32][NCOL + 1];  // (x.re, x.im | hi, lo), (-x.im, x.re | hi, lo)
  const int tid = threadIdx.x;
  const int r = tid & 63, cg = tid >> 6;
  const int row = row0 + r;
  const bool live = row < n;
  const float4* Mrow = M + (live ? row : 0);
  float2 s[CPG], t[CPG];
#pragma unroll
  for (int c = 0; c < CPG; ++c) s[c] = t[c] = make_float2(0.f, 0.f);
  auto mac = [&](const float4 m, int jj) {
    const float2 mrh = make_float2(m.x, m.x), mrl = make_float2(m.z, m.z);
    const float2 mih = make_float2(m.y, m.y), mil = make_float2(m.w, m.w);
#pragma unroll
    for (int c = 0; c < CPG; ++c) {
      const float4 P = sP[jj][cg * CPG + c], Q = sQ[jj][cg * CPG + c];
      df2_mac<XLO>(s[c], t[c], mrh, mrl, make_float2(P.x, P.y), make_float2(P.z, P.w));
      df2_mac<XLO>(s[c], t[c], mih, mil, make_float2(Q.x, Q.y), make_float2(Q.z, Q.w));
    }
  };
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int jn = min(32, n - j0);
    __syncthreads();
    for (int idx = tid; idx < 32 * NCOL; idx += 256) {
      const int jj = idx & 31, c = idx >> 5;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (jj < jn && c < NRHS) v = Xdf[(size_t)c * n + j0 + jj];
      sP[jj][c] = make_float4(v.x, v.z, v.y, v.w);
      sQ[jj][c] = make_float4(-v.z, v.x, -v.w, v.y);
    }
    __syncthreads();
    if (live) {
      if (jn == 32) {
#pragma unroll 4
        for (int jj = 0; jj < 32; ++jj) mac(Mrow[(size_t)(j0 + jj) * n], jj);
      } else {
        for (int jj = 0; jj < jn; ++jj) mac(Mrow[(size_t)(j0 + jj) * n], jj);
      }
    }
  }
  if (live) {
    const double2* B = reinterpret_cast<const double2*>(ws + u.r_off);
#pragma unroll
    for (int c = 0; c < CPG; ++c) {
      const int col = cg * CPG + c;
      if (NRHS % 4 != 0 && col >= NRHS) continue;
      double2 b;
      if (explicit_b) b = B[(size_t)col * n + row];
      else b = (row == col && col < K) ? mk(1.0, 0.0) : mk(0.0, 0.0);
      const double re = b.x - ((double)s[c].x + (double)t[c].x);
      const double im = b.y - ((double)s[c].y + (double)t[c].y);
      X32[(size_t)col * n + row] = make_float2((float)re, (float)im);
    }
  }
}

// Probe weights: w_q[c] complex Gaussian (Box-Muller on two uniforms), the
// uniforms from the integer hash "lowbias32" (C. Wellons) of (unit, sweep, q, c,
// draw): a fixed pseudo-random vector per unit and sweep.  Gaussian weights
// make ||D w|| small only with probability ~ the squared ratio, whatever the
// structure of D.
__device__ __forceinline__ uint32_t probe_hash(uint32_t h) {
  h ^= h >> 16;
  h *= 0x7feb352du;
  h ^= h >> 15;
  h *= 0x846ca68bu;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ double2 probe_weight(int64_t unit, int sweep, int q, int c) {
  const uint32_t key = (uint32_t)((((unit * 16 + sweep) * 4 + q) * 64 + c) * 2);
  const double u1 = ((double)probe_hash(key) + 1.0) * 0x1p-32;  // (0, 1]
  const double u2 = (double)probe_hash(key + 1) * 0x1p-32;      // [0, 1)
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  return make_double2(r * cs, r * sn);
}

// X += X32 (the correction); done when ||correction||_F <= tol ||X||_F.  One CTA
// per unit.  Each sweep adds 1 << 8 to the unit's status word (pass count).
// Mixed form: also keeps X's double-float copy and forms the convergence-probe
// inputs y_q = X w_q and (B w)_q for kProbe complex Gaussian vectors w_q (FP64),
// stored as [q][n] (hi, lo) float4 at p_off and [q][n] complex128 after them.
__global__ void __launch_bounds__(256) k_ir_update(const Unit* __restrict__ units, char* ws, int nrhs, int K,
                                                   bool explicit_b, int sweep, double tol, int32_t* done,
                                                   int32_t* stat) {
  const Unit u = units[blockIdx.x];
  if (done[u.stat_off]) return;
  const int n = u.n;
  const float2* D = reinterpret_cast<const float2*>(ws + u.x32_off);
  double2* X = reinterpret_cast<double2*>(ws + u.x_off);
  float4* Xdf = reinterpret_cast<float4*>(ws + u.xdf_off);
  const double2* B = reinterpret_cast<const double2*>(ws + u.r_off);
  float4* Y = reinterpret_cast<float4*>(ws + u.p_off);  // y_q as (hi, lo) pairs
  double2* BW = reinterpret_cast<double2*>(Y + (size_t)kProbe * n);
  // probe weights rounded to complex64 (exact in both products below)
  __shared__ float2 sw[kProbe][32];
  __shared__ unsigned int s_cmax[32];  // column maxima of the high parts of the updated X
  for (int idx = threadIdx.x; idx < kProbe * 32; idx += blockDim.x)
    sw[idx / 32][idx % 32] = to32(probe_weight(u.stat_off, sweep, idx / 32, idx % 32));
  if (threadIdx.x < 32) s_cmax[threadIdx.x] = 0u;
  __syncthreads();
  // the update in FP64 (X is the complex128 solution) and its double-float split;
  // the norms in FP32 (a ratio test), y = X w in double-float on the FP32 pipes,
  // (B w) in FP64
  float dn = 0.f, xn = 0.f;
  for (int i0 = 0; i0 < n; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const bool live = i < n;
    DfAcc y[kProbe];
    double2 bw[kProbe];
#pragma unroll
    for (int q = 0; q < kProbe; ++q) {
      y[q] = df_zero();
      bw[q] = mk(0.0, 0.0);
    }
    // columns in groups of 8: the group's loads are issued together, then used
    for (int c0 = 0; c0 < nrhs; c0 += 8) {
      float2 dv[8];
      double2 xv[8], bv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = c0 + j;
        if (live && c < nrhs) {
          const size_t idx = (size_t)c * n + i;
          dv[j] = D[idx];
          xv[j] = X[idx];
          if (explicit_b) bv[j] = B[idx];
        }
      }
      float cmv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = c0 + j;
        cmv[j] = 0.f;
        if (live && c < nrhs) {
          const size_t idx = (size_t)c * n + i;
          const float2 d32 = dv[j];
          const double2 x = cadd(xv[j], to64(d32));
          X[idx] = x;
          const float4 xs = df_split(x);  // split once here instead of in every residual CTA
          Xdf[idx] = xs;
          cmv[j] = fmaxf(fabsf(xs.x), fabsf(xs.z));
          dn = fmaf(d32.x, d32.x, fmaf(d32.y, d32.y, dn));
          xn = fmaf(xs.x, xs.x, fmaf(xs.z, xs.z, xn));
#pragma unroll
          for (int q = 0; q < kProbe; ++q) {
            const float2 w = sw[q][c & 31];
            dfc_mac(y[q], xs, make_float4(w.x, 0.f, w.y, 0.f));
          }
          if (explicit_b) {
#pragma unroll
            for (int q = 0; q < kProbe; ++q) bw[q] = cfma(bv[j], to64(sw[q][c & 31]), bw[q]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (c0 + j >= nrhs) break;
        const float cm = warp_max_nonneg(cmv[j]);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_cmax[c0 + j], __float_as_uint(cm));
      }
    }
    if (live) {
#pragma unroll
      for (int q = 0; q < kProbe; ++q) {
        // B = E0 (forward): (B w)_i = w_i for i < K
        if (!explicit_b && i < K && i < nrhs) bw[q] = to64(sw[q][i]);
        Y[(size_t)q * n + i] = df_value(y[q]);
        BW[(size_t)q * n + i] = bw[q];
      }
    }
  }
  __shared__ double s1[256], s2[256];
  s1[threadIdx.x] = (double)dn;
  s2[threadIdx.x] = (double)xn;
  __syncthreads();
  if (threadIdx.x < nrhs)
    reinterpret_cast<float*>(ws + u.xdf_off + colmax_rel_off(n, nrhs))[threadIdx.x] =
        __uint_as_float(s_cmax[threadIdx.x]);
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double a = s1[0], b = s2[0];
    atomicAdd(&stat[u.stat_off], 1 << 8);
    if (!isfinite(a) || !isfinite(b)) {
      atomicOr(&stat[u.stat_off], LSMS_UNIT_NONFINITE);
      done[u.stat_off] = 1;
    } else if (a <= tol * tol * b) {
      done[u.stat_off] = 1;
    }
  }
}

// Convergence probe, residual half: r_q = (B w)_q - M y_q for the kProbe vectors
// of k_ir_update, double-float as in k_residual, rounded to complex64 into X32
// columns q = 0..kProbe-1 for the probe correction solve (which permutes them).
// grid (ceil(n_max / 64), n_units), block 256: 64 rows x 4 quarters of each
// 128-column slab of M, the quarters' partial sums added in shared memory.
__global__ void __launch_bounds__(256, 3) k_probe_residual(const Unit* __restrict__ units, const char* fac_base,
                                                           char* ws, const int32_t* __restrict__ done) {
  const Unit u = units[blockIdx.y];
  if (done[u.stat_off]) return;
  const int n = u.n;
  const int row0 = blockIdx.x * 64;
  if (row0 >= n) return;
  const float4* M = reinterpret_cast<const float4*>(fac_base + u.m64_off);  // (re.hi, im.hi, re.lo, im.lo)
  const float4* Y = reinterpret_cast<const float4*>(ws + u.p_off);  // y_q as (re.hi, re.lo, im.hi, im.lo)
  const double2* BW = reinterpret_cast<const double2*>(Y + (size_t)kProbe * n);
  float2* X32 = reinterpret_cast<float2*>(ws + u.x32_off);
  // y staged as the pairs each product needs: (y.re, y.im) and (-y.im, y.re), hi and lo
  __shared__ float4 sP[128][kProbe], sQ[128][kProbe];
  __shared__ float4 sPart[3][kProbe][64];
  const int tid = threadIdx.x;
  const int r = tid & 63, grp = tid >> 6;
  const int row = row0 + r;
  const bool live = row < n;
  const float4* Mrow = M + (live ? row : 0);
  float2 s2[kProbe], t2[kProbe];
#pragma unroll
  for (int q = 0; q < kProbe; ++q) s2[q] = t2[q] = make_float2(0.f, 0.f);
  auto mac = [&](const float4 m, int jj) {
    const float2 mrh = make_float2(m.x, m.x), mrl = make_float2(m.z, m.z);
    const float2 mih = make_float2(m.y, m.y), mil = make_float2(m.w, m.w);
#pragma unroll
    for (int q = 0; q < kProbe; ++q) {
      const float4 P = sP[jj][q], Q = sQ[jj][q];
      df2_mac(s2[q], t2[q], mrh, mrl, make_float2(P.x, P.y), make_float2(P.z, P.w));
      df2_mac(s2[q], t2[q], mih, mil, make_float2(Q.x, Q.y), make_float2(Q.z, Q.w));
    }
  };
  for (int j0 = 0; j0 < n; j0 += 128) {
    const int jn = min(128, n - j0);
    __syncthreads();
    for (int idx = tid; idx < 128 * kProbe; idx += 256) {
      const int jj = idx & 127, q = idx >> 7;
      const float4 v = jj < jn ? Y[(size_t)q * n + j0 + jj] : make_float4(0.f, 0.f, 0.f, 0.f);
      sP[jj][q] = make_float4(v.x, v.z, v.y, v.w);
      sQ[jj][q] = make_float4(-v.z, v.x, -v.w, v.y);
    }
    __syncthreads();
    if (live) {
      const int ja = grp * 32, jb = min(ja + 32, jn);
      if (jb - ja == 32) {
#pragma unroll 4
        for (int jj = ja; jj < ja + 32; ++jj) mac(Mrow[(size_t)(j0 + jj) * n], jj);
      } else {
        for (int jj = ja; jj < jb; ++jj) mac(Mrow[(size_t)(j0 + jj) * n], jj);
      }
    }
  }
  float sr[kProbe], tr[kProbe], si[kProbe], ti[kProbe];
#pragma unroll
  for (int q = 0; q < kProbe; ++q) {
    sr[q] = s2[q].x;
    si[q] = s2[q].y;
    tr[q] = t2[q].x;
    ti[q] = t2[q].y;
  }
  if (grp > 0) {
#pragma unroll
    for (int q = 0; q < kProbe; ++q) sPart[grp - 1][q][r] = make_float4(sr[q], tr[q], si[q], ti[q]);
  }
  __syncthreads();
  if (grp == 0 && live) {
#pragma unroll
    for (int q = 0; q < kProbe; ++q) {
#pragma unroll
      for (int g = 0; g < 3; ++g) {
        const float4 a = sPart[g][q][r];
        df_add(sr[q], tr[q], a.x);
        tr[q] += a.y;
        df_add(si[q], ti[q], a.z);
        ti[q] += a.w;
      }
      const double2 b = BW[(size_t)q * n + row];
      const double re = b.x - ((double)sr[q] + (double)tr[q]);
      const double im = b.y - ((double)si[q] + (double)ti[q]);
      X32[(size_t)q * n + row] = make_float2((float)re, (float)im);
    }
  }
}

// Convergence probe, test half: X32 columns q now hold the corrections d_q that
// the next sweep would add to y_q = X w_q.  The unit is done when
// sum_q ||d_q||^2 <= tol^2 sum_q ||y_q||^2: E||D w||^2 = 2 ||D||_F^2 and
// E||X w||^2 = 2 ||X||_F^2 for complex Gaussian w, so this is the sweep test of
// k_ir_update taken on kProbe random combinations of the columns, pooled (a
// lower-variance estimate than requiring each probe to pass, with about the
// same chance, ~2e-8, of passing a rank-one correction 100x above tol).  Adds
// 1 << 16 to the status word.
__global__ void __launch_bounds__(256) k_probe_check(const Unit* __restrict__ units, const char* ws, double tol,
                                                     int32_t* done, int32_t* stat) {
  const Unit u = units[blockIdx.x];
  if (done[u.stat_off]) return;
  const int n = u.n;
  const float2* D = reinterpret_cast<const float2*>(ws + u.x32_off);
  const float4* Y = reinterpret_cast<const float4*>(ws + u.p_off);  // (hi, lo) pairs
  double dn[kProbe], yn[kProbe];
#pragma unroll
  for (int q = 0; q < kProbe; ++q) dn[q] = yn[q] = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
#pragma unroll
    for (int q = 0; q < kProbe; ++q) {
      const double2 d = to64(D[(size_t)q * n + i]);
      const double2 y = df_join(Y[(size_t)q * n + i]);
      dn[q] += d.x * d.x + d.y * d.y;
      yn[q] += y.x * y.x + y.y * y.y;
    }
  }
  __shared__ double s[2 * kProbe][256];
#pragma unroll
  for (int q = 0; q < kProbe; ++q) {
    s[2 * q][threadIdx.x] = dn[q];
    s[2 * q + 1][threadIdx.x] = yn[q];
  }
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int k = 0; k < 2 * kProbe; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&stat[u.stat_off], 1 << 16);
    double a = 0.0, b = 0.0;
#pragma unroll
    for (int q = 0; q < kProbe; ++q) {
      a += s[2 * q][0];
      b += s[2 * q + 1][0];
    }
    if (isfinite(a) && isfinite(b) && a <= tol * tol * b) done[u.stat_off] = 1;
  }
}

__global__ void k_ir_finish(const Unit* __restrict__ units, int n_units, const int32_t* done, int32_t* stat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_units) return;
  const Unit u = units[i];
  if (!done[u.stat_off]) atomicOr(&stat[u.stat_off], LSMS_UNIT_NOCONV);
}

// tau[e][site_off + p][L][L'] = X[L' * n + K p + L].  grid (S_max, n_units).
// conj_pairs: also tau[e + 1] = conj(tau[e]) (the partner energy conj z_e).
__global__ void k_write_tau(const Unit* __restrict__ units, const char* ws, int K, int64_t S_total, bool conj_pairs,
                            double2* __restrict__ tau) {
  const Unit u = units[blockIdx.y];
  const int p = blockIdx.x;
  if (p >= u.S) return;
  const int tid = threadIdx.x;
  const int L = tid >> 4, Lp = tid & 15;
  if (L >= K || Lp >= K) return;
  const double2* X = reinterpret_cast<const double2*>(ws + u.x_off);
  const double2 x = X[(size_t)Lp * u.n + K * p + L];
  tau[(((size_t)u.energy * S_total) + u.site_off + p) * K * K + L * K + Lp] = x;
  if (conj_pairs) tau[(((size_t)(u.energy + 1) * S_total) + u.site_off + p) * K * K + L * K + Lp] = mk(x.x, -x.y);
}

__global__ void k_status_out(const int32_t* __restrict__ stat, int n, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = stat[i];
}

// Conjugate-pair mode: flag[d] = 1 when some t^{-1} block of energy 2d + 1 is not
// the conjugate of energy 2d's (|b - conj a| > 1e-12 max|a| over the block).
// grid (n_species, n_delta), block 256.
__global__ void k_check_conj_tinv(const double2* __restrict__ tinv, int n_energy, int KK, int32_t* flag) {
  const int s = blockIdx.x, d = blockIdx.y;
  const double2* a = tinv + ((size_t)s * n_energy + 2 * d) * KK;
  const double2* b = a + KK;
  double dm = 0.0, am = 0.0;
  for (int i = threadIdx.x; i < KK; i += blockDim.x) {
    const double2 x = a[i], y = b[i];
    dm = fmax(dm, fabs(y.x - x.x) + fabs(y.y + x.y));
    am = fmax(am, fabs(x.x) + fabs(x.y));
    if (!isfinite(x.x) || !isfinite(x.y) || !isfinite(y.x) || !isfinite(y.y)) dm = INFINITY;
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
  if (threadIdx.x == 0 && !(s1[0] <= 1e-12 * s2[0])) atomicOr(&flag[d], 1);
}

// Conjugate-pair mode, status of the second energy of each pair: stat (its own
// solves in the backward, else the partner's) plus LSMS_UNIT_BAD_INPUT when the
// pair's t^{-1} is not conjugate.  One thread per (pair, atom).
__global__ void k_status_conj(const int32_t* __restrict__ stat, const int32_t* __restrict__ flag, int n_atoms,
                              int n_delta, bool from_partner, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_atoms * n_delta) return;
  const int d = i / n_atoms, m = i % n_atoms;
  const size_t minus = (size_t)(2 * d + 1) * n_atoms + m;
  const int32_t v = from_partner ? stat[(size_t)(2 * d) * n_atoms + m] : stat[minus];
  out[minus] = v | (flag[d] ? LSMS_UNIT_BAD_INPUT : 0);
}

// Conjugate-pair mode (backward): conjugate the n x nrhs complex128 block at
// r_off (which = 0) or x_off (which = 1) of the units solved with their
// partner's factors.  grid (ceil(n_max nrhs / 256), n_units).
__global__ void k_conj_block(const Unit* __restrict__ units, char* ws, int nrhs, int which) {
  const Unit u = units[blockIdx.y];
  if (!u.conj) return;
  double2* X = reinterpret_cast<double2*>(ws + (which == 0 ? u.r_off : u.x_off));
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)u.n * nrhs;
       idx += (int64_t)gridDim.x * blockDim.x)
    X[idx].y = -X[idx].y;
}

// ------------------------------------------------------------------ FP64 fallback (mixed form)
// Flags after which a mixed-form unit is re-solved in the FP64 form: a zero
// pivot or pivot growth in the complex64 factors, a refinement that did not
// converge, or a tensor-core wait that gave up.
constexpr int32_t kRetryFlags = LSMS_UNIT_ZERO_PIVOT | LSMS_UNIT_NOCONV | LSMS_UNIT_GROWTH | LSMS_UNIT_TIMEOUT;

// One warp: the first `slots` units (plan order) carrying a retry flag get a
// fallback slot; their retry flags are cleared and LSMS_UNIT_FP64_FALLBACK set
// (the FP64 kernels then flag whatever they find themselves).  Slot s factors
// at region + s * slot_bytes; unused slots get n = 0 (every kernel skips them).
// *count = the number of units that were given a slot; units beyond the slots
// keep their flags.
__global__ void __launch_bounds__(32) k_fb_select(const Unit* __restrict__ units, int n_units, int32_t* stat,
                                                  int slots, int64_t slot_bytes, int64_t off_piv, int64_t off_x,
                                                  int64_t off_b, Unit* __restrict__ fb, int32_t* count) {
  const int lane = threadIdx.x;
  int cnt = 0;
  for (int i0 = 0; i0 < n_units && cnt < slots; i0 += 32) {
    const int i = i0 + lane;
    Unit u{};
    bool f = false;
    if (i < n_units) {
      u = units[i];
      f = (stat[u.stat_off] & kRetryFlags) != 0;
    }
    const unsigned b = __ballot_sync(0xffffffffu, f);
    const int pos = cnt + __popc(b & ((1u << lane) - 1u));
    if (f && pos < slots) {
      Unit v{};
      v.atom = u.atom;
      v.energy = u.energy;
      v.n = u.n;
      v.S = u.S;
      v.site_off = u.site_off;
      v.stat_off = u.stat_off;
      v.fac_off = (int64_t)pos * slot_bytes;
      v.piv_off = v.fac_off + off_piv;
      v.x_off = v.fac_off + off_x;
      v.r_off = v.fac_off + off_b;
      fb[pos] = v;
      stat[u.stat_off] = (stat[u.stat_off] & ~kRetryFlags) | LSMS_UNIT_FP64_FALLBACK;
    }
    cnt += __popc(b);
  }
  const int used = min(cnt, slots);
  for (int s2 = used + lane; s2 < slots; s2 += 32) {
    Unit v{};
    fb[s2] = v;  // n = 0, S = 0: skipped
  }
  if (lane == 0) *count = used;
}

// ------------------------------------------------------------------ shared driver
struct Call {
  lsms_liz* liz;
  DeviceData* dd;
  int lmax, K, n_species, n_energy, precision;  // precision: LSMS_FP64 or LSMS_MIXED
  bool conj;                                    // LSMS_CONJ_PAIRS given
  const int32_t* species;
  const double2* tinv;
  EnergyTable E;
  cudaStream_t st;
};

static int check_common(const lsms_liz* liz, int lmax, const void* species, int n_species, int n_energy,
                        int precision) {
  if (!liz) return fail(LSMS_ERR_ARG, "NULL liz");
  if (lmax < 0 || lmax > kMaxLmax) return fail(LSMS_ERR_ARG, "lmax must be in 0..%d", kMaxLmax);
  if (!species || n_species < 1) return fail(LSMS_ERR_ARG, "species must be given, n_species >= 1");
  if (n_energy < 1 || n_energy > kMaxEnergies) return fail(LSMS_ERR_ARG, "n_energy must be in 1..%d", kMaxEnergies);
  if (precision != LSMS_FP64 && precision != LSMS_MIXED) return fail(LSMS_ERR_ARG, "unknown precision %d", precision);
  return LSMS_OK;
}

// Assemble + factor the units of one chunk that own factors (at fac_base); the
// mixed form also writes the double-float copy of M.
static int assemble_factor(const Call& c, const Plan& p, const Chunk& ch, char* fac_base, char* ws, int32_t* stat) {
  const NvtxRange range("lsms/assemble+lu");
  const Unit* du = p.d_fac_units + ch.f0;  // the units that own factors
  const int nu = ch.f1 - ch.f0;
  const int S_max = ch.n_max / c.K;
  const int n_at = nu / p.fac_per_atom;  // chunks hold whole atoms
  if (c.precision == LSMS_FP64) {
    LSMS_LAUNCH(k_assemble<false>, dim3(S_max, n_at), dim3(256), 0, c.st, du, p.fac_per_atom, c.dd->disp,
                c.dd->site_atom, c.species, c.tinv, c.n_species, c.n_energy, c.E, c.K, fac_base, ws, true, stat);
    return lu_factor_chunk<double>(du, nu, ch.n_max, fac_base, stat, c.st);
  }
  const dim3 gu((nu + 255) / 256);
  LSMS_LAUNCH(k_growth_init, dim3(nu), dim3(256), 0, c.st, du, nu, fac_base);
  LSMS_LAUNCH(k_assemble<true>, dim3(S_max, n_at), dim3(256), 0, c.st, du, p.fac_per_atom, c.dd->disp,
              c.dd->site_atom, c.species, c.tinv, c.n_species, c.n_energy, c.E, c.K, fac_base, ws, true, stat);
  const int rc = lu_factor_chunk<float>(du, nu, ch.n_max, fac_base, stat, c.st);
  if (rc) return rc;
  LSMS_LAUNCH(k_growth_check, gu, dim3(256), 0, c.st, du, nu, fac_base, (float)opt_growth_limit(), stat);
  return LSMS_OK;
}

// Solve M X = B for a chunk whose factors exist.  B = E0 (forward) or the explicit
// complex128 block at r_off (backward).  Result in X (complex128).
static int solve_refine(const Call& c, const Plan& p, const Chunk& ch, const char* fac_base, char* ws, int32_t* stat,
                        int32_t* done, bool explicit_b) {
  const NvtxRange range("lsms/solve+refine");
  const Unit* du = p.d_units + ch.u0;
  const int nu = ch.u1 - ch.u0;
  const int nrhs = p.nrhs;
  const dim3 g1((ch.n_max * nrhs + 255) / 256, nu);
  int rc;
  if (c.precision == LSMS_FP64) {
    if (explicit_b) LSMS_LAUNCH(k_copy_b, g1, dim3(256), 0, c.st, du, ws, nrhs, false);
    else LSMS_LAUNCH(k_rhs_identity<double2>, g1, dim3(256), 0, c.st, du, ws, (int)RHS_X, c.K, nrhs);
    return lu_solve_chunk<double>(du, nu, ch.n_max, fac_base, ws, RHS_X, nrhs, nullptr, stat, c.st);
  }
  if (explicit_b) LSMS_LAUNCH(k_copy_b, g1, dim3(256), 0, c.st, du, ws, nrhs, true);
  else LSMS_LAUNCH(k_rhs_identity<float2>, g1, dim3(256), 0, c.st, du, ws, (int)RHS_X32, c.K, nrhs);
  if ((rc = lu_solve_chunk<float>(du, nu, ch.n_max, fac_base, ws, RHS_X32, nrhs, nullptr, stat, c.st))) return rc;
  LSMS_LAUNCH(k_widen, dim3(nu), dim3(256), 0, c.st, du, ws, nrhs);
  // done flags of this chunk's units start cleared (memset by the caller)
  const int max_sweeps = opt_ir_max_sweeps();
  // the residual on the tensor cores for 9 or more right-hand sides (lmax >= 2), else double-float SIMT
  const bool tc_resid = opt_residual_tc() && nrhs >= 9;
  for (int it = 0; it < max_sweeps; ++it) {
    const dim3 gr((ch.n_max + 63) / 64, nu);
    if (tc_resid) {
      if ((rc = residual_tc_chunk(du, nu, ch.n_max, fac_base, ws, c.K, nrhs, explicit_b, done, stat, c.st))) return rc;
    } else switch (nrhs) {  // K or 2K for lmax = 0..3
#define LSMS_RESID(NR)                                                                                 \
  case NR:                                                                                             \
    if (it == 0) LSMS_LAUNCH((k_residual<NR, false>), gr, dim3(256), 0, c.st, du, fac_base, ws, c.K, explicit_b, done); \
    else LSMS_LAUNCH((k_residual<NR, true>), gr, dim3(256), 0, c.st, du, fac_base, ws, c.K, explicit_b, done);          \
    break;
      LSMS_RESID(1) LSMS_RESID(2) LSMS_RESID(4) LSMS_RESID(8) LSMS_RESID(9) LSMS_RESID(18) LSMS_RESID(16)
      LSMS_RESID(32)
#undef LSMS_RESID
      default: return fail(LSMS_ERR_ARG, "internal: no residual kernel for %d right-hand sides", nrhs);
    }
    if ((rc = lu_solve_chunk<float>(du, nu, ch.n_max, fac_base, ws, RHS_X32, nrhs, done, stat, c.st))) return rc;
    LSMS_LAUNCH(k_ir_update, dim3(nu), dim3(256), 0, c.st, du, ws, nrhs, c.K, explicit_b, it, kIrTol, done,
                stat);
    // probe: would the next sweep's correction pass the test?  If so, stop here.
    LSMS_LAUNCH(k_probe_residual, gr, dim3(256), 0, c.st, du, fac_base, ws, done);
    if ((rc = lu_solve_chunk<float>(du, nu, ch.n_max, fac_base, ws, RHS_X32, kProbe, done, stat, c.st))) return rc;
    LSMS_LAUNCH(k_probe_check, dim3(nu), dim3(256), 0, c.st, du, ws, kIrTol, done, stat);
  }
  LSMS_LAUNCH(k_ir_finish, dim3((nu + 255) / 256), dim3(256), 0, c.st, du, nu, done, stat);
  return LSMS_OK;
}

// Arguments of the adjoint right-hand sides and site products (backward only).
struct AdjArgs {
  const double2* J;
  int64_t J_dstride;
  const double2* tau;
  const double2* abar;
  int n_delta;
  double2* G;
};

// Re-solve in the FP64 form, on the GPU, the mixed-form units flagged with
// kRetryFlags (at most f.slots of them, in plan order): assemble M in FP64,
// factor, solve, and overwrite that unit's tau blocks (forward, adj == NULL) or
// its per-site gradient blocks (backward).  Runs on c.st after every chunk.
static int fallback_resolve(const Call& c, const Plan& p, char* ws, const WsHeader& h, const FbLayout& f,
                            int32_t* stat, double2* tau_out, const AdjArgs* adj) {
  if (!f.slots || p.units.empty()) return LSMS_OK;
  const NvtxRange range("lsms/fp64-fallback");
  Unit* fbu = reinterpret_cast<Unit*>(ws + h.fb + f.units_off);
  int32_t* cnt = reinterpret_cast<int32_t*>(ws + h.fb + f.count_off);
  char* region = ws + h.fb + f.region_off;
  int n_max = 0;
  for (const Chunk& ch : p.chunks) n_max = std::max(n_max, ch.n_max);
  const int S_max = n_max / c.K;
  const int slots = f.slots;
  const int nrhs = p.nrhs;
  LSMS_LAUNCH(k_fb_select, dim3(1), dim3(32), 0, c.st, p.d_units, (int)p.units.size(), stat, slots,
              (int64_t)f.slot, (int64_t)f.fac, (int64_t)(f.fac + f.piv), (int64_t)(f.fac + f.piv + f.x), fbu, cnt);
  LSMS_LAUNCH(k_assemble<false>, dim3(S_max, slots), dim3(256), 0, c.st, fbu, 1, c.dd->disp, c.dd->site_atom,
              c.species, c.tinv, c.n_species, c.n_energy, c.E, c.K, region, region, true, stat);
  int rc = lu_factor_chunk<double>(fbu, slots, n_max, region, stat, c.st);
  if (rc) return rc;
  const dim3 g1((n_max * nrhs + 255) / 256, slots);
  if (!adj) {
    LSMS_LAUNCH(k_rhs_identity<double2>, g1, dim3(256), 0, c.st, fbu, region, (int)RHS_X, c.K, nrhs);
    if ((rc = lu_solve_chunk<double>(fbu, slots, n_max, region, region, RHS_X, nrhs, nullptr, stat, c.st))) return rc;
    LSMS_LAUNCH(k_write_tau, dim3(S_max, slots), dim3(256), 0, c.st, fbu, region, c.K, c.liz->total_sites, c.conj,
                tau_out);
    return LSMS_OK;
  }
  if ((rc = adj_rhs(fbu, slots, S_max, c.dd->site_atom, c.species, c.n_species, adj->J, adj->J_dstride, adj->tau,
                    c.liz->total_sites, adj->abar, nullptr, 0, nullptr, adj->n_delta, c.K, region, false, c.st)))
    return rc;
  LSMS_LAUNCH(k_copy_b, g1, dim3(256), 0, c.st, fbu, region, nrhs, false);
  if ((rc = lu_solve_chunk<double>(fbu, slots, n_max, region, region, RHS_X, nrhs, nullptr, stat, c.st))) return rc;
  return adj_site(fbu, slots, S_max, adj->tau, c.liz->total_sites, c.K, region, adj->G, false, c.st);
}

// Conjugate-pair mode: n_energy even and z[2d + 1] = conj z[2d] exactly.
static int check_conj_energies(const lsms_complex* z, int n_energy) {
  if (n_energy & 1) return fail(LSMS_ERR_ARG, "LSMS_CONJ_PAIRS needs an even n_energy");
  for (int d = 0; d < n_energy / 2; ++d)
    if (!(z[2 * d + 1].re == z[2 * d].re && z[2 * d + 1].im == -z[2 * d].im))
      return fail(LSMS_ERR_ARG, "LSMS_CONJ_PAIRS: z[%d] is not the conjugate of z[%d]", 2 * d + 1, 2 * d);
  return LSMS_OK;
}

// The parts of a chunk run on concurrent streams: the caller's and side streams
// (per host thread and device), forked and joined by events, which a CUDA-graph
// capture records as edges.  The step is a chain of batched launches whose
// latency-bound phases (panels, interchanges, solves) leave the GPU partly idle;
// the other parts' bandwidth- and compute-bound launches fill it.  Parts hold
// whole atoms and disjoint workspace.  With the kernel timers on, everything
// stays on the caller's stream so that each launch is timed alone.
constexpr int kMaxParts = 4;
struct SideStreams {
  cudaStream_t s[kMaxParts - 1] = {};
  cudaEvent_t fork = nullptr, join[kMaxParts - 1] = {};
};

// Number of concurrent parts per chunk: the "streams" option if set, else the
// environment variable LSMS_STREAMS (1..4, read once), else 4.
static int stream_parts() {
  static const int env_parts = [] {
    const char* e = std::getenv("LSMS_STREAMS");
    const int v = e ? std::atoi(e) : 4;
    return std::min(std::max(v, 1), kMaxParts);
  }();
  const int o = g_opt_streams.load();
  return o > 0 ? std::min(o, kMaxParts) : env_parts;
}

static int side_streams(SideStreams** out) {
  static thread_local SideStreams side[64];  // per host thread: a stream is captured into one graph at a time
  int dev = 0;
  LSMS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(LSMS_ERR_CUDA, "device index %d unsupported", dev);
  SideStreams& ss = side[dev];
  if (!ss.fork) {
    for (int i = 0; i < kMaxParts - 1; ++i) {
      LSMS_CUDA_TRY(cudaStreamCreateWithFlags(&ss.s[i], cudaStreamNonBlocking));
      LSMS_CUDA_TRY(cudaEventCreateWithFlags(&ss.join[i], cudaEventDisableTiming));
    }
    LSMS_CUDA_TRY(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming));
  }
  *out = &ss;
  return LSMS_OK;
}

// Split ch at atom boundaries into up to `want` parts (units and factor units
// are atom-major, with the same number per atom).  Returns the number of parts.
static int split_chunk(const Plan& p, const Chunk& ch, int want, Chunk* part) {
  const int n_at = (ch.f1 - ch.f0) / p.fac_per_atom;
  const int np = std::max(1, std::min(want, n_at));
  const int upa = (ch.u1 - ch.u0) / std::max(n_at, 1);
  for (int i = 0; i < np; ++i) {
    const int a0 = (int)((int64_t)n_at * i / np), a1 = (int)((int64_t)n_at * (i + 1) / np);
    Chunk& c = part[i];
    c = ch;
    c.u0 = ch.u0 + a0 * upa;
    c.u1 = ch.u0 + a1 * upa;
    c.f0 = ch.f0 + a0 * p.fac_per_atom;
    c.f1 = ch.f0 + a1 * p.fac_per_atom;
    c.n_max = 0;
    for (int u = c.u0; u < c.u1; ++u) c.n_max = std::max(c.n_max, p.units[u].n);
  }
  if (np == 1) part[0] = ch;
  return np;
}

// run(chunk, stream) for the parts of ch on concurrent streams, or for ch on c.st.
template <typename F>
static int run_split(const Call& c, const Plan& p, const Chunk& ch, F run) {
  Chunk part[kMaxParts];
  const int np = g_timer_on.load(std::memory_order_relaxed) ? 1 : split_chunk(p, ch, stream_parts(), part);
  if (np == 1) return run(ch, c.st);
  SideStreams* ss = nullptr;
  int rc = side_streams(&ss);
  if (rc) return rc;
  LSMS_CUDA_TRY(cudaEventRecord(ss->fork, c.st));
  for (int i = 1; i < np; ++i) LSMS_CUDA_TRY(cudaStreamWaitEvent(ss->s[i - 1], ss->fork, 0));
  rc = run(part[0], c.st);
  for (int i = 1; i < np && !rc; ++i) rc = run(part[i], ss->s[i - 1]);
  // joined even after an error: no work stays forked from the caller's stream
  for (int i = 1; i < np; ++i) {
    LSMS_CUDA_TRY(cudaEventRecord(ss->join[i - 1], ss->s[i - 1]));
    LSMS_CUDA_TRY(cudaStreamWaitEvent(c.st, ss->join[i - 1], 0));
  }
  return rc;
}

static int begin_call(lsms_liz* liz, const lsms_complex* z, int n_energy, Call* c) {
  for (int e = 0; e < n_energy; ++e) {
    if (!std::isfinite(z[e].re) || !std::isfinite(z[e].im)) return fail(LSMS_ERR_ARG, "energy %d is not finite", e);
    c->E.z[e] = make_double2(z[e].re, z[e].im);
  }
  for (int e = n_energy; e < kMaxEnergies; ++e) c->E.z[e] = make_double2(0.0, 0.0);
  return device_data(liz, &c->dd);
}

}  // namespace lsms

using namespace lsms;

// ------------------------------------------------------------------ C ABI
extern "C" long long lsms_launch_count(void) { return g_launches.load(); }

extern "C" int lsms_set_option(const char* name, double value) {
  clear_error();
  if (!name) return fail(LSMS_ERR_ARG, "lsms_set_option: NULL name");
  const std::string n(name);
  auto in_int = [&](double lo, double hi) { return value >= lo && value <= hi && value == std::floor(value); };
  if (n == "growth_limit") {
    if (!(value > 0.0) || !std::isfinite(value)) return fail(LSMS_ERR_ARG, "growth_limit must be finite and > 0");
    g_opt_growth_limit.store(value);
  } else if (n == "fallback_slots") {
    if (!in_int(0, 4096)) return fail(LSMS_ERR_ARG, "fallback_slots must be an integer in 0..4096");
    g_opt_fallback_slots.store((int)value);
  } else if (n == "ir_max_sweeps") {
    if (!in_int(0, 64)) return fail(LSMS_ERR_ARG, "ir_max_sweeps must be an integer in 0..64");
    g_opt_ir_max_sweeps.store((int)value);
  } else if (n == "streams") {
    if (!in_int(0, kMaxParts)) return fail(LSMS_ERR_ARG, "streams must be an integer in 0..%d", kMaxParts);
    g_opt_streams.store((int)value);
  } else if (n == "residual_tc") {
    if (!in_int(0, 1)) return fail(LSMS_ERR_ARG, "residual_tc must be 0 or 1");
    g_opt_residual_tc.store((int)value);
  } else if (n == "solve_cols") {
    if (!(value == 0 || value == 8 || value == 16 || value == 32))
      return fail(LSMS_ERR_ARG, "solve_cols must be 0, 8, 16 or 32");
    g_opt_solve_cols.store((int)value);
  } else if (n == "solve_regs") {
    if (!in_int(0, 2)) return fail(LSMS_ERR_ARG, "solve_regs must be 0, 1 or 2");
    g_opt_solve_regs.store((int)value);
  } else if (n == "solve_steps") {
    if (!in_int(0, 3)) return fail(LSMS_ERR_ARG, "solve_steps must be 0, 1, 2 or 3");
    g_opt_solve_steps.store((int)value);
  } else if (n == "nvtx") {
    if (!in_int(0, 1)) return fail(LSMS_ERR_ARG, "nvtx must be 0 or 1");
    g_opt_nvtx.store((int)value);
  } else {
    return fail(LSMS_ERR_ARG, "lsms_set_option: unknown option '%s'", name);
  }
  return LSMS_OK;
}

extern "C" int lsms_get_option(const char* name, double* value) {
  clear_error();
  if (!name || !value) return fail(LSMS_ERR_ARG, "lsms_get_option: NULL argument");
  const std::string n(name);
  if (n == "growth_limit") *value = g_opt_growth_limit.load();
  else if (n == "fallback_slots") *value = g_opt_fallback_slots.load();
  else if (n == "ir_max_sweeps") *value = g_opt_ir_max_sweeps.load();
  else if (n == "streams") *value = stream_parts();
  else if (n == "residual_tc") *value = g_opt_residual_tc.load();
  else if (n == "solve_cols") *value = g_opt_solve_cols.load();
  else if (n == "solve_regs") *value = g_opt_solve_regs.load();
  else if (n == "solve_steps") *value = g_opt_solve_steps.load();
  else if (n == "nvtx") *value = g_opt_nvtx.load();
  else return fail(LSMS_ERR_ARG, "lsms_get_option: unknown option '%s'", name);
  return LSMS_OK;
}

extern "C" int lsms_unit_stats(const int32_t* unit_status, int64_t n_words, lsms_stats* stats, void* stream) {
  clear_error();
  if (!stats || n_words < 0 || (!unit_status && n_words > 0))
    return fail(LSMS_ERR_ARG, "lsms_unit_stats: NULL pointer or n < 0");
  if ((reinterpret_cast<uintptr_t>(stats) & 7) != 0) return fail(LSMS_ERR_ARG, "lsms_unit_stats: stats not 8-byte aligned");
  const NvtxRange range("lsms/unit-stats");
  LSMS_LAUNCH(k_unit_stats, dim3(1), dim3(1024), 0, reinterpret_cast<cudaStream_t>(stream), unit_status, n_words,
              stats);
  return LSMS_OK;
}

extern "C" int lsms_kernel_timer_enable(int on) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_timer_mu);
  g_timer_recs.clear();
  g_timer_next = 0;
  g_timer_on.store(on != 0);
  return LSMS_OK;
}

extern "C" int lsms_kernel_timer_report(char* buf, size_t len) {
  clear_error();
  if (!buf || len == 0) return fail(LSMS_ERR_ARG, "lsms_kernel_timer_report: empty buffer");
  std::lock_guard<std::mutex> lk(g_timer_mu);
  std::map<std::string, std::pair<double, long long>> agg;
  for (const TimerRec& r : g_timer_recs) {
    float ms = 0.f;
    if (r.ev + 1 >= (int)g_timer_next) continue;
    if (cudaEventElapsedTime(&ms, g_timer_events[r.ev], g_timer_events[r.ev + 1]) != cudaSuccess) continue;
    auto& a = agg[r.name];
    a.first += ms;
    a.second += 1;
  }
  std::string out;
  char line[512];
  for (auto& kv : agg) {
    snprintf(line, sizeof(line), "%s\t%.6f\t%lld\n", kv.first.c_str(), kv.second.first, kv.second.second);
    out += line;
  }
  if (out.size() + 1 > len) return fail(LSMS_ERR_NOMEM, "lsms_kernel_timer_report: buffer too small");
  std::memcpy(buf, out.c_str(), out.size() + 1);
  return LSMS_OK;
}

extern "C" void lsms_liz_destroy(lsms_liz* liz) {
  if (!liz) return;
  int cur = -1;
  cudaGetDevice(&cur);
  for (auto& kv : liz->dev) {
    if (cudaSetDevice(kv.first) != cudaSuccess) continue;
    DeviceData& d = kv.second;
    cudaFree(d.block);
    for (auto& pk : d.plans) cudaFree(pk.second.d_block);
  }
  if (cur >= 0) cudaSetDevice(cur);
  delete liz;
}

// Workspace of one atom's units (factors in the workspace, i.e. no store):
// largest over atoms and total.
static size_t unit_ws_max_sum(const lsms_liz* liz, int lmax, int n_energy, int precision, int nrhs, bool backward,
                              bool conj, bool store, size_t* sum) {
  const int K = (lmax + 1) * (lmax + 1);
  std::vector<int> es;
  std::vector<char> owns;
  plan_energies(n_energy, conj, backward, &es, &owns);
  size_t mx = 0, s = 0;
  for (int m = 0; m < liz->n_atoms; ++m) {
    const int n = K * (int)(liz->offsets[m + 1] - liz->offsets[m]);
    const UnitBytes ub = unit_bytes(n, precision, nrhs, backward);
    size_t b = 0;
    for (size_t i = 0; i < es.size(); ++i) b += ws_unit_bytes(ub, owns[i] && !store);
    mx = std::max(mx, b);
    s += b;
  }
  *sum = s;
  return mx;
}

// Precision argument: LSMS_FP64 or LSMS_MIXED, optionally with LSMS_CONJ_PAIRS.
static bool split_precision(int precision, int* base, bool* conj) {
  *base = precision & ~LSMS_CONJ_PAIRS;
  *conj = (precision & LSMS_CONJ_PAIRS) != 0;
  return *base == LSMS_FP64 || *base == LSMS_MIXED;
}
// The workspace-size functions also take LSMS_WS_STORE (factors kept in lu_store).
static bool split_precision_ws(int precision, int* base, bool* conj, bool* store) {
  *store = (precision & LSMS_WS_STORE) != 0;
  return split_precision(precision & ~LSMS_WS_STORE, base, conj);
}

extern "C" int lsms_tau_workspace_bytes(const lsms_liz* liz, int lmax, int n_energy, int precision, size_t* min_bytes,
                                        size_t* all_bytes) {
  clear_error();
  int base;
  bool conj, store;
  if (!liz || lmax < 0 || lmax > kMaxLmax || n_energy < 1 || n_energy > kMaxEnergies ||
      !split_precision_ws(precision, &base, &conj, &store) || (conj && (n_energy & 1)))
    return fail(LSMS_ERR_ARG, "lsms_tau_workspace_bytes: bad arguments");
  const int K = (lmax + 1) * (lmax + 1);
  size_t sum = 0;
  const size_t mx = unit_ws_max_sum(liz, lmax, n_energy, base, K, false, conj, store, &sum);
  const WsHeader h =
      ws_header(liz, n_energy, conj_extra_bytes(n_energy), fb_layout(liz, lmax, base, K, false).total);
  if (min_bytes) *min_bytes = h.total_fixed + mx;
  if (all_bytes) *all_bytes = h.total_fixed + sum;
  return LSMS_OK;
}

extern "C" int lsms_backward_workspace_bytes(const lsms_liz* liz, int lmax, int n_energy, int precision,
                                             size_t* min_bytes, size_t* all_bytes) {
  clear_error();
  int base;
  bool conj, store;
  if (!liz || lmax < 0 || lmax > kMaxLmax || n_energy < 2 || n_energy > kMaxEnergies || (n_energy & 1) ||
      !split_precision_ws(precision, &base, &conj, &store))
    return fail(LSMS_ERR_ARG, "lsms_backward_workspace_bytes: bad arguments");
  const int K = (lmax + 1) * (lmax + 1);
  size_t sum = 0;
  const size_t mx = unit_ws_max_sum(liz, lmax, n_energy, base, 2 * K, true, conj, store, &sum);
  const WsHeader h = ws_header(liz, n_energy, backward_extra_bytes(liz, lmax, n_energy) + conj_extra_bytes(n_energy),
                               fb_layout(liz, lmax, base, 2 * K, true).total);
  if (min_bytes) *min_bytes = h.total_fixed + mx;
  if (all_bytes) *all_bytes = h.total_fixed + sum;
  return LSMS_OK;
}

extern "C" int lsms_lu_store_bytes(const lsms_liz* liz, int lmax, int n_energy, int precision, size_t* bytes) {
  clear_error();
  int base;
  bool conj;
  if (!liz || !bytes || lmax < 0 || lmax > kMaxLmax || n_energy < 1 || n_energy > kMaxEnergies ||
      !split_precision(precision, &base, &conj) || (conj && (n_energy & 1)))
    return fail(LSMS_ERR_ARG, "lsms_lu_store_bytes: bad arguments");
  const int K = (lmax + 1) * (lmax + 1);
  const int n_fac = conj ? n_energy / 2 : n_energy;  // factored energies per atom
  size_t s = 0;
  for (int m = 0; m < liz->n_atoms; ++m) {
    const int n = K * (int)(liz->offsets[m + 1] - liz->offsets[m]);
    const UnitBytes ub = unit_bytes(n, base, K, false);
    s += (ub.fac + ub.piv + ub.m64) * n_fac;
  }
  *bytes = s;
  return LSMS_OK;
}

static const size_t kDefaultChunkBudget = (size_t)8 << 30;

extern "C" int lsms_tau_blocks(const lsms_liz* liz_c, int lmax, const int32_t* species, int n_species,
                               const lsms_complex* tinv, const lsms_complex* z, int n_energy, int precision,
                               lsms_complex* tau, int32_t* unit_status, void* workspace, size_t workspace_bytes,
                               void* lu_store, size_t lu_store_bytes, void* stream) {
  clear_error();
  lsms_liz* liz = const_cast<lsms_liz*>(liz_c);
  int base;
  bool conj;
  if (!split_precision(precision, &base, &conj)) return fail(LSMS_ERR_ARG, "unknown precision %d", precision);
  int rc = check_common(liz, lmax, species, n_species, n_energy, base);
  if (rc) return rc;
  if (!tinv || !z || !tau) return fail(LSMS_ERR_ARG, "lsms_tau_blocks: tinv, z and tau are required");
  if (conj && (rc = check_conj_energies(z, n_energy))) return rc;
  Call c{};
  c.liz = liz;
  c.lmax = lmax;
  c.K = (lmax + 1) * (lmax + 1);
  c.n_species = n_species;
  c.n_energy = n_energy;
  c.precision = base;
  c.conj = conj;
  c.species = species;
  c.tinv = reinterpret_cast<const double2*>(tinv);
  c.st = reinterpret_cast<cudaStream_t>(stream);
  if ((rc = begin_call(liz, z, n_energy, &c))) return rc;
  size_t need_store = 0;
  if (lu_store) {
    if ((rc = lsms_lu_store_bytes(liz, lmax, n_energy, precision, &need_store))) return rc;
    if (reinterpret_cast<uintptr_t>(lu_store) % kAlign)
      return fail(LSMS_ERR_ARG, "lu_store must be %d-byte aligned", (int)kAlign);
    if (lu_store_bytes < need_store)
      return fail(LSMS_ERR_NOMEM, "lu_store holds %zu bytes, %zu needed", lu_store_bytes, need_store);
  }
  const bool store = lu_store != nullptr;
  size_t min_b = 0, all_b = 0;
  lsms_tau_workspace_bytes(liz, lmax, n_energy, precision | (store ? LSMS_WS_STORE : 0), &min_b, &all_b);
  const FbLayout fb = fb_layout(liz, lmax, base, c.K, false);
  const WsHeader h = ws_header(liz, n_energy, conj_extra_bytes(n_energy), fb.total);
  char* ws = static_cast<char*>(workspace);
  bool own = false;
  size_t ws_bytes = workspace_bytes;
  if (!ws) {
    ws_bytes = std::min(all_b, std::max(min_b, kDefaultChunkBudget));
    LSMS_CUDA_TRY(cudaMallocAsync((void**)&ws, ws_bytes, c.st));
    own = true;
  } else if (ws_bytes < min_b) {
    return fail(LSMS_ERR_NOMEM, "workspace holds %zu bytes, at least %zu needed", ws_bytes, min_b);
  } else if (reinterpret_cast<uintptr_t>(ws) % kAlign) {
    return fail(LSMS_ERR_ARG, "workspace must be %d-byte aligned", (int)kAlign);
  }
  Plan* p = nullptr;
  if ((rc = get_plan(liz, c.dd, lmax, n_energy, base, c.K, false, store, conj, ws_bytes - h.total_fixed, &p))) {
    if (own) cudaFreeAsync(ws, c.st);
    return rc;
  }
  int32_t* stat = reinterpret_cast<int32_t*>(ws + h.stat);
  int32_t* done = reinterpret_cast<int32_t*>(ws + h.done);
  const size_t nu_all = (size_t)liz->n_atoms * n_energy;
  int32_t* conj_flag = reinterpret_cast<int32_t*>(ws + h.extra);
  rc = [&]() -> int {
    LSMS_CUDA_TRY(cudaMemsetAsync(stat, 0, nu_all * 4, c.st));
    LSMS_CUDA_TRY(cudaMemsetAsync(done, 0, nu_all * 4, c.st));
    if (conj) {
      LSMS_CUDA_TRY(cudaMemsetAsync(conj_flag, 0, conj_extra_bytes(n_energy), c.st));
      LSMS_LAUNCH(k_check_conj_tinv, dim3(n_species, n_energy / 2), dim3(256), 0, c.st, c.tinv, n_energy,
                  c.K * c.K, conj_flag);
    }
    char* chunk = ws + h.chunk;
    char* fac_base = store ? static_cast<char*>(lu_store) : chunk;
    for (const Chunk& whole : p->chunks) {
      int r2 = run_split(c, *p, whole, [&](const Chunk& ch, cudaStream_t st) -> int {
        Call cs = c;
        cs.st = st;
        int r3 = assemble_factor(cs, *p, ch, fac_base, chunk, stat);
        if (r3) return r3;
        if ((r3 = solve_refine(cs, *p, ch, fac_base, chunk, stat, done, false))) return r3;
        LSMS_LAUNCH(k_write_tau, dim3(ch.n_max / c.K, ch.u1 - ch.u0), dim3(256), 0, st, p->d_units + ch.u0, chunk,
                    c.K, liz->total_sites, conj, reinterpret_cast<double2*>(tau));
        return LSMS_OK;
      });
      if (r2) return r2;
    }
    if (base == LSMS_MIXED) {
      const int r2 = fallback_resolve(c, *p, ws, h, fb, stat, reinterpret_cast<double2*>(tau), nullptr);
      if (r2) return r2;
    }
    if (unit_status) {
      LSMS_LAUNCH(k_status_out, dim3((unsigned)((nu_all + 255) / 256)), dim3(256), 0, c.st, stat, (int)nu_all,
                  unit_status);
      if (conj)
        LSMS_LAUNCH(k_status_conj, dim3((unsigned)((nu_all / 2 + 255) / 256)), dim3(256), 0, c.st, stat, conj_flag,
                    liz->n_atoms, n_energy / 2, true, unit_status);
    }
    return LSMS_OK;
  }();
  if (own) cudaFreeAsync(ws, c.st);
  return rc;
}

extern "C" int lsms_kubo_sigma(const lsms_liz* liz_c, int lmax, const int32_t* species, int n_species,
                               const lsms_complex* J, int64_t J_delta_stride, const lsms_complex* tau, int n_delta,
                               double volume, int precision, lsms_complex* sigma_tilde, lsms_complex* sigma,
                               double* rho, void* stream) {
  clear_error();
  lsms_liz* liz = const_cast<lsms_liz*>(liz_c);
  const bool conj = (precision & LSMS_CONJ_PAIRS) != 0;  // halve the traces when J allows (checked on the device)
  precision &= ~LSMS_CONJ_PAIRS;
  int rc = check_common(liz, lmax, species, n_species, 2 * std::max(n_delta, 1), precision);
  if (rc) return rc;
  if (n_delta < 1 || !J || !tau || !sigma) return fail(LSMS_ERR_ARG, "lsms_kubo_sigma: J, tau, sigma required, n_delta >= 1");
  if (!(volume > 0.0) || !std::isfinite(volume)) return fail(LSMS_ERR_ARG, "lsms_kubo_sigma: volume must be > 0");
  if (J_delta_stride < 0) return fail(LSMS_ERR_ARG, "lsms_kubo_sigma: negative J stride");
  DeviceData* dd = nullptr;
  if ((rc = device_data(liz, &dd))) return rc;
  const int K = (lmax + 1) * (lmax + 1);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t part_bytes = align_up((size_t)n_delta * 4 * liz->n_atoms * 9 * 16);
  const size_t s_bytes = align_up((size_t)n_delta * 36 * 16);
  const size_t jdf_bytes = precision == LSMS_MIXED ? jdf_scratch_bytes(n_species, K, n_delta, J_delta_stride) : 0;
  char* scratch = nullptr;
  LSMS_CUDA_TRY(cudaMallocAsync((void**)&scratch, part_bytes + s_bytes + jdf_bytes + kAlign, st));
  const NvtxRange range("lsms/traces");
  rc = kubo_forward(dd->offsets, dd->site_atom, species, n_species, reinterpret_cast<const double2*>(J), J_delta_stride,
                    reinterpret_cast<const double2*>(tau), liz->total_sites, K, liz->n_atoms, n_delta, volume,
                    precision == LSMS_MIXED, reinterpret_cast<float4*>(scratch + part_bytes + s_bytes),
                    reinterpret_cast<double2*>(scratch), reinterpret_cast<double2*>(scratch + part_bytes),
                    reinterpret_cast<double2*>(sigma_tilde), reinterpret_cast<double2*>(sigma), rho, st,
                    conj ? reinterpret_cast<int32_t*>(scratch + part_bytes + s_bytes + jdf_bytes) : nullptr);
  cudaFreeAsync(scratch, st);
  return rc;
}

extern "C" int lsms_kubo_sigma_atoms(const lsms_liz* liz_c, int lmax, const int32_t* species, int n_species,
                                     const lsms_complex* J, int64_t J_delta_stride, const lsms_complex* tau,
                                     int n_delta, double volume, int precision, lsms_complex* sigma_tilde_atoms,
                                     void* stream) {
  clear_error();
  lsms_liz* liz = const_cast<lsms_liz*>(liz_c);
  int rc = check_common(liz, lmax, species, n_species, 2 * std::max(n_delta, 1), precision);
  if (rc) return rc;
  if (n_delta < 1 || !J || !tau || !sigma_tilde_atoms)
    return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_atoms: J, tau, sigma_tilde_atoms required, n_delta >= 1");
  if (!(volume > 0.0) || !std::isfinite(volume)) return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_atoms: volume must be > 0");
  if (J_delta_stride < 0) return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_atoms: negative J stride");
  DeviceData* dd = nullptr;
  if ((rc = device_data(liz, &dd))) return rc;
  const int K = (lmax + 1) * (lmax + 1);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  float4* jdf = nullptr;
  if (precision == LSMS_MIXED)
    LSMS_CUDA_TRY(cudaMallocAsync((void**)&jdf, jdf_scratch_bytes(n_species, K, n_delta, J_delta_stride), st));
  rc = kubo_atoms(dd->offsets, dd->site_atom, species, n_species, reinterpret_cast<const double2*>(J), J_delta_stride,
                  reinterpret_cast<const double2*>(tau), liz->total_sites, K, liz->n_atoms, n_delta, volume,
                  precision == LSMS_MIXED, jdf, reinterpret_cast<double2*>(sigma_tilde_atoms), st);
  if (jdf) cudaFreeAsync(jdf, st);
  return rc;
}

extern "C" int lsms_kubo_sigma_backward(const lsms_liz* liz_c, int lmax, const int32_t* species, int n_species,
                                        const lsms_complex* tinv, const lsms_complex* z, int n_energy, int precision,
                                        const lsms_complex* J, int64_t J_delta_stride, const lsms_complex* tau,
                                        double volume, const lsms_complex* grad_sigma, const void* lu_store,
                                        size_t lu_store_bytes, lsms_complex* grad_tinv,
                                        lsms_complex* grad_tinv_species, int32_t* unit_status,
                                        void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  lsms_liz* liz = const_cast<lsms_liz*>(liz_c);
  int base;
  bool conj;
  if (!split_precision(precision, &base, &conj)) return fail(LSMS_ERR_ARG, "unknown precision %d", precision);
  int rc = check_common(liz, lmax, species, n_species, n_energy, base);
  if (rc) return rc;
  if ((n_energy & 1) || !tinv || !z || !J || !tau || !grad_sigma || !grad_tinv)
    return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_backward: missing argument or odd n_energy");
  if (!(volume > 0.0)) return fail(LSMS_ERR_ARG, "lsms_kubo_sigma_backward: volume must be > 0");
  if (conj && (rc = check_conj_energies(z, n_energy))) return rc;
  Call c{};
  c.liz = liz;
  c.lmax = lmax;
  c.K = (lmax + 1) * (lmax + 1);
  c.n_species = n_species;
  c.n_energy = n_energy;
  c.precision = base;
  c.conj = conj;
  c.species = species;
  c.tinv = reinterpret_cast<const double2*>(tinv);
  c.st = reinterpret_cast<cudaStream_t>(stream);
  if ((rc = begin_call(liz, z, n_energy, &c))) return rc;
  const bool store = lu_store != nullptr;
  if (store) {
    size_t need = 0;
    if ((rc = lsms_lu_store_bytes(liz, lmax, n_energy, precision, &need))) return rc;
    if (reinterpret_cast<uintptr_t>(lu_store) % kAlign)
      return fail(LSMS_ERR_ARG, "lu_store must be %d-byte aligned", (int)kAlign);
    if (lu_store_bytes < need) return fail(LSMS_ERR_NOMEM, "lu_store holds %zu bytes, %zu needed", lu_store_bytes, need);
  }
  const int n_delta = n_energy / 2;
  const size_t KK = (size_t)c.K * c.K;
  size_t min_b = 0, all_b = 0;
  lsms_backward_workspace_bytes(liz, lmax, n_energy, precision | (store ? LSMS_WS_STORE : 0), &min_b, &all_b);
  const FbLayout fb = fb_layout(liz, lmax, base, 2 * c.K, true);
  const WsHeader h = ws_header(liz, n_energy, backward_extra_bytes(liz, lmax, n_energy) + conj_extra_bytes(n_energy),
                               fb.total);
  char* ws = static_cast<char*>(workspace);
  bool own = false;
  size_t ws_bytes = workspace_bytes;
  if (!ws) {
    ws_bytes = std::min(all_b, std::max(min_b, kDefaultChunkBudget));
    LSMS_CUDA_TRY(cudaMallocAsync((void**)&ws, ws_bytes, c.st));
    own = true;
  } else if (ws_bytes < min_b) {
    return fail(LSMS_ERR_NOMEM, "workspace holds %zu bytes, at least %zu needed", ws_bytes, min_b);
  } else if (reinterpret_cast<uintptr_t>(ws) % kAlign) {
    return fail(LSMS_ERR_ARG, "workspace must be %d-byte aligned", (int)kAlign);
  }
  Plan* p = nullptr;
  if ((rc = get_plan(liz, c.dd, lmax, n_energy, base, 2 * c.K, true, store, conj, ws_bytes - h.total_fixed, &p))) {
    if (own) cudaFreeAsync(ws, c.st);
    return rc;
  }
  int32_t* stat = reinterpret_cast<int32_t*>(ws + h.stat);
  int32_t* done = reinterpret_cast<int32_t*>(ws + h.done);
  const size_t abar_bytes = align_up((size_t)liz->n_atoms * n_delta * 12 * KK * 16);
  double2* abar = reinterpret_cast<double2*>(ws + h.extra);
  double2* G = reinterpret_cast<double2*>(ws + h.extra + abar_bytes);
  float4* abar_df = reinterpret_cast<float4*>(ws + h.extra + abar_bytes +
                                              align_up((size_t)n_energy * liz->total_sites * KK * 16));
  int32_t* conj_flag = reinterpret_cast<int32_t*>(ws + h.extra + backward_extra_bytes(liz, lmax, n_energy));
  const bool df = base == LSMS_MIXED;
  float4* jdf = nullptr;  // J as double-float pairs (mixed form), stream-ordered scratch
  int64_t jdf_dstride = 0;
  if (df) {
    const cudaError_t e = cudaMallocAsync((void**)&jdf, jdf_scratch_bytes(n_species, c.K, n_delta, J_delta_stride), c.st);
    if (e != cudaSuccess) {
      if (own) cudaFreeAsync(ws, c.st);
      return fail(LSMS_ERR_NOMEM, "lsms_kubo_sigma_backward: %s", cudaGetErrorString(e));
    }
  }
  const size_t nu_all = (size_t)liz->n_atoms * n_energy;
  rc = [&]() -> int {
    LSMS_CUDA_TRY(cudaMemsetAsync(stat, 0, nu_all * 4, c.st));
    LSMS_CUDA_TRY(cudaMemsetAsync(done, 0, nu_all * 4, c.st));
    if (conj) {
      LSMS_CUDA_TRY(cudaMemsetAsync(conj_flag, 0, conj_extra_bytes(n_energy), c.st));
      LSMS_LAUNCH(k_check_conj_tinv, dim3(n_species, n_energy / 2), dim3(256), 0, c.st, c.tinv, n_energy,
                  c.K * c.K, conj_flag);
    }
    int r2 = adj_abar(species, n_species, reinterpret_cast<const double2*>(J), J_delta_stride,
                      reinterpret_cast<const double2*>(grad_sigma), c.K, volume, liz->n_atoms, n_delta, abar,
                      df ? abar_df : nullptr, c.st);
    if (r2) return r2;
    if (df && (r2 = split_j(reinterpret_cast<const double2*>(J), J_delta_stride, n_species, c.K, n_delta, jdf,
                            &jdf_dstride, c.st)))
      return r2;
    char* chunk = ws + h.chunk;
    char* fac_base = store ? const_cast<char*>(static_cast<const char*>(lu_store)) : chunk;
    for (const Chunk& whole : p->chunks) {
      r2 = run_split(c, *p, whole, [&](const Chunk& ch, cudaStream_t st) -> int {
        Call cs = c;
        cs.st = st;
        const Unit* du = p->d_units + ch.u0;
        const int nu = ch.u1 - ch.u0;
        const int S_max = ch.n_max / c.K;
        int r3;
        // stored factors come with the double-float copy of M (mixed form): nothing to rebuild,
        // but their pivot-growth record is checked again for this call's status
        if (!store && (r3 = assemble_factor(cs, *p, ch, fac_base, chunk, stat))) return r3;
        if (store && df) {
          const int nf = ch.f1 - ch.f0;
          LSMS_LAUNCH(k_growth_check, dim3((nf + 255) / 256), dim3(256), 0, st, p->d_fac_units + ch.f0, nf, fac_base,
                      (float)opt_growth_limit(), stat);
        }
        {
          const NvtxRange range("lsms/adjoint-rhs");
          if ((r3 = adj_rhs(du, nu, S_max, c.dd->site_atom, species, n_species, reinterpret_cast<const double2*>(J),
                            J_delta_stride, reinterpret_cast<const double2*>(tau), liz->total_sites, abar, jdf,
                            jdf_dstride, abar_df, n_delta, c.K, chunk, df, st)))
            return r3;
        }
        const dim3 gc((ch.n_max * p->nrhs + 255) / 256, nu);
        // second energy of a conjugate pair: M(conj z) = conj M(z), so X = conj(M(z)^-1 conj B)
        if (conj) LSMS_LAUNCH(k_conj_block, gc, dim3(256), 0, st, du, chunk, p->nrhs, 0);
        if ((r3 = solve_refine(cs, *p, ch, fac_base, chunk, stat, done, true))) return r3;
        if (conj) LSMS_LAUNCH(k_conj_block, gc, dim3(256), 0, st, du, chunk, p->nrhs, 1);
        const NvtxRange range("lsms/adjoint-site");
        return adj_site(du, nu, S_max, reinterpret_cast<const double2*>(tau), liz->total_sites, c.K, chunk, G,
                        precision == LSMS_MIXED, st);
      });
      if (r2) return r2;
    }
    if (df) {
      const AdjArgs aa{reinterpret_cast<const double2*>(J), J_delta_stride, reinterpret_cast<const double2*>(tau),
                       abar, n_delta, G};
      if ((r2 = fallback_resolve(c, *p, ws, h, fb, stat, nullptr, &aa))) return r2;
    }
    if ((r2 = adj_reduce(c.dd->inv_off, c.dd->inv_sites, G, liz->total_sites, c.K, liz->n_atoms, n_energy,
                         reinterpret_cast<double2*>(grad_tinv), c.st)))
      return r2;
    if (unit_status) {
      LSMS_LAUNCH(k_status_out, dim3((unsigned)((nu_all + 255) / 256)), dim3(256), 0, c.st, stat, (int)nu_all,
                  unit_status);
      if (conj)
        LSMS_LAUNCH(k_status_conj, dim3((unsigned)((nu_all / 2 + 255) / 256)), dim3(256), 0, c.st, stat, conj_flag,
                    liz->n_atoms, n_delta, false, unit_status);
    }
    if (grad_tinv_species)
      return adj_species(species, reinterpret_cast<const double2*>(grad_tinv), c.K, liz->n_atoms, n_species, n_energy,
                         reinterpret_cast<double2*>(grad_tinv_species), c.st);
    return LSMS_OK;
  }();
  if (jdf) cudaFreeAsync(jdf, c.st);
  if (own) cudaFreeAsync(ws, c.st);
  return rc;
}
