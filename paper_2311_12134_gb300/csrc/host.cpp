// Host side of liblsmskubo: errors, the LIZ builder, and the angular tables
// (real Gaunt coefficients from the Wigner 3j closed form, the sparse coupling
// table of the free-electron propagator, Y_L normalisations, the dipole
// current-matrix model).  Plain C++17; no architecture-specific code.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>

#include "internal.h"

namespace lsms {

static thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

void clear_error() { g_last_error.clear(); }

// ---------------------------------------------------------------- angular tables
static double fact(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// Wigner 3j symbol (j1 j2 j3; m1 m2 m3) for integer arguments, Racah's formula.
static double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  const double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
  const double pre = std::sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) *
                               fact(j3 + m3) * fact(j3 - m3));
  const int kmin = std::max({0, j2 - j3 - m1, j1 - j3 + m2});
  const int kmax = std::min({j1 + j2 - j3, j1 - m1, j2 + m2});
  double s = 0.0;
  for (int k = kmin; k <= kmax; ++k) {
    const double den = fact(k) * fact(j3 - j2 + k + m1) * fact(j3 - j1 + k - m2) * fact(j1 + j2 - j3 - k) *
                       fact(j1 - k - m1) * fact(j2 - k + m2);
    s += ((k & 1) ? -1.0 : 1.0) / den;
  }
  const int ph = j1 - j2 - m3;
  return ((ph % 2 + 2) % 2 ? -1.0 : 1.0) * pre * s;
}

// Integral of three complex harmonics (Condon-Shortley phase) over the sphere.
static double gaunt_complex(int l1, int l2, int l3, int m1, int m2, int m3) {
  const double w0 = wigner3j(l1, l2, l3, 0, 0, 0);
  if (w0 == 0.0) return 0.0;
  return std::sqrt((2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / (4.0 * M_PI)) * w0 *
         wigner3j(l1, l2, l3, m1, m2, m3);
}

// Real harmonic without the Condon-Shortley phase in terms of complex ones:
// Y_{l,mu} = sum_m U[mu][m] Y_l^m.
using cd = std::complex<double>;
static void real_from_complex(int l, int mu, cd u[2], int m[2], int* cnt) {
  const double s = 1.0 / std::sqrt(2.0);
  if (mu > 0) {
    m[0] = mu; u[0] = cd((mu & 1) ? -s : s, 0.0);
    m[1] = -mu; u[1] = cd(s, 0.0);
    *cnt = 2;
  } else if (mu < 0) {
    const int a = -mu;
    // ((-1)^a Y^a - Y^{-a}) / (sqrt2 i)
    m[0] = a; u[0] = cd((a & 1) ? -s : s, 0.0) / cd(0.0, 1.0);
    m[1] = -a; u[1] = cd(-s, 0.0) / cd(0.0, 1.0);
    *cnt = 2;
  } else {
    m[0] = 0; u[0] = cd(1.0, 0.0);
    *cnt = 1;
  }
  (void)l;
}

std::vector<double> gaunt_real(int lmax) {
  const int K = (lmax + 1) * (lmax + 1);
  const int l3max = 2 * lmax;
  const int K3 = (l3max + 1) * (l3max + 1);
  std::vector<double> C((size_t)K * K * K3, 0.0);
  for (int l1 = 0; l1 <= lmax; ++l1)
    for (int mu1 = -l1; mu1 <= l1; ++mu1)
      for (int l2 = 0; l2 <= lmax; ++l2)
        for (int mu2 = -l2; mu2 <= l2; ++mu2)
          for (int l3 = 0; l3 <= l3max; ++l3)
            for (int mu3 = -l3; mu3 <= l3; ++mu3) {
              if ((l1 + l2 + l3) & 1) continue;
              if (l3 < std::abs(l1 - l2) || l3 > l1 + l2) continue;
              cd u1[2], u2[2], u3[2];
              int m1[2], m2[2], m3[2], c1, c2, c3;
              real_from_complex(l1, mu1, u1, m1, &c1);
              real_from_complex(l2, mu2, u2, m2, &c2);
              real_from_complex(l3, mu3, u3, m3, &c3);
              cd acc(0.0, 0.0);
              for (int a = 0; a < c1; ++a)
                for (int b = 0; b < c2; ++b)
                  for (int c = 0; c < c3; ++c)
                    if (m1[a] + m2[b] + m3[c] == 0)
                      acc += u1[a] * u2[b] * u3[c] * gaunt_complex(l1, l2, l3, m1[a], m2[b], m3[c]);
              double v = acc.real();
              if (std::fabs(v) < 1e-15) v = 0.0;
              const int L1 = l1 * l1 + l1 + mu1, L2 = l2 * l2 + l2 + mu2, L3 = l3 * l3 + l3 + mu3;
              C[((size_t)L1 * K + L2) * K3 + L3] = v;
            }
  return C;
}

static int l_of(int L) {
  int l = 0;
  while ((l + 1) * (l + 1) <= L) ++l;
  return l;
}

Coupling g_coupling(int lmax) {
  const int K = (lmax + 1) * (lmax + 1);
  const int K3 = (2 * lmax + 1) * (2 * lmax + 1);
  const std::vector<double> C = gaunt_real(lmax);
  Coupling cp;
  cp.start.assign(K * K + 1, 0);
  for (int L = 0; L < K; ++L)
    for (int Lp = 0; Lp < K; ++Lp) {
      for (int L3 = 0; L3 < K3; ++L3) {
        const double c = C[((size_t)L * K + Lp) * K3 + L3];
        if (c == 0.0) continue;
        const int e = l_of(L) - l_of(Lp) - l_of(L3);  // even when c != 0
        const double s = (((e / 2) % 2) == 0) ? 1.0 : -1.0;
        cp.lpp.push_back(L3);
        cp.coef.push_back(s * c);
      }
      cp.start[L * K + Lp + 1] = (int32_t)cp.lpp.size();
    }
  return cp;
}

std::vector<double> ylm_norm(int l3max) {
  std::vector<double> nrm((l3max + 1) * (l3max + 1));
  for (int l = 0; l <= l3max; ++l)
    for (int m = -l; m <= l; ++m) {
      const int am = std::abs(m);
      double v = std::sqrt((2 * l + 1) / (4.0 * M_PI) * fact(l - am) / fact(l + am));
      if (m != 0) v *= std::sqrt(2.0);
      nrm[l * l + l + m] = v;
    }
  return nrm;
}

}  // namespace lsms

using namespace lsms;

// ---------------------------------------------------------------- C ABI (host only)
extern "C" const char* lsms_last_error(void) { return g_last_error.c_str(); }

extern "C" int lsms_version(void) { return 10000; }

extern "C" int lsms_gaunt_table(int lmax, double* C) {
  clear_error();
  if (lmax < 0 || lmax > kMaxLmax || !C) return fail(LSMS_ERR_ARG, "lsms_gaunt_table: lmax must be 0..%d", kMaxLmax);
  const std::vector<double> t = gaunt_real(lmax);
  std::memcpy(C, t.data(), t.size() * sizeof(double));
  return LSMS_OK;
}

extern "C" int lsms_dipole_current(int lmax, const lsms_complex* r_ll, int n_species, lsms_complex* J) {
  clear_error();
  if (lmax < 0 || lmax > kMaxLmax) return fail(LSMS_ERR_ARG, "lsms_dipole_current: lmax must be 0..%d", kMaxLmax);
  if (n_species < 1 || !r_ll || !J) return fail(LSMS_ERR_ARG, "lsms_dipole_current: bad arguments");
  const int K = (lmax + 1) * (lmax + 1);
  const int K3 = (2 * lmax + 1) * (2 * lmax + 1);
  const std::vector<double> C = gaunt_real(lmax);
  const int mu_m[3] = {1, -1, 0};
  const int nl = lmax + 1;
  for (int s = 0; s < n_species; ++s)
    for (int c = 0; c < 4; ++c)
      for (int mu = 0; mu < 3; ++mu) {
        const int L3 = 2 + mu_m[mu];  // l = 1: L = 1*1 + 1 + m
        for (int L = 0; L < K; ++L)
          for (int Lp = 0; Lp < K; ++Lp) {
            lsms_complex v{0.0, 0.0};
            const int l = l_of(L), lp = l_of(Lp);
            if (std::abs(l - lp) == 1 && L3 < K3) {
              const double g = C[((size_t)L * K + Lp) * K3 + L3];
              const lsms_complex r = r_ll[((size_t)(s * 4 + c) * nl + l) * nl + lp];
              v.re = r.re * g;
              v.im = r.im * g;
            }
            J[((((size_t)s * 4 + c) * 3 + mu) * K + L) * K + Lp] = v;
          }
      }
  return LSMS_OK;
}

// ---------------------------------------------------------------- LIZ builder
namespace {
struct Cand {
  int32_t j;
  int32_t im[3];
  double d[3];
  bool centre;
};

bool cand_less(const Cand& a, const Cand& b) {
  if (a.centre != b.centre) return a.centre;
  if (a.j != b.j) return a.j < b.j;
  for (int k = 0; k < 3; ++k)
    if (a.im[k] != b.im[k]) return a.im[k] < b.im[k];
  return false;
}

// f(m) for m = 0 .. n - 1 on up to 8 host threads (the atoms' neighbour searches
// are independent); one thread for small n.
template <typename F>
void parallel_atoms(int n, F& f) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nt = std::min<int>({8, (int)hw, std::max(1, n / 32)});
  if (nt <= 1) {
    for (int m = 0; m < n; ++m) f(m);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(nt - 1);
  auto run = [&](int t) {
    for (int m = t; m < n; m += nt) f(m);
  };
  for (int t = 1; t < nt; ++t) th.emplace_back(run, t);
  run(0);
  for (auto& x : th) x.join();
}

bool inv3(const double a[9], double out[9]) {
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  if (!(std::fabs(det) > 1e-12)) return false;
  const double id = 1.0 / det;
  out[0] = (a[4] * a[8] - a[5] * a[7]) * id;
  out[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  out[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  out[3] = (a[5] * a[6] - a[3] * a[8]) * id;
  out[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  out[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  out[6] = (a[3] * a[7] - a[4] * a[6]) * id;
  out[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  out[8] = (a[0] * a[4] - a[1] * a[3]) * id;
  return true;
}
}  // namespace

extern "C" int lsms_build_liz(const double* pos, int n_atoms, const double* lattice, double r_liz,
                              lsms_liz** out) {
  clear_error();
  if (!out) return fail(LSMS_ERR_ARG, "lsms_build_liz: out is NULL");
  *out = nullptr;
  if (!pos || n_atoms < 1) return fail(LSMS_ERR_ARG, "lsms_build_liz: need at least one atom");
  if (!(r_liz >= 0.0) || !std::isfinite(r_liz)) return fail(LSMS_ERR_ARG, "lsms_build_liz: r_liz must be finite and >= 0");
  for (int i = 0; i < 3 * n_atoms; ++i)
    if (!std::isfinite(pos[i])) return fail(LSMS_ERR_ARG, "lsms_build_liz: non-finite position");
  const double rcut = r_liz + 1e-8;
  const double rcut2 = rcut * rcut;
  lsms_liz* z = new (std::nothrow) lsms_liz();
  if (!z) return fail(LSMS_ERR_NOMEM, "lsms_build_liz: out of host memory");
  z->n_atoms = n_atoms;
  z->periodic = lattice != nullptr;
  z->offsets.assign(n_atoms + 1, 0);

  std::vector<std::vector<Cand>> per(n_atoms);
  if (!lattice) {
    // Finite cluster: uniform grid of cell width >= rcut over the bounding box.
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) { lo[k] = hi[k] = pos[k]; }
    for (int i = 0; i < n_atoms; ++i)
      for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], pos[3 * i + k]); hi[k] = std::max(hi[k], pos[3 * i + k]); }
    const double w = std::max(rcut, 1e-6);
    int nc[3];
    for (int k = 0; k < 3; ++k) nc[k] = std::max(1, std::min(256, (int)std::floor((hi[k] - lo[k]) / w) + 1));
    std::vector<std::vector<int>> cell((size_t)nc[0] * nc[1] * nc[2]);
    auto cidx = [&](int i, int k) {
      int c = (int)std::floor((pos[3 * i + k] - lo[k]) / w);
      return std::max(0, std::min(nc[k] - 1, c));
    };
    for (int i = 0; i < n_atoms; ++i) cell[((size_t)cidx(i, 0) * nc[1] + cidx(i, 1)) * nc[2] + cidx(i, 2)].push_back(i);
    for (int m = 0; m < n_atoms; ++m) {
      const int c0 = cidx(m, 0), c1 = cidx(m, 1), c2 = cidx(m, 2);
      for (int a = std::max(0, c0 - 1); a <= std::min(nc[0] - 1, c0 + 1); ++a)
        for (int b = std::max(0, c1 - 1); b <= std::min(nc[1] - 1, c1 + 1); ++b)
          for (int c = std::max(0, c2 - 1); c <= std::min(nc[2] - 1, c2 + 1); ++c)
            for (int j : cell[((size_t)a * nc[1] + b) * nc[2] + c]) {
              Cand cd;
              double d2 = 0.0;
              for (int k = 0; k < 3; ++k) {
                cd.d[k] = pos[3 * j + k] - pos[3 * m + k];
                d2 += cd.d[k] * cd.d[k];
              }
              if (d2 > rcut2) continue;
              cd.j = j;
              cd.im[0] = cd.im[1] = cd.im[2] = 0;
              cd.centre = (j == m);
              per[m].push_back(cd);
            }
    }
  } else {
    double inv[9];
    if (!inv3(lattice, inv)) { delete z; return fail(LSMS_ERR_ARG, "lsms_build_liz: singular lattice"); }
    // plane spacing h_k = V / |a_{k+1} x a_{k+2}| = 1 / |row k of inverse^T| -> use columns of inv
    double h[3];
    for (int k = 0; k < 3; ++k) {
      const double nx = inv[0 * 3 + k], ny = inv[1 * 3 + k], nz = inv[2 * 3 + k];
      h[k] = 1.0 / std::sqrt(nx * nx + ny * ny + nz * nz);
    }
    // fractional coordinates f = pos * inv (pos as row vector, pos = f * lattice)
    std::vector<double> fw((size_t)3 * n_atoms);
    std::vector<int> wsh((size_t)3 * n_atoms);
    int nc[3], rng[3];
    for (int k = 0; k < 3; ++k) {
      nc[k] = std::max(1, std::min(256, (int)std::floor(h[k] / std::max(rcut, 1e-9))));
      rng[k] = std::max(1, (int)std::ceil(rcut * nc[k] / h[k])) + 1;  // +1: cell-boundary rounding
    }
    std::vector<std::vector<int>> cell((size_t)nc[0] * nc[1] * nc[2]);
    std::vector<int> ci((size_t)3 * n_atoms);
    for (int i = 0; i < n_atoms; ++i) {
      for (int k = 0; k < 3; ++k) {
        const double f = pos[3 * i + 0] * inv[0 * 3 + k] + pos[3 * i + 1] * inv[1 * 3 + k] + pos[3 * i + 2] * inv[2 * 3 + k];
        const double fl = std::floor(f);
        wsh[3 * i + k] = (int)fl;
        fw[3 * i + k] = f - fl;
        ci[3 * i + k] = std::max(0, std::min(nc[k] - 1, (int)std::floor((f - fl) * nc[k])));
      }
      cell[((size_t)ci[3 * i] * nc[1] + ci[3 * i + 1]) * nc[2] + ci[3 * i + 2]].push_back(i);
    }
    // wrapped Cartesian positions, for a cheap pre-test of each candidate
    std::vector<double> pw((size_t)3 * n_atoms);
    for (int i = 0; i < n_atoms; ++i)
      for (int k = 0; k < 3; ++k)
        pw[3 * i + k] = fw[3 * i] * lattice[0 * 3 + k] + fw[3 * i + 1] * lattice[1 * 3 + k] + fw[3 * i + 2] * lattice[2 * 3 + k];
    const double pre_cut2 = rcut2 * (1.0 + 1e-9) + 1e-300;
    auto search = [&](int m) {
      per[m].reserve(64);
      for (int da = -rng[0]; da <= rng[0]; ++da)
        for (int db = -rng[1]; db <= rng[1]; ++db)
          for (int dc = -rng[2]; dc <= rng[2]; ++dc) {
            // a cell |d| cells away along axis k is at least (|d| - 1) / nc[k] apart in
            // that fractional coordinate, i.e. (|d| - 1) h[k] / nc[k] in distance
            const int dd[3] = {da, db, dc};
            double gap = 0.0;
            for (int k = 0; k < 3; ++k) gap = std::max(gap, (std::abs(dd[k]) - 1) * h[k] / nc[k]);
            if (gap > rcut * (1.0 + 1e-9)) continue;
            const int raw[3] = {ci[3 * m] + da, ci[3 * m + 1] + db, ci[3 * m + 2] + dc};
            int cc[3], t[3];
            for (int k = 0; k < 3; ++k) {
              const int q = (int)std::floor((double)raw[k] / nc[k]);
              t[k] = q;
              cc[k] = raw[k] - q * nc[k];
            }
            double tw[3];  // t . lattice - wrapped position of m
            for (int k = 0; k < 3; ++k)
              tw[k] = t[0] * lattice[0 * 3 + k] + t[1] * lattice[1 * 3 + k] + t[2] * lattice[2 * 3 + k] - pw[3 * m + k];
            for (int j : cell[((size_t)cc[0] * nc[1] + cc[1]) * nc[2] + cc[2]]) {
              double q2 = 0.0;
              for (int k = 0; k < 3; ++k) {
                const double dk = pw[3 * j + k] + tw[k];
                q2 += dk * dk;
              }
              if (q2 > pre_cut2) continue;  // the exact test below decides the rest
              // relative to the wrapped centre: (fw_j + t - fw_m) * lattice == pos_j + T * lattice - pos_m
              // with T = t - floor(f_j) + floor(f_m)
              Cand cd;
              for (int k = 0; k < 3; ++k) cd.im[k] = t[k] - wsh[3 * j + k] + wsh[3 * m + k];
              double d2 = 0.0;
              for (int k = 0; k < 3; ++k) {
                const double tv = cd.im[0] * lattice[0 * 3 + k] + cd.im[1] * lattice[1 * 3 + k] + cd.im[2] * lattice[2 * 3 + k];
                cd.d[k] = (pos[3 * j + k] + tv) - pos[3 * m + k];
                d2 += cd.d[k] * cd.d[k];
              }
              if (d2 > rcut2) continue;
              cd.j = j;
              cd.centre = (j == m && cd.im[0] == 0 && cd.im[1] == 0 && cd.im[2] == 0);
              per[m].push_back(cd);
            }
          }
      std::sort(per[m].begin(), per[m].end(), cand_less);
    };
    parallel_atoms(n_atoms, search);
  }
  int64_t total = 0;
  int smax = 0, smin = 1 << 30;
  for (int m = 0; m < n_atoms; ++m) {
    if (!lattice) std::sort(per[m].begin(), per[m].end(), cand_less);  // periodic: sorted by the search
    if (per[m].empty() || !per[m][0].centre) { delete z; return fail(LSMS_ERR_ARG, "lsms_build_liz: atom %d missing from its own LIZ", m); }
    const int s = (int)per[m].size();
    smax = std::max(smax, s);
    smin = std::min(smin, s);
    total += s;
    z->offsets[m + 1] = total;
  }
  if (total > ((int64_t)1 << 31)) { delete z; return fail(LSMS_ERR_NOMEM, "lsms_build_liz: too many sites"); }
  z->total_sites = total;
  z->max_sites = smax;
  z->min_sites = smin;
  z->site_atom.resize(total);
  z->image.resize(3 * total);
  z->disp.resize(3 * total);
  z->site_centre.resize(total);
  for (int m = 0; m < n_atoms; ++m) {
    int64_t o = z->offsets[m];
    for (const Cand& c : per[m]) {
      z->site_atom[o] = c.j;
      z->site_centre[o] = m;
      for (int k = 0; k < 3; ++k) {
        z->image[3 * o + k] = c.im[k];
        z->disp[3 * o + k] = c.d[k];
      }
      ++o;
    }
  }
  // inverse map: the sites at which each atom appears, in increasing site order
  z->inv_off.assign(n_atoms + 1, 0);
  for (int64_t s = 0; s < total; ++s) z->inv_off[z->site_atom[s] + 1]++;
  for (int i = 0; i < n_atoms; ++i) z->inv_off[i + 1] += z->inv_off[i];
  z->inv_sites.resize(total);
  std::vector<int64_t> fill(z->inv_off.begin(), z->inv_off.end() - 1);
  for (int64_t s = 0; s < total; ++s) z->inv_sites[fill[z->site_atom[s]]++] = s;
  *out = z;
  return LSMS_OK;
}

extern "C" int lsms_liz_sizes(const lsms_liz* liz, int* n_atoms, int64_t* total_sites, int* max_sites,
                              int* min_sites) {
  clear_error();
  if (!liz) return fail(LSMS_ERR_ARG, "lsms_liz_sizes: NULL liz");
  if (n_atoms) *n_atoms = liz->n_atoms;
  if (total_sites) *total_sites = liz->total_sites;
  if (max_sites) *max_sites = liz->max_sites;
  if (min_sites) *min_sites = liz->min_sites;
  return LSMS_OK;
}

extern "C" int lsms_liz_export(const lsms_liz* liz, int64_t* offsets, int32_t* site_atom, int32_t* image,
                               double* disp) {
  clear_error();
  if (!liz) return fail(LSMS_ERR_ARG, "lsms_liz_export: NULL liz");
  if (offsets) std::memcpy(offsets, liz->offsets.data(), liz->offsets.size() * sizeof(int64_t));
  if (site_atom) std::memcpy(site_atom, liz->site_atom.data(), liz->site_atom.size() * sizeof(int32_t));
  if (image) std::memcpy(image, liz->image.data(), liz->image.size() * sizeof(int32_t));
  if (disp) std::memcpy(disp, liz->disp.data(), liz->disp.size() * sizeof(double));
  return LSMS_OK;
}
