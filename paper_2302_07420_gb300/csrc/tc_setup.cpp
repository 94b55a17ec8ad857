// Host setup of the TC operator (cell, mesh, spheres, tables), FP64.
//
// Conventions: reciprocal rows b_i with a_i . b_j = 2 pi delta_ij; Gamma-centred
// mesh with fractional coordinates in (-1/2, 1/2]; sphere |k+G|^2/2 <= ecut in
// lexicographic Miller order; FFT index m of the box stands for the Miller
// integer m (m <= (n-1)/2) or m - n.
#include "tc_setup.hpp"

#include <algorithm>
#include <cmath>
#include <iterator>
#include <map>
#include <tuple>

namespace tc {

static const double kPi = 3.14159265358979323846;
static const double k4Pi = 4.0 * kPi;

// --- Jastrow kernel transforms (Sec. 2.6.3, Appendix B) -----------------------
// u~(p) = 4 pi A (1/p^2 - 1/(p^2 + C^-2)) in the cancellation-free form.
double host_u_tilde(double p2, double A, double C) {
  const double c2 = 1.0 / (C * C);
  return k4Pi * A * c2 / (p2 * (p2 + c2));
}

static double lap_u(double p2, double A, double C) {
  const double c2 = 1.0 / (C * C);
  return -k4Pi * A * c2 / (p2 + c2);
}

// B(g) = -(pi/4) g^2 - (1 + g^2/2) atan(g/2) + (1 + g^2) atan(g) (Appendix B).
// g <= 1: as printed.  1 < g <= 6: atan(x) = pi/2 - atan(1/x) cancels the pi
// terms exactly.  g > 6: series in 1/g from the atan Taylor series,
// B = sum_{k>=1} c_k g^-(2k+1), c_k = (-1)^k [(2^(2k+1)-1)/(2k+1) - (2^(2k+2)-1)/(2k+3)].
static double B_of_g(double g) {
  if (g <= 1.0) return -0.25 * kPi * g * g - (1.0 + 0.5 * g * g) * std::atan(0.5 * g) + (1.0 + g * g) * std::atan(g);
  if (g <= 6.0) return (1.0 + 0.5 * g * g) * std::atan(2.0 / g) - (1.0 + g * g) * std::atan(1.0 / g);
  const double inv2 = 1.0 / (g * g);
  double pw = inv2 / g;     // g^-3
  double sum = 0.0;
  double p2k1 = 8.0;        // 2^(2k+1) at k = 1
  for (int k = 1; k < 60; ++k) {
    const double ck = ((k & 1) ? -1.0 : 1.0) * ((p2k1 - 1.0) / (2 * k + 1) - (2.0 * p2k1 - 1.0) / (2 * k + 3));
    sum += ck * pw;
    pw *= inv2;
    p2k1 *= 4.0;
    if (std::fabs(ck * pw) < 1e-30 * std::fabs(sum)) break;
  }
  return sum;
}

double host_gradu_sq(double p, double A, double C) {
  const double g = C * p;
  if (g == 0.0) return 2.0 * kPi * A * A / C;
  return k4Pi * A * A / (C * g) * B_of_g(g);
}

// D(g) = g B'(g) - 2 B(g), with B'(g) = 2/(4 + g^2) + g (2 atan g - atan(g/2) - pi/2);
// the same three branches as B_of_g (for g > 1 the bracket is atan(2/g) - 2 atan(1/g),
// for g > 6 the series gives D = -sum_k (2k + 3) c_k g^-(2k+1)).
static double D_of_g(double g) {
  if (g <= 1.0) {
    const double dB = 2.0 / (4.0 + g * g) + g * (2.0 * std::atan(g) - std::atan(0.5 * g) - 0.5 * kPi);
    return g * dB - 2.0 * B_of_g(g);
  }
  if (g <= 6.0) {
    const double dB = 2.0 / (4.0 + g * g) + g * (std::atan(2.0 / g) - 2.0 * std::atan(1.0 / g));
    return g * dB - 2.0 * B_of_g(g);
  }
  const double inv2 = 1.0 / (g * g);
  double pw = inv2 / g;
  double sum = 0.0;
  double p2k1 = 8.0;
  for (int k = 1; k < 60; ++k) {
    const double ck = ((k & 1) ? -1.0 : 1.0) * ((p2k1 - 1.0) / (2 * k + 1) - (2.0 * p2k1 - 1.0) / (2 * k + 3));
    const double t = -(2 * k + 3) * ck * pw;
    sum += t;
    pw *= inv2;
    p2k1 *= 4.0;
    if (std::fabs(t) < 1e-30 * std::fabs(sum)) break;
  }
  return sum;
}

// One Jastrow channel (A, C) and what to evaluate: the kernel (wrt = -1), its
// derivative with respect to A (wrt = 0) or C (wrt = 1), or nothing (wrt = 2,
// a channel the derivative does not touch).
struct Chan {
  double A, C;
  int wrt;
};

static double ch_u(double p2, const Chan& c) {   // u~(p), p > 0
  const double c2 = 1.0 / (c.C * c.C);
  switch (c.wrt) {
    case -1: return host_u_tilde(p2, c.A, c.C);
    case 0: return k4Pi * c2 / (p2 * (p2 + c2));
    case 1: return -2.0 * k4Pi * c.A / (c.C * c.C * c.C * (p2 + c2) * (p2 + c2));
    default: return 0.0;
  }
}

static double ch_lap(double p2, const Chan& c) {   // (lap u)~(p)
  const double c2 = 1.0 / (c.C * c.C);
  switch (c.wrt) {
    case -1: return lap_u(p2, c.A, c.C);
    case 0: return -k4Pi * c2 / (p2 + c2);
    case 1: return 2.0 * k4Pi * c.A * p2 / (c.C * c.C * c.C * (p2 + c2) * (p2 + c2));
    default: return 0.0;
  }
}

static double ch_gsq(double p, const Chan& c) {   // ((grad u)^2)~(p), p >= 0
  const double g = c.C * p;
  switch (c.wrt) {
    case -1: return host_gradu_sq(p, c.A, c.C);
    case 0: return g == 0.0 ? k4Pi * c.A / c.C : 2.0 * k4Pi * c.A / (c.C * g) * B_of_g(g);
    case 1: return g == 0.0 ? -2.0 * kPi * c.A * c.A / (c.C * c.C) : k4Pi * c.A * c.A / (c.C * c.C * c.C * p) * D_of_g(g);
    default: return 0.0;
  }
}

// finite Jastrow part of V_2a at p = 0: (lap u)~(0) - ((grad u)^2)~(0) = -4 pi A - 2 pi A^2 / C
static double ch_v0(const Chan& c) {
  switch (c.wrt) {
    case -1: return -k4Pi * c.A - 2.0 * kPi * c.A * c.A / c.C;
    case 0: return -k4Pi - k4Pi * c.A / c.C;
    case 1: return 2.0 * kPi * c.A * c.A / (c.C * c.C);
    default: return 0.0;
  }
}

// (4 pi A)^2 Gamma0 + x 4 pi A u_short / Nk with u_short = -4 pi A C^2 (Eq. u_short)
static double ch_corr(const Chan& c, double Gamma0, double x, int Nk) {
  const double a2 = k4Pi * c.A * k4Pi * c.A;
  switch (c.wrt) {
    case -1: return a2 * (Gamma0 - x * c.C * c.C / Nk);
    case 0: return 2.0 * k4Pi * k4Pi * c.A * (Gamma0 - x * c.C * c.C / Nk);
    case 1: return a2 * (-2.0 * x * c.C / Nk);
    default: return 0.0;
  }
}

static double ch_amp(const Chan& c) { return c.wrt == -1 ? c.A : (c.wrt == 0 ? 1.0 : 0.0); }

// --- small linear algebra ----------------------------------------------------
static double det3(const double M[3][3]) {
  return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
         M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

static void reciprocal(const double A[3][3], double B[3][3]) {
  // B = 2 pi (A^-1)^T: rows b_i = 2 pi (a_j x a_k) / det
  const double d = det3(A);
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    B[i][0] = 2.0 * kPi * (A[j][1] * A[k][2] - A[j][2] * A[k][1]) / d;
    B[i][1] = 2.0 * kPi * (A[j][2] * A[k][0] - A[j][0] * A[k][2]) / d;
    B[i][2] = 2.0 * kPi * (A[j][0] * A[k][1] - A[j][1] * A[k][0]) / d;
  }
}

static double norm3(const double* v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

// sum' exp(-alpha p^2)/p^2 over the reciprocal lattice of the supercell (p != 0),
// until exp(-alpha p^2) < 1e-20; terms summed in ascending order.
static double aux_sum(const Setup& S, double alpha) {
  const double pmax = std::sqrt(-std::log(1e-20) / alpha);
  int bound[3];
  double Bs[3][3];
  for (int i = 0; i < 3; ++i) {
    const double L = norm3(S.A[i]) * S.prm.kmesh[i];
    bound[i] = (int)std::ceil(pmax * L / (2.0 * kPi)) + 1;
    for (int d = 0; d < 3; ++d) Bs[i][d] = S.B[i][d] / S.prm.kmesh[i];
  }
  std::vector<double> w;
  for (int a = -bound[0]; a <= bound[0]; ++a)
    for (int b = -bound[1]; b <= bound[1]; ++b)
      for (int c = -bound[2]; c <= bound[2]; ++c) {
        if (a == 0 && b == 0 && c == 0) continue;
        double p[3];
        for (int d = 0; d < 3; ++d) p[d] = a * Bs[0][d] + b * Bs[1][d] + c * Bs[2][d];
        const double p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
        w.push_back(std::exp(-alpha * p2) / p2);
      }
  std::sort(w.begin(), w.end());
  double s = 0.0;
  for (double x : w) s += x;
  return s;
}

// Neumaier's compensated sum (terms of both signs).
namespace {
struct CompSum {
  double s = 0.0, c = 0.0;
  void add(double x) {
    const double t = s + x;
    c += std::fabs(s) >= std::fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};
}  // namespace

bool band_constants(const Setup& S, const double kcart[3], double* gamma_b, double W[3]) {
  const double alpha = S.alpha;
  const double kn = norm3(kcart);
  const double pmax = std::sqrt(-std::log(1e-20) / alpha) + kn;
  int bound[3];
  double Bs[3][3];
  for (int i = 0; i < 3; ++i) {
    const double L = norm3(S.A[i]) * S.prm.kmesh[i];
    bound[i] = (int)std::ceil(pmax * L / (2.0 * kPi)) + 1;
    for (int d = 0; d < 3; ++d) Bs[i][d] = S.B[i][d] / S.prm.kmesh[i];
  }
  std::vector<double> w;
  CompSum wv[3];
  for (int a = -bound[0]; a <= bound[0]; ++a)
    for (int b = -bound[1]; b <= bound[1]; ++b)
      for (int c = -bound[2]; c <= bound[2]; ++c) {
        double p[3];
        for (int d = 0; d < 3; ++d) p[d] = kcart[d] - (a * Bs[0][d] + b * Bs[1][d] + c * Bs[2][d]);
        const double p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
        if (p2 == 0.0) return false;
        const double t = std::exp(-alpha * p2) / p2;
        w.push_back(t);
        for (int d = 0; d < 3; ++d) wv[d].add(p[d] * t);
      }
  std::sort(w.begin(), w.end());
  double s = 0.0;
  for (double x : w) s += x;
  *gamma_b = S.Omega / (4.0 * std::sqrt(kPi * kPi * kPi * alpha)) - s / S.Nk;
  for (int d = 0; d < 3; ++d) W[d] = wv[d].value();
  return true;
}

bool sphere(const Setup& S, const double kcart[3], std::vector<std::array<int, 3>>& out) {
  out.clear();
  const int n = S.prm.fft[0];
  const double ecut = S.prm.ecut_ha;
  const double gmax = std::sqrt(2.0 * ecut) + norm3(kcart);
  int bound[3];
  for (int i = 0; i < 3; ++i) bound[i] = (int)std::ceil(gmax * norm3(S.A[i]) / (2.0 * kPi)) + 1;
  for (int a = -bound[0]; a <= bound[0]; ++a)
    for (int b = -bound[1]; b <= bound[1]; ++b)
      for (int c = -bound[2]; c <= bound[2]; ++c) {
        double kg[3];
        for (int d = 0; d < 3; ++d) kg[d] = kcart[d] + (a * S.B[0][d] + b * S.B[1][d] + c * S.B[2][d]);
        if (0.5 * (kg[0] * kg[0] + kg[1] * kg[1] + kg[2] * kg[2]) <= ecut) out.push_back({a, b, c});
      }
  for (auto& m : out)
    for (int i = 0; i < 3; ++i)
      if (std::abs(m[i]) > (n - 1) / 2) return false;
  return true;
}

int pick_split(int items, int partners, int sms) {
  int best = 1;
  double best_eff = 0.0;
  for (int s = 1; s <= std::min(8, partners); ++s) {
    const long long ctas = (long long)items * s;
    const long long waves = (ctas + sms - 1) / sms;
    const double eff = (double)ctas / (double)(waves * sms);
    if (eff > best_eff + 0.01) {
      best_eff = eff;
      best = s;
    }
  }
  return best;
}

int miller_span(const std::vector<std::vector<std::array<int, 3>>>& miller) {
  int span = 0;
  for (int i = 0; i < 3; ++i) {
    int lo = 1 << 30, hi = -(1 << 30);
    for (const auto& sph : miller)
      for (const auto& m : sph) {
        lo = std::min(lo, m[i]);
        hi = std::max(hi, m[i]);
      }
    if (hi >= lo) span = std::max(span, hi - lo);
  }
  return span;
}

bool left_from_right_exact(int n, int span) { return n % 2 == 1 || span <= n / 2 - 1; }

int pair_support_len(int n, int span) { return std::min(n, 2 * span + 1); }

size_t mirror_buffer_bytes(bool fp64, int nkb, int prune_L, int pair_support, int Nk, int no, size_t free_bytes) {
  if (!fp64 || nkb > 0 || prune_L <= 0 || pair_support > prune_L || Nk <= 0 || no <= 0) return 0;
  const size_t L = (size_t)prune_L, M = (size_t)Nk * no;
  const size_t bytes = M * M * 2 * L * L * L * 16;
  return bytes <= free_bytes / 4 ? bytes : 0;
}

int smallest_near_best(const double* t, int n) {
  double best = 1e300;
  for (int s = 1; s <= n; ++s) best = std::min(best, t[s]);
  for (int s = 1; s <= n; ++s)
    if (t[s] <= 1.02 * best) return s;
  return 1;
}

static int fft_rep(int m, int n) { return m <= (n - 1) / 2 ? m : m - n; }
static void value_tables(Setup& S);
static void build_deltas(Setup& S);
static void flatten_spheres(Setup& S);

std::string build_setup(const tc_params& p, Setup& S) {
  S.prm = p;
  if (p.fft[0] != p.fft[1] || p.fft[1] != p.fft[2]) return "unsupported: FFT box must be cubic";
  const int n = p.fft[0];
  static const int kSizes[] = {9, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 48};
  if (std::find(std::begin(kSizes), std::end(kSizes), n) == std::end(kSizes))
    return "unsupported: FFT box size (9, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32 or 48)";
  for (int i = 0; i < 3; ++i)
    if (p.kmesh[i] < 1 || p.kmesh[i] > 16) return "kmesh entries must be in [1, 16]";
  if (!(p.nocc > 0 && p.nocc <= p.nbands)) return "need 0 < nocc <= nbands";
  if (!(p.ecut_ha > 0)) return "ecut_ha must be positive";
  if (!(p.C[0] > 0 && p.C[1] > 0)) return "Jastrow C must be positive";
  if (!(p.A[0] >= 0 && p.A[1] >= 0)) return "Jastrow A must be non-negative";
  if (p.precision == TC_FP32_COMP) return "unsupported: TC_FP32_COMP (compensated FP32 accumulation) is not built";
  if (p.precision != TC_FP64 && p.precision != TC_FP32 && p.precision != TC_BF16_STORE)
    return "precision must be TC_FP64, TC_FP32 or TC_BF16_STORE";
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S.A[i][j] = p.lattice[i][j];
  S.Omega = std::fabs(det3(S.A));
  if (!(S.Omega > 0)) return "lattice is singular";
  reciprocal(S.A, S.B);
  S.n = n;
  S.N = n * n * n;
  S.nb = p.nbands;
  S.no = p.nocc;
  S.Nk = p.kmesh[0] * p.kmesh[1] * p.kmesh[2];

  // k mesh
  S.kfrac.clear();
  S.kcart.clear();
  for (int a = 0; a < p.kmesh[0]; ++a)
    for (int b = 0; b < p.kmesh[1]; ++b)
      for (int c = 0; c < p.kmesh[2]; ++c) {
        const int idx[3] = {a, b, c};
        std::array<double, 3> f{};
        for (int i = 0; i < 3; ++i) {
          f[i] = (double)idx[i] / p.kmesh[i];
          if (f[i] > 0.5) f[i] -= 1.0;
        }
        std::array<double, 3> kc{};
        for (int d = 0; d < 3; ++d) kc[d] = f[0] * S.B[0][d] + f[1] * S.B[1][d] + f[2] * S.B[2][d];
        S.kfrac.push_back(f);
        S.kcart.push_back(kc);
      }

  // spheres
  S.miller.assign(S.Nk, {});
  S.npw.assign(S.Nk, 0);
  for (int k = 0; k < S.Nk; ++k) {
    if (!sphere(S, S.kcart[k].data(), S.miller[k])) return "plane-wave sphere does not fit the FFT box";
    S.npw[k] = (int)S.miller[k].size();
  }
  S.Nkt = S.Nk;
  S.nkb = 0;
  flatten_spheres(S);

  // divergence-correction constant (Eq. correction2, k on the mesh)
  if (p.alpha > 0) {
    S.alpha = p.alpha;
  } else {
    double best = 1e300, Sup[3][3];
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d) Sup[i][d] = S.A[i][d] * p.kmesh[i];
    for (int a = -2; a <= 2; ++a)
      for (int b = -2; b <= 2; ++b)
        for (int c = -2; c <= 2; ++c) {
          if (!a && !b && !c) continue;
          double v[3];
          for (int d = 0; d < 3; ++d) v[d] = a * Sup[0][d] + b * Sup[1][d] + c * Sup[2][d];
          best = std::min(best, norm3(v));
        }
    S.alpha = (best / 12.0) * (best / 12.0);
  }
  S.Gamma0 = S.Omega / (4.0 * std::sqrt(kPi * kPi * kPi * S.alpha)) - (-S.alpha + aux_sum(S, S.alpha)) / S.Nk;

  S.Nkt = S.Nk;
  build_deltas(S);

  value_tables(S);
  return "";
}

static void value_tables(Setup& S) {
  KernelData kd;
  kernel_data(S, KD_VALUE, kd);
  S.tabV = std::move(kd.tabV);
  S.tabU = std::move(kd.tabU);
  S.hartV = std::move(kd.hartV);
  S.hartU = std::move(kd.hartU);
  S.hartUs = std::move(kd.hartUs);
  for (int s = 0; s < 2; ++s) {
    S.corr_c[s] = kd.corr_c[s];
    S.amp[s] = kd.amp[s];
  }
}

// Distinct Delta = k_out - k_part (unreduced Cartesian differences of the in-cell k of every
// k-point with orbitals) and the [Nkt][Nkt] id table; pairs of two band points get no id (never used).
static void build_deltas(Setup& S) {
  std::map<std::tuple<long long, long long, long long>, int> ids;
  S.delta_id.assign((size_t)S.Nkt * S.Nkt, 0);
  S.delta.clear();
  for (int ko = 0; ko < S.Nkt; ++ko)
    for (int kp = 0; kp < S.Nkt; ++kp) {
      if (ko >= S.Nk && kp >= S.Nk) continue;
      // mesh differences are integers in units of 1/kmesh; band points are resolved to 2^-20 of that
      long long key[3];
      for (int i = 0; i < 3; ++i)
        key[i] = std::llround((S.kfrac[ko][i] - S.kfrac[kp][i]) * S.prm.kmesh[i] * 1048576.0);
      auto t = std::make_tuple(key[0], key[1], key[2]);
      auto it = ids.find(t);
      int id;
      if (it == ids.end()) {
        id = (int)S.delta.size();
        ids[t] = id;
        std::array<double, 3> dc{};
        for (int d = 0; d < 3; ++d) dc[d] = S.kcart[ko][d] - S.kcart[kp][d];
        S.delta.push_back(dc);
      } else {
        id = it->second;
      }
      S.delta_id[(size_t)ko * S.Nkt + kp] = id;
    }
  S.ndelta = (int)S.delta.size();
}

// Flattened Miller vectors and box indices of all Nkt spheres (zero / -1 padded to npw_max).
static void flatten_spheres(Setup& S) {
  const int n = S.n;
  S.npw_max = *std::max_element(S.npw.begin(), S.npw.end());
  S.miller_flat.assign((size_t)S.Nkt * S.npw_max * 3, 0);
  S.box_index.assign((size_t)S.Nkt * S.npw_max, -1);
  for (int k = 0; k < S.Nkt; ++k)
    for (int g = 0; g < S.npw[k]; ++g) {
      const auto& m = S.miller[k][g];
      for (int i = 0; i < 3; ++i) S.miller_flat[((size_t)k * S.npw_max + g) * 3 + i] = m[i];
      const int i1 = (m[0] + n) % n, i2 = (m[1] + n) % n, i3 = (m[2] + n) % n;
      S.box_index[(size_t)k * S.npw_max + g] = (i1 * n + i2) * n + i3;
    }
}

std::string add_band_points(Setup& S, int nkb, const double* kfrac_band) {
  if (nkb < 1 || !kfrac_band) return "need at least one band point";
  if (S.nkb != 0) return "band points already added";
  S.gamma_b.assign(nkb, 0.0);
  S.Wb.assign(nkb, {});
  for (int b = 0; b < nkb; ++b) {
    std::array<double, 3> f{}, kc{};
    for (int i = 0; i < 3; ++i) f[i] = kfrac_band[3 * b + i];
    for (int d = 0; d < 3; ++d) kc[d] = f[0] * S.B[0][d] + f[1] * S.B[1][d] + f[2] * S.B[2][d];
    double W[3];
    if (!band_constants(S, kc.data(), &S.gamma_b[b], W))
      return "band point " + std::to_string(b) + " lies on the SCF mesh (modulo a reciprocal vector)";
    for (int d = 0; d < 3; ++d) S.Wb[b][d] = W[d];
    std::vector<std::array<int, 3>> m;
    if (!sphere(S, kc.data(), m)) return "plane-wave sphere of band point " + std::to_string(b) + " does not fit the FFT box";
    S.kfrac.push_back(f);
    S.kcart.push_back(kc);
    S.miller.push_back(m);
    S.npw.push_back((int)m.size());
  }
  S.nkb = nkb;
  S.Nkt = S.Nk + nkb;
  flatten_spheres(S);
  build_deltas(S);
  value_tables(S);
  return "";
}

void kernel_data(const Setup& S, int mode, KernelData& kd) {
  const tc_params& p = S.prm;
  const int n = S.n;
  const size_t N = S.N;
  const bool value = mode == KD_VALUE;
  Chan ch[2];
  for (int s = 0; s < 2; ++s) {
    ch[s] = {p.A[s], p.C[s], -1};
    if (!value) ch[s].wrt = (mode % 2 == s) ? mode / 2 : 2;
  }
  const double coul = value ? 1.0 : 0.0;   // the Coulomb part does not depend on A or C
  for (int s = 0; s < 2; ++s) {
    kd.corr_c[s] = ch_corr(ch[s], S.Gamma0, p.ushort_factor, S.Nk);
    kd.amp[s] = ch_amp(ch[s]);
  }
  // exchange tables at p = Delta + G; V uses the parallel-spin channel
  kd.tabV.assign((size_t)S.ndelta * 2 * N, 0.0);
  kd.tabU.assign((size_t)S.ndelta * 2 * N, 0.0);
  const double v0 = (ch_v0(ch[0]) + (value && p.div_correction ? k4Pi * S.Nk * S.Gamma0 : 0.0)) / S.Omega;
  for (int id = 0; id < S.ndelta; ++id)
    for (int i1 = 0; i1 < n; ++i1)
      for (int i2 = 0; i2 < n; ++i2)
        for (int i3 = 0; i3 < n; ++i3) {
          const int r1 = fft_rep(i1, n), r2 = fft_rep(i2, n), r3 = fft_rep(i3, n);
          double pv[3];
          for (int d = 0; d < 3; ++d) pv[d] = S.delta[id][d] + (r1 * S.B[0][d] + r2 * S.B[1][d] + r3 * S.B[2][d]);
          const double p2 = pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2];
          const size_t g = ((size_t)i1 * n + i2) * n + i3;
          double* V = &kd.tabV[(size_t)id * 2 * N];
          double* U = &kd.tabU[(size_t)id * 2 * N];
          if (p2 == 0.0) {
            V[g] = v0;
            V[N + g] = v0;   // the adjoint of the discrete right operator keeps V_2a(0)
            U[g] = 0.0;
            U[N + g] = 0.0;
          } else {
            const double lap = ch_lap(p2, ch[0]), gsq = ch_gsq(std::sqrt(p2), ch[0]);
            V[g] = (coul * k4Pi / p2 + lap - gsq) / S.Omega;
            V[N + g] = (coul * k4Pi / p2 - lap - gsq) / S.Omega;
            U[g] = ch_u(p2, ch[0]) / S.Omega;
            U[N + g] = ch_u(p2, ch[1]) / S.Omega;
          }
        }
  // Hartree-type tables at G (G = 0 dropped), both channels summed
  kd.hartV.assign(2 * N, 0.0);
  kd.hartU.assign(N, 0.0);
  kd.hartUs.assign(2 * N, 0.0);
  for (int i1 = 0; i1 < n; ++i1)
    for (int i2 = 0; i2 < n; ++i2)
      for (int i3 = 0; i3 < n; ++i3) {
        const size_t g = ((size_t)i1 * n + i2) * n + i3;
        if (g == 0) continue;
        const int r1 = fft_rep(i1, n), r2 = fft_rep(i2, n), r3 = fft_rep(i3, n);
        double G[3];
        for (int d = 0; d < 3; ++d) G[d] = r1 * S.B[0][d] + r2 * S.B[1][d] + r3 * S.B[2][d];
        const double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
        double vr = 0, vl = 0, u = 0;
        for (int s = 0; s < 2; ++s) {
          const double lap = ch_lap(g2, ch[s]), gsq = ch_gsq(std::sqrt(g2), ch[s]);
          vr += coul * k4Pi / g2 + lap - gsq;
          vl += coul * k4Pi / g2 - lap - gsq;
          const double us = ch_u(g2, ch[s]);
          u += us;
          kd.hartUs[(size_t)s * N + g] = us;
        }
        kd.hartV[g] = vr / S.Omega;
        kd.hartV[N + g] = vl / S.Omega;
        kd.hartU[g] = u / S.Omega;
      }
}

}  // namespace tc
