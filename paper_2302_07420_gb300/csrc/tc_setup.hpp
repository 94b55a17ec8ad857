// Host-side setup of the TC operator: cell, k mesh, plane-wave spheres, FFT
// box maps, the divergence-correction constant and the FP64 kernel tables.
#pragma once
#include <array>
#include <string>
#include <vector>

#include "../../include/tc.h"

namespace tc {

struct Setup {
  tc_params prm{};
  double A[3][3]{};        // lattice rows a_i
  double B[3][3]{};        // reciprocal rows b_i, a_i . b_j = 2 pi delta_ij
  double Omega = 0.0;
  int Nk = 0, n = 0, N = 0, nb = 0, no = 0;
  // band-structure k-points (add_band_points): nkb points after the Nk mesh points carry output
  // orbitals only; Nkt = Nk + nkb k-points have orbitals (kfrac, kcart, miller, npw, box_index,
  // and both indices of delta_id run over them)
  int nkb = 0, Nkt = 0;
  std::vector<double> gamma_b;                          // [nkb] Gamma_b of each band point
  std::vector<std::array<double, 3>> Wb;                // [nkb] W of each band point
  std::vector<std::array<double, 3>> kfrac, kcart;
  std::vector<std::vector<std::array<int, 3>>> miller;   // per k, lexicographic
  std::vector<int> npw;
  int npw_max = 0;
  std::vector<int> miller_flat;                          // [Nk][npw_max][3], zero padded
  std::vector<int> box_index;                            // [Nk][npw_max], -1 padded
  double alpha = 0.0, Gamma0 = 0.0;
  // distinct Delta = k_out - k_part (unreduced)
  int ndelta = 0;
  std::vector<int> delta_id;                             // [Nkt][Nkt] (row: output k, column: partner k)
  std::vector<std::array<double, 3>> delta;              // Cartesian
  // FP64 tables, all divided by Omega, over the box in global (unpadded) order
  std::vector<double> tabV;    // [ndelta][2][N]  V_2a (right), V_2a^dagger (left), p = 0 value incl. correction
  std::vector<double> tabU;    // [ndelta][2][N]  u~_pp, u~_ap (0 at p = 0)
  std::vector<double> hartV;   // [2][N]          (V_pp + V_ap)(G) right / left, 0 at G = 0
  std::vector<double> hartU;   // [N]             (u~pp + u~ap)(G), 0 at G = 0
  std::vector<double> hartUs;  // [2][N]          u~_s(G) (NOT divided by Omega), 0 at G = 0
  double corr_c[2]{};          // (4 pi A_s)^2 Gamma0 + x 4 pi A_s u_short,s / Nk
  double amp[2]{};             // A_s as used by the corrections (4 pi A_s / Nk)
};

// The Jastrow-dependent kernel data: the tables of Setup and the correction
// scalars.  mode -1: values at (A, C); mode 0..3: their derivatives with
// respect to A_pp, A_ap, C_pp, C_ap (zero for the other channel and for the
// Coulomb part).
struct KernelData {
  std::vector<double> tabV, tabU, hartV, hartU, hartUs;
  double corr_c[2]{}, amp[2]{};
};
enum { KD_VALUE = -1, KD_DA_PP = 0, KD_DA_AP = 1, KD_DC_PP = 2, KD_DC_AP = 3 };
void kernel_data(const Setup& S, int mode, KernelData& kd);

// Returns an empty string on success, otherwise the reason.
std::string build_setup(const tc_params& p, Setup& S);
// Appends nkb band-structure k-points (fractional coordinates kfrac_band[3 b + i]) to a built setup as
// output-only points: their spheres, the Delta tables of every band/mesh pair and the band constants
// Gamma_b and W (band_constants).  A point on the SCF mesh modulo a reciprocal vector is refused (it
// takes the SCF corrections).  Returns an empty string on success, otherwise the reason.
std::string add_band_points(Setup& S, int nkb, const double* kfrac_band);

// Constants of the divergence corrections at a band-structure k-point off the SCF mesh
// (Sec. 2.6.3 after Eq. divcorr_2ax_scf; Eqs. divcorr_2ax_band, correction_nabla), for
// kcart = k: gamma_b = Omega/(4 sqrt(pi^3 alpha)) - (1/Nk) sum_{q,G} A_aux(k - q + G) and
// W = sum_{q,G} (k - q + G) A_aux(k - q + G), A_aux(p) = exp(-alpha p^2)/p^2, q over the SCF mesh.
// Returns false when some k - q + G vanishes (k on the mesh).
bool band_constants(const Setup& S, const double kcart[3], double* gamma_b, double W[3]);

// The plane-wave sphere |k + m.B|^2/2 <= ecut of the wave vector kcart, Miller vectors m in
// lexicographic order (the order of every sphere of the library).  Returns false when a vector
// does not fit the FFT box (|m_i| > (n - 1)/2).  S needs only the lattice and the parameters.
bool sphere(const Setup& S, const double kcart[3], std::vector<std::array<int, 3>>& out);

// Default partner chunks per CTA item: the s in 1 .. min(8, partners) whose launch of items x s CTAs
// fills its last wave on `sms` SMs best (a larger s must raise the filled fraction by more than 1 %).
int pick_split(int items, int partners, int sms);
// The autotuner's rule over measured times t[1..n]: the smallest s within 2 % of the fastest, so that
// near-ties go the same way from run to run and fewer chunks (fewer partial sums) win them.
int smallest_near_best(const double* t, int n);

// Largest per-axis Miller span (max - min over the union of all spheres): a pair density
// chi_q^* phi_j has its spectrum at Miller differences -span .. span on each axis.
int miller_span(const std::vector<std::vector<std::array<int, 3>>>& miller);
// Whether the left occupied-pair fields are exactly the conjugates of the right ones on this grid
// (see k_left_from_right): an odd box, or pair densities clear of the Nyquist planes (span <= n/2 - 1).
bool left_from_right_exact(int n, int span);
// Box indices per axis that a pair-density spectrum can occupy: min(n, 2 span + 1).  The pruned
// transforms of the pair chains apply when this is at most their compiled support length.
int pair_support_len(int n, int span);
// Bytes of the reflection buffer of mirrored two-sided pair chains (k_pair_chain_pr, mirror), or 0
// for none: FP64 contexts on the SCF mesh (no band points) whose pair chains take the pruned
// transforms (0 < prune_L, pair_support <= prune_L), (Nk no)^2 x 2 x prune_L^3 complex FP64 values,
// allocated only when that is at most a quarter of free_bytes.
size_t mirror_buffer_bytes(bool fp64, int nkb, int prune_L, int pair_support, int Nk, int no, size_t free_bytes);

// Appendix B kernel pieces (host, FP64), exposed for the table tests.
double host_u_tilde(double p2, double A, double C);
double host_gradu_sq(double p, double A, double C);

}  // namespace tc
