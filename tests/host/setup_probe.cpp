// Test probe of the library's host setup (csrc/tc_setup.cpp): builds the FP64 tables for the
// parameters given on the command line and writes them as raw doubles for the Python test to compare
// with the oracle.  Usage: setup_probe out.bin a11 a12 ... a33 k1 k2 k3 ecut n nbands nocc
//                          App Aap Cpp Cap alpha div ushort_factor
// Output, all float64: Omega, alpha, Gamma0, ndelta, corr_c[2], Nk, N; delta_id[Nk*Nk];
// delta[ndelta][3]; tabV[ndelta][2][N]; tabU[ndelta][2][N]; hartV[2][N]; hartU[N]; hartUs[2][N];
// then the layout: npw_max, npw[Nk], miller_flat[Nk][npw_max][3], box_index[Nk][npw_max];
// then for each derivative mode KD_DA_PP, KD_DA_AP, KD_DC_PP, KD_DC_AP the same five tables
// followed by corr_c[2], amp[2]; then host_gradu_sq at p = 0 for the parallel-spin channel; then
// the band constants at the fractional k (0.13, 0.27, -0.31): found (1 or 0), Gamma_b, W[3].
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "tc_setup.hpp"

int main(int argc, char** argv) {
  if (argc != 2 + 9 + 3 + 1 + 1 + 2 + 4 + 3) {
    std::fprintf(stderr, "wrong number of arguments\n");
    return 2;
  }
  int a = 2;
  tc_params p{};
  for (int i = 0; i < 9; ++i) p.lattice[i / 3][i % 3] = std::atof(argv[a++]);
  for (int i = 0; i < 3; ++i) p.kmesh[i] = std::atoi(argv[a++]);
  p.ecut_ha = std::atof(argv[a++]);
  const int n = std::atoi(argv[a++]);
  p.fft[0] = p.fft[1] = p.fft[2] = n;
  p.nbands = std::atoi(argv[a++]);
  p.nocc = std::atoi(argv[a++]);
  for (int s = 0; s < 2; ++s) p.A[s] = std::atof(argv[a++]);
  for (int s = 0; s < 2; ++s) p.C[s] = std::atof(argv[a++]);
  p.alpha = std::atof(argv[a++]);
  p.div_correction = std::atoi(argv[a++]);
  p.ushort_factor = std::atof(argv[a++]);
  p.precision = TC_FP64;
  tc::Setup S;
  const std::string why = tc::build_setup(p, S);
  if (!why.empty()) {
    std::fprintf(stderr, "%s\n", why.c_str());
    return 1;
  }
  std::vector<double> out = {S.Omega, S.alpha, S.Gamma0, (double)S.ndelta, S.corr_c[0], S.corr_c[1],
                             (double)S.Nk, (double)S.N};
  for (int v : S.delta_id) out.push_back(v);
  for (const auto& d : S.delta) out.insert(out.end(), d.begin(), d.end());
  for (const std::vector<double>* t : {&S.tabV, &S.tabU, &S.hartV, &S.hartU, &S.hartUs})
    out.insert(out.end(), t->begin(), t->end());
  out.push_back(S.npw_max);
  for (int k = 0; k < S.Nk; ++k) out.push_back(S.npw[k]);
  for (int v : S.miller_flat) out.push_back(v);
  for (int v : S.box_index) out.push_back(v);
  for (int mode : {tc::KD_DA_PP, tc::KD_DA_AP, tc::KD_DC_PP, tc::KD_DC_AP}) {
    tc::KernelData kd;
    tc::kernel_data(S, mode, kd);
    for (const std::vector<double>* t : {&kd.tabV, &kd.tabU, &kd.hartV, &kd.hartU, &kd.hartUs})
      out.insert(out.end(), t->begin(), t->end());
    out.insert(out.end(), {kd.corr_c[0], kd.corr_c[1], kd.amp[0], kd.amp[1]});
  }
  out.push_back(tc::host_gradu_sq(0.0, p.A[0], p.C[0]));
  const double kf[3] = {0.13, 0.27, -0.31};
  double kc[3], gb = 0.0, W[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < 3; ++d) kc[d] = kf[0] * S.B[0][d] + kf[1] * S.B[1][d] + kf[2] * S.B[2][d];
  const bool found = tc::band_constants(S, kc, &gb, W);
  out.insert(out.end(), {found ? 1.0 : 0.0, gb, W[0], W[1], W[2]});
  FILE* f = std::fopen(argv[1], "wb");
  if (!f) return 3;
  const size_t w = std::fwrite(out.data(), sizeof(double), out.size(), f);
  std::fclose(f);
  return w == out.size() ? 0 : 4;
}
