// Test probe of the library's host setup (csrc/tc_setup.cpp): builds the FP64 tables for the
// parameters given on the command line and writes them as raw doubles for the Python test to compare
// with the oracle.  Usage: setup_probe out.bin a11 a12 ... a33 k1 k2 k3 ecut n nbands nocc
//                          App Aap Cpp Cap alpha div ushort_factor
// Output, all float64: Omega, alpha, Gamma0, ndelta, corr_c[2], Nk, N; delta_id[Nk*Nk];
// delta[ndelta][3]; tabV[ndelta][2][N]; tabU[ndelta][2][N]; hartV[2][N]; hartU[N]; hartUs[2][N].
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
  FILE* f = std::fopen(argv[1], "wb");
  if (!f) return 3;
  const size_t w = std::fwrite(out.data(), sizeof(double), out.size(), f);
  std::fclose(f);
  return w == out.size() ? 0 : 4;
}
