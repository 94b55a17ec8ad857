// Crystal symmetry (tc_set_symmetry, tc_symmetrize_orbitals).
//
// Sec. 2.3 (end) and Sec. 2.6.4: with symmorphic operations x -> S x
// (fractional coordinates, no translation) and optionally time reversal, the
// orbitals of a k-point k = tr S^T k0 - K follow from those of the irreducible
// point k0,
//   phi~_k(tr S^T m0 + K) = phi~_k0(m0)      (conjugated when tr = -1),
// and so do the occupied-pair fields h3 (3a4 kind and 3b kind) and the h6
// contribution of each q2; the occupied-pair stage then runs over irreducible
// q2 only and the other q2 are unfolded on the real-space grid (k_unfold,
// k_reduce_a4).  The map takes the mesh points in order: a point that no
// earlier irreducible point reaches is irreducible, and its images under the
// operations (then, with time reversal, under the operations times -1), tried
// in the given order, assign the points they reach first.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "tc_ctx.hpp"

namespace tc {

void free_symmetry(tc_ctx* c) {
  void* ptrs[] = {c->d_irr, c->d_symk, c->d_symrot, c->d_star_off, c->d_star_k, c->d_sym_src, c->d_symcart64,
                  c->d_symcart32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  c->d_irr = c->d_symk = c->d_symrot = c->d_star_off = c->d_star_k = c->d_sym_src = nullptr;
  c->d_symcart64 = nullptr;
  c->d_symcart32 = nullptr;
  c->sym = 0;
  c->nirr = 0;
}

int pick_split_for(int items, int partners, int device);
int rebuild_workspace(tc_ctx* c);

}  // namespace tc

namespace {

tc_status sfail(tc_ctx* c, tc_status s, const std::string& m) { return tc::fail(c, s, m); }

__global__ void k_sym_orbitals(double2* phi, double2* chi, const int* __restrict__ symk, const int* __restrict__ src,
                               int Nk, int nb, int npw_max) {
  const size_t total = (size_t)Nk * nb * npw_max;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / ((size_t)nb * npw_max));
    const int b = (int)((e / npw_max) % nb), i = (int)(e % npw_max);
    const int* m = symk + 6 * k;
    if (m[0] == k) continue;
    const int s = src[(size_t)k * npw_max + i];
    double2 p = make_double2(0.0, 0.0), q = make_double2(0.0, 0.0);
    if (s >= 0) {
      const size_t from = ((size_t)m[0] * nb + b) * npw_max + s;
      p = phi[from];
      if (chi) q = chi[from];
      if (m[2] < 0) {
        p.y = -p.y;
        q.y = -q.y;
      }
    }
    phi[e] = p;
    if (chi) chi[e] = q;
  }
}

}  // namespace

namespace tc {
int launch_sym_unfold(tc_ctx* c, double2* a, double2* b, cudaStream_t st) {
  if (!a) {
    a = b;
    b = nullptr;
  }
  if (!a) return TC_OK;
  k_sym_orbitals<<<2 * 152, 256, 0, st>>>(a, b, c->d_symk, c->d_sym_src, c->S.Nk, c->S.nb, c->S.npw_max);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->err = std::string("k_sym_orbitals: ") + cudaGetErrorString(e);
    return TC_ERR_CUDA;
  }
  return TC_OK;
}
}  // namespace tc

extern "C" {

tc_status tc_set_symmetry(tc_ctx* c, int nops, const int* rot, int time_reversal) {
  if (!c) return TC_ERR_STATE;
  if (c->batch || !c->ws_owned || c->S.nkb > 0)
    return sfail(c, TC_ERR_STATE, "symmetry needs a single-cell context from tc_init");
  if (nops < 0 || (nops > 0 && !rot)) return sfail(c, TC_ERR_ARG, "bad operation list");
  tc::free_symmetry(c);
  c->sym_ops.clear();
  c->sym_tr = 0;
  ++c->sym_version;
  if (nops == 0) {
    tc::choose_splits(c);   // never above the split the workspace was laid out for
    return TC_OK;
  }
  const tc::Setup& S = c->S;
  const int Nk = S.Nk, n = S.n;
  // 1. every operation keeps the lattice metric L L^T and maps the k mesh onto itself
  double Mt[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      Mt[a][b] = 0.0;
      for (int d = 0; d < 3; ++d) Mt[a][b] += S.A[a][d] * S.A[b][d];
    }
  double mscale = 0.0;
  for (auto& row : Mt)
    for (double v : row) mscale = std::max(mscale, std::fabs(v));
  for (int o = 0; o < nops; ++o) {
    const int* R = rot + 9 * o;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double v = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) v += R[3 * i + a] * Mt[i][j] * R[3 * j + b];
        if (std::fabs(v - Mt[a][b]) > 1e-9 * mscale)
          return sfail(c, TC_ERR_ARG, "operation " + std::to_string(o) + " does not keep the lattice metric");
      }
  }
  bool has_identity = false;
  for (int o = 0; o < nops && !has_identity; ++o) {
    const int* R = rot + 9 * o;
    has_identity = R[0] == 1 && R[4] == 1 && R[8] == 1 && R[1] == 0 && R[2] == 0 && R[3] == 0 && R[5] == 0 &&
                   R[6] == 0 && R[7] == 0;
  }
  if (!has_identity) return sfail(c, TC_ERR_ARG, "the operations must include the identity");
  // 2. the k map
  std::vector<int> k0(Nk, -1), op(Nk, 0), tr(Nk, 1), K(3 * Nk, 0), irr;
  const int nsign = time_reversal ? 2 : 1;
  for (int a = 0; a < Nk; ++a) {
    if (k0[a] >= 0) continue;
    irr.push_back(a);
    for (int sg = 0; sg < nsign; ++sg) {
      const int t = sg == 0 ? 1 : -1;
      for (int o = 0; o < nops; ++o) {
        const int* R = rot + 9 * o;
        double kap[3];
        for (int i = 0; i < 3; ++i)   // S^T kappa0
          kap[i] = t * (R[i] * S.kfrac[a][0] + R[3 + i] * S.kfrac[a][1] + R[6 + i] * S.kfrac[a][2]);
        int hit = -1, nhit = 0;
        for (int j = 0; j < Nk; ++j) {
          bool same = true;
          for (int i = 0; i < 3; ++i) {
            const double d = kap[i] - S.kfrac[j][i];
            if (std::fabs(d - std::round(d)) > 1e-9) same = false;
          }
          if (same) { hit = j; ++nhit; }
        }
        if (nhit != 1) return sfail(c, TC_ERR_ARG, "operation " + std::to_string(o) + " does not map the k mesh onto itself");
        if (k0[hit] < 0) {
          k0[hit] = a;
          op[hit] = o;
          tr[hit] = t;
          for (int i = 0; i < 3; ++i) K[3 * hit + i] = (int)std::lround(kap[i] - S.kfrac[hit][i]);
        }
      }
    }
  }
  // 3. sphere gather table, and the no-wrap condition of the pair densities
  std::vector<int> src((size_t)Nk * S.npw_max, -1);
  for (int k = 0; k < Nk; ++k) {
    if (k0[k] == k) continue;
    const int a = k0[k];
    if (S.npw[a] != S.npw[k]) return sfail(c, TC_ERR_ARG, "sphere sizes differ between symmetry-related k-points");
    std::map<long long, int> pos;
    auto key = [](int x, int y, int z) { return ((long long)(x + 4096) * 8192 + (y + 4096)) * 8192 + (z + 4096); };
    for (int i = 0; i < S.npw[k]; ++i) pos[key(S.miller[k][i][0], S.miller[k][i][1], S.miller[k][i][2])] = i;
    const int* R = rot + 9 * op[k];
    for (int i0 = 0; i0 < S.npw[a]; ++i0) {
      int m[3];
      for (int i = 0; i < 3; ++i)
        m[i] = tr[k] * (R[i] * S.miller[a][i0][0] + R[3 + i] * S.miller[a][i0][1] + R[6 + i] * S.miller[a][i0][2]) +
               K[3 * k + i];
      auto it = pos.find(key(m[0], m[1], m[2]));
      if (it == pos.end()) return sfail(c, TC_ERR_ARG, "operation does not map the plane-wave spheres onto each other");
      src[(size_t)k * S.npw_max + it->second] = i0;
    }
  }
  for (int i = 0; i < 3; ++i) {
    int lo = 1 << 30, hi = -(1 << 30);
    for (int k = 0; k < Nk; ++k)
      for (int g = 0; g < S.npw[k]; ++g) {
        lo = std::min(lo, S.miller[k][g][i]);
        hi = std::max(hi, S.miller[k][g][i]);
      }
    if (hi - lo > (n % 2 == 0 ? n / 2 - 1 : (n - 1) / 2))
      return sfail(c, TC_ERR_UNSUPPORTED, "FFT box too small for the symmetry reduction (pair densities wrap)");
  }
  // 4. stars, Cartesian S^dagger = (L^T S L^-T)^T
  std::vector<int> star_off(1, 0), star_k;
  for (size_t b = 0; b < irr.size(); ++b) {
    for (int k = 0; k < Nk; ++k)
      if (k0[k] == irr[b]) star_k.push_back(k);
    star_off.push_back((int)star_k.size());
  }
  double Linv[3][3];
  {
    const double(*L)[3] = S.A;
    const double det = L[0][0] * (L[1][1] * L[2][2] - L[1][2] * L[2][1]) - L[0][1] * (L[1][0] * L[2][2] - L[1][2] * L[2][0]) +
                       L[0][2] * (L[1][0] * L[2][1] - L[1][1] * L[2][0]);
    Linv[0][0] = (L[1][1] * L[2][2] - L[1][2] * L[2][1]) / det;
    Linv[0][1] = (L[0][2] * L[2][1] - L[0][1] * L[2][2]) / det;
    Linv[0][2] = (L[0][1] * L[1][2] - L[0][2] * L[1][1]) / det;
    Linv[1][0] = (L[1][2] * L[2][0] - L[1][0] * L[2][2]) / det;
    Linv[1][1] = (L[0][0] * L[2][2] - L[0][2] * L[2][0]) / det;
    Linv[1][2] = (L[0][2] * L[1][0] - L[0][0] * L[1][2]) / det;
    Linv[2][0] = (L[1][0] * L[2][1] - L[1][1] * L[2][0]) / det;
    Linv[2][1] = (L[0][1] * L[2][0] - L[0][0] * L[2][1]) / det;
    Linv[2][2] = (L[0][0] * L[1][1] - L[0][1] * L[1][0]) / det;
  }
  std::vector<double> cart64(9 * (size_t)nops);
  std::vector<float> cart32(9 * (size_t)nops);
  for (int o = 0; o < nops; ++o) {
    const int* R = rot + 9 * o;
    // S_c = L^T R L^-T: S_c[a][b] = sum_ij L[i][a] R[i][j] Linv[b][j]
    double Sc[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double v = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) v += S.A[i][a] * R[3 * i + j] * Linv[b][j];
        Sc[a][b] = v;
      }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        cart64[9 * o + 3 * a + b] = Sc[b][a];
        cart32[9 * o + 3 * a + b] = (float)Sc[b][a];
      }
  }
  std::vector<int> symk(6 * (size_t)Nk);
  for (int k = 0; k < Nk; ++k) {
    symk[6 * k] = k0[k];
    symk[6 * k + 1] = op[k];
    symk[6 * k + 2] = tr[k];
    for (int i = 0; i < 3; ++i) symk[6 * k + 3 + i] = K[3 * k + i];
  }
  // 5. partner chunks of the reduced launch; a larger count needs a larger workspace
  const int nirr = (int)irr.size();
  int so[2];
  for (int sides = 1; sides <= 2; ++sides)
    so[sides - 1] = tc::pick_split_for(nirr * S.no * sides, Nk * S.no, c->device);
  int sc[2];
  for (int sides = 1; sides <= 2; ++sides)
    sc[sides - 1] = tc::pick_split_for(nirr * S.nb * sides, Nk * S.no, c->device);
  const int so_old[2] = {c->split_occ[0], c->split_occ[1]}, so_max_old = c->so_max;
  const int sc_old[2] = {c->split_chain[0], c->split_chain[1]}, sc_max_old = c->sc_max;
  c->split_occ[0] = so[0];
  c->split_occ[1] = so[1];
  c->split_chain[0] = sc[0];
  c->split_chain[1] = sc[1];
  c->so_max = std::max(so_max_old, std::max(so[0], so[1]));
  c->sc_max = std::max(sc_max_old, std::max(sc[0], sc[1]));
  if (c->so_max != so_max_old || c->sc_max != sc_max_old) {
    const int r = tc::rebuild_workspace(c);
    if (r != TC_OK) {
      c->split_occ[0] = so_old[0];
      c->split_occ[1] = so_old[1];
      c->split_chain[0] = sc_old[0];
      c->split_chain[1] = sc_old[1];
      c->so_max = so_max_old;
      c->sc_max = sc_max_old;
      tc::rebuild_workspace(c);
      return (tc_status)r;
    }
  }
  // 6. device tables
  cudaError_t e = cudaSuccess;
  auto up = [&](void** dst, const void* h, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, h, bytes, cudaMemcpyHostToDevice);
  };
  up((void**)&c->d_irr, irr.data(), irr.size() * sizeof(int));
  up((void**)&c->d_symk, symk.data(), symk.size() * sizeof(int));
  up((void**)&c->d_symrot, rot, 9 * (size_t)nops * sizeof(int));
  up((void**)&c->d_star_off, star_off.data(), star_off.size() * sizeof(int));
  up((void**)&c->d_star_k, star_k.data(), star_k.size() * sizeof(int));
  up((void**)&c->d_sym_src, src.data(), src.size() * sizeof(int));
  up((void**)&c->d_symcart64, cart64.data(), cart64.size() * sizeof(double));
  up((void**)&c->d_symcart32, cart32.data(), cart32.size() * sizeof(float));
  if (e != cudaSuccess) {
    tc::free_symmetry(c);
    cudaGetLastError();
    return sfail(c, e == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA,
                 std::string("symmetry tables: ") + cudaGetErrorString(e));
  }
  c->nirr = nirr;
  c->sym = 1;
  c->sym_ops.assign(rot, rot + 9 * (size_t)nops);
  c->sym_tr = time_reversal ? 1 : 0;
  return TC_OK;
}

tc_status tc_symmetry_info(const tc_ctx* c, int* nirr, int* kmap6) {
  if (!c) return TC_ERR_STATE;
  if (nirr) *nirr = c->sym ? c->nirr : c->S.Nk;
  if (kmap6 && c->sym &&
      cudaMemcpy(kmap6, c->d_symk, 6 * (size_t)c->S.Nk * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return TC_ERR_CUDA;
  if (kmap6 && !c->sym)
    for (int k = 0; k < c->S.Nk; ++k) {
      const int v[6] = {k, 0, 1, 0, 0, 0};
      std::memcpy(kmap6 + 6 * k, v, sizeof(v));
    }
  return TC_OK;
}

tc_status tc_symmetrize_orbitals(tc_ctx* c, void* phi, void* chi, void* stream) {
  if (!c) return TC_ERR_STATE;
  if (!c->sym) return sfail(c, TC_ERR_STATE, "no symmetry set (tc_set_symmetry)");
  if (!phi || !chi) return sfail(c, TC_ERR_ARG, "null orbital pointer");
  const tc::Setup& S = c->S;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t orb = (size_t)S.Nk * S.nb * S.npw_max * sizeof(double2);
  const bool hp = !tc::device_ptr(phi), hc = !tc::device_ptr(chi);
  double2* dp = hp ? c->d_in_phi : static_cast<double2*>(phi);
  double2* dc = hc ? c->d_in_chi : static_cast<double2*>(chi);
  cudaError_t e = cudaSuccess;
  if (hp) e = cudaMemcpyAsync(dp, phi, orb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && hc) e = cudaMemcpyAsync(dc, chi, orb, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return sfail(c, TC_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
  k_sym_orbitals<<<2 * 152, 256, 0, st>>>(dp, dc, c->d_symk, c->d_sym_src, S.Nk, S.nb, S.npw_max);
  if ((e = cudaGetLastError()) != cudaSuccess) return sfail(c, TC_ERR_CUDA, std::string("k_sym_orbitals: ") + cudaGetErrorString(e));
  if (hp) e = cudaMemcpyAsync(phi, dp, orb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && hc) e = cudaMemcpyAsync(chi, dc, orb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && (hp || hc)) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return sfail(c, TC_ERR_CUDA, std::string("tc_symmetrize_orbitals: ") + cudaGetErrorString(e));
  return TC_OK;
}

}  // extern "C"
