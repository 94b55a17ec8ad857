// C ABI of the TC operator library (see include/tc.h).
#include <algorithm>
#include <array>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tc_ctx.hpp"
#include "tc_kernels.cuh"

using tc::NT;

namespace {

thread_local std::string g_init_err;   // reason of the last failed tc_init on this thread
void term_weights(const tc_ctx* c, double* tw, double two, double three);

// Box sizes with compiled specialisations.
#define TC_FOR_N(X) X(9) X(12) X(15) X(16) X(18) X(20) X(24) X(25) X(27) X(30) X(32) X(48)

template <typename T> int dispatch_prepare(tc_ctx* c, int n) {
#define CASE(NN) \
  case NN: return tc::prepare_kernels<T, NN>(c);
  switch (n) { TC_FOR_N(CASE) }
#undef CASE
  return TC_ERR_UNSUPPORTED;
}

template <typename T> size_t dispatch_scratch(const tc::Setup& S, int n, int so_max, int sc_max) {
#define CASE(NN) \
  case NN: return tc::scratch_needed<T, NN>(S, so_max, sc_max);
  switch (n) { TC_FOR_N(CASE) }
#undef CASE
  return 0;
}

template <typename T>
int dispatch_run(tc_ctx* c, const double2* a, const double2* b, double2* oR, double2* oL, const double* tw, int ns,
                 cudaStream_t st) {
#define CASE(NN) \
  case NN: return tc::run_pipeline<T, NN>(c, a, b, oR, oL, tw, ns, st);
  switch (c->S.n) { TC_FOR_N(CASE) }
#undef CASE
  return TC_ERR_UNSUPPORTED;
}

template <typename T>
int dispatch_run_band(tc_ctx* c, const double2* a, const double2* b, const double2* ba, const double2* bb, double2* oR,
                      double2* oL, const double* tw, cudaStream_t st) {
#define CASE(NN) \
  case NN: return tc::run_pipeline<T, NN>(c, a, b, oR, oL, tw, 2, st, ba, bb);
  switch (c->S.n) { TC_FOR_N(CASE) }
#undef CASE
  return TC_ERR_UNSUPPORTED;
}

template <typename T> int dispatch_fft(int n, void* data, int batch, int sign, cudaStream_t st) {
#define CASE(NN) \
  case NN: return tc::run_fft3d<T, NN>(data, batch, sign, st);
  switch (n) { TC_FOR_N(CASE) }
#undef CASE
  return TC_ERR_UNSUPPORTED;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

tc_status fail(tc_ctx* c, tc_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

tc_status cuda_fail(tc_ctx* c, cudaError_t e, const char* where) {
  return fail(c, TC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T> void* upload_as(const std::vector<double>& v, cudaError_t& err) {
  std::vector<T> h(v.size());
  for (size_t i = 0; i < v.size(); ++i) h[i] = (T)v[i];
  void* d = nullptr;
  err = cudaMalloc(&d, h.size() * sizeof(T) + 16);
  if (err != cudaSuccess) return nullptr;
  err = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return d;
}

void free_all(tc_ctx* c) {
  void* ptrs[] = {c->d_box_index, c->d_kpg, c->d_delta_id, c->d_delta, c->d_tabV, c->d_tabU, c->d_hartV,
                  c->d_hartU, c->d_hartUs, c->d_occ, c->ws_owned ? c->d_ws : nullptr, c->d_in_phi, c->d_in_chi,
                  c->d_out_R, c->d_out_L, c->d_edot, c->d_npw, c->d_status, c->d_band, c->d_bs, c->d_kd64,
                  c->d_mirror};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->occ_ev) cudaEventDestroy(c->occ_ev);
  if (c->h_occ) cudaFreeHost(c->h_occ);
  if (c->h_edot) cudaFreeHost(c->h_edot);
  if (c->h_status) cudaFreeHost(c->h_status);
}

// e[j] = sum_G conj(c_chi) (kin |k+G|^2/2 c_phi + out), FP64
__global__ void k_energy_dot(const double2* __restrict__ cphi, const double2* __restrict__ cchi,
                             const double2* __restrict__ out, const double* __restrict__ kpg, int npw_max, int nb,
                             int kin, double2* e) {
  __shared__ double rx[32], ry[32];
  const int j = blockIdx.x, k = j / nb;
  double sx = 0, sy = 0;
  for (int g = threadIdx.x; g < npw_max; g += blockDim.x) {
    const double2 x = cchi[(size_t)j * npw_max + g];
    double2 v = out ? out[(size_t)j * npw_max + g] : make_double2(0.0, 0.0);
    if (kin) {
      const double* q = kpg + ((size_t)k * npw_max + g) * 3;
      const double t = 0.5 * (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
      const double2 p = cphi[(size_t)j * npw_max + g];
      v.x += t * p.x;
      v.y += t * p.y;
    }
    sx += x.x * v.x + x.y * v.y;   // conj(x) v
    sy += x.x * v.y - x.y * v.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  if ((threadIdx.x & 31) == 0) { rx[threadIdx.x >> 5] = sx; ry[threadIdx.x >> 5] = sy; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ax = 0, ay = 0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) { ax += rx[i]; ay += ry[i]; }
    e[j] = make_double2(ax, ay);
  }
}

// Orbital gradient of E (dE = Re sum conj(g) dc):
//   g_phi = pref f (T chi + out_L),  g_chi = pref f (T phi + out_R),  T = |k+G|^2/2, pref = 2/Nk.
// g_phi may alias out_L and g_chi may alias out_R (each element is read before it is written).
__global__ void k_grad_combine(const double2* __restrict__ cphi, const double2* __restrict__ cchi, const double2* outR,
                               const double2* outL, const double* __restrict__ kpg, const double* __restrict__ occ,
                               int npw_max, int nb, double pref, size_t total, double2* gphi, double2* gchi) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t j = e / npw_max, g = e % npw_max, k = j / nb;
    const double* q = kpg + (k * npw_max + g) * 3;
    const double t = 0.5 * (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    const double w = pref * occ[j];
    if (gphi) {
      const double2 x = cchi[e], o = outL[e];
      gphi[e] = make_double2(w * (t * x.x + o.x), w * (t * x.y + o.y));
    }
    if (gchi) {
      const double2 x = cphi[e], o = outR[e];
      gchi[e] = make_double2(w * (t * x.x + o.x), w * (t * x.y + o.y));
    }
  }
}

// ---------------------------------------------------------------------------
// Biorthonormalisation per k-point (one CTA per k, FP64): modified Gram-Schmidt
// of the right orbitals in band order, then chi_j <- sum_i chi_i (M^-1)_ij with
// M_ij = <phi_i|chi_j> (Gauss-Jordan with partial pivoting on [M | I] in shared
// memory), so that <chi_j|phi_l> = delta_jl.  *status = k + 1 if a norm or a
// pivot vanishes at k-point k.
using tc::kBiorthoMaxBands;

__device__ double2 block_dot(const double2* a, const double2* b, int n, double* red) {
  // sum_g conj(a_g) b_g over the CTA; result valid in every thread
  double sx = 0.0, sy = 0.0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    const double2 x = a[g], y = b[g];
    sx += x.x * y.x + x.y * y.y;
    sy += x.x * y.y - x.y * y.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) { red[2 * w] = sx; red[2 * w + 1] = sy; }
  __syncthreads();
  double tx = 0.0, ty = 0.0;
  for (int i = 0; i < nw; ++i) { tx += red[2 * i]; ty += red[2 * i + 1]; }
  return make_double2(tx, ty);
}

__global__ void k_biortho(double2* phi, double2* chi, const int* __restrict__ npw_k, int npw_max, int nb, int* status) {
  extern __shared__ double2 aug[];   // [nb][2 nb]
  __shared__ double red[64];
  __shared__ double2 fac[kBiorthoMaxBands];
  __shared__ int piv;
  __shared__ int bad;
  const int k = blockIdx.x, n = npw_k[k], w2 = 2 * nb;
  double2* P = phi + (size_t)k * nb * npw_max;
  double2* X = chi + (size_t)k * nb * npw_max;
  if (threadIdx.x == 0) bad = 0;
  // 1. modified Gram-Schmidt of the rows of P
  for (int i = 0; i < nb; ++i) {
    double2* pi = P + (size_t)i * npw_max;
    for (int j = 0; j < i; ++j) {
      const double2* pj = P + (size_t)j * npw_max;
      const double2 r = block_dot(pj, pi, n, red);
      for (int g = threadIdx.x; g < n; g += blockDim.x) {
        const double2 a = pj[g];
        pi[g].x -= r.x * a.x - r.y * a.y;
        pi[g].y -= r.x * a.y + r.y * a.x;
      }
      __syncthreads();
    }
    const double nrm = sqrt(block_dot(pi, pi, n, red).x);
    if (!(nrm > 0.0)) {
      if (threadIdx.x == 0) *status = k + 1;
      return;   // uniform across the CTA
    }
    for (int g = threadIdx.x; g < n; g += blockDim.x) { pi[g].x /= nrm; pi[g].y /= nrm; }
    __syncthreads();
  }
  // 2. [M | I], M_ij = <phi_i|chi_j>
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      const double2 m = block_dot(P + (size_t)i * npw_max, X + (size_t)j * npw_max, n, red);
      if (threadIdx.x == 0) {
        aug[i * w2 + j] = m;
        aug[i * w2 + nb + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
      }
    }
  __syncthreads();
  double mmax = 0.0;
  for (int e = 0; e < nb * nb; ++e) mmax = fmax(mmax, hypot(aug[(e / nb) * w2 + e % nb].x, aug[(e / nb) * w2 + e % nb].y));
  // 3. Gauss-Jordan
  for (int c = 0; c < nb; ++c) {
    if (threadIdx.x == 0) {
      int p = c;
      double best = -1.0;
      for (int r = c; r < nb; ++r) {
        const double v = hypot(aug[r * w2 + c].x, aug[r * w2 + c].y);
        if (v > best) { best = v; p = r; }
      }
      piv = p;
      if (!(best > 1e-13 * mmax)) bad = 1;
    }
    __syncthreads();
    if (bad) {
      if (threadIdx.x == 0) *status = k + 1;
      return;
    }
    const int p = piv;
    if (p != c)
      for (int e = threadIdx.x; e < w2; e += blockDim.x) {
        const double2 t = aug[c * w2 + e];
        aug[c * w2 + e] = aug[p * w2 + e];
        aug[p * w2 + e] = t;
      }
    __syncthreads();
    const double2 d = aug[c * w2 + c];
    const double dd = d.x * d.x + d.y * d.y;
    const double2 inv = make_double2(d.x / dd, -d.y / dd);
    __syncthreads();
    for (int e = threadIdx.x; e < w2; e += blockDim.x) {
      const double2 a = aug[c * w2 + e];
      aug[c * w2 + e] = make_double2(a.x * inv.x - a.y * inv.y, a.x * inv.y + a.y * inv.x);
    }
    for (int r = threadIdx.x; r < nb; r += blockDim.x) fac[r] = aug[r * w2 + c];
    __syncthreads();
    for (int e = threadIdx.x; e < nb * w2; e += blockDim.x) {
      const int r = e / w2, col = e % w2;
      if (r == c) continue;
      const double2 f = fac[r], a = aug[c * w2 + col];
      aug[e].x -= f.x * a.x - f.y * a.y;
      aug[e].y -= f.x * a.y + f.y * a.x;
    }
    __syncthreads();
  }
  // 4. chi_j(G) = sum_i chi_i(G) Minv_ij   (Minv in the right half of aug)
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    double2 x[kBiorthoMaxBands];
    for (int i = 0; i < nb; ++i) x[i] = X[(size_t)i * npw_max + g];
    for (int j = 0; j < nb; ++j) {
      double sx = 0.0, sy = 0.0;
      for (int i = 0; i < nb; ++i) {
        const double2 m = aug[i * w2 + nb + j];
        sx += x[i].x * m.x - x[i].y * m.y;
        sy += x[i].x * m.y + x[i].y * m.x;
      }
      X[(size_t)j * npw_max + g] = make_double2(sx, sy);
    }
  }
}

// y = (T)(x + a dx) elementwise (FP64 arithmetic, one rounding to the compute precision)
template <typename T>
__global__ void k_displace(const double* __restrict__ x, const double* __restrict__ dx, double a, T* __restrict__ y,
                           size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (T)(x[i] + a * dx[i]);
}

// The context's kernel tables set to K + a dK_m on the device (m < 0: K), from the FP64 copies of K and
// of the four derivatives that tc_energy_grad keeps in d_kd64 (set m = 0 .. 3 after the base, set -1).
template <typename T> cudaError_t displace_tables(tc_ctx* c, int m, double a, cudaStream_t st) {
  void* dst[] = {c->d_tabV, c->d_tabU, c->d_hartV, c->d_hartU, c->d_hartUs};
  size_t set = 0;
  for (int i = 0; i < 5; ++i) set += c->kd64_len[i];
  size_t off = 0;
  for (int i = 0; i < 5; ++i) {
    const double* x = c->d_kd64 + off;
    const double* dx = m < 0 ? x : c->d_kd64 + (size_t)(m + 1) * set + off;
    k_displace<T><<<2 * 152, 256, 0, st>>>(x, dx, m < 0 ? 0.0 : a, static_cast<T*>(dst[i]), c->kd64_len[i]);
    off += c->kd64_len[i];
  }
  return cudaGetLastError();
}

}  // namespace

namespace tc {
// Sets the message returned by tc_last_error(NULL) on this thread.
void set_thread_error(const std::string& msg) { g_init_err = msg; }
}  // namespace tc

namespace tc {

WsLayout ws_layout(const tc_ctx* c) {
  const Setup& S = c->S;
  const size_t NN = (size_t)S.N, nj = (size_t)S.Nkt * S.nb, vol = NN * c->esz;   // orbitals of all k-points
  WsLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    const size_t o = off;
    off += bytes;
    return o;
  };
  L.phi = take(nj * vol);
  L.chi = take(nj * vol);
  L.gphi = take(nj * 3 * vol);
  L.gchi = take(nj * 3 * vol);
  L.side_bytes = side_field_vols(S.Nk, S.nb, S.no, c->so_max, c->sc_max, c->nj_out, S.nkb, c->so_band) * vol;
  L.side = take(2 * L.side_bytes);
  L.cs_bytes = (size_t)2 * c->nj_out * S.no * 6 * sizeof(double);
  L.cs = take(L.cs_bytes);
  L.scratch_bytes = c->prec == TC_FP64 ? dispatch_scratch<double>(S, S.n, c->so_max, c->sc_max)
                                       : dispatch_scratch<float>(S, S.n, c->so_max, c->sc_max);
  L.scratch = take(L.scratch_bytes);
  L.total = (off + 255) & ~(size_t)255;
  return L;
}

size_t side_field_vols(int Nk, int nb, int no, int so_max, int sc_max, int nj_out, int nkb, int so_band) {
  // n, m(3), nt, mt(3), vH, h1(3), vb2, t3b1, t3b2, vu(2), spec(3), h5(3), h6, vloc = 25; per occupied
  // state h3a4(3) and h3b(3) per chunk part and Z(3); per output orbital acc(1) and w(3) per part and
  // Y(3); with band points: V2 and V3 (4 per point) and both h3 kinds (3 each) of every band-point occupied
  // orbital per band chunk part
  return 25 + (size_t)Nk * no * 3 * (2 * (size_t)so_max + 1) + (size_t)nj_out * (4 * (size_t)sc_max + 3) +
         (size_t)nkb * (4 + (size_t)no * 6 * so_band);
}

// Number of partner chunks s for a launch of `items` CTA items (per chunk one CTA): the s
// (1 <= s <= min(8, partners)) that fills the last wave of CTAs over the SMs best, the
// smallest such s when several are within 1 %.
void choose_splits(tc_ctx* c) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 1;
  }
  const Setup& S = c->S;
  const int M = S.Nk * S.no, nj = c->nj_out;
  for (int sides = 1; sides <= 2; ++sides) {
    c->split_occ[sides - 1] = pick_split(M * sides, M, sms);
    c->split_chain[sides - 1] = pick_split(nj * sides, M, sms);
  }
  c->so_max = std::max(c->split_occ[0], c->split_occ[1]);
  c->sc_max = std::max(c->split_chain[0], c->split_chain[1]);
  c->so_band = S.nkb > 0 ? pick_split(2 * S.nkb * S.no, M, sms) : 1;
}

int pick_split_for(int items, int partners, int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 1;
  }
  return pick_split(items, partners, sms);
}

// Replaces the owned workspace block by one laid out for the current split counts.
int rebuild_workspace(tc_ctx* c) {
  if (!c->ws_owned) return TC_ERR_STATE;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && c->d_ws) e = cudaFree(c->d_ws);
  c->d_ws = nullptr;
  const WsLayout L = ws_layout(c);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_ws, L.total);
  if (e == cudaSuccess) e = cudaMemset(c->d_ws, 0, L.total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->err = std::string("workspace: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA;
  }
  ws_assign(c, static_cast<char*>(c->d_ws), L);
  return TC_OK;
}

void ws_assign(tc_ctx* c, char* base, const WsLayout& L) {
  c->d_phi = base + L.phi;
  c->d_chi = base + L.chi;
  c->d_gphi = base + L.gphi;
  c->d_gchi = base + L.gchi;
  c->d_side = base + L.side;
  c->side_bytes = L.side_bytes;
  c->d_cs = reinterpret_cast<double*>(base + L.cs);
  c->d_scratch = base + L.scratch;
  c->scratch_bytes = L.scratch_bytes;
}

int init_context(const tc_params* params, bool own_workspace, tc_ctx** out, std::string& err, int nkb,
                 const double* kfrac_band) {
  *out = nullptr;
  tc_ctx* c = new (std::nothrow) tc_ctx();
  if (!c) { err = "host allocation failed"; return TC_ERR_OOM; }
  std::string why = tc::build_setup(*params, c->S);
  if (why.empty() && nkb > 0) why = tc::add_band_points(c->S, nkb, kfrac_band);
  if (!why.empty()) {
    err = why;
    delete c;
    return why.rfind("unsupported", 0) == 0 ? TC_ERR_UNSUPPORTED : TC_ERR_ARG;
  }
  tc::Setup& S = c->S;
  c->nj_out = (S.nkb > 0 ? S.nkb : S.Nk) * S.nb;
  {
    // the left/right conjugation of the occupied-pair fields and the pruned pair-chain transforms
    // both depend on how far the pair-density spectra reach on the box
    const int span = tc::miller_span(S.miller);
    c->left_from_right = tc::left_from_right_exact(S.n, span);
    c->pair_support = tc::pair_support_len(S.n, span);
  }
  if (const int f = injected_fault("alloc")) {
    err = "injected fault (TC_FAULT=alloc): no device memory allocated";
    delete c;
    return f;
  }
  c->prec = params->precision;
  c->esz = c->prec == TC_FP64 ? 16 : 8;
  c->ws_owned = own_workspace;
  cudaGetDevice(&c->device);
  choose_splits(c);
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) { if (r != cudaSuccess && e == cudaSuccess) e = r; return r == cudaSuccess; };
  const size_t nj = (size_t)S.Nk * S.nb;
  // basis
  ok(cudaMalloc((void**)&c->d_box_index, S.box_index.size() * sizeof(int)));
  if (e == cudaSuccess) ok(cudaMemcpy(c->d_box_index, S.box_index.data(), S.box_index.size() * sizeof(int), cudaMemcpyHostToDevice));
  std::vector<double> kpg((size_t)S.Nkt * S.npw_max * 3, 0.0);
  for (int k = 0; k < S.Nkt; ++k)
    for (int g = 0; g < S.npw[k]; ++g)
      for (int d = 0; d < 3; ++d) {
        const auto& m = S.miller[k][g];
        kpg[((size_t)k * S.npw_max + g) * 3 + d] = S.kcart[k][d] + (m[0] * S.B[0][d] + m[1] * S.B[1][d] + m[2] * S.B[2][d]);
      }
  if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_kpg, kpg.size() * sizeof(double)));
  if (e == cudaSuccess) ok(cudaMemcpy(c->d_kpg, kpg.data(), kpg.size() * sizeof(double), cudaMemcpyHostToDevice));
  if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_delta_id, S.delta_id.size() * sizeof(int)));
  if (e == cudaSuccess) ok(cudaMemcpy(c->d_delta_id, S.delta_id.data(), S.delta_id.size() * sizeof(int), cudaMemcpyHostToDevice));
  std::vector<double> dl;
  for (auto& d : S.delta) dl.insert(dl.end(), d.begin(), d.end());
  auto up = [&](const std::vector<double>& v) -> void* {
    if (e != cudaSuccess) return nullptr;
    cudaError_t r = cudaSuccess;
    void* p = c->prec == TC_FP64 ? upload_as<double>(v, r) : upload_as<float>(v, r);
    ok(r);
    return p;
  };
  c->d_delta = up(dl);
  c->d_tabV = up(S.tabV);
  c->d_tabU = up(S.tabU);
  c->d_hartV = up(S.hartV);
  c->d_hartU = up(S.hartU);
  c->d_hartUs = up(S.hartUs);
  // occupations of the mesh points, then (band contexts) of the band points
  const size_t nj_all = (size_t)S.Nkt * S.nb;
  if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_occ, nj_all * sizeof(double)));
  if (e == cudaSuccess) ok(cudaMallocHost((void**)&c->h_occ, nj_all * sizeof(double)));
  if (S.nkb > 0) {
    std::vector<double> band((size_t)S.nkb * 4);
    for (int b = 0; b < S.nkb; ++b) {
      for (int d = 0; d < 3; ++d) band[4 * b + d] = S.Wb[b][d];
      band[4 * b + 3] = S.gamma_b[b];
    }
    if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_band, band.size() * sizeof(double)));
    if (e == cudaSuccess) ok(cudaMemcpy(c->d_band, band.data(), band.size() * sizeof(double), cudaMemcpyHostToDevice));
    const size_t nbs = (size_t)2 * S.nkb * S.no * S.nb * tc::kBandScalars;
    if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_bs, nbs * sizeof(double2)));
  }
  // workspace: real-space fields, per-side fields, correction scalars, scratch (zeroed once)
  if (own_workspace) {
    const WsLayout L = ws_layout(c);
    if (e == cudaSuccess) ok(cudaMalloc(&c->d_ws, L.total));
    if (e == cudaSuccess) ok(cudaMemset(c->d_ws, 0, L.total));
    if (e == cudaSuccess) ws_assign(c, static_cast<char*>(c->d_ws), L);
  }
  const size_t orb = nj * S.npw_max * sizeof(double2);
  if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_in_phi, orb));
  if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_in_chi, orb));
  if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_out_R, orb));
  if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_out_L, orb));
  if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_edot, nj * sizeof(double2)));
  if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_npw, S.npw.size() * sizeof(int)));
  if (e == cudaSuccess) ok(cudaMemcpy(c->d_npw, S.npw.data(), S.npw.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (e == cudaSuccess) ok(cudaMalloc((void**)&c->d_status, sizeof(int)));
  if (e == cudaSuccess) ok(cudaMallocHost((void**)&c->h_status, sizeof(int)));
  if (e == cudaSuccess) ok(cudaMallocHost((void**)&c->h_edot, nj * sizeof(double2)));
  if (e == cudaSuccess) ok(cudaEventCreateWithFlags(&c->occ_ev, cudaEventDisableTiming));
  if (e != cudaSuccess) {
    err = std::string("tc_init: ") + cudaGetErrorString(e);
    free_all(c);
    delete c;
    return (e == cudaErrorMemoryAllocation) ? TC_ERR_OOM : TC_ERR_CUDA;
  }
  const int r = c->prec == TC_FP64 ? dispatch_prepare<double>(c, S.n) : dispatch_prepare<float>(c, S.n);
  if (r != TC_OK) {
    err = c->err;
    free_all(c);
    delete c;
    return r;
  }
  c->npw_host = S.npw;
  *out = c;
  return TC_OK;
}

void destroy_context(tc_ctx* c) {
  if (!c) return;
  if (c->batch) destroy_batch(c);
  if (c->dav) destroy_davidson(c);
  free_symmetry(c);
  free_all(c);
  delete c;
}

int apply_device(tc_ctx* c, const double2* phi, const double2* chi, double2* outR, double2* outL, cudaStream_t st) {
  return apply_sides(c, phi, chi, outR, outL, 2, st);
}

int apply_sides(tc_ctx* c, const double2* phi, const double2* chi, double2* outR, double2* outL, int nsides,
                cudaStream_t st) {
  double tw[NT];
  term_weights(c, tw, 1.0, 1.0);
  return c->prec == TC_FP64 ? dispatch_run<double>(c, phi, chi, outR, outL, tw, nsides, st)
                            : dispatch_run<float>(c, phi, chi, outR, outL, tw, nsides, st);
}

int stage_occ(tc_ctx* c, const double* occ, cudaStream_t st) {
  const size_t nj = (size_t)c->S.Nk * c->S.nb;
  for (size_t i = 0; i < nj; ++i)
    if (!(occ[i] >= 0.0 && occ[i] <= 1.0)) return ::fail(c, TC_ERR_ARG, "occupations must lie in [0, 1]");
  // the previous upload may not have run yet: h_occ is its source
  if (c->occ_pending) {
    const cudaError_t w = cudaEventSynchronize(c->occ_ev);
    if (w != cudaSuccess) return cuda_fail(c, w, "occupation upload wait");
  }
  std::memcpy(c->h_occ, occ, nj * sizeof(double));
  cudaError_t e = cudaMemcpyAsync(c->d_occ, c->h_occ, nj * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && c->occ_ev) e = cudaEventRecord(c->occ_ev, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "occ upload");
  c->occ_pending = c->occ_ev != nullptr;
  return TC_OK;
}

// Band contexts: mesh occupations [Nk][nb] then band-point occupations [nkb][nb] into c->d_occ.
int stage_occ_band(tc_ctx* c, const double* occ, const double* band_occ, cudaStream_t st) {
  const size_t nm = (size_t)c->S.Nk * c->S.nb, nbnd = (size_t)c->S.nkb * c->S.nb;
  for (size_t i = 0; i < nm; ++i)
    if (!(occ[i] >= 0.0 && occ[i] <= 1.0)) return ::fail(c, TC_ERR_ARG, "occupations must lie in [0, 1]");
  for (size_t i = 0; i < nbnd; ++i)
    if (!(band_occ[i] >= 0.0 && band_occ[i] <= 1.0)) return ::fail(c, TC_ERR_ARG, "band occupations must lie in [0, 1]");
  if (c->occ_pending) {
    const cudaError_t w = cudaEventSynchronize(c->occ_ev);
    if (w != cudaSuccess) return cuda_fail(c, w, "occupation upload wait");
  }
  std::memcpy(c->h_occ, occ, nm * sizeof(double));
  std::memcpy(c->h_occ + nm, band_occ, nbnd * sizeof(double));
  cudaError_t e = cudaMemcpyAsync(c->d_occ, c->h_occ, (nm + nbnd) * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && c->occ_ev) e = cudaEventRecord(c->occ_ev, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "occ upload");
  c->occ_pending = c->occ_ev != nullptr;
  return TC_OK;
}

int launch_biortho(tc_ctx* c, double2* phi, double2* chi, int* status, cudaStream_t st) {
  const Setup& S = c->S;
  const size_t smem = (size_t)S.nb * 2 * S.nb * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_biortho, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_biortho attribute");
  k_biortho<<<S.Nk, 256, smem, st>>>(phi, chi, c->d_npw, S.npw_max, S.nb, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "k_biortho");
  return TC_OK;
}

bool device_ptr(const void* p) { return is_device_ptr(p); }

tc_status fail(tc_ctx* c, tc_status s, const std::string& msg) { return ::fail(c, s, msg); }

int injected_fault(const char* site) {
  const char* v = std::getenv("TC_FAULT");
  if (!v || !site) return TC_OK;
  const std::string f(v), at(site);
  if (at == "alloc" && f == "alloc") return TC_ERR_OOM;
  if (at == "launch" && f == "launch") return TC_ERR_CUDA;
  if (at == "launch" && f == "timeout") return TC_ERR_TIMEOUT;
  if (at == "cluster" && f == "nocluster") return TC_ERR_UNSUPPORTED;
  if (at == "mirror" && f == "nomirror") return TC_ERR_OOM;
  return TC_OK;
}

// The reflection buffer of mirrored two-sided pair chains (tc_ctx::d_mirror): for FP64 contexts
// whose pair chains run the pruned kernels on the SCF mesh, when it takes at most a quarter of the
// free device memory; otherwise (or under TC_FAULT=nomirror, as if it did not fit) none.  (FP32 pair
// chains are bound by the loads of their parallel-spin passes, which the mirror does not remove;
// measured on the 4x4x4 silicon-like cell, the right launch's stores cost more than the left launch
// saves.)
static void alloc_mirror(tc_ctx* c) {
  const Setup& S = c->S;
  if (injected_fault("mirror") != TC_OK) return;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const size_t bytes =
      mirror_buffer_bytes(c->prec == TC_FP64, S.nkb, c->plan_prune_L, c->pair_support, S.Nk, S.no, fr);
  if (bytes == 0) return;
  if (cudaMalloc(&c->d_mirror, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->d_mirror = nullptr;
    return;
  }
  c->mirror_bytes = bytes;
}

}  // namespace tc

extern "C" {

tc_status tc_init(const tc_params* params, tc_ctx** out) {
  if (!params || !out) return TC_ERR_ARG;
  std::string err;
  const int r = tc::init_context(params, true, out, err);
  if (r == TC_OK) tc::alloc_mirror(*out);
  g_init_err = err;
  return (tc_status)r;
}

tc_status tc_layout(const tc_ctx* c, int* nk, int* npw_max, const int** npw_per_k, const int** miller) {
  if (!c) return TC_ERR_STATE;
  if (c->batch) return TC_ERR_STATE;
  if (nk) *nk = c->S.Nkt;   // band contexts: the mesh points, then the band points
  if (npw_max) *npw_max = c->S.npw_max;
  if (npw_per_k) *npw_per_k = c->npw_host.data();
  if (miller) *miller = c->S.miller_flat.data();
  return TC_OK;
}

tc_status tc_setup_scalars(const tc_ctx* c, double out4[4]) {
  if (!c) return TC_ERR_STATE;
  if (c->batch) return TC_ERR_STATE;
  if (!out4) return TC_ERR_ARG;
  out4[0] = c->S.Omega;
  out4[1] = c->S.alpha;
  out4[2] = c->S.Gamma0;
  out4[3] = c->S.ndelta;
  return TC_OK;
}

static tc_status run_common(tc_ctx* c, const void* phi, const void* chi, const double* occ, void* outR, void* outL,
                            const double* tw, int nsides, cudaStream_t st, bool* host_out) {
  const tc::Setup& S = c->S;
  const size_t nj = (size_t)S.Nk * S.nb, orb = nj * S.npw_max * sizeof(double2);
  if (const int f = tc::injected_fault("launch")) return fail(c, (tc_status)f, "injected fault (TC_FAULT): no device work done");
  const int ro = tc::stage_occ(c, occ, st);
  if (ro != TC_OK) return (tc_status)ro;
  cudaError_t e = cudaSuccess;
  const double2* dphi = static_cast<const double2*>(phi);
  const double2* dchi = static_cast<const double2*>(chi);
  if (!is_device_ptr(phi)) {
    e = cudaMemcpyAsync(c->d_in_phi, phi, orb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "phi_R upload");
    dphi = c->d_in_phi;
  }
  if (!is_device_ptr(chi)) {
    e = cudaMemcpyAsync(c->d_in_chi, chi, orb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "phi_L upload");
    dchi = c->d_in_chi;
  }
  double2* oR = static_cast<double2*>(outR);
  double2* oL = static_cast<double2*>(outL);
  *host_out = false;
  if (oR && !is_device_ptr(oR)) { oR = c->d_out_R; *host_out = true; }
  if (oL && !is_device_ptr(oL)) { oL = c->d_out_L; *host_out = true; }
  const int r = c->prec == TC_FP64 ? dispatch_run<double>(c, dphi, dchi, oR, oL, tw, nsides, st)
                                   : dispatch_run<float>(c, dphi, dchi, oR, oL, tw, nsides, st);
  if (r != TC_OK) return (tc_status)r;
  if (outR && oR == c->d_out_R && outR != c->d_out_R) {
    e = cudaMemcpyAsync(outR, oR, orb, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "out_R download");
  }
  if (outL && oL == c->d_out_L && outL != c->d_out_L) {
    e = cudaMemcpyAsync(outL, oL, orb, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "out_L download");
  }
  return TC_OK;
}

// (2/Nk) Re sum_j f_j <chi_j| (kin ? T phi_j : 0) + (with_out ? out_R_j : 0) > in FP64; blocks the host.
static tc_status energy_reduce(tc_ctx* c, const double2* dphi, const double2* dchi, const double* occ, bool kin,
                               bool with_out, cudaStream_t st, double* res) {
  const tc::Setup& S = c->S;
  const int nj = S.Nk * S.nb;
  k_energy_dot<<<nj, 128, 0, st>>>(dphi, dchi, with_out ? c->d_out_R : nullptr, c->d_kpg, S.npw_max, S.nb, kin ? 1 : 0,
                                   c->d_edot);
  cudaError_t e2 = cudaGetLastError();
  if (e2 != cudaSuccess) return cuda_fail(c, e2, "k_energy_dot");
  e2 = cudaMemcpyAsync(c->h_edot, c->d_edot, nj * sizeof(double2), cudaMemcpyDeviceToHost, st);
  if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
  if (e2 != cudaSuccess) return cuda_fail(c, e2, "energy reduction");
  double s = 0.0;
  for (int j = 0; j < nj; ++j) s += occ[j] * c->h_edot[j].x;
  *res = 2.0 / S.Nk * s;
  return TC_OK;
}

}  // extern "C"

namespace {
void term_weights(const tc_ctx* c, double* tw, double two, double three) {
  const unsigned mask = c->S.prm.term_mask;
  for (int t = 0; t < NT; ++t) {
    const bool on = mask == 0u || (mask >> t) & 1u;
    tw[t] = on ? (t < 6 ? two : three) : 0.0;
  }
}
}  // namespace

extern "C" {

tc_status tc_apply(tc_ctx* c, const void* phi, const void* chi, const double* occ, void* outR, void* outL,
                   void* stream) {
  if (!c) return TC_ERR_STATE;
  if (c->batch) return fail(c, TC_ERR_STATE, "batch context: use tc_apply_batch or tc_batch_cell");
  if (c->S.nkb > 0) return fail(c, TC_ERR_STATE, "band context: use tc_apply_band");
  if (!phi || !chi || !occ) return fail(c, TC_ERR_ARG, "null input pointer");
  if (!outR && !outL) return TC_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double tw[NT];
  term_weights(c, tw, 1.0, 1.0);
  bool host_out = false;
  tc_status r = run_common(c, phi, chi, occ, outR, outL, tw, 2, st, &host_out);
  if (r != TC_OK) return r;
  if (host_out) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "tc_apply");
  }
  return TC_OK;
}

tc_status tc_init_band(const tc_params* params, int nkb, const double* kfrac_band, tc_ctx** out) {
  if (!params || !out || !kfrac_band || nkb < 1) {
    g_init_err = "tc_init_band: null pointer or nkb < 1";
    return TC_ERR_ARG;
  }
  std::string err;
  const int r = tc::init_context(params, true, out, err, nkb, kfrac_band);
  g_init_err = err;
  return (tc_status)r;
}

tc_status tc_apply_band(tc_ctx* c, const void* phi, const void* chi, const double* occ, const void* band_phi,
                        const void* band_chi, const double* band_occ, void* outR, void* outL, void* stream) {
  if (!c) return TC_ERR_STATE;
  if (c->S.nkb == 0) return fail(c, TC_ERR_STATE, "not a band context (tc_init_band)");
  if (!phi || !chi || !occ || !band_phi || !band_chi || !band_occ) return fail(c, TC_ERR_ARG, "null input pointer");
  if (!outR && !outL) return TC_OK;
  for (const void* p : {phi, chi, band_phi, band_chi, (const void*)outR, (const void*)outL})
    if (p && !is_device_ptr(p)) return fail(c, TC_ERR_ARG, "band launches take device pointers only");
  if (const int f = tc::injected_fault("launch")) return fail(c, (tc_status)f, "injected fault (TC_FAULT): no device work done");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ro = tc::stage_occ_band(c, occ, band_occ, st);
  if (ro != TC_OK) return (tc_status)ro;
  double tw[NT];
  term_weights(c, tw, 1.0, 1.0);
  const double2* a = static_cast<const double2*>(phi);
  const double2* b = static_cast<const double2*>(chi);
  const double2* ba = static_cast<const double2*>(band_phi);
  const double2* bb = static_cast<const double2*>(band_chi);
  double2* oR = static_cast<double2*>(outR);
  double2* oL = static_cast<double2*>(outL);
  const int r = c->prec == TC_FP64 ? dispatch_run_band<double>(c, a, b, ba, bb, oR, oL, tw, st)
                                   : dispatch_run_band<float>(c, a, b, ba, bb, oR, oL, tw, st);
  return (tc_status)r;
}

tc_status tc_energy(tc_ctx* c, const void* phi, const void* chi, const double* occ, double* E_total,
                    double* E_terms, void* stream) {
  if (!c) return TC_ERR_STATE;
  if (c->batch) return fail(c, TC_ERR_STATE, "batch context: use tc_apply_batch or tc_batch_cell");
  if (c->S.nkb > 0) return fail(c, TC_ERR_STATE, "band context: use tc_apply_band");
  if (!phi || !chi || !occ || !E_total) return fail(c, TC_ERR_ARG, "null pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const tc::Setup& S = c->S;
  const int nj = S.Nk * S.nb;
  const size_t orb = (size_t)nj * S.npw_max * sizeof(double2);
  // device copies of the inputs (so that the dot products can read them)
  const double2* dphi = static_cast<const double2*>(phi);
  const double2* dchi = static_cast<const double2*>(chi);
  cudaError_t e;
  if (!is_device_ptr(phi)) {
    if ((e = cudaMemcpyAsync(c->d_in_phi, phi, orb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(c, e, "upload");
    dphi = c->d_in_phi;
  }
  if (!is_device_ptr(chi)) {
    if ((e = cudaMemcpyAsync(c->d_in_chi, chi, orb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(c, e, "upload");
    dchi = c->d_in_chi;
  }
  auto reduce = [&](bool kin, bool with_out, double* res) -> tc_status {
    return energy_reduce(c, dphi, dchi, occ, kin, with_out, st, res);
  };
  double tw[NT];
  bool host_out = false;
  term_weights(c, tw, 0.5, 1.0 / 3.0);
  tc_status r = run_common(c, dphi, dchi, occ, c->d_out_R, nullptr, tw, 1, st, &host_out);
  if (r != TC_OK) return r;
  if ((r = reduce(true, true, E_total)) != TC_OK) return r;
  if (E_terms) {
    double all[NT];
    term_weights(c, all, 0.5, 1.0 / 3.0);
    for (int t = 0; t < NT; ++t) {
      if (all[t] == 0.0) { E_terms[t] = 0.0; continue; }
      double one[NT] = {0};
      one[t] = all[t];
      if ((r = run_common(c, dphi, dchi, occ, c->d_out_R, nullptr, one, 1, st, &host_out)) != TC_OK) return r;
      if ((r = reduce(false, true, &E_terms[t])) != TC_OK) return r;
    }
    if ((r = reduce(true, false, &E_terms[TC_TERM_KIN])) != TC_OK) return r;
  }
  return TC_OK;
}

tc_status tc_energy_grad(tc_ctx* c, const void* phi, const void* chi, const double* occ, void* dE_dphiR,
                         void* dE_dphiL, double* dE_dA, double* dE_dC, void* stream) {
  if (!c) return TC_ERR_STATE;
  if (c->batch) return fail(c, TC_ERR_STATE, "batch context: use tc_apply_batch or tc_batch_cell");
  if (c->S.nkb > 0) return fail(c, TC_ERR_STATE, "band context: use tc_apply_band");
  if (!phi || !chi || !occ) return fail(c, TC_ERR_ARG, "null input pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tc::Setup& S = c->S;
  const int nj = S.Nk * S.nb;
  for (int k = 0; k < S.Nk; ++k)
    for (int mu = S.no; mu < S.nb; ++mu)
      if (occ[k * S.nb + mu] != 0.0)
        return fail(c, TC_ERR_ARG, "tc_energy_grad needs occ = 0 for bands >= nocc (the partners carry the energy)");
  const bool want_orb = dE_dphiR || dE_dphiL;
  if (want_orb && S.prm.term_mask != 0u)
    return fail(c, TC_ERR_UNSUPPORTED, "the orbital gradient is the operator only with every term on (term_mask 0)");
  const size_t orb = (size_t)nj * S.npw_max * sizeof(double2);
  const double2* dphi = static_cast<const double2*>(phi);
  const double2* dchi = static_cast<const double2*>(chi);
  cudaError_t e;
  if (!is_device_ptr(phi)) {
    if ((e = cudaMemcpyAsync(c->d_in_phi, phi, orb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(c, e, "upload");
    dphi = c->d_in_phi;
  }
  if (!is_device_ptr(chi)) {
    if ((e = cudaMemcpyAsync(c->d_in_chi, chi, orb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(c, e, "upload");
    dchi = c->d_in_chi;
  }
  bool host_out = false;
  tc_status r;
  // 1. orbitals: both operator outputs, then g = (2/Nk) f (T x + out)
  if (want_orb) {
    double tw[NT];
    term_weights(c, tw, 1.0, 1.0);
    if ((r = run_common(c, dphi, dchi, occ, c->d_out_R, c->d_out_L, tw, 2, st, &host_out)) != TC_OK) return r;
    double2* gphi = dE_dphiR ? (is_device_ptr(dE_dphiR) ? static_cast<double2*>(dE_dphiR) : c->d_out_L) : nullptr;
    double2* gchi = dE_dphiL ? (is_device_ptr(dE_dphiL) ? static_cast<double2*>(dE_dphiL) : c->d_out_R) : nullptr;
    const size_t total = (size_t)nj * S.npw_max;
    k_grad_combine<<<2 * 152, 256, 0, st>>>(dphi, dchi, c->d_out_R, c->d_out_L, c->d_kpg, c->d_occ, S.npw_max, S.nb,
                                            2.0 / S.Nk, total, gphi, gchi);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "k_grad_combine");
    if (dE_dphiR && gphi == c->d_out_L &&
        (e = cudaMemcpyAsync(dE_dphiR, gphi, orb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(c, e, "dE_dphiR download");
    if (dE_dphiL && gchi == c->d_out_R &&
        (e = cudaMemcpyAsync(dE_dphiL, gchi, orb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(c, e, "dE_dphiL download");
  }
  // 2. Jastrow parameters: E is quadratic in the kernel data K, so along dK = dK/dtheta the
  //    symmetric difference [E(K + t dK) - E(K - t dK)] / 2t is exact for any t.
  if (dE_dA || dE_dC) {
    if (c->dkd.empty()) {
      try {
        c->dkd.resize(4);
        for (int m = 0; m < 4; ++m) tc::kernel_data(S, m, c->dkd[m]);
      } catch (const std::bad_alloc&) {
        c->dkd.clear();
        return fail(c, TC_ERR_OOM, "derivative tables: host allocation failed");
      }
    }
    if (!c->d_kd64) {
      // K and its four derivatives once on the device in FP64; each pass forms K + a dK there
      const std::vector<double>* base_t[5] = {&S.tabV, &S.tabU, &S.hartV, &S.hartU, &S.hartUs};
      size_t set = 0;
      for (int i = 0; i < 5; ++i) set += (c->kd64_len[i] = base_t[i]->size());
      if ((e = cudaMalloc((void**)&c->d_kd64, 5 * set * sizeof(double))) != cudaSuccess) {
        c->d_kd64 = nullptr;
        return cuda_fail(c, e, "derivative tables");
      }
      for (int m = -1; m < 4 && e == cudaSuccess; ++m) {
        const tc::KernelData* kd = m < 0 ? nullptr : &c->dkd[m];
        const std::vector<double>* src[5] = {
            m < 0 ? base_t[0] : &kd->tabV, m < 0 ? base_t[1] : &kd->tabU, m < 0 ? base_t[2] : &kd->hartV,
            m < 0 ? base_t[3] : &kd->hartU, m < 0 ? base_t[4] : &kd->hartUs};
        size_t off = (size_t)(m + 1) * set;
        for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
          if (src[i]->size() != c->kd64_len[i]) {
            e = cudaErrorInvalidValue;
            break;
          }
          e = cudaMemcpy(c->d_kd64 + off, src[i]->data(), src[i]->size() * sizeof(double), cudaMemcpyHostToDevice);
          off += src[i]->size();
        }
      }
      if (e != cudaSuccess) {
        cudaFree(c->d_kd64);
        c->d_kd64 = nullptr;
        return cuda_fail(c, e, "derivative tables");
      }
    }
    const double corr0[2] = {S.corr_c[0], S.corr_c[1]}, amp0[2] = {S.amp[0], S.amp[1]};
    double twE[NT];
    term_weights(c, twE, 0.5, 1.0 / 3.0);
    r = TC_OK;
    for (int m = 0; m < 4 && r == TC_OK; ++m) {
      double* dst = m < 2 ? dE_dA : dE_dC;
      if (!dst) continue;
      const double theta = m < 2 ? S.prm.A[m] : S.prm.C[m - 2];
      const double t = 0.5 * std::max(std::fabs(theta), 0.1);
      const tc::KernelData& dk = c->dkd[m];
      // the work of the pair stages that reads only the antiparallel u table ([delta][1][N] of tabU) is
      // the same in both passes when dK has no antiparallel part, and cancels in the difference: skip it
      bool ap_zero = true;
      const size_t nn = (size_t)S.N;
      for (size_t o = nn; ap_zero && o < dk.tabU.size(); o += 2 * nn)
        for (size_t i = 0; i < nn; ++i)
          if (dk.tabU[o + i] != 0.0) {
            ap_zero = false;
            break;
          }
      c->skip_ap = ap_zero ? 1 : 0;
      double Epm[2] = {0.0, 0.0};
      for (int sg = 0; sg < 2 && r == TC_OK; ++sg) {
        const double a = sg == 0 ? t : -t;
        e = c->prec == TC_FP64 ? displace_tables<double>(c, m, a, st) : displace_tables<float>(c, m, a, st);
        if (e != cudaSuccess) { r = cuda_fail(c, e, "displaced tables"); break; }
        for (int s = 0; s < 2; ++s) {
          S.corr_c[s] = corr0[s] + a * dk.corr_c[s];
          S.amp[s] = amp0[s] + a * dk.amp[s];
        }
        r = run_common(c, dphi, dchi, occ, c->d_out_R, nullptr, twE, 1, st, &host_out);
        if (r == TC_OK) r = energy_reduce(c, dphi, dchi, occ, false, true, st, &Epm[sg]);
      }
      if (r == TC_OK) dst[m % 2] = (Epm[0] - Epm[1]) / (2.0 * t);
    }
    // restore the kernel data of the context (also after a failure)
    c->skip_ap = 0;
    for (int s = 0; s < 2; ++s) {
      S.corr_c[s] = corr0[s];
      S.amp[s] = amp0[s];
    }
    e = c->prec == TC_FP64 ? displace_tables<double>(c, -1, 0.0, st) : displace_tables<float>(c, -1, 0.0, st);
    if (r != TC_OK) return r;
    if (e != cudaSuccess) return cuda_fail(c, e, "table restore");
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "tc_energy_grad");
  return TC_OK;
}

tc_status tc_biorthonormalize(tc_ctx* c, void* phi, void* chi, void* stream) {
  if (!c) return TC_ERR_STATE;
  if (c->batch) return fail(c, TC_ERR_STATE, "batch context: use tc_apply_batch or tc_batch_cell");
  if (c->S.nkb > 0) return fail(c, TC_ERR_STATE, "band context: use tc_apply_band");
  if (!phi || !chi) return fail(c, TC_ERR_ARG, "null orbital pointer");
  const tc::Setup& S = c->S;
  if (S.nb > kBiorthoMaxBands) return fail(c, TC_ERR_UNSUPPORTED, "tc_biorthonormalize supports at most 64 bands");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t orb = (size_t)S.Nk * S.nb * S.npw_max * sizeof(double2);
  const bool hp = !is_device_ptr(phi), hc = !is_device_ptr(chi);
  double2* dp = hp ? c->d_in_phi : static_cast<double2*>(phi);
  double2* dc = hc ? c->d_in_chi : static_cast<double2*>(chi);
  cudaError_t e = cudaSuccess;
  if (hp && (e = cudaMemcpyAsync(dp, phi, orb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(c, e, "upload");
  if (hc && (e = cudaMemcpyAsync(dc, chi, orb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(c, e, "upload");
  if ((e = cudaMemsetAsync(c->d_status, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(c, e, "status");
  const int rb = tc::launch_biortho(c, dp, dc, c->d_status, st);
  if (rb != TC_OK) return (tc_status)rb;
  int status = 0;
  if ((e = cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(c, e, "status");
  if (hp && (e = cudaMemcpyAsync(phi, dp, orb, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(c, e, "download");
  if (hc && (e = cudaMemcpyAsync(chi, dc, orb, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(c, e, "download");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "tc_biorthonormalize");
  status = *c->h_status;
  if (status != 0)
    return fail(c, TC_ERR_ARG, "biorthonormalisation: vanishing norm or singular overlap at k-point " +
                                   std::to_string(status - 1) + " (outputs undefined)");
  return TC_OK;
}

tc_status tc_fft3d(int n, int precision, int sign, void* data, int batch, void* stream) {
  if (!data || batch < 0 || (sign != 1 && sign != -1)) return TC_ERR_ARG;
  if (batch == 0) return TC_OK;
  tc_ctx tmp;
  const int pr = precision == TC_FP64 ? dispatch_prepare<double>(&tmp, n) : dispatch_prepare<float>(&tmp, n);
  if (pr != TC_OK) return (tc_status)pr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int r = precision == TC_FP64 ? dispatch_fft<double>(n, data, batch, sign, st)
                                     : dispatch_fft<float>(n, data, batch, sign, st);
  return (tc_status)r;
}

tc_status tc_band_constants(const tc_params* params, const double* kfrac_band, int nkb, double* gamma_b,
                            double* W) {
  if (!params || nkb < 0 || (nkb > 0 && (!kfrac_band || !gamma_b || !W))) {
    tc::set_thread_error("tc_band_constants: null pointer or nkb < 0");
    return TC_ERR_ARG;
  }
  tc::Setup S;
  const std::string why = tc::build_setup(*params, S);
  if (!why.empty()) {
    tc::set_thread_error("tc_band_constants: " + why);
    return why.rfind("unsupported", 0) == 0 ? TC_ERR_UNSUPPORTED : TC_ERR_ARG;
  }
  for (int i = 0; i < nkb; ++i) {
    const double* kf = kfrac_band + 3 * (size_t)i;
    for (int q = 0; q < S.Nk; ++q) {
      bool same = true;
      for (int d = 0; d < 3; ++d) {
        const double x = kf[d] - S.kfrac[q][d];
        same = same && std::fabs(x - std::round(x)) < 1e-12;
      }
      if (same) {
        tc::set_thread_error("tc_band_constants: band point " + std::to_string(i) +
                         " lies on the SCF mesh (it takes the SCF constants)");
        return TC_ERR_ARG;
      }
    }
    double k[3];
    for (int d = 0; d < 3; ++d) k[d] = kf[0] * S.B[0][d] + kf[1] * S.B[1][d] + kf[2] * S.B[2][d];
    if (!tc::band_constants(S, k, gamma_b + i, W + 3 * (size_t)i)) {
      tc::set_thread_error("tc_band_constants: band point " + std::to_string(i) + " lies on the SCF mesh");
      return TC_ERR_ARG;
    }
  }
  return TC_OK;
}

tc_status tc_band_layout(const tc_params* params, const double* kfrac_band, int nkb, int max_npw, int* npw,
                         int* miller) {
  if (!params || nkb < 0 || (nkb > 0 && (!kfrac_band || !npw)) || (miller && max_npw <= 0)) {
    tc::set_thread_error("tc_band_layout: null pointer, nkb < 0 or max_npw <= 0");
    return TC_ERR_ARG;
  }
  tc::Setup S;
  const std::string why = tc::build_setup(*params, S);
  if (!why.empty()) {
    tc::set_thread_error("tc_band_layout: " + why);
    return why.rfind("unsupported", 0) == 0 ? TC_ERR_UNSUPPORTED : TC_ERR_ARG;
  }
  std::vector<std::array<int, 3>> m;
  for (int i = 0; i < nkb; ++i) {
    const double* kf = kfrac_band + 3 * (size_t)i;
    double k[3];
    for (int d = 0; d < 3; ++d) k[d] = kf[0] * S.B[0][d] + kf[1] * S.B[1][d] + kf[2] * S.B[2][d];
    if (!tc::sphere(S, k, m)) {
      tc::set_thread_error("tc_band_layout: the sphere of band point " + std::to_string(i) +
                           " does not fit the FFT box");
      return TC_ERR_ARG;
    }
    npw[i] = (int)m.size();
    if (!miller) continue;
    if (npw[i] > max_npw) {
      tc::set_thread_error("tc_band_layout: max_npw is smaller than the sphere of band point " + std::to_string(i));
      return TC_ERR_ARG;
    }
    int* out = miller + (size_t)i * max_npw * 3;
    for (int g = 0; g < max_npw; ++g)
      for (int d = 0; d < 3; ++d) out[3 * g + d] = g < npw[i] ? m[g][d] : 0;
  }
  return TC_OK;
}

tc_status tc_profile(tc_ctx* c, int enable) {
  if (!c) return TC_ERR_STATE;
  if (c->batch) return fail(c, TC_ERR_STATE, "batch context: use tc_apply_batch or tc_batch_cell");
  for (int i = 0; i < 8; ++i) {
    c->stage_ms[i] = 0.0;
    c->stage_launch[i] = 0;
    if (enable && !c->ev[i]) {
      cudaError_t e = cudaEventCreate(&c->ev[i]);
      if (e != cudaSuccess) return cuda_fail(c, e, "tc_profile");
    }
  }
  c->profile = enable != 0;
  return TC_OK;
}

tc_status tc_autotune(tc_ctx* c, const void* phi, const void* chi, const double* occ, int* so_out, int* sc_out,
                      void* stream) {
  if (!c) return TC_ERR_STATE;
  if (c->batch || !c->ws_owned) return fail(c, TC_ERR_STATE, "autotuning needs a single-cell context from tc_init");
  if (c->S.nkb > 0) return fail(c, TC_ERR_STATE, "band context: use tc_apply_band");
  if (!phi || !chi || !occ) return fail(c, TC_ERR_ARG, "null input pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const tc::Setup& S = c->S;
  const int M = S.Nk * S.no;
  const int smax = std::min(8, M);
  const bool prof_was = c->profile;
  // workspace for the largest candidate
  c->so_max = std::max(c->so_max, smax);
  c->sc_max = std::max(c->sc_max, smax);
  int r = tc::rebuild_workspace(c);
  if (r != TC_OK) return (tc_status)r;
  tc_status rs = tc_profile(c, 1);
  if (rs != TC_OK) return rs;
  double tw[NT];
  term_weights(c, tw, 1.0, 1.0);
  bool host_out = false;
  int so[2] = {c->split_occ[0], c->split_occ[1]}, sc[2] = {c->split_chain[0], c->split_chain[1]};
  // two-sided launches (tc_apply, tc_energy_grad), then one-sided ones (tc_energy, tc_davidson_step)
  for (int nsides = 2; nsides >= 1 && rs == TC_OK; --nsides) {
    double t_occ[9] = {}, t_chain[9] = {};
    for (int s = 0; s <= smax; ++s) {
      // s = 0 is an untimed warm-up with one chunk; then one measured apply per candidate
      const int cand = s == 0 ? 1 : s;
      c->split_occ[nsides - 1] = cand;
      c->split_chain[nsides - 1] = cand;
      for (int i = 0; i < 8; ++i) c->stage_ms[i] = 0.0;
      rs = run_common(c, phi, chi, occ, c->d_out_R, nsides == 2 ? c->d_out_L : nullptr, tw, nsides, st, &host_out);
      if (rs != TC_OK) break;
      if (s == 0) continue;
      t_occ[s] = c->stage_ms[2];
      t_chain[s] = c->stage_ms[3] + c->stage_ms[4];
    }
    if (rs != TC_OK) break;
    so[nsides - 1] = tc::smallest_near_best(t_occ, smax);
    sc[nsides - 1] = tc::smallest_near_best(t_chain, smax);
  }
  tc_profile(c, prof_was ? 1 : 0);
  c->split_occ[0] = so[0];
  c->split_occ[1] = so[1];
  c->split_chain[0] = sc[0];
  c->split_chain[1] = sc[1];
  c->so_max = std::max(so[0], so[1]);
  c->sc_max = std::max(sc[0], sc[1]);
  r = tc::rebuild_workspace(c);
  if (rs != TC_OK) return rs;
  if (r != TC_OK) return (tc_status)r;
  // two-sided launches that derive the left side run the occupied-pair stage one-sided
  if (so_out) *so_out = c->left_from_right ? so[0] : so[1];
  if (sc_out) *sc_out = sc[1];
  return TC_OK;
}

tc_status tc_stage_times(const tc_ctx* c, double* ms, int* launches, int n) {
  if (!c) return TC_ERR_STATE;
  if (c->batch) return TC_ERR_STATE;
  if (!ms || n < TC_NSTAGES) return TC_ERR_ARG;
  for (int i = 0; i < TC_NSTAGES; ++i) {
    ms[i] = c->stage_ms[i];
    if (launches) launches[i] = c->stage_launch[i];
  }
  return TC_OK;
}

tc_status tc_pair_kernels(const tc_ctx* c, int* info) {
  if (!c || c->batch) return TC_ERR_STATE;
  if (!info) return TC_ERR_ARG;
  // the dispatch rule of run_pipeline
  const bool pruned = c->plan_prune_L > 0 && c->pair_support <= c->plan_prune_L;
  const bool dist = !pruned && c->plan_cl_L > 0 && c->pair_support <= c->plan_cl_L;
  for (int k = 0; k < 3; ++k) {
    int* o = info + 3 * k;
    if (pruned) {
      o[0] = 1; o[1] = c->plan_prune_L; o[2] = 1;
    } else if (dist && c->plan_cl[k] > 0 && ((c->cluster_ok >> k) & 1)) {
      o[0] = 2; o[1] = c->plan_cl_L; o[2] = c->plan_cl[k];
    } else {
      o[0] = 0; o[1] = c->S.n; o[2] = 1;
    }
  }
  return TC_OK;
}

tc_status tc_pair_mirror(const tc_ctx* c, int* active, unsigned long long* bytes) {
  if (!c || c->batch) return TC_ERR_STATE;
  if (active) *active = c->d_mirror ? 1 : 0;
  if (bytes) *bytes = (unsigned long long)c->mirror_bytes;
  return TC_OK;
}

const char* tc_last_error(const tc_ctx* c) { return c ? c->err.c_str() : g_init_err.c_str(); }

tc_status tc_destroy(tc_ctx* c) {
  if (!c) return TC_ERR_STATE;
  if (c->batch_owner) return fail(c, TC_ERR_STATE, "this context belongs to a batch: destroy the batch");
  tc::destroy_context(c);
  return TC_OK;
}

}  // extern "C"
