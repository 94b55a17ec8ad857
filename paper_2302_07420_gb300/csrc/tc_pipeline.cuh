// Host-side launch sequence of the operator for one (precision, box size).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "tc_ctx.hpp"
#include "tc_kernels_impl.cuh"
#include "tc_pruned.cuh"
#include "tc_cluster.cuh"
#include "tc_band.cuh"

namespace tc {



template <typename T, int N> static void fill_side(tc_ctx* ctx, int side, SideArgs<T>& s) {
  const size_t NN = (size_t)N * N * N;
  const auto& S = ctx->S;
  cplx<T>* base = reinterpret_cast<cplx<T>*>(reinterpret_cast<char*>(ctx->d_side) + side * ctx->side_bytes);
  size_t o = 0;
  auto take = [&](size_t vols) { cplx<T>* p = base + o * NN; o += vols; return p; };
  s.n = take(1); s.m = take(3); s.nt = take(1); s.mt = take(3); s.vH = take(1); s.h1 = take(3);
  s.vb2 = take(1); s.t3b1 = take(1); s.t3b2 = take(1); s.vu = take(2); s.spec = take(3); s.h5 = take(3);
  s.h6 = take(1); s.vloc = take(1);
  s.h3a4 = take((size_t)ctx->so_max * S.Nk * S.no * 3);
  s.h3b = take((size_t)ctx->so_max * S.Nk * S.no * 3);
  s.acc = take((size_t)ctx->sc_max * ctx->nj_out);
  s.w = take((size_t)ctx->sc_max * ctx->nj_out * 3);
  s.Z = take((size_t)S.Nk * S.no * 3);
  s.Y = take((size_t)ctx->nj_out * 3);
  s.v2 = take((size_t)S.nkb * 4);
  s.bh3a = take((size_t)ctx->so_band * S.nkb * S.no * 3);
  s.bh3b = take((size_t)ctx->so_band * S.nkb * S.no * 3);
  s.cs = ctx->d_cs + (size_t)side * ctx->nj_out * S.no * 6;
  const cplx<T>* phi = reinterpret_cast<const cplx<T>*>(ctx->d_phi);
  const cplx<T>* chi = reinterpret_cast<const cplx<T>*>(ctx->d_chi);
  const cplx<T>* gphi = reinterpret_cast<const cplx<T>*>(ctx->d_gphi);
  const cplx<T>* gchi = reinterpret_cast<const cplx<T>*>(ctx->d_gchi);
  s.ket = side == 0 ? phi : chi;
  s.bra = side == 0 ? chi : phi;
  s.gket = side == 0 ? gphi : gchi;
  s.tabV = reinterpret_cast<const T*>(ctx->d_tabV);
  s.s2b = side == 0 ? T(1) : T(-1);
  s.side = side;
}

template <typename T, int N> static Params<T> make_params(tc_ctx* ctx, const double* tw) {
  Params<T> P{};
  const auto& S = ctx->S;
  P.Nk = S.Nk; P.nb = S.nb; P.no = S.no; P.npw_max = S.npw_max; P.ndelta = S.ndelta;
  P.div = S.prm.div_correction;
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) P.Bm[i][d] = (T)S.B[i][d];
  P.invN = (T)(1.0 / ((double)N * N * N));
  P.Omega = S.Omega;
  P.invOm2 = 1.0 / (S.Omega * S.Omega);
  for (int s = 0; s < 2; ++s) { P.corr_c[s] = S.corr_c[s]; P.A[s] = S.amp[s]; }
  for (int t = 0; t < NT; ++t) P.tw[t] = (T)tw[t];
  P.delta_id = ctx->d_delta_id;
  P.delta = reinterpret_cast<const T*>(ctx->d_delta);
  P.tabU = reinterpret_cast<const T*>(ctx->d_tabU);
  P.tabV = reinterpret_cast<const T*>(ctx->d_tabV);
  P.hartV = reinterpret_cast<const T*>(ctx->d_hartV);
  P.hartU = reinterpret_cast<const T*>(ctx->d_hartU);
  P.hartUs = reinterpret_cast<const T*>(ctx->d_hartUs);
  P.occ = ctx->d_occ;
  P.scratch = reinterpret_cast<cplx<T>*>(ctx->d_scratch);
  P.sym = ctx->sym;
  P.nirr = ctx->nirr;
  P.irr = ctx->d_irr;
  P.symk = ctx->d_symk;
  P.symrot = ctx->d_symrot;
  if constexpr (sizeof(T) == 8) P.symcart = reinterpret_cast<const T*>(ctx->d_symcart64);
  else P.symcart = reinterpret_cast<const T*>(ctx->d_symcart32);
  P.star_off = ctx->d_star_off;
  P.star_k = ctx->d_star_k;
  P.kstride = S.Nkt;
  P.j0 = 0;
  P.nj_out = S.Nk * S.nb;
  P.i2_0 = 0;
  P.nq2 = S.Nk * S.no;
  P.h3_only = 0;
  P.no_ap = ctx->skip_ap;
  P.band = 0;
  P.nkb = S.nkb;
  P.bandc = ctx->d_band;
  P.bs = ctx->d_bs;
  fill_side<T, N>(ctx, 0, P.side[0]);
  fill_side<T, N>(ctx, 1, P.side[1]);
  return P;
}

template <typename T, int N> static inline int vol_bytes() { return Geo<N>::vol * (int)sizeof(cplx<T>); }
template <typename T, int N> static inline int smem_vols(int want, int static_bytes = 1024) {
  int n = (kSmemLimit - static_bytes) / vol_bytes<T, N>();
  return n < want ? n : want;
}

#define TC_SET_SMEM(kern, bytes)                                                              \
  do {                                                                                        \
    cudaError_t e_ = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (bytes)); \
    if (e_ != cudaSuccess) {                                                                  \
      ctx->err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e_);              \
      return TC_ERR_CUDA;                                                                     \
    }                                                                                         \
  } while (0)

// Launch of a cluster-distributed kernel: clusters of cl CTAs along x (grid.x a multiple of cl).
template <typename... Args>
static cudaError_t launch_cluster(void (*kern)(Args...), dim3 grid, int threads, size_t smem, int cl,
                                  cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Sets the kernel's shared-memory size and reports whether one cluster of it fits the device (never
// under the host fault switch TC_FAULT=nocluster).
template <typename K> static bool cluster_fits(tc_ctx*, K kern, int cl, int threads, size_t smem) {
  if (injected_fault("cluster") != TC_OK) return false;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

template <typename T, int N> int prepare_kernels(tc_ctx* ctx) {
  // twiddles exp(-2 pi i j/L) for every codelet length, FP64 host sin/cos
  static double tw64[2 * kTwTotal];
  static float tw32[2 * kTwTotal];
  for (int i = 0, off = 0; i < kNumTwLens; ++i) {
    const int L = kTwLens[i];
    for (int j = 0; j < L; ++j) {
      const double a = -2.0 * 3.14159265358979323846 * j / L;
      tw64[2 * (off + j)] = std::cos(a);
      tw64[2 * (off + j) + 1] = std::sin(a);
      tw32[2 * (off + j)] = (float)std::cos(a);
      tw32[2 * (off + j) + 1] = (float)std::sin(a);
    }
    off += L;
  }
  cudaError_t e1 = cudaMemcpyToSymbol(c_tw64, tw64, sizeof(tw64));
  cudaError_t e2 = cudaMemcpyToSymbol(c_tw32, tw32, sizeof(tw32));
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    ctx->err = "twiddle upload failed";
    return TC_ERR_CUDA;
  }
  const int vb = vol_bytes<T, N>();
  const int vb1 = Fit<T, N>::one ? vb : 0;   // single-volume kernels: shared memory or global scratch
  TC_SET_SMEM((k_orbitals<T, N>), vb1);
  TC_SET_SMEM((k_spec_fwd<T, N>), vb1);
  TC_SET_SMEM((k_hartree_inv<T, N>), vb1);
  TC_SET_SMEM((k_finalize<T, N>), vb1);
  TC_SET_SMEM((k_band_v2<T, N>), vb1);
  TC_SET_SMEM((k_occ_pairs<T, N>), (smem_vols<T, N>(4) * vb));
  TC_SET_SMEM((k_pair_chain<T, N>), (smem_vols<T, N>(3) * vb));
  TC_SET_SMEM((k_pair_3b4<T, N>), (smem_vols<T, N>(2) * vb));
  if constexpr (kPruneL<N> < N) {
    TC_SET_SMEM((k_pair_chain_pr<T, N, kPruneL<N>>), (int)(PrSmem<T, N, kPruneL<N>, 2, 3>::bytes));
    TC_SET_SMEM((k_pair_3b4_pr<T, N, kPruneL<N>>), (int)(PrSmem<T, N, kPruneL<N>, 1, 1>::bytes));
    TC_SET_SMEM((k_occ_pairs_pr<T, N, kPruneL<N>>), (int)(OccSmem<T, N, kPruneL<N>>::bytes));
  }
  TC_SET_SMEM((k_fft3d<T, N, -1>), vb1);
  TC_SET_SMEM((k_fft3d<T, N, +1>), vb1);
  // cluster-distributed kernels: each is used only if the device can hold one of its clusters
  ctx->cluster_ok = 0;
  using C0 = ClCfg<T, N, 0>;
  using C1 = ClCfg<T, N, 1>;
  using C2 = ClCfg<T, N, 2>;
  ctx->plan_prune_L = kPruneL<N> < N ? kPruneL<N> : 0;
  ctx->plan_cl_L = ClPlan<T, N>::L;
  ctx->plan_cl[0] = C0::CL;
  ctx->plan_cl[1] = C1::CL;
  ctx->plan_cl[2] = C2::CL;
  if constexpr (C0::CL > 0)
    ctx->cluster_ok |= cluster_fits(ctx, k_pair_chain_cl<T, N>, C0::CL, C0::threads, C0::smem) ? 1 : 0;
  if constexpr (C1::CL > 0)
    ctx->cluster_ok |= cluster_fits(ctx, k_pair_3b4_cl<T, N>, C1::CL, C1::threads, C1::smem) ? 2 : 0;
  if constexpr (C2::CL > 0)
    ctx->cluster_ok |= cluster_fits(ctx, k_occ_pairs_cl<T, N>, C2::CL, C2::threads, C2::smem) ? 4 : 0;
  return TC_OK;
}

// Global scratch: the per-CTA volumes of k_occ_pairs (6) and k_pair_chain (3)
// that are not in shared memory, and -- for boxes whose volume does not fit in
// shared memory -- the work volume of every CTA of the single-volume kernels
// (at most 8 per orbital in k_orbitals).  The uses never overlap in time.
template <typename T, int N> size_t scratch_needed(const Setup& S, int so_max, int sc_max) {
  const size_t vb = (size_t)vol_bytes<T, N>();
  // (band contexts: the band points' occupied-pair launch, at most 8 chunks)
  const size_t a = (size_t)2 * std::max(S.Nk * so_max, S.nkb * 8) * S.no * 6 * vb;
  const size_t b = (size_t)2 * std::max(S.Nk, S.nkb) * S.nb * sc_max * 3 * vb;
  const size_t c = Fit<T, N>::one ? 0 : (size_t)8 * S.Nkt * S.nb * vb;
  return std::max(a, std::max(b, c));
}

#define TC_CHECK_LAUNCH(name)                                                                 \
  do {                                                                                        \
    cudaError_t e_ = cudaGetLastError();                                                      \
    if (e_ != cudaSuccess) {                                                                  \
      ctx->err = std::string(name) + ": " + cudaGetErrorString(e_);                           \
      return TC_ERR_CUDA;                                                                     \
    }                                                                                         \
  } while (0)

#define TC_CHECK_CL(call)                                                                     \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      cudaGetLastError();                                                                     \
      ctx->err = std::string("cluster launch: ") + cudaGetErrorString(e_);                    \
      return TC_ERR_CUDA;                                                                     \
    }                                                                                         \
  } while (0)

// Records the boundary event before stage i (profiling only).
static inline void stage_mark(tc_ctx* ctx, cudaStream_t st, int i) {
  if (ctx->profile) cudaEventRecord(ctx->ev[i], st);
}

static inline int stage_collect(tc_ctx* ctx, int nstages, const int* launches) {
  if (!ctx->profile) return TC_OK;
  if (cudaEventSynchronize(ctx->ev[nstages]) != cudaSuccess) {
    ctx->err = "profiling event wait failed";
    return TC_ERR_CUDA;
  }
  for (int i = 0; i < nstages; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]);
    ctx->stage_ms[i] += ms;
    ctx->stage_launch[i] += launches[i];
  }
  return TC_OK;
}

// Band contexts (S.nkb > 0): bphi / bchi are the band points' orbitals and the outputs are theirs
// (tc_band.cuh); every partner-only stage is the mesh one.
template <typename T, int N>
int run_pipeline(tc_ctx* ctx, const double2* cphi, const double2* cchi, double2* outR, double2* outL,
                 const double* tw, int nsides, cudaStream_t st, const double2* bphi, const double2* bchi) {
  const auto& S = ctx->S;
  const int TH = Cfg<N>::threads;
  const int vb = vol_bytes<T, N>();
  const int vb1 = Fit<T, N>::one ? vb : 0;
  Params<T> P = make_params<T, N>(ctx, tw);
  P.so = ctx->split_occ[nsides - 1];
  P.sc = ctx->split_chain[nsides - 1];
  const bool band = S.nkb > 0;
  if (band && (nsides != 2 || !bphi || !bchi || P.sym || ctx->partners_from)) {
    ctx->err = "band context: two-sided launches with band-point orbitals only";
    return TC_ERR_STATE;
  }
  const int nj = S.Nk * S.nb;                       // mesh orbitals (partners)
  const int nj_all = S.Nkt * S.nb;                  // orbitals to real space
  if (band) {
    P.band = 1;
    P.j0 = nj;
    P.nj_out = S.nkb * S.nb;
  }
  // band points: every divergence correction (all need div_correction) and the fields they take
  const bool band_corr = band && P.div;
  const int pw_blocks = 2 * 152;
  int nl[6] = {1, 9, 0, 1, 1, 1};   // kernel launches per stage
  // pair densities whose spectra fit the compiled support take the pruned transforms
  constexpr int LP = kPruneL<N>;
  const bool pruned = LP < N && ctx->pair_support <= LP;
  // else, when they fit the distributed kernels' support, the cluster-distributed ones
  constexpr int LC = ClPlan<T, N>::L;
  using C0 = ClCfg<T, N, 0>;
  using C1 = ClCfg<T, N, 1>;
  using C2 = ClCfg<T, N, 2>;
  constexpr int CLc = C0::CL, CLb = C1::CL, CLo = C2::CL;
  const bool dist = !pruned && LC > 0 && ctx->pair_support <= LC;
  const bool dist_chain = dist && CLc > 0 && (ctx->cluster_ok & 1);
  const bool dist_3b4 = dist && CLb > 0 && (ctx->cluster_ok & 2);
  const bool dist_occ = dist && CLo > 0 && (ctx->cluster_ok & 4);
  // 1. orbitals to real space
  stage_mark(ctx, st, 0);
  k_orbitals<T, N><<<dim3(nj_all, 4, 2), TH, vb1, st>>>(cphi, cchi, bphi, bchi, nj, ctx->d_box_index, ctx->d_kpg,
                                                   S.npw_max, S.nb,
                                                   (cplx<T>*)ctx->d_phi, (cplx<T>*)ctx->d_chi,
                                                   (cplx<T>*)ctx->d_gphi, (cplx<T>*)ctx->d_gchi,
                                                   (cplx<T>*)ctx->d_scratch);
  TC_CHECK_LAUNCH("k_orbitals");
  if (sizeof(T) == 4 && S.prm.precision == TC_BF16_STORE) {
    const size_t no = (size_t)nj_all * S.N;   // orbitals x box points per set
    k_round_bf16<T><<<2 * pw_blocks, 256, 0, st>>>((cplx<T>*)ctx->d_phi, no);
    k_round_bf16<T><<<2 * pw_blocks, 256, 0, st>>>((cplx<T>*)ctx->d_chi, no);
    k_round_bf16<T><<<2 * pw_blocks, 256, 0, st>>>((cplx<T>*)ctx->d_gphi, 3 * no);
    k_round_bf16<T><<<2 * pw_blocks, 256, 0, st>>>((cplx<T>*)ctx->d_gchi, 3 * no);
    TC_CHECK_LAUNCH("k_round_bf16");
    nl[0] += 4;
  }
  const tc_ctx* src = ctx->partners_from;
  if (src) {
    // stages 2 and 3 up to the local potential from a context with the same partners: the 25
    // base fields of each side (n .. vloc, contiguous) and part 0 of both occupied-pair h3 kinds
    stage_mark(ctx, st, 1);
    const size_t vb_el = sizeof(cplx<T>) * (size_t)S.N;
    for (int sd = 0; sd < nsides; ++sd) {
      SideArgs<T> from{};
      fill_side<T, N>(const_cast<tc_ctx*>(src), sd, from);
      cudaError_t e = cudaMemcpyAsync(P.side[sd].n, from.n, 25 * vb_el, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.side[sd].h3a4, from.h3a4, (size_t)S.Nk * S.no * 3 * vb_el, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.side[sd].h3b, from.h3b, (size_t)S.Nk * S.no * 3 * vb_el, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) {
        ctx->err = std::string("partner fields: ") + cudaGetErrorString(e);
        return TC_ERR_CUDA;
      }
    }
    nl[1] = 0;
    nl[2] = 1;
    stage_mark(ctx, st, 2);
    k_prep_zy<T, N><<<dim3(2 * pw_blocks, nsides), 256, 0, st>>>(P);
    TC_CHECK_LAUNCH("k_prep_zy");
  } else {
  // 2. densities and Hartree-type fields
  stage_mark(ctx, st, 1);
  k_density<T, N><<<dim3(pw_blocks, nsides), 256, 0, st>>>(P);
  TC_CHECK_LAUNCH("k_density");
  k_spec_fwd<T, N><<<dim3(1, nsides), TH, vb1, st>>>(P, 0);
  k_spec_fwd<T, N><<<dim3(3, nsides), TH, vb1, st>>>(P, 1);
  TC_CHECK_LAUNCH("k_spec_fwd");
  k_hartree_inv<T, N><<<dim3(1, nsides), TH, vb1, st>>>(P, 0);
  k_hartree_inv<T, N><<<dim3(3, nsides), TH, vb1, st>>>(P, 1);
  k_hartree_inv<T, N><<<dim3(1, nsides), TH, vb1, st>>>(P, 2);
  k_hartree_inv<T, N><<<dim3(2, nsides), TH, vb1, st>>>(P, 5);
  TC_CHECK_LAUNCH("k_hartree_inv");
  k_spec_fwd<T, N><<<dim3(3, nsides), TH, vb1, st>>>(P, 2);
  k_hartree_inv<T, N><<<dim3(1, nsides), TH, vb1, st>>>(P, 3);
  TC_CHECK_LAUNCH("hartree 3b1");
  if (band_corr) {
    k_band_v2<T, N><<<dim3(4 * S.nkb, nsides), TH, vb1, st>>>(P);
    TC_CHECK_LAUNCH("k_band_v2");
    nl[1] += 1;
  }
  // 3. occupied-pair stage
  stage_mark(ctx, st, 2);
  const bool need_a4 = tw[T3A2] != 0 || tw[T3A4] != 0 || tw[T3B2] != 0 || tw[T3B5] != 0;
  if (need_a4) {
    // two-sided launches compute the right side only and conjugate it into the left one when
    // that is exact on this grid (see k_left_from_right)
    const bool derive_left = nsides == 2 && ctx->left_from_right;
    const int occ_sides = derive_left ? 1 : nsides;
    Params<T> Pa = P;
    Pa.nsmem = smem_vols<T, N>(4);
    if (derive_left) Pa.so = ctx->split_occ[0];
    const int q2_items = P.sym ? P.nirr * S.no : S.Nk * S.no;   // irreducible q2 only with symmetry
    if constexpr (LP < N) {
      if (pruned)
        k_occ_pairs_pr<T, N, LP><<<dim3(q2_items * Pa.so, occ_sides), PrCfg<T, N>::threads,
                                   OccSmem<T, N, LP>::bytes, st>>>(Pa);
    }
    if constexpr (CLo > 0) {
      if (dist_occ)
        TC_CHECK_CL(launch_cluster(k_occ_pairs_cl<T, N>, dim3(q2_items * Pa.so * CLo, occ_sides), C2::threads,
                                   C2::smem, CLo, st, Pa));
    }
    if (!pruned && !dist_occ) k_occ_pairs<T, N><<<dim3(q2_items * Pa.so, occ_sides), TH, Pa.nsmem * vb, st>>>(Pa);
    TC_CHECK_LAUNCH("k_occ_pairs");
    if (Pa.so > 1) {
      k_sum_parts<T, N><<<dim3(2 * pw_blocks, occ_sides), 256, 0, st>>>(Pa, 0);
      TC_CHECK_LAUNCH("k_sum_parts");
      nl[2] += 1;
    }
    if (P.sym && P.nirr < S.Nk) {
      k_unfold<T, N><<<dim3(2 * pw_blocks, occ_sides), 256, 0, st>>>(P);
      TC_CHECK_LAUNCH("k_unfold");
      nl[2] += 1;
    }
    k_reduce_a4<T, N><<<dim3(pw_blocks, occ_sides), 256, 0, st>>>(Pa, 0, 0);
    TC_CHECK_LAUNCH("k_reduce_a4");
    if (derive_left) {
      k_left_from_right<T, N><<<2 * pw_blocks, 256, 0, st>>>(P);
      TC_CHECK_LAUNCH("k_left_from_right");
      k_reduce_a4<T, N><<<dim3(pw_blocks, 1), 256, 0, st>>>(Pa, 1, 1);   // h5 of the left side
      TC_CHECK_LAUNCH("k_reduce_a4");
      nl[2] += 2;
    }
    k_spec_fwd<T, N><<<dim3(3, nsides), TH, vb1, st>>>(P, 3);
    k_hartree_inv<T, N><<<dim3(1, nsides), TH, vb1, st>>>(P, 4);
    TC_CHECK_LAUNCH("hartree 3b2");
    nl[2] += 4;
  }
  if (band_corr) {
    // occupied-pair fields (both h3 kinds, parallel spins) of the band points' own occupied
    // orbitals against the mesh partners, both sides, then their q1 -> k_b correction
    Params<T> Pq = P;
    Pq.nsmem = smem_vols<T, N>(4);
    Pq.i2_0 = nj / S.nb * S.no;   // items Nk no ..
    Pq.nq2 = S.nkb * S.no;
    Pq.h3_only = 1;
    Pq.so = ctx->so_band;
    for (int sd = 0; sd < 2; ++sd) {
      Pq.side[sd].h3a4 = P.side[sd].bh3a;
      Pq.side[sd].h3b = P.side[sd].bh3b;
    }
    if constexpr (LP < N) {
      if (pruned)
        k_occ_pairs_pr<T, N, LP><<<dim3(Pq.nq2 * Pq.so, 2), PrCfg<T, N>::threads, OccSmem<T, N, LP>::bytes, st>>>(Pq);
    }
    if constexpr (CLo > 0) {
      if (dist_occ)
        TC_CHECK_CL(launch_cluster(k_occ_pairs_cl<T, N>, dim3(Pq.nq2 * Pq.so * CLo, 2), C2::threads, C2::smem, CLo,
                                   st, Pq));
    }
    if (!pruned && !dist_occ) k_occ_pairs<T, N><<<dim3(Pq.nq2 * Pq.so, 2), TH, Pq.nsmem * vb, st>>>(Pq);
    TC_CHECK_LAUNCH("k_occ_pairs (band points)");
    if (Pq.so > 1) {
      k_sum_parts<T, N><<<dim3(2 * pw_blocks, 2), 256, 0, st>>>(Pq, 0);
      TC_CHECK_LAUNCH("k_sum_parts");
      nl[2] += 1;
    }
    k_band_scalars<T, N><<<dim3(S.nkb * S.no * S.nb, 2), 256, 0, st>>>(P, 0);
    k_band_h3corr<T, N><<<2 * pw_blocks, 256, 0, st>>>(P, 2);
    k_band_scalars<T, N><<<dim3(S.nkb * S.no * S.nb, 2), 256, 0, st>>>(P, 1);
    TC_CHECK_LAUNCH("band scalars");
    nl[2] += 4;
  }
  k_vloc<T, N><<<dim3(pw_blocks, nsides), 256, 0, st>>>(P);
  TC_CHECK_LAUNCH("k_vloc");
  k_prep_zy<T, N><<<dim3(2 * pw_blocks, nsides), 256, 0, st>>>(P);
  TC_CHECK_LAUNCH("k_prep_zy");
  nl[2] += 2;
  }
  // 4. pair chains (with symmetry: output orbitals of irreducible k-points only)
  stage_mark(ctx, st, 3);
  const int nj_items = P.sym ? P.nirr * S.nb : P.nj_out;
  {
    Params<T> Pc = P;
    Pc.nsmem = smem_vols<T, N>(3);
    if constexpr (LP < N) {
      // two-sided FP64: the right side first, writing the reflections the left side then reads
      const bool mirror = sizeof(T) == 8 && pruned && nsides == 2 && ctx->d_mirror && !P.sym && !band;
      if (mirror) {
        Pc.mir = reinterpret_cast<cplx<T>*>(ctx->d_mirror);
        for (int sd = 0; sd < 2; ++sd) {
          Pc.side0 = sd;
          Pc.mirror = 1 + sd;
          k_pair_chain_pr<T, N, LP><<<dim3(nj_items * P.sc, 1), PrCfg<T, N>::threads,
                                      PrSmem<T, N, LP, 2, 3>::bytes, st>>>(Pc);
        }
        nl[3] += 1;
      } else if (pruned) {
        k_pair_chain_pr<T, N, LP><<<dim3(nj_items * P.sc, nsides), PrCfg<T, N>::threads,
                                    PrSmem<T, N, LP, 2, 3>::bytes, st>>>(Pc);
      }
    }
    if constexpr (CLc > 0) {
      if (dist_chain)
        TC_CHECK_CL(launch_cluster(k_pair_chain_cl<T, N>, dim3(nj_items * P.sc * CLc, nsides), C0::threads,
                                   C0::smem, CLc, st, Pc));
    }
    if (!pruned && !dist_chain) k_pair_chain<T, N><<<dim3(nj_items * P.sc, nsides), TH, Pc.nsmem * vb, st>>>(Pc);
    TC_CHECK_LAUNCH("k_pair_chain");
    stage_mark(ctx, st, 4);
    if (P.sc > 1) {
      k_sum_parts<T, N><<<dim3(2 * pw_blocks, nsides), 256, 0, st>>>(P, 1);
      TC_CHECK_LAUNCH("k_sum_parts");
      nl[4] += 1;
    }
    if (band_corr) {
      // w_j + w_c (3a3, 3b4) and its overlaps (3b4)
      k_band_wc<T, N><<<2 * pw_blocks, 256, 0, st>>>(P, 2);
      k_band_scalars<T, N><<<dim3(S.nkb * S.no * S.nb, 2), 256, 0, st>>>(P, 2);
      TC_CHECK_LAUNCH("band w_c");
      nl[4] += 2;
    }
    Params<T> Pb = P;
    Pb.nsmem = smem_vols<T, N>(2);
    if constexpr (LP < N) {
      if (pruned)
        k_pair_3b4_pr<T, N, LP><<<dim3(nj_items * P.sc, nsides), PrCfg<T, N>::threads,
                                  PrSmem<T, N, LP, 1, 1>::bytes, st>>>(Pb);
    }
    if constexpr (CLb > 0) {
      if (dist_3b4)
        TC_CHECK_CL(launch_cluster(k_pair_3b4_cl<T, N>, dim3(nj_items * P.sc * CLb, nsides), C1::threads, C1::smem,
                                   CLb, st, Pb));
    }
    if (!pruned && !dist_3b4) k_pair_3b4<T, N><<<dim3(nj_items * P.sc, nsides), TH, Pb.nsmem * vb, st>>>(Pb);
    TC_CHECK_LAUNCH("k_pair_3b4");
    if (P.sc > 1 && tw[T3B4] != 0) {
      k_sum_parts<T, N><<<dim3(2 * pw_blocks, nsides), 256, 0, st>>>(P, 2);
      TC_CHECK_LAUNCH("k_sum_parts");
      nl[4] += 1;
    }
  }
  // 5. local terms, corrections, back to the sphere
  stage_mark(ctx, st, 5);
  if (band_corr) {
    k_band_corr<T, N><<<2 * pw_blocks, 256, 0, st>>>(P, 2);
    TC_CHECK_LAUNCH("k_band_corr");
    nl[5] += 1;
  }
  k_finalize<T, N><<<dim3(nj_items, nsides), TH, vb1, st>>>(P, outR, outL, ctx->d_box_index);
  TC_CHECK_LAUNCH("k_finalize");
  if (P.sym && P.nirr < S.Nk) {
    // outputs of the other k-points by the same unfolding as the orbitals (the operator commutes with it)
    const int ru = launch_sym_unfold(ctx, outR, nsides > 1 ? outL : nullptr, st);
    if (ru != TC_OK) return ru;
    nl[5] += 1;
  }
  stage_mark(ctx, st, 6);
  return stage_collect(ctx, 6, nl);
}

template <typename T, int N> int run_fft3d(void* data, int batch, int sign, cudaStream_t st) {
  const int vb = vol_bytes<T, N>();
  const int vb1 = Fit<T, N>::one ? vb : 0;
  cplx<T>* gwork = nullptr;   // boxes too large for shared memory: stream-ordered work volumes
  if (!Fit<T, N>::one && cudaMallocAsync((void**)&gwork, (size_t)batch * vb, st) != cudaSuccess) return TC_ERR_OOM;
  if (sign < 0)
    k_fft3d<T, N, -1><<<batch, Cfg<N>::threads, vb1, st>>>(reinterpret_cast<cplx<T>*>(data), gwork);
  else
    k_fft3d<T, N, +1><<<batch, Cfg<N>::threads, vb1, st>>>(reinterpret_cast<cplx<T>*>(data), gwork);
  const cudaError_t e = cudaGetLastError();
  if (gwork) cudaFreeAsync(gwork, st);
  return e == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

#define TC_INSTANTIATE(T, N)                                                                             \
  template int run_pipeline<T, N>(tc_ctx*, const double2*, const double2*, double2*, double2*, const double*, \
                                  int, cudaStream_t, const double2*, const double2*);                     \
  template int prepare_kernels<T, N>(tc_ctx*);                                                           \
  template int run_fft3d<T, N>(void*, int, int, cudaStream_t);                                           \
  template size_t scratch_needed<T, N>(const Setup&, int, int);

}  // namespace tc
