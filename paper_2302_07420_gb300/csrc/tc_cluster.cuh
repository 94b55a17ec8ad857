// Pair kernels distributed over a thread-block cluster (templated on precision T, box size N,
// support length L and cluster width CL), for boxes whose pruned volumes do not fit one CTA's
// shared memory.
//
// The CL CTAs of a cluster share one item of the pruned kernels of tc_pruned.cuh (one output
// orbital j and partner chunk, or one occupied q2 and partner chunk).  Their work volume
// [L][N][N|1] and compact spectra [L]^3 are split along the first index c1 (the compact axis-1
// index): rank r holds the R = ceil(L / CL) rows c1 in [r R, r R + R) in its own shared memory.
//   * The passes over axes 2 and 3 have pencils at fixed c1 and stay inside the CTA that holds
//     the row (CTA barriers only).
//   * The axis-1 passes (pencils (i2, i3) along c1) are split between the CTAs by pencil: rank r
//     takes pencils [r PEN, r PEN + PEN), PEN = ceil(N^2 / CL), and reads and writes the rows of
//     every CTA through distributed shared memory.
//   * Every pass pair (and every axis-1 pass) ends with a cluster barrier (arrive.release /
//     wait.acquire), which orders the shared-memory rows between CTAs and the global accumulator
//     writes of the cluster -- except the chain's per-component forward passes, which a
//     cluster-barrier-closed inverse pass of the same CTA always follows.  Control flow that reaches a cluster barrier depends only on the
//     launch parameters and the cluster's item, so every CTA of a cluster arrives at every barrier.
// The arithmetic per pair is that of the pruned kernels, exact for the discrete operator whenever
// the pair-density support fits L.
#pragma once
#include <cooperative_groups.h>

#include "tc_pruned.cuh"

namespace tc {

namespace cg = cooperative_groups;

// One kernel's cluster configuration: CTAs per cluster, which compact spectra sit in shared memory
// (spec 1: all; 2: the chain's pair spectrum A only, its accumulator C in the scratch slice; 0: none,
// the spectra in the item's scratch slice, each CTA touching its own rows only), the CTAs per SM its
// launch bounds ask for, the threads per CTA (0: one axis-1 pencil per thread), the elements per
// load chunk of the chain's pointwise pass (its loads for a chunk are issued together), and, for the
// occupied-pair kernel, whether the item's h6 part accumulates in shared memory (h6 = 1: by axis-1
// pencil, each element owned by one thread, written to the item's scratch slot once at the end).
struct ClChoice {
  int cl, spec, minb, thr, ch, h6 = 0;
};

// Cluster plan for box size N: the support length L of the distributed kernels (0: none built; the
// pair-density support of spheres |m| <= r is 4 r + 1, which the plan covers for the boxes of the
// batched HEG cells, 4 floor((N-1)/4) + 1, and with full transforms at 48^3) and the choice per kernel
// (kind 0 pair chain, 1 3b4 pass, 2 occupied pairs).  FP32 takes the choices below, each the fastest of
// the configurations timed per box on the batched HEG cells (2, 3, 4, 6 or 8 CTAs; spectra on chip or
// in L2; 1-3 CTAs per SM; load chunks of 1, 2 or 4): few CTAs per cluster with the spectra on chip
// where they fit generally won over more warps per SM from more, smaller CTAs, whose rows are mostly
// remote and whose barriers have more participants.  FP64 takes the smallest width whose slices fit
// one CTA per SM (with the spectra if they fit too).
template <typename T, int N> struct ClPlan {
  static constexpr int L = (N == 24) ? 21 : (N == 25 || N == 27) ? 25 : (N == 30 || N == 32) ? 29 : (N == 48) ? 48 : 0;
  static constexpr int P = N | 1;
  static constexpr size_t z = sizeof(cplx<T>);
  static constexpr size_t lim = (size_t)kSmemLimit - 2048;
  static constexpr int rows(int cl) { return cl > 0 ? (L + cl - 1) / cl : 0; }
  static constexpr int pens(int cl) { return cl > 0 ? (N * N + cl - 1) / cl : 0; }
  static constexpr int need(int cl) {
    const int t = pens(cl) > rows(cl) * N ? pens(cl) : rows(cl) * N;
    return ((t + 31) / 32) * 32;
  }
  static constexpr int nspec(int kind) { return kind == 1 ? 1 : 2; }
  // bytes of the row slices: work rows (and, for kind 2, B1 by pencil), then the spectra on chip
  static constexpr size_t bytes(int kind, int cl, int spec, int h6 = 0) {
    const size_t b = (size_t)rows(cl) * N * P * z;
    const size_t base = kind == 2 ? (size_t)(h6 ? 2 : 1) * N * pens(cl) * z + b : b;
    const int on_chip = spec == 1 ? nspec(kind) : (spec == 2 ? 1 : 0);
    return base + (size_t)on_chip * rows(cl) * L * L * z;
  }
  static constexpr ClChoice choice64(int kind) {
    if (L == 0) return ClChoice{0, 0, 0, 0, 1};
    for (int cl = 2; cl <= 8; cl *= 2)
      if (bytes(kind, cl, 1) <= lim) return ClChoice{cl, 1, 1, 0, 1};
    for (int cl = 2; cl <= 8; cl *= 2)
      if (bytes(kind, cl, 0) <= lim) return ClChoice{cl, 0, 1, 0, 1};
    return ClChoice{0, 0, 0, 0, 1};
  }
  static constexpr ClChoice choice(int kind) {
    if (sizeof(T) == 8) return choice64(kind);
    switch (N) {
      case 24: return kind == 0 ? ClChoice{2, 1, 1, 0, 4} : ClChoice{2, 1, 1, 0, 1};
      case 25: return kind == 0 ? ClChoice{2, 1, 1, 0, 4} : (kind == 1 ? ClChoice{2, 1, 1, 0, 1} : ClChoice{2, 0, 1, 0, 1, 1});
      case 27: return kind == 0 ? ClChoice{2, 1, 1, 0, 2} : (kind == 1 ? ClChoice{2, 1, 1, 0, 1} : ClChoice{2, 0, 1, 0, 1});
      case 30: return kind == 0 ? ClChoice{2, 2, 1, 0, 1} : (kind == 1 ? ClChoice{2, 1, 1, 0, 1} : ClChoice{2, 0, 1, 0, 1});
      case 32: return kind == 0 ? ClChoice{2, 2, 1, 0, 1} : (kind == 1 ? ClChoice{2, 1, 1, 0, 1} : ClChoice{3, 0, 1, 0, 1});
      case 48: return kind == 0 ? ClChoice{4, 0, 1, 288, 4} : (kind == 1 ? ClChoice{6, 0, 1, 0, 1} : ClChoice{8, 0, 1, 0, 1});
      default: return ClChoice{0, 0, 0, 0, 1};
    }
  }
};

// Compile-time configuration of one cluster kernel (KIND as in ClPlan).
template <typename T, int N, int KIND> struct ClCfg {
  using PL = ClPlan<T, N>;
  static constexpr int L = PL::L;
  static constexpr int CL = PL::choice(KIND).cl;
  static constexpr bool SPEC = PL::choice(KIND).spec == 1;     // every spectrum on chip
  static constexpr bool SPEC_A = PL::choice(KIND).spec != 0;   // the (first) pair spectrum on chip
  static constexpr int MINB = PL::choice(KIND).minb;
  static constexpr int CH = PL::choice(KIND).ch;
  // one axis-1 pencil per thread unless the choice caps the count; FP64 at most 256 threads (a double
  // pencil takes 4 N registers); the passes loop over their pencils, so any count is correct
  static constexpr int want = PL::choice(KIND).thr > 0 ? PL::choice(KIND).thr : PL::need(CL);
  static constexpr int threads = (sizeof(T) == 8 && want > 256) ? 256 : want;
  static constexpr bool H6S = KIND == 2 && PL::choice(KIND).h6 != 0;   // h6 part in shared memory
  static constexpr size_t bytes = PL::bytes(KIND, CL, PL::choice(KIND).spec, H6S ? 1 : 0);
  // kernel-table rows of the current Delta (3 for the chain, 1 for 3b4) when they fit as well
  static constexpr size_t tab_bytes = (size_t)(KIND == 0 ? 3 : 1) * PL::rows(CL) * L * L * sizeof(T);
  static constexpr bool tab = (KIND == 0 ? SPEC : (KIND == 1 && SPEC_A)) &&
                              (size_t)MINB * (bytes + tab_bytes + 2048) <= 233472;
  static constexpr size_t smem = bytes + (tab ? tab_bytes : 0);
  static_assert(CL == 0 || (size_t)MINB * (smem + 2048) <= 233472, "row slices exceed the SM's shared memory");
  static_assert(KIND != 2 || PL::choice(KIND).spec != 2, "the occupied-pair kernel keeps both spectra or none");
};

// Row slices of one CTA (rank r: compact rows [r R, r R + R) and axis-1 pencils [r PEN, r PEN + PEN)).
template <typename T, int N, int L, int CL> struct Dist {
  static constexpr int P = N | 1;
  static constexpr int R = (L + CL - 1) / CL;
  static constexpr int PEN = (N * N + CL - 1) / CL;
  static constexpr int bslab = R * N * P;     // work rows [R][N][P]
  static constexpr int cslab = R * L * L;     // compact spectrum rows [R][L][L]
  static __device__ __forceinline__ int bidx(int r, int i2, int i3) { return (r * N + i2) * P + i3; }
  static __device__ __forceinline__ int cidx(int r, int c2, int c3) { return (r * L + c2) * L + c3; }
};

// Inverse transform, axes 2 and 3, of this CTA's rows of a compact spectrum into its work rows;
// spec(r, c1, c2, c3) gives the value at local row r (compact index c1 = c1_0 + r).
template <typename T, int N, int L, int CL, typename Spec>
__device__ __forceinline__ void cinv_23(cg::cluster_group& cluster, cplx<T>* B, int c1_0, int nrow, Spec spec) {
  using S = Sup<N, L>;
  using D = Dist<T, N, L, CL>;
  for (int p = threadIdx.x; p < nrow * L; p += blockDim.x) {
    const int r = p / L, c3 = p % L;
    cplx<T> v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = cplx<T>{0, 0};
#pragma unroll
    for (int c2 = 0; c2 < L; ++c2) v[S::box(c2)] = spec(r, c1_0 + r, c2, c3);
    Codelet<T, N, +1>::run(v);
#pragma unroll
    for (int i2 = 0; i2 < N; ++i2) B[D::bidx(r, i2, c3)] = v[i2];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < nrow * N; p += blockDim.x) {
    const int r = p / N, i2 = p % N;
    cplx<T> v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = cplx<T>{0, 0};
#pragma unroll
    for (int c3 = 0; c3 < L; ++c3) v[S::box(c3)] = B[D::bidx(r, i2, c3)];
    Codelet<T, N, +1>::run(v);
#pragma unroll
    for (int i3 = 0; i3 < N; ++i3) B[D::bidx(r, i2, i3)] = v[i3];
  }
  cluster.sync();
}

// Axis-1 pass over this CTA's pencils (i2, i3); rb[k] is the work-row slice of rank k (distributed
// shared memory).  FROM_B: the pencil's L spectral values are read from the rows of every CTA and
// inverse-transformed (else load(i1, i2, i3) supplies N real-space values); body(t, i2, i3, v) then
// works on the N real-space values (t: the pencil's index within this CTA); with fwd the pencil is
// forward-transformed and its L support values are written back into the rows of every CTA.
template <typename T, int N, int L, int CL, bool FROM_B, typename Load, typename Body>
__device__ __forceinline__ void caxis1(cg::cluster_group& cluster, cplx<T>* const (&rb)[CL], int rank, Load load,
                                       Body body, bool fwd) {
  using S = Sup<N, L>;
  using D = Dist<T, N, L, CL>;
  const int p0 = rank * D::PEN;
  const int p1 = (p0 + D::PEN < N * N) ? p0 + D::PEN : N * N;
  for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const int i2 = p / N, i3 = p % N;
    cplx<T> v[N];
    if constexpr (FROM_B) {
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] = cplx<T>{0, 0};
#pragma unroll
      for (int c1 = 0; c1 < L; ++c1) v[S::box(c1)] = rb[c1 / D::R][D::bidx(c1 % D::R, i2, i3)];
      Codelet<T, N, +1>::run(v);
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] = load(i, i2, i3);
    }
    body(p - p0, i2, i3, v);
    if (fwd) {
      Codelet<T, N, -1>::run(v);
#pragma unroll
      for (int c1 = 0; c1 < L; ++c1) rb[c1 / D::R][D::bidx(c1 % D::R, i2, i3)] = v[S::box(c1)];
    }
  }
  cluster.sync();
}

// Forward transform, axes 3 and 2, of this CTA's work rows (axis 1 done) onto the support;
// emit(r, c1, c2, c3, value) receives each output of the rows once, from the thread that owns the
// compact pencil (r, c3) -- the same thread that reads it in cinv_23.  It ends with a cluster barrier
// (the next axis-1 pass may write into these rows from another CTA), or with a CTA barrier when
// CSYNC is false: allowed where a cinv_23 of this CTA, which ends with a cluster barrier, comes
// before any such pass.
template <typename T, int N, int L, int CL, bool CSYNC = true, typename Emit>
__device__ __forceinline__ void cfwd_32(cg::cluster_group& cluster, cplx<T>* B, int c1_0, int nrow, Emit emit) {
  using S = Sup<N, L>;
  using D = Dist<T, N, L, CL>;
  for (int p = threadIdx.x; p < nrow * N; p += blockDim.x) {
    const int r = p / N, i2 = p % N;
    cplx<T> v[N];
#pragma unroll
    for (int i3 = 0; i3 < N; ++i3) v[i3] = B[D::bidx(r, i2, i3)];
    Codelet<T, N, -1>::run(v);
#pragma unroll
    for (int c3 = 0; c3 < L; ++c3) B[D::bidx(r, i2, c3)] = v[S::box(c3)];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < nrow * L; p += blockDim.x) {
    const int r = p / L, c3 = p % L;
    cplx<T> v[N];
#pragma unroll
    for (int i2 = 0; i2 < N; ++i2) v[i2] = B[D::bidx(r, i2, c3)];
    Codelet<T, N, -1>::run(v);
#pragma unroll
    for (int c2 = 0; c2 < L; ++c2) emit(r, c1_0 + r, c2, c3, v[S::box(c2)]);
  }
  if constexpr (CSYNC) {
    cluster.sync();
  } else {
    __syncthreads();
  }
}

// Fused pair chains, distributed (same work, accumulators and per-pair arithmetic as
// k_pair_chain_pr; Algs. 2, 5, 6, 9, 11, 12 and the 2bx terms of Sec. 2.6.3).  Grid
// (Nk*nb*sc*CL, sides), clusters of CL CTAs along x; cluster = output orbital j and partner chunk.
template <typename T, int N>
__global__ void __launch_bounds__(ClCfg<T, N, 0>::threads, ClCfg<T, N, 0>::MINB) k_pair_chain_cl(Params<T> P) {
  using SM = ClCfg<T, N, 0>;
  constexpr int L = SM::L, CL = SM::CL;
  using G = Geo<N>;
  using S = Sup<N, L>;
  using D = Dist<T, N, L, CL>;
  constexpr int CH = SM::CH;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ T red[32];
  __shared__ T part[4];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int c1_0 = rank * D::R;
  const int nrow = L - c1_0 < D::R ? (L - c1_0 > 0 ? L - c1_0 : 0) : D::R;
  const SideArgs<T>& SD = P.side[blockIdx.y];
  const int cid = blockIdx.x / CL;
  const int jitem = cid / P.sc, chunk = cid % P.sc;
  const int jo = P.sym ? P.irr[jitem / P.nb] * P.nb + jitem % P.nb : jitem, j = P.j0 + jo, kj = j / P.nb;
  const int M = P.Nk * P.no, nj = P.nj_out;
  const int qi_begin = (int)((long long)chunk * M / P.sc), qi_end = (int)((long long)(chunk + 1) * M / P.sc);
  cplx<T>* B = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* A;
  cplx<T>* C;
  // this CTA's rows of the item's compact spectra in its scratch slots (k_pair_chain's, one item each)
  const size_t item = (size_t)blockIdx.y * (gridDim.x / CL) + blockIdx.x / CL;
  cplx<T>* gA = P.scratch + item * 3 * (size_t)Geo<N>::vol + (size_t)c1_0 * L * L;
  if constexpr (SM::SPEC) {
    A = B + D::bslab;
    C = A + D::cslab;
  } else if constexpr (SM::SPEC_A) {
    A = B + D::bslab;
    C = gA + Sup<N, L>::cvol;
  } else {
    A = gA;
    C = gA + Sup<N, L>::cvol;
  }
  T* tU = SM::tab ? reinterpret_cast<T*>(C + D::cslab) : nullptr;
  cplx<T>* rb[CL];
#pragma unroll
  for (int k = 0; k < CL; ++k) rb[k] = cluster.map_shared_rank(B, k);
  const size_t NN = G::nn;
  const cplx<T>* ketj = SD.ket + (size_t)j * NN;
  const cplx<T>* Yj = SD.Y + (size_t)jo * 3 * NN;
  cplx<T>* acc = SD.acc + ((size_t)chunk * nj + jo) * NN;
  cplx<T>* w = SD.w + ((size_t)chunk * nj + jo) * 3 * NN;
  const T* tw = P.tw;
  const bool need_w = tw[T3A3] != T(0) || tw[T3B4] != T(0);
  const bool need_z = tw[T2BX1] != T(0) || tw[T3A4] != T(0);
  const bool need_y = tw[T3B3] != T(0) || tw[T2BX2] != T(0);
  const bool need_pp = need_w || need_z || tw[T3B6] != T(0);
  const bool need_F = need_y || tw[T3B5] != T(0) || tw[T3B6] != T(0);
  const bool need_ap = tw[T3B6] != T(0) && !P.no_ap;
  const T t3b5 = tw[T3B5], t3b6 = tw[T3B6], t2ax = tw[T2AX];
  for (int r = rank * blockDim.x + threadIdx.x; r < (int)NN; r += CL * blockDim.x) {
    acc[r] = cplx<T>{0, 0};
    for (int d = 0; d < 3; ++d) w[d * NN + r] = cplx<T>{0, 0};
  }
  int staged = -1;   // Delta whose kernel-table rows are in shared memory
  for (int qi = qi_begin; qi < qi_end; ++qi) {
    const int kq = qi / P.no, mu = qi % P.no;
    const int q = kq * P.nb + mu;
    const T f = (T)(P.occ[q] / P.Nk);
    if (f == T(0)) continue;
    const int did = P.delta_id[kj * P.kstride + kq];
    const T* dl = P.delta + did * 3;
    const T* Vt = SD.tabV + ((size_t)did * 2 + SD.side) * NN;
    const T* Upp = P.tabU + ((size_t)did * 2 + 0) * NN;
    const T* Uap = P.tabU + ((size_t)did * 2 + 1) * NN;
    if constexpr (SM::tab) {
      if (did != staged) {
        // the previous pair's last reads of the rows ended before its closing barrier
        for (int c = threadIdx.x; c < nrow * L * L; c += blockDim.x) {
          const int g = gidx_c<N, L>(c1_0 + c / (L * L), (c / L) % L, c % L);
          tU[c] = Upp[g];
          tU[D::cslab + c] = Uap[g];
          tU[2 * D::cslab + c] = Vt[g];
        }
        staged = did;   // first read after the barriers of the forward transform below
      }
    }
    auto tab = [&](int which, int r, int c1, int c2, int c3) -> T {
      if constexpr (SM::tab) {
        return tU[which * D::cslab + D::cidx(r, c2, c3)];
      } else {
        const T* t = which == 0 ? Upp : (which == 1 ? Uap : Vt);
        return t[gidx_c<N, L>(c1, c2, c3)];
      }
    };
    const cplx<T>* braq = SD.bra + (size_t)q * NN;
    const cplx<T>* ketq = SD.ket + (size_t)q * NN;
    const cplx<T>* Zq = SD.Z + ((size_t)(kq * P.no + mu) * 3) * NN;
    const cplx<T>* h3bq = SD.h3b + ((size_t)(kq * P.no + mu) * 3) * NN;
    // A = FT[conj(bra_q) ket_j] on the support
    caxis1<T, N, L, CL, false>(
        cluster, rb, rank,
        [&](int a, int b, int c) { const int g = G::gidx(a, b, c); return mulc(ldg(ketj + g), ldg(braq + g)); },
        [&](int, int, int, cplx<T>(&)[N]) {}, true);
    cfwd_32<T, N, L, CL>(cluster, B, c1_0, nrow,
                         [&](int r, int, int c2, int c3, cplx<T> v) { A[D::cidx(r, c2, c3)] = P.invN * v; });
    if (P.div && kq == kj && t3b6 != T(0)) {
      // O_qj = A(0) and X_s = sum_{G != 0} u~_s(G) A(G) n~(-G) for the 3b6 corrections: partial sums
      // over this CTA's rows, added up by rank 0
      for (int s = 0; s < 2; ++s) {
        T xr = 0, xi = 0;
        for (int c = threadIdx.x; c < nrow * L * L; c += blockDim.x) {
          const int a = S::box(c1_0 + c / (L * L)), b = S::box((c / L) % L), e = S::box(c % L);
          const int gn = G::gidx((N - a) % N, (N - b) % N, (N - e) % N);
          const cplx<T> t = P.hartUs[(size_t)s * NN + G::gidx(a, b, e)] * (A[c] * SD.nt[gn]);
          xr += t.x;
          xi += t.y;
        }
        const T sr = block_sum<T>(xr, red);
        const T si = block_sum<T>(xi, red);
        if (threadIdx.x == 0) {
          part[2 * s] = sr;
          part[2 * s + 1] = si;
        }
      }
      cluster.sync();
      if (rank == 0 && threadIdx.x == 0) {
        double* cs = SD.cs + ((size_t)jo * P.no + mu) * 6;
        for (int e = 0; e < 4; ++e) {
          T sum = 0;
          for (int k = 0; k < CL; ++k) sum += cluster.map_shared_rank(part, k)[e];
          cs[2 + e] = sum;
        }
        cs[0] = A[0].x;
        cs[1] = A[0].y;
      }
    }
    for (int sp = 0; sp < 2; ++sp) {
      if (sp == 0 && !(need_pp || need_F)) continue;
      if (sp == 1 && !need_ap) continue;
      for (int d = 0; d < 3; ++d) {
        const bool first_C = (sp == 0 && d == 0);
        const PComp<T> qd = pcomp_setup<T>(P, dl, d);
        // b = FT^{-1}[U_d A]
        cinv_23<T, N, L, CL>(cluster, B, c1_0, nrow, [&](int r, int c1, int c2, int c3) {
          return mul_si<T, 1>((pcomp_c<T, N, L>(qd, c1, c2, c3) * tab(sp, r, c1, c2, c3)) * A[D::cidx(r, c2, c3)]);
        });
        const bool fwd = sp == 1 || need_F;
        caxis1<T, N, L, CL, true>(
            cluster, rb, rank, [&](int, int, int) { return cplx<T>{0, 0}; },
            [&](int, int i2, int i3, cplx<T>(&v)[N]) {
              if (sp == 0) {
#pragma unroll
                for (int c0 = 0; c0 < N; c0 += CH) {
                  cplx<T> lz[CH], lk[CH], ly[CH], lb[CH], lj[CH], lh[CH], ln[CH];
#pragma unroll
                  for (int u = 0; u < CH; ++u) {
                    if (c0 + u >= N) continue;
                    const int g = G::gidx(c0 + u, i2, i3);
                    if (need_z) lz[u] = ldg(Zq + d * NN + g);
                    lk[u] = ldg(ketq + g);
                    if (need_F) {
                      ly[u] = ldg(Yj + d * NN + g);
                      lb[u] = ldg(braq + g);
                      lj[u] = ldg(ketj + g);
                      lh[u] = ldg(h3bq + d * NN + g);
                      ln[u] = ldg(SD.n + g);
                    }
                  }
#pragma unroll
                  for (int u = 0; u < CH; ++u) {
                    if (c0 + u >= N) continue;
                    const int g = G::gidx(c0 + u, i2, i3);
                    const cplx<T> bv = v[c0 + u];
                    if (need_z) red_add_v(&acc[g], f * (lz[u] * bv));
                    if (need_w) red_add_v(&w[d * NN + g], f * (lk[u] * bv));
                    cplx<T> F = {0, 0};
                    if (need_F) {
                      if (need_y) F = mulc(ly[u], lb[u]);
                      if (t3b5 != T(0)) F = F - t3b5 * (lj[u] * lh[u]);
                      if (t3b6 != T(0)) F = F + t3b6 * (ln[u] * bv);
                    }
                    v[c0 + u] = F;
                  }
                }
              } else {
#pragma unroll
                for (int i = 0; i < N; ++i) v[i] = t3b6 * (ldg(SD.n + G::gidx(i, i2, i3)) * v[i]);
              }
            },
            fwd);
        if (!fwd) continue;
        // C += -U_d FT[F] = -i p_d u FT[F]; a cinv_23 always follows (the next component's or the
        // final one: C is then nonzero), so a CTA barrier closes the pass
        cfwd_32<T, N, L, CL, false>(cluster, B, c1_0, nrow, [&](int r, int c1, int c2, int c3, cplx<T> v) {
          const T k = pcomp_c<T, N, L>(qd, c1, c2, c3) * tab(sp, r, c1, c2, c3) * P.invN;
          const cplx<T> t = mul_si<T, -1>(k * v);
          const int s = D::cidx(r, c2, c3);
          C[s] = first_C ? t : C[s] + t;
        });
      }
    }
    const bool has_C = need_F || need_ap;
    if (has_C || t2ax != T(0)) {
      cinv_23<T, N, L, CL>(cluster, B, c1_0, nrow, [&](int r, int c1, int c2, int c3) {
        const int s = D::cidx(r, c2, c3);
        cplx<T> v = has_C ? C[s] : cplx<T>{0, 0};
        if (t2ax != T(0)) v = v - (t2ax * tab(2, r, c1, c2, c3)) * A[s];
        return v;
      });
      caxis1<T, N, L, CL, true>(
          cluster, rb, rank, [&](int, int, int) { return cplx<T>{0, 0}; },
          [&](int, int i2, int i3, cplx<T>(&v)[N]) {
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 4) {
              cplx<T> lk[4];
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (c0 + u < N) lk[u] = ldg(ketq + G::gidx(c0 + u, i2, i3));
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (c0 + u < N) red_add_v(&acc[G::gidx(c0 + u, i2, i3)], f * (lk[u] * v[c0 + u]));
            }
          },
          false);
    }
  }
  // no CTA leaves while another may still read its rows or partial sums
  cluster.sync();
}

// Pass 2 for 3b4 (Alg. 10), distributed: acc += tw3b4 f ket_q FT^{-1}[-U^pp . FT[-conj(bra_q) w_j]]
// (same grid and accumulators as k_pair_3b4, clusters of CL CTAs along x).
template <typename T, int N>
__global__ void __launch_bounds__(ClCfg<T, N, 1>::threads, ClCfg<T, N, 1>::MINB) k_pair_3b4_cl(Params<T> P) {
  using SM = ClCfg<T, N, 1>;
  constexpr int L = SM::L, CL = SM::CL;
  using G = Geo<N>;
  using D = Dist<T, N, L, CL>;
  extern __shared__ __align__(16) unsigned char smraw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int c1_0 = rank * D::R;
  const int nrow = L - c1_0 < D::R ? (L - c1_0 > 0 ? L - c1_0 : 0) : D::R;
  const SideArgs<T>& SD = P.side[blockIdx.y];
  const int cid = blockIdx.x / CL;
  const int jitem = cid / P.sc, chunk = cid % P.sc;
  const int jo = P.sym ? P.irr[jitem / P.nb] * P.nb + jitem % P.nb : jitem, j = P.j0 + jo, kj = j / P.nb;
  const int M = P.Nk * P.no, nj = P.nj_out;
  const int qi_begin = (int)((long long)chunk * M / P.sc), qi_end = (int)((long long)(chunk + 1) * M / P.sc);
  cplx<T>* B = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* A;
  if constexpr (SM::SPEC_A) {
    A = B + D::bslab;
  } else {
    const size_t item = (size_t)blockIdx.y * (gridDim.x / CL) + blockIdx.x / CL;
    A = P.scratch + item * 2 * (size_t)Geo<N>::vol + (size_t)c1_0 * L * L;
  }
  T* tU = SM::tab ? reinterpret_cast<T*>(A + D::cslab) : nullptr;
  cplx<T>* rb[CL];
#pragma unroll
  for (int k = 0; k < CL; ++k) rb[k] = cluster.map_shared_rank(B, k);
  const size_t NN = G::nn;
  cplx<T>* acc = SD.acc + ((size_t)chunk * nj + jo) * NN;
  const cplx<T>* w = SD.w + (size_t)jo * 3 * NN;
  const T t3b4 = P.tw[T3B4];
  if (t3b4 == T(0)) return;   // uniform over the launch, before any cluster access
  if (chunk > 0) {
    for (int r = rank * blockDim.x + threadIdx.x; r < (int)NN; r += CL * blockDim.x) acc[r] = cplx<T>{0, 0};
    cluster.sync();
  }
  int staged = -1;
  for (int qi = qi_begin; qi < qi_end; ++qi) {
    const int kq = qi / P.no, mu = qi % P.no;
    const int q = kq * P.nb + mu;
    const T f = (T)(P.occ[q] / P.Nk);
    if (f == T(0)) continue;
    const int did = P.delta_id[kj * P.kstride + kq];
    const T* dl = P.delta + did * 3;
    const T* Upp = P.tabU + ((size_t)did * 2 + 0) * NN;
    if constexpr (SM::tab) {
      if (did != staged) {
        for (int c = threadIdx.x; c < nrow * L * L; c += blockDim.x)
          tU[c] = Upp[gidx_c<N, L>(c1_0 + c / (L * L), (c / L) % L, c % L)];
        staged = did;
      }
    }
    auto tab = [&](int r, int c1, int c2, int c3) -> T {
      if constexpr (SM::tab) return tU[D::cidx(r, c2, c3)];
      else return Upp[gidx_c<N, L>(c1, c2, c3)];
    };
    const cplx<T>* braq = SD.bra + (size_t)q * NN;
    const cplx<T>* ketq = SD.ket + (size_t)q * NN;
    for (int d = 0; d < 3; ++d) {
      const PComp<T> qd = pcomp_setup<T>(P, dl, d);
      caxis1<T, N, L, CL, false>(
          cluster, rb, rank,
          [&](int a, int b, int c) { const int g = G::gidx(a, b, c); return mulc(ldg(w + d * NN + g), ldg(braq + g)); },
          [&](int, int, int, cplx<T>(&)[N]) {}, true);
      // -U_d FT[-conj(bra_q) w_d] = +i p_d u FT[conj(bra_q) w_d]
      cfwd_32<T, N, L, CL>(cluster, B, c1_0, nrow, [&](int r, int c1, int c2, int c3, cplx<T> v) {
        const T k = pcomp_c<T, N, L>(qd, c1, c2, c3) * tab(r, c1, c2, c3) * P.invN;
        const cplx<T> t = mul_si<T, 1>(k * v);
        const int s = D::cidx(r, c2, c3);
        A[s] = d == 0 ? t : A[s] + t;
      });
    }
    const T fw = t3b4 * f;
    cinv_23<T, N, L, CL>(cluster, B, c1_0, nrow, [&](int r, int, int c2, int c3) { return A[D::cidx(r, c2, c3)]; });
    caxis1<T, N, L, CL, true>(
        cluster, rb, rank, [&](int, int, int) { return cplx<T>{0, 0}; },
        [&](int, int i2, int i3, cplx<T>(&v)[N]) {
#pragma unroll
          for (int c0 = 0; c0 < N; c0 += 4) {
            cplx<T> lk[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (c0 + u < N) lk[u] = ldg(ketq + G::gidx(c0 + u, i2, i3));
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (c0 + u < N) red_add_v(&acc[G::gidx(c0 + u, i2, i3)], fw * (lk[u] * v[c0 + u]));
          }
        },
        false);
  }
  cluster.sync();
}

// Occupied-pair stage, distributed (same grid, outputs, per-item h6 part and arithmetic as
// k_occ_pairs_pr; Algs. 4, 6, 8, 11 and the 3a2 corrections of Eqs. divcor_3a2_first/second in the
// general-overlap form); clusters of CL CTAs along x, cluster = occupied q2 and partner chunk.
// Shared memory: B1 = P^s_d(q2, q1) in real space, held by the CTA that owns each axis-1 pencil
// ([N][PEN], element i of local pencil t at i PEN + t); the work rows; the rows of A1 and A2.  The
// 3a2 spectrum F_ab (compact, slot 2) and the h6 part (slot 4) are in the item's scratch slice.
template <typename T, int N>
__global__ void __launch_bounds__(ClCfg<T, N, 2>::threads, ClCfg<T, N, 2>::MINB) k_occ_pairs_cl(Params<T> P) {
  using SM = ClCfg<T, N, 2>;
  constexpr int L = SM::L, CL = SM::CL;
  using G = Geo<N>;
  using S = Sup<N, L>;
  using D = Dist<T, N, L, CL>;
  constexpr int NS = 6;
  constexpr int CH = sizeof(T) == 4 ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sO[2][2];
  __shared__ double sF0[2];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int c1_0 = rank * D::R;
  const int nrow = L - c1_0 < D::R ? (L - c1_0 > 0 ? L - c1_0 : 0) : D::R;
  const SideArgs<T>& SD = P.side[blockIdx.y];
  const int M = P.Nk * P.no;
  const int cid = blockIdx.x / CL;
  const int item = cid / P.so, chunk = cid % P.so;
  const int i2 = P.sym ? P.irr[item / P.no] * P.no + item % P.no : P.i2_0 + item;
  const int k2 = i2 / P.no, mu2 = i2 % P.no;
  const int q2 = k2 * P.nb + mu2;
  const int i1_begin = (int)((long long)chunk * M / P.so), i1_end = (int)((long long)(chunk + 1) * M / P.so);
  const size_t cta = (size_t)blockIdx.y * (gridDim.x / CL) + cid;   // item index of the h6 parts
  cplx<T>* slice = P.scratch + cta * NS * (size_t)G::vol;
  cplx<T>* FAB = slice + 2 * (size_t)G::vol;
  cplx<T>* H6 = slice + 4 * (size_t)G::vol;
  cplx<T>* R1 = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* H6s = R1 + (size_t)N * D::PEN;                       // used when SM::H6S
  cplx<T>* W = SM::H6S ? H6s + (size_t)N * D::PEN : H6s;
  cplx<T>* A1;
  cplx<T>* A2;
  if constexpr (SM::SPEC) {
    A1 = W + D::bslab;
    A2 = A1 + D::cslab;
  } else {
    A1 = slice + (size_t)c1_0 * L * L;
    A2 = slice + (size_t)G::vol + (size_t)c1_0 * L * L;
  }
  cplx<T>* rb[CL];
#pragma unroll
  for (int k = 0; k < CL; ++k) rb[k] = cluster.map_shared_rank(W, k);
  const size_t NN = G::nn;
  const T f2 = (T)(P.occ[q2] / P.Nk);
  cplx<T>* h3a4 = SD.h3a4 + ((size_t)chunk * P.nq2 + (i2 - P.i2_0)) * 3 * NN;
  cplx<T>* h3b = SD.h3b + ((size_t)chunk * P.nq2 + (i2 - P.i2_0)) * 3 * NN;
  const cplx<T>* bra2 = SD.bra + (size_t)q2 * NN;
  const cplx<T>* ket2 = SD.ket + (size_t)q2 * NN;
  const int tid = rank * blockDim.x + threadIdx.x, nthr = CL * blockDim.x;
  for (int r = tid; r < S::cvol; r += nthr) FAB[r] = cplx<T>{0, 0};
  if constexpr (SM::H6S) {
    for (int r = threadIdx.x; r < N * D::PEN; r += blockDim.x) H6s[r] = cplx<T>{0, 0};
  }
  for (int r = tid; r < (int)NN; r += nthr) {
    if constexpr (!SM::H6S) H6[r] = cplx<T>{0, 0};
    for (int d = 0; d < 3; ++d) {
      h3a4[d * NN + r] = cplx<T>{0, 0};
      h3b[d * NN + r] = cplx<T>{0, 0};
    }
  }
  if (threadIdx.x == 0) { sF0[0] = 0.0; sF0[1] = 0.0; }
  cluster.sync();
  for (int i1 = i1_begin; i1 < i1_end; ++i1) {
    const int k1 = i1 / P.no, mu1 = i1 % P.no;
    const int q1 = k1 * P.nb + mu1;
    const T f1 = (T)(P.occ[q1] / P.Nk);
    if (f1 == T(0) || f2 == T(0)) continue;
    const int id12 = P.delta_id[k2 * P.kstride + k1];   // Delta = k2 - k1 -> for P(q1,q2)
    const int id21 = P.delta_id[k1 * P.kstride + k2];   // Delta = k1 - k2 -> for P(q2,q1)
    const T* d12 = P.delta + id12 * 3;
    const T* d21 = P.delta + id21 * 3;
    const cplx<T>* bra1 = SD.bra + (size_t)q1 * NN;
    const cplx<T>* ket1 = SD.ket + (size_t)q1 * NN;
    // A1 = FT[conj(bra_q2) ket_q1], A2 = FT[conj(bra_q1) ket_q2]
    caxis1<T, N, L, CL, false>(
        cluster, rb, rank,
        [&](int a, int b, int c) { const int g = G::gidx(a, b, c); return mulc(ldg(ket1 + g), ldg(bra2 + g)); },
        [&](int, int, int, cplx<T>(&)[N]) {}, true);
    cfwd_32<T, N, L, CL>(cluster, W, c1_0, nrow,
                         [&](int r, int, int c2, int c3, cplx<T> v) { A1[D::cidx(r, c2, c3)] = P.invN * v; });
    caxis1<T, N, L, CL, false>(
        cluster, rb, rank,
        [&](int a, int b, int c) { const int g = G::gidx(a, b, c); return mulc(ldg(ket2 + g), ldg(bra1 + g)); },
        [&](int, int, int, cplx<T>(&)[N]) {}, true);
    cfwd_32<T, N, L, CL>(cluster, W, c1_0, nrow,
                         [&](int r, int, int c2, int c3, cplx<T> v) { A2[D::cidx(r, c2, c3)] = P.invN * v; });
    // 3a2 correction pieces for pairs at the same k (Eqs. divcor_3a2_*_density_matrix_mixing);
    // A1(0) and A2(0) are in rank 0's first row
    if (P.div && k1 == k2) {
      if (threadIdx.x == 0) {
        cplx<T> o21, o12;
        if constexpr (SM::SPEC) {
          o21 = cluster.map_shared_rank(A1, 0)[0];
          o12 = cluster.map_shared_rank(A2, 0)[0];
        } else {
          o21 = slice[0];
          o12 = slice[G::vol];
        }
        sO[0][0] = o21.x; sO[0][1] = o21.y; sO[1][0] = o12.x; sO[1][1] = o12.y;
        const double fq = P.occ[q1];
        sF0[0] += fq * ((double)o21.x * o12.x - (double)o21.y * o12.y);
        sF0[1] += fq * ((double)o21.x * o12.y + (double)o21.y * o12.x);
      }
      __syncthreads();
      const cplx<T> o21 = {(T)sO[0][0], (T)sO[0][1]}, o12 = {(T)sO[1][0], (T)sO[1][1]};
      const T fq = (T)P.occ[q1];
      cplx<T>* fab = FAB + (size_t)c1_0 * L * L;   // this CTA's rows (compact layout)
      for (int r = threadIdx.x; r < nrow * L * L; r += blockDim.x) fab[r] = fab[r] + fq * (o12 * A1[r] + o21 * A2[r]);
    }
    // antiparallel channel: each unordered pair once (see k_occ_pairs)
    const int cyc = (i1 - i2 + M) % M;
    const bool ap_here = P.sym || cyc == 0 || 2 * cyc < M || (2 * cyc == M && i2 < i1);
    const T ap_w = (P.sym || cyc == 0) ? T(1) : T(2);
    for (int sp = 0; sp < 2; ++sp) {
      if (sp == 1 && (!ap_here || P.h3_only || P.no_ap)) continue;
      const T w12 = (sp == 1 ? ap_w : T(1)) * (f1 * f2);
      const T* U21 = P.tabU + ((size_t)id21 * 2 + sp) * NN;
      const T* U12 = P.tabU + ((size_t)id12 * 2 + sp) * NN;
      for (int d = 0; d < 3; ++d) {
        const PComp<T> q21 = pcomp_setup<T>(P, d21, d), q12 = pcomp_setup<T>(P, d12, d);
        // B1 = P^s_d(q2, q1), kept in real space by the owner of each axis-1 pencil
        cinv_23<T, N, L, CL>(cluster, W, c1_0, nrow, [&](int r, int c1, int c2, int c3) {
          return mul_si<T, 1>((pcomp_c<T, N, L>(q21, c1, c2, c3) * U21[gidx_c<N, L>(c1, c2, c3)]) *
                              A1[D::cidx(r, c2, c3)]);
        });
        caxis1<T, N, L, CL, true>(
            cluster, rb, rank, [&](int, int, int) { return cplx<T>{0, 0}; },
            [&](int t, int, int, cplx<T>(&v)[N]) {
#pragma unroll
              for (int i = 0; i < N; ++i) R1[i * D::PEN + t] = v[i];
            },
            false);
        // B2 = P^s_d(q1, q2); its axis-1 pass forms the products with B1
        cinv_23<T, N, L, CL>(cluster, W, c1_0, nrow, [&](int r, int c1, int c2, int c3) {
          return mul_si<T, 1>((pcomp_c<T, N, L>(q12, c1, c2, c3) * U12[gidx_c<N, L>(c1, c2, c3)]) *
                              A2[D::cidx(r, c2, c3)]);
        });
        caxis1<T, N, L, CL, true>(
            cluster, rb, rank, [&](int, int, int) { return cplx<T>{0, 0}; },
            [&](int t, int a2, int a3, cplx<T>(&v)[N]) {
#pragma unroll
              for (int c0 = 0; c0 < N; c0 += CH) {
                cplx<T> lb1[CH], lk[CH], lr[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                  if (c0 + u >= N) continue;
                  const int g = G::gidx(c0 + u, a2, a3);
                  lb1[u] = R1[(c0 + u) * D::PEN + t];
                  if (sp == 0) {
                    lk[u] = ldg(ket1 + g);
                    lr[u] = ldg(bra1 + g);
                  }
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                  if (c0 + u >= N) continue;
                  const int g = G::gidx(c0 + u, a2, a3);
                  const cplx<T> b2 = v[c0 + u];
                  if constexpr (SM::H6S) {
                    cplx<T>& h = H6s[(c0 + u) * D::PEN + t];
                    h = h + w12 * (lb1[u] * b2);
                  } else {
                    red_add_v(&H6[g], w12 * (lb1[u] * b2));
                  }
                  if (sp == 0) {
                    red_add_v(&h3a4[d * NN + g], f1 * (b2 * lk[u]));
                    red_add_v(&h3b[d * NN + g], f1 * mulc(lb1[u], lr[u]));
                  }
                }
              }
            },
            false);
      }
    }
  }
  // 3a2 corrections of this q2: (f2/Nk)/Omega^2 sum_s [c_s F0 + (4 pi A_s/Nk) FT^{-1}[u~_s F_ab]]
  if (P.div && f2 != T(0) && !P.h3_only) {
    const T pref = (T)(f2 * P.invOm2);
    const T c0 = (T)(P.corr_c[0] + P.corr_c[1]);
    const cplx<T> cF0 = {(T)(c0 * sF0[0]), (T)(c0 * sF0[1])};
    const T a0 = (T)(4.0 * 3.14159265358979323846 * P.A[0] / P.Nk), a1 = (T)(4.0 * 3.14159265358979323846 * P.A[1] / P.Nk);
    cinv_23<T, N, L, CL>(cluster, W, c1_0, nrow, [&](int, int c1, int c2, int c3) {
      const int g = gidx_c<N, L>(c1, c2, c3);
      const T u = a0 * P.hartUs[g] + a1 * P.hartUs[NN + g];
      return u * FAB[S::cidx(c1, c2, c3)];
    });
    caxis1<T, N, L, CL, true>(
        cluster, rb, rank, [&](int, int, int) { return cplx<T>{0, 0}; },
        [&](int t, int a2, int a3, cplx<T>(&v)[N]) {
#pragma unroll
          for (int i = 0; i < N; ++i) {
            if constexpr (SM::H6S) {
              H6s[i * D::PEN + t] = H6s[i * D::PEN + t] + pref * (v[i] + cF0);
            } else {
              red_add_v(&H6[G::gidx(i, a2, a3)], pref * (v[i] + cF0));
            }
          }
        },
        false);
  }
  if constexpr (SM::H6S) {
    // the item's h6 part: this CTA's pencils, by the threads that accumulated them
    const int p0 = rank * D::PEN;
    const int p1 = (p0 + D::PEN < N * N) ? p0 + D::PEN : N * N;
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
      const int a2 = p / N, a3 = p % N, t = p - p0;
      for (int i = 0; i < N; ++i) H6[G::gidx(i, a2, a3)] = H6s[i * D::PEN + t];
    }
  }
  cluster.sync();
}

}  // namespace tc
