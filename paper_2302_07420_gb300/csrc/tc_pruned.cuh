// Pair chains with pruned transforms (templated on precision T, box size N and support length L).
//
// Every transform of a pair chain has its spectrum on the support of the pair densities: the
// forward transform of a pair density chi_q^* phi_j has nonzero coefficients only at m_j - m_q
// (sphere Miller vectors, cyclic on the box), and every spectral accumulator of the chain is
// consumed only through ket_q FT^{-1}[.], whose projection onto the sphere of k_j reads it at those
// same indices.  When the Miller span s of all spheres satisfies 2 s + 1 <= L, the support per axis
// lies in the L box indices {0 .. (L-1)/2} U {N - (L-1)/2 .. N-1}, so
//   * an inverse transform reads L^3 spectral values: the axis-2 pass runs over L^2 pencils with
//     L nonzero inputs each, the axis-3 pass over L N pencils with L nonzero inputs, and only the
//     axis-1 pass produces the full N^3 real-space values;
//   * a forward transform keeps L outputs per pencil in the same passes in reverse order;
//   * the pair spectrum A and the spectral accumulator C are stored compactly ([L]^3), next to the
//     work volume [L][N][N|1] (first index: compact axis-1 index) in shared memory.
// This is exact for the discrete operator (the dropped coefficients are zero there).  Compact
// index c maps to box index box(c) = c for c < (L+1)/2 and c + N - L otherwise; L = N means no
// pruning (box(c) = c).
#pragma once
#include "tc_kernels.cuh"

namespace tc {

template <int N, int L> struct Sup {
  static_assert(L <= N, "support longer than the box");
  static constexpr int H = (L == N) ? N : (L + 1) / 2;
  static constexpr int P = N | 1;              // row pitch of the work volume
  static constexpr int bvol = L * N * P;       // work volume [L][N][P]
  static constexpr int cvol = L * L * L;       // compact spectrum [L][L][L]
  static __host__ __device__ constexpr int box(int c) { return c < H ? c : c + N - L; }
  // Miller integer of compact index c
  static __host__ __device__ constexpr int mil(int c) {
    return (L == N) ? (c <= (N - 1) / 2 ? c : c - N) : (c < H ? c : c - L);
  }
  // compact index of the negated Miller integer (L < N: the support is symmetric and clear of the
  // Nyquist index, so -m is again on the support)
  static __host__ __device__ constexpr int refl(int c) { return c == 0 ? 0 : L - c; }
  static __device__ __forceinline__ int bidx(int c1, int i2, int i3) { return (c1 * N + i2) * P + i3; }
  static __device__ __forceinline__ int cidx(int c1, int c2, int c3) { return (c1 * L + c2) * L + c3; }
};

// Support length of the pruned kernels compiled for box size N (N: not compiled pruned): 17 at 24^3
// (the silicon-like 4x4x4 cell's spheres) and the supports 4 floor((N-1)/4) + 1 of the batched HEG
// cells' spheres at 16^3, 18^3 and 20^3.
template <int N> constexpr int kPruneL = (N == 16) ? 13 : (N == 18 || N == 20 || N == 24) ? 17 : N;

// Threads per CTA of the pruned kernels: one axis-1 pencil per thread in FP32, two in FP64
// (a pencil of N double-complex values takes 4 N registers).
template <typename T, int N> struct PrCfg {
  static constexpr int threads = sizeof(T) == 4 ? ((N * N + 31) / 32) * 32 : ((N * N / 2 + 31) / 32) * 32;
};

// Shared-memory plan: work volume B first; the compact spectra A and C and the three kernel tables
// of the current Delta (U_pp, U_ap, V on the support) follow when they fit, else A and C live in a
// per-CTA slice of the global scratch and the tables are read from the full-box tables.
template <typename T, int N, int L, int NSPEC, int NTAB> struct PrSmem {
  using S = Sup<N, L>;
  static constexpr size_t bB = (size_t)S::bvol * sizeof(cplx<T>);
  static constexpr size_t bC = (size_t)S::cvol * sizeof(cplx<T>);
  static constexpr size_t bT = (size_t)S::cvol * sizeof(T);
  static constexpr size_t lim = (size_t)kSmemLimit - 1024;
  static constexpr bool spec = bB + NSPEC * bC <= lim;
  static constexpr bool tab = spec && bB + NSPEC * bC + NTAB * bT <= lim;
  static constexpr size_t bytes = bB + (spec ? NSPEC * bC : 0) + (tab ? NTAB * bT : 0);
};

// *p += v in L2 without a return value; FP32 complex as one vector reduction.
__device__ __forceinline__ void red_add_v(cplx<float>* p, cplx<float> v) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void red_add_v(cplx<double>* p, cplx<double> v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

// Inverse transform, axes 2 and 3, of a compact spectrum spec(c1, c2, c3) into the work volume.
template <typename T, int N, int L, typename Spec>
__device__ __forceinline__ void pinv_23(cplx<T>* B, Spec spec) {
  using S = Sup<N, L>;
  for (int p = threadIdx.x; p < L * L; p += blockDim.x) {
    const int c1 = p / L, c3 = p % L;
    cplx<T> v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = cplx<T>{0, 0};
#pragma unroll
    for (int c2 = 0; c2 < L; ++c2) v[S::box(c2)] = spec(c1, c2, c3);
    Codelet<T, N, +1>::run(v);
#pragma unroll
    for (int i2 = 0; i2 < N; ++i2) B[S::bidx(c1, i2, c3)] = v[i2];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < L * N; p += blockDim.x) {
    const int c1 = p / N, i2 = p % N;
    cplx<T> v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = cplx<T>{0, 0};
#pragma unroll
    for (int c3 = 0; c3 < L; ++c3) v[S::box(c3)] = B[S::bidx(c1, i2, c3)];
    Codelet<T, N, +1>::run(v);
#pragma unroll
    for (int i3 = 0; i3 < N; ++i3) B[S::bidx(c1, i2, i3)] = v[i3];
  }
  __syncthreads();
}

// Axis-1 pass over the N^2 pencils (i2, i3).  FROM_B: the pencil's L spectral values are read from
// the work volume and inverse-transformed (else load(i1, i2, i3) supplies N real-space values);
// body(i2, i3, v) then works on the N real-space values; with fwd the pencil is forward-transformed
// and its L support values are written back into the work volume.
template <typename T, int N, int L, bool FROM_B, typename Load, typename Body>
__device__ __forceinline__ void pass_axis1(cplx<T>* B, Load load, Body body, bool fwd) {
  using S = Sup<N, L>;
  for (int p = threadIdx.x; p < N * N; p += blockDim.x) {
    const int i2 = p / N, i3 = p % N;
    cplx<T> v[N];
    if constexpr (FROM_B) {
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] = cplx<T>{0, 0};
#pragma unroll
      for (int c1 = 0; c1 < L; ++c1) v[S::box(c1)] = B[S::bidx(c1, i2, i3)];
      Codelet<T, N, +1>::run(v);
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] = load(i, i2, i3);
    }
    body(i2, i3, v);
    if (fwd) {
      Codelet<T, N, -1>::run(v);
#pragma unroll
      for (int c1 = 0; c1 < L; ++c1) B[S::bidx(c1, i2, i3)] = v[S::box(c1)];
    }
  }
  __syncthreads();
}

// Forward transform, axes 3 and 2, of the work volume (axis 1 done, L x N x N values) onto the
// support; emit(c1, c2, c3, value) receives each of the L^3 outputs once, from the thread that owns
// the compact pencil (c1, c3) -- the same thread that reads it in pinv_23.
template <typename T, int N, int L, typename Emit>
__device__ __forceinline__ void pfwd_32(cplx<T>* B, Emit emit) {
  using S = Sup<N, L>;
  for (int p = threadIdx.x; p < L * N; p += blockDim.x) {
    const int c1 = p / N, i2 = p % N;
    cplx<T> v[N];
#pragma unroll
    for (int i3 = 0; i3 < N; ++i3) v[i3] = B[S::bidx(c1, i2, i3)];
    Codelet<T, N, -1>::run(v);
#pragma unroll
    for (int c3 = 0; c3 < L; ++c3) B[S::bidx(c1, i2, c3)] = v[S::box(c3)];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < L * L; p += blockDim.x) {
    const int c1 = p / L, c3 = p % L;
    cplx<T> v[N];
#pragma unroll
    for (int i2 = 0; i2 < N; ++i2) v[i2] = B[S::bidx(c1, i2, c3)];
    Codelet<T, N, -1>::run(v);
#pragma unroll
    for (int c2 = 0; c2 < L; ++c2) emit(c1, c2, c3, v[S::box(c2)]);
  }
  __syncthreads();
}

// p_d = Delta_d + G_d at compact index (c1, c2, c3)
template <typename T, int N, int L>
__device__ __forceinline__ T pcomp_c(const PComp<T>& q, int c1, int c2, int c3) {
  using S = Sup<N, L>;
  return q.c0 + (T)S::mil(c1) * q.b1 + (T)S::mil(c2) * q.b2 + (T)S::mil(c3) * q.b3;
}

template <int N, int L> __device__ __forceinline__ int gidx_c(int c1, int c2, int c3) {
  using S = Sup<N, L>;
  return (S::box(c1) * N + S::box(c2)) * N + S::box(c3);
}

// Fused pair chains, pruned (same work, grid and accumulators as k_pair_chain):
//   A  = FT[conj(bra_q) ket_j]                                          on the support
//   for d: b = FT^{-1}[U^pp_d A];  acc += f Z(q)_d b;  w_d += f ket_q b   (2bx1, 3a4, 3a3's w_j)
//          F = conj(bra_q) Y(j)_d - tw3b5 ket_j h3b(q)_d + tw3b6 n b;  C += -U^pp_d FT[F]
//   for d: b = FT^{-1}[U^ap_d A];  C += -U^ap_d FT[tw3b6 n b]             (3b6, antiparallel)
//   acc += f ket_q FT^{-1}[C - tw2ax V A]                                 (3b3, 2bx2, 3b5, 3b6, 2ax)
// (Algs. 2, 5, 6, 9, 11, 12 and the 2bx terms of Sec. 2.6.3.)
//
// Mirrored two-sided launches (P.mirror; Eq. BITCSCFconj).  The left pair density of (output q,
// partner j) is conj(phi_j^* chi_q) -- the complex conjugate of the right pair density of (output j,
// partner q) -- and the left side's kernel momentum is -(k_j - k_q + G), so on a support symmetric
// under G -> -G its compact spectrum is A_L(c) = conj(A_R(refl c)).  With u~ real and even,
// U_d(-p) = conj(U_d(p)), so FT^{-1}[U^ap_d A_L] = conj(FT^{-1}[U^ap_d A_R]); the left density is
// conj of the right one, so the antiparallel 3b6 spectrum is C_ap,L(c) = conj(C_ap,R(refl c)) too.
// mirror = 1 (right launch): a CTA whose output j is itself a partner (band < no) stores both
// reflections for the left pair (q, j), the antiparallel one summed over d as it is emitted;
// mirror = 2 (left launch, after it): such a pair loads them as its A and initial C and skips its
// own pair-density transform and antiparallel loop (7 of its 14 transforms).  Left outputs whose
// right counterpart was skipped for a zero occupation compute their own.  The parallel-spin loop
// and the final transform stay per side: their partner fields (Y, Z, h3b, V) have no such
// relation.  Built for FP64, whose chains are bound by the FP64 pipe; in FP32 the parallel-spin
// passes' loads dominate and the mirror code is compiled out.
template <typename T, int N, int L>
__global__ void __launch_bounds__(PrCfg<T, N>::threads, 1) k_pair_chain_pr(Params<T> P) {
  using G = Geo<N>;
  using S = Sup<N, L>;
  using SM = PrSmem<T, N, L, 2, 3>;
  constexpr int CH = 1;   // elements per load chunk of the pointwise pass (1 measured fastest in FP32)
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ T red[32];
  const SideArgs<T>& SD = P.side[P.side0 + blockIdx.y];
  const int jitem = blockIdx.x / P.sc, chunk = blockIdx.x % P.sc;
  const int jo = P.sym ? P.irr[jitem / P.nb] * P.nb + jitem % P.nb : jitem, j = P.j0 + jo, kj = j / P.nb;
  const int M = P.Nk * P.no, nj = P.nj_out;
  // mirrored launches (FP64 only: the FP32 kernel is bound by the loads of its parallel-spin
  // passes, which both sides keep, and gains nothing from them): output j as a partner index; write
  // (right) or read (left) the reflections
  constexpr bool MIR = sizeof(T) == 8;
  const int jocc = kj * P.no + j % P.nb;
  const bool mw = MIR && P.mirror == 1 && j % P.nb < P.no;
  // (the right CTA of output q skipped its pair with j when f_j, in the compute precision, was 0)
  const bool mr = MIR && P.mirror == 2 && j % P.nb < P.no && (T)(P.occ[j] / P.Nk) != T(0);
  const int qi_begin = (int)((long long)chunk * M / P.sc), qi_end = (int)((long long)(chunk + 1) * M / P.sc);
  cplx<T>* B = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* A;
  if constexpr (SM::spec) {
    A = B + S::bvol;
  } else {
    const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    A = P.scratch + cta * 2 * (size_t)S::cvol;
  }
  cplx<T>* C = A + S::cvol;
  T* tU = SM::tab ? reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(smraw) + SM::bB + 2 * SM::bC) : nullptr;
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
  for (int r = threadIdx.x; r < (int)NN; r += blockDim.x) {
    acc[r] = cplx<T>{0, 0};
    for (int d = 0; d < 3; ++d) w[d * NN + r] = cplx<T>{0, 0};
  }
  int staged = -1;   // Delta whose kernel tables are in shared memory
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
        // the previous pair's last reads of the tables ended before its closing barrier
        for (int c = threadIdx.x; c < S::cvol; c += blockDim.x) {
          const int g = gidx_c<N, L>(c / (L * L), (c / L) % L, c % L);
          tU[c] = Upp[g];
          tU[S::cvol + c] = Uap[g];
          tU[2 * S::cvol + c] = Vt[g];
        }
        staged = did;   // first read after the barriers of the forward transform below
      }
    }
    auto tab = [&](int which, int c1, int c2, int c3) -> T {
      if constexpr (SM::tab) {
        return tU[which * S::cvol + S::cidx(c1, c2, c3)];
      } else {
        const T* t = which == 0 ? Upp : (which == 1 ? Uap : Vt);
        return t[gidx_c<N, L>(c1, c2, c3)];
      }
    };
    const cplx<T>* braq = SD.bra + (size_t)q * NN;
    const cplx<T>* ketq = SD.ket + (size_t)q * NN;
    const cplx<T>* Zq = SD.Z + ((size_t)(kq * P.no + mu) * 3) * NN;
    const cplx<T>* h3bq = SD.h3b + ((size_t)(kq * P.no + mu) * 3) * NN;
    // the reflections of this pair: [A][C_ap] of the left pair (q, j) (write) or of this one (read)
    cplx<T>* MA = (mw || mr) ? P.mir + ((size_t)(mw ? qi : jocc) * M + (mw ? jocc : qi)) * 2 * S::cvol : nullptr;
    if (mr) {
      for (int c = threadIdx.x; c < S::cvol; c += blockDim.x) {
        A[c] = MA[c];
        C[c] = need_ap ? MA[S::cvol + c] : cplx<T>{0, 0};
      }
      __syncthreads();
    } else {
      // A = FT[conj(bra_q) ket_j] on the support
      pass_axis1<T, N, L, false>(
          B, [&](int a, int b, int c) { const int g = G::gidx(a, b, c); return mulc(ldg(ketj + g), ldg(braq + g)); },
          [&](int, int, cplx<T>(&)[N]) {}, true);
      pfwd_32<T, N, L>(B, [&](int c1, int c2, int c3, cplx<T> v) {
        const cplx<T> a = P.invN * v;
        A[S::cidx(c1, c2, c3)] = a;
        if (mw) MA[S::cidx(S::refl(c1), S::refl(c2), S::refl(c3))] = conjg(a);
      });
    }
    if (P.div && kq == kj && t3b6 != T(0)) {
      // O_qj = A(0) and X_s = sum_{G != 0} u~_s(G) A(G) n~(-G) for the 3b6 corrections
      for (int s = 0; s < 2; ++s) {
        T xr = 0, xi = 0;
        for (int c = threadIdx.x; c < S::cvol; c += blockDim.x) {
          const int c1 = c / (L * L), c2 = (c / L) % L, c3 = c % L;
          const int a = S::box(c1), b = S::box(c2), e = S::box(c3);
          const int gn = G::gidx((N - a) % N, (N - b) % N, (N - e) % N);
          const cplx<T> t = P.hartUs[(size_t)s * NN + G::gidx(a, b, e)] * (A[c] * SD.nt[gn]);
          xr += t.x;
          xi += t.y;
        }
        const T sr = block_sum<T>(xr, red);
        const T si = block_sum<T>(xi, red);
        if (threadIdx.x == 0) {
          double* cs = SD.cs + ((size_t)jo * P.no + mu) * 6;
          cs[2 + 2 * s] = sr;
          cs[3 + 2 * s] = si;
          if (s == 0) { cs[0] = A[0].x; cs[1] = A[0].y; }
        }
      }
      __syncthreads();
    }
    // spin channels: parallel then antiparallel (a reading mirrored CTA has the antiparallel
    // spectrum in C already; a writing one also sums it, reflected, into the left pair's slot)
    for (int sp = 0; sp < 2; ++sp) {
      if (sp == 0 && !(need_pp || need_F)) continue;
      if (sp == 1 && (!need_ap || mr)) continue;
      for (int d = 0; d < 3; ++d) {
        const bool first_C = sp == 0 && d == 0 && !mr;
        const PComp<T> qd = pcomp_setup<T>(P, dl, d);
        // b = FT^{-1}[U_d A]
        pinv_23<T, N, L>(B, [&](int c1, int c2, int c3) {
          return mul_si<T, 1>((pcomp_c<T, N, L>(qd, c1, c2, c3) * tab(sp, c1, c2, c3)) * A[S::cidx(c1, c2, c3)]);
        });
        const bool fwd = sp == 1 || need_F;
        pass_axis1<T, N, L, true>(
            B, [&](int, int, int) { return cplx<T>{0, 0}; },
            [&](int i2, int i3, cplx<T>(&v)[N]) {
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
        // C += -U_d FT[F] = -i p_d u FT[F]
        pfwd_32<T, N, L>(B, [&](int c1, int c2, int c3, cplx<T> v) {
          const T k = pcomp_c<T, N, L>(qd, c1, c2, c3) * tab(sp, c1, c2, c3) * P.invN;
          const cplx<T> t = mul_si<T, -1>(k * v);
          const int s = S::cidx(c1, c2, c3);
          C[s] = first_C ? t : C[s] + t;
          if (sp == 1 && mw) {
            // the thread that emits an index emits it for every d
            cplx<T>* mc = MA + S::cvol + S::cidx(S::refl(c1), S::refl(c2), S::refl(c3));
            *mc = d == 0 ? conjg(t) : *mc + conjg(t);
          }
        });
      }
    }
    const bool has_C = need_F || need_ap;
    if (has_C || t2ax != T(0)) {
      pinv_23<T, N, L>(B, [&](int c1, int c2, int c3) {
        const int s = S::cidx(c1, c2, c3);
        cplx<T> v = has_C ? C[s] : cplx<T>{0, 0};
        if (t2ax != T(0)) v = v - (t2ax * tab(2, c1, c2, c3)) * A[s];
        return v;
      });
      pass_axis1<T, N, L, true>(
          B, [&](int, int, int) { return cplx<T>{0, 0}; },
          [&](int i2, int i3, cplx<T>(&v)[N]) {
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
}

// Pass 2 for 3b4 (Alg. 10), pruned: acc += tw3b4 f ket_q FT^{-1}[-U^pp . FT[-conj(bra_q) w_j]]
// (same grid and accumulators as k_pair_3b4).
template <typename T, int N, int L>
__global__ void __launch_bounds__(PrCfg<T, N>::threads, 1) k_pair_3b4_pr(Params<T> P) {
  using G = Geo<N>;
  using S = Sup<N, L>;
  using SM = PrSmem<T, N, L, 1, 1>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const SideArgs<T>& SD = P.side[blockIdx.y];
  const int jitem = blockIdx.x / P.sc, chunk = blockIdx.x % P.sc;
  const int jo = P.sym ? P.irr[jitem / P.nb] * P.nb + jitem % P.nb : jitem, j = P.j0 + jo, kj = j / P.nb;
  const int M = P.Nk * P.no, nj = P.nj_out;
  const int qi_begin = (int)((long long)chunk * M / P.sc), qi_end = (int)((long long)(chunk + 1) * M / P.sc);
  cplx<T>* B = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* A;
  if constexpr (SM::spec) {
    A = B + S::bvol;
  } else {
    const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    A = P.scratch + cta * (size_t)S::cvol;
  }
  T* tU = SM::tab ? reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(smraw) + SM::bB + SM::bC) : nullptr;
  const size_t NN = G::nn;
  cplx<T>* acc = SD.acc + ((size_t)chunk * nj + jo) * NN;
  const cplx<T>* w = SD.w + (size_t)jo * 3 * NN;
  const T t3b4 = P.tw[T3B4];
  if (t3b4 == T(0)) return;
  if (chunk > 0) {
    for (int r = threadIdx.x; r < (int)NN; r += blockDim.x) acc[r] = cplx<T>{0, 0};
    __syncthreads();
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
        for (int c = threadIdx.x; c < S::cvol; c += blockDim.x)
          tU[c] = Upp[gidx_c<N, L>(c / (L * L), (c / L) % L, c % L)];
        staged = did;
      }
    }
    auto tab = [&](int c1, int c2, int c3) -> T {
      if constexpr (SM::tab) return tU[S::cidx(c1, c2, c3)];
      else return Upp[gidx_c<N, L>(c1, c2, c3)];
    };
    const cplx<T>* braq = SD.bra + (size_t)q * NN;
    const cplx<T>* ketq = SD.ket + (size_t)q * NN;
    for (int d = 0; d < 3; ++d) {
      const PComp<T> qd = pcomp_setup<T>(P, dl, d);
      pass_axis1<T, N, L, false>(
          B, [&](int a, int b, int c) { const int g = G::gidx(a, b, c); return mulc(ldg(w + d * NN + g), ldg(braq + g)); },
          [&](int, int, cplx<T>(&)[N]) {}, true);
      // -U_d FT[-conj(bra_q) w_d] = +i p_d u FT[conj(bra_q) w_d]
      pfwd_32<T, N, L>(B, [&](int c1, int c2, int c3, cplx<T> v) {
        const T k = pcomp_c<T, N, L>(qd, c1, c2, c3) * tab(c1, c2, c3) * P.invN;
        const cplx<T> t = mul_si<T, 1>(k * v);
        const int s = S::cidx(c1, c2, c3);
        A[s] = d == 0 ? t : A[s] + t;
      });
    }
    const T fw = t3b4 * f;
    pinv_23<T, N, L>(B, [&](int c1, int c2, int c3) { return A[S::cidx(c1, c2, c3)]; });
    pass_axis1<T, N, L, true>(
        B, [&](int, int, int) { return cplx<T>{0, 0}; },
        [&](int i2, int i3, cplx<T>(&v)[N]) {
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
}

// Occupied-pair stage, pruned (same grid, outputs and per-CTA h6 part as k_occ_pairs; Algs. 4, 6, 8,
// 11 and the 3a2 corrections of Eqs. divcor_3a2_first/second in the general-overlap form):
//   A1 = FT[conj(bra_q2) ket_q1], A2 = FT[conj(bra_q1) ket_q2]                      on the support
//   B1 = P^s_d(q2, q1) = FT^{-1}[U^s_d(k1 - k2 + G) A1]   (real space, in shared memory)
//   B2 = P^s_d(q1, q2) = FT^{-1}[U^s_d(k2 - k1 + G) A2]   (its last pass fused with the products)
//   h6 += w f1 f2 B1 . B2;  h3a4(q2)_d += f1 B2 ket_q1;  h3b(q2)_d += f1 B1 conj(bra_q1)   (s = pp)
// Shared memory: B1 as a real-space volume [N][N][N|1] (rows c1 < L serve as its inverse work
// area), then the work volume of B2 [L][N][N|1] when it fits (FP32), else in the CTA's scratch
// slice.  The compact spectra A1, A2 and the 3a2 spectrum F_ab live in the CTA's scratch slice
// (slots 0, 1, 2; slot 4 is the h6 part that k_reduce_a4 sums, as for k_occ_pairs).
template <typename T, int N, int L> struct OccSmem {
  using S = Sup<N, L>;
  static constexpr size_t bR = (size_t)Geo<N>::vol * sizeof(cplx<T>);
  static constexpr size_t bW = (size_t)S::bvol * sizeof(cplx<T>);
  static constexpr size_t lim = (size_t)kSmemLimit - 1024;
  static constexpr bool w_smem = bR + bW <= lim;
  static constexpr size_t bytes = bR + (w_smem ? bW : 0);
};

template <typename T, int N, int L>
__global__ void __launch_bounds__(PrCfg<T, N>::threads, 1) k_occ_pairs_pr(Params<T> P) {
  using G = Geo<N>;
  using S = Sup<N, L>;
  using SM = OccSmem<T, N, L>;
  static_assert(S::bvol <= G::vol && S::cvol <= G::vol, "slots hold a full volume");
  constexpr int NS = 6;
  constexpr int CH = sizeof(T) == 4 ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sO[2][2];
  __shared__ double sF0[2];
  const SideArgs<T>& SD = P.side[blockIdx.y];
  const int M = P.Nk * P.no;
  const int item = blockIdx.x / P.so, chunk = blockIdx.x % P.so;
  const int i2 = P.sym ? P.irr[item / P.no] * P.no + item % P.no : P.i2_0 + item;
  const int k2 = i2 / P.no, mu2 = i2 % P.no;
  const int q2 = k2 * P.nb + mu2;
  const int i1_begin = (int)((long long)chunk * M / P.so), i1_end = (int)((long long)(chunk + 1) * M / P.so);
  const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
  cplx<T>* slice = P.scratch + cta * NS * (size_t)G::vol;
  cplx<T>* R1 = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* W2 = SM::w_smem ? R1 + G::vol : slice + 3 * (size_t)G::vol;
  cplx<T>* A1 = slice;
  cplx<T>* A2 = slice + G::vol;
  cplx<T>* FAB = slice + 2 * (size_t)G::vol;
  cplx<T>* H6 = slice + 4 * (size_t)G::vol;
  const size_t NN = G::nn;
  const T f2 = (T)(P.occ[q2] / P.Nk);
  cplx<T>* h3a4 = SD.h3a4 + ((size_t)chunk * P.nq2 + (i2 - P.i2_0)) * 3 * NN;
  cplx<T>* h3b = SD.h3b + ((size_t)chunk * P.nq2 + (i2 - P.i2_0)) * 3 * NN;
  const cplx<T>* bra2 = SD.bra + (size_t)q2 * NN;
  const cplx<T>* ket2 = SD.ket + (size_t)q2 * NN;
  for (int r = threadIdx.x; r < S::cvol; r += blockDim.x) FAB[r] = cplx<T>{0, 0};
  for (int r = threadIdx.x; r < (int)NN; r += blockDim.x) {
    H6[r] = cplx<T>{0, 0};
    for (int d = 0; d < 3; ++d) {
      h3a4[d * NN + r] = cplx<T>{0, 0};
      h3b[d * NN + r] = cplx<T>{0, 0};
    }
  }
  if (threadIdx.x == 0) { sF0[0] = 0.0; sF0[1] = 0.0; }
  __syncthreads();
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
    // A1 = FT[conj(bra_q2) ket_q1], A2 = FT[conj(bra_q1) ket_q2] (work area: the rows of R1)
    pass_axis1<T, N, L, false>(
        R1, [&](int a, int b, int c) { const int g = G::gidx(a, b, c); return mulc(ldg(ket1 + g), ldg(bra2 + g)); },
        [&](int, int, cplx<T>(&)[N]) {}, true);
    pfwd_32<T, N, L>(R1, [&](int c1, int c2, int c3, cplx<T> v) { A1[S::cidx(c1, c2, c3)] = P.invN * v; });
    pass_axis1<T, N, L, false>(
        R1, [&](int a, int b, int c) { const int g = G::gidx(a, b, c); return mulc(ldg(ket2 + g), ldg(bra1 + g)); },
        [&](int, int, cplx<T>(&)[N]) {}, true);
    pfwd_32<T, N, L>(R1, [&](int c1, int c2, int c3, cplx<T> v) { A2[S::cidx(c1, c2, c3)] = P.invN * v; });
    // 3a2 correction pieces for pairs at the same k (Eqs. divcor_3a2_*_density_matrix_mixing)
    if (P.div && k1 == k2) {
      if (threadIdx.x == 0) {
        const cplx<T> o21 = A1[0], o12 = A2[0];   // <bra_q2|ket_q1>, <bra_q1|ket_q2>
        sO[0][0] = o21.x; sO[0][1] = o21.y; sO[1][0] = o12.x; sO[1][1] = o12.y;
        const double fq = P.occ[q1];
        sF0[0] += fq * ((double)o21.x * o12.x - (double)o21.y * o12.y);
        sF0[1] += fq * ((double)o21.x * o12.y + (double)o21.y * o12.x);
      }
      __syncthreads();
      const cplx<T> o21 = {(T)sO[0][0], (T)sO[0][1]}, o12 = {(T)sO[1][0], (T)sO[1][1]};
      const T fq = (T)P.occ[q1];
      for (int r = threadIdx.x; r < S::cvol; r += blockDim.x) FAB[r] = FAB[r] + fq * (o12 * A1[r] + o21 * A2[r]);
      __syncthreads();
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
        // B1 = P^s_d(q2, q1), real space in R1
        pinv_23<T, N, L>(R1, [&](int c1, int c2, int c3) {
          const int s = S::cidx(c1, c2, c3);
          return mul_si<T, 1>((pcomp_c<T, N, L>(q21, c1, c2, c3) * U21[gidx_c<N, L>(c1, c2, c3)]) * A1[s]);
        });
        pass_axis1<T, N, L, true>(
            R1, [&](int, int, int) { return cplx<T>{0, 0}; },
            [&](int a2, int a3, cplx<T>(&v)[N]) {
#pragma unroll
              for (int i = 0; i < N; ++i) R1[G::sidx(i, a2, a3)] = v[i];
            },
            false);
        // B2 = P^s_d(q1, q2); its axis-1 pass forms the products with B1
        pinv_23<T, N, L>(W2, [&](int c1, int c2, int c3) {
          const int s = S::cidx(c1, c2, c3);
          return mul_si<T, 1>((pcomp_c<T, N, L>(q12, c1, c2, c3) * U12[gidx_c<N, L>(c1, c2, c3)]) * A2[s]);
        });
        pass_axis1<T, N, L, true>(
            W2, [&](int, int, int) { return cplx<T>{0, 0}; },
            [&](int a2, int a3, cplx<T>(&v)[N]) {
#pragma unroll
              for (int c0 = 0; c0 < N; c0 += CH) {
                cplx<T> lb1[CH], lk[CH], lr[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                  if (c0 + u >= N) continue;
                  const int g = G::gidx(c0 + u, a2, a3);
                  lb1[u] = R1[G::sidx(c0 + u, a2, a3)];
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
                  red_add_v(&H6[g], w12 * (lb1[u] * b2));
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
    pinv_23<T, N, L>(W2, [&](int c1, int c2, int c3) {
      const int g = gidx_c<N, L>(c1, c2, c3);
      const T u = a0 * P.hartUs[g] + a1 * P.hartUs[NN + g];
      return u * FAB[S::cidx(c1, c2, c3)];
    });
    pass_axis1<T, N, L, true>(
        W2, [&](int, int, int) { return cplx<T>{0, 0}; },
        [&](int a2, int a3, cplx<T>(&v)[N]) {
#pragma unroll
          for (int i = 0; i < N; ++i) red_add_v(&H6[G::gidx(i, a2, a3)], pref * (v[i] + cF0));
        },
        false);
  }
}

}  // namespace tc
