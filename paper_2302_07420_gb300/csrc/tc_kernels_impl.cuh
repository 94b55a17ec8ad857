// Kernels of the TC operator (templated on precision T and cubic box size N).
//
// Stage map (Sec. 2.6 of arXiv:2302.07420):
//   k_orbitals     sphere -> box gather and inverse FFT of phi, chi, grad phi, grad chi
//   k_density      n and the 2bh2 vector density m (per side)
//   k_spec_fwd     FT of a global field or of a product of two fields
//   k_hartree_inv  Hartree-type convolutions: v_H (Alg. 1), h1 (Algs. 3, 5, 7, 9),
//                  v_b2 (2bh2), the 3b1 / 3b2 tails and the 3b6 scf2 field
//   k_occ_pairs    occupied-pair stage (Algs. 4, 6, 8, 11): h6, h3 (3a4), h3 (3b), and
//                  the 3a2 corrections (Eqs. divcor_3a2_first/second, general overlaps)
//   k_reduce_a4    sum of the per-CTA h6 parts and h5 of Alg. 8
//   k_vloc         local potential of the Hartree-type terms
//   k_pair_chain   per output orbital j, all partners q: 2ax (Alg. 2), 2bx1, 2bx2, 3a3's w_j,
//                  3a4 (Alg. 6), 3b3 (Alg. 9), 3b5 (Alg. 11), 3b6 (Alg. 12) fused into one
//                  FFT chain per (j, q) pair
//   k_pair_3b4     second pass for 3b4 (Alg. 10), which needs the complete w_j
//   k_finalize     local terms, 3b6 corrections (Eqs. 3b6_div_scf1/2/3), FFT, box -> sphere
#pragma once
#include "tc_kernels.cuh"

namespace tc {

// Threads per CTA: one pencil per thread up to 384 pencils, two per thread up to
// 24^3, and 256 threads (several pencils each, up to 255 registers) above.
template <int N> struct Cfg {
  static constexpr int threads = (N * N <= 384) ? ((N * N + 31) / 32) * 32
                                                : (N <= 24 ? ((N * N / 2 + 31) / 32) * 32 : 256);
};

// Whether one n^3 work volume (padded layout) fits in a CTA's shared memory.
template <typename T, int N> struct Fit {
  static constexpr bool one = (size_t)Geo<N>::vol * sizeof(cplx<T>) + 1024 <= (size_t)kSmemLimit;
};

// Work volume of a single-volume kernel: shared memory when it fits, else this
// CTA's volume in the global scratch gwork (one volume per CTA of the launch).
template <typename T, int N> __device__ __forceinline__ cplx<T>* work_vol(unsigned char* smraw, cplx<T>* gwork) {
  if constexpr (Fit<T, N>::one) {
    return reinterpret_cast<cplx<T>*>(smraw);
  } else {
    const size_t b = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    return gwork + b * (size_t)Geo<N>::vol;
  }
}

template <typename T, int N> __device__ __forceinline__ cplx<T>* vol_slot(const Params<T>& P, cplx<T>* smem, int slot,
                                                                           int nslots, bool force_global = false) {
  if (!force_global && slot < P.nsmem) return smem + (size_t)slot * Geo<N>::vol;
  const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
  return P.scratch + (cta * nslots + slot) * (size_t)Geo<N>::vol;
}

// p = Delta + G for the FFT index (i1, i2, i3)
template <typename T, int N> __device__ __forceinline__ void pvec(const Params<T>& P, const T* dl, int i1, int i2, int i3,
                                                                   T* p) {
  const T r1 = (T)(i1 <= (N - 1) / 2 ? i1 : i1 - N);
  const T r2 = (T)(i2 <= (N - 1) / 2 ? i2 : i2 - N);
  const T r3 = (T)(i3 <= (N - 1) / 2 ? i3 : i3 - N);
#pragma unroll
  for (int d = 0; d < 3; ++d) p[d] = dl[d] + r1 * P.Bm[0][d] + r2 * P.Bm[1][d] + r3 * P.Bm[2][d];
}

// One Cartesian component d of p = Delta + G, with the per-component constants
// taken out of the element loop: p_d = c0 + r1 b1 + r2 b2 + r3 b3 (r_i the
// Miller integers of the FFT index).  Selecting the constants by d with
// constant indices keeps every array access static (no local-memory copies).
template <typename T> struct PComp {
  T c0, b1, b2, b3;
};

template <typename T>
__device__ __forceinline__ PComp<T> pcomp_setup(const Params<T>& P, const T* dl, int d) {
  PComp<T> q;
  q.c0 = dl ? dl[d] : T(0);
  q.b1 = d == 0 ? P.Bm[0][0] : (d == 1 ? P.Bm[0][1] : P.Bm[0][2]);
  q.b2 = d == 0 ? P.Bm[1][0] : (d == 1 ? P.Bm[1][1] : P.Bm[1][2]);
  q.b3 = d == 0 ? P.Bm[2][0] : (d == 1 ? P.Bm[2][1] : P.Bm[2][2]);
  return q;
}

template <typename T, int N> __device__ __forceinline__ T pcomp(const PComp<T>& q, int i1, int i2, int i3) {
  const T r1 = (T)(i1 <= (N - 1) / 2 ? i1 : i1 - N);
  const T r2 = (T)(i2 <= (N - 1) / 2 ? i2 : i2 - N);
  const T r3 = (T)(i3 <= (N - 1) / 2 ? i3 : i3 - N);
  return q.c0 + r1 * q.b1 + r2 * q.b2 + r3 * q.b3;
}

template <typename T> __device__ __forceinline__ cplx<T> ld(const cplx<T>* p, size_t i) { return p[i]; }

// *p += v performed in L2 (a reduction without a return value): the SM does not wait
// for the old value.  Each accumulator element has one owning CTA, and one thread of
// it adds to the element at a time, so the sums keep their order.
template <typename T> __device__ __forceinline__ void red_add(cplx<T>* p, cplx<T> v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

template <typename T> __device__ __forceinline__ T block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T s = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) s += red[i];
  return s;   // valid in thread 0
}

// ---------------------------------------------------------------------------
// Standalone batched 3D FFT (testing hook).
template <typename T, int N, int S>
__global__ void __launch_bounds__(Cfg<N>::threads) k_fft3d(cplx<T>* data, cplx<T>* gwork) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* V = work_vol<T, N>(smraw, gwork);
  cplx<T>* d = data + (size_t)blockIdx.x * G::nn;
  auto ld = [&](int a, int b, int c) { return d[G::gidx(a, b, c)]; };
  auto st = [&](int a, int b, int c, cplx<T> v) { d[G::gidx(a, b, c)] = v; };
  if (S < 0) fwd3d<T, N>(V, ld, st);
  else inv3d<T, N>(V, ld, st);
}

// ---------------------------------------------------------------------------
// Orbitals to real space: grid (orbitals, 4 components, 2 sets).  Component 0 is
// psi = FT^{-1}[c], components 1..3 are d_d psi = FT^{-1}[i (k+G)_d c].
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::threads)
    k_orbitals(const double2* __restrict__ cphi, const double2* __restrict__ cchi, const double2* __restrict__ bphi,
               const double2* __restrict__ bchi, int nj_mesh, const int* __restrict__ box_index,
               const double* __restrict__ kpg, int npw_max, int nb, cplx<T>* phi, cplx<T>* chi, cplx<T>* gphi,
               cplx<T>* gchi, cplx<T>* gwork) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* V = work_vol<T, N>(smraw, gwork);
  const int j = blockIdx.x, comp = blockIdx.y, set = blockIdx.z;
  const int k = j / nb;
  // orbitals j >= nj_mesh are those of band points (their own input arrays)
  const double2* c = j < nj_mesh ? (set == 0 ? cphi : cchi) + (size_t)j * npw_max
                                 : (set == 0 ? bphi : bchi) + (size_t)(j - nj_mesh) * npw_max;
  for (int i = threadIdx.x; i < G::vol; i += blockDim.x) V[i] = cplx<T>{0, 0};
  __syncthreads();
  for (int g = threadIdx.x; g < npw_max; g += blockDim.x) {
    const int bi = box_index[(size_t)k * npw_max + g];
    if (bi < 0) continue;
    double2 v = c[g];
    if (comp > 0) {   // multiply by i (k+G)_d
      const double q = kpg[((size_t)k * npw_max + g) * 3 + (comp - 1)];
      v = make_double2(-q * v.y, q * v.x);
    }
    const int i1 = bi / (N * N), i2 = (bi / N) % N, i3 = bi % N;
    V[G::sidx(i1, i2, i3)] = cplx<T>{(T)v.x, (T)v.y};
  }
  __syncthreads();
  cplx<T>* dst = comp == 0 ? (set == 0 ? phi : chi) + (size_t)j * G::nn
                           : (set == 0 ? gphi : gchi) + ((size_t)j * 3 + (comp - 1)) * G::nn;
  inv3d<T, N>(V, [&](int a, int b, int cc) { return V[G::sidx(a, b, cc)]; },
              [&](int a, int b, int cc, cplx<T> v) { dst[G::gidx(a, b, cc)] = v; });
}

// BF16 storage (TC_BF16_STORE): every value of a[0 .. n) rounded to the nearest BF16 (ties to even),
// kept in its FP32 word.
template <typename T> __global__ void k_round_bf16(cplx<T>* a, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cplx<T> v = a[i];
    v.x = (T)__bfloat162float(__float2bfloat16_rn((float)v.x));
    v.y = (T)__bfloat162float(__float2bfloat16_rn((float)v.y));
    a[i] = v;
  }
}

// ---------------------------------------------------------------------------
// Densities of both sides: n = (1/Nk) sum_{k, mu < no} f conj(bra) ket, m likewise with grad ket.
template <typename T, int N> __global__ void k_density(Params<T> P) {
  const SideArgs<T>& S = P.side[blockIdx.y];
  const int NN = N * N * N;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < NN; r += gridDim.x * blockDim.x) {
    cplx<T> n = {0, 0}, m0 = {0, 0}, m1 = {0, 0}, m2 = {0, 0};
    for (int k = 0; k < P.Nk; ++k)
      for (int mu = 0; mu < P.no; ++mu) {
        const int q = k * P.nb + mu;
        const T f = (T)(P.occ[q] / P.Nk);
        if (f == T(0)) continue;
        const cplx<T> b = conjg(S.bra[(size_t)q * NN + r]);
        n = n + f * (b * S.ket[(size_t)q * NN + r]);
        m0 = m0 + f * (b * S.gket[((size_t)q * 3 + 0) * NN + r]);
        m1 = m1 + f * (b * S.gket[((size_t)q * 3 + 1) * NN + r]);
        m2 = m2 + f * (b * S.gket[((size_t)q * 3 + 2) * NN + r]);
      }
    S.n[r] = n;
    S.m[r] = m0;
    S.m[NN + r] = m1;
    S.m[2 * NN + r] = m2;
  }
}

// ---------------------------------------------------------------------------
// dst[c] = FT[a[c] * b[c]] (1/N normalised) for c = blockIdx.x; b may be null (factor 1).
// blockIdx.y = side; a and b are given per side by offsets into the side's fields.
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::threads)
    k_spec_fwd(Params<T> P, int which) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* V = work_vol<T, N>(smraw, P.scratch);
  const SideArgs<T>& S = P.side[blockIdx.y];
  const int c = blockIdx.x;
  const cplx<T>* a;
  const cplx<T>* b = nullptr;
  cplx<T>* dst;
  if (which == 0) {          // n~
    a = S.n; dst = S.nt;
  } else if (which == 1) {   // m~_c
    a = S.m + (size_t)c * G::nn; dst = S.mt + (size_t)c * G::nn;
  } else if (which == 2) {   // FT[h1_c n]  (Alg. 7)
    a = S.h1 + (size_t)c * G::nn; b = S.n; dst = S.spec + (size_t)c * G::nn;
  } else {                   // FT[h5_c]    (Alg. 8)
    a = S.h5 + (size_t)c * G::nn; dst = S.spec + (size_t)c * G::nn;
  }
  fwd3d<T, N>(
      V,
      [&](int i, int j, int k) {
        cplx<T> v = a[G::gidx(i, j, k)];
        return b ? v * b[G::gidx(i, j, k)] : v;
      },
      [&](int i, int j, int k, cplx<T> v) { dst[G::gidx(i, j, k)] = P.invN * v; });
}

// Hartree-type convolutions (Delta = 0, G = 0 dropped), blockIdx.y = side.
//   kind 0: v_H = FT^{-1}[Vh n~]
//   kind 1: h1_c = FT^{-1}[i G_c u~h n~]                 (c = blockIdx.x)
//   kind 2: v_b2 = FT^{-1}[-i G u~h . m~]
//   kind 3: t3b1 = FT^{-1}[-i G u~h . FT[h1 n]]         (spectrum in S.spec)
//   kind 4: t3b2 = FT^{-1}[-i G u~h . FT[h5]]           (spectrum in S.spec)
//   kind 5: vu_s = FT^{-1}[u~_s n~] (no 1/Omega)        (s = blockIdx.x)
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::threads)
    k_hartree_inv(Params<T> P, int kind) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* V = work_vol<T, N>(smraw, P.scratch);
  const SideArgs<T>& S = P.side[blockIdx.y];
  const int c = blockIdx.x;
  const T zero3[3] = {0, 0, 0};
  const PComp<T> qc = pcomp_setup<T>(P, nullptr, kind == 1 ? c : 0);
  cplx<T>* dst = kind == 0 ? S.vH : kind == 1 ? S.h1 + (size_t)c * G::nn : kind == 2 ? S.vb2 : kind == 3 ? S.t3b1
               : kind == 4 ? S.t3b2 : S.vu + (size_t)c * G::nn;
  inv3d<T, N>(
      V,
      [&](int i, int j, int k) {
        const int g = G::gidx(i, j, k);
        if (kind == 0) return P.hartV[(size_t)S.side * G::nn + g] * S.nt[g];
        if (kind == 5) return P.hartUs[(size_t)c * G::nn + g] * S.nt[g];
        const T u = P.hartU[g];
        if (kind == 1) {
          const cplx<T> t = (pcomp<T, N>(qc, i, j, k) * u) * S.nt[g];
          return mul_si<T, 1>(t);
        }
        T p[3];
        pvec<T, N>(P, zero3, i, j, k, p);
        const cplx<T>* src = (kind == 2) ? S.mt : S.spec;
        cplx<T> s = {0, 0};
#pragma unroll
        for (int d = 0; d < 3; ++d) s = s + (p[d] * u) * src[(size_t)d * G::nn + g];
        return mul_si<T, -1>(s);   // -i G u . src
      },
      [&](int i, int j, int k, cplx<T> v) { dst[G::gidx(i, j, k)] = v; });
}

// ---------------------------------------------------------------------------
// Occupied-pair stage.  Grid (Nk*no*so, 2 sides); CTA = occupied q2 and one of `so` chunks
// of the q1 range (chunk parts of h3a4 / h3b, summed by k_sum_parts).
//   P^s(a, b) = FT^{-1}[U^_s(k_b - k_a + G) FT[conj(bra_a) ket_b]],  U^_s = i p u~_s / Omega
//   h6 += f1 f2 / Nk^2 sum_s P^s(q2,q1) . P^s(q1,q2)             (Alg. 4; ap part over unordered pairs)
//   h3a4(q2) += f1/Nk P^pp(q1,q2) ket_q1                         (Alg. 6)
//   h3b(q2)  += f1/Nk P^pp(q2,q1) conj(bra_q1)                   (Algs. 8, 11)
// Slots: 0 B1, 1 B2, 2 A1, 3 A2 (shared or global), 4 h6 part, 5 F_ab (global).
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::threads, 1) k_occ_pairs(Params<T> P) {
  using G = Geo<N>;
  constexpr int NS = 6;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(smraw);
  __shared__ double sO[2][2];
  __shared__ double sF0[2];
  const SideArgs<T>& S = P.side[blockIdx.y];
  const int M = P.Nk * P.no;                                   // occupied states
  // with crystal symmetry only the q2 of irreducible k-points have CTAs (the rest are unfolded)
  const int item = blockIdx.x / P.so, chunk = blockIdx.x % P.so;
  const int i2 = P.sym ? P.irr[item / P.no] * P.no + item % P.no : P.i2_0 + item;
  const int k2 = i2 / P.no, mu2 = i2 % P.no;
  const int q2 = k2 * P.nb + mu2;
  const int i1_begin = (int)((long long)chunk * M / P.so), i1_end = (int)((long long)(chunk + 1) * M / P.so);
  cplx<T>* B1 = vol_slot<T, N>(P, sm, 0, NS);
  cplx<T>* B2 = vol_slot<T, N>(P, sm, 1, NS);
  cplx<T>* A1 = vol_slot<T, N>(P, sm, 2, NS);
  cplx<T>* A2 = vol_slot<T, N>(P, sm, 3, NS);
  cplx<T>* H6 = vol_slot<T, N>(P, sm, 4, NS, true);
  cplx<T>* FAB = vol_slot<T, N>(P, sm, 5, NS, true);
  const size_t NN = G::nn;
  const T f2 = (T)(P.occ[q2] / P.Nk);
  cplx<T>* h3a4 = S.h3a4 + ((size_t)chunk * P.nq2 + (i2 - P.i2_0)) * 3 * NN;
  cplx<T>* h3b = S.h3b + ((size_t)chunk * P.nq2 + (i2 - P.i2_0)) * 3 * NN;
  const cplx<T>* bra2 = S.bra + (size_t)q2 * NN;
  const cplx<T>* ket2 = S.ket + (size_t)q2 * NN;
  for (int r = threadIdx.x; r < G::vol; r += blockDim.x) FAB[r] = cplx<T>{0, 0};   // padded layout
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
    const int id12 = P.delta_id[k2 * P.kstride + k1];   // Delta = k2 - k1 -> for P(q1,q2)
    const int id21 = P.delta_id[k1 * P.kstride + k2];   // Delta = k1 - k2 -> for P(q2,q1)
    const T* d12 = P.delta + id12 * 3;
    const T* d21 = P.delta + id21 * 3;
    {
      const int q1 = k1 * P.nb + mu1;
      const T f1 = (T)(P.occ[q1] / P.Nk);
      if (f1 == T(0) || f2 == T(0)) continue;
      const cplx<T>* bra1 = S.bra + (size_t)q1 * NN;
      const cplx<T>* ket1 = S.ket + (size_t)q1 * NN;
      // A1 = FT[conj(bra_q2) ket_q1], A2 = FT[conj(bra_q1) ket_q2]
      fwd3d<T, N>(B1, [&](int i, int j, int k) { const int g = G::gidx(i, j, k); return mulc(ldg(ket1 + g), ldg(bra2 + g)); },
                  [&](int i, int j, int k, cplx<T> v) { A1[G::sidx(i, j, k)] = P.invN * v; });
      fwd3d<T, N>(B2, [&](int i, int j, int k) { const int g = G::gidx(i, j, k); return mulc(ldg(ket2 + g), ldg(bra1 + g)); },
                  [&](int i, int j, int k, cplx<T> v) { A2[G::sidx(i, j, k)] = P.invN * v; });
      __syncthreads();
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
        for (int r = threadIdx.x; r < G::vol; r += blockDim.x) FAB[r] = FAB[r] + fq * (o12 * A1[r] + o21 * A2[r]);
        __syncthreads();
      }
      // The antiparallel channel only feeds h6, and its contribution P^ap(q2,q1) . P^ap(q1,q2) is
      // symmetric in (q1, q2): each unordered pair is taken once, by the CTA for which q1 lies
      // in the next half of the cyclic order after q2, with weight 2 (1 on the diagonal).
      // (With symmetry the part of each irreducible q2 must hold all its pairs: no halving.)
      const int cyc = (i1 - i2 + M) % M;
      const bool ap_here = P.sym || cyc == 0 || 2 * cyc < M || (2 * cyc == M && i2 < i1);
      const T ap_w = (P.sym || cyc == 0) ? T(1) : T(2);
      for (int sp = 0; sp < 2; ++sp) {
        if (sp == 1 && (!ap_here || P.h3_only || P.no_ap)) continue;
        const T w12 = (sp == 1 ? ap_w : T(1)) * (f1 * f2);
        for (int d = 0; d < 3; ++d) {
          const PComp<T> q21 = pcomp_setup<T>(P, d21, d), q12 = pcomp_setup<T>(P, d12, d);
          // B1 = P^s_d(q2, q1) (stored), B2 = P^s_d(q1, q2) (consumed with B1 in the last pass)
          inv3d<T, N>(
              B1,
              [&](int i, int j, int k) {
                const T u = P.tabU[((size_t)id21 * 2 + sp) * NN + G::gidx(i, j, k)];
                return mul_si<T, 1>((pcomp<T, N>(q21, i, j, k) * u) * A1[G::sidx(i, j, k)]);
              },
              [&](int i, int j, int k, cplx<T> v) { B1[G::sidx(i, j, k)] = v; });
          // old accumulator values, B1 and the partner fields of one element, loaded before any store
          struct Old3 { cplx<T> b1, k1, br1; };
          inv3d_rmw<T, N, 4>(
              B2,
              [&](int i, int j, int k) {
                const T u = P.tabU[((size_t)id12 * 2 + sp) * NN + G::gidx(i, j, k)];
                return mul_si<T, 1>((pcomp<T, N>(q12, i, j, k) * u) * A2[G::sidx(i, j, k)]);
              },
              [&](int i, int j, int k) {
                const int g = G::gidx(i, j, k);
                Old3 o;
                // the axis-1 pencil of B2 is owned by the thread that wrote the same pencil of B1
                o.b1 = B1[G::sidx(i, j, k)];
                if (sp == 0) {
                  o.k1 = ldg(ket1 + g);
                  o.br1 = ldg(bra1 + g);
                }
                return o;
              },
              [&](int i, int j, int k, cplx<T> b2, const Old3& o) {
                const int g = G::gidx(i, j, k);
                red_add(&H6[g], w12 * (o.b1 * b2));
                if (sp == 0) {
                  red_add(&h3a4[d * NN + g], f1 * (b2 * o.k1));
                  red_add(&h3b[d * NN + g], f1 * mulc(o.b1, o.br1));
                }
              });
          __syncthreads();
        }
      }
    }
  }
  // 3a2 corrections of this q2: (f2/Nk)/Omega^2 sum_s [c_s F0 + (4 pi A_s/Nk) FT^{-1}[u~_s F_ab]]
  if (P.div && f2 != T(0) && !P.h3_only) {
    const T pref = (T)(f2 * P.invOm2);
    const T c0 = (T)(P.corr_c[0] + P.corr_c[1]);
    const cplx<T> cF0 = {(T)(c0 * sF0[0]), (T)(c0 * sF0[1])};
    const T a0 = (T)(4.0 * 3.14159265358979323846 * P.A[0] / P.Nk), a1 = (T)(4.0 * 3.14159265358979323846 * P.A[1] / P.Nk);
    inv3d<T, N>(
        B1,
        [&](int i, int j, int k) {
          const int g = G::gidx(i, j, k);
          const T u = a0 * P.hartUs[g] + a1 * P.hartUs[NN + g];
          return u * FAB[G::sidx(i, j, k)];
        },
        [&](int i, int j, int k, cplx<T> v) {
          red_add(&H6[G::gidx(i, j, k)], pref * (v + cF0));
        });
  }
}

// Grid index of the image S x of grid point (i1, i2, i3) under a fractional operation S.
template <int N> __device__ __forceinline__ int sym_image(const int* R, int i1, int i2, int i3) {
  int y[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int v = (R[3 * a] * i1 + R[3 * a + 1] * i2 + R[3 * a + 2] * i3) % N;
    y[a] = v < 0 ? v + N : v;
  }
  return (y[0] * N + y[1]) * N + y[2];
}

// h6 = sum over CTAs of the parts; h5_d = sum_q2 f/Nk h3b(q2)_d ket_q2 (Alg. 8).
// With symmetry the part of an irreducible q2;0 stands for every q2 of its star:
// part(q2)(x) = part(q2;0)(S x), conjugated under time reversal (Sec. 2.6.4).
template <typename T, int N> __global__ void k_reduce_a4(Params<T> P, int side0, int h5_only) {
  using G = Geo<N>;
  constexpr int NS = 6;
  const int side = side0 + blockIdx.y;
  const SideArgs<T>& S = P.side[side];
  const size_t NN = G::nn;
  const int M = P.Nk * P.no, ncta = (P.sym ? P.nirr * P.no : M) * P.so;   // k_occ_pairs CTAs per side
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < (int)NN; r += gridDim.x * blockDim.x) {
    cplx<T> h6 = {0, 0}, h5[3] = {{0, 0}, {0, 0}, {0, 0}};
    if (h5_only) {
    } else if (!P.sym) {
      for (int c = 0; c < ncta; ++c) {
        const size_t cta = (size_t)side * ncta + c;
        h6 = h6 + P.scratch[(cta * NS + 4) * (size_t)Geo<N>::vol + r];
      }
    } else {
      const int i1 = r / (N * N), i2 = (r / N) % N, i3 = r % N;
      for (int c = 0; c < ncta; ++c) {
        const int b = c / (P.no * P.so);
        const cplx<T>* part = P.scratch + (((size_t)side * ncta + c) * NS + 4) * (size_t)Geo<N>::vol;
        for (int t = P.star_off[b]; t < P.star_off[b + 1]; ++t) {
          const int* e = P.symk + 6 * P.star_k[t];
          cplx<T> v = part[sym_image<N>(P.symrot + 9 * e[1], i1, i2, i3)];
          if (e[2] < 0) v.y = -v.y;
          h6 = h6 + v;
        }
      }
    }
    for (int c = 0; c < M; ++c) {
      const int k = c / P.no, mu = c % P.no;
      const int q = k * P.nb + mu;
      const T f = (T)(P.occ[q] / P.Nk);
      const cplx<T> kv = S.ket[(size_t)q * NN + r];
#pragma unroll
      for (int d = 0; d < 3; ++d) h5[d] = h5[d] + f * (S.h3b[((size_t)c * 3 + d) * NN + r] * kv);
    }
    if (!h5_only) S.h6[r] = h6;
#pragma unroll
    for (int d = 0; d < 3; ++d) S.h5[d * NN + r] = h5[d];
  }
}

// Left-side occupied-pair fields from the right side's.  With F = FT of a pair density and
// U(p) = i p u~(p) (so conj U(p) = U(-p)), the left pair field of (a, b) is the conjugate of the
// right one of (b, a), P_L(a, b) = conj P_R(b, a); summed as in the occupied-pair stage this
// gives h6_L = conj h6_R, h3(3a4)_L = conj h3(3b)_R and h3(3b)_L = conj h3(3a4)_R.  Exact on the
// grid when -m is the negated Miller vector of every box index a pair density occupies (odd n,
// or pair densities that do not reach the Nyquist planes); the pipeline uses it only then.
template <typename T, int N> __global__ void k_left_from_right(Params<T> P) {
  const SideArgs<T>& R = P.side[0];
  const SideArgs<T>& L = P.side[1];
  const size_t NN = (size_t)N * N * N, M3 = (size_t)P.Nk * P.no * 3 * NN;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < NN + M3; e += (size_t)gridDim.x * blockDim.x) {
    if (e < NN) {
      L.h6[e] = conjg(R.h6[e]);
    } else {
      const size_t i = e - NN;
      L.h3a4[i] = conjg(R.h3b[i]);
      L.h3b[i] = conjg(R.h3a4[i]);
    }
  }
}

// Occupied-pair fields of every q2 at a non-irreducible k-point from those of its q2;0
// (Sec. 2.6.4, Eqs. symope_3a2_1/2), on the real-space grid: with k2 = tr S^T k0 - K,
//   h3a4(q2)(x) = e^{+2 pi i K.x} S_c^T [conj] h3a4(q2;0)(S x)   (crystal momentum +k2)
//   h3b(q2)(x)  = e^{-2 pi i K.x} S_c^T [conj] h3b(q2;0)(S x)    (crystal momentum -k2)
// (conjugation under time reversal), written into part 0 after the parts are summed.
template <typename T, int N> __global__ void k_unfold(Params<T> P) {
  const SideArgs<T>& S = P.side[blockIdx.y];
  const size_t NN = (size_t)N * N * N;
  const size_t total = (size_t)P.Nk * P.no * NN;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int q2 = (int)(e / NN), r = (int)(e % NN);
    const int k2 = q2 / P.no, mu = q2 % P.no;
    const int* m = P.symk + 6 * k2;
    if (m[0] == k2) continue;
    const int i1 = r / (N * N), i2 = (r / N) % N, i3 = r % N;
    const int y = sym_image<N>(P.symrot + 9 * m[1], i1, i2, i3);
    int kx = (m[3] * i1 + m[4] * i2 + m[5] * i3) % N;
    if (kx < 0) kx += N;
    double sn = 0.0, cs = 1.0;
    if (kx != 0) sincospi(2.0 * kx / N, &sn, &cs);
    const T* C = P.symcart + 9 * m[1];
    const size_t src = ((size_t)m[0] * P.no + mu) * 3, dst = (size_t)q2 * 3;
    for (int kind = 0; kind < 2; ++kind) {
      cplx<T>* h = kind == 0 ? S.h3a4 : S.h3b;
      cplx<T> v[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        v[d] = h[(src + d) * NN + y];
        if (m[2] < 0) v[d].y = -v[d].y;
      }
      const cplx<T> ph = {(T)cs, (T)(kind == 0 ? sn : -sn)};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const cplx<T> o = C[3 * d] * v[0] + C[3 * d + 1] * v[1] + C[3 * d + 2] * v[2];
        h[(dst + d) * NN + r] = ph * o;
      }
    }
  }
}

// Part 0 of a chunked accumulator += parts 1 .. nparts-1 (part = `len` elements), per side.
// which: 0 h3a4 and h3b (k_occ_pairs), 1 acc and w (k_pair_chain), 2 acc only (k_pair_3b4).
template <typename T, int N> __global__ void k_sum_parts(Params<T> P, int which) {
  const SideArgs<T>& S = P.side[blockIdx.y];
  const size_t NN = (size_t)N * N * N;
  const size_t nj = (size_t)P.nj_out, M = (size_t)P.nq2;
  const int nparts = which == 0 ? P.so : P.sc;
  cplx<T>* a = which == 0 ? S.h3a4 : S.acc;
  cplx<T>* b = which == 0 ? S.h3b : S.w;
  const size_t la = which == 0 ? M * 3 * NN : nj * NN, lb = which == 0 ? M * 3 * NN : (which == 1 ? nj * 3 * NN : 0);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < la + lb; e += (size_t)gridDim.x * blockDim.x) {
    cplx<T>* base = e < la ? a + e : b + (e - la);
    const size_t len = e < la ? la : lb;
    cplx<T> v = base[0];
    for (int c = 1; c < nparts; ++c) v = v + base[c * len];
    base[0] = v;
  }
}

// Local potential: tw2ah v_H + tw2bh2 s2b v_b2 - tw3a1 h1.h1/2 + tw3a2 h6/2 - tw3b1 t3b1 + tw3b2 t3b2
template <typename T, int N> __global__ void k_vloc(Params<T> P) {
  const SideArgs<T>& S = P.side[blockIdx.y];
  const size_t NN = (size_t)N * N * N;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < (int)NN; r += gridDim.x * blockDim.x) {
    cplx<T> h1h1 = {0, 0};
#pragma unroll
    for (int d = 0; d < 3; ++d) h1h1 = h1h1 + S.h1[d * NN + r] * S.h1[d * NN + r];
    cplx<T> v = P.tw[T2AH] * S.vH[r] + (P.tw[T2BH2] * S.s2b) * S.vb2[r] - (T(0.5) * P.tw[T3A1]) * h1h1 +
                (T(0.5) * P.tw[T3A2]) * S.h6[r] - P.tw[T3B1] * S.t3b1[r] + P.tw[T3B2] * S.t3b2[r];
    S.vloc[r] = v;
  }
}

// ---------------------------------------------------------------------------
// Per-partner and per-output combinations used by the pair chains (same side):
//   Z(q)_d = -(s2b tw2bx1 d_d ket_q + tw3a4 h3a4(q)_d)          (q occupied)
//   Y(j)_d = tw3b3 h1_d ket_j - s2b tw2bx2 d_d ket_j             (every j)
template <typename T, int N> __global__ void k_prep_zy(Params<T> P) {
  const SideArgs<T>& S = P.side[blockIdx.y];
  const size_t NN = (size_t)N * N * N;
  const size_t nz = (size_t)P.Nk * P.no * 3, ny = (size_t)P.nj_out * 3;
  const T* tw = P.tw;
  const T zg = -S.s2b * tw[T2BX1], zh = -tw[T3A4], y1 = tw[T3B3], yg = -S.s2b * tw[T2BX2];
  const size_t total = (nz + ny) * NN;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t v = e / NN, r = e % NN;
    if (v < nz) {
      const size_t qd = v;                       // (k * no + mu) * 3 + d
      const size_t d = qd % 3, qo = qd / 3;
      const size_t q = (qo / P.no) * P.nb + qo % P.no;
      S.Z[e] = zg * S.gket[(q * 3 + d) * NN + r] + zh * S.h3a4[e];
    } else {
      const size_t jd = v - nz, d = jd % 3, j = P.j0 + jd / 3;   // Y is indexed by j - j0
      S.Y[jd * NN + r] = y1 * (S.h1[d * NN + r] * S.ket[j * NN + r]) + yg * S.gket[(j * 3 + d) * NN + r];
    }
  }
}

// Fused pair chains, pass 1.  Grid (Nk*nb*sc, 2 sides); CTA = output orbital j and one of `sc`
// chunks of the partner range (chunk parts of acc / w, summed by k_sum_parts).
// For every occupied partner q (f = f_q / Nk, rho = conj(bra_q) ket_j):
//   A  = FT[rho]
//   2ax : acc -= tw f ket_q FT^{-1}[V(Delta + G) A]
//   for d: b = FT^{-1}[U^pp_d A]
//        acc += f Z(q)_d b  (2bx1, 3a4);   w_d += f ket_q b
//        F   = conj(bra_q) Y(j)_d - tw3b5 ket_j h3b(q)_d + tw3b6 n b   (3b3, 2bx2, 3b5, 3b6 pp)
//        C  += -U^pp_d FT[F]
//   for d: b = FT^{-1}[U^ap_d A];  C += -U^ap_d FT[tw3b6 n b]
//   acc += f ket_q FT^{-1}[C]
// The inverse transform of b ends on axis 1 and the forward transform of F
// starts on axis 1, so one thread owns each pencil through the pointwise work.
// When k_q = k_j the CTA also stores O_qj = A(0) and X_s = sum_{G != 0} u~_s(G) A(G) n~(-G)
// for the 3b6 corrections.  Slots: 0 B (work), 1 C (spectral accumulator), 2 A.
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::threads, 1) k_pair_chain(Params<T> P) {
  using G = Geo<N>;
  constexpr int NS = 3;
  constexpr int CH = 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(smraw);
  __shared__ T red[32];
  const SideArgs<T>& S = P.side[blockIdx.y];
  // with crystal symmetry only orbitals of irreducible k-points are computed (the rest are unfolded)
  const int jitem = blockIdx.x / P.sc, chunk = blockIdx.x % P.sc;
  const int jo = P.sym ? P.irr[jitem / P.nb] * P.nb + jitem % P.nb : jitem, j = P.j0 + jo, kj = j / P.nb;
  const int M = P.Nk * P.no, nj = P.nj_out;
  const int qi_begin = (int)((long long)chunk * M / P.sc), qi_end = (int)((long long)(chunk + 1) * M / P.sc);
  cplx<T>* B = vol_slot<T, N>(P, sm, 0, NS);
  cplx<T>* C = vol_slot<T, N>(P, sm, 1, NS);
  cplx<T>* A = vol_slot<T, N>(P, sm, 2, NS);
  const size_t NN = G::nn;
  const cplx<T>* ketj = S.ket + (size_t)j * NN;
  const cplx<T>* Yj = S.Y + (size_t)jo * 3 * NN;
  cplx<T>* acc = S.acc + ((size_t)chunk * nj + jo) * NN;
  cplx<T>* w = S.w + ((size_t)chunk * nj + jo) * 3 * NN;
  const T* tw = P.tw;
  const bool need_w = tw[T3A3] != T(0) || tw[T3B4] != T(0);
  const bool need_z = tw[T2BX1] != T(0) || tw[T3A4] != T(0);
  const bool need_y = tw[T3B3] != T(0) || tw[T2BX2] != T(0);
  const bool need_pp = need_w || need_z || tw[T3B6] != T(0);
  const bool need_F = need_y || tw[T3B5] != T(0) || tw[T3B6] != T(0);
  const bool need_ap = tw[T3B6] != T(0) && !P.no_ap;
  const T t3b5 = tw[T3B5], t3b6 = tw[T3B6];
  for (int r = threadIdx.x; r < (int)NN; r += blockDim.x) {
    acc[r] = cplx<T>{0, 0};
    for (int d = 0; d < 3; ++d) w[d * NN + r] = cplx<T>{0, 0};
  }
  __syncthreads();
  for (int qi = qi_begin; qi < qi_end; ++qi) {
    const int kq = qi / P.no, mu = qi % P.no;
    const int did = P.delta_id[kj * P.kstride + kq];
    const T* dl = P.delta + did * 3;
    const T* Vt = S.tabV + ((size_t)did * 2 + S.side) * NN;
    const T* Upp = P.tabU + ((size_t)did * 2 + 0) * NN;
    const T* Uap = P.tabU + ((size_t)did * 2 + 1) * NN;
    {
      const int q = kq * P.nb + mu;
      const T f = (T)(P.occ[q] / P.Nk);
      if (f == T(0)) continue;
      const cplx<T>* braq = S.bra + (size_t)q * NN;
      const cplx<T>* ketq = S.ket + (size_t)q * NN;
      const cplx<T>* Zq = S.Z + ((size_t)(kq * P.no + mu) * 3) * NN;
      const cplx<T>* h3bq = S.h3b + ((size_t)(kq * P.no + mu) * 3) * NN;
      // A = FT[conj(bra_q) ket_j]
      fwd3d<T, N>(B, [&](int a, int b, int c) { const int g = G::gidx(a, b, c); return mulc(ldg(ketj + g), ldg(braq + g)); },
                  [&](int a, int b, int c, cplx<T> v) { A[G::sidx(a, b, c)] = P.invN * v; });
      __syncthreads();
      if (P.div && kq == kj && t3b6 != T(0)) {
        // O_qj and X_s = sum_{G != 0} u~_s(G) A(G) n~(-G)
        for (int s = 0; s < 2; ++s) {
          T xr = 0, xi = 0;
          for (int g = threadIdx.x; g < (int)NN; g += blockDim.x) {
            const int a = g / (N * N), b = (g / N) % N, c = g % N;
            const int gn = G::gidx((N - a) % N, (N - b) % N, (N - c) % N);
            const cplx<T> t = P.hartUs[(size_t)s * NN + g] * (A[G::sidx(a, b, c)] * S.nt[gn]);
            xr += t.x;
            xi += t.y;
          }
          const T sr = block_sum<T>(xr, red);
          const T si = block_sum<T>(xi, red);
          if (threadIdx.x == 0) {
            double* cs = S.cs + ((size_t)jo * P.no + mu) * 6;
            cs[2 + 2 * s] = sr;
            cs[3 + 2 * s] = si;
            if (s == 0) { cs[0] = A[0].x; cs[1] = A[0].y; }
          }
        }
        __syncthreads();
      }
      // (2ax, -f ket_q FT^{-1}[V A], shares the final inverse transform: acc += f ket_q FT^{-1}[C - V A])
      const T t2ax = tw[T2AX];
      // grad-u channels: pp (with the fused second-stage vector field) and ap (3b6)
      for (int sp = 0; sp < 2; ++sp) {
        if (sp == 0 && !(need_pp || need_F)) continue;
        if (sp == 1 && !need_ap) continue;
        const T* Ut = sp == 0 ? Upp : Uap;
        for (int d = 0; d < 3; ++d) {
          const bool first_C = (sp == 0 && d == 0);
          const PComp<T> qd = pcomp_setup<T>(P, dl, d);
          // b = FT^{-1}[U_d A]: axes 2 and 3 here, axis 1 fused below
          fft_pass<T, N, +1, 2>(
              [&](int a, int b, int c) {
                return mul_si<T, 1>((pcomp<T, N>(qd, a, b, c) * Ut[G::gidx(a, b, c)]) * A[G::sidx(a, b, c)]);
              },
              [&](int a, int b, int c, cplx<T> v) { B[G::sidx(a, b, c)] = v; });
          __syncthreads();
          fft_pass<T, N, +1, 3>([&](int a, int b, int c) { return B[G::sidx(a, b, c)]; },
                                [&](int a, int b, int c, cplx<T> v) { B[G::sidx(a, b, c)] = v; });
          __syncthreads();
          // axis 1: inverse, pointwise work, forward (one thread owns each (i2, i3) pencil)
          for (int pp = threadIdx.x; pp < N * N; pp += blockDim.x) {
            const int i2 = pp / N, i3 = pp % N;
            cplx<T> v[N];
#pragma unroll
            for (int i = 0; i < N; ++i) v[i] = B[G::sidx(i, i2, i3)];
            Codelet<T, N, +1>::run(v);
            if (sp == 0) {
#pragma unroll
              for (int c0 = 0; c0 < N; c0 += CH) {
                cplx<T> lz[CH], lk[CH], ly[CH], lb[CH], lj[CH], lh[CH], ln[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                  if (c0 + u >= N) continue;
                  const int g = G::gidx(c0 + u, i2, i3);
                  lz[u] = ldg(Zq + d * NN + g); lk[u] = ldg(ketq + g); ly[u] = ldg(Yj + d * NN + g);
                  lb[u] = ldg(braq + g); lj[u] = ldg(ketj + g); lh[u] = ldg(h3bq + d * NN + g); ln[u] = ldg(S.n + g);
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                  if (c0 + u >= N) continue;
                  const int g = G::gidx(c0 + u, i2, i3);
                  const cplx<T> bv = v[c0 + u];
                  if (need_z) red_add(&acc[g], f * (lz[u] * bv));
                  if (need_w) red_add(&w[d * NN + g], f * (lk[u] * bv));
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
              for (int i = 0; i < N; ++i) v[i] = t3b6 * (ldg(S.n + G::gidx(i, i2, i3)) * v[i]);
            }
            if (sp == 0 && !need_F) continue;
            Codelet<T, N, -1>::run(v);
#pragma unroll
            for (int i = 0; i < N; ++i) B[G::sidx(i, i2, i3)] = v[i];
          }
          __syncthreads();
          if (sp == 0 && !need_F) continue;
          fft_pass<T, N, -1, 3>([&](int a, int b, int c) { return B[G::sidx(a, b, c)]; },
                                [&](int a, int b, int c, cplx<T> v) { B[G::sidx(a, b, c)] = v; });
          __syncthreads();
          fft_pass_pre<T, N, -1, 2, 8>(
              [&](int a, int b, int c) { return B[G::sidx(a, b, c)]; },
              [&](int a, int b, int c) { return pcomp<T, N>(qd, a, b, c) * Ut[G::gidx(a, b, c)] * P.invN; },
              [&](int a, int b, int c, cplx<T> v, T k) {
                // -U_d FT[F] = -i p_d u (v / N)
                const cplx<T> t = mul_si<T, -1>(k * v);
                const int s = G::sidx(a, b, c);
                C[s] = first_C ? t : C[s] + t;
              });
          __syncthreads();
        }
      }
      const bool has_C = need_F || need_ap;
      if (has_C || t2ax != T(0)) {
        inv3d_rmw<T, N, CH>(
            B,
            [&](int a, int b, int c) {
              const int s = G::sidx(a, b, c);
              cplx<T> v = has_C ? C[s] : cplx<T>{0, 0};
              if (t2ax != T(0)) v = v - (t2ax * Vt[G::gidx(a, b, c)]) * A[s];
              return v;
            },
            [&](int a, int b, int c) { return ldg(ketq + G::gidx(a, b, c)); },
            [&](int a, int b, int c, cplx<T> v, const cplx<T>& kq) {
              red_add(&acc[G::gidx(a, b, c)], f * (kq * v));
            });
        __syncthreads();
      }
    }
  }
}

// Pass 2 for 3b4 (Alg. 10): acc += tw f ket_q FT^{-1}[-U^pp . FT[-conj(bra_q) w_j]].
// Grid (Nk*nb*sc, 2 sides): orbital j and one of `sc` chunks of the partner range.
// Slots: 0 B (work), 1 A (spectral accumulator).
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::threads, 1) k_pair_3b4(Params<T> P) {
  using G = Geo<N>;
  constexpr int NS = 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(smraw);
  const SideArgs<T>& S = P.side[blockIdx.y];
  // with crystal symmetry only orbitals of irreducible k-points are computed (the rest are unfolded)
  const int jitem = blockIdx.x / P.sc, chunk = blockIdx.x % P.sc;
  const int jo = P.sym ? P.irr[jitem / P.nb] * P.nb + jitem % P.nb : jitem, j = P.j0 + jo, kj = j / P.nb;
  const int M = P.Nk * P.no, nj = P.nj_out;
  const int qi_begin = (int)((long long)chunk * M / P.sc), qi_end = (int)((long long)(chunk + 1) * M / P.sc);
  cplx<T>* B = vol_slot<T, N>(P, sm, 0, NS);
  cplx<T>* A = vol_slot<T, N>(P, sm, 1, NS);
  const size_t NN = G::nn;
  // chunk 0 adds to the complete accumulator (part 0); the others to their own zeroed parts
  cplx<T>* acc = S.acc + ((size_t)chunk * nj + jo) * NN;
  const cplx<T>* w = S.w + (size_t)jo * 3 * NN;
  const T t3b4 = P.tw[T3B4];
  if (t3b4 == T(0)) return;
  if (chunk > 0) {
    for (int r = threadIdx.x; r < (int)NN; r += blockDim.x) acc[r] = cplx<T>{0, 0};
    __syncthreads();
  }
  for (int qi = qi_begin; qi < qi_end; ++qi) {
    const int kq = qi / P.no, mu = qi % P.no;
    const int did = P.delta_id[kj * P.kstride + kq];
    const T* dl = P.delta + did * 3;
    const T* Upp = P.tabU + ((size_t)did * 2 + 0) * NN;
    {
      const int q = kq * P.nb + mu;
      const T f = (T)(P.occ[q] / P.Nk);
      if (f == T(0)) continue;
      const cplx<T>* braq = S.bra + (size_t)q * NN;
      const cplx<T>* ketq = S.ket + (size_t)q * NN;
      for (int d = 0; d < 3; ++d) {
        const PComp<T> qd = pcomp_setup<T>(P, dl, d);
        fwd3d_pre<T, N, 8>(
            B, [&](int a, int b, int c) { const int g = G::gidx(a, b, c); return mulc(ldg(w + d * NN + g), ldg(braq + g)); },
            [&](int a, int b, int c) { return pcomp<T, N>(qd, a, b, c) * Upp[G::gidx(a, b, c)] * P.invN; },
            [&](int a, int b, int c, cplx<T> v, T k) {
              // -U_d FT[-conj(bra_q) w_d] = +i p_d u FT[conj(bra_q) w_d]
              const cplx<T> t = mul_si<T, 1>(k * v);
              const int s = G::sidx(a, b, c);
              A[s] = d == 0 ? t : A[s] + t;
            });
        __syncthreads();
      }
      const T fw = t3b4 * f;
      inv3d_rmw<T, N, 8>(
          B, [&](int a, int b, int c) { return A[G::sidx(a, b, c)]; },
          [&](int a, int b, int c) { return ldg(ketq + G::gidx(a, b, c)); },
          [&](int a, int b, int c, cplx<T> v, const cplx<T>& kq) {
            red_add(&acc[G::gidx(a, b, c)], fw * (kq * v));
          });
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Finalize: acc += vloc ket_j + s2b tw2bh1 h1 . grad ket_j + tw3a3 h1 . w_j + 3b6 corrections,
// then out(G) = FT[acc](G) on the sphere of k_j (FP64 interleaved complex).
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::threads)
    k_finalize(Params<T> P, double2* outR, double2* outL, const int* __restrict__ box_index) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* V = work_vol<T, N>(smraw, P.scratch);
  const int side = blockIdx.y;
  const SideArgs<T>& S = P.side[side];
  double2* out = side == 0 ? outR : outL;
  if (out == nullptr) return;
  const int jo = P.sym ? P.irr[blockIdx.x / P.nb] * P.nb + blockIdx.x % P.nb : blockIdx.x;
  const int j = P.j0 + jo, kj = j / P.nb;
  const size_t NN = G::nn;
  const cplx<T>* ketj = S.ket + (size_t)j * NN;
  const cplx<T>* gketj = S.gket + (size_t)j * 3 * NN;
  const cplx<T>* acc = S.acc + (size_t)jo * NN;
  const cplx<T>* w = S.w + (size_t)jo * 3 * NN;
  const T t2bh1 = P.tw[T2BH1] * S.s2b, t3a3 = P.tw[T3A3];
  const bool corr = P.div && P.tw[T3B6] != T(0) && !P.band;
  const T a0 = (T)(4.0 * 3.14159265358979323846 * P.A[0] / P.Nk), a1 = (T)(4.0 * 3.14159265358979323846 * P.A[1] / P.Nk);
  const double n0x = corr ? (double)S.nt[0].x : 0.0, n0y = corr ? (double)S.nt[0].y : 0.0;
  fwd3d<T, N>(
      V,
      [&](int a, int b, int c) {
        const int g = G::gidx(a, b, c);
        const cplx<T> kv = ketj[g];
        cplx<T> v = acc[g] + S.vloc[g] * kv;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const cplx<T> h = S.h1[d * NN + g];
          v = v + t2bh1 * (h * gketj[d * NN + g]) + t3a3 * (h * w[d * NN + g]);
        }
        if (corr) {
          // sum_q f_q ket_q (1/Omega^2) sum_s [c_s n0 O_qj + (4 pi A_s/Nk)(O_qj vu_s + X_s)]
          cplx<T> s = {0, 0};
          for (int mu = 0; mu < P.no; ++mu) {
            const int q = kj * P.nb + mu;
            const double fq = P.occ[q];
            if (fq == 0.0) continue;
            const double* cs = S.cs + ((size_t)jo * P.no + mu) * 6;
            const cplx<T> O = {(T)cs[0], (T)cs[1]};
            const cplx<T> X0 = {(T)cs[2], (T)cs[3]}, X1 = {(T)cs[4], (T)cs[5]};
            const double cc = P.corr_c[0] + P.corr_c[1];
            const cplx<T> cn = {(T)(cc * n0x), (T)(cc * n0y)};
            cplx<T> t = cn * O + a0 * (O * S.vu[g] + X0) + a1 * (O * S.vu[NN + g] + X1);
            s = s + (T)(fq * P.invOm2) * (S.ket[(size_t)q * NN + g] * t);
          }
          v = v + P.tw[T3B6] * s;
        }
        return v;
      },
      [&](int a, int b, int c, cplx<T> v) { V[G::sidx(a, b, c)] = P.invN * v; });
  __syncthreads();
  double2* o = out + (size_t)jo * P.npw_max;
  for (int g = threadIdx.x; g < P.npw_max; g += blockDim.x) {
    const int bi = box_index[(size_t)kj * P.npw_max + g];
    if (bi < 0) {
      o[g] = make_double2(0.0, 0.0);
      continue;
    }
    const int i1 = bi / (N * N), i2 = (bi / N) % N, i3 = bi % N;
    const cplx<T> v = V[G::sidx(i1, i2, i3)];
    o[g] = make_double2((double)v.x, (double)v.y);
  }
}

}  // namespace tc
