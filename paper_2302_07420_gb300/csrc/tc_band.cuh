// Band-structure k-points off the SCF mesh (Sec. 2.6.3 after Eq. divcorr_2ax_scf; Sec. 2.6.4, 3b6).
//
// A band context appends nkb band points after the Nk mesh points: their orbitals are outputs only
// (orbital index (Nk + b) nb + j), every sum over occupied q runs over the mesh, and the pair terms
// take their kernels at k_b - q + G (never zero off the mesh).  The divergence corrections use the
// band constants Gamma_b and W(k_b) = sum_{q,G} (k_b - q + G) A_aux(k_b - q + G) and the band point's
// own occupied orbitals m (occupations f_m).  With c = 4 pi A_pp / (Nk Omega), s = +1 right / -1
// left, O_mj = <bra_m|ket_j>:
//   2ax   Eq. divcorr_2ax_band:          -(4 pi Gamma_b / Omega) sum_m f_m O_mj ket_m
//   2bx1  Eq. divcorr_2bx1:              + s i c sum_m f_m O_mj (W . grad ket_m)
//   2bx2  Eq. divcorr_2bx2:              - s i c sum_m f_m (W . <bra_m|grad ket_j>) ket_m
//   3a3   Eq. divcorr_3a3 and 3b4 Eq. div_corr_3b4_2: w_j += w_c = -i c W sum_m f_m O_mj ket_m
//   3b3   Eq. div_corr_3b3_2:            + i c sum_m f_m <bra_m|(W . h1) ket_j> ket_m
//   3a4   Eqs. div_corr_3a4_2/3:         + i c sum_m f_m O_mj (W . h3a(m))
//   3b5   Eqs. 3b5_div_2/3:              - i c sum_m f_m (W . mean(ket_j h3b(m))) ket_m
//   3b4   Eq. div_corr_3b4_4:            - i c sum_m f_m (W . <bra_m|w_j + w_c>) ket_m
//   3b6   Eqs. 3b6_div_band1/2/3 (times the multiplicity 2 and the 1/2 of 3b6), per channel s:
//         sum_m f_m ket_m [(4 pi A_s)^2 Gamma_b n~(0) O_mj - a_s O_mj V2_s - a_s X3_s,mj] / Omega^2,
//         a_s = 4 pi A_s / Nk,  V2_s = FT^{-1}[(W.G) u~_s n~]  (G != 0),
//         X3_s,mj = sum_{G != 0} (W.G) u~_s(G) FT[bra_m^* ket_j](G) n~(-G) = mean(bra_m^* ket_j V3_s),
//         V3_s = sum_m (W.G_{-m}) u~_s(G_{-m}) n~(m) e^{2 pi i m.x/n}  (m box indices, G_{-m} the wave
//         vector of index -m: V3 = -V2 except on the Nyquist planes of an even box)
// (sum_m A(m) B(-m) = mean(a b) for the box spectra A, B of fields a, b).  h3a(m), h3b(m) are the occupied-pair fields of the
// band point's own occupied orbitals (partners q1 on the mesh, kernels at k_b - q1 + G and
// q1 - k_b + G), each corrected for q1 -> k_b by Eq. correction_nabla:
//   h3a(m) -= i c W sum_m' f_m' O_m'm ket_m',    h3b(m) += i c W sum_m' f_m' O_mm' bra_m'^*.
// Means are (1/N) sum over the N grid points (the G = 0 coefficient of the product); FP64 sums.
#pragma once
#include "tc_kernels_impl.cuh"

namespace tc {

constexpr int kBandSums = 13;   // scalars per (side, b, m, j); see kBandScalars in tc_ctx.hpp

template <typename T> __device__ __forceinline__ cplx<double> to_d(cplx<T> v) { return {(double)v.x, (double)v.y}; }
__device__ __forceinline__ cplx<double> ld_bs(const double2* p) { return {p->x, p->y}; }
template <typename T> __device__ __forceinline__ cplx<double> times_i(cplx<T> v) { return {-(double)v.y, (double)v.x}; }

// Fields of band point b (no 1/Omega), grid (4 nkb, sides), kind = (neg, s):
//   V2_s = FT^{-1}[(W_b . G) u~_s(G) n~(G)] (neg = 0),  V3_s = FT^{-1}[(W_b . G_{-m}) u~_s(G_{-m}) n~(m)] (neg = 1),
// G != 0; stored at v2[b][2 neg + s].
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::threads) k_band_v2(Params<T> P) {
  using G = Geo<N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* V = work_vol<T, N>(smraw, P.scratch);
  const SideArgs<T>& S = P.side[blockIdx.y];
  const int b = blockIdx.x / 4, s = blockIdx.x % 2, neg = (blockIdx.x / 2) % 2;
  const double* bc = P.bandc + 4 * b;
  const T w0 = (T)bc[0], w1 = (T)bc[1], w2 = (T)bc[2];
  const PComp<T> q0 = pcomp_setup<T>(P, nullptr, 0), q1 = pcomp_setup<T>(P, nullptr, 1),
                 q2 = pcomp_setup<T>(P, nullptr, 2);
  cplx<T>* dst = S.v2 + ((size_t)b * 4 + 2 * neg + s) * G::nn;
  inv3d<T, N>(
      V,
      [&](int i, int j, int k) {
        const int g = G::gidx(i, j, k);
        const int a = neg ? (N - i) % N : i, bb = neg ? (N - j) % N : j, c = neg ? (N - k) % N : k;
        const T wg = w0 * pcomp<T, N>(q0, a, bb, c) + w1 * pcomp<T, N>(q1, a, bb, c) + w2 * pcomp<T, N>(q2, a, bb, c);
        return (wg * P.hartUs[(size_t)s * G::nn + G::gidx(a, bb, c)]) * S.nt[g];
      },
      [&](int i, int j, int k, cplx<T> v) { dst[G::gidx(i, j, k)] = v; });
}

// Grid means of the band corrections, one CTA per (b, m, j) and side: phase 0 O, <bra_m|grad ket_j>,
// <bra_m|(W.h1) ket_j>, X3_s = mean(bra_m^* ket_j V3_s); phase 1 mean(ket_j h3b(m)) (corrected h3b);
// phase 2 <bra_m|w_j> (w_j after its correction).
template <typename T, int N> __global__ void __launch_bounds__(256) k_band_scalars(Params<T> P, int phase) {
  constexpr int NV = 14;   // doubles reduced (7 complex sums at most)
  __shared__ double red[NV][8];
  const size_t NN = (size_t)N * N * N;
  const int side = blockIdx.y;
  const SideArgs<T>& S = P.side[side];
  const int item = blockIdx.x, b = item / (P.no * P.nb), m = (item / P.nb) % P.no, j = item % P.nb;
  const size_t om = (size_t)(P.Nk + b) * P.nb + m, oj = (size_t)(P.Nk + b) * P.nb + j;
  const cplx<T>* bra_m = S.bra + om * NN;
  const cplx<T>* ket_j = S.ket + oj * NN;
  const double* bc = P.bandc + 4 * b;
  double a[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) a[i] = 0.0;
  for (size_t r = threadIdx.x; r < NN; r += blockDim.x) {
    const cplx<T> bm = conjg(bra_m[r]), kj = ket_j[r];
    if (phase == 0) {
      const cplx<T> rho = bm * kj;
      const cplx<T> hw = (T)bc[0] * S.h1[r] + (T)bc[1] * S.h1[NN + r] + (T)bc[2] * S.h1[2 * NN + r];
      cplx<T> t[7];
      t[0] = rho;
      for (int d = 0; d < 3; ++d) t[1 + d] = bm * S.gket[(oj * 3 + d) * NN + r];
      t[4] = rho * hw;
      t[5] = rho * S.v2[((size_t)b * 4 + 2) * NN + r];
      t[6] = rho * S.v2[((size_t)b * 4 + 3) * NN + r];
#pragma unroll
      for (int i = 0; i < 7; ++i) { a[2 * i] += (double)t[i].x; a[2 * i + 1] += (double)t[i].y; }
    } else if (phase == 1) {
      for (int d = 0; d < 3; ++d) {
        const cplx<T> t = kj * S.bh3b[(((size_t)b * P.no + m) * 3 + d) * NN + r];
        a[2 * d] += (double)t.x;
        a[2 * d + 1] += (double)t.y;
      }
    } else {
      const size_t jo = (size_t)b * P.nb + j;
      for (int d = 0; d < 3; ++d) {
        const cplx<T> t = bm * S.w[(jo * 3 + d) * NN + r];
        a[2 * d] += (double)t.x;
        a[2 * d + 1] += (double)t.y;
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double v = a[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[i][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    v /= (double)NN;
    const int first = phase == 0 ? 0 : (phase == 1 ? 7 : 10), count = phase == 0 ? 7 : 3;
    if (threadIdx.x < 2 * count) {
      double* dst = reinterpret_cast<double*>(P.bs + (((size_t)side * P.nkb + b) * P.no + m) * P.nb * kBandSums +
                                              (size_t)j * kBandSums + first);
      dst[threadIdx.x] = v;
    }
  }
}

template <typename T>
__device__ __forceinline__ const double2* band_sc(const Params<T>& P, int side, int b, int m, int j) {
  return P.bs + ((((size_t)side * P.nkb + b) * P.no + m) * P.nb + j) * kBandSums;
}

// Correction of the band points' occupied-pair fields for q1 -> k_b (part 0 of bh3a, bh3b).
template <typename T, int N> __global__ void k_band_h3corr(Params<T> P, int nsides) {
  const size_t NN = (size_t)N * N * N;
  const size_t per_side = (size_t)P.nkb * P.no * 3 * NN;
  const double c = 4.0 * 3.14159265358979323846 * P.A[0] / (P.Nk * P.Omega);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nsides * per_side; e += (size_t)gridDim.x * blockDim.x) {
    const int side = (int)(e / per_side);
    const size_t rest = e % per_side, r = rest % NN;
    const int d = (int)((rest / NN) % 3), m = (int)((rest / (3 * NN)) % P.no), b = (int)(rest / (3 * NN * P.no));
    const SideArgs<T>& S = P.side[side];
    const double wd = P.bandc[4 * b + d];
    cplx<double> sa = {0, 0}, sb = {0, 0};
    for (int mp = 0; mp < P.no; ++mp) {
      const size_t o = (size_t)(P.Nk + b) * P.nb + mp;
      const double f = P.occ[o];
      if (f == 0.0) continue;
      const cplx<double> Oa = ld_bs(band_sc(P, side, b, mp, m));   // <bra_m'|ket_m>
      const cplx<double> Ob = ld_bs(band_sc(P, side, b, m, mp));   // <bra_m|ket_m'>
      sa = sa + (f * Oa) * to_d(S.ket[o * NN + r]);
      sb = sb + (f * Ob) * to_d(conjg(S.bra[o * NN + r]));
    }
    // h3a -= i c W_d sa;  h3b += i c W_d sb
    const size_t idx = (((size_t)b * P.no + m) * 3 + d) * NN + r;
    const cplx<double> ta = (c * wd) * cplx<double>{-sa.y, sa.x};
    const cplx<double> tb = (c * wd) * cplx<double>{-sb.y, sb.x};
    S.bh3a[idx] = S.bh3a[idx] - cplx<T>{(T)ta.x, (T)ta.y};
    S.bh3b[idx] = S.bh3b[idx] + cplx<T>{(T)tb.x, (T)tb.y};
  }
}

// w_j += w_c = -i c W sum_m f_m O_mj ket_m (part 0 of w; before the 3b4 pass and k_finalize).
template <typename T, int N> __global__ void k_band_wc(Params<T> P, int nsides) {
  const size_t NN = (size_t)N * N * N;
  const size_t per_side = (size_t)P.nj_out * 3 * NN;
  const double c = 4.0 * 3.14159265358979323846 * P.A[0] / (P.Nk * P.Omega);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nsides * per_side; e += (size_t)gridDim.x * blockDim.x) {
    const int side = (int)(e / per_side);
    const size_t rest = e % per_side, r = rest % NN;
    const int d = (int)((rest / NN) % 3), jo = (int)(rest / (3 * NN));
    const int b = jo / P.nb, j = jo % P.nb;
    const SideArgs<T>& S = P.side[side];
    cplx<double> sm = {0, 0};
    for (int m = 0; m < P.no; ++m) {
      const size_t o = (size_t)(P.Nk + b) * P.nb + m;
      const double f = P.occ[o];
      if (f == 0.0) continue;
      sm = sm + (f * ld_bs(band_sc(P, side, b, m, j))) * to_d(S.ket[o * NN + r]);
    }
    const cplx<double> t = (c * P.bandc[4 * b + d]) * cplx<double>{-sm.y, sm.x};
    S.w[e % per_side] = S.w[e % per_side] - cplx<T>{(T)t.x, (T)t.y};
  }
}

// acc_j += every band correction but the w_c part (part 0 of acc; after the 3b4 pass).
template <typename T, int N> __global__ void k_band_corr(Params<T> P, int nsides) {
  const size_t NN = (size_t)N * N * N;
  const size_t per_side = (size_t)P.nj_out * NN;
  const double pi4 = 4.0 * 3.14159265358979323846;
  const double c = pi4 * P.A[0] / (P.Nk * P.Omega), iom2 = P.invOm2;
  const double as[2] = {pi4 * P.A[0] / P.Nk, pi4 * P.A[1] / P.Nk};
  const double tw2ax = P.tw[T2AX], tw2bx1 = P.tw[T2BX1], tw2bx2 = P.tw[T2BX2], tw3b3 = P.tw[T3B3],
               tw3a4 = P.tw[T3A4], tw3b5 = P.tw[T3B5], tw3b4 = P.tw[T3B4], tw3b6 = P.tw[T3B6];
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nsides * per_side; e += (size_t)gridDim.x * blockDim.x) {
    const int side = (int)(e / per_side);
    const size_t rest = e % per_side, r = rest % NN;
    const int jo = (int)(rest / NN), b = jo / P.nb, j = jo % P.nb;
    const SideArgs<T>& S = P.side[side];
    const double s2b = (double)S.s2b;
    const double* bc = P.bandc + 4 * b;
    const double W[3] = {bc[0], bc[1], bc[2]}, gb = bc[3];
    const cplx<double> n0 = to_d(S.nt[0]);
    const cplx<double> v2sum = as[0] * to_d(S.v2[((size_t)b * 4 + 0) * NN + r]) + as[1] * to_d(S.v2[((size_t)b * 4 + 1) * NN + r]);
    double k3b6 = 0.0;
    for (int s = 0; s < 2; ++s) k3b6 += (pi4 * P.A[s]) * (pi4 * P.A[s]) * gb;
    cplx<double> tot = {0, 0};
    for (int m = 0; m < P.no; ++m) {
      const size_t o = (size_t)(P.Nk + b) * P.nb + m;
      const double f = P.occ[o];
      if (f == 0.0) continue;
      const double2* sc = band_sc(P, side, b, m, j);
      const cplx<double> O = ld_bs(sc), E = ld_bs(sc + 4), X0 = ld_bs(sc + 5), X1 = ld_bs(sc + 6);
      cplx<double> WD = {0, 0}, WF = {0, 0}, WG = {0, 0};
      for (int d = 0; d < 3; ++d) {
        WD = WD + W[d] * ld_bs(sc + 1 + d);
        WF = WF + W[d] * ld_bs(sc + 7 + d);
        WG = WG + W[d] * ld_bs(sc + 10 + d);
      }
      // i-multiples: -s i c tw2bx2 WD + i c tw3b3 E - i c tw3b5 WF - i c tw3b4 WG
      const cplx<double> ipart = (-s2b * c * tw2bx2) * WD + (c * tw3b3) * E + (-c * tw3b5) * WF + (-c * tw3b4) * WG;
      const cplx<double> alpha = f * ((-pi4 * gb / P.Omega * tw2ax) * O + cplx<double>{-ipart.y, ipart.x} +
                                      (tw3b6 * iom2) * (k3b6 * (n0 * O) - as[0] * X0 - as[1] * X1));
      const cplx<double> iO = {-O.y, O.x};
      const cplx<double> beta = (f * s2b * c * tw2bx1) * iO;
      const cplx<double> gamma = (f * c * tw3a4) * iO;
      const cplx<double> delta = (-f * tw3b6 * iom2) * O;
      const cplx<double> km = to_d(S.ket[o * NN + r]);
      cplx<double> wg = {0, 0}, wh = {0, 0};
      for (int d = 0; d < 3; ++d) {
        wg = wg + W[d] * to_d(S.gket[(o * 3 + d) * NN + r]);
        wh = wh + W[d] * to_d(S.bh3a[(((size_t)b * P.no + m) * 3 + d) * NN + r]);
      }
      tot = tot + alpha * km + beta * wg + gamma * wh + delta * (v2sum * km);
    }
    S.acc[rest] = S.acc[rest] + cplx<T>{(T)tot.x, (T)tot.y};
  }
}

}  // namespace tc
