// Device-side parameter blocks of the TC operator kernels.
#pragma once
#include <cuda_bf16.h>

#include "tc_fft.cuh"

namespace tc {

constexpr int NT = 16;   // operator terms, order of TC_TERM_* in tc.h
constexpr int kSmemLimit = 227 * 1024;   // bytes of shared memory per CTA on sm_103a
enum { T2AH, T2BH1, T2BH2, T2AX, T2BX1, T2BX2, T3A1, T3A2, T3A3, T3A4, T3B1, T3B2, T3B3, T3B4, T3B5, T3B6 };

// Fields of one side.  Right side: ket = phi, bra = chi; left side: ket = chi,
// bra = phi (Eq. BITCSCFconj).  Real-space fields are psi(r) = sum_G c(G) e^{iG.r}
// on the unpadded n^3 grid.
template <typename T> struct SideArgs {
  const cplx<T>* ket;    // [Nk][nb][N]
  const cplx<T>* bra;    // [Nk][nb][N]
  const cplx<T>* gket;   // [Nk][nb][3][N]
  cplx<T>* n;            // [N]      n = (1/Nk) sum_q f conj(bra_q) ket_q
  cplx<T>* m;            // [3][N]   (1/Nk) sum_q f conj(bra_q) grad ket_q
  cplx<T>* nt;           // [N]      FT[n] (1/N normalised)
  cplx<T>* mt;           // [3][N]   FT[m]
  cplx<T>* vH;           // [N]
  cplx<T>* h1;           // [3][N]
  cplx<T>* vb2;          // [N]
  cplx<T>* t3b1;         // [N]
  cplx<T>* t3b2;         // [N]
  cplx<T>* vu;           // [2][N]   sum_{G != 0} u~_s(G) n~(G) e^{iG.r}  (no 1/Omega)
  cplx<T>* spec;         // [3][N]   spectral scratch
  cplx<T>* h3a4;         // [so][Nk][no][3][N]  one part per partner chunk (part 0 holds the sum)
  cplx<T>* h3b;          // [so][Nk][no][3][N]
  cplx<T>* h5;           // [3][N]
  cplx<T>* h6;           // [N]
  cplx<T>* vloc;         // [N]
  cplx<T>* acc;          // [sc][Nk][nb][N]  output accumulator (real space), one part per partner chunk
  cplx<T>* w;            // [sc][Nk][nb][3][N]
  cplx<T>* Z;            // [Nk][no][3][N]  -(s2b tw2bx1 grad ket_q + tw3a4 h3a4(q))
  cplx<T>* Y;            // [Nk][nb][3][N]  tw3b3 h1 ket_j - s2b tw2bx2 grad ket_j
  double* cs;            // [nj_out][no][6]: O_qj, X_pp, X_ap (re, im each): 3b6 correction scalars
  cplx<T>* v2;           // [nkb][4]  band points: V2_pp, V2_ap, V3_pp, V3_ap (see tc_band.cuh)
  cplx<T>* bh3a;         // [so][nkb no][3][N]  band points: h3 (3a4 kind) of their occupied orbitals
  cplx<T>* bh3b;         // [so][nkb no][3][N]  band points: h3 (3b kind)
  const T* tabV;         // [ndelta][2][N] -> this side's V at offset side*N
  T s2b;                 // +1 right, -1 left (sign of the grad u . grad terms)
  int side;
};

template <typename T> struct Params {
  int Nk, nb, no, npw_max, ndelta;
  int nsmem;             // number of n^3 volumes held in shared memory
  int so, sc;            // partner chunks per CTA item of k_occ_pairs / k_pair_chain (this launch)
  int div;
  T Bm[3][3];            // reciprocal rows b_i
  T invN;
  double Omega, invOm2;
  double corr_c[2], A[2];
  T tw[NT];              // per-term weights (1 apply, 1/2 or 1/3 energy, 0 = off)
  const int* delta_id;   // [Nk][Nk]
  const T* delta;        // [ndelta][3]
  const T* tabU;         // [ndelta][2][N] u~_pp/Omega, u~_ap/Omega
  const T* tabV;         // [ndelta][2][N]
  const T* hartV;        // [2][N]
  const T* hartU;        // [N]
  const T* hartUs;       // [2][N] (no 1/Omega)
  const double* occ;     // [Nk][nb]
  cplx<T>* scratch;      // per-CTA volumes
  // crystal symmetry of the occupied-pair stage (tc_set_symmetry); sym = 0: every q2 computed
  int sym, nirr;
  const int* irr;        // [nirr] irreducible k-points, ascending
  const int* symk;       // [Nk][6]: k0, operation, tr (+1 / -1), K (3 integers)
  const int* symrot;     // [nops][9] fractional operation S (x -> S x), row-major
  const T* symcart;      // [nops][9] Cartesian S^dagger = S_c^T, row-major
  const int* star_off;   // [nirr + 1] offsets into star_k
  const int* star_k;     // [Nk] k-points grouped by their irreducible point
  // launch ranges (a mesh apply: kstride = Nk, j0 = 0, nj_out = Nk nb, i2_0 = 0, nq2 = Nk no)
  int kstride;           // row stride of delta_id: k-points with orbitals (mesh + band points)
  int j0, nj_out;        // output orbitals j0 .. j0 + nj_out - 1 (pair chains, 3b4, finalize, Y);
                         // acc, w, Y and cs are indexed by j - j0
  int i2_0, nq2;         // occupied-pair stage: q2 items i2_0 .. i2_0 + nq2 - 1 (item = k no + mu)
  int h3_only;           // occupied-pair stage: the two h3 kinds only (parallel spins, no h6)
  int no_ap;             // pair stages without the work that reads only the antiparallel kernel table
  int band;              // outputs at band points: no SCF-mesh 3b6 corrections in k_finalize
  int nkb;               // band points (band contexts)
  const double* bandc;   // [nkb][4]: W (3), Gamma_b
  double2* bs;           // [2][nkb][no][nb][13] band correction scalars (tc_band.cuh)
  // pair chains of a two-sided apply as two launches, right side first (k_pair_chain_pr): side0 is
  // the side of blockIdx.y = 0; mirror = 1 writes, for every occupied output j, the conjugate
  // reflections of each pair spectrum and antiparallel 3b6 spectrum into mir, mirror = 2 reads them
  // as the left side's own (see k_pair_chain_pr); mirror = 0: each side computes its own
  int side0, mirror;
  cplx<T>* mir;          // [Nk no (left output)][Nk no (partner)][2][L^3] compact spectra
  SideArgs<T> side[2];
};

}  // namespace tc
