// One block-Davidson step of the non-Hermitian one-body operator (tc_davidson_step).
//
// Sec. 2.4: the SCF equation is solved per k-point as the eigenvalue problem
// of h = T + (two-body) + (three-body) for fixed partner orbitals.  One step
// with a subspace of two blocks (p_max = 1):
//   1. h v_i for the m current orbitals v (the context's own operator launch,
//      right side only, plus the kinetic term);
//   2. w_i = P (h - eps_i) v_i, eps_i = <v_i|h|v_i>, with Payne's
//      preconditioner P(x), x(G) = |k+G|^2/2 / <v_i|T|v_i>; each w_i is
//      orthogonalised against everything kept so far (classical Gram-Schmidt,
//      two passes) and kept only if its remaining norm is at least 1e-8;
//   3. h w (a second operator context whose bands are the nocc partners
//      followed by the m new vectors, unoccupied);
//   4. the subspace matrix M_ab = <b_a|h|b_b> over b = (v, kept w), reduced to
//      Hessenberg form by Householder reflections and to Schur form
//      M = Q T Q^H by single-shift complex QR; right and left eigenvectors of T
//      by back / forward substitution, rotated by Q; the m eigenpairs of lowest
//      real part are kept;
//   5. phi_i = sum_a y_ai b_a and chi_i = sum_a z_ai b_a, then Gram-Schmidt of
//      phi and chi made biorthonormal to it (the library's biorthonormaliser).
// The operator launches run in the context's precision; every other step is FP64.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tc_ctx.hpp"

namespace tc {

struct DavState {
  tc_ctx* aux = nullptr;              // nbands = nocc + nbands: partners, then the new vectors
  double2* hv = nullptr;              // [Nk][m][npw_max] h v (operator + kinetic)
  double2* w = nullptr;               // [Nk][m][npw_max] kept new vectors, zero rows after the last
  double2* aux_phi = nullptr;         // [Nk][nocc + m][npw_max] partners phi, then w
  double2* aux_chi = nullptr;         // [Nk][nocc + m][npw_max] partners chi, then w
  double2* hw = nullptr;              // [Nk][nocc + m][npw_max] operator on the aux bands
  double2* Y = nullptr;               // [Nk][2m][m] right eigenvector coefficients
  double2* Z = nullptr;               // [Nk][2m][m] left eigenvector coefficients
  double2* lam = nullptr;             // [Nk][m] Ritz values, ascending real part
  double2* eig_scratch = nullptr;     // [Nk][eig_words] when the solver's arrays exceed shared memory
  int* cnt = nullptr;                 // [Nk] kept new vectors
  int* dim = nullptr;                 // [Nk] subspace dimension, -1 if the eigen-solver failed
  int* status = nullptr;              // biorthonormalisation status
  double2* h_lam = nullptr;           // pinned staging
  int* h_dim = nullptr;
  int* h_status = nullptr;
  std::vector<double> occ_aux;        // host [Nk][nocc + m]
  int aux_sym_version = 0;            // the context's symmetry version last given to aux
  size_t eig_words = 0;               // double2 words of the solver's arrays per k
  bool eig_in_smem = true;
};

void destroy_davidson(tc_ctx* c) {
  DavState* D = c->dav;
  if (!D) return;
  if (D->aux) destroy_context(D->aux);
  void* ptrs[] = {D->hv, D->w, D->aux_phi, D->aux_chi, D->hw, D->Y, D->Z, D->lam, D->eig_scratch,
                  D->cnt, D->dim, D->status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (D->h_lam) cudaFreeHost(D->h_lam);
  if (D->h_dim) cudaFreeHost(D->h_dim);
  if (D->h_status) cudaFreeHost(D->h_status);
  delete D;
  c->dav = nullptr;
}

}  // namespace tc

namespace {

constexpr double kNormCut = 1e-8;              // Sec. 2.4: vectors below this norm are left out
constexpr double kUlp = 2.220446049250313e-16;  // 2^-52
constexpr int kDavThreads = 256;
constexpr int kEigThreads = 128;
constexpr int kSmemCap = 200 * 1024;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // a / b with the larger component of b factored out (Smith's method)
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y, d = b.y + b.x * r;
  return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__device__ __forceinline__ double2 csqrt_(double2 z) {
  const double r = hypot(z.x, z.y);
  const double re = sqrt(0.5 * (r + z.x));
  const double im = sqrt(0.5 * fmax(r - z.x, 0.0));
  return make_double2(re, z.y < 0.0 ? -im : im);
}

__device__ __forceinline__ double payne(double x) {
  const double num = 27.0 + x * (18.0 + x * (12.0 + x * 8.0));
  return num / (num + 16.0 * x * x * x * x);
}

// Sum of a (up to 3 values) over the CTA; result valid in every thread.
template <int K> __device__ void block_sum(double (&a)[K], double* red) {
  for (int o = 16; o > 0; o >>= 1)
    for (int i = 0; i < K; ++i) a[i] += __shfl_xor_sync(0xffffffffu, a[i], o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
    for (int i = 0; i < K; ++i) red[K * w + i] = a[i];
  __syncthreads();
  for (int i = 0; i < K; ++i) {
    double t = 0.0;
    for (int j = 0; j < nw; ++j) t += red[K * j + i];
    a[i] = t;
  }
}

__device__ __forceinline__ double kin(const double* kpg, int k, int npw_max, int g) {
  const double* q = kpg + ((size_t)k * npw_max + g) * 3;
  return 0.5 * (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
}

// Steps 1-2 for one k-point per CTA: adds T v to hv, builds the kept new vectors
// w, and writes the second operator launch's inputs (partners, then w).
__global__ void __launch_bounds__(kDavThreads) k_dav_expand(const double2* __restrict__ v, const double2* __restrict__ vchi,
                                                            double2* hv, const double* __restrict__ kpg,
                                                            const int* __restrict__ npw_k, int npw_max, int m, int no,
                                                            double2* w, double2* aux_phi, double2* aux_chi, int* cnt_out) {
  __shared__ double red[3 * 32];
  __shared__ double2 coef[128];
  const int k = blockIdx.x, n = npw_k[k];
  const size_t row = npw_max;
  const double2* V = v + (size_t)k * m * row;
  double2* HV = hv + (size_t)k * m * row;
  double2* W = w + (size_t)k * m * row;
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int i = e / n, g = e % n;
    const double t = kin(kpg, k, npw_max, g);
    const double2 x = V[(size_t)i * row + g];
    double2& h = HV[(size_t)i * row + g];
    h.x += t * x.x;
    h.y += t * x.y;
  }
  __syncthreads();
  int cnt = 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int i = 0; i < m; ++i) {
    const double2* vi = V + (size_t)i * row;
    const double2* hi = HV + (size_t)i * row;
    double s[3] = {0.0, 0.0, 0.0};   // Re, Im <v|h v>, <v|T|v>
    for (int g = threadIdx.x; g < n; g += blockDim.x) {
      const double2 a = vi[g], b = hi[g];
      s[0] += a.x * b.x + a.y * b.y;
      s[1] += a.x * b.y - a.y * b.x;
      s[2] += kin(kpg, k, npw_max, g) * (a.x * a.x + a.y * a.y);
    }
    block_sum<3>(s, red);
    const double2 eps = make_double2(s[0], s[1]);
    const double ekin = s[2];
    double2* u = W + (size_t)cnt * row;
    for (int g = threadIdx.x; g < n; g += blockDim.x) {
      const double t = kin(kpg, k, npw_max, g);
      const double p = ekin > 0.0 ? payne(t / ekin) : (t == 0.0 ? 1.0 : 0.0);
      const double2 r = csub(hi[g], cmul(eps, vi[g]));
      u[g] = cscale(r, p);
    }
    __syncthreads();
    const int nbasis = m + cnt;
    for (int pass = 0; pass < 2; ++pass) {
      for (int b = warp; b < nbasis; b += nwarp) {
        const double2* pb = b < m ? V + (size_t)b * row : W + (size_t)(b - m) * row;
        double cx = 0.0, cy = 0.0;
        for (int g = lane; g < n; g += 32) {
          const double2 q = cmulc(pb[g], u[g]);
          cx += q.x;
          cy += q.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
          cx += __shfl_xor_sync(0xffffffffu, cx, o);
          cy += __shfl_xor_sync(0xffffffffu, cy, o);
        }
        if (lane == 0) coef[b] = make_double2(cx, cy);
      }
      __syncthreads();
      for (int g = threadIdx.x; g < n; g += blockDim.x) {
        double2 x = u[g];
        for (int b = 0; b < nbasis; ++b) {
          const double2* pb = b < m ? V + (size_t)b * row : W + (size_t)(b - m) * row;
          x = csub(x, cmul(coef[b], pb[g]));
        }
        u[g] = x;
      }
      __syncthreads();
    }
    double q[1] = {0.0};
    for (int g = threadIdx.x; g < n; g += blockDim.x) q[0] += u[g].x * u[g].x + u[g].y * u[g].y;
    block_sum<1>(q, red);
    const double nrm = sqrt(q[0]);
    if (nrm >= kNormCut) {
      const double inv = 1.0 / nrm;
      for (int g = threadIdx.x; g < n; g += blockDim.x) u[g] = cscale(u[g], inv);
      ++cnt;
    }
    __syncthreads();
  }
  // zero the unused rows and every row's padding
  for (int e = threadIdx.x; e < m * npw_max; e += blockDim.x) {
    const int i = e / npw_max, g = e % npw_max;
    if (i >= cnt || g >= n) W[e] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int na = no + m;
  for (int e = threadIdx.x; e < na * npw_max; e += blockDim.x) {
    const int b = e / npw_max, g = e % npw_max;
    double2 x, y;
    if (b < no) {
      x = v[((size_t)k * m + b) * row + g];
      y = vchi[((size_t)k * m + b) * row + g];
    } else {
      x = y = W[(size_t)(b - no) * row + g];
    }
    aux_phi[((size_t)k * na + b) * row + g] = x;
    aux_chi[((size_t)k * na + b) * row + g] = y;
  }
  if (threadIdx.x == 0) cnt_out[k] = cnt;
}

// ---------------------------------------------------------------------------
// Dense complex eigen-solver of one d x d matrix per CTA (A, Q row-major, leading
// dimension ld, in shared or global memory).

// Householder reduction of A to upper Hessenberg form, Q <- Q H_j (Q = I on entry).
__device__ void hessenberg(double2* A, double2* Q, int d, int ld, double2* hv, double* sh) {
  for (int j = 0; j + 2 < d; ++j) {
    if (threadIdx.x == 0) {
      double alpha2 = 0.0;
      for (int r = j + 1; r < d; ++r) alpha2 += A[r * ld + j].x * A[r * ld + j].x + A[r * ld + j].y * A[r * ld + j].y;
      const double2 x0 = A[(j + 1) * ld + j];
      const double ax0 = hypot(x0.x, x0.y);
      const double tail = alpha2 - ax0 * ax0;
      if (tail <= 0.0 || alpha2 == 0.0) {
        sh[0] = 0.0;   // column already reduced
      } else {
        const double alpha = sqrt(alpha2);
        const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
        const double2 beta = make_double2(-ph.x * alpha, -ph.y * alpha);
        for (int r = j + 1; r < d; ++r) hv[r] = A[r * ld + j];
        hv[j + 1] = csub(x0, beta);
        double vn2 = 0.0;
        for (int r = j + 1; r < d; ++r) vn2 += hv[r].x * hv[r].x + hv[r].y * hv[r].y;
        sh[0] = 2.0 / vn2;
        sh[1] = beta.x;
        sh[2] = beta.y;
      }
    }
    __syncthreads();
    const double tau = sh[0];
    if (tau == 0.0) {
      __syncthreads();
      continue;
    }
    // A <- (I - tau v v^H) A on columns j .. d-1
    for (int c = j + threadIdx.x; c < d; c += blockDim.x) {
      double2 s = make_double2(0.0, 0.0);
      for (int r = j + 1; r < d; ++r) s = cadd(s, cmulc(hv[r], A[r * ld + c]));
      s = cscale(s, tau);
      for (int r = j + 1; r < d; ++r) A[r * ld + c] = csub(A[r * ld + c], cmul(hv[r], s));
    }
    __syncthreads();
    // A <- A (I - tau v v^H), Q <- Q (I - tau v v^H) on every row
    for (int e = threadIdx.x; e < 2 * d; e += blockDim.x) {
      double2* M = e < d ? A : Q;
      const int r = e < d ? e : e - d;
      double2 s = make_double2(0.0, 0.0);
      for (int c = j + 1; c < d; ++c) s = cadd(s, cmul(M[r * ld + c], hv[c]));
      s = cscale(s, tau);
      for (int c = j + 1; c < d; ++c) M[r * ld + c] = csub(M[r * ld + c], cmul(s, cconj(hv[c])));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      A[(j + 1) * ld + j] = make_double2(sh[1], sh[2]);
      for (int r = j + 2; r < d; ++r) A[r * ld + j] = make_double2(0.0, 0.0);
    }
    __syncthreads();
  }
}

// Single-shift complex QR on the Hessenberg A (Wilkinson shift, exceptional shifts
// after 10 and 20 iterations without deflation), accumulating Q.  On return A is
// upper triangular (entries below the diagonal are ignored by the callers).
// Returns false if it did not converge within 30 max(10, d) iterations.
__device__ bool schur(double2* A, double2* Q, int d, int ld, int* si, double2* sc) {
  // sc[0] = (c, 0), sc[1] = s, sc[2] = shift; si[0] = lo, si[1] = action, si[2] = hi
  if (threadIdx.x == 0) {
    double an = 0.0;
    for (int r = 0; r < d; ++r)
      for (int c = (r > 0 ? r - 1 : 0); c < d; ++c) an = fmax(an, cabs1(A[r * ld + c]));
    sc[3] = make_double2(an, 0.0);
    si[2] = d - 1;
    si[3] = 0;   // iterations since the last deflation
    si[4] = 0;   // total iterations
  }
  __syncthreads();
  const int itmax = 30 * (d > 10 ? d : 10);
  while (true) {
    if (threadIdx.x == 0) {
      const int hi = si[2];
      int action = 0;   // 0: sweep, 1: deflate, 2: done, 3: fail
      int lo = 0;
      if (hi <= 0) {
        action = 2;
      } else {
        int l = hi;
        for (; l > 0; --l) {
          double s = cabs1(A[(l - 1) * ld + l - 1]) + cabs1(A[l * ld + l]);
          if (s == 0.0) s = sc[3].x;
          if (cabs1(A[l * ld + l - 1]) <= kUlp * s) {
            A[l * ld + l - 1] = make_double2(0.0, 0.0);
            break;
          }
        }
        lo = l;
        if (lo == hi) {
          action = 1;
        } else if (si[4] >= itmax) {
          action = 3;
        } else {
          si[3] += 1;
          si[4] += 1;
          double2 mu;
          const double2 hh = A[hi * ld + hi];
          if (si[3] == 10 || si[3] == 20) {
            mu = make_double2(hh.x + 0.75 * fabs(A[hi * ld + hi - 1].x), hh.y);
          } else {
            const double2 a = A[(hi - 1) * ld + hi - 1], b = A[(hi - 1) * ld + hi], c = A[hi * ld + hi - 1];
            const double2 half = cscale(csub(a, hh), 0.5);
            const double2 disc = csqrt_(cadd(cmul(half, half), cmul(b, c)));
            const double2 mid = cscale(cadd(a, hh), 0.5);
            const double2 m1 = cadd(mid, disc), m2 = csub(mid, disc);
            mu = cabs1(csub(m1, hh)) <= cabs1(csub(m2, hh)) ? m1 : m2;
          }
          sc[2] = mu;
        }
      }
      si[0] = lo;
      si[1] = action;
    }
    __syncthreads();
    const int action = si[1], lo = si[0], hi = si[2];
    if (action == 2) return true;
    if (action == 3) return false;
    if (action == 1) {
      __syncthreads();
      if (threadIdx.x == 0) {
        si[2] = hi - 1;
        si[3] = 0;
      }
      __syncthreads();
      continue;
    }
    const double2 mu = sc[2];
    for (int k = lo; k < hi; ++k) {
      if (threadIdx.x == 0) {
        double2 x, y;
        if (k == lo) {
          x = csub(A[lo * ld + lo], mu);
          y = A[(lo + 1) * ld + lo];
        } else {
          x = A[k * ld + k - 1];
          y = A[(k + 1) * ld + k - 1];
        }
        const double ax = hypot(x.x, x.y), ay = hypot(y.x, y.y);
        const double nn = hypot(ax, ay);
        double c;
        double2 s;
        if (nn == 0.0) {
          c = 1.0;
          s = make_double2(0.0, 0.0);
        } else if (ax == 0.0) {
          c = 0.0;
          s = make_double2(1.0, 0.0);
        } else {
          const double2 al = make_double2(x.x / ax, x.y / ax);
          c = ax / nn;
          s = cscale(cmul(al, cconj(y)), 1.0 / nn);
        }
        sc[0] = make_double2(c, 0.0);
        sc[1] = s;
      }
      __syncthreads();
      const double c = sc[0].x;
      const double2 s = sc[1];
      const int c0 = k == lo ? lo : k - 1;
      // rows k, k+1: [c s; -conj(s) c]
      for (int col = c0 + threadIdx.x; col < d; col += blockDim.x) {
        const double2 a = A[k * ld + col], b = A[(k + 1) * ld + col];
        A[k * ld + col] = cadd(cscale(a, c), cmul(s, b));
        A[(k + 1) * ld + col] = (k > lo && col == k - 1) ? make_double2(0.0, 0.0)
                                                          : csub(cscale(b, c), cmul(cconj(s), a));
      }
      __syncthreads();
      // columns k, k+1 of A (rows 0 .. min(k+2, hi)) and of Q (every row): times [c -s; conj(s) c]
      const int rA = (k + 2 < hi ? k + 2 : hi) + 1;
      for (int e = threadIdx.x; e < rA + d; e += blockDim.x) {
        double2* M = e < rA ? A : Q;
        const int r = e < rA ? e : e - rA;
        const double2 a = M[r * ld + k], b = M[r * ld + k + 1];
        M[r * ld + k] = cadd(cscale(a, c), cmul(cconj(s), b));
        M[r * ld + k + 1] = csub(cscale(b, c), cmul(s, a));
      }
      __syncthreads();
    }
  }
}

// Steps 4-5 for one k-point per CTA.
__global__ void __launch_bounds__(kEigThreads) k_dav_subspace(
    const double2* __restrict__ v, const double2* __restrict__ hv, const double2* __restrict__ w,
    const double2* __restrict__ hw, const double* __restrict__ kpg, const int* __restrict__ npw_k, int npw_max, int m,
    int no, const int* __restrict__ cnt_k, double2* Yout, double2* Zout, double2* lam_out, int* dim_out,
    double2* gscratch, size_t words) {
  extern __shared__ double2 dsm[];
  __shared__ double2 hvec[128];
  __shared__ double sh[4];
  __shared__ int si[8];
  __shared__ double2 sc[4];
  __shared__ int order[128];
  const int k = blockIdx.x, n = npw_k[k], d = m + cnt_k[k], ld = d;
  const size_t row = npw_max;
  double2* base = gscratch ? gscratch + (size_t)k * words : dsm;
  double2* A = base;
  double2* Q = A + (size_t)d * d;
  double2* X = Q + (size_t)d * d;      // [m][d] right vectors of T, then of M
  double2* U = X + (size_t)m * d;      // [m][d] left vectors of T, then of M
  const double2* V = v + (size_t)k * m * row;
  const double2* HV = hv + (size_t)k * m * row;
  const double2* W = w + (size_t)k * m * row;
  const double2* HW = hw + ((size_t)k * (no + m) + no) * row;
  // M[a][b] = <b_a | h b_b>, h w = operator output + T w
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int e = warp; e < d * d; e += nwarp) {
    const int a = e / d, b = e % d;
    const double2* pa = a < m ? V + (size_t)a * row : W + (size_t)(a - m) * row;
    double sx = 0.0, sy = 0.0;
    if (b < m) {
      const double2* pb = HV + (size_t)b * row;
      for (int g = lane; g < n; g += 32) {
        const double2 q = cmulc(pa[g], pb[g]);
        sx += q.x;
        sy += q.y;
      }
    } else {
      const double2* pb = HW + (size_t)(b - m) * row;
      const double2* pw = W + (size_t)(b - m) * row;
      for (int g = lane; g < n; g += 32) {
        const double t = kin(kpg, k, npw_max, g);
        const double2 hb = make_double2(pb[g].x + t * pw[g].x, pb[g].y + t * pw[g].y);
        const double2 q = cmulc(pa[g], hb);
        sx += q.x;
        sy += q.y;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) A[a * ld + b] = make_double2(sx, sy);
  }
  for (int e = threadIdx.x; e < d * d; e += blockDim.x)
    Q[e] = make_double2((e / d) == (e % d) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  hessenberg(A, Q, d, ld, hvec, sh);
  const bool ok = schur(A, Q, d, ld, si, sc);
  if (!ok) {
    for (int e = threadIdx.x; e < 2 * d * m; e += blockDim.x) {
      Yout[(size_t)k * 2 * m * m + e] = make_double2(0.0, 0.0);
      Zout[(size_t)k * 2 * m * m + e] = make_double2(0.0, 0.0);
    }
    if (threadIdx.x == 0) dim_out[k] = -1;
    return;
  }
  // order by real part (stable), and the largest |T_ij| for the substitution floor
  if (threadIdx.x == 0) {
    for (int i = 0; i < d; ++i) order[i] = i;
    for (int i = 1; i < d; ++i) {
      const int t = order[i];
      const double key = A[t * ld + t].x;
      int j = i - 1;
      while (j >= 0 && A[order[j] * ld + order[j]].x > key) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = t;
    }
    double tn = 0.0;
    for (int r = 0; r < d; ++r)
      for (int c = r; c < d; ++c) tn = fmax(tn, cabs1(A[r * ld + c]));
    sh[3] = fmax(kUlp * tn, 1e-300);
  }
  __syncthreads();
  const double smin = sh[3];
  // right (T x = lambda x) and left (u T = lambda u) vectors of T, one thread per kept eigenpair
  for (int s = threadIdx.x; s < m; s += blockDim.x) {
    const int p = order[s];
    const double2 lp = A[p * ld + p];
    double2* x = X + (size_t)s * d;
    double2* u = U + (size_t)s * d;
    for (int i = 0; i < d; ++i) x[i] = u[i] = make_double2(0.0, 0.0);
    x[p] = u[p] = make_double2(1.0, 0.0);
    for (int i = p - 1; i >= 0; --i) {
      double2 acc = make_double2(0.0, 0.0);
      for (int j = i + 1; j <= p; ++j) acc = cadd(acc, cmul(A[i * ld + j], x[j]));
      double2 den = csub(A[i * ld + i], lp);
      if (cabs1(den) < smin) den = make_double2(smin, 0.0);
      x[i] = cdiv(make_double2(-acc.x, -acc.y), den);
      if (cabs1(x[i]) > 1e100)
        for (int j = i; j <= p; ++j) x[j] = cscale(x[j], 1e-100);
    }
    for (int j = p + 1; j < d; ++j) {
      double2 acc = make_double2(0.0, 0.0);
      for (int i = p; i < j; ++i) acc = cadd(acc, cmul(u[i], A[i * ld + j]));
      double2 den = csub(A[j * ld + j], lp);
      if (cabs1(den) < smin) den = make_double2(smin, 0.0);
      u[j] = cdiv(make_double2(-acc.x, -acc.y), den);
      if (cabs1(u[j]) > 1e100)
        for (int i = p; i <= j; ++i) u[i] = cscale(u[i], 1e-100);
    }
    lam_out[(size_t)k * m + s] = lp;
  }
  __syncthreads();
  // y = Q x, z = Q conj(u) (each into registers, then back over x / u once every thread has read them)
  double2* Yk = Yout + (size_t)k * 2 * m * m;   // [2m][m]
  double2* Zk = Zout + (size_t)k * 2 * m * m;
  for (int e = threadIdx.x; e < 2 * m * m; e += blockDim.x) {
    Yk[e] = make_double2(0.0, 0.0);
    Zk[e] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < d * m; e += blockDim.x) {
    const int r = e / m, s = e % m;
    double2 y = make_double2(0.0, 0.0), z = make_double2(0.0, 0.0);
    for (int j = 0; j < d; ++j) {
      y = cadd(y, cmul(Q[r * ld + j], X[(size_t)s * d + j]));
      z = cadd(z, cmul(Q[r * ld + j], cconj(U[(size_t)s * d + j])));
    }
    Yk[(size_t)r * m + s] = y;
    Zk[(size_t)r * m + s] = z;
  }
  __syncthreads();
  // |y| = 1 and z^H y = 1 per eigenpair
  for (int s = threadIdx.x; s < m; s += blockDim.x) {
    double ny = 0.0;
    for (int r = 0; r < d; ++r) ny += Yk[(size_t)r * m + s].x * Yk[(size_t)r * m + s].x + Yk[(size_t)r * m + s].y * Yk[(size_t)r * m + s].y;
    const double iy = 1.0 / sqrt(ny);
    double2 zy = make_double2(0.0, 0.0);
    for (int r = 0; r < d; ++r) {
      Yk[(size_t)r * m + s] = cscale(Yk[(size_t)r * m + s], iy);
      zy = cadd(zy, cmulc(Zk[(size_t)r * m + s], Yk[(size_t)r * m + s]));
    }
    const double2 f = cconj(zy);
    for (int r = 0; r < d; ++r) Zk[(size_t)r * m + s] = cdiv(Zk[(size_t)r * m + s], f);
  }
  if (threadIdx.x == 0) dim_out[k] = d;
}

// With crystal symmetry: every k-point takes the kept-vector count of its irreducible point.
__global__ void k_dav_sym_cnt(int* cnt, const int* __restrict__ symk, int Nk) {
  for (int k = threadIdx.x; k < Nk; k += blockDim.x) {
    const int k0 = symk[6 * k];
    if (k0 != k) cnt[k] = cnt[k0];
  }
}

// phi_s = sum_a Y_as b_a, chi_s = sum_a Z_as b_a; one thread per plane wave.
__global__ void k_dav_rotate(const double2* __restrict__ v, const double2* __restrict__ w, const double2* __restrict__ Y,
                             const double2* __restrict__ Z, const int* __restrict__ dim_k, const int* __restrict__ npw_k,
                             int npw_max, int m, double2* phi, double2* chi) {
  const int k = blockIdx.y, g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npw_max) return;
  const int d = dim_k[k], n = npw_k[k];
  const size_t row = npw_max;
  const double2* Yk = Y + (size_t)k * 2 * m * m;
  const double2* Zk = Z + (size_t)k * 2 * m * m;
  for (int s = 0; s < m; ++s) {
    double2 p = make_double2(0.0, 0.0), q = make_double2(0.0, 0.0);
    if (g < n)
      for (int a = 0; a < d; ++a) {
        const double2 b = a < m ? v[((size_t)k * m + a) * row + g] : w[((size_t)k * m + a - m) * row + g];
        p = cadd(p, cmul(Yk[(size_t)a * m + s], b));
        q = cadd(q, cmul(Zk[(size_t)a * m + s], b));
      }
    phi[((size_t)k * m + s) * row + g] = p;
    chi[((size_t)k * m + s) * row + g] = q;
  }
}

tc_status dav_fail(tc_ctx* c, tc_status s, const std::string& m) { return tc::fail(c, s, m); }
tc_status dav_cuda(tc_ctx* c, cudaError_t e, const char* where) {
  return tc::fail(c, TC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Creates the Davidson buffers and the partner + new-vector context on first use.
tc_status ensure_davidson(tc_ctx* c) {
  if (c->dav) return TC_OK;
  const tc::Setup& S = c->S;
  const int m = S.nb, no = S.no, na = no + m;
  tc_params p = S.prm;
  p.nbands = na;
  p.nocc = no;
  tc::DavState* D = new (std::nothrow) tc::DavState();
  if (!D) return dav_fail(c, TC_ERR_OOM, "host allocation failed");
  c->dav = D;
  std::string err;
  const int r = tc::init_context(&p, true, &D->aux, err);
  if (r != TC_OK) {
    tc::destroy_davidson(c);
    return dav_fail(c, (tc_status)r, "Davidson operator context: " + err);
  }
  const size_t Nk = S.Nk, row = S.npw_max;
  const int dmax = 2 * m;
  D->eig_words = (size_t)2 * dmax * dmax + (size_t)2 * m * dmax;
  D->eig_in_smem = D->eig_words * sizeof(double2) <= (size_t)kSmemCap;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  al((void**)&D->hv, Nk * m * row * sizeof(double2));
  al((void**)&D->w, Nk * m * row * sizeof(double2));
  al((void**)&D->aux_phi, Nk * na * row * sizeof(double2));
  al((void**)&D->aux_chi, Nk * na * row * sizeof(double2));
  al((void**)&D->hw, Nk * na * row * sizeof(double2));
  al((void**)&D->Y, Nk * dmax * m * sizeof(double2));
  al((void**)&D->Z, Nk * dmax * m * sizeof(double2));
  al((void**)&D->lam, Nk * m * sizeof(double2));
  if (!D->eig_in_smem) al((void**)&D->eig_scratch, Nk * D->eig_words * sizeof(double2));
  al((void**)&D->cnt, Nk * sizeof(int));
  al((void**)&D->dim, Nk * sizeof(int));
  al((void**)&D->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&D->h_lam, Nk * m * sizeof(double2));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&D->h_dim, Nk * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&D->h_status, sizeof(int));
  if (e != cudaSuccess) {
    tc::destroy_davidson(c);
    cudaGetLastError();
    return dav_fail(c, e == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA,
                    std::string("Davidson buffers: ") + cudaGetErrorString(e));
  }
  D->occ_aux.assign(Nk * na, 0.0);
  return TC_OK;
}

}  // namespace

extern "C" {

tc_status tc_davidson_step(tc_ctx* c, const void* phi, const void* chi, const double* occ, void* phi_out,
                           void* chi_out, void* eig_out, int* dim_out, void* stream) {
  if (!c) return TC_ERR_STATE;
  if (c->batch) return dav_fail(c, TC_ERR_STATE, "batch context: use a single-cell context");
  if (c->S.nkb > 0) return dav_fail(c, TC_ERR_STATE, "band context: use a context from tc_init");
  if (!phi || !chi || !occ || !phi_out || !chi_out) return dav_fail(c, TC_ERR_ARG, "null pointer");
  if (phi_out == phi || phi_out == chi || chi_out == phi || chi_out == chi || phi_out == chi_out)
    return dav_fail(c, TC_ERR_ARG, "output arrays must not alias the inputs or each other");
  const tc::Setup& S = c->S;
  const int m = S.nb, no = S.no, na = no + m;
  if (m > tc::kBiorthoMaxBands) return dav_fail(c, TC_ERR_UNSUPPORTED, "tc_davidson_step supports at most 64 bands");
  if (const int f = tc::injected_fault("launch"))
    return dav_fail(c, (tc_status)f, "injected fault (TC_FAULT): no device work done");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tc_status r = ensure_davidson(c);
  if (r != TC_OK) return r;
  tc::DavState* D = c->dav;
  const size_t Nk = S.Nk, row = S.npw_max, orb = Nk * m * row * sizeof(double2);
  cudaError_t e = cudaSuccess;
  // inputs on the device
  const double2* dphi = static_cast<const double2*>(phi);
  const double2* dchi = static_cast<const double2*>(chi);
  if (!tc::device_ptr(phi)) {
    if ((e = cudaMemcpyAsync(c->d_in_phi, phi, orb, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return dav_cuda(c, e, "phi upload");
    dphi = c->d_in_phi;
  }
  if (!tc::device_ptr(chi)) {
    if ((e = cudaMemcpyAsync(c->d_in_chi, chi, orb, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return dav_cuda(c, e, "chi upload");
    dchi = c->d_in_chi;
  }
  const bool hp = !tc::device_ptr(phi_out), hc = !tc::device_ptr(chi_out);
  double2* ophi = hp ? c->d_out_R : static_cast<double2*>(phi_out);
  double2* ochi = hc ? c->d_out_L : static_cast<double2*>(chi_out);
  // 1. h v
  int rr = tc::stage_occ(c, occ, st);
  if (rr != TC_OK) return (tc_status)rr;
  rr = tc::apply_sides(c, dphi, dchi, D->hv, nullptr, 1, st);
  if (rr != TC_OK) return (tc_status)rr;
  // 2. new vectors, second launch's inputs
  k_dav_expand<<<S.Nk, kDavThreads, 0, st>>>(dphi, dchi, D->hv, c->d_kpg, c->d_npw, S.npw_max, m, no, D->w,
                                              D->aux_phi, D->aux_chi, D->cnt);
  if ((e = cudaGetLastError()) != cudaSuccess) return dav_cuda(c, e, "k_dav_expand");
  if (D->aux_sym_version != c->sym_version) {
    // the second operator context takes the same symmetry (it reduces h w as the first launch reduces h v)
    const int nops = (int)(c->sym_ops.size() / 9);
    const tc_status rs = tc_set_symmetry(D->aux, c->sym ? nops : 0, c->sym ? c->sym_ops.data() : nullptr, c->sym_tr);
    if (rs != TC_OK) return dav_fail(c, rs, "Davidson operator context: " + D->aux->err);
    D->aux_sym_version = c->sym_version;
  }
  if (c->sym) {
    // new vectors of the other k-points by symmetry, so that both launches see one symmetric set
    k_dav_sym_cnt<<<1, 128, 0, st>>>(D->cnt, c->d_symk, S.Nk);
    if ((e = cudaGetLastError()) != cudaSuccess) return dav_cuda(c, e, "k_dav_sym_cnt");
    int ru = tc::launch_sym_unfold(c, D->w, nullptr, st);
    if (ru == TC_OK) ru = tc::launch_sym_unfold(D->aux, D->aux_phi, D->aux_chi, st);
    if (ru != TC_OK) return (tc_status)ru;
  }
  // 3. h w with the same partners
  for (size_t k = 0; k < Nk; ++k)
    for (int b = 0; b < na; ++b) D->occ_aux[k * na + b] = b < no ? occ[k * m + b] : 0.0;
  rr = tc::stage_occ(D->aux, D->occ_aux.data(), st);
  if (rr != TC_OK) return dav_fail(c, (tc_status)rr, D->aux->err);
  // same partners as the h v launch: its partner-only fields (densities, Hartree-type fields, the
  // occupied-pair stage) are copied rather than recomputed
  D->aux->partners_from = c;
  rr = tc::apply_sides(D->aux, D->aux_phi, D->aux_chi, D->hw, nullptr, 1, st);
  D->aux->partners_from = nullptr;
  if (rr != TC_OK) return dav_fail(c, (tc_status)rr, D->aux->err);
  // 4. subspace eigenpairs
  const size_t eig_smem = D->eig_in_smem ? D->eig_words * sizeof(double2) : 0;
  if ((e = cudaFuncSetAttribute(k_dav_subspace, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eig_smem)) !=
      cudaSuccess)
    return dav_cuda(c, e, "k_dav_subspace attribute");
  k_dav_subspace<<<S.Nk, kEigThreads, eig_smem, st>>>(
      dphi, D->hv, D->w, D->hw, c->d_kpg, c->d_npw, S.npw_max, m, no, D->cnt, D->Y, D->Z, D->lam, D->dim,
      D->eig_in_smem ? nullptr : D->eig_scratch, D->eig_words);
  if ((e = cudaGetLastError()) != cudaSuccess) return dav_cuda(c, e, "k_dav_subspace");
  // 5. Ritz vectors, then Gram-Schmidt and biorthonormalisation
  k_dav_rotate<<<dim3((S.npw_max + 127) / 128, S.Nk), 128, 0, st>>>(dphi, D->w, D->Y, D->Z, D->dim, c->d_npw,
                                                                   S.npw_max, m, ophi, ochi);
  if ((e = cudaGetLastError()) != cudaSuccess) return dav_cuda(c, e, "k_dav_rotate");
  if ((e = cudaMemsetAsync(D->status, 0, sizeof(int), st)) != cudaSuccess) return dav_cuda(c, e, "status");
  rr = tc::launch_biortho(c, ophi, ochi, D->status, st);
  if (rr != TC_OK) return (tc_status)rr;
  if (c->sym && (rr = tc::launch_sym_unfold(c, ophi, ochi, st)) != TC_OK) return (tc_status)rr;
  // outputs
  if (hp && (e = cudaMemcpyAsync(phi_out, ophi, orb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return dav_cuda(c, e, "phi download");
  if (hc && (e = cudaMemcpyAsync(chi_out, ochi, orb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return dav_cuda(c, e, "chi download");
  if (eig_out) {
    const cudaMemcpyKind kind = tc::device_ptr(eig_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if ((e = cudaMemcpyAsync(eig_out, D->lam, Nk * m * sizeof(double2), kind, st)) != cudaSuccess)
      return dav_cuda(c, e, "eigenvalue copy");
  }
  if (dim_out && tc::device_ptr(dim_out) &&
      (e = cudaMemcpyAsync(dim_out, D->dim, Nk * sizeof(int), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return dav_cuda(c, e, "dimension copy");
  if ((e = cudaMemcpyAsync(D->h_dim, D->dim, Nk * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(D->h_status, D->status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return dav_cuda(c, e, "status copy");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return dav_cuda(c, e, "tc_davidson_step");
  if (dim_out && !tc::device_ptr(dim_out)) std::memcpy(dim_out, D->h_dim, Nk * sizeof(int));
  for (size_t k = 0; k < Nk; ++k)
    if (D->h_dim[k] < 0)
      return dav_fail(c, TC_ERR_NUMERIC,
                      "subspace eigen-solver did not converge at k-point " + std::to_string(k) + " (outputs undefined)");
  if (*D->h_status != 0)
    return dav_fail(c, TC_ERR_NUMERIC, "Ritz vectors: vanishing norm or singular overlap at k-point " +
                                           std::to_string(*D->h_status - 1) + " (outputs undefined)");
  return TC_OK;
}

}  // extern "C"
