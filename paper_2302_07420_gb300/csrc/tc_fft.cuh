// Register-resident mixed-radix DFT codelets and CTA-level 3D FFT passes.
//
// One thread transforms whole pencils held in registers; a CTA transforms a
// full n^3 volume held in shared memory, one axis per pass.  Layout of a
// shared-memory volume: element (i1, i2, i3) at (i1 * n + i2) * P + i3 with
// P = n | 1 (odd row pitch, so the row-per-thread axis-3 pass is free of bank
// conflicts).  Global fields use the unpadded layout (i1 * n + i2) * n + i3.
//
// Conventions (periodic transform of Sec. 2.2 on the grid): the forward
// transform computes sum_r f(r) e^{-2 pi i m.r/n} (SIGN = -1, unnormalised;
// callers fold the 1/N of FT into their kernel factors) and the inverse
// computes sum_m F(m) e^{+2 pi i m.r/n} (SIGN = +1).
#pragma once
#include <cuda_runtime.h>

namespace tc {

template <typename T> struct cplx { T x, y; };

template <typename T> __device__ __forceinline__ cplx<T> mk(T a, T b) { return {a, b}; }
template <typename T> __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return {s * a.x, s * a.y}; }
template <typename T> __device__ __forceinline__ cplx<T> conjg(cplx<T> a) { return {a.x, -a.y}; }
// a * (s i) for s = +-1
template <typename T, int S> __device__ __forceinline__ cplx<T> mul_si(cplx<T> a) {
  return S > 0 ? cplx<T>{-a.y, a.x} : cplx<T>{a.y, -a.x};
}
// Read-only (non-coherent) load of a complex value: lets the compiler hoist it
// above stores to other arrays.
template <typename T> __device__ __forceinline__ cplx<T> ldg(const cplx<T>* p) {
  if constexpr (sizeof(T) == 4) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
  } else {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
  }
}
// a * conj(b)
template <typename T> __device__ __forceinline__ cplx<T> mulc(cplx<T> a, cplx<T> b) {
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

// ---------------------------------------------------------------------------
// Twiddle tables: exp(-2 pi i j / N), j < N, computed on the host in FP64
// (glibc sin/cos) and stored in constant memory per supported length.
constexpr int kTwLens[] = {2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 36, 40, 45, 48};
constexpr int kNumTwLens = sizeof(kTwLens) / sizeof(int);
__host__ __device__ constexpr int tw_offset(int N) {
  int off = 0;
  for (int i = 0; i < kNumTwLens; ++i) {
    if (kTwLens[i] == N) return off;
    off += kTwLens[i];
  }
  return -1;
}
constexpr int kTwTotal = tw_offset(48) + 48;

// One copy per translation unit (internal linkage); each instantiation unit
// uploads its own copy in prepare_kernels.
static __constant__ double c_tw64[2 * kTwTotal];
static __constant__ float c_tw32[2 * kTwTotal];

template <typename T> __device__ __forceinline__ cplx<T> tw_load(int idx);
template <> __device__ __forceinline__ cplx<double> tw_load<double>(int idx) { return {c_tw64[2 * idx], c_tw64[2 * idx + 1]}; }
template <> __device__ __forceinline__ cplx<float> tw_load<float>(int idx) { return {c_tw32[2 * idx], c_tw32[2 * idx + 1]}; }

// v * exp(S 2 pi i e / N)
template <typename T, int N, int S> __device__ __forceinline__ cplx<T> twiddle(int e, cplx<T> v) {
  e %= N;
  if (e == 0) return v;
  if ((4 * e) % N == 0) {
    const int q = (4 * e) / N;              // quarter turns
    if (q == 2) return cplx<T>{-v.x, -v.y};
    return (q == 1) ? mul_si<T, S>(v) : mul_si<T, -S>(v);
  }
  cplx<T> w = tw_load<T>(tw_offset(N) + e);   // exp(-2 pi i e/N)
  if (S > 0) w.y = -w.y;
  return v * w;
}

// ---------------------------------------------------------------------------
// Small butterflies (in place, natural order), exponent sign S.
template <typename T, int R, int S> struct Small;

template <typename T, int S> struct Small<T, 2, S> {
  static __device__ __forceinline__ void run(cplx<T>* z) {
    cplx<T> a = z[0], b = z[1];
    z[0] = a + b;
    z[1] = a - b;
  }
};

template <typename T, int S> struct Small<T, 3, S> {
  static __device__ __forceinline__ void run(cplx<T>* z) {
    const T h = T(0.5), s3 = T(0.86602540378443864676372317075294);   // sqrt(3)/2
    cplx<T> t1 = z[1] + z[2], t2 = z[1] - z[2];
    cplx<T> a = z[0];
    cplx<T> m = a - h * t1;
    cplx<T> r = mul_si<T, S>(s3 * t2);
    z[0] = a + t1;
    z[1] = m + r;
    z[2] = m - r;
  }
};

template <typename T, int S> struct Small<T, 4, S> {
  static __device__ __forceinline__ void run(cplx<T>* z) {
    cplx<T> a = z[0] + z[2], b = z[0] - z[2], c = z[1] + z[3], d = mul_si<T, S>(z[1] - z[3]);
    z[0] = a + c;
    z[2] = a - c;
    z[1] = b + d;
    z[3] = b - d;
  }
};

template <typename T, int S> struct Small<T, 5, S> {
  static __device__ __forceinline__ void run(cplx<T>* z) {
    // cos(2 pi/5), cos(4 pi/5), sin(2 pi/5), sin(4 pi/5)
    const T c1 = T(0.30901699437494742410229341718282), c2 = T(-0.80901699437494742410229341718282);
    const T s1 = T(0.95105651629515357211643933337938), s2 = T(0.58778525229247312916870595463907);
    cplx<T> x0 = z[0];
    cplx<T> t1 = z[1] + z[4], t2 = z[2] + z[3], t3 = z[1] - z[4], t4 = z[2] - z[3];
    cplx<T> a1 = x0 + c1 * t1 + c2 * t2, a2 = x0 + c2 * t1 + c1 * t2;
    cplx<T> b1 = mul_si<T, S>(s1 * t3 + s2 * t4), b2 = mul_si<T, S>(s2 * t3 - s1 * t4);
    z[0] = x0 + t1 + t2;
    z[1] = a1 + b1;
    z[4] = a1 - b1;
    z[2] = a2 + b2;
    z[3] = a2 - b2;
  }
};

__host__ __device__ constexpr int pick_radix(int n) {
  return (n % 4 == 0) ? 4 : (n % 3 == 0 ? 3 : (n % 2 == 0 ? 2 : (n % 5 == 0 ? 5 : n)));
}

// Mixed-radix decimation in time: X[k + M s] = sum_r W_R^{rs} (W_N^{rk} Y_r[k]),
// Y_r = DFT_M of x[r::R].
template <typename T, int N, int S> struct Codelet {
  static __device__ __forceinline__ void run(cplx<T>* x) {
    constexpr int R = pick_radix(N);
    constexpr int M = N / R;
    if constexpr (M == 1) {
      Small<T, R, S>::run(x);
    } else {
      cplx<T> y[N];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        cplx<T> sub[M];
#pragma unroll
        for (int m = 0; m < M; ++m) sub[m] = x[m * R + r];
        Codelet<T, M, S>::run(sub);
#pragma unroll
        for (int k = 0; k < M; ++k) y[r * M + k] = sub[k];
      }
#pragma unroll
      for (int k = 0; k < M; ++k) {
        cplx<T> z[R];
#pragma unroll
        for (int r = 0; r < R; ++r) z[r] = twiddle<T, N, S>(r * k, y[r * M + k]);
        Small<T, R, S>::run(z);
#pragma unroll
        for (int s = 0; s < R; ++s) x[k + M * s] = z[s];
      }
    }
  }
};

// ---------------------------------------------------------------------------
// CTA-level passes over an n^3 volume.  Pencil index p enumerates the n^2
// pencils of the pass; each thread takes p = tid, tid + blockDim.x, ...
//
//   axis 1: pencil (i2, i3), elements i1 = 0..n-1
//   axis 2: pencil (i1, i3), elements i2
//   axis 3: pencil (i1, i2), elements i3
//
// load(i1, i2, i3) -> cplx<T>;  store(i1, i2, i3, value).  Both are called
// with the element's coordinates; the pass performs the 1D DFT in between.
template <int N> struct Geo {
  static constexpr int n = N;
  static constexpr int P = N | 1;                 // shared-memory row pitch
  static constexpr int vol = N * N * P;           // shared-memory complex elements
  static constexpr int nn = N * N * N;            // global (unpadded) elements
  static __device__ __forceinline__ int sidx(int i1, int i2, int i3) { return (i1 * N + i2) * P + i3; }
  static __device__ __forceinline__ int gidx(int i1, int i2, int i3) { return (i1 * N + i2) * N + i3; }
};

template <typename T, int N, int S, int AXIS, typename Load, typename Store>
__device__ __forceinline__ void fft_pass(Load load, Store store) {
  for (int p = threadIdx.x; p < N * N; p += blockDim.x) {
    const int a = p / N, b = p % N;
    cplx<T> v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (AXIS == 1) v[i] = load(i, a, b);
      else if (AXIS == 2) v[i] = load(a, i, b);
      else v[i] = load(a, b, i);
    }
    Codelet<T, N, S>::run(v);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (AXIS == 1) store(i, a, b, v[i]);
      else if (AXIS == 2) store(a, i, b, v[i]);
      else store(a, b, i, v[i]);
    }
  }
}

// Full 3D transforms through a shared-memory work volume W.  Global memory is
// touched only in axis-1 and axis-2 passes, whose pencils put consecutive
// threads on consecutive i3 (coalesced); the axis-3 pass stays in shared memory.
//   forward  (SIGN -1): axes 1, 3, 2   load = real-space input, emit = spectrum
//   inverse  (SIGN +1): axes 2, 3, 1   load = spectrum,         emit = real-space output
// The caller synchronises after emit when it reuses W.
template <typename T, int N, typename Load, typename Emit>
__device__ __forceinline__ void fwd3d(cplx<T>* W, Load load, Emit emit) {
  using G = Geo<N>;
  fft_pass<T, N, -1, 1>(load, [&](int a, int b, int c, cplx<T> v) { W[G::sidx(a, b, c)] = v; });
  __syncthreads();
  fft_pass<T, N, -1, 3>([&](int a, int b, int c) { return W[G::sidx(a, b, c)]; },
                        [&](int a, int b, int c, cplx<T> v) { W[G::sidx(a, b, c)] = v; });
  __syncthreads();
  fft_pass<T, N, -1, 2>([&](int a, int b, int c) { return W[G::sidx(a, b, c)]; }, emit);
}

template <typename T, int N, typename Load, typename Emit>
__device__ __forceinline__ void inv3d(cplx<T>* W, Load load, Emit emit) {
  using G = Geo<N>;
  fft_pass<T, N, +1, 2>(load, [&](int a, int b, int c, cplx<T> v) { W[G::sidx(a, b, c)] = v; });
  __syncthreads();
  fft_pass<T, N, +1, 3>([&](int a, int b, int c) { return W[G::sidx(a, b, c)]; },
                        [&](int a, int b, int c, cplx<T> v) { W[G::sidx(a, b, c)] = v; });
  __syncthreads();
  fft_pass<T, N, +1, 1>([&](int a, int b, int c) { return W[G::sidx(a, b, c)]; }, emit);
}

// A pass whose store needs per-element data from global memory: after the
// transform of a pencil, pre(i1, i2, i3) is evaluated for a chunk of CH
// elements before store(i1, i2, i3, v, pre_value) runs on any of them, so the
// loads of a chunk are in flight together (each store through a generic
// pointer would otherwise hold back every later load).
template <typename T, int N, int S, int AXIS, int CH, typename Load, typename Pre, typename Store>
__device__ __forceinline__ void fft_pass_pre(Load load, Pre pre, Store store) {
  for (int p = threadIdx.x; p < N * N; p += blockDim.x) {
    const int a = p / N, b = p % N;
    cplx<T> v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (AXIS == 1) v[i] = load(i, a, b);
      else if (AXIS == 2) v[i] = load(a, i, b);
      else v[i] = load(a, b, i);
    }
    Codelet<T, N, S>::run(v);
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += CH) {
      decltype(pre(0, 0, 0)) o[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int i = c0 + u;
        if (i >= N) continue;
        if (AXIS == 1) o[u] = pre(i, a, b);
        else if (AXIS == 2) o[u] = pre(a, i, b);
        else o[u] = pre(a, b, i);
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int i = c0 + u;
        if (i >= N) continue;
        if (AXIS == 1) store(i, a, b, v[i], o[u]);
        else if (AXIS == 2) store(a, i, b, v[i], o[u]);
        else store(a, b, i, v[i], o[u]);
      }
    }
  }
}

// Forward transform whose emit needs per-element global data (see fft_pass_pre).
template <typename T, int N, int CH, typename Load, typename Pre, typename Emit>
__device__ __forceinline__ void fwd3d_pre(cplx<T>* W, Load load, Pre pre, Emit emit) {
  using G = Geo<N>;
  fft_pass<T, N, -1, 1>(load, [&](int a, int b, int c, cplx<T> v) { W[G::sidx(a, b, c)] = v; });
  __syncthreads();
  fft_pass<T, N, -1, 3>([&](int a, int b, int c) { return W[G::sidx(a, b, c)]; },
                        [&](int a, int b, int c, cplx<T> v) { W[G::sidx(a, b, c)] = v; });
  __syncthreads();
  fft_pass_pre<T, N, -1, 2, CH>([&](int a, int b, int c) { return W[G::sidx(a, b, c)]; }, pre, emit);
}

// Last (axis-1) pass of an inverse transform that feeds a read-modify-write of
// global arrays.  Per pencil and chunk of CH elements, pre(i1, i2, i3) loads
// every old value first and post(i1, i2, i3, v, old) then computes and stores,
// so the loads of a chunk are in flight together instead of one at a time.
template <typename T, int N, int CH, typename Pre, typename Post>
__device__ __forceinline__ void inv_axis1_rmw(cplx<T>* W, Pre pre, Post post) {
  using G = Geo<N>;
  for (int p = threadIdx.x; p < N * N; p += blockDim.x) {
    const int a = p / N, b = p % N;
    cplx<T> v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = W[G::sidx(i, a, b)];
    Codelet<T, N, +1>::run(v);
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += CH) {
      decltype(pre(0, 0, 0)) o[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u)
        if (c0 + u < N) o[u] = pre(c0 + u, a, b);
#pragma unroll
      for (int u = 0; u < CH; ++u)
        if (c0 + u < N) post(c0 + u, a, b, v[c0 + u], o[u]);
    }
  }
}

template <typename T, int N, int CH, typename Load, typename Pre, typename Post>
__device__ __forceinline__ void inv3d_rmw(cplx<T>* W, Load load, Pre pre, Post post) {
  using G = Geo<N>;
  fft_pass<T, N, +1, 2>(load, [&](int a, int b, int c, cplx<T> v) { W[G::sidx(a, b, c)] = v; });
  __syncthreads();
  fft_pass<T, N, +1, 3>([&](int a, int b, int c) { return W[G::sidx(a, b, c)]; },
                        [&](int a, int b, int c, cplx<T> v) { W[G::sidx(a, b, c)] = v; });
  __syncthreads();
  inv_axis1_rmw<T, N, CH>(W, pre, post);
}

// Pass on a pencil without a transform (pointwise work in the same thread mapping).
template <typename T, int N, int AXIS, typename Body>
__device__ __forceinline__ void pointwise_pass(Body body) {
  for (int p = threadIdx.x; p < N * N; p += blockDim.x) {
    const int a = p / N, b = p % N;
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      if (AXIS == 1) body(i, a, b);
      else if (AXIS == 2) body(a, i, b);
      else body(a, b, i);
    }
  }
}

}  // namespace tc
