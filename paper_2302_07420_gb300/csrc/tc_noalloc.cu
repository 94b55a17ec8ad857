// tc_apply_noalloc: the operator of tc_apply for callers that cannot allocate
// device memory (see include/tc.h).  Every device buffer of the call -- the
// basis maps, the kernel tables, the real-space fields and the pipeline's
// workspace -- is carved out of one file-scope device array of fixed size, so
// the call makes no cudaMalloc/cudaFree and no allocating library call.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "tc_ctx.hpp"

namespace tc {
void set_thread_error(const std::string& msg);   // defined in tc_api.cu (tc_last_error(NULL))
}

namespace {

constexpr size_t kNoallocBytes = (size_t)TC_NOALLOC_MAX_BYTES;
constexpr int kMaxDevices = 64;

// Scratch of every tc_apply_noalloc call on this device.  In host code the
// name `g_noalloc_arena` is only a host-side stand-in for the symbol: device
// addresses come from cudaGetSymbolAddress (g_arena_addr below).
static __device__ __align__(256) unsigned char g_noalloc_arena[kNoallocBytes];

std::mutex g_mu;
void* g_arena_addr[kMaxDevices] = {};
unsigned g_prepared[kMaxDevices] = {};   // bit (prec * 16 + size slot): kernel attributes and twiddles set

#define TC_FOR_N(X) \
  X(0, 9) X(1, 12) X(2, 15) X(3, 16) X(4, 18) X(5, 20) X(6, 24) X(7, 25) X(8, 27) X(9, 30) X(10, 32) X(11, 48)

template <typename T> int prepare(tc_ctx* c, int n) {
#define CASE(SLOT, NN) \
  case NN: return tc::prepare_kernels<T, NN>(c);
  switch (n) { TC_FOR_N(CASE) }
#undef CASE
  return TC_ERR_UNSUPPORTED;
}

template <typename T>
int run(tc_ctx* c, const double2* a, const double2* b, double2* oR, double2* oL, const double* tw, cudaStream_t st) {
#define CASE(SLOT, NN) \
  case NN: return tc::run_pipeline<T, NN>(c, a, b, oR, oL, tw, 2, st);
  switch (c->S.n) { TC_FOR_N(CASE) }
#undef CASE
  return TC_ERR_UNSUPPORTED;
}

int size_slot(int n) {
#define CASE(SLOT, NN) \
  case NN: return SLOT;
  switch (n) { TC_FOR_N(CASE) }
#undef CASE
  return -1;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

tc_status fail(tc_status s, const std::string& msg) {
  tc::set_thread_error("tc_apply_noalloc: " + msg);
  return s;
}

// Offsets into the arena (256-byte aligned pieces).
struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    const size_t o = off;
    off += bytes;
    return o;
  }
};

struct Layout {
  size_t box, kpg, did, delta, tabV, tabU, hartV, hartU, hartUs, occ, ws, total;
  tc::WsLayout W;   // the context's workspace block (fields, per-side fields, scratch) at offset ws
};

Layout plan(const tc_ctx& ctx, size_t rsz) {
  const tc::Setup& S = ctx.S;
  Layout L{};
  Carve c;
  const size_t nj = (size_t)S.Nk * S.nb;
  L.box = c.take(S.box_index.size() * sizeof(int));
  L.kpg = c.take((size_t)S.Nk * S.npw_max * 3 * sizeof(double));
  L.did = c.take(S.delta_id.size() * sizeof(int));
  L.delta = c.take((size_t)S.ndelta * 3 * rsz);
  L.tabV = c.take(S.tabV.size() * rsz);
  L.tabU = c.take(S.tabU.size() * rsz);
  L.hartV = c.take(S.hartV.size() * rsz);
  L.hartU = c.take(S.hartU.size() * rsz);
  L.hartUs = c.take(S.hartUs.size() * rsz);
  L.occ = c.take(nj * sizeof(double));
  L.W = tc::ws_layout(&ctx);
  L.ws = c.take(L.W.total);
  L.total = (c.off + 255) & ~(size_t)255;
  return L;
}

// Host FP64 vector -> arena piece in the compute precision (pageable copy on st).
template <typename T> cudaError_t put(char* dst, const std::vector<double>& v, cudaStream_t st) {
  if (v.empty()) return cudaSuccess;
  std::vector<T> h(v.size());
  for (size_t i = 0; i < v.size(); ++i) h[i] = (T)v[i];
  return cudaMemcpyAsync(dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

// Device address of this device's arena (looked up once per device, device current).
void* arena_address(int dev, cudaError_t& err) {
  err = cudaSuccess;
  if (dev < 0 || dev >= kMaxDevices) {
    err = cudaErrorInvalidDevice;
    return nullptr;
  }
  if (!g_arena_addr[dev]) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_noalloc_arena);
    if (err != cudaSuccess) return nullptr;
    g_arena_addr[dev] = p;
  }
  return g_arena_addr[dev];
}

}  // namespace

extern "C" tc_status tc_apply_noalloc(const tc_params* params, const void* phi_R, const void* phi_L,
                                      const double* occ, void* out_R, void* out_L, void* cuda_stream) {
  if (!params || !phi_R || !phi_L || !occ) return fail(TC_ERR_ARG, "null argument");
  if (!out_R && !out_L) return TC_OK;
  if (const int f = tc::injected_fault("launch")) return fail((tc_status)f, "injected fault (TC_FAULT): no device work done");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  {
    // the per-call uploads read host memory that lives only during the call: not capturable
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(st, &cap);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      // the legacy default stream while another stream captures in global mode
      if (ce == cudaErrorStreamCaptureImplicit)
        return fail(TC_ERR_STATE, "a graph capture is in progress: the per-call host uploads cannot be captured");
      return fail(TC_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
    }
    if (cap != cudaStreamCaptureStatusNone)
      return fail(TC_ERR_STATE, "the stream is capturing a graph: the per-call host uploads cannot be captured");
  }
  tc_ctx c;
  const std::string why = tc::build_setup(*params, c.S);
  if (!why.empty()) return fail(why.rfind("unsupported", 0) == 0 ? TC_ERR_UNSUPPORTED : TC_ERR_ARG, why);
  const tc::Setup& S = c.S;
  const size_t nj = (size_t)S.Nk * S.nb;
  for (size_t i = 0; i < nj; ++i)
    if (!(occ[i] >= 0.0 && occ[i] <= 1.0)) return fail(TC_ERR_ARG, "occupations must lie in [0, 1]");
  c.prec = params->precision;
  const bool f64 = c.prec == TC_FP64;
  c.esz = f64 ? 16 : 8;
  const size_t rsz = f64 ? 8 : 4;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(TC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  c.device = dev;
  c.nj_out = S.Nk * S.nb;
  {
    // the same grid rules as tc_init: derived left occupied-pair fields, pruned pair chains
    const int span = tc::miller_span(S.miller);
    c.left_from_right = tc::left_from_right_exact(S.n, span);
    c.pair_support = tc::pair_support_len(S.n, span);
  }
  tc::choose_splits(&c);
  Layout L = plan(c, rsz);
  if (L.total > kNoallocBytes) {   // partner chunks multiply the accumulators: fall back to one chunk
    c.split_occ[0] = c.split_occ[1] = c.split_chain[0] = c.split_chain[1] = 1;
    c.so_max = c.sc_max = 1;
    L = plan(c, rsz);
  }
  if (L.total > kNoallocBytes)
    return fail(TC_ERR_UNSUPPORTED, "problem needs " + std::to_string(L.total) + " bytes of device scratch; the "
                                    "static arena holds " + std::to_string(kNoallocBytes) + " (TC_NOALLOC_MAX_BYTES)");
  for (const void* p : {phi_R, phi_L, (const void*)out_R, (const void*)out_L})
    if (p && !on_device(p)) return fail(TC_ERR_ARG, "orbital and output arrays must be device pointers");

  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    base = static_cast<char*>(arena_address(dev, e));
    if (!base)
      return fail(TC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e) +
                                   (e == cudaErrorMemoryAllocation
                                        ? " (the static array is placed in device memory at the first call on a device "
                                          "under lazy module loading: make that call before reserving device memory)"
                                        : ""));
    const unsigned bit = 1u << ((f64 ? 0 : 16) + size_slot(S.n));
    if (!(g_prepared[dev] & bit)) {
      const int r = f64 ? prepare<double>(&c, S.n) : prepare<float>(&c, S.n);
      if (r != TC_OK) return fail((tc_status)r, c.err);
      g_prepared[dev] |= bit;
    }
  }
  // basis maps and tables
  std::vector<double> kpg((size_t)S.Nk * S.npw_max * 3, 0.0);
  for (int k = 0; k < S.Nk; ++k)
    for (int g = 0; g < S.npw[k]; ++g)
      for (int d = 0; d < 3; ++d) {
        const auto& m = S.miller[k][g];
        kpg[((size_t)k * S.npw_max + g) * 3 + d] = S.kcart[k][d] + (m[0] * S.B[0][d] + m[1] * S.B[1][d] + m[2] * S.B[2][d]);
      }
  std::vector<double> dl;
  for (auto& d : S.delta) dl.insert(dl.end(), d.begin(), d.end());
  auto ok = [&](cudaError_t r) { if (r != cudaSuccess && e == cudaSuccess) e = r; };
  ok(cudaMemcpyAsync(base + L.box, S.box_index.data(), S.box_index.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  ok(cudaMemcpyAsync(base + L.kpg, kpg.data(), kpg.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  ok(cudaMemcpyAsync(base + L.did, S.delta_id.data(), S.delta_id.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  const std::vector<double> occ_copy(occ, occ + nj);   // pageable: consumed before the copy call returns
  ok(cudaMemcpyAsync(base + L.occ, occ_copy.data(), nj * sizeof(double), cudaMemcpyHostToDevice, st));
  const std::vector<double>* tabs[] = {&dl, &S.tabV, &S.tabU, &S.hartV, &S.hartU, &S.hartUs};
  const size_t offs[] = {L.delta, L.tabV, L.tabU, L.hartV, L.hartU, L.hartUs};
  for (int i = 0; i < 6; ++i) ok(f64 ? put<double>(base + offs[i], *tabs[i], st) : put<float>(base + offs[i], *tabs[i], st));
  // the arena keeps the previous call's contents: start from the zeroed state of a fresh context
  ok(cudaMemsetAsync(base + L.ws + L.W.side, 0, 2 * L.W.side_bytes, st));
  ok(cudaMemsetAsync(base + L.ws + L.W.cs, 0, L.W.cs_bytes, st));
  if (e != cudaSuccess) return fail(TC_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));

  c.d_box_index = reinterpret_cast<int*>(base + L.box);
  c.d_kpg = reinterpret_cast<double*>(base + L.kpg);
  c.d_delta_id = reinterpret_cast<int*>(base + L.did);
  c.d_delta = base + L.delta;
  c.d_tabV = base + L.tabV;
  c.d_tabU = base + L.tabU;
  c.d_hartV = base + L.hartV;
  c.d_hartU = base + L.hartU;
  c.d_hartUs = base + L.hartUs;
  c.d_occ = reinterpret_cast<double*>(base + L.occ);
  tc::ws_assign(&c, base + L.ws, L.W);
  double tw[TC_NTERMS_OP];
  const unsigned mask = S.prm.term_mask;
  for (int t = 0; t < TC_NTERMS_OP; ++t) tw[t] = (mask == 0u || ((mask >> t) & 1u)) ? 1.0 : 0.0;
  const double2* a = static_cast<const double2*>(phi_R);
  const double2* b = static_cast<const double2*>(phi_L);
  double2* oR = static_cast<double2*>(out_R);
  double2* oL = static_cast<double2*>(out_L);
  const int r = f64 ? run<double>(&c, a, b, oR, oL, tw, st) : run<float>(&c, a, b, oR, oL, tw, st);
  if (r != TC_OK) return fail((tc_status)r, c.err);
  return TC_OK;
}
