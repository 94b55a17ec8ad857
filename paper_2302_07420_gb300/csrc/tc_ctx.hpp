// Library context: setup, device tables and workspace (all allocated in tc_init).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "tc_setup.hpp"

namespace tc {
struct BatchState;
struct DavState;
// Offsets of the workspace pieces of one context inside its workspace block.
struct WsLayout {
  size_t phi, chi, gphi, gchi, side, cs, scratch, total;
  size_t side_bytes, cs_bytes, scratch_bytes;
};
}  // namespace tc

struct tc_ctx {
  tc::Setup S;
  int prec = TC_FP64;
  size_t esz = 16;                 // bytes per complex element of the compute precision
  std::string err;
  int device = 0;
  // basis
  int* d_box_index = nullptr;      // [Nkt][npw_max] (mesh and band points)
  double* d_kpg = nullptr;         // [Nkt][npw_max][3]
  int* d_delta_id = nullptr;       // [Nkt][Nkt]
  void* d_delta = nullptr;         // [ndelta][3] T
  void* d_tabV = nullptr;          // [ndelta][2][N] T
  void* d_tabU = nullptr;          // [ndelta][2][N] T
  void* d_hartV = nullptr;         // [2][N] T
  void* d_hartU = nullptr;         // [N] T
  void* d_hartUs = nullptr;        // [2][N] T
  // tc_energy_grad: the base kernel data and its four derivatives (FP64, device, built by the first
  // call) and the element counts of the five tables
  double* d_kd64 = nullptr;
  size_t kd64_len[5] = {0, 0, 0, 0, 0};
  double* d_occ = nullptr;         // [Nk][nb]
  double* h_occ = nullptr;         // pinned [Nk][nb]
  // real-space orbitals
  void *d_phi = nullptr, *d_chi = nullptr, *d_gphi = nullptr, *d_gchi = nullptr;
  // per side fields (2 sides), each a separate allocation block
  void* d_side = nullptr;          // packed per-side global fields
  size_t side_bytes = 0;
  double* d_cs = nullptr;          // [2][Nk*nb][no][6]
  void* d_scratch = nullptr;
  size_t scratch_bytes = 0;
  // partner-chunk counts of k_occ_pairs / k_pair_chain for one-sided [0] and two-sided [1]
  // launches (chosen from the SM count, see choose_splits) and the largest of each
  int split_occ[2] = {1, 1}, split_chain[2] = {1, 1};
  int so_max = 1, sc_max = 1;
  // workspace block holding d_phi .. d_scratch (owned unless the context belongs to a batch)
  void* d_ws = nullptr;
  bool ws_owned = true;
  // staging for host pointers and energy
  double2 *d_in_phi = nullptr, *d_in_chi = nullptr, *d_out_R = nullptr, *d_out_L = nullptr;
  double2* d_edot = nullptr;       // [Nk*nb]
  double2* h_edot = nullptr;       // pinned
  int* d_npw = nullptr;            // [Nk]
  int* d_status = nullptr;         // device status word (tc_biorthonormalize)
  int* h_status = nullptr;         // pinned
  std::vector<int> npw_host;
  // derivative kernel data d/dA_pp, d/dA_ap, d/dC_pp, d/dC_ap (host, FP64), built by the first tc_energy_grad
  std::vector<tc::KernelData> dkd;
  // batch contexts (tc_init_batch): the cells and their shared workspace; nullptr otherwise
  tc::BatchState* batch = nullptr;
  bool batch_owner = false;        // a cell of a batch (destroyed with the batch)
  // crystal symmetry (tc_set_symmetry): maps and tables on the device, 0 / nullptr when off
  int sym = 0, nirr = 0;
  std::vector<int> sym_ops;        // host copy of the operations [nops][9] and the time-reversal flag
  int sym_tr = 0, sym_version = 0; // version: incremented by every tc_set_symmetry
  int *d_irr = nullptr, *d_symk = nullptr, *d_symrot = nullptr, *d_star_off = nullptr, *d_star_k = nullptr;
  int* d_sym_src = nullptr;        // [Nk][npw_max] sphere index at k0 of each coefficient at k (-1 pad)
  double* d_symcart64 = nullptr;   // [nops][9]
  float* d_symcart32 = nullptr;
  // two-sided launches derive the left occupied-pair fields from the right ones (exact here:
  // odd box, or pair densities clear of the Nyquist planes)
  bool left_from_right = false;
  // box indices per axis that a pair-density spectrum can occupy (tc::pair_support_len); the pair
  // chains use their pruned transforms when it fits the compiled support length (large: never)
  int pair_support = 1 << 30;
  // two-sided applies with the pruned pair kernels: the left pair chains take their pair spectra
  // and antiparallel 3b6 spectra from the right ones (k_pair_chain_pr, mirror); this buffer holds
  // them ([Nk no][Nk no][2][L^3] in the compute precision), allocated by tc_init when it fits in a
  // quarter of the free device memory, else null (each side computes its own)
  void* d_mirror = nullptr;
  size_t mirror_bytes = 0;
  // cluster-distributed pair kernels that can be scheduled on this device (bit 0 chain, 1 3b4,
  // 2 occupied pairs; tc_cluster.cuh), set by prepare_kernels
  int cluster_ok = 0;
  // set by tc_energy_grad for its passes along a derivative that is zero in the antiparallel kernel
  // table: the pair stages skip the work that reads only that table (it cancels in the difference)
  int skip_ap = 0;
  // compiled plans of the box: support length of the one-CTA pruned kernels (0: none), of the
  // cluster kernels (0: none) and the cluster widths of the chain, 3b4 and occupied-pair kernels
  int plan_prune_L = 0, plan_cl_L = 0;
  int plan_cl[3] = {0, 0, 0};
  // output orbitals of an apply: Nk nb at the mesh points, or nkb nb at the band points of a band
  // context (tc_init_band); band h3 chunks; band constants [nkb][4] = (W, Gamma_b) and the band
  // correction scalars [2][nkb][nocc][nbands][kBandScalars] (device)
  int nj_out = 0;
  int so_band = 1;
  double* d_band = nullptr;
  double2* d_bs = nullptr;
  // when set for one launch: a context with the same partners (occupied bands, occupations, cell,
  // precision) whose last launch left its partner-only fields (densities, Hartree-type fields,
  // occupied-pair stage) for the same sides; they are copied instead of recomputed
  const tc_ctx* partners_from = nullptr;
  // the last occupation upload from h_occ (h_occ is rewritten only after it has run)
  cudaEvent_t occ_ev = nullptr;
  bool occ_pending = false;
  // block-Davidson buffers and the partner + new-vector operator context (first tc_davidson_step)
  tc::DavState* dav = nullptr;
  // profiling (tc_profile / tc_stage_times)
  bool profile = false;
  cudaEvent_t ev[8] = {};
  double stage_ms[8] = {};
  int stage_launch[8] = {};
};

namespace tc {
// Context construction without the public wrapper: all tables, staging buffers
// and -- if own_workspace -- the workspace block.  Returns a tc_status; on
// failure *out is null and err holds the reason.
int init_context(const tc_params* p, bool own_workspace, tc_ctx** out, std::string& err, int nkb = 0,
                 const double* kfrac_band = nullptr);
// Complex FP64 scalars per (side, band point, occupied m, output j) of the band corrections:
// 0 <bra_m|ket_j>, 1-3 <bra_m|grad ket_j>, 4 <bra_m|(W.h1) ket_j>, 5-6 mean(bra_m^* ket_j V2_s),
// 7-9 mean(ket_j h3b(m)), 10-12 <bra_m|w_j> (w_j including its correction).
constexpr int kBandScalars = 13;
void destroy_context(tc_ctx* c);
WsLayout ws_layout(const tc_ctx* c);
// Chooses the partner-chunk counts of c for the current device (needs c->S).
void choose_splits(tc_ctx* c);
// n^3 volumes of one side's field block (see fill_side).
size_t side_field_vols(int Nk, int nb, int no, int so_max, int sc_max, int nj_out, int nkb, int so_band);
void ws_assign(tc_ctx* c, char* base, const WsLayout& L);
// Both operator sides into outR / outL (device pointers) on st, all terms of term_mask.
int apply_device(tc_ctx* c, const double2* phi, const double2* chi, double2* outR, double2* outL, cudaStream_t st);
void destroy_batch(tc_ctx* c);
void destroy_davidson(tc_ctx* c);
void free_symmetry(tc_ctx* c);
// Overwrites the coefficient arrays a, b ([Nk][nb][npw_max], device; b may be null) at every
// non-irreducible k-point by the symmetry image of its irreducible point.
int launch_sym_unfold(tc_ctx* c, double2* a, double2* b, cudaStream_t st);
// Validates occ (Nk*nb values in [0, 1]) and enqueues its upload into c->d_occ on st.
int stage_occ(tc_ctx* c, const double* occ, cudaStream_t st);
// Band contexts: mesh occupations, then those of the band points.
int stage_occ_band(tc_ctx* c, const double* occ, const double* band_occ, cudaStream_t st);
// Operator on nsides sides (1: right only into outR; 2: both) for orbitals already on the device.
int apply_sides(tc_ctx* c, const double2* phi, const double2* chi, double2* outR, double2* outL, int nsides,
                cudaStream_t st);
// Biorthonormalises phi / chi (device, [Nk][nb][npw_max]) in place on st; *status <- k + 1 on failure at k.
int launch_biortho(tc_ctx* c, double2* phi, double2* chi, int* status, cudaStream_t st);
constexpr int kBiorthoMaxBands = 64;
bool device_ptr(const void* p);
tc_status fail(tc_ctx* c, tc_status s, const std::string& msg);
// Host-side fault injection for tests of a caller's error handling (no device fault): the
// environment variable TC_FAULT, read on every call, names the failure.  site "alloc" (context
// creation, before any device allocation): TC_FAULT=alloc gives TC_ERR_OOM; site "launch" (the
// operator calls, before any device work): TC_FAULT=launch gives TC_ERR_CUDA, TC_FAULT=timeout
// TC_ERR_TIMEOUT.  Returns TC_OK when nothing is injected at that site.
int injected_fault(const char* site);
void set_thread_error(const std::string& msg);

// Runs the operator pipeline on the given stream.  tw: per-term weights;
// nsides: 2 (right and left) or 1 (right only).
template <typename T, int N>
int run_pipeline(tc_ctx* ctx, const double2* cphi, const double2* cchi, double2* outR, double2* outL,
                 const double* tw, int nsides, cudaStream_t st, const double2* bphi = nullptr,
                 const double2* bchi = nullptr);
template <typename T, int N> int prepare_kernels(tc_ctx* ctx);
template <typename T, int N> int run_fft3d(void* data, int batch, int sign, cudaStream_t st);
template <typename T, int N> size_t scratch_needed(const Setup& S, int so_max, int sc_max);
}  // namespace tc
