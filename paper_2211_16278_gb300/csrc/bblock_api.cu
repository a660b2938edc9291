// Host side of the C ABI declared in include/bblock.h: argument checks, spin-operator
// analysis, workspace, phase cache, job tables and the launch sequence
//   phase table (cached) -> projection (Eq. 2) -> contraction (Eq. 1/3) -> slab reduction.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/bblock.h"
#include "bblock_internal.h"

using namespace bb;

struct bblock_ctx {
  bblock_config cfg{};
  int X = 0, rows = 0, num_sms = 0;
  std::string err;
  cudaStream_t last_stream = nullptr;
  int* d_status = nullptr;
  // phase cache
  std::vector<int32_t> phase_mom;
  double2* d_phase = nullptr;     // FP64 phases [n_mom][X], then their FP32 copy
  float2* d_phase_f = nullptr;
  float4* d_phase_df = nullptr;    // Ozaki form: the phases as double-float float4
  size_t phase_cap = 0;
  int* d_mom = nullptr;
  size_t mom_cap = 0;
  // workspace (fields + partials)
  char* d_ws = nullptr;
  size_t ws_cap = 0;
  // job tables: device copy + pinned host staging guarded by an event
  char* d_tab = nullptr;
  size_t tab_cap = 0;
  char* h_tab = nullptr;
  size_t h_tab_cap = 0;
  cudaEvent_t tab_free = nullptr;
  // device staging for bblock_compute_host, and the stream its copies run on
  char* d_io = nullptr;
  size_t io_cap = 0;
  cudaStream_t copy_stream = nullptr;
  // mode-triplet ordering: identity coefficients [4 n_ev][n_ev] and the mode-product
  // intermediates (folded phi3, T x3 phi3', then x2 phi2)
  double2* d_ident = nullptr;
  char* d_tri = nullptr;
  size_t tri_cap = 0;
  int last_launches = 0;
  int last_waves = 0;         // waves of jobs the last compute call ran in
  int last_path = -1;         // contraction path of the last compute call (BBLOCK_PATH_*)
  int graph_path = -1;
  size_t ws_budget = 0;
  // launch timing (bblock_profile_enable)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Timed { int kind; cudaEvent_t a, b; int kernels; };   // one timed step, its kernels
  std::vector<Timed> timed;
  // launch timing of CUDA-graph replays: event pairs captured as event-record nodes of the
  // graph (owned while the graph lives); a replay re-records them, so their times are
  // harvested into graph_ms / graph_cnt before the next replay or at bblock_profile_read
  std::vector<Timed> graph_timed;
  bool graph_pending = false;
  double graph_ms[8] = {};
  int graph_cnt[8] = {};
  // options (bblock_set_option)
  int opt_graphs = 1, opt_tc_nc = 0, opt_tc_chunk = 0, opt_slabs = 0, opt_checks = 0;
  unsigned long long* d_dbg = nullptr;  // first index violation of a checked launch
  // CUDA graph of a repeated call: captured on the second call with an identical
  // signature, replayed while the signature and the buffers it points to stay the same
  std::vector<uint64_t> last_sig, graph_sig;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_launches = 0;
  int graph_waves = 0;
  bool capturing = false;
  // pinned staging that a captured graph's table copies read at every replay: each upload
  // of the captured call (one per wave) keeps its own slot, at graph_tab_off onwards
  char* h_graph_tab = nullptr;
  size_t h_graph_tab_cap = 0;
  size_t graph_tab_off = 0;
  size_t call_tab_bytes = 0;  // slots the last call's uploads took, summed over its waves
  size_t opt_wave_bytes = 0;  // workspace budget per wave set by the caller (0: default)
  int opt_wait_us = 0;        // test hook: bounded-wait limit in microseconds (0: default)
  int opt_fail_alloc = 0;     // test hook: the next device allocation fails once
  int opt_corrupt_canary = 0; // test hook: the next call overwrites its first canary once
  int opt_tc_cluster = 0;     // tensor-core cluster size: 0 automatic, 1 none, 2 / 4 / 8
  int opt_host_chunks = 0;    // bblock_compute_host chunks of time slices (0: kHostChunks)
  // mixed forms' Eq. 2: tiled tensor-core projection (0), per-stage tensor-core projection
  // (1), FP32 FMA (2)
  int opt_tc_proj = 0;
  int opt_tc_rows = 0;        // FP16 form: row-factored phase 0 where it pays, 1 where it fits, 2 never
  long long cycles_per_us = 2070;
};

namespace {
// bblock_compute_host moves its time slices in at most this many chunks
constexpr int kHostChunks = 8;
enum KernelKind { K_PHASE = 0, K_PROJECT, K_CONTRACT, K_REDUCE, K_CONVERT, K_CANARY, K_COUNT };
const char* const kKernelNames[K_COUNT] = {"phase", "project", "contract", "reduce", "convert",
                                           "canary"};
static_assert(K_COUNT <= 8, "graph launch-time slots");

cudaEvent_t take_event(bblock_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

// Enqueue `launch` on `s`; when timing is on, bracket it with events. Under stream capture
// the events become event-record nodes of the graph (cudaEventRecordExternal), so every
// replay times its launches too.
template <class F>
cudaError_t timed_launch(bblock_ctx* c, int kind, cudaStream_t s, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  const unsigned rec_flags = c->capturing ? cudaEventRecordExternal : 0u;
  if (c->prof) {
    a = take_event(c);
    b = take_event(c);
    if (a && b && cudaEventRecordWithFlags(a, s, rec_flags) != cudaSuccess) {
      cudaGetLastError();
      c->ev_pool.push_back(a);
      c->ev_pool.push_back(b);
      a = b = nullptr;
    }
  }
  const long long n0 = t_kernel_launches;
  cudaError_t e = launch();
  c->last_launches += (int)(t_kernel_launches - n0);   // a step may launch several kernels
  if (a && b) {
    if (cudaEventRecordWithFlags(b, s, rec_flags) == cudaSuccess) {
      (c->capturing ? c->graph_timed : c->timed)
          .push_back({kind, a, b, (int)(t_kernel_launches - n0)});
    } else {
      cudaGetLastError();
      c->ev_pool.push_back(a);
      c->ev_pool.push_back(b);
    }
  } else {
    if (a) c->ev_pool.push_back(a);
    if (b) c->ev_pool.push_back(b);
  }
  return e;
}

// Add the launch times of the last graph replay (if not yet read) to graph_ms / graph_cnt.
// Waits for that replay to finish.
cudaError_t harvest_graph_times(bblock_ctx* c) {
  if (!c->graph_pending) return cudaSuccess;
  c->graph_pending = false;
  cudaError_t rc = cudaSuccess;
  for (const auto& t : c->graph_timed) {
    float m = 0.f;
    cudaError_t e = cudaEventSynchronize(t.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m, t.a, t.b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (rc == cudaSuccess) rc = e;
      continue;
    }
    c->graph_ms[t.kind] += m;
    c->graph_cnt[t.kind] += t.kernels;
  }
  return rc;
}
}  // namespace

namespace {

int fail(bblock_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

int cuda_fail(bblock_ctx* c, cudaError_t e, const char* what) {
  return fail(c, BBLOCK_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(ctx, call)                                             \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);      \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The FP64 and double-float forms share fields, tiles, units and the FP64 reduction.
bool fp64_like(const bblock_config& cfg) {
  return cfg.precision == BBLOCK_FP64 || cfg.precision == BBLOCK_DF64 ||
         cfg.precision == BBLOCK_OZAKI;
}

// Workspace one wave of jobs may take: the caller's limit, else half the free memory seen at
// creation (at most 96 GiB). A job larger than the budget still runs, alone in its wave.
size_t wave_budget(const bblock_ctx* c) { return c->opt_wave_bytes ? c->opt_wave_bytes : c->ws_budget; }

void drop_graph(bblock_ctx* c) {
  // the last replay's launch times are kept; its events then go back to the pool
  if (c->graph_pending && harvest_graph_times(c) != cudaSuccess) cudaGetLastError();
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  c->graph_sig.clear();
  for (const auto& t : c->graph_timed) {
    c->ev_pool.push_back(t.a);
    c->ev_pool.push_back(t.b);
  }
  c->graph_timed.clear();
}

int grow_device(bblock_ctx* c, char** p, size_t* cap, size_t need) {
  if (need <= *cap) return BBLOCK_OK;
  if (c->capturing) return fail(c, BBLOCK_ERR_UNSUPPORTED, "workspace growth during graph capture");
  if (c->opt_fail_alloc) {
    c->opt_fail_alloc = 0;
    return fail(c, BBLOCK_ERR_OOM, "allocation of %zu bytes failed (forced by the test hook)", need);
  }
  drop_graph(c);  // the graph holds the old addresses
  if (*p) {
    cudaError_t e = cudaStreamSynchronize(c->last_stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize before workspace growth");
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
  }
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, BBLOCK_ERR_OOM, "cudaMalloc of %zu bytes failed", need);
  }
  *cap = need;
  return BBLOCK_OK;
}

// Whether `p` is device-accessible memory of the context's device.
bool is_device_ptr(const bblock_ctx* c, const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == c->cfg.device;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Whether [p, p + bytes) lies inside the device allocation that contains p (driver query
// cuMemGetAddressRange, reached through the runtime's entry-point lookup; if the query is
// unavailable the extent is not checked).
typedef int (*MemRangeFn)(unsigned long long* base, size_t* size, unsigned long long ptr);
MemRangeFn mem_range_fn() {
  static MemRangeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<MemRangeFn>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

bool within_allocation(const void* p, size_t bytes) {
  const MemRangeFn fn = mem_range_fn();
  if (!fn) return true;
  unsigned long long base = 0;
  size_t size = 0;
  if (fn(&base, &size, reinterpret_cast<unsigned long long>(p)) != 0) return false;
  return reinterpret_cast<unsigned long long>(p) + bytes <= base + size;
}

// Whether [p, p + bytes) lies inside the context workspace.
bool within_workspace(const bblock_ctx* c, const void* p, size_t bytes) {
  const char* q = static_cast<const char*>(p);
  return q >= c->d_ws && q + bytes <= c->d_ws + c->ws_cap;
}

// Spin operator of Eq. (1) reduced to what the kernels consume.
struct SpinPlan {
  int n1 = 0, n2 = 0;                 // distinct alpha (line 1), beta (line 2)
  int slot1[4], slot2[4];             // spin -> slot, -1 if unused
  int alpha_of1[4], beta_of2[4];      // slot -> spin
  int n_pairs = 0;
  int a_slot[kMaxPairs], b_slot[kMaxPairs];
  int pair_alpha[kMaxPairs], pair_beta[kMaxPairs];
  // terms of each folded line-3 field, per momentum set index (1 if broadcast, P if per-momentum)
  int n_coef_sets = 1;
  std::vector<std::vector<std::vector<std::pair<int, double2>>>> terms;  // [set][pair] -> (gamma, c)
};

int plan_spins(bblock_ctx* c, const int32_t* spin_idx, const double* coeffs, int n_spin,
               int per_mom, int n_mom, SpinPlan* sp) {
  for (int i = 0; i < 4; ++i) sp->slot1[i] = sp->slot2[i] = -1;
  std::vector<int> pair_of(n_spin);
  for (int s = 0; s < n_spin; ++s) {
    const int al = spin_idx[3 * s], be = spin_idx[3 * s + 1], ga = spin_idx[3 * s + 2];
    if (al < 0 || al > 3 || be < 0 || be > 3 || ga < 0 || ga > 3)
      return fail(c, BBLOCK_ERR_INVALID_ARG, "spin triple %d = (%d,%d,%d) outside 0..3", s, al, be, ga);
    if (sp->slot1[al] < 0) { sp->alpha_of1[sp->n1] = al; sp->slot1[al] = sp->n1++; }
    if (sp->slot2[be] < 0) { sp->beta_of2[sp->n2] = be; sp->slot2[be] = sp->n2++; }
    int pr = -1;
    for (int k = 0; k < sp->n_pairs; ++k)
      if (sp->pair_alpha[k] == al && sp->pair_beta[k] == be) pr = k;
    if (pr < 0) {
      pr = sp->n_pairs++;
      sp->pair_alpha[pr] = al;
      sp->pair_beta[pr] = be;
      sp->a_slot[pr] = sp->slot1[al];
      sp->b_slot[pr] = sp->slot2[be];
    }
    pair_of[s] = pr;
  }
  sp->n_coef_sets = per_mom ? n_mom : 1;
  sp->terms.assign(sp->n_coef_sets, std::vector<std::vector<std::pair<int, double2>>>(sp->n_pairs));
  for (int set = 0; set < sp->n_coef_sets; ++set)
    for (int s = 0; s < n_spin; ++s) {
      const double* cz = coeffs + 2 * ((size_t)set * n_spin + s);
      const int ga = spin_idx[3 * s + 2];
      auto& tl = sp->terms[set][pair_of[s]];
      bool merged = false;
      for (auto& t : tl)
        if (t.first == ga) { t.second.x += cz[0]; t.second.y += cz[1]; merged = true; }
      if (!merged) tl.push_back({ga, make_double2(cz[0], cz[1])});
    }
  return BBLOCK_OK;
}

int ensure_phase(bblock_ctx* c, const int32_t* momenta, int n_mom, cudaStream_t s) {
  std::vector<int32_t> key(momenta, momenta + 3 * n_mom);
  if (c->d_phase && key == c->phase_mom) return BBLOCK_OK;
  const size_t n_ph = (size_t)c->X * n_mom;
  const bool oz = c->cfg.precision == BBLOCK_OZAKI;
  const size_t df_ofs = align_up((sizeof(double2) + sizeof(float2)) * n_ph, 256);
  int rc = grow_device(c, reinterpret_cast<char**>(&c->d_phase), &c->phase_cap,
                       df_ofs + (oz ? sizeof(float4) * n_ph : 0));
  if (rc) return rc;
  c->d_phase_f = reinterpret_cast<float2*>(c->d_phase + n_ph);
  c->d_phase_df = oz ? reinterpret_cast<float4*>(reinterpret_cast<char*>(c->d_phase) + df_ofs)
                     : nullptr;
  rc = grow_device(c, reinterpret_cast<char**>(&c->d_mom), &c->mom_cap, sizeof(int) * 3 * n_mom);
  if (rc) return rc;
  CK(c, cudaMemcpyAsync(c->d_mom, momenta, sizeof(int) * 3 * n_mom, cudaMemcpyHostToDevice, s));
  CK(c, timed_launch(c, K_PHASE, s, [&] { return launch_phase_table(c->cfg.L, n_mom, c->d_mom, c->d_phase, c->d_phase_f, s); }));
  if (oz)
    CK(c, timed_launch(c, K_PHASE, s, [&] { return launch_phase_df(c->d_phase, c->d_phase_df, (long long)n_ph, s); }));
  // the host momentum array may be reused by the caller right after return
  CK(c, cudaStreamSynchronize(s));
  c->phase_mom = key;
  return BBLOCK_OK;
}

// Copy `bytes` of host tables into the device table buffer on `s` via pinned staging.
int upload_tables(bblock_ctx* c, const void* src, size_t bytes, cudaStream_t s) {
  const size_t slot = align_up(bytes, 256);
  c->call_tab_bytes += slot;
  if (c->capturing) {
    // The graph's memcpy node reads its slot at every replay, so every wave of the captured
    // call needs a slot of its own: a shared one would hand every wave the last wave's tables.
    if (c->graph_tab_off + bytes > c->h_graph_tab_cap || bytes > c->tab_cap)
      return fail(c, BBLOCK_ERR_UNSUPPORTED, "table growth during graph capture");
    char* h = c->h_graph_tab + c->graph_tab_off;
    memcpy(h, src, bytes);
    CK(c, cudaMemcpyAsync(c->d_tab, h, bytes, cudaMemcpyHostToDevice, s));
    c->graph_tab_off += slot;
    return BBLOCK_OK;
  }
  if (c->tab_free) CK(c, cudaEventSynchronize(c->tab_free));  // previous upload has drained
  if (bytes > c->h_tab_cap) {
    if (c->h_tab) cudaFreeHost(c->h_tab);
    c->h_tab = nullptr;
    c->h_tab_cap = 0;
    if (cudaHostAlloc(&c->h_tab, bytes, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, BBLOCK_ERR_OOM, "cudaHostAlloc of %zu bytes failed", bytes);
    }
    c->h_tab_cap = bytes;
  }
  int rc = grow_device(c, &c->d_tab, &c->tab_cap, bytes);
  if (rc) return rc;
  memcpy(c->h_tab, src, bytes);
  CK(c, cudaMemcpyAsync(c->d_tab, c->h_tab, bytes, cudaMemcpyHostToDevice, s));
  CK(c, cudaEventRecord(c->tab_free, s));
  return BBLOCK_OK;
}

// Pick the slab count so that the work units fill the persistent grid evenly.
int choose_slabs(long long tiles, int grid, int X, int xc, int max_slabs) {
  const int s_hi = std::max(1, std::min(max_slabs, (X + xc - 1) / xc));
  const int s_lo = std::max(1, (int)std::min<long long>(s_hi, (4LL * grid + tiles - 1) / tiles));
  int best = s_lo;
  double best_eff = 0.0;
  for (int s = s_lo; s <= s_hi; ++s) {
    const long long units = tiles * s;
    const long long waves = (units + grid - 1) / grid;
    const double eff = (double)units / (double)(waves * grid);
    if (eff > best_eff + 1e-9) { best_eff = eff; best = s; }
    if (eff >= 0.97) break;
  }
  return best;
}

struct JobIn {
  const double2* V;
  const double2* phi[3];
  int nd[3];
  double2* B;
};

int validate_common(bblock_ctx* c, const int32_t* momenta, int n_mom, const int32_t* spin_idx,
                    const double* coeffs, int n_spin, int per_mom) {
  if (n_mom < 0) return fail(c, BBLOCK_ERR_INVALID_ARG, "n_mom = %d < 0", n_mom);
  if (n_mom > 0 && !momenta) return fail(c, BBLOCK_ERR_INVALID_ARG, "momenta is NULL");
  if (n_spin < 1 || n_spin > 64) return fail(c, BBLOCK_ERR_INVALID_ARG, "n_spin = %d outside 1..64", n_spin);
  if (!spin_idx || !coeffs) return fail(c, BBLOCK_ERR_INVALID_ARG, "spin_idx / spin_coeffs is NULL");
  if (per_mom != 0 && per_mom != 1) return fail(c, BBLOCK_ERR_INVALID_ARG, "coeff_per_mom must be 0 or 1");
  return BBLOCK_OK;
}

int validate_job(bblock_ctx* c, const JobIn& j, int idx, bool device, int n_mom = 0,
                 int n_t = 1) {
  const void* ptrs[5] = {j.V, j.phi[0], j.phi[1], j.phi[2], j.B};
  const char* names[5] = {"V", "phi1", "phi2", "phi3", "B_out"};
  for (int k = 0; k < 5; ++k) {
    if (!ptrs[k]) return fail(c, BBLOCK_ERR_INVALID_ARG, "job %d: %s is NULL", idx, names[k]);
    if (!aligned16(ptrs[k]))
      return fail(c, BBLOCK_ERR_INVALID_ARG, "job %d: %s is not 16-byte aligned", idx, names[k]);
    if (device && !is_device_ptr(c, ptrs[k]))
      return fail(c, BBLOCK_ERR_INVALID_ARG, "job %d: %s is not device memory of device %d", idx,
                  names[k], c->cfg.device);
  }
  for (int i = 0; i < 3; ++i)
    if (j.nd[i] < 1 || j.nd[i] > c->cfg.max_ndil)
      return fail(c, BBLOCK_ERR_INVALID_ARG, "job %d: nd%d = %d outside 1..max_ndil (%d)", idx,
                  i + 1, j.nd[i], c->cfg.max_ndil);
  if (device) {
    const size_t sz = sizeof(double2) * (size_t)n_t;
    const size_t ext[5] = {sz * c->cfg.n_ev * c->rows, sz * 4 * c->cfg.n_ev * j.nd[0],
                           sz * 4 * c->cfg.n_ev * j.nd[1], sz * 4 * c->cfg.n_ev * j.nd[2],
                           sz * n_mom * j.nd[0] * j.nd[1] * j.nd[2]};
    for (int k = 0; k < 5; ++k)
      if (ext[k] && !within_allocation(ptrs[k], ext[k]))
        return fail(c, BBLOCK_ERR_INVALID_ARG, "job %d: %s does not hold %zu bytes", idx,
                    names[k], ext[k]);
  }
  return BBLOCK_OK;
}

int tc_form_of(const bblock_config& cfg) {
  if (cfg.precision == BBLOCK_TF32X3) return TC_TF32_3;
  if (cfg.precision == BBLOCK_FP16X3) return TC_F16_3;
  return cfg.bf16_products == 3 ? TC_BF16_3 : cfg.bf16_products == 9 ? TC_BF16_9 : TC_BF16_6;
}

// Complex columns per tensor-core tile: the N tile that wastes the fewest padded columns,
// counting a fixed per-tile cost of 16 columns for building the shared diquark tile.
struct TcTiling {
  int cluster = 1;       // CTAs of a cluster (1: none)
  int nc = 48;           // complex (p, d3) columns per CTA
  bool share_b = false;  // cluster = 2 CTA pairs sharing the third-quark tile (FP16 form)
};

// Cluster size and N tile for jobs [b, e).
//
// N tile: the widest that fits TMEM (48 complex columns) unless fewer, narrower tiles
// cover the (p, d3) columns with less padding; every extra N tile rebuilds the 128-pair
// diquark tile, the producers' dominant cost (a tile costs ~ 128 + nc row-units).
// Cluster: no cluster unless the caller asks for one (BBLOCK_OPT_TC_CLUSTER). Measured on
// GB300, clusters that share each diquark tile do not pay robustly: with 2 CTAs the whole
// step is 2-4 % faster for the 3-piece BF16 forms at 448 columns (L = 48, 7 momenta,
// N_dil = 64), 14 % slower for the 2-piece form, and unchanged at 96 or 320 columns;
// clusters of 4 or 8 are slower, because the stage time barely falls with the diquark
// work per CTA.
//
// FP16 form: CTA pairs that share the third-quark tile unless the caller asks for no
// cluster, for index checks or for the wait-limit test hook. A pair builds 2 x 128 diquark
// rows and NC third-quark rows per stage for an N tile of up to 80 columns, so the N tile
// is the one with the least (256 + nc) x tiles over the wave's jobs.
TcTiling choose_tc_tiling(const bblock_ctx* c, const std::vector<JobIn>& jobs, size_t b,
                          size_t e, int P, int form, int nc_fixed) {
  if (form == TC_F16_3 && !c->opt_checks && c->opt_wait_us == 0 && c->opt_tc_cluster != 1) {
    TcTiling pair;
    pair.cluster = 2;
    pair.share_b = true;
    pair.nc = nc_fixed > 0 ? nc_fixed : 80;
    if (nc_fixed <= 0) {
      long long best_cost = -1;
      for (int nc = tc_max_nc(form, true); nc >= 16; nc -= 16) {
        long long cost = 0;
        for (size_t k = b; k < e; ++k) {
          const long long N = (long long)P * jobs[k].nd[2];
          const long long mp = (((long long)jobs[k].nd[0] * jobs[k].nd[1] + 127) / 128 + 1) / 2;
          cost += mp * ((N + nc - 1) / nc) * (nc + 256);
        }
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; pair.nc = nc; }
      }
    }
    return pair;
  }
  const bool can_cluster = form != TC_TF32_3 && form != TC_F16_3 && !c->opt_checks &&
                           c->opt_wait_us == 0 && c->opt_tc_cluster != 1;
  TcTiling best;
  best.nc = nc_fixed > 0 ? nc_fixed : 48;
  if (nc_fixed <= 0) {
    long long best_cost = -1;
    for (int nc = 48; nc >= 16; nc -= 16) {
      long long cost = 0;
      for (size_t k = b; k < e; ++k) {
        const long long N = (long long)P * jobs[k].nd[2];
        const long long mt = ((long long)jobs[k].nd[0] * jobs[k].nd[1] + 127) / 128;
        cost += mt * ((N + nc - 1) / nc) * (nc + 128);
      }
      if (best_cost < 0 || cost < best_cost) { best_cost = cost; best.nc = nc; }
    }
  }
  if (can_cluster && c->opt_tc_cluster > 1) best.cluster = c->opt_tc_cluster;
  return best;
}

// The row-factored phase of the FP16 form: e^{-i p.x} = w^{n0 x0} w^{n1 x1 + n2 x2}. The
// contraction's N tile holds NC = nidx * nc columns (idx0, d3) for the nidx distinct n0 of
// the momenta, and TMEM holds the chunk accumulators (4 NC columns) and a running sum per
// momentum (2 nc each). It pays when the momenta are at least twice as many as their
// distinct n0: the MMAs then cover nidx instead of P phase columns per d3.
struct RfPlan {
  bool on = false;
  int nc = 16, nidx = 0, spr = 0;
  int n0[kMaxRfIdx] = {};
  int pidx0[kMaxRfP] = {}, pn1[kMaxRfP] = {}, pn2[kMaxRfP] = {};
};

RfPlan plan_rf(const bblock_ctx* c, int n_mom, int per_mom, int form, int n_pairs, int G,
               int nc_opt) {
  RfPlan r;
  if (form != TC_F16_3 || per_mom || c->opt_checks || c->opt_wait_us || c->opt_tc_rows == 2 ||
      n_mom < 1 || n_mom > kMaxRfP || c->phase_mom.size() != (size_t)3 * n_mom)
    return r;
  const int L = c->cfg.L;
  auto md = [L](int v) { const int m = v % L; return m < 0 ? m + L : m; };
  for (int p = 0; p < n_mom; ++p) {
    const int n0 = md(c->phase_mom[3 * p]);
    int idx = -1;
    for (int k = 0; k < r.nidx; ++k)
      if (r.n0[k] == n0) idx = k;
    if (idx < 0) {
      if (r.nidx == kMaxRfIdx) return RfPlan{};
      idx = r.nidx;
      r.n0[r.nidx++] = n0;
    }
    r.pidx0[p] = idx;
    r.pn1[p] = md(c->phase_mom[3 * p + 1]);
    r.pn2[p] = md(c->phase_mom[3 * p + 2]);
  }
  if (c->opt_tc_rows == 0 && n_mom < 2 * r.nidx) return RfPlan{};
  auto fits = [&](int nc) {
    // B rows (idx0, d3) are built by the plain kernel's third-quark producers: <= 48
    return nc >= 16 && nc % 16 == 0 && r.nidx * nc <= tc_max_nc(form, false) &&
           4 * r.nidx * nc + 2 * n_mom * nc <= 512;
  };
  if (nc_opt > 0) {
    if (!fits(nc_opt)) return RfPlan{};
    r.nc = nc_opt;
  } else {
    r.nc = 0;
    for (int nc = 48; nc >= 16 && !r.nc; nc -= 16)
      if (fits(nc)) r.nc = nc;
    if (!r.nc) return RfPlan{};
  }
  r.spr = (L * n_pairs + G - 1) / G;
  r.on = true;
  return r;
}

// Tensor-core forms: FP32 projection, tcgen05 contraction, FP64 slab reduction.
int run_jobs_tc(bblock_ctx* c, const std::vector<JobIn>& jobs, const SpinPlan& sp, int n_mom,
                int per_mom, cudaStream_t s) {
  const int X = c->X, rows = c->rows, n_ev = c->cfg.n_ev;
  const int form = tc_form_of(c->cfg);
  const int G = tc_groups_per_stage(form);
  // 12 leading accumulations between drains by default
  const int chunk_stages = c->opt_tc_chunk > 0 ? c->opt_tc_chunk : 2;
  const int n3_fields = sp.n_pairs * sp.n_coef_sets;
  const int P_launch = per_mom ? 1 : n_mom;
  const int grid_cap = c->num_sms;            // one CTA per SM (all of TMEM, ~200 KB smem)
  // at most 256 drains into the FP32 running sum per work unit
  const long long max_groups_per_unit = 256LL * chunk_stages * G;
  const int min_slabs = (int)std::min<long long>(
      X, ((long long)X * sp.n_pairs + max_groups_per_unit - 1) / max_groups_per_unit);
  const int max_slabs = std::max(64, min_slabs);
  // the row-factored phase (FP16 form): slabs are ranges of lattice rows, each unit drains
  // at most 256 times
  const int L = c->cfg.L, n_rows = L * L;
  const RfPlan rp = plan_rf(c, n_mom, per_mom, form, sp.n_pairs, G, c->opt_tc_nc);
  const int rf_cpr = rp.on ? (rp.spr + chunk_stages - 1) / chunk_stages : 1;
  const int rf_min_slabs = rp.on ? (n_rows + std::max(1, 256 / rf_cpr) - 1) / std::max(1, 256 / rf_cpr) : 1;
  // checks option: a canary after the converted inputs and every field and partial block
  const size_t canary_bytes = c->opt_checks ? (size_t)(sp.n1 + sp.n2 + n3_fields + 2) * kCanaryBytes : 0;
  // the tiled tensor-core projection (the default): V and the folded phi as BF16 piece tiles,
  // V once per distinct V of a wave
  const bool tiled = !c->opt_checks && c->opt_tc_proj == 0;
  auto phi_tile_bytes = [&](const JobIn& j) -> size_t {
    return align_up(sp.n1 * tiled_phi_bytes(j.nd[0], tiled_ncp(j.nd[0]), n_ev) +
                        sp.n2 * tiled_phi_bytes(j.nd[1], tiled_ncp(j.nd[1]), n_ev) +
                        n3_fields * tiled_phi_bytes(j.nd[2], tiled_ncp(j.nd[2]), n_ev),
                    256);
  };
  // FP32 copies of a job's inputs (V and the three phi_i), converted once per call; tiled:
  // the fields' phi tiles (the V tiles, one set per distinct V, precede the jobs)
  const size_t v_tile_bytes = align_up(tiled_v_bytes(rows, n_ev), 256);
  auto in_bytes = [&](const JobIn& j) -> size_t {
    if (tiled) return phi_tile_bytes(j);
    return align_up((size_t)rows * n_ev * sizeof(float2), 256) +
           align_up((size_t)4 * n_ev * (j.nd[0] + j.nd[1] + j.nd[2]) * sizeof(float2), 256);
  };
  auto job_bytes = [&](const JobIn& j, int n_slab) {
    size_t f = (size_t)rows * (sp.n1 * j.nd[0] + sp.n2 * j.nd[1] + n3_fields * j.nd[2]) * sizeof(float2);
    size_t p = (size_t)n_slab * P_launch * j.nd[0] * j.nd[1] * j.nd[2] * sizeof(float2);
    return in_bytes(j) + align_up(f, 256) + align_up(p, 256) + canary_bytes;
  };
  size_t job_idx = 0;
  int rc;
  while (job_idx < jobs.size()) {
    size_t end = job_idx, need = 0;
    std::vector<const double2*> wave_vs;   // tiled projection: the wave's distinct V
    while (end < jobs.size()) {
      size_t b = job_bytes(jobs[end], max_slabs);
      const bool new_v = tiled && std::find(wave_vs.begin(), wave_vs.end(), jobs[end].V) == wave_vs.end();
      if (new_v) b += v_tile_bytes;
      if (end > job_idx && need + b > wave_budget(c)) break;
      need += b;
      if (new_v) wave_vs.push_back(jobs[end].V);
      ++end;
    }
    ++c->last_waves;
    const int nj = (int)(end - job_idx);
    TcTiling tt = choose_tc_tiling(c, jobs, job_idx, end, P_launch, form, c->opt_tc_nc);
    if (rp.on) {   // row-factored: B rows (idx0, d3); plain CTAs or clusters of 2 that share
                   // each diquark tile and take adjacent d3 tiles (by default when every job
                   // of the wave has at least two d3 tiles: 6 % faster on the batched
                   // L = 32 workload, where the diquark tiles are the producers' largest cost)
      bool two = true;
      for (size_t k = job_idx; k < end; ++k) two = two && jobs[k].nd[2] > rp.nc;
      tt.cluster = (c->opt_tc_cluster == 2 || (c->opt_tc_cluster == 0 && two)) ? 2 : 1;
      tt.share_b = false;
      tt.nc = rp.nidx * rp.nc;
    }
    const int NC = tt.nc, CL = tt.cluster;
    if (NC > tc_max_nc(form, tt.share_b))
      return fail(c, BBLOCK_ERR_INVALID_ARG, "N tile of %d columns exceeds this form's %d", NC,
                  tc_max_nc(form, tt.share_b));
    // M tiles of 128 (d1, d2) pairs per unit (two adjacent ones for CTA pairs) and N tiles
    // per unit (CL adjacent ones for clusters sharing the diquark tile)
    auto unit_m_tiles = [&](const JobIn& j) -> long long {
      const long long mt = ((long long)j.nd[0] * j.nd[1] + 127) / 128;
      return tt.share_b ? (mt + 1) / 2 : mt;
    };
    const int n_group = tt.share_b ? NC : CL * NC;
    // N tiles of a job: groups of (p, d3) columns, or (row-factored) of d3 columns
    auto unit_n_tiles = [&](const JobIn& j) -> long long {
      if (rp.on) return ((j.nd[2] + rp.nc - 1) / rp.nc + CL - 1) / CL;
      return ((long long)P_launch * j.nd[2] + n_group - 1) / n_group;
    };
    long long tiles = 0, max_elems = 0;
    int max_ndf = 0;
    for (size_t k = job_idx; k < end; ++k) {
      const JobIn& j = jobs[k];
      tiles += unit_m_tiles(j) * unit_n_tiles(j);
      for (int i = 0; i < 3; ++i) max_ndf = std::max(max_ndf, j.nd[i]);
      max_elems = std::max(max_elems, (long long)P_launch * j.nd[0] * j.nd[1] * j.nd[2]);
    }
    int n_slab, sites_per_slab, rows_per_slab = 0;
    if (rp.on) {
      n_slab = c->opt_slabs > 0 ? std::max(rf_min_slabs, std::min(c->opt_slabs, n_rows))
                                : std::max(rf_min_slabs, choose_slabs(tiles, grid_cap / CL, n_rows, 1, max_slabs));
      rows_per_slab = (n_rows + n_slab - 1) / n_slab;
      n_slab = (n_rows + rows_per_slab - 1) / rows_per_slab;
      sites_per_slab = rows_per_slab * L;
    } else {
      n_slab = c->opt_slabs > 0 ? std::max(min_slabs, std::min(c->opt_slabs, X))
                                : std::max(min_slabs, choose_slabs(tiles, grid_cap / CL, X, 1, max_slabs));
      sites_per_slab = (X + n_slab - 1) / n_slab;
      n_slab = (X + sites_per_slab - 1) / sites_per_slab;
    }
    // FP16 form: three per-line maxima per job (the operand scales), at the wave's start
    const bool amax_on = tc_form_needs_amax(form);
    const size_t amax_bytes = amax_on ? align_up((size_t)3 * nj * sizeof(uint32_t), 256) : 0;
    const size_t vt_bytes = wave_vs.size() * v_tile_bytes;
    size_t ws_need = amax_bytes + vt_bytes;
    for (size_t k = job_idx; k < end; ++k) ws_need += job_bytes(jobs[k], n_slab);
    rc = grow_device(c, &c->d_ws, &c->ws_cap, ws_need);
    if (rc) return rc;
    uint32_t* d_amax = amax_on ? reinterpret_cast<uint32_t*>(c->d_ws) : nullptr;

    std::vector<ProjFieldF> fields;
    std::vector<std::vector<TcJob>> tjobs(sp.n_coef_sets, std::vector<TcJob>(nj));
    std::vector<uint32_t*> canaries;
    std::vector<F32ConvSeg> segs;
    long long max_seg = 0;
    char* ws = c->d_ws + amax_bytes + vt_bytes;
    long long unit = 0;
    // tiled projection: the distinct V of the wave (tiles after the maxima) and every field's
    // phi tiles
    std::vector<TileV> tvs;
    for (size_t q = 0; q < wave_vs.size(); ++q)
      tvs.push_back(TileV{wave_vs[q], reinterpret_cast<uint16_t*>(c->d_ws + amax_bytes + q * v_tile_bytes)});
    std::vector<TiledField> tfields;
    std::vector<int> tfield_v;
    for (int k = 0; k < nj; ++k) {
      const JobIn& j = jobs[job_idx + k];
      char* base = ws;
      auto canary = [&](char*& at) {
        if (!c->opt_checks) return;
        canaries.push_back(reinterpret_cast<uint32_t*>(at));
        at += kCanaryBytes;
      };
      const float2* Vf = nullptr;
      const float2* phif[3] = {};
      char* phi_tiles = nullptr;
      int vidx = -1;
      if (tiled) {
        for (size_t q = 0; q < tvs.size(); ++q)
          if (tvs[q].V == j.V) vidx = (int)q;
        if (vidx < 0) return fail(c, BBLOCK_ERR_INVALID_ARG, "internal: V of a job not in its wave");
        phi_tiles = base;
      } else {
        // the job's inputs in FP32: V, then phi_1..3 packed
        Vf = reinterpret_cast<const float2*>(base);
        segs.push_back(F32ConvSeg{j.V, reinterpret_cast<float2*>(base), (long long)rows * n_ev});
        max_seg = std::max(max_seg, (long long)rows * n_ev);
        char* pb = base + align_up((size_t)rows * n_ev * sizeof(float2), 256);
        for (int i = 0; i < 3; ++i) {
          phif[i] = reinterpret_cast<const float2*>(pb);
          const long long n = 4LL * n_ev * j.nd[i];
          segs.push_back(F32ConvSeg{j.phi[i], reinterpret_cast<float2*>(pb), n});
          max_seg = std::max(max_seg, n);
          pb += (size_t)n * sizeof(float2);
        }
      }
      base += in_bytes(j);
      canary(base);
      auto add_field = [&](const float2* phi, int nd, int n_terms, const int* offs,
                           const double2* w, int line) -> float2* {
        ProjFieldF f{};
        f.V = Vf;
        f.phi = phi;
        f.q = reinterpret_cast<float2*>(base);
        f.amax = d_amax ? d_amax + 3 * k + line : nullptr;
        f.nd = nd;
        f.n_terms = n_terms;
        for (int t = 0; t < n_terms; ++t) { f.row_off[t] = offs[t]; f.w[t] = w[t]; }
        if (tiled) {
          TiledField tf{};
          tf.phi = j.phi[line];
          for (int t = 0; t < n_terms; ++t) { tf.row_off[t] = offs[t]; tf.w[t] = w[t]; }
          tf.n_terms = n_terms;
          tf.nd = nd;
          tf.ncp = tiled_ncp(nd);
          tf.n_tiles = (nd + tf.ncp - 1) / tf.ncp;
          tf.btiles = reinterpret_cast<uint16_t*>(phi_tiles);
          phi_tiles += tiled_phi_bytes(nd, tf.ncp, n_ev);
          tf.q = f.q;
          tf.amax = f.amax;
          tfields.push_back(tf);
          tfield_v.push_back(vidx);
        }
        base += (size_t)rows * nd * sizeof(float2);
        canary(base);
        fields.push_back(f);
        return f.q;
      };
      const double2 one = make_double2(1.0, 0.0);
      const float2* q1[4] = {};
      const float2* q2[4] = {};
      for (int sl = 0; sl < sp.n1; ++sl) {
        int off = sp.alpha_of1[sl] * n_ev;
        q1[sl] = add_field(phif[0], j.nd[0], 1, &off, &one, 0);
      }
      for (int sl = 0; sl < sp.n2; ++sl) {
        int off = sp.beta_of2[sl] * n_ev;
        q2[sl] = add_field(phif[1], j.nd[1], 1, &off, &one, 1);
      }
      std::vector<std::vector<const float2*>> q3(sp.n_coef_sets, std::vector<const float2*>(sp.n_pairs));
      for (int set = 0; set < sp.n_coef_sets; ++set)
        for (int pr = 0; pr < sp.n_pairs; ++pr) {
          const auto& tlist = sp.terms[set][pr];
          if ((int)tlist.size() > kMaxTerms) return fail(c, BBLOCK_ERR_UNSUPPORTED, "too many terms");
          int offs[kMaxTerms];
          double2 w[kMaxTerms];
          for (size_t t = 0; t < tlist.size(); ++t) { offs[t] = tlist[t].first * n_ev; w[t] = tlist[t].second; }
          q3[set][pr] = add_field(phif[2], j.nd[2], (int)tlist.size(), offs, w, 2);
        }
      base = c->d_ws + align_up((size_t)(base - c->d_ws), 256);
      float2* partial = reinterpret_cast<float2*>(base);
      base += align_up((size_t)n_slab * P_launch * j.nd[0] * j.nd[1] * j.nd[2] * sizeof(float2), 256);
      canary(base);
      ws = base;
      const int m_tiles = (int)unit_m_tiles(j);                       // (d1, d2) pairs
      // groups of CL N tiles of NC (p, d3) columns: a cluster unit covers one group
      const int n_tiles = (int)unit_n_tiles(j);
      for (int set = 0; set < sp.n_coef_sets; ++set) {
        TcJob& tj = tjobs[set][k];
        for (int i = 0; i < 4; ++i) { tj.q1[i] = q1[i]; tj.q2[i] = q2[i]; }
        for (int pr = 0; pr < sp.n_pairs; ++pr) tj.q3[pr] = q3[set][pr];
        tj.amax = d_amax ? d_amax + 3 * k : nullptr;
        tj.partial = partial;
        // per-momentum coefficient sets run one momentum per launch into their slice of B
        tj.B = j.B + (per_mom ? (size_t)set * j.nd[0] * j.nd[1] * j.nd[2] : 0);
        tj.nd1 = j.nd[0]; tj.nd2 = j.nd[1]; tj.nd3 = j.nd[2];
        tj.m_tiles = m_tiles;
        tj.n_tiles = n_tiles;
        tj.unit_begin = unit;
      }
      unit += (long long)m_tiles * n_tiles * n_slab;
    }
    // every field and partial block the kernels will touch lies inside the workspace
    for (const ProjFieldF& f : fields)
      if (!within_workspace(c, f.q, (size_t)rows * f.nd * sizeof(float2)))
        return fail(c, BBLOCK_ERR_INVALID_ARG, "internal: field outside the workspace");
    for (int k = 0; k < nj; ++k) {
      const TcJob& tj = tjobs[0][k];
      if (!within_workspace(c, tj.partial, (size_t)n_slab * P_launch * tj.nd1 * tj.nd2 * tj.nd3 * sizeof(float2)))
        return fail(c, BBLOCK_ERR_INVALID_ARG, "internal: partial block outside the workspace");
    }
    for (uint32_t* cn : canaries)
      if (!within_workspace(c, cn, kCanaryBytes))
        return fail(c, BBLOCK_ERR_INVALID_ARG, "internal: canary outside the workspace");
    for (const F32ConvSeg& g : segs)
      if (!within_workspace(c, g.dst, (size_t)g.n * sizeof(float2)))
        return fail(c, BBLOCK_ERR_INVALID_ARG, "internal: converted input outside the workspace");
    const size_t fbytes = align_up(fields.size() * sizeof(ProjFieldF), 256);
    const size_t jbytes = align_up((size_t)nj * sizeof(TcJob), 256);
    const size_t sofs = fbytes + jbytes * sp.n_coef_sets;
    const size_t cofs = sofs + align_up(segs.size() * sizeof(F32ConvSeg), 256);
    // row-factored: w^k = e^{-2 pi i k / L}, k = 0..L-1, in FP64 rounded to FP32
    const size_t wofs = align_up(cofs + canaries.size() * sizeof(uint32_t*), 256);
    // tiled projection: the field tiles grouped by V (units: 128-row tile outermost within a
    // group, so the CTAs running at once share their V tiles in L2)
    std::vector<FieldTile> tfts;
    std::vector<PGroup> tgroups;
    TiledProjParams tpp{};
    if (tiled) {
      tpp.rows = rows;
      tpp.n_ev = n_ev;
      tpp.k_stages = (n_ev + 31) / 32;
      tpp.m_tiles = (rows + 127) / 128;
      long long ub = 0;
      for (int v = 0; v < (int)tvs.size(); ++v) {
        PGroup g{ub, (int)tfts.size(), 0, v};
        for (size_t f = 0; f < tfields.size(); ++f)
          if (tfield_v[f] == v)
            for (int nt = 0; nt < tfields[f].n_tiles; ++nt) tfts.push_back(FieldTile{(int)f, nt});
        g.ft_count = (int)tfts.size() - g.ft_first;
        if (g.ft_count == 0) continue;
        ub += (long long)tpp.m_tiles * g.ft_count;
        tgroups.push_back(g);
      }
      tpp.n_groups = (int)tgroups.size();
      tpp.total_units = ub;
    }
    const size_t tofs = align_up(wofs + (rp.on ? (size_t)L * sizeof(float2) : 0), 256);
    const size_t tv_ofs = tofs;
    const size_t tf_ofs = align_up(tv_ofs + tvs.size() * sizeof(TileV), 256);
    const size_t tft_ofs = align_up(tf_ofs + tfields.size() * sizeof(TiledField), 256);
    const size_t tg_ofs = align_up(tft_ofs + tfts.size() * sizeof(FieldTile), 256);
    std::vector<char> tab(tiled ? tg_ofs + tgroups.size() * sizeof(PGroup)
                                : wofs + (rp.on ? (size_t)L * sizeof(float2) : 0));
    if (tiled) {
      memcpy(tab.data() + tv_ofs, tvs.data(), tvs.size() * sizeof(TileV));
      memcpy(tab.data() + tf_ofs, tfields.data(), tfields.size() * sizeof(TiledField));
      memcpy(tab.data() + tft_ofs, tfts.data(), tfts.size() * sizeof(FieldTile));
      memcpy(tab.data() + tg_ofs, tgroups.data(), tgroups.size() * sizeof(PGroup));
    }
    if (rp.on) {
      float2* om = reinterpret_cast<float2*>(tab.data() + wofs);
      const double two_pi = 6.283185307179586476925286766559;
      for (int k = 0; k < L; ++k)
        om[k] = make_float2((float)std::cos(two_pi * k / L), (float)-std::sin(two_pi * k / L));
    }
    memcpy(tab.data(), fields.data(), fields.size() * sizeof(ProjFieldF));
    for (int set = 0; set < sp.n_coef_sets; ++set)
      memcpy(tab.data() + fbytes + jbytes * set, tjobs[set].data(), (size_t)nj * sizeof(TcJob));
    memcpy(tab.data() + sofs, segs.data(), segs.size() * sizeof(F32ConvSeg));
    if (!canaries.empty()) memcpy(tab.data() + cofs, canaries.data(), canaries.size() * sizeof(uint32_t*));
    rc = upload_tables(c, tab.data(), tab.size(), s);
    if (rc) return rc;
    const ProjFieldF* d_fields = reinterpret_cast<const ProjFieldF*>(c->d_tab);
    uint32_t* const* d_canaries = reinterpret_cast<uint32_t* const*>(c->d_tab + cofs);
    if (!canaries.empty()) {
      CK(c, timed_launch(c, K_CANARY, s, [&] {
        return launch_canaries(d_canaries, (int)canaries.size(), false, c->d_status, s);
      }));
      if (c->opt_corrupt_canary && !c->capturing) {   // test hook: a simulated overrun
        c->opt_corrupt_canary = 0;
        CK(c, cudaMemsetAsync(canaries[0], 0x5a, 4, s));
      }
    }
    if (!tiled)
      CK(c, timed_launch(c, K_CONVERT, s, [&] {
        return launch_convert_f32(reinterpret_cast<const F32ConvSeg*>(c->d_tab + sofs),
                                  (int)segs.size(), max_seg, s);
      }));
    if (amax_on) CK(c, cudaMemsetAsync(d_amax, 0, (size_t)3 * nj * sizeof(uint32_t), s));
    if (tiled) {
      // Eq. 2 on the tensor cores from pre-tiled BF16 pieces (it also writes the FP16 form's
      // field maxima)
      tpp.vs = reinterpret_cast<const TileV*>(c->d_tab + tv_ofs);
      tpp.fields = reinterpret_cast<const TiledField*>(c->d_tab + tf_ofs);
      tpp.fts = reinterpret_cast<const FieldTile*>(c->d_tab + tft_ofs);
      tpp.groups = reinterpret_cast<const PGroup*>(c->d_tab + tg_ofs);
      tpp.status = c->d_status;
      tpp.wait_limit = c->opt_wait_us > 0 ? (long long)c->opt_wait_us * c->cycles_per_us
                                          : 4000000000LL;
      const int pgrid = (int)std::min<long long>(tpp.total_units, c->num_sms);
      CK(c, timed_launch(c, K_PROJECT, s, [&] {
        return launch_project_tiled(tpp, (int)tvs.size(), (int)tfts.size(), pgrid, s);
      }));
    } else if (c->opt_checks || c->opt_tc_proj == 2 || amax_on) {
      // the FP32 projection: the checked variant (it checks every index), on request, and for
      // the FP16 form when the per-stage projection is asked for (it takes its operand scales
      // from the FP32 projection's field maxima)
      // the FP32 projection (the default, and the checked variant: it checks every index)
      CK(c, timed_launch(c, K_PROJECT, s, [&] {
        return launch_project_f32(d_fields, (int)fields.size(), rows, n_ev, max_ndf,
                                  c->opt_checks, c->d_dbg, c->d_status, s);
      }));
    } else {
      // Eq. 2 on the tensor cores in the form's split, drained every stage; the N tile
      // with the fewest tiles over the fields (the narrower one on a tie)
      TcParams pp{};
      int best_tiles = 0;
      for (int nc = 16; nc <= 48; nc += 16) {   // the N tiles the kernel accepts
        int t = 0;
        for (const ProjFieldF& f : fields) t = std::max(t, (f.nd + nc - 1) / nc);
        if (best_tiles == 0 || t < best_tiles) { best_tiles = t; pp.NC = nc; }
      }
      pp.pfields = d_fields;
      pp.p_n_fields = (int)fields.size();
      pp.p_rows = rows;
      pp.p_n_ev = n_ev;
      pp.p_m_tiles = (rows + 127) / 128;
      pp.p_n_tiles = best_tiles;
      pp.total_units = (long long)fields.size() * pp.p_m_tiles * pp.p_n_tiles;
      pp.chunk_stages = 1;
      pp.status = c->d_status;
      pp.dbg = c->d_dbg;
      pp.wait_limit = c->opt_wait_us > 0 ? (long long)c->opt_wait_us * c->cycles_per_us
                                         : 4000000000LL;
      const int pgrid = (int)std::min<long long>(pp.total_units, c->num_sms);
      CK(c, timed_launch(c, K_PROJECT, s, [&] { return launch_project_tc(pp, form, pgrid, s); }));
    }
    TcParams prm{};
    prm.n_jobs = nj;
    prm.total_units = unit;
    prm.X = X;
    prm.n_slab = n_slab;
    prm.sites_per_slab = sites_per_slab;
    prm.n_pairs = sp.n_pairs;
    for (int pr = 0; pr < sp.n_pairs; ++pr) { prm.a_slot[pr] = sp.a_slot[pr]; prm.b_slot[pr] = sp.b_slot[pr]; }
    prm.P = P_launch;
    prm.NC = NC;
    prm.share_b = tt.share_b ? 1 : 0;
    prm.chunk_stages = chunk_stages;
    c->last_path = rp.on ? (CL > 1 ? BBLOCK_PATH_TC_ROWS_CLUSTER : BBLOCK_PATH_TC_ROWS)
                         : tt.share_b ? BBLOCK_PATH_TC_PAIRS
                                      : CL > 1 ? BBLOCK_PATH_TC_CLUSTER : BBLOCK_PATH_TC;
    if (rp.on) {
      prm.rf = 1;
      prm.L = L;
      prm.rf_spr = rp.spr;
      prm.rf_rows_per_slab = rows_per_slab;
      prm.rf_nc = rp.nc;
      prm.rf_nidx = rp.nidx;
      for (int k = 0; k < rp.nidx; ++k) prm.rf_n0[k] = rp.n0[k];
      for (int p = 0; p < n_mom; ++p) {
        prm.rf_pidx0[p] = rp.pidx0[p];
        prm.rf_pn1[p] = rp.pn1[p];
        prm.rf_pn2[p] = rp.pn2[p];
      }
      prm.rf_omega = reinterpret_cast<const float2*>(c->d_tab + wofs);
    }
    prm.status = c->d_status;
    prm.checks = c->opt_checks;
    prm.dbg = c->d_dbg;
    prm.wait_limit = c->opt_wait_us > 0 ? (long long)c->opt_wait_us * c->cycles_per_us
                                        : 4000000000LL;
    // CTAs wanted: CL per cluster unit, at most one per SM (the launch caps it further at
    // the clusters that can be resident at once)
    const int grid = (int)std::min<long long>(unit * CL, grid_cap / CL * CL);
    for (int set = 0; set < sp.n_coef_sets; ++set) {
      const TcJob* d_jobs = reinterpret_cast<const TcJob*>(c->d_tab + fbytes + jbytes * set);
      prm.jobs = d_jobs;
      prm.phase = c->d_phase_f + (per_mom ? (size_t)set * X : 0);
      CK(c, timed_launch(c, K_CONTRACT, s, [&] { return launch_contract_tc(prm, form, CL, grid, s); }));
      CK(c, timed_launch(c, K_REDUCE, s, [&] {
        return launch_reduce_slabs_f32(d_jobs, nj, n_slab, P_launch, max_elems, c->opt_checks,
                                       c->d_dbg, c->d_status, s);
      }));
    }
    if (!canaries.empty())
      CK(c, timed_launch(c, K_CANARY, s, [&] {
        return launch_canaries(d_canaries, (int)canaries.size(), true, c->d_status, s);
      }));
    job_idx = end;
  }
  return BBLOCK_OK;
}

// The whole launch sequence for a list of jobs sharing momenta and spin operator.
// Ozaki form: clusters of C CTAs share each diquark tile across C adjacent N tiles; each
// builds 1/C of the tile's rows, with shorter per-thread chains, which sets the stage time.
// Measured on GB300 (L = 32, 9 momenta, N_dil 32-64): pairs are the fastest, 1.6x the plain
// CTA; clusters of 3 and 4 are 10 % and 3 % slower than pairs (fewer resident CTAs: 138 and
// 144 of 152 SMs, and N tiles padded to a multiple of C). Auto: pairs unless their ragged
// last clusters pad the N tiles by more than 20 %.
int oz_cluster_for(const bblock_ctx* c, const std::vector<JobIn>& jobs, size_t b, size_t e,
                   int P_launch, int nc) {
  if (c->opt_tc_cluster >= 1 && c->opt_tc_cluster <= 4) return c->opt_tc_cluster;
  long long tiles = 0, padded = 0;
  for (size_t k = b; k < e; ++k) {
    const long long nt = ((long long)P_launch * jobs[k].nd[2] + nc - 1) / nc;
    const long long mt = ((long long)jobs[k].nd[0] * jobs[k].nd[1] + kOzM - 1) / kOzM;
    tiles += mt * nt;
    padded += mt * ((nt + 1) / 2) * 2;
  }
  return tiles > 0 && (double)(padded - tiles) / tiles <= 0.2 ? 2 : 1;
}

int run_jobs(bblock_ctx* c, const std::vector<JobIn>& jobs, const int32_t* momenta, int n_mom,
             const int32_t* spin_idx, const double* coeffs, int n_spin, int per_mom,
             cudaStream_t s) {
  c->last_launches = 0;
  c->last_waves = 0;
  c->last_path = c->cfg.precision == BBLOCK_OZAKI ? BBLOCK_PATH_OZAKI
                 : fp64_like(c->cfg)               ? BBLOCK_PATH_FP64
                                                   : -1;
  c->last_stream = s;
  c->call_tab_bytes = 0;
  if (jobs.empty() || n_mom == 0) return BBLOCK_OK;
  CK(c, cudaSetDevice(c->cfg.device));
  SpinPlan sp;
  int rc = plan_spins(c, spin_idx, coeffs, n_spin, per_mom, n_mom, &sp);
  if (rc) return rc;
  if (sp.n_pairs > kMaxPairs) return fail(c, BBLOCK_ERR_UNSUPPORTED, "more than %d spin pairs", kMaxPairs);
  rc = ensure_phase(c, momenta, n_mom, s);
  if (rc) return rc;
  if (!fp64_like(c->cfg)) return run_jobs_tc(c, jobs, sp, n_mom, per_mom, s);
  // the Ozaki form runs on the double-float form's converted inputs and fields
  const bool oz = c->cfg.precision == BBLOCK_OZAKI;
  const bool df = c->cfg.precision == BBLOCK_DF64 || oz;

  const int X = c->X, rows = c->rows, n_ev = c->cfg.n_ev;
  const int n3_fields = sp.n_pairs * sp.n_coef_sets;
  // momenta per contraction launch: the Ozaki form takes them all as N columns
  const int P_launch = per_mom ? 1
                       : oz    ? n_mom
                               : p_group_size(n_mom, c->cfg.precision == BBLOCK_DF64 ? kMaxPGroupDf
                                                                                     : kMaxPGroup);
  const int xc = oz ? 1 : fp64_sites_per_chunk(sp.n_pairs);
  const Fp64Tile tl = fp64_tile_for(oz ? 1 : P_launch);  // one tile shape for every momentum group
  // Ozaki form: units run one per CTA (clusters: one per cluster of oz_cl CTAs)
  const int ctas = oz ? c->num_sms : fp64_contract_ctas_per_sm(P_launch, tl.rn, sp.n_pairs) * c->num_sms;
  const int max_slabs = 64;
  const int oz_nc = c->opt_tc_nc > 0 && c->opt_tc_nc <= kOzMaxNC ? c->opt_tc_nc : kOzMaxNC;
  int oz_cl = 1;   // Ozaki form: CTAs per cluster of the current wave
  // M tiles and N tiles (Ozaki form: clusters of oz_cl N tiles) of a job's contraction
  auto job_tiles = [&](const JobIn& j, int& mt, int& nt) {
    if (oz) {
      mt = (j.nd[0] * j.nd[1] + kOzM - 1) / kOzM;
      nt = ((P_launch * j.nd[2] + oz_nc - 1) / oz_nc + oz_cl - 1) / oz_cl;
    } else {
      mt = (j.nd[0] * j.nd[1] + 16 * tl.rm - 1) / (16 * tl.rm);
      nt = (j.nd[2] + 16 * tl.rn - 1) / (16 * tl.rn);
    }
  };
  // Ozaki form: the column and row maxima of every job, [n_slab][nd1 + nd2 + nd3] and
  // [n_slab][nd1 nd2] floats
  auto oz_bytes = [&](const JobIn& j, int n_slab) -> size_t {
    return oz ? align_up((size_t)n_slab * (j.nd[0] + j.nd[1] + j.nd[2] + j.nd[0] * j.nd[1]) *
                             sizeof(float), 256)
              : 0;
  };

  // double-float inputs of a job: V and the three phi_i as float4 planes
  auto df_in_bytes = [&](const JobIn& j) -> size_t {
    if (!df) return 0;
    return align_up((size_t)rows * n_ev * sizeof(float4), 256) +
           align_up((size_t)4 * n_ev * (j.nd[0] + j.nd[1] + j.nd[2]) * sizeof(float4), 256);
  };
  // checks option: a canary after every field, the partial block and the converted inputs
  const size_t canary_bytes =
      c->opt_checks ? (size_t)(sp.n1 + sp.n2 + n3_fields + 1 + (df ? 1 : 0)) * kCanaryBytes : 0;
  // bytes per job: fields + partials at the largest slab count (+ double-float inputs)
  auto job_bytes = [&](const JobIn& j, int n_slab) {
    size_t f = (size_t)rows * (sp.n1 * j.nd[0] + sp.n2 * j.nd[1] + n3_fields * j.nd[2]) * sizeof(double2);
    size_t p = (size_t)n_slab * n_mom * j.nd[0] * j.nd[1] * j.nd[2] * sizeof(double2);
    return align_up(f, 256) + align_up(p, 256) + df_in_bytes(j) + canary_bytes + oz_bytes(j, n_slab);
  };

  size_t job_idx = 0;
  while (job_idx < jobs.size()) {
    // wave of jobs whose workspace fits the budget
    size_t end = job_idx, need = 0;
    while (end < jobs.size()) {
      size_t b = job_bytes(jobs[end], max_slabs);
      if (end > job_idx && need + b > wave_budget(c)) break;
      need += b;
      ++end;
    }
    ++c->last_waves;
    const int nj = (int)(end - job_idx);
    if (oz) oz_cl = oz_cluster_for(c, jobs, job_idx, end, P_launch, oz_nc);
    long long tiles = 0;
    int max_nd3 = 0, max_ndf = 0;
    long long max_elems = 0;
    for (size_t k = job_idx; k < end; ++k) {
      const JobIn& j = jobs[k];
      int mt, nt;
      job_tiles(j, mt, nt);
      tiles += (long long)mt * nt;
      max_nd3 = std::max(max_nd3, j.nd[2]);
      for (int i = 0; i < 3; ++i) max_ndf = std::max(max_ndf, j.nd[i]);
      max_elems = std::max(max_elems, (long long)n_mom * j.nd[0] * j.nd[1] * j.nd[2]);
    }
    const int unit_slots = oz ? ctas / oz_cl : ctas;
    int n_slab = c->opt_slabs > 0 ? std::min(c->opt_slabs, (X + xc - 1) / xc)
                                   : choose_slabs(tiles, unit_slots, X, xc, max_slabs);
    int sites_per_slab = (X + n_slab - 1) / n_slab;
    sites_per_slab = (sites_per_slab + xc - 1) / xc * xc;
    n_slab = (X + sites_per_slab - 1) / sites_per_slab;

    size_t ws_need = 0, oz_need = 0;
    for (size_t k = job_idx; k < end; ++k) {
      ws_need += job_bytes(jobs[k], n_slab);
      oz_need += oz_bytes(jobs[k], n_slab);
    }
    rc = grow_device(c, &c->d_ws, &c->ws_cap, ws_need);
    if (rc) return rc;
    // Ozaki form: every job's column maxima in one block at the end (one memset)
    char* oz_base = c->d_ws + (ws_need - oz_need);
    std::vector<OzMaxSeg> ozsegs;

    // field and job tables
    std::vector<ProjField> fields;
    std::vector<std::vector<ContractJob>> cjobs(sp.n_coef_sets, std::vector<ContractJob>(nj));
    std::vector<DfConvSeg> segs;
    std::vector<uint32_t*> canaries;
    long long max_seg = 0;
    char* ws = c->d_ws;
    long long unit = 0;
    for (int k = 0; k < nj; ++k) {
      const JobIn& j = jobs[job_idx + k];
      char* base = ws;
      auto canary = [&](char*& at) {
        if (!c->opt_checks) return;
        canaries.push_back(reinterpret_cast<uint32_t*>(at));
        at += kCanaryBytes;
      };
      // double-float form: the job's inputs are converted to float4 planes first
      const double2* Vin = j.V;
      const double2* phin[3] = {j.phi[0], j.phi[1], j.phi[2]};
      if (df) {
        char* dbase = base;
        auto add_seg = [&](const double2* src, long long n) -> const double2* {
          float4* dst = reinterpret_cast<float4*>(dbase);
          segs.push_back(DfConvSeg{src, dst, n});
          max_seg = std::max(max_seg, n);
          dbase += align_up((size_t)n * sizeof(float4), 256);
          return reinterpret_cast<const double2*>(dst);
        };
        Vin = add_seg(j.V, (long long)rows * n_ev);
        char* phi_base = dbase;
        for (int i = 0; i < 3; ++i) {
          phin[i] = reinterpret_cast<const double2*>(phi_base);
          segs.push_back(DfConvSeg{j.phi[i], reinterpret_cast<float4*>(phi_base), 4LL * n_ev * j.nd[i]});
          max_seg = std::max(max_seg, 4LL * n_ev * j.nd[i]);
          phi_base += (size_t)4 * n_ev * j.nd[i] * sizeof(float4);
        }
        base += df_in_bytes(j);
        canary(base);
      }
      auto add_field = [&](const double2* phi, int nd, int n_terms, const int* offs,
                           const double2* w) -> double2* {
        ProjField f{};
        f.V = Vin;
        f.phi = phi;
        f.q = reinterpret_cast<double2*>(base);
        f.nd = nd;
        f.n_terms = n_terms;
        for (int t = 0; t < n_terms; ++t) { f.row_off[t] = offs[t]; f.w[t] = w[t]; }
        base += (size_t)rows * nd * sizeof(double2);
        canary(base);
        fields.push_back(f);
        return f.q;
      };
      const double2 one = make_double2(1.0, 0.0);
      const double2* q1[4] = {};
      const double2* q2[4] = {};
      for (int sl = 0; sl < sp.n1; ++sl) {
        int off = sp.alpha_of1[sl] * n_ev;
        q1[sl] = add_field(phin[0], j.nd[0], 1, &off, &one);
      }
      for (int sl = 0; sl < sp.n2; ++sl) {
        int off = sp.beta_of2[sl] * n_ev;
        q2[sl] = add_field(phin[1], j.nd[1], 1, &off, &one);
      }
      std::vector<std::vector<const double2*>> q3(sp.n_coef_sets, std::vector<const double2*>(sp.n_pairs));
      for (int set = 0; set < sp.n_coef_sets; ++set)
        for (int pr = 0; pr < sp.n_pairs; ++pr) {
          const auto& tlist = sp.terms[set][pr];
          if ((int)tlist.size() > kMaxTerms) return fail(c, BBLOCK_ERR_UNSUPPORTED, "too many terms");
          int offs[kMaxTerms];
          double2 w[kMaxTerms];
          for (size_t t = 0; t < tlist.size(); ++t) { offs[t] = tlist[t].first * n_ev; w[t] = tlist[t].second; }
          q3[set][pr] = add_field(phin[2], j.nd[2], (int)tlist.size(), offs, w);
        }
      base = c->d_ws + align_up((size_t)(base - c->d_ws), 256);
      double2* partial = reinterpret_cast<double2*>(base);
      base += align_up((size_t)n_slab * n_mom * j.nd[0] * j.nd[1] * j.nd[2] * sizeof(double2), 256);
      canary(base);
      ws = base;
      int m_tiles, n_tiles;
      job_tiles(j, m_tiles, n_tiles);
      float* oz_max = nullptr;
      if (oz) {
        oz_max = reinterpret_cast<float*>(oz_base);
        oz_base += oz_bytes(j, n_slab);
        const int stride = j.nd[0] + j.nd[1] + j.nd[2];
        auto seg = [&](const double2* q, int nd, int off, int modulus) {
          ozsegs.push_back(
              OzMaxSeg{reinterpret_cast<const float4*>(q), oz_max, nd, off, stride, modulus});
        };
        for (int sl = 0; sl < sp.n1; ++sl) seg(q1[sl], j.nd[0], 0, 0);
        for (int sl = 0; sl < sp.n2; ++sl) seg(q2[sl], j.nd[1], j.nd[0], 0);
        for (int set = 0; set < sp.n_coef_sets; ++set)
          for (int pr = 0; pr < sp.n_pairs; ++pr) seg(q3[set][pr], j.nd[2], j.nd[0] + j.nd[1], 1);
      }
      for (int set = 0; set < sp.n_coef_sets; ++set) {
        ContractJob& cj = cjobs[set][k];
        cj.oz_max = oz_max;
        for (int i = 0; i < 4; ++i) { cj.q1[i] = q1[i]; cj.q2[i] = q2[i]; }
        for (int pr = 0; pr < sp.n_pairs; ++pr) cj.q3[pr] = q3[set][pr];
        cj.partial = partial;
        cj.B = j.B;
        cj.nd1 = j.nd[0]; cj.nd2 = j.nd[1]; cj.nd3 = j.nd[2];
        cj.m_tiles = m_tiles;
        cj.n_tiles = n_tiles;
        cj.unit_begin = unit;
      }
      unit += (long long)m_tiles * n_tiles * n_slab;
    }
    // one contiguous table upload: fields, then one job table per coefficient set
    for (const ProjField& f : fields)
      if (!within_workspace(c, f.q, (size_t)rows * f.nd * sizeof(double2)))
        return fail(c, BBLOCK_ERR_INVALID_ARG, "internal: field outside the workspace");
    for (int k = 0; k < nj; ++k) {
      const ContractJob& cj = cjobs[0][k];
      if (!within_workspace(c, cj.partial, (size_t)n_slab * n_mom * cj.nd1 * cj.nd2 * cj.nd3 * sizeof(double2)))
        return fail(c, BBLOCK_ERR_INVALID_ARG, "internal: partial block outside the workspace");
    }
    for (const DfConvSeg& g : segs)
      if (!within_workspace(c, g.dst, (size_t)g.n * sizeof(float4)))
        return fail(c, BBLOCK_ERR_INVALID_ARG, "internal: converted input outside the workspace");
    for (uint32_t* cn : canaries)
      if (!within_workspace(c, cn, kCanaryBytes))
        return fail(c, BBLOCK_ERR_INVALID_ARG, "internal: canary outside the workspace");
    const size_t fbytes = align_up(fields.size() * sizeof(ProjField), 256);
    const size_t jbytes = align_up((size_t)nj * sizeof(ContractJob), 256);
    const size_t sofs = fbytes + jbytes * sp.n_coef_sets;
    const size_t cofs = sofs + align_up(segs.size() * sizeof(DfConvSeg), 256);
    const size_t zofs = cofs + align_up(canaries.size() * sizeof(uint32_t*), 256);
    std::vector<char> tab(zofs + ozsegs.size() * sizeof(OzMaxSeg));
    memcpy(tab.data(), fields.data(), fields.size() * sizeof(ProjField));
    for (int set = 0; set < sp.n_coef_sets; ++set)
      memcpy(tab.data() + fbytes + jbytes * set, cjobs[set].data(), (size_t)nj * sizeof(ContractJob));
    if (!segs.empty()) memcpy(tab.data() + sofs, segs.data(), segs.size() * sizeof(DfConvSeg));
    if (!canaries.empty()) memcpy(tab.data() + cofs, canaries.data(), canaries.size() * sizeof(uint32_t*));
    if (!ozsegs.empty()) memcpy(tab.data() + zofs, ozsegs.data(), ozsegs.size() * sizeof(OzMaxSeg));
    rc = upload_tables(c, tab.data(), tab.size(), s);
    if (rc) return rc;
    const ProjField* d_fields = reinterpret_cast<const ProjField*>(c->d_tab);
    uint32_t* const* d_canaries = reinterpret_cast<uint32_t* const*>(c->d_tab + cofs);
    if (!canaries.empty()) {
      CK(c, timed_launch(c, K_CANARY, s, [&] {
        return launch_canaries(d_canaries, (int)canaries.size(), false, c->d_status, s);
      }));
      if (c->opt_corrupt_canary && !c->capturing) {   // test hook: a simulated overrun
        c->opt_corrupt_canary = 0;
        CK(c, cudaMemsetAsync(canaries[0], 0x5a, 4, s));
      }
    }

    if (df) {
      CK(c, timed_launch(c, K_CONVERT, s, [&] {
        return launch_convert_df(reinterpret_cast<const DfConvSeg*>(c->d_tab + sofs),
                                 (int)segs.size(), max_seg, s);
      }));
    }
    CK(c, timed_launch(c, K_PROJECT, s, [&] {
      return df ? launch_project_df(d_fields, (int)fields.size(), rows, n_ev, max_ndf, s)
                : launch_project_fp64(d_fields, (int)fields.size(), rows, n_ev, max_ndf, s);
    }));
    if (oz) {
      // the slabs' column maxima of every field, from which the contraction takes its scales
      CK(c, cudaMemsetAsync(c->d_ws + (ws_need - oz_need), 0, oz_need, s));
      CK(c, timed_launch(c, K_PROJECT, s, [&] {
        return launch_oz_colmax(reinterpret_cast<const OzMaxSeg*>(c->d_tab + zofs),
                                (int)ozsegs.size(), X, sites_per_slab, s);
      }));
    }

    ContractParams prm{};
    prm.n_jobs = nj;
    prm.total_units = unit;
    prm.X = X;
    prm.n_slab = n_slab;
    prm.sites_per_slab = sites_per_slab;
    prm.n_pairs = sp.n_pairs;
    for (int pr = 0; pr < sp.n_pairs; ++pr) { prm.a_slot[pr] = sp.a_slot[pr]; prm.b_slot[pr] = sp.b_slot[pr]; }
    prm.phase = c->d_phase;
    prm.P_total = n_mom;
    prm.status = c->d_status;
    prm.phase_df = c->d_phase_df;
    prm.NC = oz_nc;
    prm.wait_limit = c->opt_wait_us > 0 ? (long long)c->opt_wait_us * c->cycles_per_us
                                        : 4000000000LL;
    const int grid = (int)std::min<long long>(unit, ctas);
    if (oz) {
      // the diquark's row maxima (from the line-1 and line-2 fields of any coefficient set)
      int max_mt = 0;
      for (int k = 0; k < nj; ++k) max_mt = std::max(max_mt, cjobs[0][k].m_tiles);
      prm.jobs = reinterpret_cast<const ContractJob*>(c->d_tab + fbytes);
      CK(c, timed_launch(c, K_PROJECT, s, [&] { return launch_oz_rowmax(prm, max_mt, s); }));
      // every momentum as N columns of one launch (one launch per momentum with per-momentum
      // coefficient sets)
      for (int set = 0; set < sp.n_coef_sets; ++set) {
        prm.jobs = reinterpret_cast<const ContractJob*>(c->d_tab + fbytes + jbytes * set);
        prm.p0 = per_mom ? set : 0;
        prm.P = per_mom ? 1 : n_mom;
        CK(c, timed_launch(c, K_CONTRACT, s, [&] {
          return launch_contract_oz(prm, oz_cl, (int)std::min<long long>(unit, unit_slots), s);
        }));
      }
    } else if (per_mom) {
      for (int p = 0; p < n_mom; ++p) {
        prm.jobs = reinterpret_cast<const ContractJob*>(c->d_tab + fbytes + jbytes * p);
        prm.p0 = p;
        CK(c, timed_launch(c, K_CONTRACT, s, [&] {
          return df ? launch_contract_df(prm, 1, tl.rn, grid, s) : launch_contract_fp64(prm, 1, tl.rn, grid, s);
        }));
      }
    } else {
      prm.jobs = reinterpret_cast<const ContractJob*>(c->d_tab + fbytes);
      const int pg = P_launch;
      for (int p0 = 0; p0 < n_mom; p0 += pg) {
        const int Pg = std::min(pg, n_mom - p0);
        prm.p0 = p0;
        CK(c, timed_launch(c, K_CONTRACT, s, [&] {
          return df ? launch_contract_df(prm, Pg, tl.rn, grid, s) : launch_contract_fp64(prm, Pg, tl.rn, grid, s);
        }));
      }
    }
    CK(c, timed_launch(c, K_REDUCE, s, [&] {
      return launch_reduce_slabs(reinterpret_cast<const ContractJob*>(c->d_tab + fbytes), nj,
                                 n_slab, n_mom, max_elems, s);
    }));
    if (!canaries.empty())
      CK(c, timed_launch(c, K_CANARY, s, [&] {
        return launch_canaries(d_canaries, (int)canaries.size(), true, c->d_status, s);
      }));
    job_idx = end;
  }
  return BBLOCK_OK;
}

// Everything a call's launch sequence depends on, as a flat key.
std::vector<uint64_t> call_signature(const bblock_ctx* c, const std::vector<JobIn>& jobs,
                                     const int32_t* momenta, int n_mom, const int32_t* spin_idx,
                                     const double* coeffs, int n_spin, int per_mom) {
  std::vector<uint64_t> k;
  k.reserve(16 + jobs.size() * 8 + 3 * n_mom + 3 * n_spin);
  k.push_back((uint64_t)c->cfg.precision | ((uint64_t)c->cfg.bf16_products << 8) |
              ((uint64_t)per_mom << 16) | ((uint64_t)c->opt_tc_nc << 24) |
              ((uint64_t)c->opt_tc_chunk << 32) | ((uint64_t)c->opt_slabs << 40));
  k.push_back((uint64_t)n_mom | ((uint64_t)n_spin << 32));
  k.push_back((uint64_t)wave_budget(c) ^ ((uint64_t)c->opt_tc_cluster << 60) ^
              ((uint64_t)c->opt_tc_proj << 56) ^ ((uint64_t)c->prof << 52) ^
              ((uint64_t)c->opt_tc_rows << 48));
  for (int i = 0; i < 3 * n_mom; ++i) k.push_back((uint64_t)(uint32_t)momenta[i]);
  for (int i = 0; i < 3 * n_spin; ++i) k.push_back((uint64_t)(uint32_t)spin_idx[i]);
  const int n_coef = 2 * n_spin * (per_mom ? n_mom : 1);
  for (int i = 0; i < n_coef; ++i) {
    uint64_t b;
    memcpy(&b, &coeffs[i], sizeof(b));
    k.push_back(b);
  }
  for (const JobIn& j : jobs) {
    k.push_back(reinterpret_cast<uint64_t>(j.V));
    for (int i = 0; i < 3; ++i) k.push_back(reinterpret_cast<uint64_t>(j.phi[i]));
    k.push_back(reinterpret_cast<uint64_t>(j.B));
    k.push_back((uint64_t)j.nd[0] | ((uint64_t)j.nd[1] << 20) | ((uint64_t)j.nd[2] << 40));
  }
  return k;
}

// run_jobs with CUDA-graph reuse: the second call with an identical signature is captured
// (thread-local capture mode) and every later identical call replays the graph.
int run_jobs_cached(bblock_ctx* c, const std::vector<JobIn>& jobs, const int32_t* momenta,
                    int n_mom, const int32_t* spin_idx, const double* coeffs, int n_spin,
                    int per_mom, cudaStream_t s) {
  // the legacy and per-thread default streams cannot be captured
  const bool capturable = s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
  if (!c->opt_graphs || !capturable || jobs.empty() || n_mom == 0)
    return run_jobs(c, jobs, momenta, n_mom, spin_idx, coeffs, n_spin, per_mom, s);
  std::vector<uint64_t> sig = call_signature(c, jobs, momenta, n_mom, spin_idx, coeffs, n_spin,
                                             per_mom);
  if (c->graph_exec && sig == c->graph_sig) {
    CK(c, cudaSetDevice(c->cfg.device));
    int rc = ensure_phase(c, momenta, n_mom, s);   // a call in between may have replaced it
    if (rc) return rc;
    if (!c->graph_exec) return run_jobs(c, jobs, momenta, n_mom, spin_idx, coeffs, n_spin, per_mom, s);
    // the graph's timing events are re-recorded by this replay: read the last one's first
    if (c->graph_pending) CK(c, harvest_graph_times(c));
    CK(c, cudaGraphLaunch(c->graph_exec, s));
    c->graph_pending = !c->graph_timed.empty();
    c->last_launches = c->graph_launches;
    c->last_waves = c->graph_waves;
    c->last_path = c->graph_path;
    c->last_stream = s;
    return BBLOCK_OK;
  }
  if (sig != c->last_sig) {
    c->last_sig = sig;
    return run_jobs(c, jobs, momenta, n_mom, spin_idx, coeffs, n_spin, per_mom, s);
  }
  // second identical call: every buffer already has its size, so capture it
  drop_graph(c);
  if (c->h_graph_tab_cap < c->call_tab_bytes) {
    if (c->h_graph_tab) {
      // an older graph that read this staging has been dropped, but a replay may be in flight
      if (c->last_stream) CK(c, cudaStreamSynchronize(c->last_stream));
      cudaFreeHost(c->h_graph_tab);
    }
    c->h_graph_tab = nullptr;
    c->h_graph_tab_cap = 0;
    if (cudaHostAlloc(&c->h_graph_tab, c->call_tab_bytes, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return run_jobs(c, jobs, momenta, n_mom, spin_idx, coeffs, n_spin, per_mom, s);
    }
    c->h_graph_tab_cap = c->call_tab_bytes;
  }
  CK(c, cudaSetDevice(c->cfg.device));
  // the previous plain upload must have drained before the capture reuses the device tables
  if (c->tab_free) CK(c, cudaEventSynchronize(c->tab_free));
  c->graph_tab_off = 0;
  CK(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  c->capturing = true;
  int rc = run_jobs(c, jobs, momenta, n_mom, spin_idx, coeffs, n_spin, per_mom, s);
  c->capturing = false;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (rc != BBLOCK_OK || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    drop_graph(c);
    c->last_sig.clear();
    c->err.clear();
    return run_jobs(c, jobs, momenta, n_mom, spin_idx, coeffs, n_spin, per_mom, s);
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    drop_graph(c);
    c->last_sig.clear();
    return run_jobs(c, jobs, momenta, n_mom, spin_idx, coeffs, n_spin, per_mom, s);
  }
  c->graph_exec = exec;
  c->graph_sig = sig;
  c->graph_launches = c->last_launches;
  c->graph_waves = c->last_waves;
  c->graph_path = c->last_path;
  CK(c, cudaGraphLaunch(exec, s));
  c->graph_pending = !c->graph_timed.empty();
  c->last_stream = s;
  return BBLOCK_OK;
}

// ---------------------------------------------------------------- autotuner

// How one bblock_compute call with uniform dilution sizes is cut into work units for a
// given set of tile options (the same rules as run_jobs / run_jobs_tc, one wave).
struct CallPlan {
  int nc = 0, chunk = 0, n_slab = 0;
  long long units = 0;
  double pad = 0.0;  // padded / actual columns - 1
};

CallPlan plan_call(const bblock_ctx* c, int n_t, const int nd[3], int n_mom, int pairs,
                   int nc_opt, int chunk_opt, int slabs_opt) {
  CallPlan pl;
  const int X = c->X;
  if (c->cfg.precision == BBLOCK_OZAKI) {
    // units (job, 128-row tile, N tile over every momentum's columns, slab)
    const int nc = nc_opt > 0 && nc_opt <= kOzMaxNC ? nc_opt : kOzMaxNC;
    const long long nt = ((long long)n_mom * nd[2] + nc - 1) / nc;
    const long long tiles = (long long)n_t * ((nd[0] * nd[1] + kOzM - 1) / kOzM) * nt;
    pl.nc = nc;
    pl.n_slab = slabs_opt > 0 ? std::min(slabs_opt, X) : choose_slabs(tiles, c->num_sms, X, 1, 64);
    const int sps = (X + pl.n_slab - 1) / pl.n_slab;
    pl.n_slab = (X + sps - 1) / sps;
    pl.units = tiles * pl.n_slab;
    pl.pad = (double)(nt * nc) / ((double)n_mom * nd[2]) - 1.0;
    return pl;
  }
  if (fp64_like(c->cfg)) {
    const int P = p_group_size(n_mom, c->cfg.precision == BBLOCK_DF64 ? kMaxPGroupDf : kMaxPGroup);
    const Fp64Tile tl = fp64_tile_for(P);
    const int xc = fp64_sites_per_chunk(pairs);
    const int ctas = fp64_contract_ctas_per_sm(P, tl.rn, pairs) * c->num_sms;
    const long long tiles = (long long)n_t * ((nd[0] * nd[1] + 16 * tl.rm - 1) / (16 * tl.rm)) *
                            ((nd[2] + 16 * tl.rn - 1) / (16 * tl.rn));
    int ns = slabs_opt > 0 ? std::min(slabs_opt, (X + xc - 1) / xc) : choose_slabs(tiles, ctas, X, xc, 64);
    int sps = (X + ns - 1) / ns;
    sps = (sps + xc - 1) / xc * xc;
    pl.n_slab = (X + sps - 1) / sps;
    pl.units = tiles * pl.n_slab;
    pl.pad = (double)(((nd[2] + 16 * tl.rn - 1) / (16 * tl.rn)) * 16 * tl.rn) / nd[2] - 1.0;
    return pl;
  }
  const int G = tc_groups_per_stage(tc_form_of(c->cfg));
  pl.chunk = chunk_opt > 0 ? chunk_opt : 2;
  const long long max_groups_per_unit = 256LL * pl.chunk * G;
  const int min_slabs = (int)std::min<long long>(X, ((long long)X * pairs + max_groups_per_unit - 1) / max_groups_per_unit);
  const int max_slabs = std::max(64, min_slabs);
  std::vector<JobIn> one(1);
  one[0].nd[0] = nd[0]; one[0].nd[1] = nd[1]; one[0].nd[2] = nd[2];
  const RfPlan rp = plan_rf(c, n_mom, 0, tc_form_of(c->cfg), pairs, G, nc_opt);
  if (rp.on) {   // row-factored: units over d3 tiles and slabs of lattice rows
    const int L = c->cfg.L, n_rows = L * L;
    const int cpr = (rp.spr + pl.chunk - 1) / pl.chunk;
    const int min_s = (n_rows + std::max(1, 256 / cpr) - 1) / std::max(1, 256 / cpr);
    pl.nc = rp.nidx * rp.nc;
    const int cl = (c->opt_tc_cluster == 2 || (c->opt_tc_cluster == 0 && nd[2] > rp.nc)) ? 2 : 1;
    const long long n_tiles = ((nd[2] + rp.nc - 1) / rp.nc + cl - 1) / cl;
    const long long tiles = (long long)n_t * (((long long)nd[0] * nd[1] + 127) / 128) * n_tiles;
    int ns = slabs_opt > 0 ? std::max(min_s, std::min(slabs_opt, n_rows))
                           : std::max(min_s, choose_slabs(tiles, c->num_sms / cl, n_rows, 1, max_slabs));
    const int rps = (n_rows + ns - 1) / ns;
    pl.n_slab = (n_rows + rps - 1) / rps;
    pl.units = tiles * pl.n_slab;
    pl.pad = (double)(n_tiles * cl * rp.nc) / nd[2] - 1.0;
    return pl;
  }
  // the tiling run_jobs_tc would pick with this candidate's N tile
  const TcTiling tt = choose_tc_tiling(c, one, 0, 1, n_mom, tc_form_of(c->cfg), nc_opt);
  pl.nc = tt.nc;
  const long long N = (long long)n_mom * nd[2];                   // (p, d3) columns
  const long long n_group = tt.share_b ? pl.nc : (long long)tt.cluster * pl.nc;
  const long long n_tiles = (N + n_group - 1) / n_group;
  const long long mt = ((long long)nd[0] * nd[1] + 127) / 128;
  const long long tiles = (long long)n_t * (tt.share_b ? (mt + 1) / 2 : mt) * n_tiles;
  int ns = slabs_opt > 0 ? std::max(min_slabs, std::min(slabs_opt, X))
                         : std::max(min_slabs, choose_slabs(tiles, c->num_sms / tt.cluster, X, 1, max_slabs));
  const int sps = (X + ns - 1) / ns;
  pl.n_slab = (X + sps - 1) / sps;
  pl.units = tiles * pl.n_slab;
  pl.pad = (double)(n_tiles * n_group) / N - 1.0;
  return pl;
}

int form_code(const bblock_config& cfg) {
  if (cfg.precision == BBLOCK_FP64) return 0;
  if (cfg.precision == BBLOCK_DF64) return 5;
  if (cfg.precision == BBLOCK_TF32X3) return 4;
  if (cfg.precision == BBLOCK_FP16X3) return 6;
  if (cfg.precision == BBLOCK_OZAKI) return 7;
  return cfg.bf16_products == 3 ? 1 : cfg.bf16_products == 9 ? 3 : 2;
}

void tune_features(const bblock_ctx* c, int n_t, const int nd[3], int n_mom, int pairs,
                   const CallPlan& pl, float* f) {
  auto lg = [](double v) { return (float)std::log2(std::max(v, 1.0)); };
  f[0] = lg((double)nd[0] * nd[1]) / 12.f;
  f[1] = lg((double)n_mom * nd[2]) / 12.f;
  f[2] = lg((double)c->X) / 20.f;
  f[3] = pairs / 16.f;
  f[4] = pl.nc / 48.f;
  f[5] = pl.chunk / 4.f;
  f[6] = lg(pl.n_slab) / 12.f;
  f[7] = lg((double)pl.units / c->num_sms) / 8.f;
  f[8] = form_code(c->cfg) / 4.f;
  f[9] = (float)pl.pad;
  f[10] = lg(n_t) / 8.f;
  f[11] = lg(c->cfg.n_ev) / 10.f;
}

}  // namespace

extern "C" {

int bblock_create(bblock_ctx** out, const bblock_config* cfg) {
  if (!out) return BBLOCK_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg) return BBLOCK_ERR_INVALID_ARG;
  if (cfg->L < 1 || cfg->L > 128) return BBLOCK_ERR_INVALID_ARG;
  const long long X = (long long)cfg->L * cfg->L * cfg->L;
  if (cfg->n_ev < 1 || cfg->n_ev > 3 * X) return BBLOCK_ERR_INVALID_ARG;
  if (cfg->max_ndil < 1 || cfg->max_ndil > 256) return BBLOCK_ERR_INVALID_ARG;
  if (cfg->precision < BBLOCK_FP64 || cfg->precision > BBLOCK_OZAKI) return BBLOCK_ERR_INVALID_ARG;
  if (cfg->precision == BBLOCK_BF16_SPLIT && cfg->bf16_products != 3 && cfg->bf16_products != 6 &&
      cfg->bf16_products != 9)
    return BBLOCK_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return BBLOCK_ERR_CUDA;
  }
  if (cfg->device < 0 || cfg->device >= ndev) return BBLOCK_ERR_INVALID_ARG;
  bblock_ctx* c = new bblock_ctx();
  c->cfg = *cfg;
  c->X = (int)X;
  c->rows = (int)(3 * X);
  if (cudaSetDevice(cfg->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, cfg->device) != cudaSuccess ||
      cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess || cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->d_dbg, 4 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(c->d_dbg, 0, 4 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->tab_free, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    bblock_destroy(c);
    return BBLOCK_ERR_CUDA;
  }
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  c->ws_budget = std::min<size_t>(free_b / 2, (size_t)96 << 30);
  int khz = 0;   // SM clock: converts the wait-limit test hook from microseconds to cycles
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, cfg->device) == cudaSuccess && khz > 0)
    c->cycles_per_us = std::max(1, khz / 1000);
  else
    cudaGetLastError();
  *out = c;
  return BBLOCK_OK;
}

void bblock_destroy(bblock_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->cfg.device);
  cudaDeviceSynchronize();
  cudaFree(c->d_status);
  cudaFree(c->d_dbg);
  cudaFree(c->d_phase);
  cudaFree(c->d_mom);
  cudaFree(c->d_ws);
  cudaFree(c->d_tab);
  cudaFree(c->d_io);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  cudaFree(c->d_ident);
  cudaFree(c->d_tri);
  if (c->h_tab) cudaFreeHost(c->h_tab);
  if (c->tab_free) cudaEventDestroy(c->tab_free);
  drop_graph(c);
  if (c->h_graph_tab) cudaFreeHost(c->h_graph_tab);
  for (auto& t : c->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  cudaGetLastError();
  delete c;
}

const char* bblock_last_error(const bblock_ctx* c) { return c ? c->err.c_str() : "null context"; }

int bblock_status(bblock_ctx* c) {
  if (!c) return BBLOCK_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(c->cfg.device);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "bblock_status");
  int st = 0;
  e = cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "bblock_status readback");
  if (st) {
    unsigned long long d[4] = {0, 0, 0, 0};
    if (cudaMemcpy(d, c->d_dbg, sizeof(d), cudaMemcpyDeviceToHost) != cudaSuccess) cudaGetLastError();
    // reported once: clear the word and the index record so the next call starts clean
    if (cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->d_dbg, 0, 4 * sizeof(unsigned long long)) != cudaSuccess)
      cudaGetLastError();
    if (st & kStatusTimeout)
      return fail(c, BBLOCK_ERR_TIMEOUT, "a bounded device wait gave up (status word 0x%x)", st);
    if (st & kStatusCanary)
      return fail(c, BBLOCK_ERR_DEVICE_FLAG,
                  "a workspace canary was overwritten: a kernel wrote past its block (status word 0x%x)", st);
    return fail(c, BBLOCK_ERR_DEVICE_FLAG,
                "device status word 0x%x (index check: site %llu job %llu index %llu bound %llu)",
                st, d[0], d[1], d[2], d[3]);
  }
  return BBLOCK_OK;
}

int bblock_compute(bblock_ctx* c, int n_t, const void* V, const void* phi1, const void* phi2,
                   const void* phi3, int nd1, int nd2, int nd3, const int32_t* momenta, int n_mom,
                   const int32_t* spin_idx, const double* spin_coeffs, int n_spin, int coeff_per_mom,
                   void* B_out, void* stream) {
  if (!c) return BBLOCK_ERR_INVALID_ARG;
  c->err.clear();
  if (n_t < 0) return fail(c, BBLOCK_ERR_INVALID_ARG, "n_t = %d < 0", n_t);
  int rc = validate_common(c, momenta, n_mom, spin_idx, spin_coeffs, n_spin, coeff_per_mom);
  if (rc) return rc;
  if (n_t == 0 || n_mom == 0) { c->last_launches = 0; c->last_waves = 0; return BBLOCK_OK; }
  const size_t vstride = (size_t)c->cfg.n_ev * c->rows;
  const size_t pst[3] = {(size_t)4 * c->cfg.n_ev * nd1, (size_t)4 * c->cfg.n_ev * nd2,
                         (size_t)4 * c->cfg.n_ev * nd3};
  const size_t bstride = (size_t)n_mom * nd1 * nd2 * nd3;
  if (!V || !phi1 || !phi2 || !phi3 || !B_out)
    return fail(c, BBLOCK_ERR_INVALID_ARG, "a data pointer is NULL");
  std::vector<JobIn> jobs(n_t);
  for (int t = 0; t < n_t; ++t) {
    JobIn& j = jobs[t];
    j.V = static_cast<const double2*>(V) + t * vstride;
    j.phi[0] = static_cast<const double2*>(phi1) + t * pst[0];
    j.phi[1] = static_cast<const double2*>(phi2) + t * pst[1];
    j.phi[2] = static_cast<const double2*>(phi3) + t * pst[2];
    j.nd[0] = nd1; j.nd[1] = nd2; j.nd[2] = nd3;
    j.B = static_cast<double2*>(B_out) + t * bstride;
    if (t == 0) {
      rc = validate_job(c, j, 0, true, n_mom, n_t);
      if (rc) return rc;
    }
  }
  return run_jobs_cached(c, jobs, momenta, n_mom, spin_idx, spin_coeffs, n_spin, coeff_per_mom,
                  static_cast<cudaStream_t>(stream));
}

int bblock_compute_batch(bblock_ctx* c, const bblock_job* jobs_in, int n_jobs,
                         const int32_t* momenta, int n_mom, const int32_t* spin_idx,
                         const double* spin_coeffs, int n_spin, int coeff_per_mom, void* stream) {
  if (!c) return BBLOCK_ERR_INVALID_ARG;
  c->err.clear();
  if (n_jobs < 0 || (n_jobs > 0 && !jobs_in)) return fail(c, BBLOCK_ERR_INVALID_ARG, "bad job list");
  int rc = validate_common(c, momenta, n_mom, spin_idx, spin_coeffs, n_spin, coeff_per_mom);
  if (rc) return rc;
  std::vector<JobIn> jobs(n_jobs);
  for (int k = 0; k < n_jobs; ++k) {
    JobIn& j = jobs[k];
    j.V = static_cast<const double2*>(jobs_in[k].V);
    j.phi[0] = static_cast<const double2*>(jobs_in[k].phi1);
    j.phi[1] = static_cast<const double2*>(jobs_in[k].phi2);
    j.phi[2] = static_cast<const double2*>(jobs_in[k].phi3);
    j.nd[0] = jobs_in[k].nd1; j.nd[1] = jobs_in[k].nd2; j.nd[2] = jobs_in[k].nd3;
    j.B = static_cast<double2*>(jobs_in[k].B_out);
    rc = validate_job(c, j, k, true, n_mom);
    if (rc) return rc;
  }
  // dilution sizes may differ per job: larger jobs first so the persistent grid ends evenly
  std::stable_sort(jobs.begin(), jobs.end(), [](const JobIn& a, const JobIn& b) {
    return (long long)a.nd[0] * a.nd[1] * a.nd[2] > (long long)b.nd[0] * b.nd[1] * b.nd[2];
  });
  return run_jobs_cached(c, jobs, momenta, n_mom, spin_idx, spin_coeffs, n_spin, coeff_per_mom,
                  static_cast<cudaStream_t>(stream));
}

// Eq. (4): T[t][p] is the contraction with q_i = V, i.e. identity coefficients and the
// single spin triple (0, 0, 0), computed by the context's form for every time slice.
int bblock_mode_triplet(bblock_ctx* c, int n_t, const void* V, const int32_t* momenta, int n_mom,
                        void* T_out, void* stream) {
  if (!c) return BBLOCK_ERR_INVALID_ARG;
  c->err.clear();
  const int n_ev = c->cfg.n_ev;
  if (n_t < 0) return fail(c, BBLOCK_ERR_INVALID_ARG, "n_t = %d < 0", n_t);
  if (n_ev > c->cfg.max_ndil)
    return fail(c, BBLOCK_ERR_INVALID_ARG, "the mode triplet needs max_ndil >= n_ev (%d)", n_ev);
  const int32_t spin[3] = {0, 0, 0};
  const double one[2] = {1.0, 0.0};
  int rc = validate_common(c, momenta, n_mom, spin, one, 1, 0);
  if (rc) return rc;
  if (n_t == 0 || n_mom == 0) { c->last_launches = 0; c->last_waves = 0; return BBLOCK_OK; }
  CK(c, cudaSetDevice(c->cfg.device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!c->d_ident) {
    if (c->capturing) return fail(c, BBLOCK_ERR_UNSUPPORTED, "allocation during graph capture");
    if (cudaMalloc(&c->d_ident, sizeof(double2) * 4 * (size_t)n_ev * n_ev) != cudaSuccess) {
      cudaGetLastError();
      c->d_ident = nullptr;
      return fail(c, BBLOCK_ERR_OOM, "identity coefficients");
    }
    CK(c, launch_fill_identity(c->d_ident, n_ev, s));
  }
  const size_t vstride = (size_t)n_ev * c->rows;
  const size_t tstride = (size_t)n_mom * n_ev * n_ev * n_ev;
  std::vector<JobIn> jobs(n_t);
  for (int t = 0; t < n_t; ++t) {
    JobIn& j = jobs[t];
    j.V = static_cast<const double2*>(V) + t * vstride;
    j.phi[0] = j.phi[1] = j.phi[2] = c->d_ident;
    j.nd[0] = j.nd[1] = j.nd[2] = n_ev;
    j.B = static_cast<double2*>(T_out) + t * tstride;
    rc = validate_job(c, j, t, true, n_mom);
    if (rc) return rc;
  }
  return run_jobs_cached(c, jobs, momenta, n_mom, spin, one, 1, 0, s);
}

// Eq. (3) through the mode triplet: for every time slice and (alpha, beta) pair,
//   U1 = T x3 phi3'   (phi3' = the pair's folded line-3 coefficients),
//   U2 = U1 x2 phi2[beta],  B += U2 x1 phi1[alpha],
// three batched complex GEMMs in FP64.
int bblock_from_triplet(bblock_ctx* c, int n_t, const void* T, const void* phi1, const void* phi2,
                        const void* phi3, int nd1, int nd2, int nd3, int n_mom,
                        const int32_t* spin_idx, const double* spin_coeffs, int n_spin,
                        int coeff_per_mom, void* B_out, void* stream) {
  if (!c) return BBLOCK_ERR_INVALID_ARG;
  c->err.clear();
  const int n_ev = c->cfg.n_ev;
  if (n_t < 0) return fail(c, BBLOCK_ERR_INVALID_ARG, "n_t = %d < 0", n_t);
  // momenta are not needed (T already carries them); any valid array satisfies the check
  std::vector<int32_t> mom_dummy(3 * (size_t)std::max(n_mom, 1), 0);
  int rc = validate_common(c, mom_dummy.data(), n_mom, spin_idx, spin_coeffs, n_spin, coeff_per_mom);
  if (rc) return rc;
  if (n_t == 0 || n_mom == 0) { c->last_launches = 0; c->last_waves = 0; return BBLOCK_OK; }
  const int nds[3] = {nd1, nd2, nd3};
  for (int i = 0; i < 3; ++i)
    if (nds[i] < 1 || nds[i] > c->cfg.max_ndil)
      return fail(c, BBLOCK_ERR_INVALID_ARG, "nd%d = %d outside 1..max_ndil", i + 1, nds[i]);
  const size_t tstride = (size_t)n_mom * n_ev * n_ev * n_ev;
  const size_t pst[3] = {(size_t)4 * n_ev * nd1, (size_t)4 * n_ev * nd2, (size_t)4 * n_ev * nd3};
  const size_t bstride = (size_t)n_mom * nd1 * nd2 * nd3;
  const void* ptrs[5] = {T, phi1, phi2, phi3, B_out};
  const size_t ext[5] = {tstride * n_t, pst[0] * n_t, pst[1] * n_t, pst[2] * n_t, bstride * n_t};
  const char* names[5] = {"T", "phi1", "phi2", "phi3", "B_out"};
  for (int k = 0; k < 5; ++k) {
    if (!ptrs[k] || !aligned16(ptrs[k]) || !is_device_ptr(c, ptrs[k]))
      return fail(c, BBLOCK_ERR_INVALID_ARG, "%s must be 16-byte aligned device memory", names[k]);
    if (!within_allocation(ptrs[k], ext[k] * sizeof(double2)))
      return fail(c, BBLOCK_ERR_INVALID_ARG, "%s extends past its allocation", names[k]);
  }
  SpinPlan sp;
  rc = plan_spins(c, spin_idx, spin_coeffs, n_spin, coeff_per_mom, n_mom, &sp);
  if (rc) return rc;
  CK(c, cudaSetDevice(c->cfg.device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  // intermediates for the momenta of one coefficient set
  const int P_set = coeff_per_mom ? 1 : n_mom;
  const size_t f_bytes = align_up(sizeof(double2) * (size_t)n_ev * nd3, 256);
  const size_t u1_bytes = align_up(sizeof(double2) * (size_t)P_set * n_ev * n_ev * nd3, 256);
  const size_t u2_bytes = align_up(sizeof(double2) * (size_t)P_set * n_ev * nd2 * nd3, 256);
  rc = grow_device(c, &c->d_tri, &c->tri_cap, f_bytes + u1_bytes + u2_bytes);
  if (rc) return rc;
  double2* fold = reinterpret_cast<double2*>(c->d_tri);
  double2* U1 = reinterpret_cast<double2*>(c->d_tri + f_bytes);
  double2* U2 = reinterpret_cast<double2*>(c->d_tri + f_bytes + u1_bytes);
  int launches = 0;
  const double2 one = make_double2(1.0, 0.0);
  for (int t = 0; t < n_t; ++t) {
    const double2* Tt = static_cast<const double2*>(T) + t * tstride;
    const double2* p1 = static_cast<const double2*>(phi1) + t * pst[0];
    const double2* p2 = static_cast<const double2*>(phi2) + t * pst[1];
    const double2* p3 = static_cast<const double2*>(phi3) + t * pst[2];
    double2* Bt = static_cast<double2*>(B_out) + t * bstride;
    for (int set = 0; set < sp.n_coef_sets; ++set) {
      const int p0 = coeff_per_mom ? set : 0;
      for (int pr = 0; pr < sp.n_pairs; ++pr) {
        FoldTerms ft{};
        const auto& tl = sp.terms[set][pr];
        ft.n = (int)tl.size();
        for (int k = 0; k < ft.n; ++k) { ft.row[k] = tl[k].first; ft.w[k] = tl[k].second; }
        CK(c, launch_fold_phi(p3, n_ev, nd3, ft, fold, s));
        // U1[(p, l1, l2)][d3] = sum_l3 T[p][l1][l2][l3] phi3'[l3][d3]
        ZgemmParams g{};
        g.M = P_set * n_ev * n_ev; g.N = nd3; g.K = n_ev; g.batch = 1;
        g.A = Tt + (size_t)p0 * n_ev * n_ev * n_ev; g.a_m = n_ev; g.a_k = 1;
        g.B = fold; g.b_k = nd3; g.b_n = 1;
        g.C = U1; g.c_m = nd3; g.c_n = 1;
        g.alpha = one; g.accumulate = 0;
        CK(c, launch_zgemm(g, s));
        // U2[(p, l1)][d2][d3] = sum_l2 phi2[beta n_ev + l2][d2] U1[(p, l1, l2)][d3]
        g = ZgemmParams{};
        g.M = nd2; g.N = nd3; g.K = n_ev; g.batch = (long long)P_set * n_ev;
        g.A = p2 + (size_t)sp.pair_beta[pr] * n_ev * nd2; g.a_m = 1; g.a_k = nd2; g.a_b = 0;
        g.B = U1; g.b_k = nd3; g.b_n = 1; g.b_b = (long long)n_ev * nd3;
        g.C = U2; g.c_m = nd3; g.c_n = 1; g.c_b = (long long)nd2 * nd3;
        g.alpha = one; g.accumulate = 0;
        CK(c, launch_zgemm(g, s));
        // B[p][d1][(d2, d3)] (+)= sum_l1 phi1[alpha n_ev + l1][d1] U2[(p, l1)][(d2, d3)]
        g = ZgemmParams{};
        g.M = nd1; g.N = nd2 * nd3; g.K = n_ev; g.batch = P_set;
        g.A = p1 + (size_t)sp.pair_alpha[pr] * n_ev * nd1; g.a_m = 1; g.a_k = nd1; g.a_b = 0;
        g.B = U2; g.b_k = (long long)nd2 * nd3; g.b_n = 1; g.b_b = (long long)n_ev * nd2 * nd3;
        g.C = Bt + (size_t)p0 * nd1 * nd2 * nd3; g.c_m = (long long)nd2 * nd3; g.c_n = 1;
        g.c_b = (long long)nd1 * nd2 * nd3;
        g.alpha = one; g.accumulate = pr > 0;
        CK(c, launch_zgemm(g, s));
        launches += 4;
      }
    }
  }
  c->last_launches = launches;
  return BBLOCK_OK;
}

int bblock_compute_host(bblock_ctx* c, int n_t, const void* V, const void* phi1, const void* phi2,
                        const void* phi3, int nd1, int nd2, int nd3, const int32_t* momenta,
                        int n_mom, const int32_t* spin_idx, const double* spin_coeffs, int n_spin,
                        int coeff_per_mom, void* B_out, void* stream) {
  if (!c) return BBLOCK_ERR_INVALID_ARG;
  c->err.clear();
  if (n_t < 0) return fail(c, BBLOCK_ERR_INVALID_ARG, "n_t = %d < 0", n_t);
  int rc = validate_common(c, momenta, n_mom, spin_idx, spin_coeffs, n_spin, coeff_per_mom);
  if (rc) return rc;
  if (n_t == 0 || n_mom == 0) { c->last_launches = 0; c->last_waves = 0; return BBLOCK_OK; }
  if (!V || !phi1 || !phi2 || !phi3 || !B_out) return fail(c, BBLOCK_ERR_INVALID_ARG, "a data pointer is NULL");
  const int nds[3] = {nd1, nd2, nd3};
  for (int i = 0; i < 3; ++i)
    if (nds[i] < 1 || nds[i] > c->cfg.max_ndil)
      return fail(c, BBLOCK_ERR_INVALID_ARG, "nd%d = %d outside 1..max_ndil", i + 1, nds[i]);
  const size_t vb = sizeof(double2) * (size_t)n_t * c->cfg.n_ev * c->rows;
  size_t pb[3];
  for (int i = 0; i < 3; ++i) pb[i] = sizeof(double2) * (size_t)n_t * 4 * c->cfg.n_ev * nds[i];
  const size_t bb_ = sizeof(double2) * (size_t)n_t * n_mom * nd1 * nd2 * nd3;
  const size_t off[5] = {0, align_up(vb, 256), align_up(vb, 256) + align_up(pb[0], 256),
                         align_up(vb, 256) + align_up(pb[0], 256) + align_up(pb[1], 256),
                         align_up(vb, 256) + align_up(pb[0], 256) + align_up(pb[1], 256) + align_up(pb[2], 256)};
  CK(c, cudaSetDevice(c->cfg.device));
  rc = grow_device(c, &c->d_io, &c->io_cap, off[4] + align_up(bb_, 256));
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!c->copy_stream) CK(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  cudaStream_t cs = c->copy_stream;
  // Time slices are independent, so the call runs in chunks of them: every chunk's inputs
  // are enqueued at once on the copy stream, each chunk is computed on `stream` as soon as
  // its inputs have landed, and its blocks go back while later chunks compute. Only the
  // first chunk's inputs and the last chunk's blocks are exposed.
  const int n_chunks = std::min(n_t, c->opt_host_chunks > 0 ? c->opt_host_chunks : kHostChunks);
  std::vector<cudaEvent_t> ev(2 * n_chunks + 2, nullptr);
  for (auto& e : ev)
    if (!(e = take_event(c))) {
      for (auto x : ev) if (x) c->ev_pool.push_back(x);
      return fail(c, BBLOCK_ERR_CUDA, "cudaEventCreate failed");
    }
  auto give_back = [&] { for (auto x : ev) c->ev_pool.push_back(x); };
  auto t_of = [&](int k) { return (long long)n_t * k / n_chunks; };
  const size_t v_t = vb / n_t, b_t = bb_ / n_t;
  size_t p_t[3];
  for (int i = 0; i < 3; ++i) p_t[i] = pb[i] / n_t;
  const void* hp[3] = {phi1, phi2, phi3};
  // the staging may still be read by work the caller enqueued earlier on `stream`
  cudaError_t e = cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[0], 0);
  for (int k = 0; k < n_chunks && e == cudaSuccess; ++k) {
    const long long t0 = t_of(k), nt = t_of(k + 1) - t0;
    e = cudaMemcpyAsync(c->d_io + off[0] + t0 * v_t, static_cast<const char*>(V) + t0 * v_t,
                        nt * v_t, cudaMemcpyHostToDevice, cs);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(c->d_io + off[1 + i] + t0 * p_t[i],
                          static_cast<const char*>(hp[i]) + t0 * p_t[i], nt * p_t[i],
                          cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1 + k], cs);
  }
  if (e != cudaSuccess) {
    cudaStreamSynchronize(cs);
    give_back();
    return cuda_fail(c, e, "enqueueing the input copies");
  }
  int launches = 0, waves = 0;
  for (int k = 0; k < n_chunks && rc == BBLOCK_OK && e == cudaSuccess; ++k) {
    const long long t0 = t_of(k), nt = t_of(k + 1) - t0;
    e = cudaStreamWaitEvent(s, ev[1 + k], 0);
    if (e != cudaSuccess) break;
    rc = bblock_compute(c, (int)nt, c->d_io + off[0] + t0 * v_t, c->d_io + off[1] + t0 * p_t[0],
                        c->d_io + off[2] + t0 * p_t[1], c->d_io + off[3] + t0 * p_t[2], nd1, nd2,
                        nd3, momenta, n_mom, spin_idx, spin_coeffs, n_spin, coeff_per_mom,
                        c->d_io + off[4] + t0 * b_t, stream);
    if (rc) break;
    launches += c->last_launches;
    waves += c->last_waves;
    e = cudaEventRecord(ev[1 + n_chunks + k], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[1 + n_chunks + k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(static_cast<char*>(B_out) + t0 * b_t, c->d_io + off[4] + t0 * b_t,
                          nt * b_t, cudaMemcpyDeviceToHost, cs);
  }
  // both streams drain before the call returns, also after an error
  cudaError_t e2 = cudaEventRecord(ev[2 * n_chunks + 1], cs);
  if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, ev[2 * n_chunks + 1], 0);
  cudaError_t e3 = cudaStreamSynchronize(cs);
  cudaError_t e4 = cudaStreamSynchronize(s);
  give_back();
  if (rc) return rc;
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = e3;
  if (e == cudaSuccess) e = e4;
  if (e != cudaSuccess) return cuda_fail(c, e, "pipelined host copies");
  c->last_launches = launches;
  c->last_waves = waves;
  return BBLOCK_OK;
}

size_t bblock_workspace_bytes(const bblock_ctx* c) {
  if (!c) return 0;
  return c->ws_cap + c->phase_cap + c->mom_cap + c->tab_cap + c->io_cap + sizeof(int);
}

int bblock_last_launch_count(const bblock_ctx* c) { return c ? c->last_launches : 0; }
int bblock_last_wave_count(const bblock_ctx* c) { return c ? c->last_waves : 0; }
int bblock_last_path(const bblock_ctx* c) { return c ? c->last_path : -1; }

int bblock_autotune(bblock_ctx* c, int n_t, const void* V, const void* phi1, const void* phi2,
                    const void* phi3, int nd1, int nd2, int nd3, const int32_t* momenta,
                    int n_mom, const int32_t* spin_idx, const double* spin_coeffs, int n_spin,
                    void* B_out, void* stream, bblock_costmodel* model, int top_k, int repeats,
                    bblock_tune_entry* report, int max_report, int* n_report) {
  if (!c) return BBLOCK_ERR_INVALID_ARG;
  c->err.clear();
  if (n_report) *n_report = 0;
  if (n_t < 1 || n_mom < 1 || repeats < 1 || (model && top_k < 1) || (max_report > 0 && !report))
    return fail(c, BBLOCK_ERR_INVALID_ARG, "bad autotune arguments");
  int rc = validate_common(c, momenta, n_mom, spin_idx, spin_coeffs, n_spin, 0);
  if (rc) return rc;
  SpinPlan sp;
  rc = plan_spins(c, spin_idx, spin_coeffs, n_spin, 0, n_mom, &sp);
  if (rc) return rc;
  const int nd[3] = {nd1, nd2, nd3};
  // candidate option sets
  std::vector<std::array<int, 3>> cand;
  const CallPlan base = plan_call(c, n_t, nd, n_mom, sp.n_pairs, 0, 0, 0);
  const int a = std::max(1, base.n_slab);
  const int slab_choices[4] = {0, std::max(1, a / 2), 2 * a, 4 * a};
  if (fp64_like(c->cfg)) {
    for (int k = 0; k < 4; ++k) cand.push_back({0, 0, slab_choices[k]});
  } else {
    const int form = tc_form_of(c->cfg);
    const bool pairs_on = form == TC_F16_3 && !c->opt_checks && c->opt_wait_us == 0 &&
                          c->opt_tc_cluster != 1;
    // drain intervals: up to 3 stages; the FP16 form up to 2, which keeps its per-block
    // errors well inside 1e-6 (3 stages measured 8.9e-7 at the largest of 162 full-size
    // blocks, 2 stages about 7e-7, for 6 % more time)
    const int max_chunk = form == TC_F16_3 ? 2 : 3;
    for (int nc = 16; nc <= tc_max_nc(form, pairs_on); nc += 16)
      for (int ch = 1; ch <= max_chunk; ++ch)
        for (int k = 0; k < 3; ++k) cand.push_back({nc, ch, slab_choices[k]});
  }
  const int n_c = (int)cand.size();
  std::vector<bblock_tune_entry> ent(n_c);
  std::vector<float> feat((size_t)n_c * BBLOCK_TUNE_FEATURES);
  for (int i = 0; i < n_c; ++i) {
    ent[i].nc = cand[i][0];
    ent[i].chunk = cand[i][1];
    ent[i].slabs = cand[i][2];
    const CallPlan pl = plan_call(c, n_t, nd, n_mom, sp.n_pairs, cand[i][0], cand[i][1], cand[i][2]);
    tune_features(c, n_t, nd, n_mom, sp.n_pairs, pl, ent[i].features);
    std::copy(ent[i].features, ent[i].features + BBLOCK_TUNE_FEATURES, feat.begin() + (size_t)i * BBLOCK_TUNE_FEATURES);
    ent[i].predicted = 0.f;
    ent[i].ms = -1.0;
  }
  std::vector<int> order(n_c);
  for (int i = 0; i < n_c; ++i) order[i] = i;
  int n_time = n_c;
  if (model) {
    std::vector<float> pred(n_c);
    rc = bblock_costmodel_predict(model, feat.data(), n_c, pred.data());
    if (rc) return fail(c, rc, "cost-model prediction failed");
    for (int i = 0; i < n_c; ++i) ent[i].predicted = pred[i];
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return pred[x] < pred[y]; });
    n_time = std::min(top_k, n_c);
  }
  // time the chosen candidates with plain launches
  const int saved[4] = {c->opt_graphs, c->opt_tc_nc, c->opt_tc_chunk, c->opt_slabs};
  const bool saved_prof = c->prof;
  c->opt_graphs = 0;
  c->prof = false;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    rc = fail(c, BBLOCK_ERR_CUDA, "cudaEventCreate failed");
  }
  int best = -1;
  for (int r = 0; r < n_time && rc == BBLOCK_OK; ++r) {
    const int i = order[r];
    c->opt_tc_nc = cand[i][0];
    c->opt_tc_chunk = cand[i][1];
    c->opt_slabs = cand[i][2];
    std::vector<float> t;
    for (int k = 0; k <= repeats && rc == BBLOCK_OK; ++k) {
      if (k > 0) cudaEventRecord(e0, s);
      rc = bblock_compute(c, n_t, V, phi1, phi2, phi3, nd1, nd2, nd3, momenta, n_mom, spin_idx,
                          spin_coeffs, n_spin, 0, B_out, stream);
      if (rc == BBLOCK_OK && k > 0) {
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          cudaGetLastError();
          rc = fail(c, BBLOCK_ERR_CUDA, "timing failed");
        }
        t.push_back(ms);
      }
    }
    if (rc != BBLOCK_OK) break;
    std::sort(t.begin(), t.end());
    ent[i].ms = t[t.size() / 2];
    if (best < 0 || ent[i].ms < ent[best].ms) best = i;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->opt_graphs = saved[0];
  c->prof = saved_prof;
  if (rc == BBLOCK_OK && best >= 0) {
    c->opt_tc_nc = cand[best][0];
    c->opt_tc_chunk = cand[best][1];
    c->opt_slabs = cand[best][2];
  } else {
    c->opt_tc_nc = saved[1];
    c->opt_tc_chunk = saved[2];
    c->opt_slabs = saved[3];
  }
  drop_graph(c);
  c->last_sig.clear();
  const int n_out = std::min(max_report, n_c);
  for (int i = 0; i < n_out; ++i) report[i] = ent[i];
  if (n_report) *n_report = n_out;
  return rc;
}

int bblock_set_option(bblock_ctx* c, int option, int value) {
  if (!c) return BBLOCK_ERR_INVALID_ARG;
  switch (option) {
    case BBLOCK_OPT_GRAPHS:
      if (value != 0 && value != 1) break;
      c->opt_graphs = value;
      if (!value) drop_graph(c);
      return BBLOCK_OK;
    case BBLOCK_OPT_TC_NC:
      if (value != 0 && value != 16 && value != 32 && value != 48 &&
          !(c->cfg.precision == BBLOCK_FP16X3 && (value == 64 || value == 80)))
        break;
      c->opt_tc_nc = value;
      return BBLOCK_OK;
    case BBLOCK_OPT_TC_CHUNK:
      if (value < 0 || value > 8) break;
      c->opt_tc_chunk = value;
      return BBLOCK_OK;
    case BBLOCK_OPT_SLABS:
      if (value < 0 || value > 4096) break;
      c->opt_slabs = value;
      return BBLOCK_OK;
    case BBLOCK_OPT_CHECKS:
      if (value != 0 && value != 1) break;
      c->opt_checks = value;
      drop_graph(c);
      c->last_sig.clear();
      return BBLOCK_OK;
    case BBLOCK_OPT_WAVE_MB:
      if (value < 0) break;
      c->opt_wave_bytes = (size_t)value << 20;
      return BBLOCK_OK;
    case BBLOCK_OPT_WAIT_LIMIT_US:
      if (value < 0) break;
      c->opt_wait_us = value;
      drop_graph(c);            // the limit is a kernel parameter captured in the graph
      c->last_sig.clear();
      return BBLOCK_OK;
    case BBLOCK_OPT_FAIL_NEXT_ALLOC:
      if (value != 0 && value != 1) break;
      c->opt_fail_alloc = value;
      return BBLOCK_OK;
    case BBLOCK_OPT_TC_CLUSTER:
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 &&
          !(c->cfg.precision == BBLOCK_OZAKI && value == 3))
        break;
      c->opt_tc_cluster = value;
      return BBLOCK_OK;
    case BBLOCK_OPT_TC_ROWS:
      if (value < 0 || value > 2) break;
      c->opt_tc_rows = value;
      drop_graph(c);
      return BBLOCK_OK;
    case BBLOCK_OPT_TC_PROJECTION:
      if (value < 0 || value > 2) break;
      c->opt_tc_proj = value;
      return BBLOCK_OK;
    case BBLOCK_OPT_HOST_CHUNKS:
      if (value < 0 || value > 64) break;
      c->opt_host_chunks = value;
      return BBLOCK_OK;
    case BBLOCK_OPT_CORRUPT_CANARY:
      if (value != 0 && value != 1) break;
      c->opt_corrupt_canary = value;
      drop_graph(c);            // the hook acts on plain launches only
      c->last_sig.clear();
      return BBLOCK_OK;
    default:
      break;
  }
  return fail(c, BBLOCK_ERR_INVALID_ARG, "option %d does not take the value %d", option, value);
}

int bblock_get_option(const bblock_ctx* c, int option) {
  if (!c) return BBLOCK_ERR_INVALID_ARG;
  switch (option) {
    case BBLOCK_OPT_GRAPHS: return c->opt_graphs;
    case BBLOCK_OPT_TC_NC: return c->opt_tc_nc;
    case BBLOCK_OPT_TC_CHUNK: return c->opt_tc_chunk;
    case BBLOCK_OPT_SLABS: return c->opt_slabs;
    case BBLOCK_OPT_WAVE_MB: return (int)(c->opt_wave_bytes >> 20);
    case BBLOCK_OPT_WAIT_LIMIT_US: return c->opt_wait_us;
    case BBLOCK_OPT_FAIL_NEXT_ALLOC: return c->opt_fail_alloc;
    case BBLOCK_OPT_CORRUPT_CANARY: return c->opt_corrupt_canary;
    case BBLOCK_OPT_TC_CLUSTER: return c->opt_tc_cluster;
    case BBLOCK_OPT_HOST_CHUNKS: return c->opt_host_chunks;
    case BBLOCK_OPT_TC_PROJECTION: return c->opt_tc_proj;
    case BBLOCK_OPT_TC_ROWS: return c->opt_tc_rows;
    case BBLOCK_OPT_CHECKS: return c->opt_checks;
    default: return BBLOCK_ERR_INVALID_ARG;
  }
}

int bblock_profile_enable(bblock_ctx* c, int enable) {
  if (!c) return BBLOCK_ERR_INVALID_ARG;
  c->prof = enable != 0;
  return BBLOCK_OK;
}

int bblock_profile_read(bblock_ctx* c, bblock_kernel_stat* out, int max_entries, int* n_entries) {
  if (!c || (!out && max_entries > 0) || !n_entries) return BBLOCK_ERR_INVALID_ARG;
  double ms[K_COUNT] = {};
  int cnt[K_COUNT] = {};
  int rc = BBLOCK_OK;
  if (c->graph_pending) {
    cudaError_t e = harvest_graph_times(c);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "bblock_profile_read");
  }
  for (int k = 0; k < K_COUNT; ++k) {
    ms[k] += c->graph_ms[k];
    cnt[k] += c->graph_cnt[k];
    c->graph_ms[k] = 0.0;
    c->graph_cnt[k] = 0;
  }
  for (auto& t : c->timed) {
    float m = 0.f;
    cudaError_t e = cudaEventSynchronize(t.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&m, t.a, t.b);
    if (e != cudaSuccess && rc == BBLOCK_OK) rc = cuda_fail(c, e, "bblock_profile_read");
    ms[t.kind] += m;
    cnt[t.kind] += t.kernels;
    c->ev_pool.push_back(t.a);
    c->ev_pool.push_back(t.b);
  }
  c->timed.clear();
  int n = 0;
  for (int k = 0; k < K_COUNT; ++k) {
    if (!cnt[k]) continue;
    if (n < max_entries) {
      snprintf(out[n].name, sizeof(out[n].name), "%s", kKernelNames[k]);
      out[n].launches = cnt[k];
      out[n].total_ms = ms[k];
    }
    ++n;
  }
  *n_entries = n < max_entries ? n : max_entries;
  return rc;
}

}  // extern "C"
