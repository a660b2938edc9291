// bblock_contract_noalloc: the FP64 contraction (fused diquark + colour singlet + momentum
// projection, then the fixed-order slab reduction) for callers that cannot allocate device
// memory. Its per-slab partial sums live in one file-scope __device__ array instead of a
// context workspace, so the entry point needs no context and calls no allocator.
#include <cstdio>
#include <mutex>

#include "../../include/bblock.h"
#include "bblock_internal.h"
#include "fp64_contract.cuh"

namespace bb {
namespace {

// Fixed scratch for the per-slab partial blocks. Every device that loads the library
// holds this array for the life of the process.
constexpr size_t kNoallocScratchBytes = (size_t)BBLOCK_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) double2 g_noalloc_scratch[kNoallocScratchBytes / sizeof(double2)];

constexpr int kNaMaxP = 8;
constexpr int kNaMaxDevices = 64;

// The launch: the shared FP64 contraction body's parameters (one job, embedded below; no
// status word) plus what this entry point takes instead of a context's tables.
struct NoallocParams {
  ContractParams base;    // jobs = nullptr, status = nullptr, P_total = P, p0 = 0
  ContractJob job;        // q1/q2 slots = spins 0..3 of the caller's arrays; partial = scratch
  const double2* q3;      // [4][X][3][nd3]
  int L;
  int n_terms[kMaxPairs];
  int term_gamma[kMaxPairs][kMaxTerms];
  double2 term_w[kMaxPairs][kMaxTerms];
  int mom[kNaMaxP][3];
};

// Where the shared body's inputs come from without a context: the single job of the
// launch, the third quark folded with its pair's spin coefficients while the tile is
// staged, and the phase evaluated per site from the integer momentum ((n.x) mod L in
// integers, then sincospi).
struct NoallocSource {
  const NoallocParams* np;
  __device__ const ContractJob& job(long long) const { return np->job; }
  __device__ double2 third(const ContractJob& J, int pr, int x, int c, int n) const {
    const int X = np->base.X;
    double2 b = make_double2(0.0, 0.0);
    for (int t = 0; t < np->n_terms[pr]; ++t) {
      const double2 f = np->q3[(((size_t)np->term_gamma[pr][t] * X + x) * 3 + c) * J.nd3 + n];
      const double2 w = np->term_w[pr][t];
      b.x = fma(w.x, f.x, fma(-w.y, f.y, b.x));
      b.y = fma(w.x, f.y, fma(w.y, f.x, b.y));
    }
    return b;
  }
  __device__ double2 phase(int p, int x) const {
    const int L = np->L;
    const long long x0 = x % L, x1 = (x / L) % L, x2 = x / ((long long)L * L);
    long long kk = np->mom[p][0] * x0 + np->mom[p][1] * x1 + np->mom[p][2] * x2;
    kk %= L;
    if (kk < 0) kk += L;
    double sn, cs;
    sincospi(2.0 * (double)kk / (double)L, &sn, &cs);
    return make_double2(cs, -sn);
  }
};

template <int P, int RN>
__global__ void __launch_bounds__(kThreads, 2)
k_contract_fp64_noalloc(const __grid_constant__ NoallocParams prm) {
  fp64c::contract_body<P, 2, RN>(prm.base, NoallocSource{&prm});
}

// B[e] = sum over slabs of partial[slab][e], slabs in index order.
__global__ void k_reduce_noalloc(const double2* __restrict__ partial, double2* __restrict__ B,
                                 long long per, int n_slab) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per;
       e += (long long)gridDim.x * blockDim.x) {
    double2 s = partial[e];
    for (int sl = 1; sl < n_slab; ++sl) {
      const double2 v = partial[(size_t)sl * per + e];
      s.x += v.x;
      s.y += v.y;
    }
    B[e] = s;
  }
}


template <int P, int RN>
cudaError_t na_launch(const NoallocParams& prm, int grid, cudaStream_t s) {
  const size_t smem = fp64_contract_smem_bytes(P, RN, prm.base.n_pairs);
  cudaError_t e = cudaFuncSetAttribute(k_contract_fp64_noalloc<P, RN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_contract_fp64_noalloc<P, RN><<<grid, kThreads, smem, s>>>(prm);
  note_launch();
  return cudaGetLastError();
}

cudaError_t na_dispatch(const NoallocParams& prm, int P, int rn, int grid, cudaStream_t s) {
  if (rn == 2) {
    switch (P) {
      case 1: return na_launch<1, 2>(prm, grid, s);
      case 2: return na_launch<2, 2>(prm, grid, s);
      case 3: return na_launch<3, 2>(prm, grid, s);
      case 4: return na_launch<4, 2>(prm, grid, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (P) {
    case 5: return na_launch<5, 1>(prm, grid, s);
    case 6: return na_launch<6, 1>(prm, grid, s);
    case 7: return na_launch<7, 1>(prm, grid, s);
    case 8: return na_launch<8, 1>(prm, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

// Per-device device address of g_noalloc_scratch. In host code the array's name stands
// for a host-side shadow, not device memory, so the address must be looked up with
// cudaGetSymbolAddress once per device while that device is current.
std::mutex g_na_mu;
void* g_na_addr[kNaMaxDevices] = {};
void* g_na_ctx[kNaMaxDevices] = {};   // the CUDA context each address was looked up in

// The calling thread's current CUDA context (driver API, reached through the runtime's
// entry-point query so that the library needs no link against libcuda), or nullptr.
void* na_current_context() {
  typedef int (*CtxGetCurrentFn)(void**);
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(f);
    else
      cudaGetLastError();
  }
  void* ctx = nullptr;
  if (fn && fn(&ctx) != 0) ctx = nullptr;
  return ctx;
}

int na_fail(char* err, size_t err_len, int code, const char* msg) {
  if (err && err_len) snprintf(err, err_len, "%s", msg);
  return code;
}

bool na_device_ptr(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

}  // namespace
}  // namespace bb

using namespace bb;

extern "C" int bblock_contract_noalloc(int L, const void* q1, const void* q2, const void* q3,
                                       int nd1, int nd2, int nd3, const int32_t* momenta,
                                       int n_mom, const int32_t* spin_idx,
                                       const double* spin_coeffs, int n_spin, void* B_out,
                                       void* stream, char* err, size_t err_len) {
  if (err && err_len) err[0] = '\0';
  if (L < 1 || L > 128) return na_fail(err, err_len, BBLOCK_ERR_INVALID_ARG, "L outside 1..128");
  if (nd1 < 1 || nd2 < 1 || nd3 < 1 || nd1 > 256 || nd2 > 256 || nd3 > 256)
    return na_fail(err, err_len, BBLOCK_ERR_INVALID_ARG, "dilution sizes must be 1..256");
  if (n_mom < 0 || n_mom > kNaMaxP)
    return na_fail(err, err_len, BBLOCK_ERR_TOO_LARGE, "n_mom must be 0..8 for this entry point");
  if (n_spin < 1 || n_spin > 64 || !spin_idx || !spin_coeffs || (n_mom > 0 && !momenta))
    return na_fail(err, err_len, BBLOCK_ERR_INVALID_ARG, "bad momentum or spin arguments");
  if (n_mom == 0) return BBLOCK_OK;
  if (!q1 || !q2 || !q3 || !B_out)
    return na_fail(err, err_len, BBLOCK_ERR_INVALID_ARG, "a data pointer is NULL");
  const void* ptrs[4] = {q1, q2, q3, B_out};
  for (const void* p : ptrs)
    if ((reinterpret_cast<uintptr_t>(p) & 15u) != 0)
      return na_fail(err, err_len, BBLOCK_ERR_INVALID_ARG, "a data pointer is not 16-byte aligned");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
    cudaGetLastError();
    return na_fail(err, err_len, BBLOCK_ERR_CUDA, "no usable current CUDA device");
  }
  for (const void* p : ptrs)
    if (!na_device_ptr(p, dev))
      return na_fail(err, err_len, BBLOCK_ERR_INVALID_ARG,
                     "q1, q2, q3 and B_out must be device memory of the current device");

  NoallocParams prm{};
  ContractParams& base = prm.base;
  ContractJob& job = prm.job;
  const int X = L * L * L;
  // the q1 / q2 slots are the four spins of the caller's arrays; a pair names its spins
  for (int a = 0; a < 4; ++a) {
    job.q1[a] = static_cast<const double2*>(q1) + (size_t)a * X * 3 * nd1;
    job.q2[a] = static_cast<const double2*>(q2) + (size_t)a * X * 3 * nd2;
  }
  job.nd1 = nd1; job.nd2 = nd2; job.nd3 = nd3;
  job.unit_begin = 0;
  prm.q3 = static_cast<const double2*>(q3);
  prm.L = L;
  base.X = X;
  base.n_jobs = 1;
  base.P_total = n_mom;
  base.p0 = 0;
  for (int p = 0; p < n_mom; ++p)
    for (int i = 0; i < 3; ++i) prm.mom[p][i] = momenta[3 * p + i];
  // spin triples -> (alpha, beta) pairs with the coefficient-weighted gamma terms
  for (int s = 0; s < n_spin; ++s) {
    const int al = spin_idx[3 * s], be = spin_idx[3 * s + 1], ga = spin_idx[3 * s + 2];
    if (al < 0 || al > 3 || be < 0 || be > 3 || ga < 0 || ga > 3)
      return na_fail(err, err_len, BBLOCK_ERR_INVALID_ARG, "spin index outside 0..3");
    int pr = -1;
    for (int k = 0; k < base.n_pairs; ++k)
      if (base.a_slot[k] == al && base.b_slot[k] == be) pr = k;
    if (pr < 0) {
      pr = base.n_pairs++;
      base.a_slot[pr] = al;
      base.b_slot[pr] = be;
    }
    int t = -1;
    for (int k = 0; k < prm.n_terms[pr]; ++k)
      if (prm.term_gamma[pr][k] == ga) t = k;
    if (t < 0) {
      t = prm.n_terms[pr]++;
      prm.term_gamma[pr][t] = ga;
      prm.term_w[pr][t] = make_double2(0.0, 0.0);
    }
    prm.term_w[pr][t].x += spin_coeffs[2 * s];
    prm.term_w[pr][t].y += spin_coeffs[2 * s + 1];
  }

  const Fp64Tile tl = fp64_tile_for(n_mom);
  job.m_tiles = (nd1 * nd2 + 16 * tl.rm - 1) / (16 * tl.rm);
  job.n_tiles = (nd3 + 16 * tl.rn - 1) / (16 * tl.rn);
  const size_t per = (size_t)n_mom * nd1 * nd2 * nd3;
  const size_t max_slabs_fit = kNoallocScratchBytes / (per * sizeof(double2));
  if (max_slabs_fit < 1)
    return na_fail(err, err_len, BBLOCK_ERR_TOO_LARGE,
                   "n_mom*nd1*nd2*nd3*16 bytes exceeds the static scratch of this entry point");

  // set-up once per device and CUDA context: the device address of the static scratch
  // (looked up again if the device's context was reset and recreated since)
  {
    std::lock_guard<std::mutex> lock(g_na_mu);
    void* ctx = na_current_context();
    if (!g_na_addr[dev] || ctx != g_na_ctx[dev]) {
      void* addr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess || !addr) {
        cudaGetLastError();
        return na_fail(err, err_len, BBLOCK_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed");
      }
      g_na_addr[dev] = addr;
      g_na_ctx[dev] = ctx;
    }
    job.partial = static_cast<double2*>(g_na_addr[dev]);
  }

  int num_sms = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return na_fail(err, err_len, BBLOCK_ERR_CUDA, "device query failed");
  }
  const int xc = fp64_sites_per_chunk(base.n_pairs);
  const int grid_cap = 2 * num_sms;
  const long long tiles = (long long)job.m_tiles * job.n_tiles;
  long long want = (4LL * grid_cap + tiles - 1) / tiles;
  long long n_slab = want;
  if (n_slab > (long long)max_slabs_fit) n_slab = (long long)max_slabs_fit;
  if (n_slab > (X + xc - 1) / xc) n_slab = (X + xc - 1) / xc;
  if (n_slab < 1) n_slab = 1;
  int sps = (int)((X + n_slab - 1) / n_slab);
  sps = (sps + xc - 1) / xc * xc;
  base.sites_per_slab = sps;
  base.n_slab = (X + sps - 1) / sps;
  base.total_units = tiles * base.n_slab;
  const int grid = (int)(base.total_units < grid_cap ? base.total_units : grid_cap);

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = na_dispatch(prm, n_mom, tl.rn, grid, s);
  if (e == cudaSuccess) {
    long long bx = ((long long)per + kThreads - 1) / kThreads;
    if (bx > 4096) bx = 4096;
    k_reduce_noalloc<<<(unsigned)bx, kThreads, 0, s>>>(job.partial, static_cast<double2*>(B_out),
                                                       (long long)per, base.n_slab);
    note_launch();
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    if (err && err_len) snprintf(err, err_len, "launch failed: %s", cudaGetErrorString(e));
    return BBLOCK_ERR_CUDA;
  }
  return BBLOCK_OK;
}
