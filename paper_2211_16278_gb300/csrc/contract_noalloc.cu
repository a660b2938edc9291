// bblock_contract_noalloc: the FP64 contraction (fused diquark + colour singlet + momentum
// projection, then the fixed-order slab reduction) for callers that cannot allocate device
// memory. Its per-slab partial sums live in one file-scope __device__ array instead of a
// context workspace, so the entry point needs no context and calls no allocator.
#include <cstdio>
#include <mutex>

#include "../../include/bblock.h"
#include "bblock_internal.h"

namespace bb {
namespace {

// Fixed scratch for the per-slab partial blocks. Every device that loads the library
// holds this array for the life of the process.
constexpr size_t kNoallocScratchBytes = (size_t)BBLOCK_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) double2 g_noalloc_scratch[kNoallocScratchBytes / sizeof(double2)];

constexpr int kNaMaxP = 8;
constexpr int kNaMaxDevices = 64;

struct NoallocParams {
  const double2* q1;      // [4][X][3][nd1]
  const double2* q2;      // [4][X][3][nd2]
  const double2* q3;      // [4][X][3][nd3]
  double2* partial;       // device address of g_noalloc_scratch: [n_slab][P][nd1*nd2][nd3]
  int L, X, nd1, nd2, nd3;
  int m_tiles, n_tiles, n_slab, sites_per_slab;
  long long total_units;
  int n_pairs;
  int pair_alpha[kMaxPairs], pair_beta[kMaxPairs];
  int n_terms[kMaxPairs];
  int term_gamma[kMaxPairs][kMaxTerms];
  double2 term_w[kMaxPairs][kMaxTerms];
  int mom[kNaMaxP][3];
};

__device__ __forceinline__ double2 na_cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// Same arithmetic as k_contract_fp64 for one job; differences: the line fields are read
// per spin from the caller's [4][X][3][nd] arrays, the spin coefficients are folded into
// the third-quark tile while it is staged, and the phases are evaluated per site.
template <int P, int RN>
__global__ void __launch_bounds__(kThreads, 2)
k_contract_fp64_noalloc(const __grid_constant__ NoallocParams prm) {
  constexpr int RM = 2, MT = 16 * RM, NT = 16 * RN;
  extern __shared__ __align__(16) double smem[];
  const int np = prm.n_pairs;
  const int XC = np >= 16 ? 1 : 16 / np;
  const int KC = XC * np * 3;
  double* Ar = smem;
  double* Ai = Ar + KC * MT;
  double* As = Ai + KC * MT;
  double* Bc = As + KC * MT;
  double* Bd = Bc + KC * NT;
  double* Be = Bd + KC * NT;
  double2* ph = reinterpret_cast<double2*>(Be + KC * NT);
  const int tid = threadIdx.x, tn = tid % 16, tm = tid / 16;
  const int X = prm.X, L = prm.L;
  const int nd1 = prm.nd1, nd2 = prm.nd2, nd3 = prm.nd3, M = nd1 * nd2;

  for (long long u = blockIdx.x; u < prm.total_units; u += gridDim.x) {
    long long r = u;
    const int mt = (int)(r % prm.m_tiles);
    r /= prm.m_tiles;
    const int nt = (int)(r % prm.n_tiles);
    const int slab = (int)(r / prm.n_tiles);
    const int x_begin = slab * prm.sites_per_slab;
    const int x_end = min(X, x_begin + prm.sites_per_slab);

    double2 acc[RM][RN][P];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j)
#pragma unroll
        for (int p = 0; p < P; ++p) acc[i][j][p] = make_double2(0.0, 0.0);

    for (int xs = x_begin; xs < x_end; xs += XC) {
      for (int idx = tid; idx < XC * np * MT; idx += kThreads) {
        const int ml = idx % MT;
        const int t2 = idx / MT;
        const int pr = t2 % np, xc = t2 / np;
        const int x = xs + xc, m = mt * MT + ml;
        double2 dq0 = make_double2(0.0, 0.0), dq1 = dq0, dq2 = dq0;
        if (x < x_end && m < M) {
          const int d1 = m / nd2, d2 = m - d1 * nd2;
          const double2* u1 = prm.q1 + ((size_t)prm.pair_alpha[pr] * X + x) * 3 * nd1 + d1;
          const double2* v1 = prm.q2 + ((size_t)prm.pair_beta[pr] * X + x) * 3 * nd2 + d2;
          const double2 a0 = u1[0], a1 = u1[nd1], a2 = u1[2 * nd1];
          const double2 b0 = v1[0], b1 = v1[nd2], b2 = v1[2 * nd2];
          const double2 p12 = na_cmul(a1, b2), p21 = na_cmul(a2, b1);
          const double2 p20 = na_cmul(a2, b0), p02 = na_cmul(a0, b2);
          const double2 p01 = na_cmul(a0, b1), p10 = na_cmul(a1, b0);
          dq0 = make_double2(p12.x - p21.x, p12.y - p21.y);
          dq1 = make_double2(p20.x - p02.x, p20.y - p02.y);
          dq2 = make_double2(p01.x - p10.x, p01.y - p10.y);
        }
        const int k = (xc * np + pr) * 3;
        Ar[(k + 0) * MT + ml] = dq0.x; Ai[(k + 0) * MT + ml] = dq0.y; As[(k + 0) * MT + ml] = dq0.x + dq0.y;
        Ar[(k + 1) * MT + ml] = dq1.x; Ai[(k + 1) * MT + ml] = dq1.y; As[(k + 1) * MT + ml] = dq1.x + dq1.y;
        Ar[(k + 2) * MT + ml] = dq2.x; Ai[(k + 2) * MT + ml] = dq2.y; As[(k + 2) * MT + ml] = dq2.x + dq2.y;
      }
      for (int idx = tid; idx < KC * NT; idx += kThreads) {
        const int nl = idx % NT;
        const int k = idx / NT;
        const int c = k % 3, t2 = k / 3;
        const int pr = t2 % np, xc = t2 / np;
        const int x = xs + xc, n = nt * NT + nl;
        double2 b = make_double2(0.0, 0.0);
        if (x < x_end && n < nd3) {
          for (int t = 0; t < prm.n_terms[pr]; ++t) {
            const double2 f = prm.q3[(((size_t)prm.term_gamma[pr][t] * X + x) * 3 + c) * nd3 + n];
            const double2 w = prm.term_w[pr][t];
            b.x = fma(w.x, f.x, fma(-w.y, f.y, b.x));
            b.y = fma(w.x, f.y, fma(w.y, f.x, b.y));
          }
        }
        Bc[k * NT + nl] = b.x;
        Bd[k * NT + nl] = b.y - b.x;
        Be[k * NT + nl] = b.x + b.y;
      }
      for (int idx = tid; idx < XC * P; idx += kThreads) {
        const int p = idx % P, xc = idx / P;
        const int x = xs + xc;
        double2 e = make_double2(0.0, 0.0);
        if (x < x_end) {
          const long long x0 = x % L, x1 = (x / L) % L, x2 = x / ((long long)L * L);
          long long kk = prm.mom[p][0] * x0 + prm.mom[p][1] * x1 + prm.mom[p][2] * x2;
          kk %= L;
          if (kk < 0) kk += L;
          double sn, cs;
          sincospi(2.0 * (double)kk / (double)L, &sn, &cs);
          e = make_double2(cs, -sn);
        }
        ph[idx] = e;
      }
      __syncthreads();

      for (int xc = 0; xc < XC; ++xc) {
        double k1[RM][RN], k2[RM][RN], k3[RM][RN];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
          for (int j = 0; j < RN; ++j) k1[i][j] = k2[i][j] = k3[i][j] = 0.0;
        const int kbeg = xc * np * 3, kend = kbeg + np * 3;
        for (int k = kbeg; k < kend; ++k) {
          double ar[RM], ai[RM], as[RM], bc[RN], bd[RN], be[RN];
#pragma unroll
          for (int i = 0; i < RM; ++i) {
            ar[i] = Ar[k * MT + tm + 16 * i];
            ai[i] = Ai[k * MT + tm + 16 * i];
            as[i] = As[k * MT + tm + 16 * i];
          }
#pragma unroll
          for (int j = 0; j < RN; ++j) {
            bc[j] = Bc[k * NT + tn + 16 * j];
            bd[j] = Bd[k * NT + tn + 16 * j];
            be[j] = Be[k * NT + tn + 16 * j];
          }
#pragma unroll
          for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RN; ++j) {
              k1[i][j] = fma(bc[j], as[i], k1[i][j]);
              k2[i][j] = fma(ar[i], bd[j], k2[i][j]);
              k3[i][j] = fma(ai[i], be[j], k3[i][j]);
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const double2 e = ph[xc * P + p];
#pragma unroll
          for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RN; ++j) {
              const double sr = k1[i][j] - k3[i][j], si = k1[i][j] + k2[i][j];
              acc[i][j][p].x = fma(e.x, sr, fma(-e.y, si, acc[i][j][p].x));
              acc[i][j][p].y = fma(e.x, si, fma(e.y, sr, acc[i][j][p].y));
            }
        }
      }
      __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < RM; ++i) {
      const int m = mt * MT + tm + 16 * i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < RN; ++j) {
        const int n = nt * NT + tn + 16 * j;
        if (n >= nd3) continue;
#pragma unroll
        for (int p = 0; p < P; ++p)
          prm.partial[(((size_t)slab * P + p) * M + m) * nd3 + n] = acc[i][j][p];
      }
    }
  }
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

size_t na_smem_bytes(int P, int rn, int n_pairs) {
  const int xc = fp64_sites_per_chunk(n_pairs);
  const int kc = xc * n_pairs * 3;
  return sizeof(double) * 3 * (size_t)kc * (32 + 16 * rn) + sizeof(double2) * xc * P;
}

template <int P, int RN>
cudaError_t na_launch(const NoallocParams& prm, int grid, cudaStream_t s) {
  const size_t smem = na_smem_bytes(P, RN, prm.n_pairs);
  cudaError_t e = cudaFuncSetAttribute(k_contract_fp64_noalloc<P, RN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_contract_fp64_noalloc<P, RN><<<grid, kThreads, smem, s>>>(prm);
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
  prm.q1 = static_cast<const double2*>(q1);
  prm.q2 = static_cast<const double2*>(q2);
  prm.q3 = static_cast<const double2*>(q3);
  prm.L = L;
  prm.X = L * L * L;
  prm.nd1 = nd1; prm.nd2 = nd2; prm.nd3 = nd3;
  for (int p = 0; p < n_mom; ++p)
    for (int i = 0; i < 3; ++i) prm.mom[p][i] = momenta[3 * p + i];
  // spin triples -> (alpha, beta) pairs with the coefficient-weighted gamma terms
  for (int s = 0; s < n_spin; ++s) {
    const int al = spin_idx[3 * s], be = spin_idx[3 * s + 1], ga = spin_idx[3 * s + 2];
    if (al < 0 || al > 3 || be < 0 || be > 3 || ga < 0 || ga > 3)
      return na_fail(err, err_len, BBLOCK_ERR_INVALID_ARG, "spin index outside 0..3");
    int pr = -1;
    for (int k = 0; k < prm.n_pairs; ++k)
      if (prm.pair_alpha[k] == al && prm.pair_beta[k] == be) pr = k;
    if (pr < 0) {
      pr = prm.n_pairs++;
      prm.pair_alpha[pr] = al;
      prm.pair_beta[pr] = be;
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
  prm.m_tiles = (nd1 * nd2 + 31) / 32;
  prm.n_tiles = (nd3 + 16 * tl.rn - 1) / (16 * tl.rn);
  const size_t per = (size_t)n_mom * nd1 * nd2 * nd3;
  const size_t max_slabs_fit = kNoallocScratchBytes / (per * sizeof(double2));
  if (max_slabs_fit < 1)
    return na_fail(err, err_len, BBLOCK_ERR_TOO_LARGE,
                   "n_mom*nd1*nd2*nd3*16 bytes exceeds the static scratch of this entry point");

  // one-time set-up on this device: device address of the static scratch
  {
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_addr[dev]) {
      void* addr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess || !addr) {
        cudaGetLastError();
        return na_fail(err, err_len, BBLOCK_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed");
      }
      g_na_addr[dev] = addr;
    }
    prm.partial = static_cast<double2*>(g_na_addr[dev]);
  }

  int num_sms = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return na_fail(err, err_len, BBLOCK_ERR_CUDA, "device query failed");
  }
  const int xc = fp64_sites_per_chunk(prm.n_pairs);
  const int grid_cap = 2 * num_sms;
  const long long tiles = (long long)prm.m_tiles * prm.n_tiles;
  long long want = (4LL * grid_cap + tiles - 1) / tiles;
  long long n_slab = want;
  if (n_slab > (long long)max_slabs_fit) n_slab = (long long)max_slabs_fit;
  if (n_slab > (prm.X + xc - 1) / xc) n_slab = (prm.X + xc - 1) / xc;
  if (n_slab < 1) n_slab = 1;
  int sps = (int)((prm.X + n_slab - 1) / n_slab);
  sps = (sps + xc - 1) / xc * xc;
  prm.sites_per_slab = sps;
  prm.n_slab = (prm.X + sps - 1) / sps;
  prm.total_units = tiles * prm.n_slab;
  const int grid = (int)(prm.total_units < grid_cap ? prm.total_units : grid_cap);

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = na_dispatch(prm, n_mom, tl.rn, grid, s);
  if (e == cudaSuccess) {
    long long bx = ((long long)per + kThreads - 1) / kThreads;
    if (bx > 4096) bx = 4096;
    k_reduce_noalloc<<<(unsigned)bx, kThreads, 0, s>>>(prm.partial, static_cast<double2*>(B_out),
                                                       (long long)per, prm.n_slab);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    if (err && err_len) snprintf(err, err_len, "launch failed: %s", cudaGetErrorString(e));
    return BBLOCK_ERR_CUDA;
  }
  return BBLOCK_OK;
}
