// FP64 form of the baryon-block hot path on sm_103a.
//
//   k_phase_table     e^{-i p.x} for integer momenta (Eq. 1/3; the paper precomputes the
//                     phase once per momentum set instead of using an FFT, Sec. 3)
//   k_project_fp64    Eq. (2) as a complex GEMM, q = V^T Phi, one launch for every field
//   k_contract_fp64   fused diquark + colour singlet + momentum projection (Eq. 1/3,
//                     Algorithm 1's diq / singlet / phase-GEMM steps), site-split into slabs
//   k_reduce_slabs    fixed-order sum of the per-slab partial blocks
//
// GB300 runs IEEE double at 1/64 of the FP32 rate (measured: DFMA ~1.19 TFLOP/s, DMMA
// ~1.04 TFLOP/s), so these kernels are bound by the FP64 pipe and are written to
// execute as few FP64 operations as possible:
//   * complex products inside the long sums use the three-multiplication form
//     (re = k1 - k3, im = k1 + k2 with k1 = c(a+b), k2 = a(d-c), k3 = b(c+d));
//     the operand-side sums are formed once when a tile is staged in shared memory;
//   * the spin-pair sum is taken inside the colour singlet, before the phase (the
//     phase does not depend on the spin pair), so each (d1,d2,d3,x) costs
//     9*n_pairs + 2 + 4*P FP64 operations instead of n_pairs*(12 + 4P);
//   * the diquark of a (d1,d2) tile is built once per site and reused for every d3.
#include "bblock_internal.h"
#include "fp64_contract.cuh"

namespace bb {

// ------------------------------------------------------------------ phases

__global__ void k_phase_table(int L, int n_mom, const int* __restrict__ mom,
                              double2* __restrict__ ph, float2* __restrict__ ph_f) {
  const long long X = (long long)L * L * L;
  const long long total = X * n_mom;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i / X);
    const long long x = i - (long long)p * X;
    const long long x0 = x % L, x1 = (x / L) % L, x2 = x / ((long long)L * L);
    long long k = mom[3 * p] * x0 + mom[3 * p + 1] * x1 + mom[3 * p + 2] * x2;
    k %= L;
    if (k < 0) k += L;
    double s, c;
    sincospi(2.0 * (double)k / (double)L, &s, &c);
    ph[i] = make_double2(c, -s);
    if (ph_f) ph_f[i] = make_float2((float)c, (float)-s);
  }
}

cudaError_t launch_phase_table(int L, int n_mom, const int* d_mom, double2* ph, float2* ph_f,
                               cudaStream_t s) {
  const long long total = (long long)L * L * L * n_mom;
  if (total == 0) return cudaSuccess;
  const int grid = (int)((total + kThreads - 1) / kThreads < 65536 ? (total + kThreads - 1) / kThreads : 65536);
  k_phase_table<<<grid, kThreads, 0, s>>>(L, n_mom, d_mom, ph, ph_f);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ projection (Eq. 2)

constexpr int PBM = 64, PBN = 32, PBK = 16;

__global__ void __launch_bounds__(kThreads) k_project_fp64(const ProjField* __restrict__ fields,
                                                           int rows, int n_ev) {
  __shared__ double Ar[PBK][PBM], Ai[PBK][PBM], As[PBK][PBM];
  __shared__ double Bc[PBK][PBN], Bd[PBK][PBN], Be[PBK][PBN];
  const ProjField& F = fields[blockIdx.z];
  const int nd = F.nd;
  const int n0 = blockIdx.y * PBN;
  if (n0 >= nd) return;
  const int m0 = blockIdx.x * PBM;
  const int tid = threadIdx.x, tn = tid % 8, tm = tid / 8;
  const int n_terms = F.n_terms;

  double k1[2][4], k2[2][4], k3[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) k1[i][j] = k2[i][j] = k3[i][j] = 0.0;

  for (int kb = 0; kb < n_ev; kb += PBK) {
    for (int idx = tid; idx < PBK * PBM; idx += kThreads) {
      const int r = idx % PBM, kk = idx / PBM;
      const int l = kb + kk, row = m0 + r;
      double2 v = make_double2(0.0, 0.0);
      if (l < n_ev && row < rows) v = F.V[(size_t)l * rows + row];
      Ar[kk][r] = v.x;
      Ai[kk][r] = v.y;
      As[kk][r] = v.x + v.y;
    }
    for (int idx = tid; idx < PBK * PBN; idx += kThreads) {
      const int c = idx % PBN, kk = idx / PBN;
      const int l = kb + kk, col = n0 + c;
      double2 b = make_double2(0.0, 0.0);
      if (l < n_ev && col < nd) {
        for (int t = 0; t < n_terms; ++t) {
          const double2 f = F.phi[(size_t)(F.row_off[t] + l) * nd + col];
          const double2 w = F.w[t];
          b.x = fma(w.x, f.x, fma(-w.y, f.y, b.x));
          b.y = fma(w.x, f.y, fma(w.y, f.x, b.y));
        }
      }
      Bc[kk][c] = b.x;
      Bd[kk][c] = b.y - b.x;
      Be[kk][c] = b.x + b.y;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < PBK; ++kk) {
      double ar[2], ai[2], as[2], bc[4], bd[4], be[4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        ar[i] = Ar[kk][tm + 32 * i];
        ai[i] = Ai[kk][tm + 32 * i];
        as[i] = As[kk][tm + 32 * i];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        bc[j] = Bc[kk][tn + 8 * j];
        bd[j] = Bd[kk][tn + 8 * j];
        be[j] = Be[kk][tn + 8 * j];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          k1[i][j] = fma(bc[j], as[i], k1[i][j]);
          k2[i][j] = fma(ar[i], bd[j], k2[i][j]);
          k3[i][j] = fma(ai[i], be[j], k3[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int row = m0 + tm + 32 * i;
    if (row >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = n0 + tn + 8 * j;
      if (col < nd)
        F.q[(size_t)row * nd + col] = make_double2(k1[i][j] - k3[i][j], k1[i][j] + k2[i][j]);
    }
  }
}

cudaError_t launch_project_fp64(const ProjField* d_fields, int n_fields, int rows, int n_ev,
                                int max_nd, cudaStream_t s) {
  if (n_fields == 0 || rows == 0) return cudaSuccess;
  for (int f0 = 0; f0 < n_fields; f0 += 65535) {  // grid.z limit
    const int nf = n_fields - f0 < 65535 ? n_fields - f0 : 65535;
    dim3 grid((rows + PBM - 1) / PBM, (max_nd + PBN - 1) / PBN, nf);
    k_project_fp64<<<grid, kThreads, 0, s>>>(d_fields + f0, rows, n_ev);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------ contraction (Eq. 1/3)
//
// The body is fp64c::contract_body (fp64_contract.cuh); here the work units come from the
// context's job table, the third quark from the coefficient-folded line-3 fields and the
// phases from the cached table.

size_t fp64_contract_smem_bytes(int P, int rn, int n_pairs) {
  const int xc = fp64_sites_per_chunk(n_pairs);
  const int kc = xc * n_pairs * 3;
  return sizeof(double) * 3 * (size_t)kc * (16 * 2 + 16 * rn) + sizeof(double2) * xc * P;
}

struct TableSource {
  const ContractParams* prm;
  __device__ const ContractJob& job(long long u) const {
    return prm->jobs[fp64c::find_job(prm->jobs, prm->n_jobs, u)];
  }
  __device__ double2 third(const ContractJob& J, int pr, int x, int c, int n) const {
    return J.q3[pr][((size_t)x * 3 + c) * J.nd3 + n];
  }
  __device__ double2 phase(int p, int x) const {
    return prm->phase[(size_t)(prm->p0 + p) * prm->X + x];
  }
};

template <int P, int RM, int RN>
__global__ void __launch_bounds__(kThreads, 2) k_contract_fp64(const __grid_constant__ ContractParams prm) {
  fp64c::contract_body<P, RM, RN>(prm, TableSource{&prm});
}

template <int P, int RN>
static cudaError_t launch_contract_p(const ContractParams& prm, int grid, cudaStream_t s) {
  const size_t smem = fp64_contract_smem_bytes(P, RN, prm.n_pairs);
  cudaError_t e = cudaFuncSetAttribute(k_contract_fp64<P, 2, RN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_contract_fp64<P, 2, RN><<<grid, kThreads, smem, s>>>(prm);
  note_launch();
  return cudaGetLastError();
}

// (P, RN) instantiations: RN = 2 only for P <= 4 (register budget of 128 per thread);
// RN = 1 up to P = 10, the largest momentum group that runs without spills.
cudaError_t launch_contract_fp64(const ContractParams& prm, int P, int rn, int grid,
                                 cudaStream_t s) {
  if (prm.total_units == 0) return cudaSuccess;
  if (rn == 2) {
    switch (P) {
      case 1: return launch_contract_p<1, 2>(prm, grid, s);
      case 2: return launch_contract_p<2, 2>(prm, grid, s);
      case 3: return launch_contract_p<3, 2>(prm, grid, s);
      case 4: return launch_contract_p<4, 2>(prm, grid, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (P) {
    case 1: return launch_contract_p<1, 1>(prm, grid, s);
    case 2: return launch_contract_p<2, 1>(prm, grid, s);
    case 3: return launch_contract_p<3, 1>(prm, grid, s);
    case 4: return launch_contract_p<4, 1>(prm, grid, s);
    case 5: return launch_contract_p<5, 1>(prm, grid, s);
    case 6: return launch_contract_p<6, 1>(prm, grid, s);
    case 7: return launch_contract_p<7, 1>(prm, grid, s);
    case 8: return launch_contract_p<8, 1>(prm, grid, s);
    case 9: return launch_contract_p<9, 1>(prm, grid, s);
    case 10: return launch_contract_p<10, 1>(prm, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int fp64_contract_ctas_per_sm(int P, int rn, int n_pairs) {
  const size_t smem = fp64_contract_smem_bytes(P, rn, n_pairs);
  int dev = 0, per_sm_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  int by_smem = (int)(per_sm_smem / (smem + 1024));
  int ctas = by_smem < 2 ? by_smem : 2;  // __launch_bounds__(256, 2)
  return ctas < 1 ? 1 : ctas;
}

// ------------------------------------------------------------------ slab reduction

__global__ void k_reduce_slabs(const ContractJob* __restrict__ jobs, int n_slab, int P_total) {
  const ContractJob& J = jobs[blockIdx.y];
  const long long per = (long long)P_total * J.nd1 * J.nd2 * J.nd3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per;
       e += (long long)gridDim.x * blockDim.x) {
    double2 s = J.partial[e];
    for (int sl = 1; sl < n_slab; ++sl) {   // fixed order: the result is run-to-run identical
      const double2 v = J.partial[(size_t)sl * per + e];
      s.x += v.x;
      s.y += v.y;
    }
    J.B[e] = s;
  }
}

cudaError_t launch_reduce_slabs(const ContractJob* d_jobs, int n_jobs, int n_slab, int P_total,
                                long long max_elems, cudaStream_t s) {
  if (n_jobs == 0 || max_elems == 0) return cudaSuccess;
  long long bx = (max_elems + kThreads - 1) / kThreads;
  if (bx > 4096) bx = 4096;
  dim3 grid((unsigned)bx, n_jobs);
  k_reduce_slabs<<<grid, kThreads, 0, s>>>(d_jobs, n_slab, P_total);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bb
