// Mode-triplet ordering of Eq. (3) (Sec. 2, Eq. 4): the baryon block as
//   B[p][d1][d2][d3] = sum_s c_s sum_{l1 l2 l3} T[p][l1][l2][l3]
//                      phi1[alpha_s N_ev + l1][d1] phi2[beta_s N_ev + l2][d2] phi3[gamma_s N_ev + l3][d3]
// with the eigenvector mode triplet
//   T[p][l1][l2][l3] = sum_x e^{-ip.x} eps_abc V[l1][x][a] V[l2][x][b] V[l3][x][c].
//
// T is the contraction of Eq. (1) with q_i = V, i.e. with identity coefficients
// (phi = [I; 0; 0; 0]) and the single spin triple (0, 0, 0): the host computes it with the
// contraction kernels of the context's form. This file holds what the second step needs:
//   k_fill_identity   the identity coefficient matrix [4 N_ev][N_ev]
//   k_fold_phi        phi3' = sum_t w_t phi3[gamma_t N_ev + l][d]  (line-3 coefficients of one
//                     (alpha, beta) pair, as in the projection's fold)
//   k_zgemm           batched complex GEMM with arbitrary strides, FP64, for the three mode
//                     products T x3 phi3', x2 phi2, x1 phi1
#include "bblock_internal.h"

namespace bb {
namespace {

__global__ void k_fill_identity(double2* __restrict__ id, int n_ev) {
  const long long total = 4LL * n_ev * n_ev;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / n_ev, c = i - r * n_ev;
    id[i] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
}

__global__ void k_fold_phi(const double2* __restrict__ phi, int n_ev, int nd, FoldTerms terms,
                           double2* __restrict__ out) {
  const long long total = (long long)n_ev * nd;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long l = i / nd, d = i - l * nd;
    double re = 0.0, im = 0.0;
    for (int t = 0; t < terms.n; ++t) {
      const double2 f = phi[((long long)terms.row[t] * n_ev + l) * nd + d];
      const double2 w = terms.w[t];
      re = fma(w.x, f.x, fma(-w.y, f.y, re));
      im = fma(w.x, f.y, fma(w.y, f.x, im));
    }
    out[i] = make_double2(re, im);
  }
}

constexpr int ZBM = 64, ZBN = 32, ZBK = 16;

__global__ void __launch_bounds__(kThreads) k_zgemm(const ZgemmParams p) {
  __shared__ double2 As[ZBK][ZBM];
  __shared__ double2 Bs[ZBK][ZBN];
  const int m0 = blockIdx.x * ZBM, n0 = blockIdx.y * ZBN;
  const long long bt = blockIdx.z;
  const double2* __restrict__ A = p.A + bt * p.a_b;
  const double2* __restrict__ B = p.B + bt * p.b_b;
  double2* __restrict__ C = p.C + bt * p.c_b;
  const int tid = threadIdx.x, tn = tid % 8, tm = tid / 8;
  double2 acc[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = 0; k0 < p.K; k0 += ZBK) {
    for (int idx = tid; idx < ZBK * ZBM; idx += kThreads) {
      const int r = idx % ZBM, kk = idx / ZBM;
      const int m = m0 + r, k = k0 + kk;
      As[kk][r] = (m < p.M && k < p.K) ? A[(long long)m * p.a_m + (long long)k * p.a_k]
                                         : make_double2(0.0, 0.0);
    }
    for (int idx = tid; idx < ZBK * ZBN; idx += kThreads) {
      const int c = idx % ZBN, kk = idx / ZBN;
      const int n = n0 + c, k = k0 + kk;
      Bs[kk][c] = (n < p.N && k < p.K) ? B[(long long)k * p.b_k + (long long)n * p.b_n]
                                         : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < ZBK; ++kk) {
      double2 a[2], b[4];
#pragma unroll
      for (int i = 0; i < 2; ++i) a[i] = As[kk][tm + 32 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tn + 8 * j];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int m = m0 + tm + 32 * i;
    if (m >= p.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tn + 8 * j;
      if (n >= p.N) continue;
      double2& c = C[(long long)m * p.c_m + (long long)n * p.c_n];
      const double2 v = acc[i][j];
      double2 r = make_double2(p.alpha.x * v.x - p.alpha.y * v.y, p.alpha.x * v.y + p.alpha.y * v.x);
      if (p.accumulate) { r.x += c.x; r.y += c.y; }
      c = r;
    }
  }
}

int grid_for(long long total) {
  long long g = (total + kThreads - 1) / kThreads;
  return (int)(g < 1 ? 1 : (g > 65536 ? 65536 : g));
}

}  // namespace

cudaError_t launch_fill_identity(double2* id, int n_ev, cudaStream_t s) {
  k_fill_identity<<<grid_for(4LL * n_ev * n_ev), kThreads, 0, s>>>(id, n_ev);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_fold_phi(const double2* phi, int n_ev, int nd, const FoldTerms& terms,
                            double2* out, cudaStream_t s) {
  k_fold_phi<<<grid_for((long long)n_ev * nd), kThreads, 0, s>>>(phi, n_ev, nd, terms, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_zgemm(const ZgemmParams& p, cudaStream_t s) {
  if (p.M <= 0 || p.N <= 0 || p.batch <= 0) return cudaSuccess;
  for (long long b0 = 0; b0 < p.batch; b0 += 65535) {  // grid.z limit
    ZgemmParams q = p;
    q.A += b0 * p.a_b;
    q.B += b0 * p.b_b;
    q.C += b0 * p.c_b;
    q.batch = (int)(p.batch - b0 < 65535 ? p.batch - b0 : 65535);
    dim3 grid((p.M + ZBM - 1) / ZBM, (p.N + ZBN - 1) / ZBN, q.batch);
    k_zgemm<<<grid, kThreads, 0, s>>>(q);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace bb
