// The FP64 contraction body (fused diquark + colour singlet + momentum projection, Eq. 1/3,
// Algorithm 1's diq / singlet / phase steps) shared by the context path (k_contract_fp64)
// and the allocation-free entry point (bblock_contract_noalloc). The two differ only in
// where a unit's job, a third-quark element and a phase come from, which a source policy
// supplies:
//   const ContractJob& job(long long u)             the job of work unit u
//   double2 third(const ContractJob&, pr, x, c, n)  folded third quark of pair pr at site x,
//                                                   colour c, dilution index n
//   double2 phase(int p, int x)                     e^{-i p.x} of the launch's momentum p
//
// Work unit = (job, slab of sites, 16*RM (d1,d2) pairs, 16*RN d3 columns). Per chunk of XC
// sites the CTA stages in shared memory
//   A[k][m] = diquark  (q1_alpha x q2_beta)_c (x) for pair index m = d1*nd2 + d2,
//   B[k][n] = third quark of the pair at (x, c, d3 = n),
// with k = (site, pair, colour). Each thread then owns RM x RN (m, n) outputs and per site
//   singlet = sum_{pair, c} A[k][m] * B[k][n]          (three-multiplication form)
//   acc[p] += e^{-i p.x} * singlet                      for the P momenta of the launch,
// and writes its sums as the unit's partial block (slab-major, reduced in index order).
#pragma once

#include "bblock_internal.h"

namespace bb {
namespace fp64c {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}

__device__ __forceinline__ int find_job(const ContractJob* jobs, int n_jobs, long long u) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int P, int RM, int RN, class Src>
__device__ __forceinline__ void contract_body(const ContractParams& prm, const Src& src) {
  constexpr int MT = 16 * RM, NT = 16 * RN;
  extern __shared__ __align__(16) double smem[];
  const int np = prm.n_pairs;
  const int XC = np >= 16 ? 1 : 16 / np;
  const int KC = XC * np * 3;
  double* __restrict__ Ar = smem;
  double* __restrict__ Ai = Ar + KC * MT;
  double* __restrict__ As = Ai + KC * MT;
  double* __restrict__ Bc = As + KC * MT;
  double* __restrict__ Bd = Bc + KC * NT;
  double* __restrict__ Be = Bd + KC * NT;
  double2* __restrict__ ph = reinterpret_cast<double2*>(Be + KC * NT);

  const int tid = threadIdx.x, tn = tid % 16, tm = tid / 16;
  const int X = prm.X;

  for (long long u = blockIdx.x; u < prm.total_units; u += gridDim.x) {
    const ContractJob& J = src.job(u);
    const int nd1 = J.nd1, nd2 = J.nd2, nd3 = J.nd3;
    const int M = nd1 * nd2;
    long long r = u - J.unit_begin;
    const int mt = (int)(r % J.m_tiles);
    r /= J.m_tiles;
    const int nt = (int)(r % J.n_tiles);
    const int slab = (int)(r / J.n_tiles);
    if (slab >= prm.n_slab) {  // inconsistent job table: flag it, skip the unit
      if (tid == 0 && prm.status) atomicOr(prm.status, kStatusBadJob);
      continue;
    }
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
      // --- diquark tile: A[(xc, pair, c)][m]
      for (int idx = tid; idx < XC * np * MT; idx += kThreads) {
        const int ml = idx % MT;
        const int t2 = idx / MT;
        const int pr = t2 % np, xc = t2 / np;
        const int x = xs + xc, m = mt * MT + ml;
        double2 dq0 = make_double2(0.0, 0.0), dq1 = dq0, dq2 = dq0;
        if (x < x_end && m < M) {
          const int d1 = m / nd2, d2 = m - d1 * nd2;
          const double2* u1 = J.q1[prm.a_slot[pr]] + (size_t)x * 3 * nd1 + d1;
          const double2* v1 = J.q2[prm.b_slot[pr]] + (size_t)x * 3 * nd2 + d2;
          const double2 u0 = u1[0], uu1 = u1[nd1], u2 = u1[2 * nd1];
          const double2 v0 = v1[0], vv1 = v1[nd2], v2 = v1[2 * nd2];
          dq0 = csub(cmul(uu1, v2), cmul(u2, vv1));   // eps_{120}, eps_{210}
          dq1 = csub(cmul(u2, v0), cmul(u0, v2));     // eps_{201}, eps_{021}
          dq2 = csub(cmul(u0, vv1), cmul(uu1, v0));   // eps_{012}, eps_{102}
        }
        const int k = (xc * np + pr) * 3;
        Ar[(k + 0) * MT + ml] = dq0.x; Ai[(k + 0) * MT + ml] = dq0.y; As[(k + 0) * MT + ml] = dq0.x + dq0.y;
        Ar[(k + 1) * MT + ml] = dq1.x; Ai[(k + 1) * MT + ml] = dq1.y; As[(k + 1) * MT + ml] = dq1.x + dq1.y;
        Ar[(k + 2) * MT + ml] = dq2.x; Ai[(k + 2) * MT + ml] = dq2.y; As[(k + 2) * MT + ml] = dq2.x + dq2.y;
      }
      // --- third quark tile: B[(xc, pair, c)][n]
      for (int idx = tid; idx < KC * NT; idx += kThreads) {
        const int nl = idx % NT;
        const int k = idx / NT;
        const int c = k % 3, t2 = k / 3;
        const int pr = t2 % np, xc = t2 / np;
        const int x = xs + xc, n = nt * NT + nl;
        double2 b = make_double2(0.0, 0.0);
        if (x < x_end && n < nd3) b = src.third(J, pr, x, c, n);
        Bc[k * NT + nl] = b.x;
        Bd[k * NT + nl] = b.y - b.x;
        Be[k * NT + nl] = b.x + b.y;
      }
      // --- phases of the chunk's sites
      for (int idx = tid; idx < XC * P; idx += kThreads) {
        const int p = idx % P, xc = idx / P;
        const int x = xs + xc;
        ph[idx] = x < x_end ? src.phase(p, x) : make_double2(0.0, 0.0);
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
          J.partial[(((size_t)slab * prm.P_total + prm.p0 + p) * M + m) * nd3 + n] = acc[i][j][p];
      }
    }
  }
}

}  // namespace fp64c
}  // namespace bb
