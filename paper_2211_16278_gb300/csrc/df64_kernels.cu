// Double-float form of the fused diquark + colour singlet + momentum projection (Eq. 1/3).
//
// GB300 executes IEEE double at 1/64 of the FP32 rate, and the FP64 contraction already
// runs at that pipe's roofline. This kernel computes the same sums in double-float
// arithmetic (dfloat.cuh: h + l, FP32 pairs, error-free products and sums, about 48
// significant bits) on the FP32 pipe, and converts to FP64 only for the per-slab partial
// blocks, which the FP64 slab reduction sums in a fixed order.
//
// Work decomposition, tiles and shared-memory layout are those of k_contract_fp64 (one
// (job, d1d2 tile, d3 tile, site slab) unit per CTA iteration, the diquark tile built per
// chunk of sites and reused for every d3, the spin-pair sum inside the colour singlet, the
// three-multiplication complex product for the singlet), with each double replaced by a
// double-float of the same 8 bytes. Accumulators are renormalised once per site chunk, so
// their low parts never grow beyond a few ulp of the high parts.
#include "bblock_internal.h"
#include "dfloat.cuh"

namespace bb {
namespace {

__device__ __forceinline__ int df_find_job(const ContractJob* jobs, int n_jobs, long long u) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ dcomplex load_dc(const double2* field, size_t i) {
  const float4 v = reinterpret_cast<const float4*>(field)[i];
  return dcomplex{dfloat{v.x, v.y}, dfloat{v.z, v.w}};
}

__device__ __forceinline__ void store_df(float2* a, int i, dfloat v) { a[i] = make_float2(v.h, v.l); }
__device__ __forceinline__ dfloat load_df(const float2* a, int i) {
  const float2 v = a[i];
  return dfloat{v.x, v.y};
}

template <int P, int RM, int RN>
__global__ void __launch_bounds__(kThreads, 2) k_contract_df(const __grid_constant__ ContractParams prm) {
  constexpr int MT = 16 * RM, NT = 16 * RN;
  extern __shared__ __align__(16) float2 smem_df[];
  const int np = prm.n_pairs;
  const int XC = np >= 16 ? 1 : 16 / np;
  const int KC = XC * np * 3;
  float2* __restrict__ Ar = smem_df;
  float2* __restrict__ Ai = Ar + KC * MT;
  float2* __restrict__ As = Ai + KC * MT;
  float2* __restrict__ Bc = As + KC * MT;
  float2* __restrict__ Bd = Bc + KC * NT;
  float2* __restrict__ Be = Bd + KC * NT;
  float4* __restrict__ ph = reinterpret_cast<float4*>(Be + KC * NT);

  const int tid = threadIdx.x, tn = tid % 16, tm = tid / 16;
  const int X = prm.X;

  for (long long u = blockIdx.x; u < prm.total_units; u += gridDim.x) {
    const ContractJob& J = prm.jobs[df_find_job(prm.jobs, prm.n_jobs, u)];
    const int nd1 = J.nd1, nd2 = J.nd2, nd3 = J.nd3;
    const int M = nd1 * nd2;
    long long r = u - J.unit_begin;
    const int mt = (int)(r % J.m_tiles);
    r /= J.m_tiles;
    const int nt = (int)(r % J.n_tiles);
    const int slab = (int)(r / J.n_tiles);
    if (slab >= prm.n_slab) {  // inconsistent job table: flag it, skip the unit
      if (tid == 0) atomicOr(prm.status, kStatusBadJob);
      continue;
    }
    const int x_begin = slab * prm.sites_per_slab;
    const int x_end = min(X, x_begin + prm.sites_per_slab);

    dfloat acc_r[RM][RN][P], acc_i[RM][RN][P];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j)
#pragma unroll
        for (int p = 0; p < P; ++p) acc_r[i][j][p] = acc_i[i][j][p] = df_zero();

    for (int xs = x_begin; xs < x_end; xs += XC) {
      // --- diquark tile: A[(xc, pair, c)][m]
      for (int idx = tid; idx < XC * np * MT; idx += kThreads) {
        const int ml = idx % MT;
        const int t2 = idx / MT;
        const int pr = t2 % np, xc = t2 / np;
        const int x = xs + xc, m = mt * MT + ml;
        dcomplex dq[3];
        if (x < x_end && m < M) {
          const int d1 = m / nd2, d2 = m - d1 * nd2;
          const double2* uf = J.q1[prm.a_slot[pr]];
          const double2* vf = J.q2[prm.b_slot[pr]];
          const size_t ub = (size_t)x * 3 * nd1 + d1, vb = (size_t)x * 3 * nd2 + d2;
          const dcomplex u0 = load_dc(uf, ub), u1 = load_dc(uf, ub + nd1), u2 = load_dc(uf, ub + 2 * nd1);
          const dcomplex v0 = load_dc(vf, vb), v1 = load_dc(vf, vb + nd2), v2 = load_dc(vf, vb + 2 * nd2);
          dq[0] = dc_sub(dc_mul(u1, v2), dc_mul(u2, v1));   // eps_{120}, eps_{210}
          dq[1] = dc_sub(dc_mul(u2, v0), dc_mul(u0, v2));   // eps_{201}, eps_{021}
          dq[2] = dc_sub(dc_mul(u0, v1), dc_mul(u1, v0));   // eps_{012}, eps_{102}
        } else {
          dq[0] = dq[1] = dq[2] = dcomplex{df_zero(), df_zero()};
        }
        const int k = (xc * np + pr) * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int o = (k + c) * MT + ml;
          store_df(Ar, o, dq[c].re);
          store_df(Ai, o, dq[c].im);
          store_df(As, o, df_norm(df_add(dq[c].re, dq[c].im)));
        }
      }
      // --- third quark tile: B[(xc, pair, c)][n]
      for (int idx = tid; idx < KC * NT; idx += kThreads) {
        const int nl = idx % NT;
        const int k = idx / NT;
        const int c = k % 3, t2 = k / 3;
        const int pr = t2 % np, xc = t2 / np;
        const int x = xs + xc, n = nt * NT + nl;
        dcomplex b{df_zero(), df_zero()};
        if (x < x_end && n < nd3) b = load_dc(J.q3[pr], ((size_t)x * 3 + c) * nd3 + n);
        store_df(Bc, k * NT + nl, b.re);
        store_df(Bd, k * NT + nl, df_norm(df_sub(b.im, b.re)));
        store_df(Be, k * NT + nl, df_norm(df_add(b.re, b.im)));
      }
      // --- phases of the chunk's sites (the table is FP64; converted once per chunk)
      for (int idx = tid; idx < XC * P; idx += kThreads) {
        const int p = idx % P, xc = idx / P;
        const int x = xs + xc;
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x < x_end) {
          const dcomplex z = dc_from_double2(prm.phase[(size_t)(prm.p0 + p) * X + x]);
          e = make_float4(z.re.h, z.re.l, z.im.h, z.im.l);
        }
        ph[idx] = e;
      }
      __syncthreads();

      for (int xc = 0; xc < XC; ++xc) {
        dfloat k1[RM][RN], k2[RM][RN], k3[RM][RN];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
          for (int j = 0; j < RN; ++j) k1[i][j] = k2[i][j] = k3[i][j] = df_zero();
        const int kbeg = xc * np * 3, kend = kbeg + np * 3;
        for (int k = kbeg; k < kend; ++k) {
          dfloat ar[RM], ai[RM], as[RM], bc[RN], bd[RN], be[RN];
#pragma unroll
          for (int i = 0; i < RM; ++i) {
            ar[i] = load_df(Ar, k * MT + tm + 16 * i);
            ai[i] = load_df(Ai, k * MT + tm + 16 * i);
            as[i] = load_df(As, k * MT + tm + 16 * i);
          }
#pragma unroll
          for (int j = 0; j < RN; ++j) {
            bc[j] = load_df(Bc, k * NT + tn + 16 * j);
            bd[j] = load_df(Bd, k * NT + tn + 16 * j);
            be[j] = load_df(Be, k * NT + tn + 16 * j);
          }
          // three-multiplication form: re = k1 - k3, im = k1 + k2 with
          // k1 = c (a + b), k2 = a (d - c), k3 = b (c + d) for (a + ib)(c + id)
#pragma unroll
          for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RN; ++j) {
              df_fma(k1[i][j], bc[j], as[i]);
              df_fma(k2[i][j], ar[i], bd[j]);
              df_fma(k3[i][j], ai[i], be[j]);
            }
        }
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
          for (int j = 0; j < RN; ++j) {
            const dfloat sr = df_sub(k1[i][j], k3[i][j]), si = df_add(k1[i][j], k2[i][j]);
#pragma unroll
            for (int p = 0; p < P; ++p) {
              const float4 ev = ph[xc * P + p];
              const dfloat er{ev.x, ev.y}, ei{ev.z, ev.w};
              df_fma(acc_r[i][j][p], er, sr);
              df_fms(acc_r[i][j][p], ei, si);
              df_fma(acc_i[i][j][p], er, si);
              df_fma(acc_i[i][j][p], ei, sr);
            }
          }
      }
      // renormalise once per chunk of sites
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j)
#pragma unroll
          for (int p = 0; p < P; ++p) {
            acc_r[i][j][p] = df_norm(acc_r[i][j][p]);
            acc_i[i][j][p] = df_norm(acc_i[i][j][p]);
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
          J.partial[(((size_t)slab * prm.P_total + prm.p0 + p) * M + m) * nd3 + n] =
              make_double2(df_to_double(acc_r[i][j][p]), df_to_double(acc_i[i][j][p]));
      }
    }
  }
}

template <int P, int RN>
cudaError_t launch_df_p(const ContractParams& prm, int grid, cudaStream_t s) {
  // same layout as the FP64 tiles: every double becomes a float2 of the same size
  const size_t smem = fp64_contract_smem_bytes(P, RN, prm.n_pairs);
  cudaError_t e = cudaFuncSetAttribute(k_contract_df<P, 2, RN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_contract_df<P, 2, RN><<<grid, kThreads, smem, s>>>(prm);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_contract_df(const ContractParams& prm, int P, int rn, int grid, cudaStream_t s) {
  if (prm.total_units == 0) return cudaSuccess;
  if (rn == 2) {
    switch (P) {
      case 1: return launch_df_p<1, 2>(prm, grid, s);
      case 2: return launch_df_p<2, 2>(prm, grid, s);
      case 3: return launch_df_p<3, 2>(prm, grid, s);
      case 4: return launch_df_p<4, 2>(prm, grid, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (P) {
    case 1: return launch_df_p<1, 1>(prm, grid, s);
    case 2: return launch_df_p<2, 1>(prm, grid, s);
    case 3: return launch_df_p<3, 1>(prm, grid, s);
    case 4: return launch_df_p<4, 1>(prm, grid, s);
    case 5: return launch_df_p<5, 1>(prm, grid, s);
    case 6: return launch_df_p<6, 1>(prm, grid, s);
    case 7: return launch_df_p<7, 1>(prm, grid, s);
    case 8: return launch_df_p<8, 1>(prm, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bb
