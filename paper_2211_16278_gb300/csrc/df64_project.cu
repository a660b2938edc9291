// Double-float form, input side: conversion of the complex128 inputs to double-float
// planes, and Eq. (2) as a complex GEMM in double-float arithmetic on the FP32 pipe.
//
//   k_convert_df    every input array of a call (each job's V and phi_i) to float4
//                   elements (re.h, re.l, im.h, im.l), one launch over a segment table; the
//                   only FP64 arithmetic of the step besides the phase table and the slab
//                   reduction (one subtraction per component)
//   k_project_df    q = V^T Phi with the line-3 spin-coefficient fold, the same tiles and
//                   three-multiplication form as the FP64 projection, each double replaced
//                   by a double-float; writes the float4 fields the double-float
//                   contraction reads
#include "bblock_internal.h"
#include "dfloat.cuh"

namespace bb {
namespace {

__global__ void k_convert_df(const DfConvSeg* __restrict__ segs) {
  const DfConvSeg sg = segs[blockIdx.y];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < sg.n;
       i += (long long)gridDim.x * blockDim.x) {
    const dcomplex z = dc_from_double2(sg.src[i]);
    sg.dst[i] = make_float4(z.re.h, z.re.l, z.im.h, z.im.l);
  }
}

constexpr int DBM = 64, DBN = 32, DBK = 16;

__device__ __forceinline__ dcomplex ld4(const float4* p, size_t i) {
  const float4 v = p[i];
  return dcomplex{dfloat{v.x, v.y}, dfloat{v.z, v.w}};
}

__global__ void __launch_bounds__(kThreads, 2) k_project_df(const ProjField* __restrict__ fields,
                                                            int rows, int n_ev) {
  __shared__ float2 Ar[DBK][DBM], Ai[DBK][DBM], As[DBK][DBM];
  __shared__ float2 Bc[DBK][DBN], Bd[DBK][DBN], Be[DBK][DBN];
  __shared__ dcomplex wt[kMaxTerms];
  const ProjField& F = fields[blockIdx.z];
  const int nd = F.nd;
  const int n0 = blockIdx.y * DBN;
  if (n0 >= nd) return;
  const int m0 = blockIdx.x * DBM;
  const int tid = threadIdx.x, tn = tid % 8, tm = tid / 8;
  const int n_terms = F.n_terms;
  // this field's inputs are double-float planes (k_convert_df), its output too
  const float4* __restrict__ V = reinterpret_cast<const float4*>(F.V);
  const float4* __restrict__ phi = reinterpret_cast<const float4*>(F.phi);
  if (tid < n_terms) wt[tid] = dc_from_double2(F.w[tid]);
  __syncthreads();

  dfloat k1[2][4], k2[2][4], k3[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) k1[i][j] = k2[i][j] = k3[i][j] = df_zero();

  for (int kb = 0; kb < n_ev; kb += DBK) {
    for (int idx = tid; idx < DBK * DBM; idx += kThreads) {
      const int r = idx % DBM, kk = idx / DBM;
      const int l = kb + kk, row = m0 + r;
      dcomplex v{df_zero(), df_zero()};
      if (l < n_ev && row < rows) v = ld4(V, (size_t)l * rows + row);
      Ar[kk][r] = make_float2(v.re.h, v.re.l);
      Ai[kk][r] = make_float2(v.im.h, v.im.l);
      const dfloat s = df_norm(df_add(v.re, v.im));
      As[kk][r] = make_float2(s.h, s.l);
    }
    for (int idx = tid; idx < DBK * DBN; idx += kThreads) {
      const int c = idx % DBN, kk = idx / DBN;
      const int l = kb + kk, col = n0 + c;
      dfloat br = df_zero(), bi = df_zero();
      if (l < n_ev && col < nd) {
        for (int t = 0; t < n_terms; ++t) {
          const dcomplex f = ld4(phi, (size_t)(F.row_off[t] + l) * nd + col);
          const dcomplex w = wt[t];
          df_fma(br, w.re, f.re);
          df_fms(br, w.im, f.im);
          df_fma(bi, w.re, f.im);
          df_fma(bi, w.im, f.re);
        }
        br = df_norm(br);
        bi = df_norm(bi);
      }
      Bc[kk][c] = make_float2(br.h, br.l);
      const dfloat d = df_norm(df_sub(bi, br)), e = df_norm(df_add(br, bi));
      Bd[kk][c] = make_float2(d.h, d.l);
      Be[kk][c] = make_float2(e.h, e.l);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < DBK; ++kk) {
      dfloat ar[2], ai[2], as[2], bc[4], bd[4], be[4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float2 a = Ar[kk][tm + 32 * i], b = Ai[kk][tm + 32 * i], s = As[kk][tm + 32 * i];
        ar[i] = dfloat{a.x, a.y};
        ai[i] = dfloat{b.x, b.y};
        as[i] = dfloat{s.x, s.y};
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 c = Bc[kk][tn + 8 * j], d = Bd[kk][tn + 8 * j], e = Be[kk][tn + 8 * j];
        bc[j] = dfloat{c.x, c.y};
        bd[j] = dfloat{d.x, d.y};
        be[j] = dfloat{e.x, e.y};
      }
      // three-multiplication form: re = k1 - k3, im = k1 + k2 (see the FP64 projection)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          df_fma(k1[i][j], bc[j], as[i]);
          df_fma(k2[i][j], ar[i], bd[j]);
          df_fma(k3[i][j], ai[i], be[j]);
        }
    }
    // renormalise once per K block
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        k1[i][j] = df_norm(k1[i][j]);
        k2[i][j] = df_norm(k2[i][j]);
        k3[i][j] = df_norm(k3[i][j]);
      }
    __syncthreads();
  }
  float4* __restrict__ q = reinterpret_cast<float4*>(F.q);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int row = m0 + tm + 32 * i;
    if (row >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = n0 + tn + 8 * j;
      if (col >= nd) continue;
      const dfloat re = df_norm(df_sub(k1[i][j], k3[i][j]));
      const dfloat im = df_norm(df_add(k1[i][j], k2[i][j]));
      q[(size_t)row * nd + col] = make_float4(re.h, re.l, im.h, im.l);
    }
  }
}

}  // namespace

cudaError_t launch_convert_df(const DfConvSeg* d_segs, int n_segs, long long max_n,
                              cudaStream_t s) {
  if (n_segs == 0 || max_n == 0) return cudaSuccess;
  for (int s0 = 0; s0 < n_segs; s0 += 65535) {  // grid.y limit
    const int ns = n_segs - s0 < 65535 ? n_segs - s0 : 65535;
    long long bx = (max_n + kThreads - 1) / kThreads;
    if (bx > 1024) bx = 1024;
    dim3 grid((unsigned)bx, ns);
    k_convert_df<<<grid, kThreads, 0, s>>>(d_segs + s0);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_project_df(const ProjField* d_fields, int n_fields, int rows, int n_ev,
                              int max_nd, cudaStream_t s) {
  if (n_fields == 0 || rows == 0) return cudaSuccess;
  for (int f0 = 0; f0 < n_fields; f0 += 65535) {  // grid.z limit
    const int nf = n_fields - f0 < 65535 ? n_fields - f0 : 65535;
    dim3 grid((rows + DBM - 1) / DBM, (max_nd + DBN - 1) / DBN, nf);
    k_project_df<<<grid, kThreads, 0, s>>>(d_fields + f0, rows, n_ev);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace bb
