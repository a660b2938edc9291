// Eq. (2) for the tensor-core forms: q = V^T Phi in FP32 with FP32 accumulation.
//
//   k_convert_f32   the input-conversion step of the mixed forms: every complex128 input
//                   array of a call (each job's V and phi_i) to complex64, once per call,
//                   in one launch over a segment table
//   k_project_f32   q = V^T Phi from the FP32 copies; the spin coefficients of line 3 are
//                   folded into the staged Phi tile as in the FP64 projection. One CTA
//                   computes a 128-row x 32-column tile of one field (4 x 4 adjacent
//                   outputs per thread, the next K block's loads in flight while the
//                   current one is multiplied); the grid runs the fields of a row tile back
//                   to back (blockIdx.x = field) so that the V tile they share is served
//                   from L2. Optionally it also records the largest |Re| or |Im| of each
//                   field it writes (the FP16 form's operand scales).
#include "bblock_internal.h"

namespace bb {

constexpr int FBM = 128, FBN = 32, FBK = 16;

__device__ __forceinline__ bool f32_idx_ok(long long i, long long n, int code, int field,
                                           unsigned long long* dbg, int* status) {
  if (i >= 0 && i < n) return true;
  if (atomicCAS(dbg, 0ull, (unsigned long long)code) == 0ull) {
    dbg[1] = (unsigned long long)field;
    dbg[2] = (unsigned long long)i;
    dbg[3] = (unsigned long long)n;
  }
  atomicOr(status, kStatusBadIndex);
  return false;
}

__global__ void __launch_bounds__(kThreads) k_project_f32(const ProjFieldF* __restrict__ fields,
                                                          int rows, int n_ev, int checks,
                                                          unsigned long long* dbg, int* status) {
  __shared__ __align__(16) float2 As[FBK][FBM];
  __shared__ __align__(16) float2 Bs[FBK][FBN];
  const ProjFieldF& F = fields[blockIdx.x];
  const int nd = F.nd;
  const int n0 = blockIdx.z * FBN;
  if (n0 >= nd) return;
  const int m0 = blockIdx.y * FBM;
  // 32 x 8 threads; each owns 4 adjacent rows x 4 adjacent columns, read from shared memory
  // as two 16-byte loads per operand and k
  const int tid = threadIdx.x, tn = tid % 8, tm = tid / 8;
  const int n_terms = F.n_terms;
  float2 wt[kMaxTerms];
  for (int t = 0; t < kMaxTerms; ++t)
    wt[t] = make_float2((float)F.w[t].x, (float)F.w[t].y);
  // staging of one K block: 8 V elements and 2 folded Phi elements per thread
  constexpr int kAPer = FBK * FBM / kThreads, kBPer = FBK * FBN / kThreads;
  float2 va[kAPer], vb[kBPer];
  auto load_block = [&](int kb) {
#pragma unroll
    for (int j = 0; j < kAPer; ++j) {
      const int idx = tid + kThreads * j;
      const int r = idx % FBM, kk = idx / FBM;
      const int l = kb + kk, row = m0 + r;
      float2 v = make_float2(0.f, 0.f);
      if (l < n_ev && row < rows &&
          (!checks || f32_idx_ok((long long)l * rows + row, (long long)n_ev * rows, 11, blockIdx.x, dbg, status)))
        v = F.V[(size_t)l * rows + row];
      va[j] = v;
    }
#pragma unroll
    for (int j = 0; j < kBPer; ++j) {
      const int idx = tid + kThreads * j;
      const int c = idx % FBN, kk = idx / FBN;
      const int l = kb + kk, col = n0 + c;
      float2 b = make_float2(0.f, 0.f);
      if (l < n_ev && col < nd) {
        for (int t = 0; t < n_terms; ++t) {
          if (checks && !f32_idx_ok((long long)(F.row_off[t] + l) * nd + col, 4LL * n_ev * nd, 12,
                                    blockIdx.x, dbg, status))
            continue;
          const float2 f = F.phi[(size_t)(F.row_off[t] + l) * nd + col];
          b.x = fmaf(wt[t].x, f.x, fmaf(-wt[t].y, f.y, b.x));
          b.y = fmaf(wt[t].x, f.y, fmaf(wt[t].y, f.x, b.y));
        }
      }
      vb[j] = b;
    }
  };
  auto store_block = [&] {
#pragma unroll
    for (int j = 0; j < kAPer; ++j) {
      const int idx = tid + kThreads * j;
      As[idx / FBM][idx % FBM] = va[j];
    }
#pragma unroll
    for (int j = 0; j < kBPer; ++j) {
      const int idx = tid + kThreads * j;
      Bs[idx / FBN][idx % FBN] = vb[j];
    }
  };
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  load_block(0);
  for (int kb = 0; kb < n_ev; kb += FBK) {
    store_block();
    __syncthreads();
    // the next block's global loads are in flight while this block is multiplied
    if (kb + FBK < n_ev) load_block(kb + FBK);
#pragma unroll 4
    for (int kk = 0; kk < FBK; ++kk) {
      const float4* ar = reinterpret_cast<const float4*>(&As[kk][4 * tm]);
      const float4* br = reinterpret_cast<const float4*>(&Bs[kk][4 * tn]);
      const float4 a01 = ar[0], a23 = ar[1], b01 = br[0], b23 = br[1];
      const float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w),
                           make_float2(a23.x, a23.y), make_float2(a23.z, a23.w)};
      const float2 b[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w),
                           make_float2(b23.x, b23.y), make_float2(b23.z, b23.w)};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
  // largest |Re| or |Im| written by this thread, as FP32 bits (the integer order of
  // non-negative floats; NaN above infinity above every finite value)
  uint32_t amax = 0u;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = m0 + 4 * tm + i;
    if (row >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = n0 + 4 * tn + j;
      if (col < nd && (!checks || f32_idx_ok((long long)row * nd + col, (long long)rows * nd, 13,
                                              blockIdx.x, dbg, status))) {
        F.q[(size_t)row * nd + col] = acc[i][j];
        amax = max(amax, max(__float_as_uint(fabsf(acc[i][j].x)),
                             __float_as_uint(fabsf(acc[i][j].y))));
      }
    }
  }
  if (F.amax) {   // uniform over the CTA
    amax = __reduce_max_sync(0xffffffffu, amax);
    if ((threadIdx.x & 31) == 0 && amax) atomicMax(F.amax, amax);
  }
}
__global__ void k_convert_f32(const F32ConvSeg* __restrict__ segs) {
  const F32ConvSeg sg = segs[blockIdx.y];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < sg.n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 d = sg.src[i];
    sg.dst[i] = make_float2((float)d.x, (float)d.y);
  }
}

cudaError_t launch_convert_f32(const F32ConvSeg* d_segs, int n_segs, long long max_n,
                               cudaStream_t s) {
  if (n_segs == 0 || max_n == 0) return cudaSuccess;
  for (int s0 = 0; s0 < n_segs; s0 += 65535) {  // grid.y limit
    const int ns = n_segs - s0 < 65535 ? n_segs - s0 : 65535;
    long long bx = (max_n + kThreads - 1) / kThreads;
    if (bx > 1024) bx = 1024;
    dim3 grid((unsigned)bx, ns);
    k_convert_f32<<<grid, kThreads, 0, s>>>(d_segs + s0);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_project_f32(const ProjFieldF* d_fields, int n_fields, int rows, int n_ev,
                               int max_nd, int checks, unsigned long long* dbg, int* status,
                               cudaStream_t s) {
  if (n_fields == 0 || rows == 0) return cudaSuccess;
  dim3 grid(n_fields, (rows + FBM - 1) / FBM, (max_nd + FBN - 1) / FBN);
  k_project_f32<<<grid, kThreads, 0, s>>>(d_fields, rows, n_ev, checks, dbg, status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bb
