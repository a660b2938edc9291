// Eq. (2) for the mixed forms on the tensor cores, with both operands pre-tiled in the MMA's
// shared-memory layout and staged by asynchronous bulk copies:
//   q[m][n] = sum_l V[l][m] Phi[l][n],   m = (site, colour) row of V, n = dilution column,
//   Phi = sum_t w_t phi[row_off_t + l][n] (line 3 folds the spin coefficients of a pair).
//
// * k_tile_v     every distinct V of a wave: FP64 -> FP32 -> three BF16 pieces
//                v = v0 + v1 + v2 (successive 8-bit truncations; every subtraction is exact,
//                so the three pieces represent the FP32 value exactly), written as the A
//                operand: per (128-row tile, 32-deep K stage) one contiguous 48 KB block of six
//                K-major core-matrix planes (piece x {re, im}).
// * k_tile_phi   every field's folded Phi (the fold in FP64), split the same way, as the B
//                operand: per (N tile of ncp columns, K stage) nine planes (piece x
//                {-Bi, Br, Bi}), so that [Br | Bi] and [-Bi | Br] are contiguous 2 ncp-row
//                operands.
// * k_project_tt units (V, 128-row tile, field N tile): one thread copies each K stage's two
//                blocks with cp.async.bulk into a two-stage ring (completion counted as
//                transaction bytes on the stage's mbarrier), one thread issues the MMAs of the
//                six piece products i + j <= 2, each complex product two MMAs of
//                M = 128, N = 2 ncp, K = 16:
//                  [Cr | Ci] += Ar [Br | Bi],   [Cr | Ci] += Ai [-Bi | Br],
//                the leading product (0, 0) into four TMEM accumulators in turn (K steps
//                g = 0, 1, 2, 3 mod 4) and the other five into a fifth (5 x 2 ncp <= 480
//                columns at ncp <= 48, single-buffered), and four epilogue warps add the
//                five in FP32 (round to nearest) into the field q and record the field's
//                largest |Re| or |Im| (the FP16 form's operand scales).
// Accuracy: the three pieces represent the FP32 inputs exactly and the dropped products
// (i + j >= 3) are below 3 x 2^-24 of each term. The tensor memory accumulates with
// truncation: measured, one leading accumulator over the 8 K steps of N_ev = 128 gave fields
// about twice as far from the exact sums as the FP32 FMA projection (block errors 1.4x);
// with four, each takes a quarter of the truncations of smaller partial sums, which brings
// them back to the FP32 projection's level. Every wait is bounded; on a timeout the CTA
// raises an abort flag and a status bit, and the MMA thread waits (bounded) for its own MMAs
// before TMEM is freed.
#include <cstdint>

#include "bblock_internal.h"
#include "tc_ptx.cuh"

namespace bb {
namespace {

constexpr int kPM = 128;                       // rows per A tile
constexpr int kPK = 32;                        // K elements (eigenvectors) per stage
constexpr int kPAPlane = kPM * kPK * 2;        // 8 KB: one piece plane of the A tile
constexpr int kPABytes = 6 * kPAPlane;         // 48 KB
constexpr int kPBPlaneMax = kTiledMaxNC * kPK * 2;
constexpr int kPStageBytes = kPABytes + 9 * kPBPlaneMax;   // 84 KB
constexpr int kPStages = 2;
constexpr uint32_t kPSbo = 8 * kPK * 2;        // bytes per 8-row group (K = 32)
constexpr int kPThreads = 192;                 // producer warp, MMA warp, 4 epilogue warps
constexpr int kPEpiBar = 1;
constexpr int kPLeads = 4;                     // leading accumulators, taken in turn by K step
static_assert((kPLeads + 1) * 2 * kTiledMaxNC <= 512, "accumulators fit the tensor memory");
static_assert(kPStages * kPStageBytes <= 227 * 1024, "stages fit the shared memory");

// byte offset of (row r, 8-element K segment ks8) in a plane of K = 32 core matrices
__device__ __forceinline__ uint32_t tile_ofs(int r, int ks8) {
  return (uint32_t)((r >> 3) * kPSbo + ks8 * 128 + (r & 7) * 16);
}

// FP32 -> three BF16 pieces, each an 8-significant-bit truncation of what is left
__device__ __forceinline__ void split3(float v, uint16_t (&p)[3]) {
  const uint32_t b0 = __float_as_uint(v) & 0xFFFF0000u;
  const float r1 = v - __uint_as_float(b0);
  const uint32_t b1 = __float_as_uint(r1) & 0xFFFF0000u;
  const float r2 = r1 - __uint_as_float(b1);
  p[0] = (uint16_t)(b0 >> 16);
  p[1] = (uint16_t)(b1 >> 16);
  p[2] = (uint16_t)(__float_as_uint(r2) >> 16);   // at most 8 significant bits: exact
}

// Eight values (K run) of one row as the three pieces' 16-byte core-matrix rows, re and im.
__device__ __forceinline__ void pieces8(const float2 (&v)[8], uint4 (&re)[3], uint4 (&im)[3]) {
  uint16_t pr[8][3], pi[8][3];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    split3(v[j].x, pr[j]);
    split3(v[j].y, pi[j]);
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    re[q] = make_uint4(pr[0][q] | (uint32_t)pr[1][q] << 16, pr[2][q] | (uint32_t)pr[3][q] << 16,
                       pr[4][q] | (uint32_t)pr[5][q] << 16, pr[6][q] | (uint32_t)pr[7][q] << 16);
    im[q] = make_uint4(pi[0][q] | (uint32_t)pi[1][q] << 16, pi[2][q] | (uint32_t)pi[3][q] << 16,
                       pi[4][q] | (uint32_t)pi[5][q] << 16, pi[6][q] | (uint32_t)pi[7][q] << 16);
  }
}

// One block per (V, 128-row tile, K stage); thread = (row, 8-element K segment).
__global__ void __launch_bounds__(512) k_tile_v(const TiledProjParams prm) {
  const int ks = blockIdx.x % prm.k_stages;
  const int mt = (blockIdx.x / prm.k_stages) % prm.m_tiles;
  const int vi = blockIdx.x / (prm.k_stages * prm.m_tiles);
  const TileV tv = prm.vs[vi];
  const int r = threadIdx.x % kPM, ks8 = threadIdx.x / kPM;
  const int m = mt * kPM + r;
  float2 v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int l = ks * kPK + ks8 * 8 + j;
    v[j] = make_float2(0.f, 0.f);
    if (m < prm.rows && l < prm.n_ev) {
      const double2 d = tv.V[(size_t)l * prm.rows + m];
      v[j] = make_float2((float)d.x, (float)d.y);
    }
  }
  uint4 re[3], im[3];
  pieces8(v, re, im);
  uint8_t* tile = reinterpret_cast<uint8_t*>(tv.tiles) +
                  ((size_t)mt * prm.k_stages + ks) * kPABytes + tile_ofs(r, ks8);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    *reinterpret_cast<uint4*>(tile + (2 * q + 0) * kPAPlane) = re[q];
    *reinterpret_cast<uint4*>(tile + (2 * q + 1) * kPAPlane) = im[q];
  }
}

// One block per (field N tile, K stage); thread = (column, 8-element K segment).
__global__ void __launch_bounds__(256) k_tile_phi(const TiledProjParams prm) {
  const FieldTile ft = prm.fts[blockIdx.x / prm.k_stages];
  const int ks = blockIdx.x % prm.k_stages;
  const TiledField& F = prm.fields[ft.field];
  const int ncp = F.ncp;
  const int c = threadIdx.x % ncp, ks8 = threadIdx.x / ncp;
  if (threadIdx.x >= 4 * ncp) return;
  const int n = ft.nt * ncp + c;
  float2 v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int l = ks * kPK + ks8 * 8 + j;
    double re = 0.0, im = 0.0;
    if (n < F.nd && l < prm.n_ev) {
      for (int t = 0; t < F.n_terms; ++t) {
        const double2 f = F.phi[(size_t)(F.row_off[t] + l) * F.nd + n];
        re += F.w[t].x * f.x - F.w[t].y * f.y;
        im += F.w[t].x * f.y + F.w[t].y * f.x;
      }
    }
    v[j] = make_float2((float)re, (float)im);
  }
  uint4 re[3], im[3];
  pieces8(v, re, im);
  const size_t plane = (size_t)ncp * kPK * 2;
  uint8_t* tile = reinterpret_cast<uint8_t*>(F.btiles) +
                  ((size_t)ft.nt * prm.k_stages + ks) * 9 * plane + tile_ofs(c, ks8);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const uint4 neg = make_uint4(im[q].x ^ 0x80008000u, im[q].y ^ 0x80008000u,
                                 im[q].z ^ 0x80008000u, im[q].w ^ 0x80008000u);
    *reinterpret_cast<uint4*>(tile + (3 * q + 0) * plane) = neg;     // -Bi
    *reinterpret_cast<uint4*>(tile + (3 * q + 1) * plane) = re[q];   // Br
    *reinterpret_cast<uint4*>(tile + (3 * q + 2) * plane) = im[q];   // Bi
  }
}

struct PUnit {
  int mt, ft;
  const uint8_t* a;   // the unit's A tiles, K stage 0
  const uint8_t* b;   // its B tiles, K stage 0
  int ncp;
};
__device__ __forceinline__ PUnit p_decode(const TiledProjParams& prm, long long u) {
  int lo = 0, hi = prm.n_groups - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prm.groups[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
  }
  const PGroup g = prm.groups[lo];
  const long long r = u - g.unit_begin;
  PUnit w;
  w.mt = (int)(r / g.ft_count);
  w.ft = g.ft_first + (int)(r % g.ft_count);
  const FieldTile ft = prm.fts[w.ft];
  const TiledField& F = prm.fields[ft.field];
  w.ncp = F.ncp;
  w.a = reinterpret_cast<const uint8_t*>(prm.vs[g.vidx].tiles) +
        (size_t)w.mt * prm.k_stages * kPABytes;
  w.b = reinterpret_cast<const uint8_t*>(F.btiles) +
        (size_t)ft.nt * prm.k_stages * 9 * ((size_t)F.ncp * kPK * 2);
  return w;
}

__global__ void __launch_bounds__(kPThreads, 1) k_project_tt(const __grid_constant__ TiledProjParams prm) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_full[kPStages], bar_empty[kPStages];
  __shared__ __align__(8) uint64_t bar_acc_full[2], bar_acc_empty[2], bar_final;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  if (tid == 0) {
    for (int s = 0; s < kPStages; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_acc_full[b]), 1);
      mbar_init(smem_u32(&bar_acc_empty[b]), 1);
    }
    mbar_init(smem_u32(&bar_final), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&tmem_slot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t smem_base = smem_u32(smem);

  if (warp == 0) {
    // ------------------------------------------------------------ producer (one thread)
    if (lane == 0) {
      long long s_g = 0;
      bool stop = false;
      for (long long u = blockIdx.x; u < prm.total_units && !stop; u += gridDim.x) {
        const PUnit w = p_decode(prm, u);
        const uint32_t bbytes = (uint32_t)(9 * w.ncp * kPK * 2);
        for (int ks = 0; ks < prm.k_stages; ++ks, ++s_g) {
          const int slot = (int)(s_g % kPStages);
          if (s_g >= kPStages &&
              !wait_bounded(smem_u32(&bar_empty[slot]), (uint32_t)(((s_g / kPStages) + 1) & 1),
                            &abort_flag, prm.status, prm.wait_limit)) { stop = true; break; }
          const uint32_t full = smem_u32(&bar_full[slot]);
          const uint32_t dst = smem_base + (uint32_t)(slot * kPStageBytes);
          mbar_arrive_expect_tx(full, (uint32_t)kPABytes + bbytes);
          bulk_g2s(dst, w.a + (size_t)ks * kPABytes, (uint32_t)kPABytes, full);
          bulk_g2s(dst + kPABytes, w.b + (size_t)ks * bbytes, bbytes, full);
        }
      }
      if (stop) {
        // copies already issued land before the CTA leaves (bounded)
        for (int i = 0; i < kPStages; ++i) {
          const long long k = s_g - 1 - i;
          if (k < 0) break;
          wait_bounded(smem_u32(&bar_full[k % kPStages]), (uint32_t)((k / kPStages) & 1), nullptr,
                       prm.status, kDrainCycles);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue (one thread)
    if (lane == 0) {
      long long s_g = 0, c_g = 0;
      bool stop = false;
      for (long long u = blockIdx.x; u < prm.total_units && !stop; u += gridDim.x) {
        const PUnit w = p_decode(prm, u);
        const int ncp = w.ncp;
        // FP32 accumulate, BF16 A and B, K-major, M = 128, N = 2 ncp
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                               ((uint32_t)(2 * ncp) >> 3 << 17) | ((uint32_t)(kPM >> 4) << 24);
        // the single accumulator set must have been drained (the previous unit's)
        if (c_g >= 1 &&
            !wait_bounded(smem_u32(&bar_acc_empty[0]), (uint32_t)((c_g + 1) & 1),
                          &abort_flag, prm.status, prm.wait_limit)) { stop = true; break; }
        const uint32_t corr = tmem + (uint32_t)(kPLeads * 2 * ncp);
        const uint32_t bplane = (uint32_t)(ncp * kPK * 2);
        for (int ks = 0; ks < prm.k_stages; ++ks, ++s_g) {
          const int slot = (int)(s_g % kPStages);
          if (!wait_bounded(smem_u32(&bar_full[slot]), (uint32_t)((s_g / kPStages) & 1),
                            &abort_flag, prm.status, prm.wait_limit)) { stop = true; break; }
          tc_fence_after();
          const uint32_t sa = smem_base + (uint32_t)(slot * kPStageBytes);
          const uint32_t sb = sa + kPABytes;
#pragma unroll
          for (int kk = 0; kk < kPK / 16; ++kk) {
            const uint32_t kofs = (uint32_t)(kk * 256);
            // piece products (i, j), i + j <= 2: (0,0) leading, then the corrections
            constexpr int PI[6] = {0, 0, 1, 1, 0, 2};
            constexpr int PJ[6] = {0, 1, 0, 1, 2, 0};
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              const int g = ks * (kPK / 16) + kk;   // K step of the unit
              const uint32_t d = q == 0 ? tmem + (uint32_t)((g % kPLeads) * 2 * ncp) : corr;
              const bool first = q == 0 ? g < kPLeads : (g == 0 && q == 1);
              const uint64_t ar = smem_desc(sa + (uint32_t)((2 * PI[q] + 0) * kPAPlane) + kofs, kPSbo);
              const uint64_t ai = smem_desc(sa + (uint32_t)((2 * PI[q] + 1) * kPAPlane) + kofs, kPSbo);
              const uint32_t bj = sb + (uint32_t)(3 * PJ[q]) * bplane;
              const uint64_t b_ri = smem_desc(bj + bplane + kofs, kPSbo);   // [Br | Bi]
              const uint64_t b_nr = smem_desc(bj + kofs, kPSbo);            // [-Bi | Br]
              mma<false>(d, ar, b_ri, idesc, first ? 0u : 1u);
              mma<false>(d, ai, b_nr, idesc, 1u);
            }
          }
          tc_commit(smem_u32(&bar_empty[slot]));
        }
        if (stop) break;
        tc_commit(smem_u32(&bar_acc_full[0]));
        ++c_g;
      }
      tc_commit(smem_u32(&bar_final));
      wait_bounded(smem_u32(&bar_final), 0u, nullptr, prm.status, kWaitCycles);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (TMEM lanes)
    const int quad = warp % 4;
    const int row = quad * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
    long long c_g = 0;
    for (long long u = blockIdx.x; u < prm.total_units; u += gridDim.x, ++c_g) {
      const PUnit w = p_decode(prm, u);
      const FieldTile ft = prm.fts[w.ft];
      const TiledField& F = prm.fields[ft.field];
      const int ncp = w.ncp;
      // leading accumulators the unit's K steps wrote
      const int n_leads = min(kPLeads, prm.k_stages * (kPK / 16));
      bool ok = !abort_flag;
      if (ok)
        ok = wait_bounded(smem_u32(&bar_acc_full[0]), (uint32_t)(c_g & 1), &abort_flag,
                          prm.status, prm.wait_limit);
      ok = __all_sync(0xffffffffu, ok);
      if (ok) {
        tc_fence_after();
        const int m = w.mt * kPM + row;
        uint32_t amax = 0u;
        const uint32_t corr = lane_base + (uint32_t)(kPLeads * 2 * ncp);
        for (int col = 0; col < ncp; col += 16) {
          __syncwarp();   // tcgen05.ld is warp-aligned; the stores below may diverge
          float lr[16], li[16], cr[16], ci[16];
          tmem_ld16(corr + col, cr);
          tmem_ld16(corr + ncp + col, ci);
          tmem_wait_ld();
          // the leading accumulators, summed pairwise in FP32 (round to nearest)
          float sr[16] = {}, si[16] = {};
          for (int a = 0; a < n_leads; a += 2) {
            float ar[16], ai[16], br[16], bi[16];
            tmem_ld16(lane_base + (uint32_t)(a * 2 * ncp + col), ar);
            tmem_ld16(lane_base + (uint32_t)(a * 2 * ncp + ncp + col), ai);
            if (a + 1 < n_leads) {
              tmem_ld16(lane_base + (uint32_t)((a + 1) * 2 * ncp + col), br);
              tmem_ld16(lane_base + (uint32_t)((a + 1) * 2 * ncp + ncp + col), bi);
            }
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float pr = a + 1 < n_leads ? ar[i] + br[i] : ar[i];
              const float pi = a + 1 < n_leads ? ai[i] + bi[i] : ai[i];
              sr[i] += pr;
              si[i] += pi;
            }
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) { lr[i] = sr[i]; li[i] = si[i]; }
          if (m < prm.rows) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int n = ft.nt * ncp + col + i;
              if (n < F.nd) {
                const float2 v = make_float2(lr[i] + cr[i], li[i] + ci[i]);
                F.q[(size_t)m * F.nd + n] = v;
                amax = max(amax, max(__float_as_uint(fabsf(v.x)), __float_as_uint(fabsf(v.y))));
              }
            }
          }
        }
        if (F.amax) {
          amax = __reduce_max_sync(0xffffffffu, amax);
          if (lane == 0 && amax) atomicMax(F.amax, amax);
        }
      }
      tc_fence_before();
      __syncwarp();
      named_bar(kPEpiBar, 128);
      if (tid == 64) mbar_arrive(smem_u32(&bar_acc_empty[0]));
      __syncwarp();
    }
  }

  tc_fence_before();
  __syncwarp();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

}  // namespace

cudaError_t launch_project_tiled(const TiledProjParams& prm, int n_vs, int n_fts, int grid,
                                 cudaStream_t s) {
  if (prm.total_units == 0) return cudaSuccess;
  k_tile_v<<<(unsigned)(n_vs * prm.m_tiles * prm.k_stages), 512, 0, s>>>(prm);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_tile_phi<<<(unsigned)(n_fts * prm.k_stages), 256, 0, s>>>(prm);
  note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)kPStages * kPStageBytes;
  e = cudaFuncSetAttribute(k_project_tt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_project_tt<<<grid, kPThreads, smem, s>>>(prm);
  note_launch();
  return cudaGetLastError();
}

size_t tiled_v_bytes(int rows, int n_ev) {
  return (size_t)((rows + kPM - 1) / kPM) * ((n_ev + kPK - 1) / kPK) * kPABytes;
}
size_t tiled_phi_bytes(int nd, int ncp, int n_ev) {
  return (size_t)((nd + ncp - 1) / ncp) * ((n_ev + kPK - 1) / kPK) * 9 * ((size_t)ncp * kPK * 2);
}

}  // namespace bb
