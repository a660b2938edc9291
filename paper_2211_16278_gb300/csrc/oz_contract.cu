// FP64-accurate form of the fused diquark + contraction (Eq. 1/3) on the BF16 tensor cores:
// the Ozaki scheme (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012) — both operands
// split error-free into short integer digits whose products the tensor cores sum exactly.
//
// The contraction is the complex GEMM of the other tensor-core forms,
//   C[(d1,d2)][(p,d3)] = sum_k A[(d1,d2)][k] Bop[k][(p,d3)],   k = (site, spin pair, colour),
// A the diquark (q1_alpha x q2_beta)_c(x) and Bop = e^{-i p.x} q3_(alpha beta)[x][c][d3], built
// here from the double-float fields and phases (about 48 significant bits) of the
// double-float projection.
//
// * Scales. Every row m = (d1, d2) of A gets, per site slab, a power of two 2^eA bounding
//   |Re| and |Im| of its entries: |(u_b v_c - u_c v_b)| <= |u_b||v_c| + |u_c||v_b|
//   <= 2 max|u|_1 max|v|_1 with |z|_1 = |Re z| + |Im z| and the maxima taken over the slab's
//   sites and colours of column d1 (line 1) and d2 (line 2). Every column (p, d3) gets 2^eB
//   with 2^eB >= max|q3|_1 over the slab, which bounds the phase-folded entries (|e^{ipx}| = 1).
//   k_oz_colmax writes those column maxima; a 2^-20 margin covers their rounding.
// * Digits. A scaled entry v = h + l (|v| <= 1) is written as seven digits
//   v = sum_i a_i + r,  a_i = d_i 2^(-7-8i),  d_i integer, |d_i| <= 130, |r| <= 2^-56:
//   a_i is the multiple of 2^(-7-8i) nearest the remainder (found exactly by adding and
//   subtracting 1.5 * 2^(16-8i)), the subtraction is exact, and the low part l joins the
//   remainder by TwoSum before digits 2 and 4. Each a_i (8 significant bits) is exact in BF16.
// * Products. a_i b_j is exact on the tensor cores, a multiple of 2^(-14-8(i+j)); the 28
//   products with i + j <= 6 are kept (the rest are below 2^-56 of the scales). Levels
//   i + j = 0, 1, 2, 3 have one FP32 accumulator each in tensor memory, which sums them
//   exactly while the sums stay below 2^24 units of 2^(-14-8 level): at most 4 products
//   of |d_i d_j| <= 130 * 128 per K element, so a drain every 240 K elements (15 stages of
//   16) keeps 4 * 240 * 16640 < 2^24. Levels 4..6 (18 products, at most 2^-32 of the
//   scales) share a fifth accumulator, whose FP32 rounding stays below 2^-50 of them.
// * Drains. Every 15 stages the epilogue adds the five accumulators (TwoSum of the exact
//   levels) into a double-float running sum per element, kept in the unit's partial block
//   itself (float4 re.h, re.l, im.h, im.l); a unit's last drain writes the FP64 value times
//   2^(eA + eB). The FP64 slab reduction of the FP64 form sums the slabs in index order.
//
// A stage holds K = 16 (site, pair, colour) elements: for each of the 7 digits, the real and
// imaginary planes of the 128-row diquark tile and the -Bi | Br | Bi planes of the NC-row
// third-quark tile, as K-major 8 x 16-byte core matrices (two per 8-row group). The diquark
// planes are interleaved by row group (group g of plane (digit, re/im) at g * 3584 +
// (2 digit + re/im) * 256), so that any run of row groups of every plane is one contiguous
// block; the third-quark planes are plain (group g at g * 256), so that [Br | Bi] and
// [-Bi | Br] are contiguous 2 NC-row operands. A complex product of digits (i, j) is two MMAs
// of M = 128, N = 2 NC, K = 16 into [Cr | Ci]:
//   [Cr | Ci] += Ar_i [Br_j | Bi_j],   [Cr | Ci] += Ai_i [-Bi_j | Br_j].
//
// Clusters (C = 2, 3, 4): the C CTAs of a cluster take the same (job, M tile, slab) and C
// adjacent N tiles. The diquark tile is the same for all of them, and its digits are the
// costliest part of a stage: each CTA builds the row groups [16 r / C, 16 (r + 1) / C) of it
// and pushes them, one bulk shared::cta -> shared::cluster copy per warp and peer, into the
// peers' stage, counted as transaction bytes on their stage barriers; every CTA's MMA
// completion arrives on the stage-free barriers of all C CTAs. N tiles past a job's last
// (a ragged cluster) run with zero third-quark rows and write nothing.
//
// Warp roles: epilogue (4 warps, or 8 in clusters: warp e drains TMEM lanes 32 (e % 4) ..
// +31 and half of the columns), one MMA issue and TMEM allocation warp, then the producers:
// diquark warps (16 rows x 2 halves of 8 K elements each) and 3 third-quark warps (up to 48
// rows x 2 halves). Every wait is bounded; on a timeout the CTA raises its abort flag and a
// status bit, the roles run out their loops, the MMA thread waits (bounded) for its own MMAs
// and for peer copies still landing in its stages, and the allocating warp frees TMEM.
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>

#include "bblock_internal.h"
#include "dfloat.cuh"
#include "tc_ptx.cuh"

namespace bb {
namespace {

constexpr int kDigits = 7;
constexpr int kAcc = 5;                               // levels 0, 1, 2, 3 and 4..6
constexpr int kK = 16;                                // K elements per stage
constexpr int kStages = 2;
constexpr int kChunk = 15;                            // stages between drains
constexpr int kAGroup = kDigits * 2 * 256;            // one 8-row group of every diquark plane
constexpr int kAStage = (kOzM / 8) * kAGroup;
constexpr int kBPlaneMax = kOzMaxNC * kK * 2;         // one digit plane of the third quark
constexpr int kStageBytes = kAStage + kDigits * 3 * kBPlaneMax;   // + -Bi, Br, Bi
constexpr uint32_t kSboB = 256;                       // bytes per 8-row group (K = 16)
constexpr int kBarProd = 1, kBarEpi = 2;
static_assert(kAcc * 2 * kOzMaxNC <= 512, "accumulators fit the tensor memory");
static_assert(kStages * kStageBytes <= 227 * 1024, "stages fit the shared memory");

template <int C> struct OzRoles {
  static constexpr int kEpiWarps = 4;
  static constexpr int kMmaWarp = 4;
  static constexpr int kProdWarp0 = 5;
  // K elements per producer thread: a stage's time is the latency-bound time of each
  // producer thread's chain of elements, so the rows a cluster frees go to more threads with
  // shorter chains: 8 elements (two 8-element halves of a row) or 4 (four quarters), within
  // 16 warps in all (below)
  static constexpr int kEA = C == 1 ? 8 : 4;
  static constexpr int kEB = C >= 4 ? 4 : 8;
  static constexpr int kARowsPerWarp = 32 * kEA / kK;           // 16 or 8 rows per warp
  static constexpr int kMaxGroups = (kOzM / 8 + C - 1) / C;     // diquark row groups per CTA
  static constexpr int kAWarps = (kMaxGroups * 8 + kARowsPerWarp - 1) / kARowsPerWarp;
  static constexpr int kAThreads = kAWarps * 32;
  static constexpr int kBThreads = kOzMaxNC * (kK / kEB);
  static constexpr int kProdThreads = kAThreads + kBThreads;
  static constexpr int kThreads = kProdWarp0 * 32 + kProdThreads;
  // registers: each of the 4 SM sub-partitions has 16384 registers for its ceil(warps / 4)
  // warps, so 16 warps allow 128 registers per thread (measured on GB300: 15 warps at 136 or
  // 17 warps at 120 registers are not resident at all)
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kMaxRegs = 128;
  static_assert(kWarps <= 16, "16 warps of 128 registers fill the register file");
  static_assert(kProdThreads % 32 == 0 && kBThreads % 32 == 0, "whole producer warps");
};
__host__ __device__ constexpr int group_begin(int r, int C) { return (kOzM / 8) * r / C; }

// 1.5 * 2^(16 - 8 i): adding and subtracting it rounds |v| < 2^(15 - 8 i) to the nearest
// multiple of 2^(-7 - 8 i).
__device__ __forceinline__ float round_const(int i) {
  constexpr float r[kDigits] = {0x1.8p16f, 0x1.8p8f, 0x1.8p0f, 0x1.8p-8f, 0x1.8p-16f,
                                0x1.8p-24f, 0x1.8p-32f};
  return r[i];
}

// Packed (re, im) FP32 arithmetic; a - b as fma(-1, b, a) rounds exactly like a subtraction.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(make_float2(-1.f, -1.f), b, a);
}
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& t) {
  s = __fadd2_rn(a, b);
  const float2 bv = sub2(s, a);
  const float2 av = sub2(s, bv);
  t = __fadd2_rn(sub2(a, av), sub2(b, bv));
}

// ceil(log2 y) for the bound y > 0, clamped to [-120, 120]; 0 for a zero bound (all
// entries zero) or a non-finite one (non-finite inputs stay non-finite).
__device__ __forceinline__ int ceil_log2(float y) {
  const uint32_t b = __float_as_uint(y);
  const int be = (int)((b >> 23) & 0xFFu);
  if (be == 0xFF || (b & 0x7FFFFFFFu) == 0u) return 0;
  int e = be == 0 ? -126 : be - 127 + ((b & 0x7FFFFFu) != 0u ? 1 : 0);
  return min(120, max(-120, e));
}
__device__ __forceinline__ float pow2(int e) { return __int_as_float((127 + e) << 23); }
// Row exponent of the diquark: M = the row's largest |Re D|, |Im D| computed in FP32 from the
// fields' high parts (k_oz_rowmax), u, v = the line-1 and line-2 column maxima of |.|_1. The
// FP32 evaluation and the double-float low parts move |Re D|, |Im D| by less than
// 2^-21 (|u_b||v_c| + |u_c||v_b|) <= 2^-20 u v, so 2^eA >= (M + 2^-19 u v)(1 + 2^-20) bounds
// every entry. Column exponent of the third quark: w = the largest |q3| (FP32 modulus of the
// high parts, within 2^-22 of the exact modulus; |e^{-ip.x}| = 1), 2^eB >= w (1 + 2^-18).
// The same arithmetic runs in the producers and the epilogue.
__device__ __forceinline__ int exp_a(float M, float u, float v) {
  return ceil_log2(__fmul_rn(__fmaf_rn(0x1p-19f * u, v, M), 1.f + 0x1p-20f));
}
__device__ __forceinline__ int exp_b(float w) { return ceil_log2(__fmul_rn(w, 1.f + 0x1p-18f)); }

// acc = a * b (double-float, three leading partial products)
__device__ __forceinline__ dfloat df_prod(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return dfloat{p, e};
}
__device__ __forceinline__ dfloat df_neg(dfloat a) { return dfloat{-a.h, -a.l}; }
__device__ __forceinline__ dfloat dre(float4 z) { return dfloat{z.x, z.y}; }
__device__ __forceinline__ dfloat dim(float4 z) { return dfloat{z.z, z.w}; }

// Packed double-float products, (re, im) in the two lanes: acc = a * b and acc += a * b with
// a = (ah, al), b = (bh, bl) pairs of FP32x2 (the three leading partial products; the low
// part is normalised lazily, as df_fma).
struct df2 {
  float2 h, l;
};
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ df2 df2_prod(float2 ah, float2 al, float2 bh, float2 bl) {
  const float2 p = __fmul2_rn(ah, bh);
  float2 e = __ffma2_rn(ah, bh, neg2(p));
  e = __ffma2_rn(ah, bl, e);
  e = __ffma2_rn(al, bh, e);
  return df2{p, e};
}
__device__ __forceinline__ void df2_fma(df2& acc, float2 ah, float2 al, float2 bh, float2 bl) {
  const float2 p = __fmul2_rn(ah, bh);
  float2 e = __ffma2_rn(ah, bh, neg2(p));
  e = __ffma2_rn(ah, bl, e);
  e = __ffma2_rn(al, bh, e);
  float2 s, t;
  two_sum2(acc.h, p, s, t);
  acc.h = s;
  acc.l = __fadd2_rn(acc.l, __fadd2_rn(t, e));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ int find_job(const ContractJob* jobs, int n_jobs, long long u) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct OzUnit {
  int job, mt, nt, slab, x_begin, x_end, n_stages;
};
__device__ __forceinline__ OzUnit decode(const ContractParams& prm, long long u) {
  OzUnit w;
  w.job = find_job(prm.jobs, prm.n_jobs, u);
  const ContractJob& J = prm.jobs[w.job];
  long long r = u - J.unit_begin;
  w.mt = (int)(r % J.m_tiles);
  r /= J.m_tiles;
  w.nt = (int)(r % J.n_tiles);
  w.slab = (int)(r / J.n_tiles);
  w.x_begin = w.slab * prm.sites_per_slab;
  w.x_end = min(prm.X, w.x_begin + prm.sites_per_slab);
  const long long k_total = (long long)(w.x_end - w.x_begin) * prm.n_pairs * 3;
  w.n_stages = w.slab < prm.n_slab ? (int)((k_total + kK - 1) / kK) : 0;
  return w;
}

// Shared-memory state the producer roles use.
struct OzShared {
  uint8_t* smem;
  uint32_t smem_base;
  uint64_t* bar_full;
  uint64_t* bar_empty;
  volatile int* abort_flag;
  const float4** s_q1;
  const float4** s_q2;
  const float4** s_q3;
};

// Stores of one K run of E BF16 digits (E = 8: 16 bytes, E = 4: 8 bytes).
template <int E> __device__ __forceinline__ void store_run(uint8_t* dst, const uint32_t (&w)[E / 2]) {
  if constexpr (E == 8) *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  else *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
}

// One producer role. A = true: the diquark rows of this CTA's share (lanes: kEA-element
// segments of 32 kEA / 16 rows); A = false: the third-quark rows (48 rows x 16 / E segments).
// Each thread builds E consecutive K elements of its row per stage, splits them into digits
// and stores every digit's run; a diquark warp then pushes its row groups to the peers.
template <int C, int E, bool A>
__device__ __forceinline__ void oz_produce(const ContractParams& prm, const OzShared& sh, int pt,
                                           int lane, uint32_t rank, int gb, int ge,
                                           uint32_t peer_tx) {
  using R = OzRoles<C>;
  constexpr int kRW = 32 * E / kK;          // rows per warp (diquark)
  constexpr int kSegs = kK / E;             // K segments per row
  const int NC = prm.NC;
  const int np = prm.n_pairs;
  const long long u0 = blockIdx.x / C, du = gridDim.x / C;
  int rr, seg, a_g0 = 0, a_ng = 0;
  bool row_used;
  if (A) {
    const int wa = pt / 32;
    a_g0 = gb + wa * (kRW / 8);
    a_ng = max(0, min(kRW / 8, ge - a_g0));
    rr = a_g0 * 8 + lane % kRW;
    seg = lane / kRW;
    row_used = rr < ge * 8;
  } else {
    const int b = pt - R::kAThreads;
    rr = b % kOzMaxNC;
    seg = b / kOzMaxNC;
    row_used = rr < NC;
  }
  // byte offset of this thread's run within a plane's row: 16-byte core-matrix column
  // (seg E / 8) and, for E = 4, its half
  const uint32_t in_row = (uint32_t)((seg * E / 8) * 128 + (E == 4 ? (seg & 1) * 8 : 0));
  const uint32_t a_row = (uint32_t)((rr >> 3) * kAGroup + (rr & 7) * 16) + in_row;
  const uint32_t b_row = (uint32_t)((rr >> 3) * kSboB + (rr & 7) * 16) + in_row;
  (void)kSegs;
  long long s_g = 0;
  for (long long u = u0; u < prm.total_units; u += du) {
    const OzUnit w = decode(prm, u);
    const ContractJob& J = prm.jobs[w.job];
    const int nd1 = J.nd1, nd2 = J.nd2, nd3 = J.nd3;
    const int stride = nd1 + nd2 + nd3;
    const int slab = w.slab < prm.n_slab ? w.slab : 0;
    const float* mx = J.oz_max + (size_t)slab * stride;
    // the slab's row maxima follow every slab's column maxima
    const float* rmx = J.oz_max + (size_t)prm.n_slab * stride + (size_t)slab * nd1 * nd2;
    bool row_ok;
    int o1 = 0, o2 = 0, s1 = 0, s2 = 0, p = 0;
    float sc = 1.f;
    if (A) {
      const int m = w.mt * kOzM + rr;
      row_ok = row_used && m < nd1 * nd2;
      const int d1 = row_ok ? m / nd2 : 0, d2 = row_ok ? m - d1 * nd2 : 0;
      o1 = d1; o2 = d2; s1 = nd1; s2 = nd2;
      if (row_ok) sc = pow2(-exp_a(rmx[m], mx[d1], mx[nd1 + d2]));
    } else {
      const int n = (w.nt * C + (int)rank) * NC + rr;
      row_ok = row_used && n < prm.P * nd3;
      p = row_ok ? n / nd3 : 0;
      const int d3 = row_ok ? n - p * nd3 : 0;
      o1 = d3; s1 = nd3;
      if (row_ok) sc = pow2(-exp_b(mx[nd1 + nd2 + d3]));
    }
    const float4* ph = prm.phase_df + (size_t)(prm.p0 + p) * prm.X;
    // the unit's field table (producer warps meet before and after rewriting it)
    __syncwarp();
    named_bar(kBarProd, R::kProdThreads);
    if (pt < np) {
      sh.s_q1[pt] = reinterpret_cast<const float4*>(J.q1[prm.a_slot[pt]]);
      sh.s_q2[pt] = reinterpret_cast<const float4*>(J.q2[prm.b_slot[pt]]);
      sh.s_q3[pt] = reinterpret_cast<const float4*>(J.q3[pt]);
    }
    __syncwarp();
    named_bar(kBarProd, R::kProdThreads);
    // K elements of the unit (< 2^31: at most 3 L^3 kMaxPairs) and the (site, pair, colour)
    // of this thread's first element of the current stage; field offsets fit in 32 bits
    // (3 L^3 nd < 2^31 for L <= 128, nd <= 256)
    const int k_total = (w.x_end - w.x_begin) * np * 3;
    int kk0 = seg * E;
    int c0 = kk0 % 3, pr0 = (kk0 / 3) % np, x0 = w.x_begin + (kk0 / 3) / np;

    for (int st = 0; st < w.n_stages; ++st, ++s_g) {
      if (st > 0) {
        // advance the state by one stage: 16 = 5 groups of 3 + 1 colour
        int groups = 5;
        if (++c0 == 3) { c0 = 0; ++groups; }
        pr0 += groups;
        while (pr0 >= np) { pr0 -= np; ++x0; }
        kk0 += kK;
      }
      const int slot = (int)(s_g % kStages);
      bool ok = !*sh.abort_flag;
      if (ok && s_g >= kStages)
        ok = wait_bounded(smem_u32(&sh.bar_empty[slot]), (uint32_t)(((s_g / kStages) + 1) & 1),
                          sh.abort_flag, prm.status, prm.wait_limit);
      ok = __all_sync(0xffffffffu, ok);
      if (ok && row_used) {
        // this thread's E K elements: k = 16 st + E seg + j = ((x - x_begin) np + pair) 3 + c,
        // from the (site, pair, colour) state of its first element. They span at most
        // G = (E + 4) / 3 (site, pair) groups, whose field pointers are read once; the loads
        // of a batch of elements (4 diquark elements, 8 third-quark ones) are all issued
        // before its arithmetic, so that their latencies overlap.
        constexpr int G = (E + 4) / 3;
        constexpr int LB = A ? 4 : 8;
        const float4* pa[G];
        const float4* pb[G];
        int xg[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {
          int pr = pr0 + k, xx = x0;
          while (pr >= np) { pr -= np; ++xx; }
          pa[k] = A ? sh.s_q1[pr] : sh.s_q3[pr];
          pb[k] = A ? sh.s_q2[pr] : nullptr;
          xg[k] = xx;
        }
        float2 va[E], vb[E];   // scaled entries (re, im): high parts, low parts
        int c = c0, gi = 0, kk = kk0;
#pragma unroll
        for (int b0 = 0; b0 < E; b0 += LB) {
          float4 ld[LB][A ? 4 : 2];
          bool vld[LB];
#pragma unroll
          for (int jj = 0; jj < LB; ++jj) {
            vld[jj] = row_ok && kk < k_total;
            const float4* fa = pa[0];
            const float4* fb = pb[0];
            int x = xg[0];
#pragma unroll
            for (int k = 1; k < G; ++k)
              if (gi == k) { fa = pa[k]; fb = pb[k]; x = xg[k]; }
            if (!vld[jj]) x = w.x_begin;   // zero elements read a valid site
            if (A) {
              const int c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
              const float4* uq = fa + (x * 3 * s1 + o1);
              const float4* vq = fb + (x * 3 * s2 + o2);
              ld[jj][0] = __ldg(uq + c1 * s1);
              ld[jj][1] = __ldg(uq + c2 * s1);
              ld[jj][2] = __ldg(vq + c1 * s2);
              ld[jj][3] = __ldg(vq + c2 * s2);
            } else {
              ld[jj][0] = __ldg(fa + ((x * 3 + c) * s1 + o1));
              ld[jj][1] = __ldg(ph + x);
            }
            ++kk;
            if (++c == 3) { c = 0; ++gi; }
          }
#pragma unroll
          for (int jj = 0; jj < LB; ++jj) {
            const int j = b0 + jj;
            df2 v;
            if (A) {
              // colour c of the diquark: D = u_c1 v_c2 - u_c2 v_c1, (c, c1, c2) cyclic;
              // lanes (Re D, Im D):
              //   Re = u1r v2r - u1i v2i - u2r v1r + u2i v1i
              //   Im = u1r v2i + u1i v2r - u2r v1i - u2i v1r
              const float4 u1 = ld[jj][0], u2 = ld[jj][1], v1 = ld[jj][2], v2 = ld[jj][3];
              v = df2_prod(make_float2(u1.x, u1.x), make_float2(u1.y, u1.y),
                           make_float2(v2.x, v2.z), make_float2(v2.y, v2.w));
              df2_fma(v, make_float2(-u1.z, u1.z), make_float2(-u1.w, u1.w),
                      make_float2(v2.z, v2.x), make_float2(v2.w, v2.y));
              df2_fma(v, make_float2(-u2.x, -u2.x), make_float2(-u2.y, -u2.y),
                      make_float2(v1.x, v1.z), make_float2(v1.y, v1.w));
              df2_fma(v, make_float2(u2.z, -u2.z), make_float2(u2.w, -u2.w),
                      make_float2(v1.z, v1.x), make_float2(v1.w, v1.y));
            } else {
              // e^{-ip.x} q3: Re = er qr - ei qi, Im = er qi + ei qr
              const float4 q = ld[jj][0], e = ld[jj][1];
              v = df2_prod(make_float2(e.x, e.x), make_float2(e.y, e.y),
                           make_float2(q.x, q.z), make_float2(q.y, q.w));
              df2_fma(v, make_float2(-e.z, e.z), make_float2(-e.w, e.w),
                      make_float2(q.z, q.x), make_float2(q.w, q.y));
            }
            // elements past the unit's K or of an unused row are zero
            const float s = vld[jj] ? sc : 0.f;
            va[j] = __fmul2_rn(v.h, make_float2(s, s));
            vb[j] = __fmul2_rn(v.l, make_float2(s, s));
          }
        }
        // digits, most significant first; each digit's E values are one K run of the row
#pragma unroll
        for (int i = 0; i < kDigits; ++i) {
          const float Rc = round_const(i);
          const float2 R2 = make_float2(Rc, Rc);
          float2 d[E];
#pragma unroll
          for (int j = 0; j < E; ++j) {
            if (i == 2 || i == 4) two_sum2(va[j], vb[j], va[j], vb[j]);
            d[j] = sub2(__fadd2_rn(va[j], R2), R2);
            va[j] = sub2(va[j], d[j]);
          }
          uint32_t wr[E / 2], wi[E / 2];
#pragma unroll
          for (int q = 0; q < E / 2; ++q) {
            wr[q] = pack_bf16(d[2 * q].x, d[2 * q + 1].x);
            wi[q] = pack_bf16(d[2 * q].y, d[2 * q + 1].y);
          }
          const uint32_t stage = (uint32_t)(slot * kStageBytes);
          if (A) {
            store_run<E>(sh.smem + stage + (uint32_t)((i * 2 + 0) * 256) + a_row, wr);
            store_run<E>(sh.smem + stage + (uint32_t)((i * 2 + 1) * 256) + a_row, wi);
          } else {
            uint32_t wn[E / 2];
#pragma unroll
            for (int q = 0; q < E / 2; ++q) wn[q] = wi[q] ^ 0x80008000u;
            // third-quark digit i, planes -Bi, Br, Bi (NC rows each, adjacent)
            uint8_t* bp = sh.smem + stage + kAStage + (uint32_t)(i * 3 * kBPlaneMax) + b_row;
            store_run<E>(bp, wn);
            store_run<E>(bp + NC * kK * 2, wr);
            store_run<E>(bp + 2 * NC * kK * 2, wi);
          }
        }
      }
      // every lane's stores are made visible to the async proxy; then one lane acts for the
      // warp: its diquark row groups (every plane: one contiguous block) go to every peer
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        if (C > 1 && A && ok && a_ng > 0) {
          const uint32_t src = sh.smem_base + (uint32_t)(slot * kStageBytes + a_g0 * kAGroup);
          const uint32_t full_local = smem_u32(&sh.bar_full[slot]);
          for (uint32_t q = 0; q < (uint32_t)C; ++q) {
            if (q == rank) continue;
            copy_to_peer(map_to_rank(src, q), src, (uint32_t)(a_ng * kAGroup),
                         map_to_rank(full_local, q));
          }
        }
        if (C > 1 && pt == 0)
          mbar_arrive_expect_tx(smem_u32(&sh.bar_full[slot]), peer_tx);
        else
          mbar_arrive(smem_u32(&sh.bar_full[slot]));
      }
      __syncwarp();
    }
  }
}

template <int C>
__global__ void __maxnreg__(OzRoles<C>::kMaxRegs)
k_contract_oz(const __grid_constant__ ContractParams prm) {
  using R = OzRoles<C>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages];
  __shared__ __align__(8) uint64_t bar_acc_full, bar_acc_empty, bar_final;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ const float4* s_q1[kMaxPairs];
  __shared__ const float4* s_q2[kMaxPairs];
  __shared__ const float4* s_q3[kMaxPairs];

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int NC = prm.NC;
  const int np = prm.n_pairs;
  const uint32_t rank = C > 1 ? cluster_rank() : 0u;
  const int gb = group_begin((int)rank, C), ge = group_begin((int)rank + 1, C);
  // transaction bytes the peers' diquark row groups bring into each stage
  const uint32_t peer_tx = (uint32_t)((kOzM / 8 - (ge - gb)) * kAGroup);

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&bar_full[s]), R::kProdThreads / 32);
      mbar_init(smem_u32(&bar_empty[s]), C);   // the MMA completion of every CTA of the cluster
    }
    mbar_init(smem_u32(&bar_acc_full), 1);
    mbar_init(smem_u32(&bar_acc_empty), 1);
    mbar_init(smem_u32(&bar_final), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == R::kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&tmem_slot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  if (C > 1) cluster_sync_all();   // peers signal this CTA's barriers only once they exist
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t smem_base = smem_u32(smem);
  const long long u0 = blockIdx.x / C, du = gridDim.x / C;

  if (warp >= R::kProdWarp0) {
    // ------------------------------------------------------------ producers
    const int pt = tid - R::kProdWarp0 * 32;
    OzShared sh{smem, smem_base, bar_full, bar_empty, &abort_flag, s_q1, s_q2, s_q3};
    if (pt < R::kAThreads)
      oz_produce<C, R::kEA, true>(prm, sh, pt, lane, rank, gb, ge, peer_tx);
    else
      oz_produce<C, R::kEB, false>(prm, sh, pt, lane, rank, gb, ge, peer_tx);
  } else if (warp == R::kMmaWarp) {
    // ------------------------------------------------------------ MMA issue (one thread)
    if (lane == 0) {
      // FP32 accumulate, BF16 A and B, K-major, M = 128, N = 2 NC
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                             ((uint32_t)(2 * NC) >> 3 << 17) | ((uint32_t)(kOzM >> 4) << 24);
      long long s_g = 0, c_g = 0;
      bool stop = false;
      for (long long u = u0; u < prm.total_units && !stop; u += du) {
        const OzUnit w = decode(prm, u);
        for (int st = 0; st < w.n_stages; ++st, ++s_g) {
          const int slot = (int)(s_g % kStages);
          const bool chunk_first = st % kChunk == 0;
          const bool chunk_last = st % kChunk == kChunk - 1 || st == w.n_stages - 1;
          if (chunk_first && c_g >= 1 &&
              !wait_bounded(smem_u32(&bar_acc_empty), (uint32_t)((c_g + 1) & 1), &abort_flag,
                            prm.status, prm.wait_limit)) { stop = true; break; }
          if (!wait_bounded(smem_u32(&bar_full[slot]), (uint32_t)((s_g / kStages) & 1),
                            &abort_flag, prm.status, prm.wait_limit)) { stop = true; break; }
          tc_fence_after();
          const uint32_t sa = smem_base + (uint32_t)(slot * kStageBytes);
          const uint32_t sb = sa + kAStage;
          // the 28 digit products (i, j), i + j <= 6, level by level; levels >= 4 share the
          // last accumulator, and the first product into an accumulator in a chunk's first
          // stage overwrites it
#pragma unroll
          for (int lv = 0; lv < kDigits; ++lv) {
            const int t = lv < kAcc - 1 ? lv : kAcc - 1;
            const uint32_t d = tmem + (uint32_t)(t * 2 * NC);
#pragma unroll
            for (int i = 0; i <= lv; ++i) {
              const int j = lv - i;
              const uint32_t acc = (chunk_first && i == 0 && lv <= kAcc - 1) ? 0u : 1u;
              const uint64_t ar = smem_desc(sa + (uint32_t)((i * 2 + 0) * 256), kAGroup);
              const uint64_t ai = smem_desc(sa + (uint32_t)((i * 2 + 1) * 256), kAGroup);
              const uint32_t bj = sb + (uint32_t)(j * 3 * kBPlaneMax);
              const uint64_t b_ri = smem_desc(bj + (uint32_t)(NC * kK * 2), kSboB);   // [Br | Bi]
              const uint64_t b_nr = smem_desc(bj, kSboB);                             // [-Bi | Br]
              mma<false>(d, ar, b_ri, idesc, acc);
              mma<false>(d, ai, b_nr, idesc, 1u);
            }
          }
          if (C > 1)
            tc_commit_multicast(smem_u32(&bar_empty[slot]), (uint16_t)((1u << C) - 1u));
          else
            tc_commit(smem_u32(&bar_empty[slot]));
          if (chunk_last) {
            tc_commit(smem_u32(&bar_acc_full));
            ++c_g;
          }
        }
      }
      // every MMA this thread issued completes before TMEM is freed, also after an abort
      tc_commit(smem_u32(&bar_final));
      wait_bounded(smem_u32(&bar_final), 0u, nullptr, prm.status, kWaitCycles);
      if (C > 1 && stop) {
        // after an abort, peers may still be copying into the stages this CTA no longer
        // consumes: let those copies land (bounded) before the cluster leaves
        for (int i = 0; i < kStages; ++i) {
          const long long k = s_g + i;
          wait_bounded(smem_u32(&bar_full[k % kStages]), (uint32_t)((k / kStages) & 1), nullptr,
                       prm.status, kDrainCycles);
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (TMEM lanes)
    const int row = warp * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const int ncols = NC, col0 = 0;
    long long c_g = 0;
    for (long long u = u0; u < prm.total_units; u += du) {
      const OzUnit w = decode(prm, u);
      if (w.slab >= prm.n_slab && tid == 0) atomicOr(prm.status, kStatusBadJob);
      const ContractJob& J = prm.jobs[w.job];
      const int nd1 = J.nd1, nd2 = J.nd2, nd3 = J.nd3, M = nd1 * nd2;
      const int Ncols = prm.P * nd3;
      const int m = w.mt * kOzM + row;
      const bool row_ok = m < M;
      const int n_base = (w.nt * C + (int)rank) * NC;
      const int stride = nd1 + nd2 + nd3;
      const int slab = w.slab < prm.n_slab ? w.slab : 0;
      const float* mx = J.oz_max + (size_t)slab * stride;
      const float* rmx = J.oz_max + (size_t)prm.n_slab * stride + (size_t)slab * M;
      int eA = 0;
      if (row_ok) {
        const int d1 = m / nd2, d2 = m - d1 * nd2;
        eA = exp_a(rmx[m], mx[d1], mx[nd1 + d2]);
      }
      const int n_chunks = (w.n_stages + kChunk - 1) / kChunk;
      for (int ch = 0; ch < n_chunks; ++ch, ++c_g) {
        bool ok = !abort_flag;
        if (ok)
          ok = wait_bounded(smem_u32(&bar_acc_full), (uint32_t)(c_g & 1), &abort_flag,
                            prm.status, prm.wait_limit);
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
          tc_fence_after();
          const bool last = ch == n_chunks - 1;
          // the partial block of this unit's slab, row m, momentum p0 (element p * M nd3 + d3)
          float4* prow = reinterpret_cast<float4*>(J.partial) +
                         (((size_t)w.slab * prm.P_total + prm.p0) * M + (row_ok ? m : 0)) * nd3;
          const int pstride = M * nd3;
          for (int col = col0; col < col0 + ncols; col += 4) {
            __syncwarp();   // tcgen05.ld is warp-aligned; the stores below may diverge
            // the running sums of the 4 columns first (their loads overlap the TMEM reads)
            float4 run[4];
            int ofs[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int n = n_base + col + i;
              const int p = n / nd3;
              ofs[i] = p * pstride + (n - p * nd3);
              run[i] = make_float4(0.f, 0.f, 0.f, 0.f);
              if (ch > 0 && row_ok && n < Ncols) run[i] = prow[ofs[i]];
            }
            float ar[kAcc][4], ai[kAcc][4];
#pragma unroll
            for (int t = 0; t < kAcc; ++t) {
              tmem_ld4(lane_base + (uint32_t)(t * 2 * NC + col), ar[t]);
              tmem_ld4(lane_base + (uint32_t)(t * 2 * NC + NC + col), ai[t]);
            }
            tmem_wait_ld();
            if (!row_ok) continue;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int n = n_base + col + i;
              if (n >= Ncols) break;
              // the chunk's sum: TwoSum of the exact levels, the shared level into the tail
              float2 s0, e0, s1, e1;
              two_sum2(make_float2(ar[0][i], ai[0][i]), make_float2(ar[1][i], ai[1][i]), s0, e0);
              two_sum2(make_float2(ar[2][i], ai[2][i]), make_float2(ar[3][i], ai[3][i]), s1, e1);
              e1 = __fadd2_rn(e1, make_float2(ar[4][i], ai[4][i]));
              float2 h, l;
              two_sum2(s0, s1, h, l);
              l = __fadd2_rn(l, __fadd2_rn(e0, e1));
              if (ch > 0) {
                // running sum += chunk sum (double-float)
                float2 rh, rl;
                two_sum2(make_float2(run[i].x, run[i].z), h, rh, rl);
                rl = __fadd2_rn(rl, __fadd2_rn(make_float2(run[i].y, run[i].w), l));
                two_sum2(rh, rl, h, l);
              }
              if (!last) {
                prow[ofs[i]] = make_float4(h.x, l.x, h.y, l.y);
              } else {
                const int d3 = n - (n / nd3) * nd3;
                const double scale =
                    __longlong_as_double((long long)(1023 + eA + exp_b(mx[nd1 + nd2 + d3])) << 52);
                reinterpret_cast<double2*>(prow)[ofs[i]] =
                    make_double2(((double)h.x + (double)l.x) * scale, ((double)h.y + (double)l.y) * scale);
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        named_bar(kBarEpi, R::kEpiWarps * 32);
        if (tid == 0) mbar_arrive(smem_u32(&bar_acc_empty));
        __syncwarp();
      }
    }
  }

  // ------------------------------------------------------------ teardown
  tc_fence_before();
  __syncwarp();
  __syncthreads();
  // no CTA leaves while a peer may still address its shared memory
  if (C > 1) cluster_sync_all();
  if (warp == R::kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// Column maxima of the fields per site slab (see the header): one block per (field, 64
// sites); thread t takes column t % nd of rows t / nd + lanes * i.
constexpr int kColmaxSites = 64;
__global__ void __launch_bounds__(256) k_oz_colmax(const OzMaxSeg* __restrict__ segs, int X,
                                                    int sites_per_slab) {
  const OzMaxSeg g = segs[blockIdx.y];
  const int nd = g.nd;
  const int lanes = blockDim.x / nd;
  const int t = threadIdx.x;
  if (lanes == 0 || t >= lanes * nd) return;
  const int d = t % nd, lane = t / nd;
  const int x0 = blockIdx.x * kColmaxSites, x1 = min(X, x0 + kColmaxSites);
  float m = 0.f;
  int slab = -1;
  for (int x = x0 + lane; x < x1; x += lanes) {
    const int s = x / sites_per_slab;
    if (s != slab) {
      if (slab >= 0)
        atomicMax(reinterpret_cast<unsigned int*>(g.out + (size_t)slab * g.stride + g.col_off + d),
                  __float_as_uint(m));
      slab = s;
      m = 0.f;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 v = __ldg(g.field + ((size_t)x * 3 + c) * nd + d);
      m = fmaxf(m, g.modulus ? sqrtf(fmaf(v.x, v.x, v.z * v.z)) : fabsf(v.x) + fabsf(v.z));
    }
  }
  if (slab >= 0)
    atomicMax(reinterpret_cast<unsigned int*>(g.out + (size_t)slab * g.stride + g.col_off + d),
              __float_as_uint(m));
}

// Row maxima of the diquark per site slab: for row m = (d1, d2), the largest |Re D_c| or
// |Im D_c| over the slab's sites, spin pairs and colours, D evaluated in FP32 from the
// fields' high parts. Block (site chunk, job x M tile), thread = row; one atomicMax per row
// and slab a chunk touches (the maxima are zeroed before).
constexpr int kRowmaxSites = 32;
__global__ void __launch_bounds__(128) k_oz_rowmax(const __grid_constant__ ContractParams prm,
                                                    int max_m_tiles) {
  const int job = blockIdx.y / max_m_tiles, mt = blockIdx.y % max_m_tiles;
  const ContractJob& J = prm.jobs[job];
  const int M = J.nd1 * J.nd2;
  const int m = mt * kOzM + threadIdx.x;
  if (mt * kOzM >= M || m >= M) return;
  const int nd1 = J.nd1, nd2 = J.nd2, d1 = m / nd2, d2 = m - d1 * nd2;
  const int x0 = blockIdx.x * kRowmaxSites, x1 = min(prm.X, x0 + kRowmaxSites);
  float* rmx = J.oz_max + (size_t)prm.n_slab * (nd1 + nd2 + J.nd3);
  float mxv = 0.f;
  int slab = -1;
  for (int x = x0; x < x1; ++x) {
    const int s = x / prm.sites_per_slab;
    if (s != slab) {
      if (slab >= 0)
        atomicMax(reinterpret_cast<unsigned int*>(rmx + (size_t)slab * M + m), __float_as_uint(mxv));
      slab = s;
      mxv = 0.f;
    }
    for (int pr = 0; pr < prm.n_pairs; ++pr) {
      const float4* uq = reinterpret_cast<const float4*>(J.q1[prm.a_slot[pr]]) + (size_t)x * 3 * nd1 + d1;
      const float4* vq = reinterpret_cast<const float4*>(J.q2[prm.b_slot[pr]]) + (size_t)x * 3 * nd2 + d2;
      float2 u[3], v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 a = __ldg(uq + (size_t)c * nd1), b = __ldg(vq + (size_t)c * nd2);
        u[c] = make_float2(a.x, a.z);
        v[c] = make_float2(b.x, b.z);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
        const float re = u[c1].x * v[c2].x - u[c1].y * v[c2].y - (u[c2].x * v[c1].x - u[c2].y * v[c1].y);
        const float im = u[c1].x * v[c2].y + u[c1].y * v[c2].x - (u[c2].x * v[c1].y + u[c2].y * v[c1].x);
        mxv = fmaxf(mxv, fmaxf(fabsf(re), fabsf(im)));
      }
    }
  }
  if (slab >= 0)
    atomicMax(reinterpret_cast<unsigned int*>(rmx + (size_t)slab * M + m), __float_as_uint(mxv));
}

__global__ void k_phase_df(const double2* __restrict__ ph, float4* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const dcomplex z = dc_from_double2(ph[i]);
    out[i] = make_float4(z.re.h, z.re.l, z.im.h, z.im.l);
  }
}

template <int C>
cudaError_t launch_oz_c(const ContractParams& prm, int grid, cudaStream_t s) {
  using R = OzRoles<C>;
  const size_t smem = (size_t)kStages * kStageBytes;
  auto kern = k_contract_oz<C>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (C == 1) {
    kern<<<grid, R::kThreads, smem, s>>>(prm);
    note_launch();
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(R::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // as many clusters as can be resident at once (a cluster needs C SMs of one GPC)
  cfg.gridDim = dim3((unsigned)(C * grid));
  int max_clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (max_clusters < 1) return cudaErrorInvalidConfiguration;
  cfg.gridDim = dim3((unsigned)(C * std::min(grid, max_clusters)));
  e = cudaLaunchKernelEx(&cfg, kern, prm);
  note_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace


// grid: units wanted at once (clusters of `cluster` CTAs), capped at what is resident
cudaError_t launch_contract_oz(const ContractParams& prm, int cluster, int grid, cudaStream_t s) {
  if (prm.total_units == 0) return cudaSuccess;
  if (prm.NC < 16 || prm.NC > kOzMaxNC || prm.NC % 16 != 0 || prm.n_pairs < 1 ||
      prm.n_pairs > kMaxPairs)
    return cudaErrorInvalidValue;
  switch (cluster) {
    case 1: return launch_oz_c<1>(prm, grid, s);
    case 2: return launch_oz_c<2>(prm, grid, s);
    case 3: return launch_oz_c<3>(prm, grid, s);
    case 4: return launch_oz_c<4>(prm, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_oz_colmax(const OzMaxSeg* d_segs, int n_segs, int X, int sites_per_slab,
                             cudaStream_t s) {
  if (n_segs == 0) return cudaSuccess;
  dim3 grid((unsigned)((X + kColmaxSites - 1) / kColmaxSites), (unsigned)n_segs);
  k_oz_colmax<<<grid, 256, 0, s>>>(d_segs, X, sites_per_slab);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_oz_rowmax(const ContractParams& prm, int max_m_tiles, cudaStream_t s) {
  if (prm.n_jobs == 0 || max_m_tiles == 0) return cudaSuccess;
  dim3 grid((unsigned)((prm.X + kRowmaxSites - 1) / kRowmaxSites), (unsigned)(prm.n_jobs * max_m_tiles));
  k_oz_rowmax<<<grid, 128, 0, s>>>(prm, max_m_tiles);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_phase_df(const double2* ph, float4* out, long long n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  k_phase_df<<<blocks, 256, 0, s>>>(ph, out, n);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bb
