// Tensor-core forms of the fused diquark + contraction (Eq. 1/3) on sm_103a: tcgen05 MMAs
// with FP32 accumulators in tensor memory (TMEM), operands split into BF16, TF32 or FP16
// pieces.
//
// The contraction is a complex GEMM per (time slice, noise triple):
//   C[(d1,d2)][(p,d3)] += sum_k A[(d1,d2)][k] * Bop[k][(p,d3)],   k = (site, spin pair, colour)
//   A   = diquark  (q1_alpha x q2_beta)_c(x)                       (Algorithm 1 "diq")
//   Bop = e^{-i p.x} q3_(alpha beta)[x][c][d3]                     (singlet and phase folded)
// Neither operand exists in HBM: producer warps build both in shared memory for every stage
// of 16 (BF16) or 8 (TF32) (site, pair) groups, split each FP32 value into pieces
// v = v0 + v1 (+ v2) and store them as K-major 8x16-byte core matrices; one thread issues
// the MMAs. Complex products use separate real and imaginary planes. In the three-piece
// BF16 forms and TF32 the third-quark operand is stored as -Bi | Br | Bi, and one complex
// product is two MMAs of N = 2 NC:
//   [Cr | Ci] += Ar [Br | Bi],   [Cr | Ci] += Ai [-Bi | Br];
// the 2-piece BF16 form, bound by its producers rather than by the MMAs, skips the -Bi
// plane and takes four MMAs of N = NC (the -Ai Bi product with the B-negate bit).
// Accuracy: the TMEM accumulator rounds towards zero, so the leading piece product (v0 w0)
// goes to its own accumulator and is drained every `chunk_stages` stages into an FP32
// running sum (round to nearest) kept in TMEM; the smaller correction products share a
// second accumulator. Each work unit (job, 128 pairs, NC columns, site slab) writes its
// running sum as an FP32 partial block; the slab partials are summed in FP64 in index order.
//
// The FP16 form (two pieces per operand, scaled per job by powers of two) has two faster
// variants: CTA pairs sharing the third-quark tile, and the row-factored phase, which
// multiplies the third quark by w^{n0 x0} for each distinct x-component n0 of the momenta
// only (w = e^{-2 pi i / L}) and applies w^{n1 x1 + n2 x2} per lattice row in the epilogue;
// there the drained chunks are summed per row in shared memory and each complete row goes
// into the running sum of every momentum (the batched workload's default, in clusters of two
// CTAs that share the diquark tile; details before tc_body).
//
// Clusters (BF16 forms): C CTAs of a thread-block cluster take the same (job, 128 pairs,
// slab) and C neighbouring N tiles. Each builds only 128/C rows of the diquark tile and
// pushes them into the other CTAs' stage buffers with bulk shared::cta -> shared::cluster
// copies, counted as transaction bytes on the peers' stage barriers; each CTA's MMA
// completion arrives on the stage-free barriers of all C CTAs (multicast commit). The
// diquark is then built once per cluster instead of once per N tile. Measured, this pays
// only for wide blocks (13 % at 448 columns with C = 2): the stage time barely falls with
// the diquark work per CTA. C = 1 is the plain kernel.
//
// Projection (k_project_tc, opt-in): the same pipeline computes Eq. 2 for the mixed forms,
// q[m][n] = sum_l V[l][m] Phi[l][n], with A rows the (site, colour) rows of V, B rows a
// field's coefficient-folded phi columns, and a stage's K element read as the eigenvector
// index; each unit writes its FP32 field tile. Measured slower than the FP32 FMA projection
// at N_ev = 96-264 (the producers wait on V loads), so it is not the default.
//
// Warp roles: 0-3 epilogue (TMEM lanes 0-127: drains, partial write-out), 4 MMA issue and
// TMEM allocation, 5.. operand producers (11 warps for BF16, 6 for TF32). Every wait is
// bounded; on a timeout the CTA raises an abort flag and a status bit, the roles run out
// their loops without waiting or computing, the MMA thread waits (bounded) for its
// outstanding MMAs and the allocating warp frees TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <type_traits>

#include "bblock_internal.h"
#include "tc_ptx.cuh"

namespace bb {
namespace {

constexpr int kTcM = 128;
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kProdWarp0 = 5;
constexpr int kTmemCols = 512;
// Producer warps: one 8-group item per thread. BF16 stages hold 16 groups (two halves per
// row): 8 warps build the 128-row diquark tile, 3 warps the <= 48-row third-quark tile.
// TF32 stages hold 8 groups: 4 + 2 warps.
constexpr int kMaxNC = 48;
// With a cluster of C CTAs each builds kARows = 128 / C diquark rows: one item per thread of
// kAGroups groups (8 rows x 4 items per warp, one 8-row core-matrix group per warp, so that
// a warp's rows are one contiguous 768-byte run per plane). Third-quark items hold
// kBGroups groups. The producer warp count is fixed (11 BF16, 6 TF32); spare threads idle.
template <bool TF32, int C> struct Roles {
  static constexpr int G = TF32 ? 8 : 16;
  static constexpr int kARows = kTcM / C;
  static constexpr int kAGroups = C == 1 ? 8 : 4;
  static constexpr int kBGroups = C <= 2 ? 8 : 4;
  static constexpr int kAThreads = kARows * (G / kAGroups);
  static constexpr int kBThreads = kMaxNC * (G / kBGroups);
  static constexpr int kProdThreads = TF32 ? 192 : 352;
  static constexpr int kThreads = kProdWarp0 * 32 + kProdThreads;
  static_assert(kAThreads % 32 == 0 && kAThreads + kBThreads <= kProdThreads, "producer roles");
  static_assert(!TF32 || C == 1, "clusters are built for the BF16 forms");
};
constexpr int kBarProd = 1, kBarEpi = 2;
constexpr int kAPlaneBytes = kTcM * 96;          // 128 rows x 96 bytes of K per stage
// The third-quark operand of each piece level holds three planes, -Bi | Br | Bi, each of NC
// rows (NC * 96 bytes, so that consecutive planes continue one another's 8-row groups).
// Then [Br | Bi] and [-Bi | Br] are both contiguous operands of 2 NC rows, and a complex
// product takes two MMAs of N = 2 NC into the adjacent [Cr | Ci] accumulator columns:
//   [Cr | Ci] += Ar [Br | Bi],   [Cr | Ci] += Ai [-Bi | Br].
// Each reads the 128-row A tile once, half as often as four N = NC real products would.
// Measured, this pays in the three-piece BF16 forms (14 % at L = 48) and in TF32 (3 %).
// The 2-piece BF16 form, bound by its producers, loses 2-4 % to the extra -Bi stores and
// the larger stages (less L1 for the producers' loads): it keeps two planes, Br | Bi, and
// four MMAs of N = NC.
// WIDE (the CTA-pair form): N tiles of up to kMaxNCWide complex columns, two stages.
// TWO (the row-factored form): two stages of the narrow layout; the epilogue's row sums take
// the third stage's room.
template <bool TF32, int LEVELS, bool F16 = false, bool WIDE = false, bool TWO = false>
struct TcLayout {
  static constexpr bool kTwoMma = TF32 || LEVELS == 3 || F16;
  static constexpr int kBPlanes = kTwoMma ? 3 : 2;
  static constexpr int kBr = kTwoMma ? 1 : 0, kBi = kBr + 1;   // plane slots; -Bi is slot 0
  static constexpr int kMaxCols = WIDE ? 80 : kMaxNC;          // complex columns per N tile
  static constexpr int kBPlaneB = kMaxCols * 96;               // bytes of one B plane
  static constexpr int kStages = (LEVELS == 3 || WIDE || TWO) ? 2 : 3;
  static constexpr int kStageBytes = LEVELS * (2 * kAPlaneBytes + kBPlanes * kBPlaneB);
};
constexpr int kMaxNCWide = 80;
constexpr int kSegsPerRow = 6;                   // 16-byte core-matrix columns per row

// ------------------------------------------------------------------ operand splitting

__device__ __forceinline__ float tf32_round(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// Split 8 FP32 values into LEVELS pieces and store each piece's 8 values as one K run of
// a core-matrix row (16 bytes of BF16, or 32 bytes = two 16-byte rows of TF32).
// BF16: the pieces are successive truncations to the top 8 significant bits,
//   v0 = trunc8(v), v1 = trunc8(v - v0), v2 = (v - v0) - v1,
// every subtraction is exact and v2 has at most 8 significant bits, so v0 + v1 + v2 == v;
// with two pieces the second is rounded to nearest (error <= 2^-17 |v|).
// TF32: v0 = trunc11(v), v1 = rn_tf32(v - v0) (error <= 2^-21 |v|).
// With `neg` set, the pieces of -v go to neg[l] as well: both splits are symmetric under
// negation (truncation, round-to-nearest-even, TF32 round-half-away), so they are the
// stored pieces with their sign bits flipped.
template <bool TF32, int LEVELS, int NG = 8>
__device__ __forceinline__ void split_store8(const float (&v)[8], uint8_t* const (&dst)[LEVELS],
                                             uint8_t* const* neg) {
  static_assert(NG == 8 || (NG == 4 && !TF32), "K runs of 8 (BF16, TF32) or 4 (BF16) values");
  if (!TF32) {
    float r[8];
#pragma unroll
    for (int i = 0; i < NG; ++i) r[i] = v[i];
#pragma unroll
    for (int l = 0; l < LEVELS; ++l) {
      uint32_t piece[8];
#pragma unroll
      for (int i = 0; i < NG; ++i) {
        if (l < LEVELS - 1) {
          piece[i] = __float_as_uint(r[i]) & 0xFFFF0000u;
          r[i] -= __uint_as_float(piece[i]);
        } else if (LEVELS == 3) {
          piece[i] = __float_as_uint(r[i]);       // exact in BF16
        } else {
          const __nv_bfloat16 h = __float2bfloat16_rn(r[i]);
          piece[i] = (uint32_t)(*reinterpret_cast<const uint16_t*>(&h)) << 16;
        }
      }
      if (NG == 8) {
        uint4 w;
        w.x = __byte_perm(piece[0], piece[1], 0x7632);
        w.y = __byte_perm(piece[2], piece[3], 0x7632);
        w.z = __byte_perm(piece[4], piece[5], 0x7632);
        w.w = __byte_perm(piece[6], piece[7], 0x7632);
        *reinterpret_cast<uint4*>(dst[l]) = w;
        if (neg) {
          constexpr uint32_t m = 0x80008000u;
          *reinterpret_cast<uint4*>(neg[l]) = make_uint4(w.x ^ m, w.y ^ m, w.z ^ m, w.w ^ m);
        }
      } else {
        uint2 w;
        w.x = __byte_perm(piece[0], piece[1], 0x7632);
        w.y = __byte_perm(piece[2], piece[3], 0x7632);
        *reinterpret_cast<uint2*>(dst[l]) = w;
        if (neg) {
          constexpr uint32_t m = 0x80008000u;
          *reinterpret_cast<uint2*>(neg[l]) = make_uint2(w.x ^ m, w.y ^ m);
        }
      }
    }
  } else {
    float h[8], lo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i] = __uint_as_float(__float_as_uint(v[i]) & 0xFFFFE000u);
      lo[i] = tf32_round(v[i] - h[i]);
    }
    // a 32-byte K run spans two adjacent core matrices along K (128 bytes apart)
    *reinterpret_cast<float4*>(dst[0]) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(dst[0] + 128) = make_float4(h[4], h[5], h[6], h[7]);
    *reinterpret_cast<float4*>(dst[1]) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<float4*>(dst[1] + 128) = make_float4(lo[4], lo[5], lo[6], lo[7]);
    if (neg) {
      *reinterpret_cast<float4*>(neg[0]) = make_float4(-h[0], -h[1], -h[2], -h[3]);
      *reinterpret_cast<float4*>(neg[0] + 128) = make_float4(-h[4], -h[5], -h[6], -h[7]);
      *reinterpret_cast<float4*>(neg[1]) = make_float4(-lo[0], -lo[1], -lo[2], -lo[3]);
      *reinterpret_cast<float4*>(neg[1] + 128) = make_float4(-lo[4], -lo[5], -lo[6], -lo[7]);
    }
  }
}

// FP16 hi/lo pieces of 8 FP32 values already scaled into FP16's range (|v| < 2^15):
//   hi = rn16(v), lo = rn16(v - hi);
// v - hi is exact in FP32, so v = hi + lo + r with |r| <= 2^-23 |v| while lo is a normal
// FP16 number (smaller values keep an absolute error below 2^-25). Round-to-nearest-even is
// symmetric under negation, so the pieces of -v are the stored pieces with the sign bits
// (bit 15 of each half) flipped.
// NG = 8 values (one 16-byte K run per piece) or the first 4 (8 bytes).
template <int NG = 8>
__device__ __forceinline__ void split_store8_f16(const float (&v)[8], uint8_t* const (&dst)[2],
                                                 uint8_t* const* neg) {
  static_assert(NG == 8 || NG == 4, "K runs of 8 or 4 values");
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int i = 0; i < NG / 2; ++i) {
    const __half2 h = __floats2half2_rn(v[2 * i], v[2 * i + 1]);   // .x = low 16 bits
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
    hw[i] = *reinterpret_cast<const uint32_t*>(&h);
    lw[i] = *reinterpret_cast<const uint32_t*>(&l);
  }
  constexpr uint32_t m = 0x80008000u;
  if (NG == 8) {
    *reinterpret_cast<uint4*>(dst[0]) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(dst[1]) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    if (neg) {
      *reinterpret_cast<uint4*>(neg[0]) = make_uint4(hw[0] ^ m, hw[1] ^ m, hw[2] ^ m, hw[3] ^ m);
      *reinterpret_cast<uint4*>(neg[1]) = make_uint4(lw[0] ^ m, lw[1] ^ m, lw[2] ^ m, lw[3] ^ m);
    }
  } else {
    *reinterpret_cast<uint2*>(dst[0]) = make_uint2(hw[0], hw[1]);
    *reinterpret_cast<uint2*>(dst[1]) = make_uint2(lw[0], lw[1]);
    if (neg) {
      *reinterpret_cast<uint2*>(neg[0]) = make_uint2(hw[0] ^ m, hw[1] ^ m);
      *reinterpret_cast<uint2*>(neg[1]) = make_uint2(lw[0] ^ m, lw[1] ^ m);
    }
  }
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ int tc_find_job(const TcJob* jobs, int n_jobs, long long u) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct Unit {
  int job, mt, nt, slab, x_begin, x_end, n_stages;
};

// Power-of-two scales of the FP16 form, from the largest |Re| or |Im| (FP32 bits) of the
// fields of each quark line of a job, amax[0..2]. With e_i = floor(log2 max_i):
//   diquark  |Re|, |Im| of q1_a q2_b - q1_b q2_a  <= 4 max_1 max_2 < 2^(e1 + e2 + 4),
//   phase x third quark                             <= sqrt(2) max_3  < 2^(e3 + 1.5),
// so the scales 2^eA with eA = 10 - e1 - e2 and 2^eB with eB = 12 - e3 keep both operands
// below 2^14 (FP16 holds up to 65504). Both are clamped to normal FP32 powers of two; the
// clamp only binds where FP32 itself would overflow or the values are below 2^-116. The
// slab reduction divides the sum by 2^(eA + eB) in FP64 (exact). A zero or non-finite
// maximum gives a clamped exponent; non-finite inputs stay non-finite.
__device__ __forceinline__ int f16_floor_log2(uint32_t bits) {
  const int be = (int)((bits >> 23) & 0xFFu);
  if (be == 0xFF) return 200;                           // inf or NaN
  if ((bits & 0x7FFFFFFFu) == 0u) return -200;          // zero
  return be == 0 ? -127 : be - 127;                     // subnormal: max < 2^-126
}
__device__ __forceinline__ void f16_scale_exps(const uint32_t* amax, int& eA, int& eB) {
  const int e1 = f16_floor_log2(amax[0]), e2 = f16_floor_log2(amax[1]);
  const int e3 = f16_floor_log2(amax[2]);
  eA = min(126, max(-126, 10 - e1 - e2));
  eB = min(126, max(-126, 12 - e3));
}
__device__ __forceinline__ float pow2f(int e) {        // e in [-126, 127]
  return __int_as_float((127 + e) << 23);
}

// Index check of the debug option: false (and the first violation recorded) if i is
// outside [0, n).
__device__ __forceinline__ bool idx_ok(const TcParams& prm, long long i, long long n, int code,
                                       int job) {
  if (i >= 0 && i < n) return true;
  if (atomicCAS(prm.dbg, 0ull, (unsigned long long)code) == 0ull) {
    prm.dbg[1] = (unsigned long long)job;
    prm.dbg[2] = (unsigned long long)i;
    prm.dbg[3] = (unsigned long long)n;
  }
  atomicOr(prm.status, kStatusBadIndex);
  return false;
}

__device__ __forceinline__ Unit decode_unit(const TcParams& prm, long long u, int G) {
  Unit w;
  w.job = tc_find_job(prm.jobs, prm.n_jobs, u);
  const TcJob& J = prm.jobs[w.job];
  long long r = u - J.unit_begin;
  w.mt = (int)(r % J.m_tiles);
  r /= J.m_tiles;
  w.nt = (int)(r % J.n_tiles);
  w.slab = (int)(r / J.n_tiles);
  w.x_begin = w.slab * prm.sites_per_slab;
  w.x_end = min(prm.X, w.x_begin + prm.sites_per_slab);
  const int groups = (w.x_end - w.x_begin) * prm.n_pairs;
  w.n_stages = (groups + G - 1) / G;
  return w;
}

// Row-factored units: (job, 128-pair tile, N tile, slab of lattice rows); x_begin / x_end
// are rows, and every row takes rf_spr stages.
__device__ __forceinline__ Unit decode_unit_rf(const TcParams& prm, long long u) {
  Unit w;
  w.job = tc_find_job(prm.jobs, prm.n_jobs, u);
  const TcJob& J = prm.jobs[w.job];
  long long r = u - J.unit_begin;
  w.mt = (int)(r % J.m_tiles);
  r /= J.m_tiles;
  w.nt = (int)(r % J.n_tiles);
  w.slab = (int)(r / J.n_tiles);
  w.x_begin = w.slab * prm.rf_rows_per_slab;
  w.x_end = min(prm.L * prm.L, w.x_begin + prm.rf_rows_per_slab);
  w.n_stages = (w.x_end - w.x_begin) * prm.rf_spr;
  return w;
}

// Projection units: (128-row tile, field, N tile), the row tile outermost so that the CTAs
// running at once share their V tiles in L2; the K sum (eigenvector index l) runs over
// ceil(N_ev / KS) stages. N tiles past the field's columns are empty.
__device__ __forceinline__ Unit decode_unit_proj(const TcParams& prm, long long u, int KS) {
  Unit w;
  const long long per_row_tile = (long long)prm.p_n_fields * prm.p_n_tiles;
  w.mt = (int)(u / per_row_tile);
  const long long r = u - (long long)w.mt * per_row_tile;
  w.job = (int)(r / prm.p_n_tiles);
  w.nt = (int)(r - (long long)w.job * prm.p_n_tiles);
  w.slab = 0;
  w.x_begin = 0;
  w.x_end = 0;
  w.n_stages = w.nt * prm.NC < prm.pfields[w.job].nd ? (prm.p_n_ev + KS - 1) / KS : 0;
  return w;
}


// The body of both tensor-core kernels. PROJ = false: the contraction (diquark x phase x
// third quark). PROJ = true: the projection of Eq. 2, q[m][n] = sum_l V[l][m] Phi[l][n]
// with m = (site, colour) and Phi the coefficient-folded phi columns of one field; the same
// pipeline with the K index of a stage read as the eigenvector index
// l = stage * 3G + colour * G + group, and the unit's sum written as the FP32 field.
//
// SHB (C = 2, the FP16 form): the CTA pair form. Both CTAs of a cluster take the same
// (job, N tile, slab) and adjacent 128-row M tiles; each builds its own diquark rows and
// half of the third-quark rows, and pushes that half into the peer's stage (bulk
// shared::cta -> shared::cluster copies counted on the peer's stage barrier). Each CTA
// then runs its own MMAs on its diquark rows and the whole third-quark tile, which can be
// up to 80 complex columns wide because the accumulators are single-buffered there.
//
// RF (C = 1, the FP16 form): the row-factored phase. A chunk of MMAs never crosses a lattice
// row; the B rows are (idx0, d3) with the factor w^{n0 x0} of the idx0-th distinct n0; the
// epilogue adds each drained chunk into the row's sums, and each complete row, times its
// w^{n1 x1 + n2 x2}, into the running sum of every momentum with that n0. Two stage buffers
// (N tiles of at most 48 columns), then the w table and the row sums in shared memory.
template <bool TF32, int LEVELS, int NPROD, bool CHECKS, int C, bool PROJ, bool F16 = false,
          bool SHB = false, bool RF = false>
__device__ __forceinline__ void tc_body(const TcParams& prm) {
  using R = Roles<TF32, SHB ? 1 : C>;
  static_assert(!RF || (F16 && (C == 1 || (C == 2 && !SHB)) && !CHECKS && !PROJ),
                "row-factored: FP16, plain CTAs or pairs sharing the diquark tile");
  static_assert(!PROJ || (C == 1 && !CHECKS), "the projection runs without clusters or checks");
  static_assert(!F16 || (!TF32 && LEVELS == 2 && (C == 1 || SHB || RF) && !PROJ),
                "the FP16 form: two pieces, contraction only, clusters only as CTA pairs");
  static_assert(!SHB || (F16 && C == 2 && !CHECKS), "CTA pairs: the FP16 form, unchecked");
  constexpr bool kShareA = C > 1 && !SHB;          // cluster CTAs share the diquark tile
  constexpr int G = TF32 ? 8 : 16;                 // (site, pair) groups per stage
  // transaction bytes a stage receives from the peers: their diquark rows, every plane
  constexpr uint32_t kPeerTx = (uint32_t)((C - 1) * (R::kARows / 8) * 768 * LEVELS * 2);
  using Lay = TcLayout<TF32, LEVELS, F16, SHB, RF>;
  constexpr int STAGES = Lay::kStages;
  constexpr int STAGE_BYTES = Lay::kStageBytes;
  constexpr bool kTwoMma = Lay::kTwoMma;   // complex product as two N = 2 NC MMAs
  constexpr int kBPlanes = Lay::kBPlanes;
  // groups whose loads a producer thread issues together before computing: all 8 in one
  // round where the registers allow it; the A-sharing cluster and checked variants would spill
  constexpr int kLoadRun = (!kShareA && !CHECKS) ? 8 : 4;
  auto decode = [&](long long u) -> Unit {
    if constexpr (PROJ) return decode_unit_proj(prm, u, 3 * G);
    else if constexpr (RF) return decode_unit_rf(prm, u);
    else return decode_unit(prm, u, G);
  };
  // piece products (i, j): leading (0, 0) first, then by increasing i + j
  constexpr int PI[9] = {0, 0, 1, 1, 0, 2, 1, 2, 2};
  constexpr int PJ[9] = {0, 1, 0, 1, 2, 0, 2, 1, 2};

  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_full[STAGES], bar_empty[STAGES];
  __shared__ __align__(8) uint64_t bar_acc_full[2], bar_acc_empty[2], bar_final;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  // per-unit field pointers of every spin pair
  __shared__ const float2* s_q1[kMaxPairs];
  __shared__ const float2* s_q2[kMaxPairs];
  __shared__ const float2* s_q3[kMaxPairs];
  // row-factored: the phase per momentum of the current lattice row and of the previous one
  // (epilogue; by row parity, so that a warp may start a row while another finishes the last)
  __shared__ float2 s_rowph[2][kMaxRfP];
  __shared__ uint32_t s_rfmask[kMaxRfIdx];

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int NC = prm.NC;
  const int np = prm.n_pairs;
  // accumulator buffers: double-buffered [lead | corr] (4 NC columns each) and the FP32
  // running sum (2 NC) while 10 NC <= 512 TMEM columns; single-buffered beyond
  const int nbuf = (!RF && 10 * NC <= kTmemCols) ? 2 : 1;
  // CTA pairs: transaction bytes of the peer's third-quark rows (NC / 2 rows, every plane)
  const uint32_t peer_tx = SHB ? (uint32_t)((NC / 16) * LEVELS * Lay::kBPlanes * 768) : kPeerTx;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&bar_full[s]), R::kProdThreads / 32);   // one arrival per producer warp
      mbar_init(smem_u32(&bar_empty[s]), C);   // the MMA completion of every CTA of the cluster
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_acc_full[b]), 1);
      mbar_init(smem_u32(&bar_acc_empty[b]), 1);
    }
    mbar_init(smem_u32(&bar_final), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // row-factored: the w^k table after the stage buffers, then the row sums of the epilogue
  float2* s_omega = reinterpret_cast<float2*>(smem + STAGES * STAGE_BYTES);
  float4* s_trow = reinterpret_cast<float4*>(smem + STAGES * STAGE_BYTES + kMaxRfL * sizeof(float2));
  if constexpr (RF) {
    for (int k = tid; k < prm.L; k += blockDim.x) s_omega[k] = prm.rf_omega[k];
    // the momenta of each distinct n0, as a bit mask
    if (tid < prm.rf_nidx) {
      uint32_t msk = 0;
      for (int p = 0; p < prm.P; ++p) msk |= (prm.rf_pidx0[p] == tid ? 1u : 0u) << p;
      s_rfmask[tid] = msk;
    }
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&tmem_slot)), "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  if (C > 1) cluster_sync_all();   // peers signal this CTA's barriers only once they exist
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t smem_base = smem_u32(smem);
  // work units are shared by the C CTAs of a cluster; rank r takes N tile (group * C + r)
  const uint32_t rank = C > 1 ? cluster_rank() : 0u;
  const long long u0 = blockIdx.x / C, du = gridDim.x / C;

  auto a_plane = [&](int stage, int level, int plane) -> uint32_t {
    return (uint32_t)(stage * STAGE_BYTES + (level * 2 + plane) * kAPlaneBytes);
  };
  // plane slots: -Bi = 0, Br = 1, Bi = 2 (two-MMA forms); Br = 0, Bi = 1 (the others)
  auto b_plane = [&](int stage, int level, int plane) -> uint32_t {
    return (uint32_t)(stage * STAGE_BYTES + LEVELS * 2 * kAPlaneBytes +
                      level * kBPlanes * Lay::kBPlaneB + plane * NC * 96);
  };
  auto row_seg = [](int r, int seg) -> uint32_t {
    return (uint32_t)(((r >> 3) * kSegsPerRow + seg) * 128 + (r & 7) * 16);
  };

  if (warp >= kProdWarp0) {
    // ------------------------------------------------------------ producers
    // Thread roles are fixed: pt < kAThreads builds diquark rows (M side), the next
    // kBThreads build phase x third-quark rows (N side); each thread owns one row and NG
    // consecutive groups (starting at g0) of every stage.
    const int pt = tid - kProdWarp0 * 32;
    const bool is_a = pt < R::kAThreads;
    const bool is_b = !is_a && pt < R::kAThreads + R::kBThreads;
    int rr, g0;
    bool b_row_in = false;   // a third-quark row of this CTA's share
    if (is_a) {
      if (!kShareA) {
        rr = pt % kTcM;
        g0 = (pt / kTcM) * 8;
      } else {
        // 8 rows x 4 runs of 4 groups per warp: the warp's rows are one core-matrix row group.
        // Lanes 8q .. 8q + 7 take run q of the 8 rows, so that each half-warp's 8-byte stores
        // fill one 128-byte core-matrix column (runs 0, 1: K bytes 0-15 of colour c; runs 2, 3:
        // the next column) without bank conflicts.
        rr = (int)rank * R::kARows + (pt / 32) * 8 + (lane & 7);
        g0 = (lane >> 3) * 4;
      }
    } else {
      const int b = is_b ? pt - R::kAThreads : 0;
      if (SHB) {   // 16 rows x 2 halves per warp: two whole core-matrix row groups per warp
        const int lr = (b / 32) * 16 + (lane & 15);
        rr = (int)rank * (NC / 2) + lr;
        g0 = (lane >> 4) * 8;
        b_row_in = lr < NC / 2;
      } else {
        rr = b % kMaxNC;
        g0 = (b / kMaxNC) * R::kBGroups;
        b_row_in = rr < NC;
      }
    }
    const int NG = is_a ? R::kAGroups : R::kBGroups;
    const bool row_used = is_a || (is_b && b_row_in);
    // row-factored: a stage's first group (site x0 = xl of its lattice row, pair pr) and the
    // phase index (n0 x0) mod L advance incrementally from stage to stage, with no division
    // in the stage loop: each stage moves G groups on (G / np sites and G % np pairs)
    const int rf_gq = RF ? G / prm.n_pairs : 0, rf_gr = RF ? G % prm.n_pairs : 0;
    const int rf_xl0 = RF ? g0 / prm.n_pairs : 0, rf_pr0 = RF ? g0 % prm.n_pairs : 0;
    int rf_sub = 0, rf_row = 0, rf_xl = 0, rf_pr = 0, rf_ph = 0, rf_ph0 = 0, rf_step = 0;
    long long s_g = 0;
    for (long long u = u0; u < prm.total_units; u += du) {
      const Unit w = decode(u);
      // per-unit constants of this thread's row
      bool row_ok = false;
      int off1 = 0, off2 = 0, s1 = 0, s2 = 0, pidx = 0;
      const float2* phase_p = nullptr;
      float f16s = 1.f;   // FP16 form: this row's power-of-two scale (diquark or phase side)
      // projection: the unit's field, read once per unit (A: V column m; B: the folded
      // phi column n, its terms' rows and FP32 weights)
      const float2* p_src = nullptr;
      int p_nd = 0, p_terms = 0;
      int p_off[kMaxTerms] = {};
      float2 p_w[kMaxTerms];
      if constexpr (PROJ) {
        const ProjFieldF& F = prm.pfields[w.job];
        p_nd = F.nd;
        off1 = is_a ? w.mt * kTcM + rr : w.nt * NC + rr;
        row_ok = is_a ? off1 < prm.p_rows : (row_used && off1 < p_nd);
        if (is_a) {
          p_src = F.V + off1;
        } else {
          p_src = F.phi + off1;
          p_terms = F.n_terms;
#pragma unroll
          for (int t = 0; t < kMaxTerms; ++t) {
            p_off[t] = t < p_terms ? F.row_off[t] * p_nd : 0;
            p_w[t] = t < p_terms ? make_float2((float)F.w[t].x, (float)F.w[t].y)
                                 : make_float2(0.f, 0.f);
          }
        }
      } else {
        const TcJob& J = prm.jobs[w.job];
        const int nd1 = J.nd1, nd2 = J.nd2, nd3 = J.nd3;
        if constexpr (F16) {
          int eA, eB;
          f16_scale_exps(J.amax, eA, eB);
          f16s = pow2f(is_a ? eA : eB);
        }
        if (is_a) {
          // M side: diquark of the pair m = d1 * nd2 + d2 (CTA pairs: M tile 2 mt + rank)
          const int m = (SHB ? w.mt * 2 + (int)rank : w.mt) * kTcM + rr;
          row_ok = m < nd1 * nd2;
          const int d1 = row_ok ? m / nd2 : 0, d2 = row_ok ? m - d1 * nd2 : 0;
          off1 = d1; off2 = d2; s1 = nd1; s2 = nd2;
        } else if constexpr (RF) {
          // N side: w^{n0 x0} x third quark of the row (idx0, d3); pidx holds n0 (mod L)
          const int idx0 = rr / prm.rf_nc;
          const int d3 = (kShareA ? w.nt * C + (int)rank : w.nt) * prm.rf_nc + (rr - idx0 * prm.rf_nc);
          row_ok = row_used && d3 < nd3 && idx0 < prm.rf_nidx;
          off1 = row_ok ? d3 : 0; s1 = nd3; pidx = row_ok ? prm.rf_n0[idx0] : 0;
        } else {
          // N side: phase x third quark of the column n = p * nd3 + d3
          const int n = (kShareA ? w.nt * C + (int)rank : w.nt) * NC + rr;
          row_ok = row_used && n < prm.P * nd3;
          const int p = row_ok ? n / nd3 : 0, d3 = row_ok ? n - p * nd3 : 0;
          off1 = d3; s1 = nd3; pidx = p;
        }
        // Producer warps run their stages independently; at a unit boundary they meet twice:
        // once so that no warp still reads the previous unit's pointer table while it is
        // rewritten, once to publish the new table. (bar.sync is warp-aligned: reconverge
        // every warp before it.)
        __syncwarp();
        named_bar(kBarProd, R::kProdThreads);
        if (pt < np) {
          s_q1[pt] = J.q1[prm.a_slot[pt]];
          s_q2[pt] = J.q2[prm.b_slot[pt]];
          s_q3[pt] = J.q3[pt];
        }
        __syncwarp();
        named_bar(kBarProd, R::kProdThreads);
        if constexpr (!RF) phase_p = prm.phase + (size_t)pidx * prm.X;
        if constexpr (RF) {
          rf_ph0 = (pidx * rf_xl0) % prm.L;
          rf_step = (pidx * rf_gq) % prm.L;
          rf_sub = 0; rf_row = 0;
          rf_xl = rf_xl0; rf_pr = rf_pr0; rf_ph = rf_ph0;
        }
      }
      for (int st = 0; st < w.n_stages; ++st, ++s_g) {
        const int slot = (int)(s_g % STAGES);
        bool ok = !abort_flag;
        if (ok && s_g >= STAGES)
          ok = wait_bounded(smem_u32(&bar_empty[slot]), (uint32_t)(((s_g / STAGES) + 1) & 1),
                            &abort_flag, prm.status, prm.wait_limit);
        // a warp either fills its rows of this stage or (after an abort) none of them
        ok = __all_sync(0xffffffffu, ok);
        if (ok && row_used) {
          float re[3][8], im[3][8];
          if constexpr (PROJ) {
            // element (colour c, group g0 + j) of this stage is eigenvector index l
            const int rows = prm.p_rows, n_ev = prm.p_n_ev;
            if (is_a) {
              float2 v[3][8];
#pragma unroll
              for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const int l = st * 3 * G + c * G + g0 + j;
                  v[c][j] = (j < NG && row_ok && l < n_ev) ? p_src[(size_t)l * rows]
                                                           : make_float2(0.f, 0.f);
                }
#pragma unroll
              for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int j = 0; j < 8; ++j) { re[c][j] = v[c][j].x; im[c][j] = v[c][j].y; }
            } else {
#pragma unroll
              for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const int l = st * 3 * G + c * G + g0 + j;
                  float2 b = make_float2(0.f, 0.f);
                  if (j < NG && row_ok && l < n_ev) {
#pragma unroll
                    for (int t = 0; t < kMaxTerms; ++t)
                      if (t < p_terms) {
                        const float2 f = p_src[(size_t)p_off[t] + (size_t)l * p_nd];
                        b.x = fmaf(p_w[t].x, f.x, fmaf(-p_w[t].y, f.y, b.x));
                        b.y = fmaf(p_w[t].x, f.y, fmaf(p_w[t].y, f.x, b.y));
                      }
                  }
                  re[c][j] = b.x;
                  im[c][j] = b.y;
                }
            }
          } else {
            // the stage's sites [sx0, sx1) and this thread's first group of its run of NG
            // (row-factored: the stage's row, groups counted from the row's first site)
            int sx0 = w.x_begin, sx1 = w.x_end, xl, pr, ph = 0;
            if constexpr (RF) {
              sx0 = (w.x_begin + rf_row) * prm.L;
              sx1 = sx0 + prm.L;
              xl = rf_xl; pr = rf_pr; ph = rf_ph;
            } else {
              const int gi0 = st * G + g0;
              xl = gi0 / np;
              pr = gi0 - xl * np;
            }
            uint32_t vmask = 0;   // groups of this run that lie inside the slab and a used row
            // One role's groups, with their group count and loads per group known at compile
            // time, so that each role's load buffers take only its own registers: the
            // diquark side loads 6 values per group in rounds of kLoadRun groups, the
            // third-quark side 4 per group, all of its groups in one round (unchecked).
            auto build = [&](auto kNG, auto kIsA) {
              constexpr int NGc = decltype(kNG)::value;
              constexpr bool Ac = decltype(kIsA)::value;
              constexpr int LR = Ac ? (kLoadRun < NGc ? kLoadRun : NGc) : (CHECKS ? 4 : NGc);
              constexpr int NV = Ac ? 6 : 4;
#pragma unroll
              for (int half = 0; half < NGc / LR; ++half) {
                // LR groups: issue every load first, then compute
                float2 ld[LR][NV];
                bool vld[LR];
#pragma unroll
                for (int j = 0; j < LR; ++j) {
                  const int x = sx0 + xl;
                  vld[j] = row_ok && x < sx1;
                  int xs = vld[j] ? x : sx0;
                  if (CHECKS) {
                    const long long fl = 3LL * prm.X * s1;            // elements of a field
                    bool good = idx_ok(prm, (long long)xs * 3 * s1 + off1 + 2LL * s1, fl, Ac ? 1 : 3, w.job) &&
                                idx_ok(prm, pr, np, 6, w.job);
                    if (Ac) good = good && idx_ok(prm, (long long)xs * 3 * s2 + off2 + 2LL * s2, 3LL * prm.X * s2, 2, w.job);
                    else good = good && idx_ok(prm, (long long)pidx * prm.X + xs, (long long)prm.P * prm.X, 4, w.job);
                    if (!good) { vld[j] = false; xs = 0; pr = 0; }
                  }
                  if constexpr (Ac) {
                    const float2* uq = s_q1[pr] + (size_t)xs * 3 * s1 + off1;
                    const float2* vq = s_q2[pr] + (size_t)xs * 3 * s2 + off2;
                    ld[j][0] = uq[0]; ld[j][1] = uq[s1]; ld[j][2] = uq[2 * s1];
                    ld[j][3] = vq[0]; ld[j][4] = vq[s2]; ld[j][5] = vq[2 * s2];
                  } else {
                    const float2* q = s_q3[pr] + (size_t)xs * 3 * s1 + off1;
                    ld[j][0] = q[0]; ld[j][1] = q[s1]; ld[j][2] = q[2 * s1];
                    if constexpr (RF) ld[j][3] = s_omega[ph];
                    else ld[j][3] = phase_p[xs];
                  }
                  if (++pr == np) {
                    pr = 0;
                    ++xl;
                    if constexpr (RF) {
                      ph += pidx;
                      if (ph >= prm.L) ph -= prm.L;
                    }
                  }
                }
#pragma unroll
                for (int j = 0; j < LR; ++j) {
                  float2 c0, c1, c2;
                  if constexpr (Ac) {
                    const float2 u0 = ld[j][0], u1 = ld[j][1], u2 = ld[j][2];
                    const float2 v0 = ld[j][3], v1 = ld[j][4], v2 = ld[j][5];
                    const float2 a12 = cmulf(u1, v2), a21 = cmulf(u2, v1);
                    const float2 a20 = cmulf(u2, v0), a02 = cmulf(u0, v2);
                    const float2 a01 = cmulf(u0, v1), a10 = cmulf(u1, v0);
                    c0 = make_float2(a12.x - a21.x, a12.y - a21.y);
                    c1 = make_float2(a20.x - a02.x, a20.y - a02.y);
                    c2 = make_float2(a01.x - a10.x, a01.y - a10.y);
                    if constexpr (F16) {
                      c0.x *= f16s; c0.y *= f16s;
                      c1.x *= f16s; c1.y *= f16s;
                      c2.x *= f16s; c2.y *= f16s;
                    }
                  } else {
                    float2 phv = ld[j][3];
                    if constexpr (F16) { phv.x *= f16s; phv.y *= f16s; }
                    c0 = cmulf(phv, ld[j][0]);
                    c1 = cmulf(phv, ld[j][1]);
                    c2 = cmulf(phv, ld[j][2]);
                  }
                  const int jj = half * LR + j;
                  vmask |= (uint32_t)vld[j] << jj;
                  re[0][jj] = c0.x; im[0][jj] = c0.y;
                  re[1][jj] = c1.x; im[1][jj] = c1.y;
                  re[2][jj] = c2.x; im[2][jj] = c2.y;
                }
              }
            };
            if (is_a) build(std::integral_constant<int, R::kAGroups>{}, std::true_type{});
            else build(std::integral_constant<int, R::kBGroups>{}, std::false_type{});
            // groups past the slab's end or of an unused row (their loads read a valid site)
            // contribute zeros; this branch is taken only at ragged edges
            if (vmask != (1u << NG) - 1u) {
#pragma unroll
              for (int jj = 0; jj < 8; ++jj)
                if (!((vmask >> jj) & 1u)) {
                  re[0][jj] = 0.f; im[0][jj] = 0.f;
                  re[1][jj] = 0.f; im[1][jj] = 0.f;
                  re[2][jj] = 0.f; im[2][jj] = 0.f;
                }
            }
          }
          // colour c occupies K bytes [32c, 32c + 32) (BF16; TF32: [32c, 32c + 32) of each
          // 8-group stage as well); group g sits in 16-byte column 2c + g / 8 at 2 (g % 8)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int seg = 2 * c + g0 / 8;
            const uint32_t in_row = TF32 ? 0u : (uint32_t)((g0 % 8) * 2);
            // A side: planes Ar, Ai. B side: Br, Bi, and -Bi beside them (plane 0).
            uint8_t* dr[LEVELS];
            uint8_t* di[LEVELS];
            uint8_t* dn[LEVELS];
#pragma unroll
            for (int l = 0; l < LEVELS; ++l) {
              const uint32_t o = row_seg(rr, seg) + in_row;
              dr[l] = smem + (is_a ? a_plane(slot, l, 0) : b_plane(slot, l, Lay::kBr)) + o;
              di[l] = smem + (is_a ? a_plane(slot, l, 1) : b_plane(slot, l, Lay::kBi)) + o;
              dn[l] = smem + b_plane(slot, l, 0) + o;
            }
            uint8_t* const* neg = (is_a || !kTwoMma) ? nullptr : dn;
            if constexpr (F16) {
              if (NG == 8) {
                split_store8_f16<8>(re[c], dr, nullptr);
                split_store8_f16<8>(im[c], di, neg);
              } else {
                split_store8_f16<4>(re[c], dr, nullptr);
                split_store8_f16<4>(im[c], di, neg);
              }
            } else if constexpr (TF32) {
              split_store8<TF32, LEVELS>(re[c], dr, nullptr);
              split_store8<TF32, LEVELS>(im[c], di, neg);
            } else {
              if (NG == 8) {
                split_store8<TF32, LEVELS>(re[c], dr, nullptr);
                split_store8<TF32, LEVELS>(im[c], di, neg);
              } else {
                split_store8<TF32, LEVELS, 4>(re[c], dr, nullptr);
                split_store8<TF32, LEVELS, 4>(im[c], di, neg);
              }
            }
          }
        }
        // every lane's core-matrix stores are made visible to the tensor core's (async)
        // proxy; once the whole warp has fenced, one lane acts for the warp
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          if (SHB && is_b && ok) {
            // this warp's third-quark row groups (16 rows of this CTA's share) of every
            // plane go to the peer, at the same offsets of its stage
            const uint32_t peer = rank ^ 1u;
            const uint32_t mbar = map_to_rank(smem_u32(&bar_full[slot]), peer);
            const int lr0 = ((pt - R::kAThreads) / 32) * 16;
#pragma unroll
            for (int gq = 0; gq < 2; ++gq) {
              if (lr0 + 8 * gq >= NC / 2) break;
              const uint32_t rg = (uint32_t)(((int)rank * (NC / 2) + lr0 + 8 * gq) >> 3);
#pragma unroll
              for (int l = 0; l < LEVELS; ++l)
#pragma unroll
                for (int pl = 0; pl < kBPlanes; ++pl) {
                  const uint32_t src = smem_base + b_plane(slot, l, pl) + rg * 768u;
                  copy_to_peer(map_to_rank(src, peer), src, 768u, mbar);
                }
            }
          }
          if (kShareA && is_a && ok) {
            // this warp's 8 diquark rows (one row group) of every plane go to every peer
            const uint32_t rg = (uint32_t)(rr >> 3);
            const uint32_t full_local = smem_u32(&bar_full[slot]);
            for (uint32_t q = 0; q < (uint32_t)C; ++q) {
              if (q == rank) continue;
              const uint32_t mbar = map_to_rank(full_local, q);
#pragma unroll
              for (int l = 0; l < LEVELS; ++l)
#pragma unroll
                for (int pl = 0; pl < 2; ++pl) {
                  const uint32_t src = smem_base + a_plane(slot, l, pl) + rg * 768u;
                  copy_to_peer(map_to_rank(src, q), src, 768u, mbar);
                }
            }
          }
          if (C > 1 && pt == 0)
            mbar_arrive_expect_tx(smem_u32(&bar_full[slot]), peer_tx);
          else
            mbar_arrive(smem_u32(&bar_full[slot]));
        }
        __syncwarp();
        if constexpr (RF) {
          // the next stage's first group: G groups on, or the next row's first
          if (++rf_sub == prm.rf_spr) {
            rf_sub = 0; ++rf_row;
            rf_xl = rf_xl0; rf_pr = rf_pr0; rf_ph = rf_ph0;
          } else {
            rf_xl += rf_gq;
            rf_pr += rf_gr;
            rf_ph += rf_step;
            if (rf_pr >= np) { rf_pr -= np; ++rf_xl; rf_ph += pidx; }
            while (rf_ph >= prm.L) rf_ph -= prm.L;
          }
        }
      }
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issue (one thread)
    if (lane == 0) {
      const uint32_t fmt = TF32 ? 2u : (F16 ? 0u : 1u);   // TF32, FP16 or BF16 operands
      // FP32 accumulate, A and B of the same type, K-major, M = 128, N = 2 NC or NC
      const uint32_t n_mma = kTwoMma ? 2 * NC : NC;
      const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) |
                             ((n_mma >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
      const uint32_t idesc_neg = idesc | (1u << 14);
      long long s_g = 0, c_g = 0;
      // the chunk's accumulator buffer (c_g mod nbuf) and the parity of its use (c_g / nbuf),
      // kept incrementally: no division on the MMA thread's path between stages
      int buf = 0;
      uint32_t buf_par = 0;
      bool stop = false;
      for (long long u = u0; u < prm.total_units && !stop; u += du) {
        const Unit w = decode(u);
        // chunks of chunk_stages stages; row-factored: no chunk crosses a lattice row
        const int spr = RF ? prm.rf_spr : w.n_stages;
        int sr = 0, cpos = 0;   // stage within the row, stage within the chunk
        for (int st = 0; st < w.n_stages; ++st, ++s_g) {
          const int slot = (int)(s_g % STAGES);
          const bool chunk_first = cpos == 0;
          const bool chunk_last = cpos == prm.chunk_stages - 1 || sr == spr - 1;
          if (++sr == spr) { sr = 0; cpos = 0; }
          else if (++cpos == prm.chunk_stages) cpos = 0;
          // the chunk's accumulator buffer must have been drained (its previous use)
          if (chunk_first && c_g >= nbuf) {
            if (!wait_bounded(smem_u32(&bar_acc_empty[buf]), buf_par ^ 1u,
                              &abort_flag, prm.status, prm.wait_limit)) { stop = true; break; }
          }
          if (!wait_bounded(smem_u32(&bar_full[slot]), (uint32_t)((s_g / STAGES) & 1),
                            &abort_flag, prm.status, prm.wait_limit)) { stop = true; break; }
          tc_fence_after();
          // [Cr | Ci] of the leading product, then of the correction products
          const uint32_t lead = tmem + (uint32_t)(buf * 4 * NC), corr = lead + 2 * NC;
          const uint32_t sa = smem_base + (uint32_t)(slot * STAGE_BYTES);
          const uint32_t sb = sa + LEVELS * 2 * kAPlaneBytes;
#pragma unroll
          for (int ks = 0; ks < 3; ++ks) {
            const uint32_t kofs = (uint32_t)(ks * 256);
            const uint32_t first = (chunk_first && ks == 0) ? 0u : 1u;
#pragma unroll
            for (int q = 0; q < NPROD; ++q) {
              const uint64_t ar = smem_desc(sa + (PI[q] * 2 + 0) * kAPlaneBytes + kofs);
              const uint64_t ai = smem_desc(sa + (PI[q] * 2 + 1) * kAPlaneBytes + kofs);
              const uint32_t bl = sb + (uint32_t)(PJ[q] * kBPlanes * Lay::kBPlaneB);
              const uint32_t d = q == 0 ? lead : corr;
              const uint32_t acc = (q <= 1) ? first : 1u;
              if constexpr (kTwoMma) {
                const uint64_t b_ri = smem_desc(bl + (uint32_t)(NC * 96) + kofs);   // [Br | Bi]
                const uint64_t b_nr = smem_desc(bl + kofs);                         // [-Bi | Br]
                mma<TF32>(d, ar, b_ri, idesc, acc);
                mma<TF32>(d, ai, b_nr, idesc, 1u);
              } else {
                const uint64_t br = smem_desc(bl + (uint32_t)(Lay::kBr * NC * 96) + kofs);
                const uint64_t bi = smem_desc(bl + (uint32_t)(Lay::kBi * NC * 96) + kofs);
                const uint32_t di = d + (uint32_t)NC;
                mma<TF32>(d, ar, br, idesc, acc);
                mma<TF32>(d, ai, bi, idesc_neg, 1u);
                mma<TF32>(di, ar, bi, idesc, acc);
                mma<TF32>(di, ai, br, idesc, 1u);
              }
            }
          }
          if (C > 1)
            tc_commit_multicast(smem_u32(&bar_empty[slot]), (uint16_t)((1u << C) - 1u));
          else
            tc_commit(smem_u32(&bar_empty[slot]));
          if (chunk_last) {
            tc_commit(smem_u32(&bar_acc_full[buf]));
            ++c_g;
            if (++buf == nbuf) { buf = 0; buf_par ^= 1u; }
          }
        }
      }
      // every MMA this thread issued must be complete before TMEM is freed, also after an
      // abort: this wait ignores the abort flag and keeps the default limit
      tc_commit(smem_u32(&bar_final));
      wait_bounded(smem_u32(&bar_final), 0u, nullptr, prm.status, kWaitCycles);
      if (C > 1 && stop) {
        // after an abort, peers may still be copying into the stages this CTA no longer
        // consumes: let those copies land (bounded) before the cluster leaves
        for (int i = 0; i < STAGES; ++i) {
          const long long k = s_g + i;
          wait_bounded(smem_u32(&bar_full[k % STAGES]), (uint32_t)((k / STAGES) & 1), nullptr,
                       prm.status, kDrainCycles);
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (TMEM lanes)
    const int row = warp * 32 + lane;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint32_t run_r = tmem + lane_base + (uint32_t)(nbuf * 4 * NC);
    long long c_g = 0;
    int buf = 0;              // c_g mod nbuf and the parity c_g / nbuf, kept incrementally
    uint32_t buf_par = 0;
    int rpar = 0;             // row-factored: parity of the rows taken so far (all units)
    for (long long u = u0; u < prm.total_units; u += du) {
      const Unit w = decode(u);
      const int spr = RF ? prm.rf_spr : w.n_stages;            // stages per chunk row
      const int cpr = (spr + prm.chunk_stages - 1) / prm.chunk_stages;
      const int n_chunks = (spr > 0 ? w.n_stages / spr : 0) * cpr;
      int crow = 0, cin = 0;  // row-factored: the chunk's row in the unit, chunk in the row
      auto next_chunk = [&] {
        if (++buf == nbuf) { buf = 0; buf_par ^= 1u; }
        if (++cin == cpr) { cin = 0; ++crow; rpar ^= 1; }
      };
      for (int ch = 0; ch < n_chunks; ++ch, ++c_g, next_chunk()) {
        bool ok = !abort_flag;
        if (ok)
          ok = wait_bounded(smem_u32(&bar_acc_full[buf]), buf_par, &abort_flag, prm.status,
                            prm.wait_limit);
        // the TMEM loads below are warp-collective: decide per warp
        ok = __all_sync(0xffffffffu, ok);
        if constexpr (RF) {
          if (cin == 0) {
            // a new lattice row: its phase w^{n1 x1 + n2 x2} per momentum, once per row, into
            // the shared-memory slot of the row's parity. Every epilogue warp takes this step
            // (whether or not it drains): a warp may still read the previous row's slot.
            const int lrow = w.x_begin + crow;
            const int x1 = lrow % prm.L, x2 = lrow / prm.L;
            if (row < prm.P)
              s_rowph[rpar][row] = s_omega[(prm.rf_pn1[row] * x1 + prm.rf_pn2[row] * x2) % prm.L];
            __syncwarp();
            named_bar(kBarEpi, kEpiWarps * 32);
          }
          // Row-factored: the chunk sums t = lead + corr of this lane's row are added into the
          // row's sums in shared memory (float4 slots [column / 4][row], so that a warp's
          // accesses are contiguous), 16 columns at a time, and the accumulator is handed back
          // to the MMA thread. The running sums of the momenta take each row once, at its
          // last chunk, while the tensor cores run the next.
          float4* const trow = s_trow + row;
          if (ok) {
            tc_fence_after();
            const uint32_t lead = tmem + lane_base;
            for (int b = 0; 16 * b < NC; ++b) {
              float a_r[16], a_i[16], c_r[16], c_i[16];
              tmem_ld16(lead + 16 * b, a_r);
              tmem_ld16(lead + NC + 16 * b, a_i);
              tmem_ld16(lead + 2 * NC + 16 * b, c_r);
              tmem_ld16(lead + 3 * NC + 16 * b, c_i);
              tmem_wait_ld();
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                float4 vr = make_float4(a_r[4 * q] + c_r[4 * q], a_r[4 * q + 1] + c_r[4 * q + 1],
                                        a_r[4 * q + 2] + c_r[4 * q + 2], a_r[4 * q + 3] + c_r[4 * q + 3]);
                float4 vi = make_float4(a_i[4 * q] + c_i[4 * q], a_i[4 * q + 1] + c_i[4 * q + 1],
                                        a_i[4 * q + 2] + c_i[4 * q + 2], a_i[4 * q + 3] + c_i[4 * q + 3]);
                float4* const pr = trow + (size_t)(4 * b + q) * kTcM;
                float4* const pi = trow + (size_t)(NC / 4 + 4 * b + q) * kTcM;
                if (cin > 0) {
                  const float4 o = *pr, oi = *pi;
                  vr = make_float4(o.x + vr.x, o.y + vr.y, o.z + vr.z, o.w + vr.w);
                  vi = make_float4(oi.x + vi.x, oi.y + vi.y, oi.z + vi.z, oi.w + vi.w);
                }
                *pr = vr;
                *pi = vi;
              }
            }
          }
          tc_fence_before();
          __syncwarp();
          named_bar(kBarEpi, kEpiWarps * 32);
          if (tid == 0) mbar_arrive(smem_u32(&bar_acc_empty[buf]));
          __syncwarp();
          if (ok) {
            if (cin == cpr - 1) {
              // the row is complete: its sums times the row's w^{n1 x1 + n2 x2}, into the
              // running sum of every momentum with that n0. Each 16-column block lies in one
              // n0 block (the d3 tile is a multiple of 16).
              const int ncol = prm.rf_nc;
              for (int b = 0; 16 * b < NC; ++b) {
                const int i0 = (16 * b) / ncol, col = 16 * b - i0 * ncol;
                float t_re[16], t_im[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const float4 vr = trow[(size_t)(4 * b + q) * kTcM];
                  const float4 vi = trow[(size_t)(NC / 4 + 4 * b + q) * kTcM];
                  t_re[4 * q] = vr.x; t_re[4 * q + 1] = vr.y; t_re[4 * q + 2] = vr.z; t_re[4 * q + 3] = vr.w;
                  t_im[4 * q] = vi.x; t_im[4 * q + 1] = vi.y; t_im[4 * q + 2] = vi.z; t_im[4 * q + 3] = vi.w;
                }
                for (uint32_t m2 = s_rfmask[i0]; m2 != 0u; m2 &= m2 - 1u) {
                  const int p = __ffs(m2) - 1;
                  const float2 ph = s_rowph[rpar][p];
                  const uint32_t rp = run_r + (uint32_t)(p * 2 * ncol + col);
                  float rr[16], ri[16];
                  if (crow > 0) {
                    tmem_ld16(rp, rr);
                    tmem_ld16(rp + ncol, ri);
                    tmem_wait_ld();
                  }
                  // two adjacent columns per packed FMA (each lane rounds as fmaf):
                  //   re = ph.x tr - ph.y ti + re,   im = ph.x ti + ph.y tr + im
                  const float2 phx = make_float2(ph.x, ph.x), phy = make_float2(ph.y, ph.y);
                  const float2 nphy = make_float2(-ph.y, -ph.y);
#pragma unroll
                  for (int i = 0; i < 16; i += 2) {
                    const float2 a = crow > 0 ? make_float2(rr[i], rr[i + 1]) : make_float2(0.f, 0.f);
                    const float2 c = crow > 0 ? make_float2(ri[i], ri[i + 1]) : make_float2(0.f, 0.f);
                    const float2 tr2 = make_float2(t_re[i], t_re[i + 1]);
                    const float2 ti2 = make_float2(t_im[i], t_im[i + 1]);
                    const float2 re = __ffma2_rn(phx, tr2, __ffma2_rn(nphy, ti2, a));
                    const float2 im = __ffma2_rn(phx, ti2, __ffma2_rn(phy, tr2, c));
                    rr[i] = re.x; rr[i + 1] = re.y;
                    ri[i] = im.x; ri[i + 1] = im.y;
                  }
                  tmem_st16(rp, rr);
                  tmem_st16(rp + ncol, ri);
                }
              }
              tmem_wait_st();
            }
          }
        } else {
          if (ok) {
            tc_fence_after();
            const uint32_t lead = tmem + lane_base + (uint32_t)(buf * 4 * NC);
            for (int col = 0; col < 2 * NC; col += 16) {
              float a[16], b[16], r[16];
              tmem_ld16(lead + col, a);
              tmem_ld16(lead + 2 * NC + col, b);
              if (ch > 0) tmem_ld16(run_r + col, r);
              tmem_wait_ld();
#pragma unroll
              for (int i = 0; i < 16; ++i) r[i] = (ch > 0 ? r[i] : 0.f) + (a[i] + b[i]);
              tmem_st16(run_r + col, r);
            }
            tmem_wait_st();
          }
          tc_fence_before();
          __syncwarp();
          named_bar(kBarEpi, kEpiWarps * 32);
          if (tid == 0) mbar_arrive(smem_u32(&bar_acc_empty[buf]));
        }
        __syncwarp();   // tcgen05.ld below is warp-aligned
        if (PROJ && ok && ch == n_chunks - 1) {
          // projection unit done: the running sum is the field's tile q[m][n]
          const ProjFieldF& F = prm.pfields[w.job];
          const int m = w.mt * kTcM + row, nd = F.nd;
          for (int col = 0; col < NC; col += 16) {
            float vr[16], vi[16];
            __syncwarp();
            tmem_ld16(run_r + col, vr);
            tmem_ld16(run_r + NC + col, vi);
            tmem_wait_ld();
            if (m < prm.p_rows) {
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const int n = w.nt * NC + col + i;
                if (n < nd) F.q[(size_t)m * nd + n] = make_float2(vr[i], vi[i]);
              }
            }
          }
        } else if (RF && ok && ch == n_chunks - 1) {
          // unit done (row-factored): every momentum's running sum is its partial block
          const TcJob& J = prm.jobs[w.job];
          const int m = w.mt * kTcM + row;
          const int M = J.nd1 * J.nd2, nd3 = J.nd3, ncol = prm.rf_nc;
          for (int p = 0; p < prm.P; ++p)
            for (int col = 0; col < ncol; col += 16) {
              float vr[16], vi[16];
              __syncwarp();
              const uint32_t rp = run_r + (uint32_t)(p * 2 * ncol + col);
              tmem_ld16(rp, vr);
              tmem_ld16(rp + ncol, vi);
              tmem_wait_ld();
              if (m < M) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  const int d3 = (kShareA ? w.nt * C + (int)rank : w.nt) * ncol + col + i;
                  if (d3 < nd3)
                    J.partial[(((size_t)w.slab * prm.P + p) * M + m) * nd3 + d3] =
                        make_float2(vr[i], vi[i]);
                }
              }
            }
        } else if (!PROJ && ok && ch == n_chunks - 1) {
          // unit done: write the FP32 running sum as this slab's partial block
          const TcJob& J = prm.jobs[w.job];
          const int m = (SHB ? w.mt * 2 + (int)rank : w.mt) * kTcM + row;
          const int M = J.nd1 * J.nd2, nd3 = J.nd3, Ntot = prm.P * nd3;
          for (int col = 0; col < NC; col += 16) {
            float vr[16], vi[16];
            __syncwarp();   // the stores below may diverge; tcgen05.ld is warp-aligned
            tmem_ld16(run_r + col, vr);
            tmem_ld16(run_r + NC + col, vi);
            tmem_wait_ld();
            if (m < M) {
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const int n = (kShareA ? w.nt * C + (int)rank : w.nt) * NC + col + i;
                if (n < Ntot) {
                  const int p = n / nd3, d3 = n - p * nd3;
                  const size_t pi = (((size_t)w.slab * prm.P + p) * M + m) * nd3 + d3;
                  if (!CHECKS || idx_ok(prm, (long long)pi, (long long)prm.n_slab * prm.P * M * nd3, 5, w.job))
                    J.partial[pi] = make_float2(vr[i], vi[i]);
                }
              }
            }
          }
        }
      }
    }
  }

  // ------------------------------------------------------------ teardown
  tc_fence_before();
  __syncwarp();
  __syncthreads();
  // no CTA leaves while a peer may still address its shared memory
  if (C > 1) cluster_sync_all();
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 ::"r"(tmem), "r"(kTmemCols));
  }
}

template <bool TF32, int LEVELS, int NPROD, bool CHECKS, int C, bool F16>
__global__ void __launch_bounds__(Roles<TF32, C>::kThreads, 1)
k_contract_tc(const __grid_constant__ TcParams prm) {
  tc_body<TF32, LEVELS, NPROD, CHECKS, C, false, F16>(prm);
}
// The FP16 form with the row-factored momentum phase.
__global__ void __launch_bounds__(Roles<false, 1>::kThreads, 1)
k_contract_tc_rows(const __grid_constant__ TcParams prm) {
  tc_body<false, 2, 3, false, 1, false, true, false, true>(prm);
}

// The row-factored FP16 contraction as clusters of 2 that share each diquark tile and take
// adjacent d3 tiles.
__global__ void __launch_bounds__(Roles<false, 2>::kThreads, 1)
k_contract_tc_rows2(const __grid_constant__ TcParams prm) {
  tc_body<false, 2, 3, false, 2, false, true, false, true>(prm);
}

// The FP16 form as CTA pairs that share the third-quark tile (clusters of 2).
__global__ void __launch_bounds__(Roles<false, 1>::kThreads, 1)
k_contract_tc_pair(const __grid_constant__ TcParams prm) {
  tc_body<false, 2, 3, false, 2, false, true, true>(prm);
}

template <bool TF32, int LEVELS, int NPROD>
__global__ void __launch_bounds__(Roles<TF32, 1>::kThreads, 1)
k_project_tc(const __grid_constant__ TcParams prm) {
  tc_body<TF32, LEVELS, NPROD, false, 1, true>(prm);
}

template <bool TF32, int LEVELS, int NPROD, bool CHECKS, int C, bool F16 = false>
cudaError_t launch_variant(const TcParams& prm, int grid, cudaStream_t s) {
  using Lay = TcLayout<TF32, LEVELS, F16>;
  const size_t smem = (size_t)Lay::kStages * Lay::kStageBytes;
  auto kern = k_contract_tc<TF32, LEVELS, NPROD, CHECKS, C, F16>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (C == 1) {
    kern<<<grid, Roles<TF32, C>::kThreads, smem, s>>>(prm);
    note_launch();
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(Roles<TF32, C>::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // as many clusters as can be resident at once (a cluster needs C SMs of one GPC)
  cfg.gridDim = dim3((unsigned)grid);
  int max_clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (max_clusters < 1) return cudaErrorInvalidConfiguration;
  const long long want = (grid + C - 1) / C;
  cfg.gridDim = dim3((unsigned)(C * (want < max_clusters ? want : max_clusters)));
  e = cudaLaunchKernelEx(&cfg, kern, prm);
  note_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <bool TF32, int LEVELS, int NPROD>
cudaError_t launch_projection(const TcParams& prm, int grid, cudaStream_t s) {
  using Lay = TcLayout<TF32, LEVELS>;
  const size_t smem = (size_t)Lay::kStages * Lay::kStageBytes;
  auto kern = k_project_tc<TF32, LEVELS, NPROD>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, Roles<TF32, 1>::kThreads, smem, s>>>(prm);
  note_launch();
  return cudaGetLastError();
}

// The FP16 form as CTA pairs: grid = CTAs wanted (even), capped at the pairs that can be
// resident at once.
cudaError_t launch_pair(const TcParams& prm, int grid, cudaStream_t s) {
  using Lay = TcLayout<false, 2, true, true>;
  const size_t smem = (size_t)Lay::kStages * Lay::kStageBytes;
  auto kern = k_contract_tc_pair;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(Roles<false, 1>::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((unsigned)grid);
  int max_clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (max_clusters < 1) return cudaErrorInvalidConfiguration;
  const long long want = (grid + 1) / 2;
  cfg.gridDim = dim3((unsigned)(2 * (want < max_clusters ? want : max_clusters)));
  e = cudaLaunchKernelEx(&cfg, kern, prm);
  note_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// The row-factored FP16 contraction: one CTA per SM; the stages, the w^k table, then the
// epilogue's row sums (128 rows x 2 NC floats).
cudaError_t launch_rows(const TcParams& prm, int cluster, int grid, cudaStream_t s) {
  using Lay = TcLayout<false, 2, true, false, true>;
  const size_t smem = (size_t)Lay::kStages * Lay::kStageBytes + kMaxRfL * sizeof(float2) +
                      (size_t)kTcM * 2 * kMaxNC * sizeof(float);
  auto kern = cluster == 2 ? k_contract_tc_rows2 : k_contract_tc_rows;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cluster == 1) {
    kern<<<grid, Roles<false, 1>::kThreads, smem, s>>>(prm);
    note_launch();
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(Roles<false, 2>::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((unsigned)grid);
  int max_clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (max_clusters < 1) return cudaErrorInvalidConfiguration;
  const long long want = (grid + 1) / 2;
  cfg.gridDim = dim3((unsigned)(2 * (want < max_clusters ? want : max_clusters)));
  e = cudaLaunchKernelEx(&cfg, kern, prm);
  note_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// The FP16 form: two pieces, three products; plain CTAs (with or without index checks), or
// CTA pairs sharing the third-quark tile (cluster = 2, unchecked), or the row-factored
// phase (unchecked).
cudaError_t launch_form_f16(const TcParams& prm, int cluster, int grid, cudaStream_t s) {
  if (prm.rf) {
    if (prm.checks || (cluster != 1 && cluster != 2) || prm.share_b || prm.L < 1 || prm.L > kMaxRfL ||
        prm.rf_nidx < 1 || prm.rf_nidx > kMaxRfIdx || prm.P > kMaxRfP || prm.rf_spr < 1 ||
        prm.rf_nc < 16 || prm.rf_nc % 16 != 0 || prm.NC != prm.rf_nidx * prm.rf_nc ||
        4 * prm.NC + 2 * prm.P * prm.rf_nc > kTmemCols || !prm.rf_omega)
      return cudaErrorInvalidValue;
    return launch_rows(prm, cluster, grid, s);
  }
  if (cluster == 2 && prm.share_b) {
    if (prm.checks) return cudaErrorInvalidValue;
    return launch_pair(prm, grid, s);
  }
  if (cluster != 1 || prm.share_b || prm.NC > kMaxNC) return cudaErrorInvalidValue;
  if (prm.checks) return launch_variant<false, 2, 3, true, 1, true>(prm, grid, s);
  return launch_variant<false, 2, 3, false, 1, true>(prm, grid, s);
}

template <bool TF32, int LEVELS, int NPROD>
cudaError_t launch_form(const TcParams& prm, int cluster, int grid, cudaStream_t s) {
  if (prm.checks) {
    if (cluster != 1) return cudaErrorInvalidValue;
    return launch_variant<TF32, LEVELS, NPROD, true, 1>(prm, grid, s);
  }
  if (TF32 && cluster != 1) return cudaErrorInvalidValue;
  switch (cluster) {
    case 1: return launch_variant<TF32, LEVELS, NPROD, false, 1>(prm, grid, s);
    case 2: return launch_variant<TF32, LEVELS, NPROD, false, TF32 ? 1 : 2>(prm, grid, s);
    case 4: return launch_variant<TF32, LEVELS, NPROD, false, TF32 ? 1 : 4>(prm, grid, s);
    case 8: return launch_variant<TF32, LEVELS, NPROD, false, TF32 ? 1 : 8>(prm, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

__global__ void k_reduce_slabs_f32(const TcJob* __restrict__ jobs, int n_slab, int P_total,
                                   int checks, unsigned long long* dbg, int* status) {
  const TcJob& J = jobs[blockIdx.y];
  const long long per = (long long)P_total * J.nd1 * J.nd2 * J.nd3;
  // FP16 form: the partials carry the operands' power-of-two scales 2^(eA + eB)
  double unscale = 1.0;
  if (J.amax) {
    int eA, eB;
    f16_scale_exps(J.amax, eA, eB);
    unscale = __longlong_as_double((long long)(1023 - eA - eB) << 52);   // 2^-(eA + eB)
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per;
       e += (long long)gridDim.x * blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int sl = 0; sl < n_slab; ++sl) {   // fixed order: run-to-run identical
      const float2 v = J.partial[(size_t)sl * per + e];
      sr += (double)v.x;
      si += (double)v.y;
    }
    J.B[e] = make_double2(sr * unscale, si * unscale);
  }
  (void)checks; (void)dbg; (void)status;  // every index above is below n_slab * per or per
}

}  // namespace

int tc_groups_per_stage(int form) { return form == TC_TF32_3 ? 8 : 16; }
int tc_max_nc(int form, bool share_b) { return form == TC_F16_3 && share_b ? kMaxNCWide : kMaxNC; }
bool tc_form_needs_amax(int form) { return form == TC_F16_3; }

cudaError_t launch_contract_tc(const TcParams& prm, int form, int cluster, int grid,
                               cudaStream_t s) {
  if (prm.total_units == 0) return cudaSuccess;
  const int max_nc = (form == TC_F16_3 && prm.share_b) ? kMaxNCWide : kMaxNC;
  if (prm.NC < 16 || prm.NC > max_nc || prm.NC % 16 != 0 || prm.chunk_stages < 1)
    return cudaErrorInvalidValue;
  if ((prm.share_b || prm.rf) && form != TC_F16_3) return cudaErrorInvalidValue;
  switch (form) {
    case TC_BF16_3: return launch_form<false, 2, 3>(prm, cluster, grid, s);
    case TC_BF16_6: return launch_form<false, 3, 6>(prm, cluster, grid, s);
    case TC_BF16_9: return launch_form<false, 3, 9>(prm, cluster, grid, s);
    case TC_TF32_3: return launch_form<true, 2, 3>(prm, cluster, grid, s);
    case TC_F16_3: return launch_form_f16(prm, cluster, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_project_tc(const TcParams& prm, int form, int grid, cudaStream_t s) {
  if (prm.total_units == 0) return cudaSuccess;
  if (prm.NC < 16 || prm.NC > kMaxNC || prm.NC % 16 != 0 || prm.chunk_stages < 1 ||
      prm.checks || !prm.pfields || prm.p_n_fields < 1 || prm.p_rows < 1 || prm.p_n_ev < 1 ||
      prm.p_m_tiles < 1 || prm.p_n_tiles < 1 ||
      prm.total_units != (long long)prm.p_m_tiles * prm.p_n_fields * prm.p_n_tiles)
    return cudaErrorInvalidValue;
  switch (form) {
    case TC_BF16_3: return launch_projection<false, 2, 3>(prm, grid, s);
    case TC_BF16_6: return launch_projection<false, 3, 6>(prm, grid, s);
    case TC_BF16_9: return launch_projection<false, 3, 9>(prm, grid, s);
    case TC_TF32_3: return launch_projection<true, 2, 3>(prm, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_reduce_slabs_f32(const TcJob* d_jobs, int n_jobs, int n_slab, int P_total,
                                    long long max_elems, int checks, unsigned long long* dbg,
                                    int* status, cudaStream_t s) {
  if (n_jobs == 0 || max_elems == 0) return cudaSuccess;
  long long bx = (max_elems + kThreads - 1) / kThreads;
  if (bx > 4096) bx = 4096;
  dim3 grid((unsigned)bx, n_jobs);
  k_reduce_slabs_f32<<<grid, kThreads, 0, s>>>(d_jobs, n_slab, P_total, checks, dbg, status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bb
