// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace bb {

constexpr int kMaxTerms = 4;    // distinct gamma spins folded into one line-3 field
constexpr int kMaxPairs = 16;   // distinct (alpha, beta) spin pairs
// Row-factored tensor-core contraction: momenta per launch and distinct n0 values.
constexpr int kMaxRfP = 16;
constexpr int kMaxRfIdx = 8;
constexpr int kMaxRfL = 128;    // lattice extent (the w^k table follows the stage buffers)
// Momenta handled by one contraction launch of the FP64 form (10) and of the double-float
// form (8): the largest counts whose accumulators fit the registers without spills.
constexpr int kMaxPGroup = 10;
constexpr int kMaxPGroupDf = 8;
// Momenta of the first launch: n_mom split into the fewest groups of at most max_group, as
// evenly as possible (each launch recomputes the colour singlet that its momenta share).
inline int p_group_size(int n_mom, int max_group) {
  const int groups = (n_mom + max_group - 1) / max_group;
  return groups > 0 ? (n_mom + groups - 1) / groups : 0;
}
constexpr int kThreads = 256;   // threads per CTA of the FP64 kernels

// Kernel launches made by the calling host thread, counted at every launch site of the
// library (a call's launch count is the difference across it).
inline thread_local long long t_kernel_launches = 0;
inline void note_launch() { ++t_kernel_launches; }

// Device-side status bits (OR-ed into the context's status word).
constexpr int kStatusBadJob = 1;
constexpr int kStatusTimeout = 2;   // a bounded wait of the tensor-core kernel gave up
constexpr int kStatusBadIndex = 4;  // a checked kernel found an index outside its buffer
constexpr int kStatusCanary = 8;    // a workspace canary was overwritten (checks option)
constexpr int kCanaryBytes = 256;   // canary after every workspace block (checks option)

// One reconstructed field of Eq. (2):
//   q[r][d] = sum_l V[l][r] * Phi[l][d],   Phi[l][d] = sum_t w[t] * phi[row_off[t] + l][d],
// r = 3x + a running over the 3X (site, colour) rows. Lines 1 and 2 use one term
// (row_off = alpha * n_ev, w = 1); line 3 folds the spin coefficients of every
// triple that shares an (alpha, beta) pair into one field (Eq. 1 is linear in q3).
struct ProjField {
  const double2* V;     // [n_ev][3X]
  const double2* phi;   // [4 n_ev][nd]
  double2* q;           // [3X][nd]
  int nd;
  int n_terms;
  int row_off[kMaxTerms];
  double2 w[kMaxTerms];
};

// Same field for the tensor-core forms: V and phi are the FP32 copies made by
// launch_convert_f32 (complex64), q is written in FP32.
struct ProjFieldF {
  const float2* V;
  const float2* phi;
  float2* q;
  // if set: the largest |Re| or |Im| written to q is max-ed into *amax (FP32 bits, zeroed
  // before the projection); the FP16 form scales its operands from it
  uint32_t* amax;
  int nd;
  int n_terms;
  int row_off[kMaxTerms];
  double2 w[kMaxTerms];
};

// One job = one time slice of one noise triple.
struct ContractJob {
  const double2* q1[4];          // line-1 fields, one per distinct alpha (slot order)
  const double2* q2[4];          // line-2 fields, one per distinct beta
  const double2* q3[kMaxPairs];  // folded line-3 field per (alpha, beta) pair
  double2* partial;              // [n_slab][P_total][nd1*nd2][nd3]
  double2* B;                    // [P_total][nd1][nd2][nd3]
  // Ozaki form: per site slab, the column maxima of the job's line-1 and line-2 fields
  // (|Re| + |Im|) and line-3 fields (modulus) of the high parts, [n_slab][nd1 + nd2 + nd3],
  // then the diquark's row maxima, [n_slab][nd1 nd2]; null in the other forms
  float* oz_max;
  int nd1, nd2, nd3;
  int m_tiles, n_tiles;
  long long unit_begin;          // first global work-unit index of this job
};

struct ContractParams {
  const ContractJob* jobs;
  int n_jobs;
  long long total_units;
  int X;                         // sites per time slice
  int n_slab;
  int sites_per_slab;
  int n_pairs;
  int a_slot[kMaxPairs];         // pair -> line-1 slot
  int b_slot[kMaxPairs];         // pair -> line-2 slot
  const double2* phase;          // [P_total][X]
  int p0;                        // first momentum of this launch
  int P_total;
  int* status;
  // Ozaki form: the phases as double-float float4 (re.h, re.l, im.h, im.l), [P_total][X];
  // P momenta per launch (columns n = p * nd3 + d3, p < P), NC complex columns per N tile,
  // and the limit of every bounded wait in SM cycles
  const float4* phase_df;
  int P;
  int NC;
  long long wait_limit;
};

// Tiles of the FP64 contraction for a momentum count (per launch).
struct Fp64Tile { int rm, rn; };
inline Fp64Tile fp64_tile_for(int P) { return P <= 4 ? Fp64Tile{2, 2} : Fp64Tile{2, 1}; }
inline int fp64_sites_per_chunk(int n_pairs) { return n_pairs >= 16 ? 1 : 16 / n_pairs; }
size_t fp64_contract_smem_bytes(int P, int rn, int n_pairs);

// ---------------------------------------------------------------- tensor-core forms

// One job of the tensor-core contraction: FP32 fields [(x,a)][d] and FP32 per-slab partials.
struct TcJob {
  const float2* q1[4];
  const float2* q2[4];
  const float2* q3[kMaxPairs];
  // FP16 form: largest |Re| or |Im| of the job's line-1, line-2 and line-3 fields (FP32
  // bits, written by the projection); null in the other forms
  const uint32_t* amax;
  float2* partial;               // [n_slab][P][nd1*nd2][nd3]
  double2* B;                    // [P][nd1][nd2][nd3]
  int nd1, nd2, nd3;
  int m_tiles, n_tiles;
  long long unit_begin;
};

struct TcParams {
  const TcJob* jobs;
  int n_jobs;
  long long total_units;
  int X;
  int n_slab;
  int sites_per_slab;
  int n_pairs;
  int a_slot[kMaxPairs];
  int b_slot[kMaxPairs];
  const float2* phase;           // [P][X], the FP64 phases rounded to FP32
  int P;                         // momenta (columns n = p*nd3 + d3)
  int NC;                        // complex columns per tile: 16, 32 or 48 (up to 80 in pairs)
  int chunk_stages;              // stages accumulated in TMEM between drains
  // CTA pairs (FP16 form, cluster = 2): the two CTAs of a cluster share the third-quark tile
  // of one N tile and take adjacent M tiles; a job's m_tiles then counts pairs of M tiles
  int share_b;
  // Row-factored phase (FP16 form): e^{-i p.x} = w^{n0 x0} w^{n1 x1 + n2 x2}, w = e^{-2 pi i/L}.
  // The MMA sums one lattice row (x1, x2 fixed, x0 = 0..L-1) against the third quark times
  // w^{n0 x0} for each distinct n0 of the momenta (B rows (idx0, d3), NC = rf_nidx * rf_nc);
  // the epilogue multiplies each row's sums by w^{n1 x1 + n2 x2} into one FP32 running sum
  // per momentum. A unit's slab is a range of rows [x_begin, x_end) of the L^2 rows; a row
  // takes rf_spr stages of groups (x0, pair), the last one padded.
  int rf;                        // 1: the row-factored FP16 contraction (launch_contract_tc)
  int L;
  int rf_spr;
  int rf_rows_per_slab;
  int rf_nc;                     // d3 columns per N tile
  int rf_nidx;                   // distinct n0 (mod L) of the momenta
  int rf_n0[kMaxRfIdx];          // those n0, reduced to [0, L)
  int rf_pidx0[kMaxRfP];         // momentum p: index of its n0
  int rf_pn1[kMaxRfP], rf_pn2[kMaxRfP];   // momentum p: n1, n2 reduced to [0, L)
  const float2* rf_omega;        // w^k, k = 0..L-1, FP64 rounded to FP32
  int* status;
  // index checks (debug option): every global access is checked against its buffer; the
  // first violation is recorded in dbg[0..3] = (site code, job, index, bound) and skipped
  int checks;
  unsigned long long* dbg;
  // limit of every bounded wait, in SM cycles (about 2 s by default; a test hook shortens it)
  long long wait_limit;
  // projection mode (launch_project_tc): fields of Eq. 2 and their tiling; units are
  // (128-row tile, field, N tile of NC columns), p_m_tiles x fields x p_n_tiles in all
  const ProjFieldF* pfields;
  int p_n_fields;
  int p_rows;                    // 3 L^3 rows (site, colour) of V
  int p_n_ev;                    // eigenvectors: the K extent
  int p_m_tiles, p_n_tiles;
};

enum TcForm { TC_BF16_3 = 0, TC_BF16_6 = 1, TC_BF16_9 = 2, TC_TF32_3 = 3, TC_F16_3 = 4 };

// One input array of a call converted to FP32: n complex128 elements from src to dst.
struct F32ConvSeg {
  const double2* src;
  float2* dst;
  long long n;
};
cudaError_t launch_convert_f32(const F32ConvSeg* d_segs, int n_segs, long long max_n,
                               cudaStream_t s);
cudaError_t launch_project_f32(const ProjFieldF* d_fields, int n_fields, int rows, int n_ev,
                               int max_nd, int checks, unsigned long long* dbg, int* status,
                               cudaStream_t s);
// cluster: 1 (plain kernel) or 2, 4, 8 CTAs sharing each diquark tile (BF16 forms, no
// index checks); grid: CTAs wanted, capped at the clusters that fit at once
cudaError_t launch_contract_tc(const TcParams& p, int form, int cluster, int grid, cudaStream_t s);
// Eq. 2 for the mixed forms on the tensor cores: every field of p.pfields, in the form's
// operand split, accumulated as in the contraction; writes each field's FP32 q.
cudaError_t launch_project_tc(const TcParams& p, int form, int grid, cudaStream_t s);
int tc_groups_per_stage(int form);
// true for the forms that scale their operands from the fields' maxima (TcJob::amax)
bool tc_form_needs_amax(int form);
// widest N tile (complex columns) of a form, plain CTAs or CTA pairs sharing the B tile
int tc_max_nc(int form, bool share_b);
cudaError_t launch_reduce_slabs_f32(const TcJob* d_jobs, int n_jobs, int n_slab, int P_total,
                                    long long max_elems, int checks, unsigned long long* dbg,
                                    int* status, cudaStream_t s);

// ---------------------------------------------------------------- mode-triplet ordering

// Line-3 coefficients of one (alpha, beta) pair: phi3' = sum_t w[t] phi3[row[t] N_ev + l][d].
struct FoldTerms {
  int n;
  int row[kMaxTerms];
  double2 w[kMaxTerms];
};

// Batched complex GEMM, FP64: for b < batch,
//   C_b[m][n] = alpha * sum_k A_b[m][k] B_b[k][n]  (+ C_b[m][n] if accumulate),
// element (m, k) of A_b at A + b * a_b + m * a_m + k * a_k (strides in elements), likewise B, C.
struct ZgemmParams {
  int M, N, K;
  long long batch;
  const double2* A;
  long long a_m, a_k, a_b;
  const double2* B;
  long long b_k, b_n, b_b;
  double2* C;
  long long c_m, c_n, c_b;
  double2 alpha;
  int accumulate;
};

cudaError_t launch_fill_identity(double2* id, int n_ev, cudaStream_t s);
cudaError_t launch_fold_phi(const double2* phi, int n_ev, int nd, const FoldTerms& terms,
                            double2* out, cudaStream_t s);
cudaError_t launch_zgemm(const ZgemmParams& p, cudaStream_t s);

// Fill (check == false) or verify (check == true) the n canaries listed at d_list.
cudaError_t launch_canaries(uint32_t* const* d_list, int n, bool check, int* status,
                            cudaStream_t s);

// ph: FP64 phases [n_mom][X]; ph_f (optional): the same rounded to FP32
cudaError_t launch_phase_table(int L, int n_mom, const int* d_mom, double2* ph, float2* ph_f,
                               cudaStream_t s);
cudaError_t launch_project_fp64(const ProjField* d_fields, int n_fields, int rows, int n_ev,
                                int max_nd, cudaStream_t s);
cudaError_t launch_contract_fp64(const ContractParams& p, int P, int rn, int grid, cudaStream_t s);
// Double-float form: same units, tiles, shared memory and partial layout as the FP64
// contraction; fields hold double-float pairs (float4 per complex element).
cudaError_t launch_contract_df(const ContractParams& p, int P, int rn, int grid, cudaStream_t s);

// One input array of a call converted to double-float planes: n complex128 elements
// from src to float4 (re.h, re.l, im.h, im.l) at dst.
struct DfConvSeg {
  const double2* src;
  float4* dst;
  long long n;
};
cudaError_t launch_convert_df(const DfConvSeg* d_segs, int n_segs, long long max_n,
                              cudaStream_t s);
// Eq. (2) in double-float arithmetic: the fields' V and phi point to converted float4
// planes (cast to const double2*), q receives float4 double-float elements.
cudaError_t launch_project_df(const ProjField* d_fields, int n_fields, int rows, int n_ev,
                              int max_nd, cudaStream_t s);
int fp64_contract_ctas_per_sm(int P, int rn, int n_pairs);

// ---------------------------------------------------------------- tiled tensor-core projection

// Eq. 2 for the mixed forms with pre-tiled BF16 piece operands (proj_tiled.cu).
constexpr int kTiledMaxNC = 48;   // widest N tile (complex columns)
struct TileV {                    // one distinct V of a wave
  const double2* V;               // [n_ev][rows] FP64 (the caller's buffer)
  uint16_t* tiles;                // [m_tiles][k_stages] 48 KB blocks of A pieces
};
struct TiledField {               // one field q of Eq. 2
  const double2* phi;             // [4 n_ev][nd] FP64 (the caller's buffer)
  double2 w[kMaxTerms];           // folded coefficients, rows row_off[t] + l
  int row_off[kMaxTerms];
  int n_terms;
  int nd, ncp, n_tiles;           // columns, N tile width (16..64), N tiles
  uint16_t* btiles;               // [n_tiles][k_stages] blocks of B pieces (9 ncp 64 bytes)
  float2* q;                      // [rows][nd] FP32 output
  uint32_t* amax;                 // FP16 form: the quark line's largest |Re| or |Im| (or null)
};
struct FieldTile { int field, nt; };
struct PGroup {                   // the field tiles of one V: units (128-row tile, field tile)
  long long unit_begin;
  int ft_first, ft_count, vidx;
};
struct TiledProjParams {
  const TileV* vs;
  const TiledField* fields;
  const FieldTile* fts;
  const PGroup* groups;
  int n_groups;
  long long total_units;
  int rows, n_ev, k_stages, m_tiles;
  int* status;
  long long wait_limit;
};
cudaError_t launch_project_tiled(const TiledProjParams& p, int n_vs, int n_fts, int grid,
                                 cudaStream_t s);
size_t tiled_v_bytes(int rows, int n_ev);
size_t tiled_phi_bytes(int nd, int ncp, int n_ev);
// the N tile (16, 32 or 48 columns) with the fewest padded columns, the wider on a tie
inline int tiled_ncp(int nd) {
  int best = 48, pad = 1 << 30;
  for (int nc = 48; nc >= 16; nc -= 16) {
    const int p = (nd + nc - 1) / nc * nc - nd;
    if (p < pad) { pad = p; best = nc; }
  }
  return best;
}

// ---------------------------------------------------------------- Ozaki form

// FP64-accurate contraction on the BF16 tensor cores (oz_contract.cu): units (job, 128-row
// M tile, NC-column N tile over the launch's P * nd3 columns, site slab); fields are
// double-float float4 planes, partial blocks are written in FP64 like the FP64 form's.
constexpr int kOzMaxNC = 48;
constexpr int kOzM = 128;
// cluster: 1 (plain CTAs) or 2, 3, 4 CTAs sharing each diquark tile; grid: units (clusters)
// wanted at once, capped at the clusters that can be resident
cudaError_t launch_contract_oz(const ContractParams& p, int cluster, int grid, cudaStream_t s);
// One field's contribution to a job's column maxima: max over the slab's rows (x, c) of
// |Re| + |Im| (high parts) of column d, max-ed into out[slab * stride + col_off + d]
// (zeroed before).
struct OzMaxSeg {
  const float4* field;           // [3X][nd] double-float
  float* out;
  int nd;
  int col_off;
  int stride;
  int modulus;                   // 1: the modulus, 0: |Re| + |Im|
};
cudaError_t launch_oz_colmax(const OzMaxSeg* d_segs, int n_segs, int X, int sites_per_slab,
                             cudaStream_t s);
// The diquark's row maxima (see ContractJob::oz_max) of every job of p.jobs; max_m_tiles:
// the largest job's 128-row tiles
cudaError_t launch_oz_rowmax(const ContractParams& p, int max_m_tiles, cudaStream_t s);
// FP64 phases to double-float float4, n elements
cudaError_t launch_phase_df(const double2* ph, float4* out, long long n, cudaStream_t s);
cudaError_t launch_reduce_slabs(const ContractJob* d_jobs, int n_jobs, int n_slab, int P_total,
                                long long max_elems, cudaStream_t s);

}  // namespace bb
