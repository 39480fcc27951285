// tdc_common.cuh -- device-side plan structures and helpers shared by the
// CUDA translation units of libtdc (never by the CPU oracle).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/tdc.h"

namespace tdc {

// ---------------------------------------------------------------------------
// Plan.  Problems are sorted by tree depth, deepest first, so that the
// problems taking part in merge level l (depth > l) form a prefix.  The tree
// of a problem of order n and depth t has node boundaries floor(i n / 2^l) on
// level l; node i of level l splits at floor((2i+1) n / 2^(l+1)).
// ---------------------------------------------------------------------------
struct Problem {
  int64_t n;       // order
  int64_t off_de;  // caller's offset of d, e and lam
  int64_t off_q;   // caller's offset of Q (buffer 0)
  int64_t ld0;     // leading dimension in buffer 0
  int64_t voff;    // offset in the internal vectors (prefix of n)
  int64_t qoff1;   // offset in the internal Q buffer (prefix of n^2)
  int64_t leaf0;   // first global leaf index of the problem
  int32_t depth;   // tree depth t
  int32_t escale;  // input scale: d, e enter as x 2^-escale, eigenvalues leave times 2^escale (0: none)
};

struct Vecs {  // per-slot vectors of length N (sum of n); a merge owns [voff+lo, voff+hi)
  double* dmod;    // corner-modified diagonal
  double* lam;     // eigenvalues of the current nodes
  double* Dc;      // poles by merge column (rotated)
  double* zc;      // z by merge column (rotated)
  double* Ds;      // poles in ascending order
  double* zs;      // z in ascending pole order
  double* Dk;      // non-deflated poles (ascending), K of them
  double* zk;      // non-deflated z
  double* tau;     // root offsets
  double* zhat;    // Loewner zhat
  double* scol;    // column normalisers
  float2* xz;      // FP32 pole coordinate d_i - d_centre (high part) and z_i^2 (secular pre-iteration)
  float* xlo;      // low part of that coordinate (xz.x + xlo = d_i - d_centre to about 2^-48)
  double* zz;      // z_i^2 of the non-deflated poles
  double* bf;      // first row of each node's eigenvector matrix (by output column)
  double* bl;      // last row of it
  double* rbf;     // first row of the children's block matrix after the deflating rotations
  double* rbl;     // last row of it
  double* pf;      // rbf at the column of non-deflated pole i where it has top support, else 0
  double* pl;      // rbl at that column where it has bottom support, else 0
  double* rf;      // the node's first row at root j's column (by root index, before ordering)
  double* rl;      // its last row there
  double* dval;    // deflated eigenvalues (scan order)
  double* rcs;     // rotations: (c, s) pairs, 2 per slot
  double* skey;    // sort scratch keys, 2 slots per vector slot
  int32_t* stag;   // sort scratch tags, 2 slots per vector slot
  int32_t* perm;   // merge columns in ascending pole order
  int32_t* kept;   // merge column of non-deflated pole j
  int32_t* org;    // origin pole index of root j (j or j+1)
  int32_t* dcol;   // merge column of deflated entry q
  int32_t* tlist;  // non-deflated indices with support in the top half
  int32_t* blist;  // ... in the bottom half
  int32_t* posr;   // output column of root j
  int32_t* posd;   // output column of deflated entry q
  int32_t* rij;    // rotations: (pj, i, supports) triples, 4 ints per slot
  int32_t* rch;    // first rotation of each independent rotation chain
  uint8_t* kseg;   // support bits of non-deflated pole j (1 top, 2 bottom)
  uint8_t* dseg;   // support bits of deflated entry q
  uint8_t* cseg;   // support bits scratch by merge column
};

struct MergeInfo {  // per merge of the current level
  int32_t* K;       // non-deflated count
  int32_t* nd;      // deflated count
  int32_t* nrot;    // rotations
  int32_t* ntop;    // |S_top|
  int32_t* nbot;    // |S_bot|
  int32_t* nchain;  // independent rotation chains
  int64_t* tiles;   // GEMM tile prefix (M + 1 entries)
  int64_t* roff;    // prefix of the roots of small merges (thread-per-root kernels), M + 1 entries,
                    // then the count of roots handed to the warp-per-root fix-up
  int64_t* boff;    // prefix of the 8-root blocks of the other merges (warp per root), M + 1 entries
  int64_t* ioff;    // split path, levels cut into passes: prefix of the merges' digit-image elements
  int64_t* spass;   // split path: pass count, then the merge range [g0, g1) of each pass
  int64_t* sseg;    // split path: segments of the pass being processed
};

struct Stats {  // device-side per-call statistics (index 0 = top level)
  unsigned long long sum_n[TDC_MAX_LEVELS];
  unsigned long long sum_K[TDC_MAX_LEVELS];
  unsigned long long n_rot[TDC_MAX_LEVELS];
  unsigned long long n_type1[TDC_MAX_LEVELS];
  unsigned long long n_merges[TDC_MAX_LEVELS];
  int max_K[TDC_MAX_LEVELS];
  unsigned long long gemm_flops[TDC_MAX_LEVELS];
  unsigned long long split_flops;
  unsigned long long split_bytes;
  unsigned long long struct_flops;
  unsigned long long iter_sum;
  unsigned long long iter_roots;
  int iter_max;
  unsigned long long handoffs;
  unsigned int split_level_max;  // FP32 bits of the largest |level sum| of a split hand-off (levels 0-4)
  unsigned long long srrsc[4];   // far tiles, sum of ranks, dense fallbacks, largest rank
  unsigned long long ss_parts[2];  // structured split path: merge parts taken, parts left to the split path
};

// One GEMM segment C(rows x K) = A(rows x kk) * Qhat(list, :) of the merge
// update: list position q names pole p = plist[q] (identity when NULL), whose
// column of A is acol[p] (identity when NULL); Qhat_pj = zhat_p scol_j /
// ((D_p - D_org(j)) - tau_j); output column of root j is cpos[j] (identity when
// NULL).  near_m > 0 marks a structured segment: its dense product only covers
// the poles within one tile of size near_m of each output column (the rest is
// low rank).  a_img / b_img / it_* place the segment in the split path's digit
// images and work lists.
struct GemmSeg {
  const double* A;
  int64_t lda;
  const int32_t* acol;
  const int32_t* plist;
  int32_t rows, kk, K, near_m;
  const double* D;
  const int32_t* org;
  const double* tau;
  const double* zhat;
  const double* scol;
  double* C;
  int64_t ldc;
  const int32_t* cpos;
  int64_t a_img, b_img;    // element offsets (bf16) of the digit images
  int64_t it_a, it_b, it_t;  // first item in the digit-A, digit-B and tile work lists
  // split path with plain dense operands (the adjoint's products): A(row, col) =
  // A[row * ars + col * lda] (ars = 1 on the merge path); when Bd is set, B(k, j) =
  // Bd[k + j * ldb] 2^-cexp[j] replaces the generated Cauchy-like entries, and the
  // product's column j is scaled back by 2^cexp[j]
  int64_t ars;
  const double* Bd;
  int64_t ldb;
  const int32_t* cexp;
  // generated B with its columns drawn from a root list: column jj is root bcol[jj]
  // (the structured path's W products, Qhat(I, pivot roots)); NULL = identity
  const int32_t* bcol;
  int32_t acc;  // 1: the product is added to C (the structured path's low-rank part)
  // shared A image: a_kt > 0 makes the segment read the A digits written for another
  // segment (a_img points at its first k-tile, a_kt is that image's k-tiles per row
  // tile), and the first bq0 rows of B are zero (the segment's poles start there)
  int32_t bq0;
  int32_t a_kt;
  int32_t part;  // the structured path's segment builder: the part a segment belongs to
  // general Cauchy-like products: A enters the split product as A 2^-aexp, and column j
  // of the product is scaled back by a further 2^oexp[j] (NULL: none)
  int32_t aexp;
  const int32_t* oexp;
  // structured B from generators (struct_entry below); NULL: the Cauchy-like or dense B
  const double* tgen;
  int64_t toff;
  int32_t tkind;
};

// Entry (k, j) of a structured B given by generators: Toeplitz tgen[k - j + toff] (kind 1),
// Hankel tgen[k + j] (2), Vandermonde tgen[k]^j by binary powering (3), or a cyclic table
// tgen[(k j) mod toff] (4: the real or imaginary part of the DFT matrix of order toff).
__device__ __forceinline__ double struct_entry(const GemmSeg& sg, int64_t k, int64_t j) {
  if (sg.tkind == 1) return sg.tgen[k - j + sg.toff];
  if (sg.tkind == 2) return sg.tgen[k + j];
  if (sg.tkind == 3) {
    double x = sg.tgen[k], r = 1.0;
    for (int64_t e = j; e > 0; e >>= 1) {
      if (e & 1) r *= x;
      x *= x;
    }
    return r;
  }
  return sg.tgen[(k * j) % sg.toff];
}

struct Plan {
  const Problem* prob;  // sorted problems (device)
  int32_t nprob;        // problems in the plan
  int32_t leaf;         // leaf size
  int64_t nslots;       // N
  double* Q0;           // caller's Q (buffer 0)
  double* Q1;           // internal Q (buffer 1)
  const double* d;      // caller's d
  const double* e;      // caller's e
  double* lam_out;      // caller's lam
  Vecs v;               // vectors of the level being processed (one of two sets by level parity)
  MergeInfo m;
  const double* clam;   // the children's level: eigenvalues and boundary rows, i.e. the other set
  const double* cbf;
  const double* cbl;
  double* lam2[2];      // leaves: both sets (a leaf writes the set of its problem's depth parity)
  double* bf2[2];
  double* bl2[2];
  Stats* stats;         // NULL when statistics are off
  int* status;          // device status word
  int32_t max_iter;
  int32_t split_min_K;  // merges with K >= this use the split path (0: never)
  int32_t split_slices; // BF16 digit slices per operand
  int32_t split_chunk_steps;  // > 0: drain the split accumulators every this many k-steps
  GemmSeg* segs;        // 2 M + 1 segments of the current level (split and structured paths)
  __nv_bfloat16* img;   // digit images (split path)
  int64_t img_cap;      // capacity of img in elements
  long long spin_budget;
  int32_t struct_min_K; // merges with K >= this use the structured path (0: never)
  int32_t struct_m;     // tile size of the structured path
  int32_t struct_split; // 1: the structured path's products run on the split tensor-core GEMM
  int32_t pad_;
  const int32_t* ss_accept;  // per merge part (2g + p): 1 if the structured split path took it
};

// Scratch of the structured path: one slot per (segment, row tile I, column tile J).
struct StructArgs {
  int m;          // tile size
  int rmax;       // largest rank kept in low-rank form (larger: dense tile)
  int Tmax;       // tiles per dimension allotted per segment
  double tol;     // SRRSC stopping tolerance relative to the tile's largest entry
  int* srank;     // per slot: rank r, -1 = dense fallback, 0 = empty
  int* spiv;      // per slot x rmax: root index of pivot column a
  double* sy;     // per slot x rmax: Theorem-2 generator y_a
  double* svr;    // per slot x m: column generator v^(r) of the tile's columns
  int* scolpiv;   // per slot x m: pivot position of the column, -1 if not a pivot
  double* W;      // per (segment, I) x rmax columns of ldw rows: Qtilde(:, I) Qhat(I, pivots)
  int64_t ldw;
  int* status;
  unsigned long long* flops;  // executed multiply-add flops (statistics; NULL when off)
  unsigned long long* ranks;  // statistics (NULL when off): far tiles, sum of their ranks,
                              // dense fallbacks, largest rank kept
  int fallback_only;          // k_struct_apply: only the tiles that stayed dense (the split variant)
  int all_offdiag;            // k_srrsc: every tile off the diagonal (rank profile), not only |I - J| >= 2
};

// Scratch and outputs of the structured path on the split GEMM (one level, or one
// stand-alone product): from the SRRSC results of the structured segments it builds
// three lists of split segments -- the near-diagonal products (written), the W
// products Qtilde(:, I) Qhat(I, pivot roots) (into W), and the applications
// C(:, J) += W_J R_J (added) -- and the R_J blocks with their column scales.
struct SSArgs {
  const GemmSeg* ssegs;  // structured segments (near_m > 0 marks a part on the structured path)
  int nseg;
  StructArgs S;          // the SRRSC results and tile geometry
  int digits;            // split slices per operand
  GemmSeg* img_segs;     // nseg + 1: one per part, owning its A digit image (no products)
  GemmSeg* near_segs;    // each list: nseg * Tmax segments + the terminator
  GemmSeg* w_segs;
  GemmSeg* ap_segs;
  int64_t* counts;       // [4]: segments of the near, W, apply and image lists (device)
  int32_t* wcol0;        // per slot: first W column of its pivots
  int32_t* bcol;         // root of each W column, in W-product order
  int32_t* wpos;         // W column of each W-product column
  int64_t bcap;          // capacity of bcol / wpos
  double* W;             // ldw x wcap
  int64_t ldw, wcap;
  double* R;             // R_J blocks, column-major with ld = the block's rows
  int64_t rcap;
  int32_t* cexp;         // per (segment, J) x m: column scale exponents of R_J
  int64_t* item;         // per (segment, tile) scratch: 6 x nseg x Tmax
  int32_t* accept;       // per segment: 1 if this path takes the part (else the plain split path)
  int64_t img_cap;       // digit-image capacity (elements) of each of the three products
  int* status;
  unsigned long long* flops;  // statistics: executed flops of the three products (NULL when off)
  unsigned long long* bytes;  // statistics: their algorithmic HBM bytes (NULL when off)
  unsigned long long* parts;  // statistics: parts taken, parts left (NULL when off)
};

// Exclusive scan of four int64 values over the block (warp shuffles, then the
// warp totals scanned by warp 0); blockDim.x a multiple of 32, at most 1024.
__device__ __forceinline__ void block_excl_scan4(int64_t (&v)[4], int64_t (&sc)[4][32]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t inc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    inc[q] = v[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, inc[q], o);
      if (lane >= o) inc[q] += t;
    }
    if (lane == 31) sc[q][w] = inc[q];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int64_t x = lane < nw ? sc[q][lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
      }
      if (lane < nw) sc[q][lane] = x;  // inclusive over warps
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = inc[q] - v[q] + (w > 0 ? sc[q][w - 1] : 0);
}

// A merge (node) of level l: node i of problem p splits at mid.
struct Node {
  int64_t lo, mid, hi;  // problem-local rows/columns
  int64_t v0;           // first vector slot (p.voff + lo)
  const Problem* p;
  double* src;          // children's eigenvectors: element (r, c) of the node at src[r + c*lds]
  double* dst;          // the node's eigenvectors
  int64_t lds, ldd;
  double b;             // coupling entry e[mid-1]
};

__device__ __forceinline__ int64_t node_bound(int64_t i, int64_t n, int level) {
  return (i * n) >> level;
}

// Power-of-two scales of the split products.  exp_above(mx) is an e with mx < 2^e
// (0 for mx = 0), kept in [-1000, 1022] so that 2^e and 2^-e are both normal: a
// subnormal mx gets 2^-1000, which still bounds it; mx >= 2^1022 is out of range.
// pow2c(e) is 2^e built from its exponent bits for e in [-1022, 1023] and clamped
// there (bare bit building gives inf at e = +-1024 and wraps the sign bit beyond, so
// a 0 * inf in a scaled product becomes NaN).  scale2(x, e) = x 2^e for |e| <= 2044,
// in two such factors, for exponents that are sums of two scales.
__device__ __forceinline__ int exp_above(double mx) {
  const int e = mx > 0.0 ? ilogb(mx) + 1 : 0;
  return e < -1000 ? -1000 : (e > 1022 ? 1022 : e);
}
__device__ __forceinline__ double pow2c(int e) {
  e = e < -1022 ? -1022 : (e > 1023 ? 1023 : e);
  return __hiloint2double((1023 + e) << 20, 0);
}
__device__ __forceinline__ double scale2(double x, int e) {
  const int h = e / 2;
  return (x * pow2c(h)) * pow2c(e - h);
}

// A non-finite d or e entry is read as zero wherever the eigensolver reads the
// caller's arrays (the corner-modified diagonal, the leaves, each merge's coupling)
// and the call reports TDC_ENONFINITE: that problem's results are then not those of
// its input, but no NaN or infinity reaches the orderings, counts and ranks that
// later kernels index with.
__device__ __forceinline__ double finite_or_zero(double x) { return isfinite(x) ? x : 0.0; }

// An entry of the caller's d or e as the solver reads it: non-finite as zero, then times
// 2^-escale (exact).  A problem whose largest finite |d|, |e| lies outside
// [2^-400, 2^400] is solved scaled by the power of two that brings it into [1, 2), so
// that no square, product or sum of its entries overflows or underflows; escale is 0
// otherwise and the values enter unchanged.
__device__ __forceinline__ double input_entry(double x, int escale) {
  return escale ? scale2(finite_or_zero(x), -escale) : finite_or_zero(x);
}

__device__ __forceinline__ Node make_node(const Plan& P, int level, int64_t g) {
  Node nd;
  const Problem* p = P.prob + (g >> level);
  int64_t i = g & ((((int64_t)1) << level) - 1);
  nd.p = p;
  nd.lo = node_bound(i, p->n, level);
  nd.hi = node_bound(i + 1, p->n, level);
  nd.mid = node_bound(2 * i + 1, p->n, level + 1);
  nd.v0 = p->voff + nd.lo;
  double* b0 = P.Q0 + p->off_q;
  double* b1 = P.Q1 + p->qoff1;
  int64_t l0 = p->ld0, l1 = p->n;
  // level l writes buffer (l & 1); its children (level l+1) live in the other one
  if (level & 1) {
    nd.dst = b1 + nd.lo + nd.lo * l1; nd.ldd = l1;
    nd.src = b0 + nd.lo + nd.lo * l0; nd.lds = l0;
  } else {
    nd.dst = b0 + nd.lo + nd.lo * l0; nd.ldd = l0;
    nd.src = b1 + nd.lo + nd.lo * l1; nd.lds = l1;
  }
  nd.b = input_entry(P.e[p->off_de + nd.mid - 1], p->escale);
  return nd;
}

// binary search: index of the problem (among the first cnt) owning vector slot s
__device__ __forceinline__ int find_problem_by_slot(const Problem* prob, int cnt, int64_t s) {
  int lo = 0, hi = cnt - 1;
  while (lo < hi) {
    int m = (lo + hi + 1) >> 1;
    if (prob[m].voff <= s) lo = m; else hi = m - 1;
  }
  return lo;
}

// node index on level l containing local row r of a problem of order n
__device__ __forceinline__ int64_t node_of_row(int64_t r, int64_t n, int level) {
  int64_t i = (((r + 1) << level) - 1) / n;  // floor(i n / 2^l) <= r
  while (node_bound(i, n, level) > r) --i;
  while (node_bound(i + 1, n, level) <= r) ++i;
  return i;
}

// ---------------------------------------------------------------------------
// Arithmetic helpers
// ---------------------------------------------------------------------------
// Reciprocal of x: hardware estimate r (rcp.approx.ftz.f64, relative error e of
// about 2^-20) followed by one third-order refinement r <- r + r (e + e^2) with
// e = 1 - x r, which leaves a relative error e^3 (about 2^-60) before the final
// rounding: within an ulp of 1/x for normal, finite x, in three FP64 operations
// instead of the four of two Newton-Raphson steps.
__device__ __forceinline__ double rcp_nr(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// 1/sqrt(x): hardware estimate (rsqrt.approx.ftz.f64) followed by two Newton-Raphson
// refinements y <- y (3 - x y^2) / 2, each of which squares the relative error.
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double h = 0.5 * x;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_prod(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// A call's status slot is two words: status[0] the first error (first writer wins),
// status[1] warning bits (results written, accuracy possibly reduced).
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}
constexpr int kWarnSplitLevel = 1;  // a split-path level sum reached 2^23 (half its exact FP32 range)
__device__ __forceinline__ void set_warning(int* status, int bit) {
  if (status) atomicOr(status + 1, bit);
}

}  // namespace tdc

// Host-side launchers (one translation unit each).
namespace tdc {
struct LevelLaunch {
  int level;
  int64_t merges;     // M
  int32_t nprob_act;  // problems taking part (prefix)
  int64_t nslots;     // vector slots of the active problems
  int64_t max_n;      // largest merge order on the level
  int64_t min_n;      // smallest merge order on the level
};
cudaError_t launch_dmod(const Plan& P, cudaStream_t s);
cudaError_t launch_leaves(const Plan& P, int64_t nleaves, int max_leaf, cudaStream_t s);
// levels with at least this many slots also run the thread-per-root kernels
constexpr int64_t kSmallMinSlots = 32768;
cudaError_t launch_prepare(const Plan& P, const LevelLaunch& L, cudaStream_t s);
cudaError_t launch_rotate(const Plan& P, const LevelLaunch& L, cudaStream_t s);
cudaError_t launch_boundary_rot(const Plan& P, const LevelLaunch& L, cudaStream_t s);
cudaError_t launch_boundary_out(const Plan& P, const LevelLaunch& L, cudaStream_t s);
cudaError_t launch_secular(const Plan& P, const LevelLaunch& L, cudaStream_t s);
cudaError_t launch_lowner(const Plan& P, const LevelLaunch& L, cudaStream_t s);
cudaError_t launch_finalize(const Plan& P, const LevelLaunch& L, cudaStream_t s);
cudaError_t launch_copy_deflated(const Plan& P, const LevelLaunch& L, int sign_normalise, cudaStream_t s);
cudaError_t launch_sign_and_output(const Plan& P, int sign_normalise, cudaStream_t s);
// Rank-one eigenproblem: secular roots, Loewner zhat, column normalisers.  zz (K doubles),
// xz (K float2) and xlo (K floats) are scratch for the FP32 pre-iteration of the roots
// (NULL: the roots iterate in FP64 only).
cudaError_t launch_rank_one(const double* D, const double* z, int64_t K, double rho, int max_iter, int* org,
                            double* tau, double* zhat, double* s, double* zz, float2* xz, float* xlo, int* status,
                            cudaStream_t st);
// bytes of that scratch for K poles (three 256-byte aligned arrays)
size_t rank_one_scratch_bytes(int64_t K);
cudaError_t launch_gemm_dense(const Plan& P, const LevelLaunch& L, int64_t max_tiles, cudaStream_t s);
cudaError_t launch_gemm_tiny(const Plan& P, const LevelLaunch& L, cudaStream_t s);
cudaError_t launch_split_pack(const Plan& P, const LevelLaunch& L, int max_pass, cudaStream_t s);
cudaError_t launch_gemm_split(const Plan& P, const LevelLaunch& L, int64_t g0, int64_t g1, int pass, cudaStream_t s,
                              cudaEvent_t mid);
cudaError_t launch_seg_split(const GemmSeg* segs_dev, int nseg, int S, int* status, long long spin_budget,
                             __nv_bfloat16* img, int chunk_steps, cudaStream_t s);
cudaError_t launch_split_list(const GemmSeg* segs, int nseg_bound, const int64_t* dcount, int S, int* status,
                              long long spin_budget, __nv_bfloat16* img, int chunk_steps, unsigned int* lvl_max,
                              cudaStream_t s, cudaEvent_t mid);
cudaError_t launch_srrsc(const GemmSeg* segs, int nseg, const StructArgs& A, cudaStream_t s);
cudaError_t launch_struct_fallback(const GemmSeg* segs, int nseg, const StructArgs& A, cudaStream_t s);
cudaError_t launch_ss_build(const SSArgs& A, cudaStream_t s);
cudaError_t launch_ss_gate(const int32_t* accept, GemmSeg* plain_list, cudaStream_t s);
cudaError_t launch_cauchy_like_prep(int64_t m, int64_t n, const double* A, int64_t lda, const double* d,
                                    const double* w, const double* u, const double* v, int32_t* org, double* tau,
                                    double* scol, int32_t* eb, int32_t* cexp, int32_t* eA,
                                    unsigned long long* maxsq, bool scale, cudaStream_t s);
cudaError_t launch_cauchy_like_patch(GemmSeg* seg, const int32_t* eA, cudaStream_t s);
cudaError_t launch_seg_dense(const GemmSeg& seg, cudaStream_t s);
cudaError_t launch_struct(const GemmSeg* segs, int nseg, const StructArgs& A, cudaStream_t s);
cudaError_t launch_struct_segs(const Plan& P, const LevelLaunch& L, cudaStream_t s);
constexpr int kStructRmax = 64;
// digits of the adjoint's split products and their image size for a batch
constexpr int kAdjSlices = 7;
int64_t adjoint_split_img_elems(int batch, int64_t n);
cudaError_t launch_adjoint(int batch, int n, const double* lam, const double* Q, int64_t ldq, int64_t sQ,
                           const double* lam_bar, const double* Q_bar, int64_t sQb, double* d_bar,
                           double* e_bar, double* ws, int* status, long long spin_budget, cudaStream_t s);
int64_t split_img_elems(int64_t rows_top, int64_t rows_bot, int64_t kk_bound, int64_t K_bound, int S);
constexpr int kSplitBM = 128, kSplitBN = 64, kSplitBK = 16;
// dense symmetric reduction to tridiagonal form and its back-transform (tdc_sytrd.cu)
constexpr int kTrdNb = 128;        // reflectors per panel
constexpr int kTrdThreads = 512;   // threads of a panel block (one block per SM)
constexpr int64_t kTrdSmemV = 16384;  // the column is staged in shared memory up to this order
constexpr int kTrdMaxBlocks = 1024;
constexpr int kTrdSplitMin = 512;  // trailing updates of this order and above take the split product
constexpr int kTrdSlices = 7;      // digits of the reduction's split products
constexpr int64_t kTrdMaxLd = (int64_t)1 << 27;  // the panel kernel's column offsets are 32-bit
constexpr int kOrmKb = 128;        // reflectors per back-transform block
constexpr int kOrmZThreads = 512;
constexpr int kOrmTileTarget = 304;  // split-K: aim at this many output tiles for V^T X
struct TrdPanel {
  double* A;
  int64_t lda, n, p;
  int32_t nbp;          // reflectors in the panel (columns p .. p + nbp - 1)
  double* V;            // n x kTrdNb, ld n, rows indexed globally
  double* W;
  double* Vr;           // the same panels row-major (ld kTrdNb) for the row updates
  double* Wr;
  int32_t vsm;          // v staged in shared memory (n <= kTrdSmemV)
  double* d;
  double* e;
  double* tau;
  double* x;            // the current column (n)
  double* y;            // A22 v (n)
  double* ps;           // per-block partial sums (kTrdMaxBlocks each)
  double* pvy;
  double* pw;           // W^T v, V^T v of the current column (kTrdNb each)
  double* pv;
  unsigned* bar;        // grid barrier counter
  int* status;
  long long budget;
};
struct TrdUpdate {
  double* A;
  int64_t lda, n, t0;  // trailing matrix A(t0:n, t0:n)
  int32_t nb;
  const double* V;
  const double* W;
  int64_t ld;
  double* Aop;
  double* Bop;
  int32_t* cexp;
  unsigned long long* wmax;
  GemmSeg* segs;
  __nv_bfloat16* img;
  int* status;
  long long budget;
  int chunk_steps;
};
struct OrmStep {
  int64_t n, b0, mb, ncols;  // reflectors b0 .. b0 + kbp - 1 act on rows b0 + 1 .. n - 1 (mb rows)
  int32_t kbp;
  double* Vb;
  int64_t ldv;
  double* X;
  int64_t ldx;
  const int32_t* xexp;
  const double* tau;
  double* G;  // ns x kbp x kbp partial Gram matrices
  double* Y;  // ns x kbp x ncols partial V^T X
  double* Z;  // kbp x ncols
  int32_t* zexp;
  int32_t ns;
  int64_t kper;
  GemmSeg* list1;
  GemmSeg* list2;
  __nv_bfloat16* img;
  int64_t img2;
  int S;
  int* status;
  long long budget;
  int chunk_steps;
};
int trd_panel_grid();
cudaError_t launch_sym_fill(int64_t n, double* A, int64_t lda, cudaStream_t s);
cudaError_t launch_trd_panel(const TrdPanel& P, int grid, cudaStream_t s);
cudaError_t launch_trd_update(const TrdUpdate& U, cudaStream_t s);
cudaError_t launch_trd_tail(int64_t n, const double* A, int64_t lda, double* d, double* e, double* tau,
                            cudaStream_t s);
cudaError_t launch_orm_xexp(int64_t rows, int64_t ncols, const double* X, int64_t ldx, int32_t* xexp,
                            cudaStream_t s);
cudaError_t launch_orm_step(const OrmStep& O, const double* A, int64_t lda, cudaStream_t s);
size_t orm_z_smem(int kbp);
// structured operands (tdc_operands.cu): per-column exponents of the generated B and A's
// row-norm exponent; the DFT tables
cudaError_t launch_operand_prep(int64_t m, int64_t n, const double* A, int64_t lda, const double* t, int kind,
                                double* winmax, int32_t* cexp, int32_t* oexp, int32_t* eA,
                                unsigned long long* maxsq, cudaStream_t s);
cudaError_t launch_dft_tables(int64_t n, double* cosv, double* msinv, cudaStream_t s);
// symmetric band divide and conquer (tdc_banded.cu)
cudaError_t launch_bd_copy_band(int64_t n, int b, const double* AB, int64_t ldab, double* ABw, cudaStream_t s);
cudaError_t launch_bd_tear(double* ABw, int64_t ldab, int b, int64_t m, double* wv, cudaStream_t s);
// The leaves of the band tree, all at once: dense block of leaf t (rows [lo, lo + L) of the
// torn band) at Ab + lo lmax (ld L), its tridiagonal in d, e and reflector scalars in tau at
// offset lo; the tridiagonal eigenvectors Zb + lo lmax (ld L) back-transformed into the
// diagonal block of Q.
constexpr int kBdLeafChunk = 1024;
constexpr int kBdLeafThreads = 512;
struct BdLeafTable {
  int64_t lo[kBdLeafChunk];
  int32_t L[kBdLeafChunk];
};
struct BdLeafArgs {
  const double* ABw;
  int64_t ldab;
  int32_t b;
  int32_t nleaf;  // leaves in this launch's table
  int64_t lmax;
  double* Ab;
  double* d;
  double* e;
  double* tau;
  const double* Zb;
  double* Q;
  int64_t ldq;
};
cudaError_t launch_bd_leaf_trd(const BdLeafArgs& A, const BdLeafTable& T, cudaStream_t s);
cudaError_t launch_bd_leaf_back(const BdLeafArgs& A, const BdLeafTable& T, cudaStream_t s);
cudaError_t launch_bd_z(int64_t nn, const double* Q, int64_t ldq, int64_t ra, int64_t rb, int b, const double* w,
                        double* z, cudaStream_t s);
// Overflow guard of the dense and band solvers: the largest finite |entry| of a column-major
// rows x cols block (lower != 0: its lower triangle only) and, when that lies outside
// [2^-400, 2^400], the block times the power of two 2^-escale that puts it in [1, 2)
// (exact); *escale = 0 otherwise.  mx and escale: 8 and 4 bytes of device scratch.
// launch_range_unscale: x[0:n) times 2^escale.
cudaError_t launch_range_scale(double* A, int64_t rows, int64_t cols, int64_t ld, int lower, unsigned long long* mx,
                               int* escale, cudaStream_t s);
cudaError_t launch_range_unscale(double* x, int64_t n, const int* escale, cudaStream_t s);
// Scratch of the band sort and deflation (arrays of nn entries, free while they run).
struct BdScratch {
  double* sk;      // sort: the chunks' sorted keys
  int32_t* si;     // sort: their indices
  int32_t* surv;   // deflation: sorted positions of the poles surviving type 1
  int32_t* slot;   // deflation: deflated entry keyed by the position at which the scan deflates it
  double* c;       // deflation: speculative rotation of each consecutive survivor pair: c, s,
  double* s;       //   the combined weight and the two new poles
  double* w;
  double* dp;
  double* dn;
};
cudaError_t launch_bd_sort(int64_t nn, const double* D, const double* z, double* Ds, double* zs, int32_t* perm,
                           const BdScratch& S, cudaStream_t s);
cudaError_t launch_bd_deflate(int64_t nn, double* Ds, double* zs, int32_t* kept, int32_t* defl, int32_t* rotp,
                              double* rotcs, int32_t* cnt, double* rho, const BdScratch& S, int* status,
                              cudaStream_t s);
cudaError_t launch_bd_rotate(int64_t nrows, double* Q, int64_t ldq, const int32_t* perm, const int32_t* rotp,
                             const double* rotcs, int nr, int* status, cudaStream_t s);
cudaError_t launch_bd_gather(int64_t nrows, const double* Q, int64_t ldq, const int32_t* perm, const int32_t* kept,
                             int K, const int32_t* defl, int nd, const double* Ds, const double* zs, double* Qw,
                             double* DK, double* zK, double* Dd, int* status, cudaStream_t s);
cudaError_t launch_bd_finish(int64_t nrows, const double* Qw, double* Q, int64_t ldq, int K, int nd, const double* DK,
                             const int32_t* org, const double* tau, const double* Dd, double* D, cudaStream_t s);
cudaError_t launch_bd_copy_back(int64_t nrows, int64_t ncols, const double* Qw, double* Q, int64_t ldq,
                                cudaStream_t s);
cudaError_t launch_bd_zero(int64_t rows, int64_t cols, double* Q, int64_t ldq, cudaStream_t s);
// bidiagonal SVD through the Golub-Kahan tridiagonal (tdc_bdsdc.cu)
cudaError_t launch_gk_build(int64_t n, const double* d, const double* e, double* td, double* te, cudaStream_t s);
cudaError_t launch_gk_extract(int64_t n, const double* lam, const double* Q, int64_t ldq, double* sigma, double* U,
                              int64_t ldu, double* VT, int64_t ldvt, cudaStream_t s);
constexpr int kDenseBM = 128, kDenseBN = 64, kDenseBK = 16;
// merges of order n <= kDenseSmallN take 32 x 32 tiles: their halves have at most 64
// rows, so a 128-row tile would leave most of its FP64 multiply-adds on padding
constexpr int kDenseSmallN = 128, kDenseSmallBM = 32, kDenseSmallBN = 32;
__host__ __device__ inline void dense_tile_dims(int64_t n, int& bm, int& bn) {
  bm = n <= kDenseSmallN ? kDenseSmallBM : kDenseBM;
  bn = n <= kDenseSmallN ? kDenseSmallBN : kDenseBN;
}
// merges of order n <= kTinyN (halves of at most 16 rows and poles, K <= 32) off the
// split and structured paths take a warp each (k_gemm_tiny) instead of tiles
constexpr int kTinyN = 32;
__host__ __device__ inline bool tiny_merge(int64_t n, int K, int ntop, int nbot, int split_min_K,
                                           int struct_min_K) {
  return n <= kTinyN && K > 0 && ntop <= kTinyN / 2 && nbot <= kTinyN / 2 &&
         !(split_min_K > 0 && K >= split_min_K) && !(struct_min_K > 0 && K >= struct_min_K);
}
}  // namespace tdc
