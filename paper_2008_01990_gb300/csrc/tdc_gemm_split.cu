// tdc_gemm_split.cu -- split-precision eigenvector update C = A * Qhat on the
// BF16 tensor cores (tcgen05, FP32 accumulators in TMEM), FP64 result.
//
// Both operands are written as fixed-point numbers with scale 1 (every entry of
// an orthogonal matrix and of the orthonormal Cauchy-like Qhat has |x| <= 1) and
// cut into S balanced base-256 digits:  x = sum_s 2^(-8(s+1)) a_s with integer
// digits |a_0| <= 256 and a_s in [-128, 127] (x 2^56 rounded to an integer),
// each exact in BF16.  Then
//     C = sum_{s+t <= S-1} 2^(-8(s+t+2)) (a_s . u_t),
// and every product of digits is an integer of magnitude at most 2^16.  All
// products of one level m = s+t accumulate in their own FP32 TMEM accumulator
// over the whole reduction, which is exact while the level's partial sums stay
// below 2^24.  By Cauchy-Schwarz on the unit-norm rows of A and columns of Qhat
// the sums of levels 0 and 1 do; the digits below the top one are zero-mean, so on
// random and weakly structured spectra the higher levels are random walks of about
// 2^12.4 sqrt((m+1) kk), far below 2^24 (signed-magnitude digits would not do:
// their mean follows sign(A U), which is coherent for smooth eigenvectors).  That
// argument fails in the rows next to a merge's split when the eigenvectors are
// smooth: there the rows of A are nearly parallel to z, so A U sums the secular
// terms z_k zhat_k / delta_kj, which share their sign over long runs of k.  On the
// Clement, Hermite and spherical-harmonic matrices of order 16384 those level-3
// sums exceed 2^24 and round (orthogonality ratio about 1e4).  Draining the
// accumulators every ck k-steps (the kChunk instance) bounds every level sum by
// the chunk's length instead of the whole reduction; until that schedule is the
// default, the FP64 merge is the path for such inputs.  The S level accumulators
// (S x 64 TMEM columns) are combined in FP64 once per tile (once per chunk with
// drains).  Dropped levels (m >= S) and the rounded digits cost about 2^-8S
// absolute per entry.
//
// Data flow per merge part: k_split_a writes the digits of the gathered A
// columns, k_split_b generates Qhat from its generators in FP64 (once per entry)
// and writes its digits; both images are laid out tile by tile in exactly the
// shared-memory form the tensor core reads (K-major 8 x 16-byte core matrices),
// so k_gemm_split moves each 16-deep k-step of a tile (S A-slices of 4 KB and S
// B-slices of 2 KB, contiguous) with two bulk copies and keeps a 4-stage ring of
// shared-memory buffers in flight with mbarriers.  A tcgen05 MMA with M = 128
// costs about the same issue time for any N up to 128, so the S(S+1)/2 digit
// products of a step are issued as S wide MMAs (A_s against the stacked B slices,
// N = 64 (S - s), split at 256): 10 MMAs per step for S = 7 instead of 28.
// Sixteen epilogue warps read the accumulators (four per TMEM lane quarter):
// on shallow tiles the epilogue, not the MMAs, sets the time.
#include <float.h>

#include "tdc_common.cuh"
#include "tdc_umma.cuh"

namespace tdc {

namespace {
constexpr int BM = kSplitBM, BN = kSplitBN, BK = kSplitBK;
constexpr int kATileElems = BM * BK;  // 2048 per slice (4 KB)
constexpr int kBTileElems = BN * BK;  // 1024 per slice (2 KB)
constexpr int kMaxS = 7;
constexpr int kStages = 4;
constexpr int kGroupRows = 8;

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// element offset of (row, k) inside one K-major core-matrix tile (8 rows x 8 k per core
// matrix, core matrices along K 64 elements apart, 8-row groups BK*8 elements apart)
__device__ __forceinline__ int core_off(int r, int k) { return (r >> 3) * (BK * 8) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7); }


// The S leading balanced base-256 digits of x (|x| <= 1 + O(eps)), as BF16 bit
// patterns: F = round(x 2^56) as a two's-complement integer, written as
// F = sum_s d_s 256^(6-s) with d_s in [-128, 127] for s >= 1 (the top digit carries
// the rest, |d_0| <= 256).  Below the top digit the digits are zero-mean whatever
// the sign of x, so sums of their products behave like random walks.  With
// G = F + 128 (1 + 256 + ... + 256^5) the bytes of G below bit 48 are d_s + 128 and
// G >> 48 is d_0, so the digits come out of 32-bit field extractions; a small
// integer d becomes a float as (2^23 + 2^22 + d) - (2^23 + 2^22) on the FP32 pipe,
// and its BF16 pattern is the float's upper half (exact: |d| <= 256).
__device__ __forceinline__ void digits_bf16(double x, int S, uint32_t (&dg)[kMaxS]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const bool neg = (b >> 63) != 0;
  int e = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (e) m |= 1ull << 52; else e = 1;
  const int sh = e - 1019;  // |x| 2^56 = m * 2^(e - 1075 + 56)
  unsigned long long mag;
  if (sh >= 0) mag = (sh < 8) ? (m << sh) : 0ull;
  else if (sh > -63) mag = ((m >> (-sh - 1)) + 1ull) >> 1;  // round half up
  else mag = 0ull;
  const long long F = neg ? -(long long)mag : (long long)mag;
  const long long G = F + 0x808080808080ll;
  const uint32_t lo = (uint32_t)G;
  const int hi = (int)(G >> 32);
  int d[kMaxS];
  d[0] = hi >> 16;
  d[1] = ((hi >> 8) & 255) - 128;
  d[2] = (hi & 255) - 128;
  d[3] = (int)(lo >> 24) - 128;
  d[4] = (int)((lo >> 16) & 255) - 128;
  d[5] = (int)((lo >> 8) & 255) - 128;
  d[6] = (int)(lo & 255) - 128;
#pragma unroll
  for (int s = 0; s < kMaxS; ++s) {
    const float f = __int_as_float(0x4B400000 + d[s]) - 12582912.0f;
    dg[s] = (s < S) ? (__float_as_uint(f) >> 16) : 0u;
  }
}

// Eight BF16 patterns (low halves of v[0..7]) into one 16-byte store.
__device__ __forceinline__ uint4 pack8(const uint32_t* v) {
  uint4 o;
  o.x = v[0] | (v[1] << 16);
  o.y = v[2] | (v[3] << 16);
  o.z = v[4] | (v[5] << 16);
  o.w = v[6] | (v[7] << 16);
  return o;
}

__device__ __forceinline__ int find_seg(const GemmSeg* segs, int nseg, int64_t w, int which) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int m = (lo + hi + 1) >> 1;
    const int64_t v = which == 0 ? segs[m].it_a : (which == 1 ? segs[m].it_b : segs[m].it_t);
    if (v <= w) lo = m; else hi = m - 1;
  }
  return lo;
}

}  // namespace

int64_t split_img_elems(int64_t rows_top, int64_t rows_bot, int64_t kk_bound, int64_t K_bound, int S) {
  const int64_t KB = cdiv(kk_bound, BK), CT = cdiv(K_bound, BN);
  const int64_t a = (cdiv(rows_top, BM) + cdiv(rows_bot, BM)) * KB * S * kATileElems;
  const int64_t b = 2 * CT * KB * S * kBTileElems;
  return a + b;
}

// ---------------------------------------------------------------------------
// Segments of a tree level: one per (merge, top/bottom part).
// ---------------------------------------------------------------------------
// One block: each thread counts the digit tiles, output tiles and image elements
// of a contiguous range of merges, a block scan gives every range its offsets,
// then the threads write their segments.
// When every non-deflated pole has support in both halves (cross rotations pair
// each pole of one child with one of the other, as for equal spectra), the two
// pole lists are the same and the bottom part reuses the top part's Qhat image.
__device__ __forceinline__ bool shared_b(const Plan& P, int64_t g) {
  const int K = P.m.K[g];
  return P.m.ntop[g] == K && P.m.nbot[g] == K;
}

__device__ __forceinline__ void split_seg_counts(const Plan& P, int level, int64_t g, int S, int p, int64_t& ta,
                                                 int64_t& tb, int64_t& tt, int64_t& el) {
  ta = tb = tt = el = 0;
  const int K = P.m.K[g];
  if (!(P.split_min_K > 0 && K >= P.split_min_K)) return;
  // parts the structured split path took (it leaves the others to this path)
  if (P.struct_split && P.struct_min_K > 0 && K >= P.struct_min_K && P.ss_accept && P.ss_accept[2 * g + p]) return;
  const Node nd = make_node(P, level, g);
  const int n = (int)(nd.hi - nd.lo), n1 = (int)(nd.mid - nd.lo);
  const int64_t rows = p ? n - n1 : n1, kk = p ? P.m.nbot[g] : P.m.ntop[g];
  const int64_t RT = cdiv(rows, BM), KB = cdiv(kk, BK), CT = cdiv(K, BN);
  ta = RT * KB;
  tb = (p == 1 && shared_b(P, g)) ? 0 : CT * KB;
  tt = RT * CT;
  el = ta * S * kATileElems + tb * S * kBTileElems;
}

// Merges [g0, g1), or (pass >= 0) the merge range of that pass from k_split_pack
// (none past the pass count).  Only merge parts on the split path get a segment
// (the list is compacted: on many-merge levels most merges are below the
// threshold); the count goes to P.m.sseg, which the digit and product kernels read.
__global__ void __launch_bounds__(1024) k_split_segs(Plan P, int level, int64_t g0, int64_t g1, int pass) {
  __shared__ int64_t sc[4][32];
  const int S = P.split_slices;
  if (pass >= 0) {
    const bool live = pass < P.m.spass[0];
    g0 = live ? P.m.spass[1 + 2 * pass] : 0;
    g1 = live ? P.m.spass[2 + 2 * pass] : 0;
  }
  const int64_t M = g1 - g0, items = 2 * M;
  const int64_t per = (items + blockDim.x - 1) / blockDim.x;
  const int64_t w0 = min(items, (int64_t)threadIdx.x * per), w1 = min(items, w0 + per);
  int64_t cta = 0, ctb = 0, ctt = 0, cel = 0, cns = 0;
  for (int64_t w = w0; w < w1; ++w) {
    int64_t ta, tb, tt, el;
    split_seg_counts(P, level, g0 + w / 2, S, (int)(w & 1), ta, tb, tt, el);
    cta += ta; ctb += tb; ctt += tt; cel += el;
    cns += el > 0 ? 1 : 0;
  }
  int64_t v[4] = {cta, ctb, ctt, cel};
  block_excl_scan4(v, sc);
  __syncthreads();
  int64_t vn[4] = {cns, 0, 0, 0};
  block_excl_scan4(vn, sc);
  int64_t ia = v[0], ib = v[1], it = v[2], e = v[3], ns = vn[0];
  for (int64_t w = w0; w < w1; ++w) {
    const int64_t g = g0 + w / 2;
    const int p = (int)(w & 1);
    int64_t ta, tb, tt, el;
    split_seg_counts(P, level, g, S, p, ta, tb, tt, el);
    if (el == 0) continue;
    const Node nd = make_node(P, level, g);
    const int n = (int)(nd.hi - nd.lo), n1 = (int)(nd.mid - nd.lo);
    const int K = P.m.K[g];
    GemmSeg sg;
    memset(&sg, 0, sizeof(sg));
    sg.ars = 1;
    sg.rows = p ? n - n1 : n1;
    sg.kk = p ? P.m.nbot[g] : P.m.ntop[g];
    sg.K = K;
    sg.near_m = 0;
    sg.A = nd.src + (p ? n1 : 0);
    sg.lda = nd.lds;
    sg.acol = P.v.kept + nd.v0;
    sg.plist = (p ? P.v.blist : P.v.tlist) + nd.v0;
    sg.D = P.v.Dk + nd.v0;
    sg.org = P.v.org + nd.v0;
    sg.tau = P.v.tau + nd.v0;
    sg.zhat = P.v.zhat + nd.v0;
    sg.scol = P.v.scol + nd.v0;
    sg.C = nd.dst + (p ? n1 : 0);
    sg.ldc = nd.ldd;
    sg.cpos = P.v.posr + nd.v0;
    sg.it_a = ia;
    sg.it_b = ib;
    sg.it_t = it;
    sg.a_img = e;
    sg.b_img = e + ta * S * kATileElems;
    if (p == 1 && tb == 0) {  // the top part's image: it ends where this part's starts
      int64_t ta0, tb0, tt0, el0;
      split_seg_counts(P, level, g, S, 0, ta0, tb0, tt0, el0);
      sg.b_img = e - el0 + ta0 * S * kATileElems;
    }
    if (el > 0 && P.stats) {
      const unsigned long long r = (unsigned long long)sg.rows, kq = (unsigned long long)sg.kk,
                               kc = (unsigned long long)K;
      atomicAdd(&P.stats->split_flops, 2ull * r * kq * kc);
      atomicAdd(&P.stats->split_bytes, 2ull * S * (r * kq + kq * kc) + 8ull * r * kc);
    }
    ia += ta; ib += tb; it += tt; e += el;
    P.segs[ns++] = sg;
  }
  if (threadIdx.x == blockDim.x - 1) {
    *P.m.sseg = ns;
    GemmSeg last;
    memset(&last, 0, sizeof(last));
    last.it_a = ia;
    last.it_b = ib;
    last.it_t = it;
    last.a_img = e;
    if (e > P.img_cap) {  // cannot happen with the host's bound; never write past the images
      last.it_a = last.it_b = last.it_t = 0;
      set_status(P.status, TDC_EUNSUPPORTED);
    }
    P.segs[ns] = last;
  }
}

// Levels the host cut into passes on a bound of every merge's digit images (its
// order): after deflation the actual images are known, usually far smaller, so
// the merges are packed again, greedily in order, into as few passes as fit the
// image buffer.  Greedy packing of smaller items never needs more passes than
// the host's packing of the bounds; passes beyond the count find no merges.
__global__ void __launch_bounds__(1024) k_split_pack(Plan P, int level, int64_t M, int max_pass) {
  __shared__ int64_t sc[4][32];
  const int S = P.split_slices;
  const int64_t per = (M + blockDim.x - 1) / blockDim.x;
  const int64_t a = min(M, (int64_t)threadIdx.x * per), b = min(M, a + per);
  int64_t cel = 0;
  for (int64_t g = a; g < b; ++g)
    for (int p = 0; p < 2; ++p) {
      int64_t ta, tb, tt, el;
      split_seg_counts(P, level, g, S, p, ta, tb, tt, el);
      cel += el;
    }
  int64_t v[4] = {cel, 0, 0, 0};
  block_excl_scan4(v, sc);
  int64_t run = v[0];
  for (int64_t g = a; g < b; ++g) {
    P.m.ioff[g] = run;
    for (int p = 0; p < 2; ++p) {
      int64_t ta, tb, tt, el;
      split_seg_counts(P, level, g, S, p, ta, tb, tt, el);
      run += el;
    }
  }
  if (threadIdx.x == blockDim.x - 1) P.m.ioff[M] = run;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int64_t* io = P.m.ioff;
  const int64_t cap = P.img_cap;
  int64_t g = 0;
  int c = 0;
  while (g < M && c < max_pass) {
    // last e in (g, M] with io[e] - io[g] <= cap (at least g + 1)
    int64_t lo = g + 1, hi = M;
    while (lo < hi) {
      const int64_t m = (lo + hi + 1) >> 1;
      if (io[m] - io[g] <= cap) lo = m; else hi = m - 1;
    }
    P.m.spass[1 + 2 * c] = g;
    P.m.spass[2 + 2 * c] = lo;
    ++c;
    g = lo;
  }
  if (g < M) set_status(P.status, TDC_EUNSUPPORTED);  // cannot happen (see above)
  P.m.spass[0] = c;
}

// ---------------------------------------------------------------------------
// Digit images
// ---------------------------------------------------------------------------
// A level sum I (an integer count of 2^-58 units) times 2^adj as a double: the scale enters
// the exponent field of double(I) by an integer addition, no FP64 multiply, while the
// result stays a normal number (else two power-of-two factors).
__device__ __forceinline__ int col_adj(const GemmSeg& sg, int j) {
  return j < sg.K ? (sg.cexp ? sg.cexp[j] : 0) + (sg.oexp ? sg.oexp[j] : 0) : 0;
}
__device__ __forceinline__ double level_value(long long I, int adj) {
  if (I == 0) return 0.0;
  const long long b = __double_as_longlong(__ll2double_rn(I));
  const int f = (int)((b >> 52) & 0x7ff) + adj - 58;
  if (f >= 1 && f <= 2046) return __longlong_as_double(b + ((long long)(adj - 58) << 52));
  return scale2(__longlong_as_double(b - (58ll << 52)), adj);
}

__global__ void __launch_bounds__(256) k_split_a(const GemmSeg* segs, int nseg, const int64_t* dnseg, int S,
                                                 __nv_bfloat16* img, int* status) {
  if (dnseg) nseg = (int)*dnseg;
  const int64_t total = segs[nseg].it_a;
  const int tid = threadIdx.x;
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int si = find_seg(segs, nseg, w, 0);
    const GemmSeg& sg = segs[si];
    const int64_t local = w - sg.it_a;
    const int KB = (int)cdiv(sg.kk, BK);
    const int rt = (int)(local / KB), kb = (int)(local % KB);
    const int64_t toff = sg.a_img + ((int64_t)rt * KB + kb) * S * kATileElems;
    if (toff < 0 || toff + (int64_t)S * kATileElems > segs[nseg].a_img) {  // never write outside the images
      if (threadIdx.x == 0) set_status(status, TDC_EUNSUPPORTED);
      continue;
    }
    __nv_bfloat16* tile = img + toff;
    for (int u = tid; u < BM * (BK / 8); u += blockDim.x) {
      const int r = u % BM, kg = u / BM;  // BK/8 groups of 8 consecutive k
      const int row = rt * BM + r;
      uint32_t dig[8][kMaxS];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int q = kb * BK + kg * 8 + i;
        double x = 0.0;
        if (q < sg.kk && row < sg.rows) {
          const int p = sg.plist ? sg.plist[q] : q;
          const int col = sg.acol ? sg.acol[p] : p;
          x = sg.A[(int64_t)row * sg.ars + (int64_t)col * sg.lda];
          if (sg.aexp) x *= pow2c(-sg.aexp);
        }
        digits_bf16(x, S, dig[i]);
      }
      const int off = core_off(r, kg * 8);
#pragma unroll
      for (int s = 0; s < kMaxS; ++s) {
        if (s >= S) break;
        uint32_t v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = dig[i][s];
        *reinterpret_cast<uint4*>(tile + (int64_t)s * kATileElems + off) = pack8(v);
      }
    }
  }
}

// Two B tiles per block iteration: threads 0-127 and 128-255 each take one
// (64 columns x BK/8 groups of 8 poles).
static_assert(BN * (BK / 8) == 128, "k_split_b maps 128 threads onto one B tile");
__global__ void __launch_bounds__(256) k_split_b(const GemmSeg* segs, int nseg, const int64_t* dnseg, int S,
                                                 __nv_bfloat16* img, int* status) {
  if (dnseg) nseg = (int)*dnseg;
  const int64_t total = segs[nseg].it_b;
  const int tid = threadIdx.x & 127;
  for (int64_t w = 2 * (int64_t)blockIdx.x + (threadIdx.x >> 7); w < total; w += 2 * (int64_t)gridDim.x) {
    const int si = find_seg(segs, nseg, w, 1);
    const GemmSeg& sg = segs[si];
    const int64_t local = w - sg.it_b;
    const int KB = (int)cdiv(sg.kk, BK);
    const int ct = (int)(local / KB), kb = (int)(local % KB);
    const int64_t toff = sg.b_img + ((int64_t)ct * KB + kb) * S * kBTileElems;
    if (toff < 0 || toff + (int64_t)S * kBTileElems > segs[nseg].a_img) {  // never write outside the images
      if ((threadIdx.x & 127) == 0) set_status(status, TDC_EUNSUPPORTED);
      continue;
    }
    __nv_bfloat16* tile = img + toff;
    const int j = tid % BN, kg = tid / BN;  // 64 columns x BK/8 groups of 8 poles
    const int jj = ct * BN + j;
    double dorg = 0.0, tj = 1.0, sj = 0.0;
    if (jj < sg.K) {
      if (sg.Bd || sg.tgen) {
        sj = sg.cexp ? pow2c(-sg.cexp[jj]) : 1.0;
      } else {
        const int jr = sg.bcol ? sg.bcol[jj] : jj;
        dorg = sg.D[sg.org[jr]];
        tj = sg.tau[jr];
        sj = sg.scol[jr];
      }
    }
    uint32_t dig[8][kMaxS];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = kb * BK + kg * 8 + i;
      double u = 0.0;
      if (q < sg.kk && q >= sg.bq0 && jj < sg.K) {
        const int p = sg.plist ? sg.plist[q] : q;
        if (sg.Bd) u = sg.Bd[p + (int64_t)jj * sg.ldb] * sj;
        else if (sg.tgen) u = struct_entry(sg, p, jj) * sj;
        else u = (sg.zhat[p] * sj) * rcp_nr((sg.D[p] - dorg) - tj);
      }
      digits_bf16(u, S, dig[i]);
    }
    const int off = core_off(j, kg * 8);
#pragma unroll
    for (int s = 0; s < kMaxS; ++s) {
      if (s >= S) break;
      uint32_t v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = dig[i][s];
      *reinterpret_cast<uint4*>(tile + (int64_t)s * kBTileElems + off) = pack8(v);
    }
  }
}

// ---------------------------------------------------------------------------
// The tensor-core GEMM over the digit images: one CTA per SM, persistent over
// the tile list, three roles in separate warps so that no role waits on another
// one's bookkeeping:
//   warp 17 (one thread) producer: bulk copies of one k-step (S A-slices + S
//                        B-slices, contiguous) into a kStages ring, completion
//                        on full[st]; a stage is reused once empty[st] fires;
//   warp 16 (one thread) MMA issuer: waits full[st], issues the S wide MMAs of the
//                        step, commits them to empty[st]; after a tile's last
//                        step (with chunked drains: after every ck steps)
//                        commits to tfull, and reuses the accumulators only
//                        after the epilogue has released them (tempty);
//   warps 0-15           epilogue: warp w takes TMEM lane quarter w mod 4 (the
//                        lanes a warp may read) and column quarter w / 4 of the
//                        tile, combines the S level accumulators, releases
//                        them, then stores (four warps per lane quarter cut the
//                        epilogue, which sets the time of shallow tiles).
// The producer runs ahead into the next tile while the epilogue drains, and S is
// a compile-time constant so that the issue loop is straight-line code (every
// descriptor a constant offset of the stage base).  Every wait is bounded; a
// role that gives up raises s_fail, which the other roles poll, and the CTA
// reports TDC_ETIMEOUT after its copies and MMAs in flight have landed.
// ---------------------------------------------------------------------------
namespace {
constexpr int kEpiWarps = 16, kMmaWarp = 16, kLoadWarp = 17, kSplitThreads = 576;
constexpr int kEpiCols = BN / (kEpiWarps / 4);  // columns per epilogue warp
static_assert(kEpiCols == 16, "epilogue column split: one 16-column TMEM load per level");

// Level m < 5 of one hand-off (16 columns, exact integers held in FP32) into the
// 64-bit running sums: hi += P_m 2^sh with sh = 8 (4 - m).  An FP32 integer v with
// |v| < 2^22 becomes an integer without the conversion unit (16 per clock per SM):
// v + 1.5 2^23 lies in [2^23, 2^24), where the float's ulp is 1, so its bit pattern
// is 0x4B400000 + v exactly; bias collects the 0x4B400000 2^sh this adds, removed
// once per tile.  A thread holding a larger value (a level sum near the 2^24 limit)
// forms the same 0x4B400000 + v with cvt instead.  The sums are kept modulo 2^64
// (unsigned) and are exact once the bias is removed.
__device__ __forceinline__ void add_level_int(const uint32_t (&r)[16], int sh, unsigned long long (&hi)[16],
                                              unsigned long long& bias, float& gmax) {
  float mx = 0.0f;
#pragma unroll
  for (int i = 0; i < 16; ++i) mx = fmaxf(mx, fabsf(__uint_as_float(r[i])));
  gmax = fmaxf(gmax, mx);
  if (mx < 4194304.0f) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      hi[i] += (unsigned long long)__float_as_uint(__uint_as_float(r[i]) + 12582912.0f) << sh;
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      hi[i] += (unsigned long long)((long long)__float2int_rn(__uint_as_float(r[i])) + 0x4B400000ll) << sh;
  }
  bias += 0x4B400000ull << sh;
}

// One hand-off of the S level accumulators (this warp's 32 TMEM lanes, 16 columns at
// ta): hi += sum_{m<5} P_m 2^(8(4-m)), lo += P_6 2^-8 then += P_5.  One level at a
// time (16 registers; sixteen epilogue warps hide the load latency).  Summing these
// per hand-off gives the same integers as the per-tile Horner combination, and lo
// the same FP32 roundings.
template <int S>
__device__ __forceinline__ void drain_levels(uint32_t ta, unsigned long long (&hi)[16], float (&lo)[16],
                                             unsigned long long& bias, float& gmax) {
  uint32_t a[16];
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    if (m < S) {
      umma::tmem_ld16_nowait(ta + (uint32_t)(m * BN), a);
      umma::tmem_wait_ld(a);
      add_level_int(a, 8 * (4 - m), hi, bias, gmax);
    }
  }
#pragma unroll
  for (int m = 6; m >= 5; --m) {
    if (m < S) {
      umma::tmem_ld16_nowait(ta + (uint32_t)(m * BN), a);
      umma::tmem_wait_ld(a);
#pragma unroll
      for (int i = 0; i < 16; ++i) lo[i] += m == 6 ? __uint_as_float(a[i]) * 0.00390625f : __uint_as_float(a[i]);
    }
  }
}

// Bound of the waits on the give-up path (copies and MMAs already issued, which
// complete in microseconds): independent of the caller's spin budget, so that a
// small budget can only make the roles give up, never leave a copy or an MMA in
// flight when the CTA releases its TMEM and exits.
constexpr long long kDrainBudget = 1ll << 24;

__device__ __forceinline__ bool wait_or_fail(uint64_t* bar, uint32_t parity, long long budget,
                                             volatile int* fail) {
  for (long long i = 0; i < budget; ++i) {
    if (umma::mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && *fail) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_u32(bar)) : "memory");
}

struct TileRef {
  const GemmSeg* sg;
  int rt, ct, KB;
};

// tile w of the level: tiles in groups of kGroupRows row tiles, column tile by
// column tile, so that the CTAs running together share A row tiles and B column
// tiles in L2
__device__ __forceinline__ TileRef tile_ref(const GemmSeg* segs, int nseg, int64_t w) {
  TileRef t;
  t.sg = &segs[find_seg(segs, nseg, w, 2)];
  const int64_t local = w - t.sg->it_t;
  const int CT = (int)cdiv(t.sg->K, BN);
  const int RT = (int)cdiv(t.sg->rows, BM);
  t.KB = (int)cdiv(t.sg->kk, BK);
  const int grp = (int)(local / ((int64_t)kGroupRows * CT));
  const int within = (int)(local % ((int64_t)kGroupRows * CT));
  const int gr = min(kGroupRows, RT - grp * kGroupRows);
  t.rt = grp * kGroupRows + within % gr;
  t.ct = within / gr;
  return t;
}
}  // namespace

// kChunk: the accumulators are drained into the epilogue's running sums every ck
// k-steps of a tile (the MMA warp waits for each drain), so that every level sum
// covers at most 16 ck terms; without it they cover the tile's whole reduction.
template <int S, bool kChunk>
__global__ void __launch_bounds__(kSplitThreads, 1) k_gemm_split(const GemmSeg* segs, int nseg, const int64_t* dnseg,
                                                                 const __nv_bfloat16* img, int* status,
                                                                 long long budget, int ck, unsigned int* lvl_max) {
  if (dnseg) nseg = (int)*dnseg;
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr uint32_t a_bytes = S * kATileElems * 2, b_bytes = S * kBTileElems * 2;
  constexpr uint32_t stage_bytes = a_bytes + b_bytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t total = segs[nseg].it_t;
  if ((int64_t)blockIdx.x >= total) return;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * stage_bytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 1;
  uint64_t* done = tempty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int s_fail;
  volatile int* vfail = &s_fail;
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      umma::mbar_init(&full[i], 1);
      umma::mbar_init(&empty[i], 1);
    }
    umma::mbar_init(tfull, 1);
    umma::mbar_init(tempty, kEpiWarps);
    umma::mbar_init(done, 1);
    umma::fence_mbar_init();
    s_fail = 0;
  }
  if (warp == 0) {
    umma::tmem_alloc(tmem_slot, 512);
    umma::tmem_relinquish();
  }
  umma::tc_fence_before();
  __syncthreads();
  umma::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = umma::smem_u32(smem);

  if (warp == kLoadWarp) {
    if (lane == 0) {
      long long g = 0;  // k-steps loaded by this CTA (stage g % kStages, use g / kStages)
      bool ok = true;
      const int64_t img_end = segs[nseg].a_img;  // the list's images end here (the terminator)
      for (int64_t w = blockIdx.x; w < total && ok; w += gridDim.x) {
        const TileRef t = tile_ref(segs, nseg, w);
        const int akt = t.sg->a_kt > 0 ? t.sg->a_kt : t.KB;  // k-tiles per row tile of the A image
        const int64_t a0 = t.sg->a_img + (int64_t)t.rt * akt * S * kATileElems;
        const int64_t b0 = t.sg->b_img + (int64_t)t.ct * t.KB * S * kBTileElems;
        if (a0 < 0 || b0 < 0 || a0 + (int64_t)t.KB * S * kATileElems > img_end ||
            b0 + (int64_t)t.KB * S * kBTileElems > img_end) {  // cannot happen for a built list; never read
          set_status(status, TDC_EUNSUPPORTED);                 // outside the images
          ok = false;
          break;
        }
        const uint8_t* ai = reinterpret_cast<const uint8_t*>(img + a0);
        const uint8_t* bi = reinterpret_cast<const uint8_t*>(img + b0);
        for (int kb = 0; kb < t.KB; ++kb, ++g) {
          const int st = (int)(g % kStages);
          if (g >= kStages && !wait_or_fail(&empty[st], (uint32_t)(((g - kStages) / kStages) & 1), budget, vfail)) {
            ok = false;
            break;
          }
          uint8_t* dst = smem + st * stage_bytes;
          umma::mbar_arrive_expect_tx(&full[st], stage_bytes);
          umma::bulk_g2s(dst, ai + (int64_t)kb * a_bytes, a_bytes, &full[st]);
          umma::bulk_g2s(dst + a_bytes, bi + (int64_t)kb * b_bytes, b_bytes, &full[st]);
        }
      }
      if (!ok) *vfail = 1;
      // copies issued but not consumed (only after a failure) land before the CTA exits
      for (long long q = g > kStages ? g - kStages : 0; q < g; ++q)
        umma::mbar_wait(&full[q % kStages], (uint32_t)((q / kStages) & 1), kDrainBudget);
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      long long g = 0;
      int it = 0;
      bool ok = true, issued = false;
      // shared-memory descriptor of slice 0 of stage 0 (K-major core matrices:
      // 128 bytes between the two core matrices along K, 256 between 8-row groups);
      // the start-address field (bits 0-13, address / 16) absorbs every offset below
      // without carrying, as all of shared memory lies below 2^18 bytes
      const uint64_t desc0 = umma::sdesc(sbase, 128, BK * 16);
      for (int64_t w = blockIdx.x; w < total && ok; w += gridDim.x, ++it) {
        const TileRef t = tile_ref(segs, nseg, w);
        // one accumulator hand-off per chunk of ck k-steps (kChunk), else per tile
        const int nch = kChunk && t.KB > 0 ? (t.KB + ck - 1) / ck : 1;
        int kb0 = 0;
        for (int c = 0; c < nch; ++c) {
          if (kChunk && c > 0) ++it;
          if (it > 0 && !wait_or_fail(tempty, (uint32_t)((it - 1) & 1), budget, vfail)) {
            ok = false;
            break;
          }
          umma::tc_fence_after();
          const int kb1 = kChunk ? min(t.KB, kb0 + ck) : t.KB;
          for (int kb = kb0; kb < kb1; ++kb, ++g) {
            const int st = (int)(g % kStages);
            if (!wait_or_fail(&full[st], (uint32_t)((g / kStages) & 1), budget, vfail)) {
              ok = false;
              break;
            }
            umma::tc_fence_after();
            // The S B-slices are stacked along N in shared memory and level m's
            // accumulator starts at TMEM column m*BN, so A_s against the stacked slices
            // B_0..B_{S-1-s} (N = BN (S - s)) drops every product A_s B_t into level
            // s+t: one wide MMA per A-slice (split at N = 256) instead of one per pair.
            // Every operand descriptor is the stage-0 descriptor plus a constant, so
            // the issue loop is a handful of integer adds per MMA.
            const uint64_t dst = desc0 + (uint64_t)((st * stage_bytes) >> 4);
#pragma unroll
            for (int s = 0; s < S; ++s) {
              const uint64_t ad = dst + (uint64_t)((s * kATileElems * 2) >> 4);
#pragma unroll
              for (int off = 0; off < BN * (S - s); off += 256) {
                const int nn = BN * (S - s) - off < 256 ? BN * (S - s) - off : 256;
                const uint64_t bd = dst + (uint64_t)((a_bytes + (off / BN) * kBTileElems * 2) >> 4);
                umma::mma_bf16(tmem + s * BN + off, ad, bd, umma::idesc_bf16(BM, nn), (kb > kb0 || s > 0) ? 1u : 0u);
              }
            }
            umma::mma_commit(&empty[st]);
            issued = true;
          }
          if (!ok) break;
          if (kb1 > kb0) umma::mma_commit(tfull);
          else mbar_arrive(tfull);
          kb0 = kb1;
        }
      }
      if (!ok) *vfail = 1;
      // every MMA issued has completed before the accumulators are released
      if (issued) {
        umma::mma_commit(done);
        umma::mbar_wait(done, 0, kDrainBudget);
      }
    }
  } else {
    // epilogue: C = 2^-16 sum_m 2^-8m P_m with P_m the exact FP32 integer sums of
    // level m.  The first five levels combine exactly in a 64-bit integer
    // hi = (((P0 2^8 + P1) 2^8 + P2) 2^8 + P3) 2^8 + P4, the last two in FP32 as
    // lo = P5 + 2^-8 P6 (rounding near 2^-60 absolute), C = 2^-48 hi + 2^-56 lo.
    // The FP64 pipe retires 2 operations per clock per SM, which shallow tiles feel:
    // where |hi| < 2^52 (merge products: unit rows times unit columns give
    // |hi| <= 2^48) C is formed as I = 2^10 hi + round(4 lo) (error <= 2^-59),
    // one conversion to double, and the factor 2^-58 applied to the exponent
    // field (I != 0 gives |I| >= 1, so the result stays normal); otherwise, e.g.
    // for the adjoint's column-scaled products, in FP64 as written.
    int it = 0;
    float gmax = 0.0f;  // largest |level sum| (levels 0-4) this thread drained
    const int quarter = warp & 3, c0 = (warp >> 2) * kEpiCols;
    const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x, ++it) {
      const TileRef t = tile_ref(segs, nseg, w);
      if constexpr (kChunk) {
        // the same combination, accumulated over the tile's chunks: level m of a
        // chunk adds P_m 2^(8(4-m)) to hi (m < 5, exact) or its share to lo
        const int nch = t.KB > 0 ? (t.KB + ck - 1) / ck : 1;
        unsigned long long hu[kEpiCols], bias = 0;
        float lo[kEpiCols];
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) {
          hu[i] = 0;
          lo[i] = 0.0f;
        }
        bool okc = true;
        for (int c = 0; c < nch; ++c) {
          if (c > 0) ++it;
          okc = __all_sync(0xffffffffu, wait_or_fail(tfull, (uint32_t)(it & 1), budget, vfail));
          if (!okc) break;
          umma::tc_fence_after();
          if (t.KB > 0) drain_levels<S>(tl + (uint32_t)c0, hu, lo, bias, gmax);
          umma::tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty);
        }
        if (!okc) {
          if (lane == 0) *vfail = 1;
          break;
        }
        long long hi[kEpiCols];
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) hi[i] = (long long)(hu[i] - bias);
        double val[kEpiCols];
        bool fits = true;
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) fits = fits && hi[i] < (1ll << 52) && hi[i] > -(1ll << 52);
        // the column's scale (2^cexp_j 2^oexp_j) goes into the exponent field of the value
        if (__all_sync(0xffffffffu, fits)) {
#pragma unroll
          for (int i = 0; i < kEpiCols; ++i)
            val[i] = level_value(hi[i] * 1024 + (long long)__float2int_rn(4.0f * lo[i]), col_adj(*t.sg, t.ct * BN + c0 + i));
        } else {
#pragma unroll
          for (int i = 0; i < kEpiCols; ++i)
            val[i] = scale2(fma((double)lo[i], 0x1p-56, __ll2double_rn(hi[i]) * 0x1p-48), col_adj(*t.sg, t.ct * BN + c0 + i));
        }
        const GemmSeg& sg = *t.sg;
        const int row = t.rt * BM + quarter * 32 + lane;
        if (row < sg.rows) {
#pragma unroll
          for (int i = 0; i < kEpiCols; ++i) {
            const int j = t.ct * BN + c0 + i;
            if (j < sg.K) {
              const int pos = sg.cpos ? sg.cpos[j] : j;
              double* cp = sg.C + row + (int64_t)pos * sg.ldc;
              if (sg.acc) *cp += val[i]; else *cp = val[i];
            }
          }
        }
        continue;
      }
      const bool okw = __all_sync(0xffffffffu, wait_or_fail(tfull, (uint32_t)(it & 1), budget, vfail));
      if (!okw) {
        if (lane == 0) *vfail = 1;
        break;
      }
      umma::tc_fence_after();
      double val[kEpiCols];
      {
        unsigned long long hu[kEpiCols], bias = 0;
        float lo[kEpiCols];
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) {
          hu[i] = 0;
          lo[i] = 0.0f;
        }
        if (t.KB > 0) drain_levels<S>(tl + (uint32_t)c0, hu, lo, bias, gmax);
        long long hi[kEpiCols];
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) hi[i] = (long long)(hu[i] - bias);
        bool fits = true;
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) fits = fits && hi[i] < (1ll << 52) && hi[i] > -(1ll << 52);
        // the column's scale (2^cexp_j 2^oexp_j) goes into the exponent field of the value
        if (__all_sync(0xffffffffu, fits)) {
#pragma unroll
          for (int i = 0; i < kEpiCols; ++i)
            val[i] = level_value(hi[i] * 1024 + (long long)__float2int_rn(4.0f * lo[i]), col_adj(*t.sg, t.ct * BN + c0 + i));
        } else {
#pragma unroll
          for (int i = 0; i < kEpiCols; ++i)
            val[i] = scale2(fma((double)lo[i], 0x1p-56, __ll2double_rn(hi[i]) * 0x1p-48), col_adj(*t.sg, t.ct * BN + c0 + i));
        }
      }
      umma::tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty);
      const GemmSeg& sg = *t.sg;
      const int row = t.rt * BM + quarter * 32 + lane;
      if (row < sg.rows) {
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) {
          const int j = t.ct * BN + c0 + i;
          if (j < sg.K) {
            const int pos = sg.cpos ? sg.cpos[j] : j;
            double* cp = sg.C + row + (int64_t)pos * sg.ldc;
            if (sg.acc) *cp += val[i]; else *cp = val[i];
          }
        }
      }
    }
    // the level sums' margin: statistics, and a warning once a hand-off reached 2^23
    const float wmax = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(gmax)));
    if (lane == 0) {
      if (lvl_max) atomicMax(lvl_max, __float_as_uint(wmax));
      if (wmax >= 8388608.0f) set_warning(status, kWarnSplitLevel);
    }
  }
  umma::tc_fence_before();
  __syncthreads();
  if (tid == 0 && s_fail) set_status(status, TDC_ETIMEOUT);
  if (warp == 0) umma::tmem_dealloc(tmem, 512);
}

static cudaError_t launch_split_digits(const GemmSeg* segs, int nseg, const int64_t* dnseg, int S, int* status,
                                       __nv_bfloat16* img, cudaStream_t s) {
  k_split_a<<<152 * 8, 256, 0, s>>>(segs, nseg, dnseg, S, img, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_split_b<<<152 * 8, 256, 0, s>>>(segs, nseg, dnseg, S, img, status);
  return cudaGetLastError();
}

template <int S, bool kChunk>
static cudaError_t launch_split_mma_s(const GemmSeg* segs, int nseg, const int64_t* dnseg, int* status,
                                      long long budget, const __nv_bfloat16* img, int sms, int ck,
                                      unsigned int* lvl_max, cudaStream_t s) {
  const int smem = kStages * S * (kATileElems + kBTileElems) * 2 + 128;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_split<S, kChunk>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_gemm_split<S, kChunk><<<sms, kSplitThreads, smem, s>>>(segs, nseg, dnseg, img, status, budget, ck, lvl_max);
  return cudaGetLastError();
}

// ck > 0: drain the accumulators every ck k-steps
static cudaError_t launch_split_mma(const GemmSeg* segs, int nseg, const int64_t* dnseg, int S, int* status,
                                    long long budget, const __nv_bfloat16* img, int ck, unsigned int* lvl_max,
                                    cudaStream_t s) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (ck > 0) {
    switch (S) {
      case 3: return launch_split_mma_s<3, true>(segs, nseg, dnseg, status, budget, img, sms, ck, lvl_max, s);
      case 4: return launch_split_mma_s<4, true>(segs, nseg, dnseg, status, budget, img, sms, ck, lvl_max, s);
      case 5: return launch_split_mma_s<5, true>(segs, nseg, dnseg, status, budget, img, sms, ck, lvl_max, s);
      case 6: return launch_split_mma_s<6, true>(segs, nseg, dnseg, status, budget, img, sms, ck, lvl_max, s);
      case 7: return launch_split_mma_s<7, true>(segs, nseg, dnseg, status, budget, img, sms, ck, lvl_max, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (S) {
    case 3: return launch_split_mma_s<3, false>(segs, nseg, dnseg, status, budget, img, sms, 0, lvl_max, s);
    case 4: return launch_split_mma_s<4, false>(segs, nseg, dnseg, status, budget, img, sms, 0, lvl_max, s);
    case 5: return launch_split_mma_s<5, false>(segs, nseg, dnseg, status, budget, img, sms, 0, lvl_max, s);
    case 6: return launch_split_mma_s<6, false>(segs, nseg, dnseg, status, budget, img, sms, 0, lvl_max, s);
    case 7: return launch_split_mma_s<7, false>(segs, nseg, dnseg, status, budget, img, sms, 0, lvl_max, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_split_pack(const Plan& P, const LevelLaunch& L, int max_pass, cudaStream_t s) {
  if (P.split_min_K <= 0 || P.segs == nullptr || L.merges == 0) return cudaSuccess;
  k_split_pack<<<1, 1024, 0, s>>>(P, L.level, L.merges, max_pass);
  return cudaGetLastError();
}

// Merges [g0, g1) of the level, or (pass >= 0) the device-packed pass of that number.
cudaError_t launch_gemm_split(const Plan& P, const LevelLaunch& L, int64_t g0, int64_t g1, int pass, cudaStream_t s,
                              cudaEvent_t mid) {
  if (P.split_min_K <= 0 || P.segs == nullptr || g1 <= g0) return cudaSuccess;
  k_split_segs<<<1, 1024, 0, s>>>(P, L.level, g0, g1, pass);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nseg = (int)(2 * (g1 - g0));  // bound; the kernels read the compacted count
  const int64_t* dn = P.m.sseg;
  e = launch_split_digits(P.segs, nseg, dn, P.split_slices, P.status, P.img, s);
  if (e != cudaSuccess) return e;
  if (mid) cudaEventRecord(mid, s);
  return launch_split_mma(P.segs, nseg, dn, P.split_slices, P.status, P.spin_budget, P.img, P.split_chunk_steps,
                          P.stats ? &P.stats->split_level_max : nullptr, s);
}

// A segment list whose count lives on the device (*dcount; nseg_bound bounds it):
// digit images, then the products; `mid` (optional) is recorded between the two.
cudaError_t launch_split_list(const GemmSeg* segs, int nseg_bound, const int64_t* dcount, int S, int* status,
                              long long spin_budget, __nv_bfloat16* img, int chunk_steps, unsigned int* lvl_max,
                              cudaStream_t s, cudaEvent_t mid) {
  if (nseg_bound <= 0) return cudaSuccess;
  cudaError_t e = launch_split_digits(segs, nseg_bound, dcount, S, status, img, s);
  if (e != cudaSuccess) return e;
  if (mid) cudaEventRecord(mid, s);
  return launch_split_mma(segs, nseg_bound, dcount, S, status, spin_budget, img, chunk_steps, lvl_max, s);
}

cudaError_t launch_seg_split(const GemmSeg* segs_dev, int nseg, int S, int* status, long long spin_budget,
                             __nv_bfloat16* img, int chunk_steps, cudaStream_t s) {
  cudaError_t e = launch_split_digits(segs_dev, nseg, nullptr, S, status, img, s);
  if (e != cudaSuccess) return e;
  return launch_split_mma(segs_dev, nseg, nullptr, S, status, spin_budget, img, chunk_steps, nullptr, s);
}

}  // namespace tdc
