// tdc_gemm_dense.cu -- eigenvector update of a merge, C = Qtilde * Qhat (Eq. (evect)),
// in FP64, with Qhat generated from its generators inside the kernel
// (Eq. (Q_Cauchy), Eq. (d-lambda)) so that it never exists in memory:
//   Qhat_qj = zhat_q s_j / ((D_q - D_org(j)) - tau_j).
// The rows of the node split into the top child's rows, which only see the
// non-deflated columns with support there (S_top), and the bottom child's
// rows (S_bot); each part is a GEMM over its own list of poles.  Output
// column j goes to the node's eigenvector column posr[j].
//
// One CTA computes a 128 x 64 tile with 256 threads (8 x 4 outputs each) on
// the FP64 pipe -- 32 x 32 (2 x 2 each) for merges of order <= 128, whose halves
// have at most 64 rows; per 16-deep k-step it stages the Qtilde tile in shared
// memory and generates the 16 x 64 (16 x 32) Qhat tile there (8 FP64 operations
// per entry, amortised over the tile's rows).  Tiles of all merges of the level
// form one work list (prefix in MergeInfo::tiles) that a fixed grid walks.
// Merges of order <= 32 take a warp each instead (k_gemm_tiny).
#include <float.h>

#include "tdc_common.cuh"

namespace tdc {

namespace {
constexpr int BM = kDenseBM, BN = kDenseBN, BK = kDenseBK;
constexpr int kThreads = 256;

__device__ __forceinline__ int lower_bound_i(const int* a, int n, int x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// List positions [qlo, qhi) of the poles within one structured tile (size m) of
// the tile holding output column j0 (pole indices in [(J-1) m, (J+2) m)).
__device__ __forceinline__ void near_range(const int* list, int nl, int j0, int m, int K, int& qlo, int& qhi) {
  const int J = j0 / m;
  const int plo = J >= 1 ? (J - 1) * m : 0;
  const int phi = min(K, (J + 2) * m);
  if (list) {
    qlo = lower_bound_i(list, nl, plo);
    qhi = lower_bound_i(list, nl, phi);
  } else {
    qlo = min(plo, nl);
    qhi = min(phi, nl);
  }
}

// Per-column and per-pole values of the tile being computed.
struct DenseCols {
  double Do[BN], Tau[BN], S[BN];
  int Pos[BN];
  int Col[BK];
  double Dq[BK], Zq[BK];
};

// One TBM x TBN output tile (tile number `local` of merge g) on 256 threads,
// TM x TN outputs each.  kRowFast puts consecutive threads on consecutive row
// groups, so that a warp's stores of one column are contiguous.
template <int TBM, int TBN, bool kRowFast>
__device__ __forceinline__ void dense_tile(const Plan& P, const Node& nd, int64_t g, int64_t local, double* As,
                                           double* Us, DenseCols& sc) {
  constexpr int TM = TBM / 16, TN = TBN / 16;
  static_assert(TBM % 16 == 0 && TBN % 16 == 0 && TBN <= BN && TBM * BK <= BM * BK, "tile shape");
  const int tid = threadIdx.x;
  const int ty = kRowFast ? (tid & 15) : (tid >> 4);  // row group: TM rows
  const int tx = kRowFast ? (tid >> 4) : (tid & 15);  // column group: TN columns
  const int n = (int)(nd.hi - nd.lo), n1 = (int)(nd.mid - nd.lo);
  const int K = P.m.K[g];
  const int ct = (K + TBN - 1) / TBN;
  const int rtt = (int)(local / ct), ctile = (int)(local % ct);
  const int rt0 = (n1 + TBM - 1) / TBM;
  int r0, rend, nl;
  const int* list;
  if (rtt < rt0) { r0 = rtt * TBM; rend = n1; list = P.v.tlist + nd.v0; nl = P.m.ntop[g]; }
  else { r0 = n1 + (rtt - rt0) * TBM; rend = n; list = P.v.blist + nd.v0; nl = P.m.nbot[g]; }
  const int j0 = ctile * TBN;
  const double* Dk = P.v.Dk + nd.v0;
  // structured merge: only the poles within one tile of the output columns here
  // (TBN divides the structured tile size, a multiple of 64)
  int qlo = 0, qhi = nl;
  const bool structured = P.struct_min_K > 0 && K >= P.struct_min_K;
  if (structured) {
    near_range(list, nl, j0, P.struct_m, K, qlo, qhi);
    if (P.stats && tid == 0)
      atomicAdd(&P.stats->struct_flops, 2ull * (unsigned long long)min(TBM, rend - r0) *
                                             (unsigned long long)(qhi - qlo) * (unsigned long long)min(TBN, K - j0));
  }
  __syncthreads();
  if (tid < TBN) {
    const int j = j0 + tid;
    if (j < K) {
      sc.Do[tid] = Dk[P.v.org[nd.v0 + j]];
      sc.Tau[tid] = P.v.tau[nd.v0 + j];
      sc.S[tid] = P.v.scol[nd.v0 + j];
      sc.Pos[tid] = P.v.posr[nd.v0 + j];
    } else {
      sc.Do[tid] = 0.0; sc.Tau[tid] = 1.0; sc.S[tid] = 0.0; sc.Pos[tid] = -1;
    }
  }
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[i][c] = 0.0;
  for (int k0 = qlo; k0 < qhi; k0 += BK) {
    __syncthreads();
    if (tid < BK) {
      const int k = k0 + tid;
      if (k < qhi) {
        const int q = list[k];
        sc.Col[tid] = P.v.kept[nd.v0 + q];
        sc.Dq[tid] = Dk[q];
        sc.Zq[tid] = P.v.zhat[nd.v0 + q];
      } else {
        sc.Col[tid] = -1; sc.Dq[tid] = 0.0; sc.Zq[tid] = 0.0;
      }
    }
    __syncthreads();
    // Qtilde tile: BK columns x TBM rows (each column contiguous)
#pragma unroll
    for (int e = 0; e < (BK * TBM) / kThreads; ++e) {
      const int idx = tid + e * kThreads;
      const int k = idx / TBM, r = idx % TBM;
      const int col = sc.Col[k];
      const int row = r0 + r;
      As[k * TBM + r] = (col >= 0 && row < rend) ? nd.src[row + (int64_t)col * nd.lds] : 0.0;
    }
    // Qhat tile generated from the generators
#pragma unroll
    for (int e = 0; e < (BK * TBN) / kThreads; ++e) {
      const int idx = tid + e * kThreads;
      const int k = idx / TBN, c = idx % TBN;
      const double del = (sc.Dq[k] - sc.Do[c]) - sc.Tau[c];
      Us[k * TBN + c] = (sc.Zq[k] * sc.S[c]) * rcp_nr(del);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double av[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) av[i] = As[k * TBM + ty * TM + i];
#pragma unroll
      for (int c = 0; c < TN; ++c) bv[c] = Us[k * TBN + tx * TN + c];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[i][c] = fma(av[i], bv[c], acc[i][c]);
    }
  }
  // epilogue: write to the node's output columns
#pragma unroll
  for (int c = 0; c < TN; ++c) {
    const int pos = sc.Pos[tx * TN + c];
    if (pos < 0 || pos >= n) continue;
    double* out = nd.dst + (int64_t)pos * nd.ldd;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int row = r0 + ty * TM + i;
      if (row < rend) out[row] = acc[i][c];
    }
  }
}
}  // namespace

__global__ void __launch_bounds__(kThreads, 2) k_gemm_dense(Plan P, int level, int64_t M) {
  __shared__ double As[BK * BM];
  __shared__ double Us[BK * BN];
  __shared__ DenseCols sc;
  const int64_t total = P.m.tiles[M];
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    // merge owning tile w
    int64_t a = 0, b = M - 1;
    while (a < b) {
      int64_t m = (a + b + 1) >> 1;
      if (P.m.tiles[m] <= w) a = m; else b = m - 1;
    }
    const int64_t g = a;
    const Node nd = make_node(P, level, g);
    int bm, bn;
    dense_tile_dims(nd.hi - nd.lo, bm, bn);
    if (bm == kDenseSmallBM)
      dense_tile<kDenseSmallBM, kDenseSmallBN, true>(P, nd, g, w - P.m.tiles[g], As, Us, sc);
    else
      dense_tile<BM, BN, false>(P, nd, g, w - P.m.tiles[g], As, Us, sc);
  }
}

// Merges of order <= kTinyN: a warp per merge, lane c computing output column c
// (K <= 32) for every row of a half, its Qhat entries generated in registers and
// the half's Qtilde block (at most 16 x 16) staged in shared memory.  Same
// products in the same order as the tiled kernel; no tile search, no block
// barriers.
constexpr int kTinyWarps = 4, kTinyRows = kTinyN / 2;
__global__ void __launch_bounds__(32 * kTinyWarps) k_gemm_tiny(Plan P, int level, int64_t M) {
  __shared__ double sA[kTinyWarps][kTinyRows * kTinyRows];
  __shared__ double sDq[kTinyWarps][kTinyRows], sZq[kTinyWarps][kTinyRows];
  __shared__ int sCol[kTinyWarps][kTinyRows];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * kTinyWarps + wid;
  if (g >= M) return;
  const int K = P.m.K[g];
  const Node nd = make_node(P, level, g);
  const int n = (int)(nd.hi - nd.lo), n1 = (int)(nd.mid - nd.lo);
  if (!tiny_merge(n, K, P.m.ntop[g], P.m.nbot[g], P.split_min_K, P.struct_min_K)) return;
  const double* Dk = P.v.Dk + nd.v0;
  double Do = 0.0, Tau = 1.0, S = 0.0;
  int pos = -1;
  if (lane < K) {
    Do = Dk[P.v.org[nd.v0 + lane]];
    Tau = P.v.tau[nd.v0 + lane];
    S = P.v.scol[nd.v0 + lane];
    pos = P.v.posr[nd.v0 + lane];
  }
  double* A = sA[wid];
  for (int h = 0; h < 2; ++h) {
    const int r0 = h ? n1 : 0, rows = h ? n - n1 : n1;
    const int* list = (h ? P.v.blist : P.v.tlist) + nd.v0;
    const int nl = h ? P.m.nbot[g] : P.m.ntop[g];  // poles with support in this half (<= rows)
    __syncwarp();
    if (lane < nl) {
      const int q = list[lane];
      sCol[wid][lane] = P.v.kept[nd.v0 + q];
      sDq[wid][lane] = Dk[q];
      sZq[wid][lane] = P.v.zhat[nd.v0 + q];
    }
    __syncwarp();
    for (int e = lane; e < kTinyRows * nl; e += 32) {
      const int k = e / kTinyRows, r = e % kTinyRows;
      A[e] = r < rows ? nd.src[(r0 + r) + (int64_t)sCol[wid][k] * nd.lds] : 0.0;
    }
    __syncwarp();
    double acc[kTinyRows];
#pragma unroll
    for (int r = 0; r < kTinyRows; ++r) acc[r] = 0.0;
    for (int k = 0; k < nl; ++k) {
      const double u = (sZq[wid][k] * S) * rcp_nr((sDq[wid][k] - Do) - Tau);
#pragma unroll
      for (int r = 0; r < kTinyRows; ++r) acc[r] = fma(A[k * kTinyRows + r], u, acc[r]);
    }
    if (lane < K && pos >= 0 && pos < n) {
      double* out = nd.dst + (int64_t)pos * nd.ldd + r0;
#pragma unroll
      for (int r = 0; r < kTinyRows; ++r)
        if (r < rows) out[r] = acc[r];
    }
  }
}

// The same FP64 product for one stand-alone segment (tdc_cauchy_gemm; with tgen set, the
// structured-operand products of tdc_structured_gemm and tdc_dft_gemm).
__global__ void __launch_bounds__(kThreads, 2) k_gemm_dense_seg(GemmSeg sg) {
  __shared__ double As[BK][BM];
  __shared__ double Us[BK][BN];
  __shared__ double sDo[BN], sTau[BN], sS[BN];
  __shared__ int sCol[BK], sP[BK];
  __shared__ double sDq[BK], sZq[BK];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int rtiles = (sg.rows + BM - 1) / BM, ctiles = (sg.K + BN - 1) / BN;
  const bool gen_t = sg.tgen != nullptr;  // a structured B from generators instead of the Cauchy-like one
  for (int64_t w = blockIdx.x; w < (int64_t)rtiles * ctiles; w += gridDim.x) {
    const int r0 = (int)(w / ctiles) * BM, j0 = (int)(w % ctiles) * BN;
    __syncthreads();
    if (tid < BN && !gen_t) {
      const int j = j0 + tid;
      if (j < sg.K) { sDo[tid] = sg.D[sg.org[j]]; sTau[tid] = sg.tau[j]; sS[tid] = sg.scol[j]; }
      else { sDo[tid] = 0.0; sTau[tid] = 1.0; sS[tid] = 0.0; }
    }
    double acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][c] = 0.0;
    int qlo = 0, qhi = sg.kk;
    if (sg.near_m > 0) near_range(sg.plist, sg.kk, j0, sg.near_m, sg.K, qlo, qhi);
    for (int k0 = qlo; k0 < qhi; k0 += BK) {
      __syncthreads();
      if (tid < BK) {
        const int k = k0 + tid;
        if (k < qhi) {
          const int p = sg.plist ? sg.plist[k] : k;
          sCol[tid] = sg.acol ? sg.acol[p] : p;
          sP[tid] = p;
          sDq[tid] = gen_t ? 0.0 : sg.D[p];
          sZq[tid] = gen_t ? 0.0 : sg.zhat[p];
        } else {
          sCol[tid] = -1; sP[tid] = -1; sDq[tid] = 0.0; sZq[tid] = 0.0;
        }
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < (BK * BM) / kThreads; ++e) {
        const int idx = tid + e * kThreads;
        const int k = idx / BM, r = idx % BM;
        const int col = sCol[k], row = r0 + r;
        As[k][r] = (col >= 0 && row < sg.rows) ? sg.A[row + (int64_t)col * sg.lda] : 0.0;
      }
#pragma unroll
      for (int e = 0; e < (BK * BN) / kThreads; ++e) {
        const int idx = tid + e * kThreads;
        const int k = idx / BN, c = idx % BN;
        if (gen_t) {
          const int p = sP[k], j = j0 + c;
          Us[k][c] = (p >= 0 && j < sg.K) ? struct_entry(sg, p, j) : 0.0;
        } else {
          Us[k][c] = (sZq[k] * sS[c]) * rcp_nr((sDq[k] - sDo[c]) - sTau[c]);
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        double av[8], bv[4];
#pragma unroll
        for (int i = 0; i < 8; ++i) av[i] = As[k][ty * 8 + i];
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = Us[k][tx * 4 + c];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][c] = fma(av[i], bv[c], acc[i][c]);
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (j >= sg.K) continue;
      const int pos = sg.cpos ? sg.cpos[j] : j;
      double* out = sg.C + (int64_t)pos * sg.ldc;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int row = r0 + ty * 8 + i;
        if (row < sg.rows) out[row] = acc[i][c];
      }
    }
  }
}

cudaError_t launch_seg_dense(const GemmSeg& seg, cudaStream_t s) {
  const int64_t tiles = (int64_t)((seg.rows + BM - 1) / BM) * ((seg.K + BN - 1) / BN);
  if (tiles == 0) return cudaSuccess;
  k_gemm_dense_seg<<<(unsigned)(tiles < 152 * 8 ? tiles : 152 * 8), kThreads, 0, s>>>(seg);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tiny(const Plan& P, const LevelLaunch& L, cudaStream_t s) {
  if (L.merges == 0 || L.min_n > kTinyN) return cudaSuccess;
  k_gemm_tiny<<<(unsigned)((L.merges + kTinyWarps - 1) / kTinyWarps), 32 * kTinyWarps, 0, s>>>(P, L.level, L.merges);
  return cudaGetLastError();
}

cudaError_t launch_gemm_dense(const Plan& P, const LevelLaunch& L, int64_t max_tiles, cudaStream_t s) {
  if (max_tiles <= 0) return cudaSuccess;
  int64_t grid = max_tiles;
  const int64_t cap = 152 * 8;
  if (grid > cap) grid = cap;
  k_gemm_dense<<<(unsigned)grid, kThreads, 0, s>>>(P, L.level, L.merges);
  return cudaGetLastError();
}

}  // namespace tdc
